"""GPU runtime behaviour: bounded waits, launch configuration, autotuner."""
import numpy as np
import pytest

import lst_synth as S
import paper_2407_18231_gb300 as lst

pytestmark = pytest.mark.gpu


def _device_batch(torch, evs, dev):
    cat = lambda k: torch.from_numpy(np.ascontiguousarray(np.concatenate([getattr(e, k) for e in evs]))).to(dev)  # noqa
    x, y, z = cat("x"), cat("y"), cat("z")
    det = torch.from_numpy(np.concatenate([e.det for e in evs]).view(np.int32)).to(dev)
    pls = torch.from_numpy(np.concatenate([e.pls for e in evs]).view(np.uint8)).to(dev)
    hoff = torch.tensor(np.concatenate([[0], np.cumsum([e.n_hits for e in evs])]).astype(np.int32), device=dev)
    poff = torch.tensor(np.concatenate([[0], np.cumsum([e.n_pls for e in evs])]).astype(np.int32), device=dev)
    desc = lst.lst_batch_dev(len(evs), int(hoff[-1]), int(poff[-1]), 0, x.data_ptr(), y.data_ptr(), z.data_ptr(),
                             det.data_ptr(), hoff.data_ptr(), pls.data_ptr(), poff.data_ptr())
    return desc, (x, y, z, det, pls, hoff, poff)


def test_bounded_wait_times_out_and_batch_stays_in_flight(full_geom):
    """A wait that runs out returns LST_ERR_TIMEOUT without touching the device; the batch
    is still in flight and a later unbounded wait completes it with the right results."""
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda:0")
    evs = [S.make_event("highocc", i) for i in range(12)]  # several ms of device work
    s = lst.Session(full_geom.modules)
    ref = [s.candidates(r) for r in s.run_batch(evs)]
    desc, keep = _device_batch(torch, evs, dev)
    s.run_batch_device(desc)
    with pytest.raises(lst.LstError) as e:
        s.batch_finish(len(evs), timeout_ms=1)
    assert e.value.status == -7
    # a second batch cannot start while one is in flight
    with pytest.raises(lst.LstError) as e2:
        s.run_batch_device(desc)
    assert e2.value.status == -1
    ntc, ids = s.batch_finish(len(evs), timeout_ms=0, keep_results=True)
    for i in range(len(evs)):
        assert ntc[i] == len(ref[i])
        assert s.candidates(ids[i]).tobytes() == ref[i].tobytes()
    s.close()


def test_tuning_space_gives_identical_results(full_geom):
    ev = S.make_event("pu200", 30, n_tracks=2500, with_pls=True)
    s = lst.Session(full_geom.modules, keep_objects=True)
    ref_tc = ref_ls = None
    for bs, bps, cap in ((256, 4, 512), (128, 2, 1), (512, 8, 128), (64, 4, 32), (256, 1, 1), (512, 4, 1024),
                         (256, 8, 1024)):
        s.set_tuning(bs, bps, cap)
        rid = s.run_event(ev)
        tc = s.candidates(rid).tobytes()
        ls = s.objects(rid, lst.OBJ_LS).tobytes()
        if ref_tc is None:
            ref_tc, ref_ls = tc, ls
        assert tc == ref_tc and ls == ref_ls, (bs, bps, cap)
    with pytest.raises(lst.LstError):
        s.set_tuning(100, 4, 0)  # not a multiple of 32
    s.close()


def test_autotuner_picks_a_configuration(full_geom, tmp_path):
    from paper_2407_18231_gb300 import autotune
    evs = [S.make_event("pu200", 40 + i, n_tracks=1500, with_pls=True) for i in range(4)]
    space = {"block_size": [128, 256], "blocks_per_sm": [2, 4], "ls_list_cap": [1, 512]}
    cache = str(tmp_path / "tune.json")
    res = autotune.tune(full_geom.modules, evs, space=space, reps=2, cache=cache)
    assert len(res["table"]) == 8 and all(r["ms"] > 0 for r in res["table"])
    assert autotune.cached(cache) == res["best"]
    s = lst.Session(full_geom.modules, **res["best"])
    assert len(s.candidates(s.run_event(evs[0]))) > 0
    s.close()


def test_bounded_scan_wait_reports_timeout(full_geom, monkeypatch):
    """The single-pass scans wait for the chunk states of blocks that started earlier, every
    wait bounded.  The test hook makes the first run's scan blocks wait for a state that
    nothing writes (no block takes chunk 0): their polls run out (about a second), the run
    returns LST_ERR_TIMEOUT, and the next run on the same context equals the oracle."""
    import oracle
    monkeypatch.setenv("LST_TEST_STALL_SCAN", "1")
    s = lst.Session(full_geom.modules)
    monkeypatch.delenv("LST_TEST_STALL_SCAN")
    ev = S.make_event("pu200", 46, with_pls=True)  # one event: single-pass scans
    with pytest.raises(lst.LstError) as e:
        s.run_event(ev)
    assert e.value.status == -7 and "wait ran out" in str(e.value)
    tc = s.candidates(s.run_event(ev))
    ora = oracle.run(oracle.Geometry(full_geom.modules), ev)
    assert np.array_equal(tc["ot"], ora["tc_ot"]) and tc["score"].tobytes() == ora["tc_score"].tobytes()
    s.close()


def test_exhausted_partner_arena_rejoins_anchors(full_geom, ora_full, monkeypatch):
    """The LS count pass stores each anchor group's partner lists in a scratch arena; an
    anchor whose lists find it exhausted is joined again by the fill pass.  The test hook
    holds the arena at 4096 words and never lets it grow, so nearly every anchor of these
    runs takes that path: a single event, a batch, and the same batch again all equal the
    oracle list by list."""
    import oracle
    from test_gpu_parity import compare
    monkeypatch.setenv("LST_TEST_MASK_WORDS", "4096")
    s = lst.Session(full_geom.modules, keep_objects=True)
    monkeypatch.delenv("LST_TEST_MASK_WORDS")
    evs = [S.make_event("pu200", 47 + i, n_tracks=2000 + 1000 * i, with_pls=True) for i in range(3)]
    refs = [oracle.run(ora_full, ev) for ev in evs]
    compare(s, s.run_event(evs[0]), refs[0], evs[0], "arena single event")
    for rep in range(2):
        for i, (ev, rid) in enumerate(zip(evs, s.run_batch(evs))):
            compare(s, rid, refs[i], ev, f"arena batch {rep} event {i}")
            s.release(rid)
    s.close()


def test_bounded_large_scan_wait_reports_timeout(full_geom, ora_full, monkeypatch):
    """The same on a batch, whose scans span hundreds of chunks (one block per 8192
    elements), each looking back over the chunks before its own: with the test hook no block
    takes chunk 0, the run returns LST_ERR_TIMEOUT, and the next run on the same context
    equals the oracle."""
    import oracle
    from test_gpu_parity import compare
    monkeypatch.setenv("LST_TEST_STALL_SCAN", "1")
    s = lst.Session(full_geom.modules, keep_objects=True)
    monkeypatch.delenv("LST_TEST_STALL_SCAN")
    evs = [S.make_event("pu200", 70 + i, with_pls=True) for i in range(16)]
    assert sum(e.n_hits for e in evs) > 100 * 8192  # the hit scan takes more than 100 chunks
    with pytest.raises(lst.LstError) as e:
        s.run_batch(evs)
    assert e.value.status == -7 and "wait ran out" in str(e.value)
    ids = s.run_batch(evs)
    for i in (0, 15):
        compare(s, ids[i], oracle.run(ora_full, evs[i]), evs[i], f"after the stalled run, event {i}")
    s.close()
