"""GPU parity: every object list of the CUDA path equals the oracle's element by element.

Integer fields (hit, MD, object indices, flags) must be identical; float fields (scores,
curvatures, pT) must be identical bit for bit -- the cut arithmetic is IEEE binary32 with
one fixed evaluation order on both sides and no contraction, so the tolerance is zero.
Object order is canonical on both sides (sorted by first MD, then candidate order).
"""
import numpy as np
import pytest

import lst_synth as S
import oracle
import paper_2407_18231_gb300 as lst
from lst_synth import events as E

pytestmark = pytest.mark.gpu


def _bits(a):
    return np.ascontiguousarray(a, np.float32).view(np.uint32)


def compare(sess, rid, ora, ev, label=""):
    md = sess.objects(rid, lst.OBJ_MD)
    assert len(md) == len(ora["md"]), f"{label} MD count {len(md)} vs {len(ora['md'])}"
    assert np.array_equal(np.stack([md["module"], md["lo"], md["up"]], 1), ora["md"]), label
    ls = sess.objects(rid, lst.OBJ_LS)
    assert len(ls) == len(ora["ls"]), f"{label} LS count {len(ls)} vs {len(ora['ls'])}"
    assert np.array_equal(ls["md"], ora["ls"]), label
    t3 = sess.objects(rid, lst.OBJ_T3)
    assert len(t3) == len(ora["t3"]), f"{label} T3 count {len(t3)} vs {len(ora['t3'])}"
    assert np.array_equal(t3["md"], ora["t3"]), label
    t5 = sess.objects(rid, lst.OBJ_T5)
    assert len(t5) == len(ora["t5"]), f"{label} T5 count {len(t5)} vs {len(ora['t5'])}"
    assert np.array_equal(t5["md"], ora["t5"]), label
    assert np.array_equal(_bits(t5["score"]), _bits(ora["t5_score"])), label
    assert np.array_equal(_bits(t5["kfull"]), _bits(ora["t5_kfull"])), label
    assert np.array_equal(t5["alive"], ora["alive_t5"]), label
    pl = sess.objects(rid, lst.OBJ_PLS)
    assert len(pl) == ev.n_pls
    assert np.array_equal(pl["n_cand"], ora["pls_cand_n"]), label
    for p in range(ev.n_pls):
        n = ora["pls_cand_n"][p]
        assert np.array_equal(pl["cand"][p][:n], ora["pls_cand"][p][:n]), (label, p)
    assert np.array_equal(pl["is_tc"], ora["pls_tc"]), label
    for kind, key in ((lst.OBJ_PT3, "pt3"), (lst.OBJ_PT5, "pt5")):
        o = sess.objects(rid, kind)
        assert len(o) == len(ora[key]), f"{label} {key} count {len(o)} vs {len(ora[key])}"
        assert np.array_equal(np.stack([o["pls"], o["obj"]], 1), ora[key]), label
        assert np.array_equal(_bits(o["score"]), _bits(ora[key + "_score"])), label
        assert np.array_equal(o["alive"], ora["alive_" + key]), label
    tc = sess.candidates(rid)
    assert len(tc) == len(ora["tc_type"]), f"{label} TC count {len(tc)} vs {len(ora['tc_type'])}"
    assert np.array_equal(tc["type"], ora["tc_type"]), label
    assert np.array_equal(tc["obj"], ora["tc_obj"]), label
    assert np.array_equal(tc["pls"], ora["tc_pls"]), label
    assert np.array_equal(tc["ot"], ora["tc_ot"]), label
    assert np.array_equal(tc["pix"], ora["tc_pix"]), label
    assert np.array_equal(_bits(tc["pt"]), _bits(ora["tc_pt"])), label
    assert np.array_equal(_bits(tc["score"]), _bits(ora["tc_score"])), label
    assert np.all(tc["n_ot"] == (tc["ot"] != lst.NONE).sum(1))
    assert np.all(tc["n_pix"] == (tc["pix"] != lst.NONE).sum(1))


@pytest.fixture(scope="module")
def built():
    lst.build()
    return True


@pytest.fixture(scope="module")
def sess_barrel(built, barrel_geom):
    return lst.Session(barrel_geom.modules, keep_objects=True)


@pytest.fixture(scope="module")
def sess_full(built, full_geom):
    return lst.Session(full_geom.modules, keep_objects=True)


def test_tiny_parity(sess_barrel, ora_barrel):
    for pls in (False, True):
        ev = S.make_event("tiny", with_pls=pls)
        compare(sess_barrel, sess_barrel.run_event(ev), oracle.run(ora_barrel, ev), ev, f"tiny pls={pls}")


@pytest.mark.parametrize("n_tracks", [1000, 4000])
def test_pu200_parity(sess_full, ora_full, n_tracks):
    ev = S.make_event("pu200", 0, n_tracks=n_tracks, with_pls=True)
    compare(sess_full, sess_full.run_event(ev), oracle.run(ora_full, ev), ev, f"pu200 {n_tracks}")


def test_highocc_full_size_parity(sess_full, ora_full):
    ev = S.make_event("highocc", 0)  # 12000 tracks, 30 % noise, pixel seeds
    compare(sess_full, sess_full.run_event(ev), oracle.run(ora_full, ev), ev, "highocc")


def test_batch_equals_oracle_per_event(sess_full, ora_full):
    evs = [S.make_event("pu200", 1, n_tracks=300, with_pls=True),
           E.Event(np.zeros(0, np.float32), np.zeros(0, np.float32), np.zeros(0, np.float32),
                   np.zeros(0, np.uint32), np.zeros(0, np.int32), np.zeros(0, E.TRACK_DTYPE)),
           S.make_event("serving", 2, n_tracks=2500, with_pls=True),
           S.make_event("pu200", 3, n_tracks=50, with_pls=False),
           S.make_event("highocc", 1, n_tracks=3000)]
    ids = sess_full.run_batch(evs)
    for i, (ev, rid) in enumerate(zip(evs, ids)):
        compare(sess_full, rid, oracle.run(ora_full, ev), ev, f"batch event {i}")
    # replaying the captured graph on the same batch gives the same answer
    ids2 = sess_full.run_batch(evs)
    for a, b in zip(ids, ids2):
        assert sess_full.candidates(a).tobytes() == sess_full.candidates(b).tobytes()


def test_dense_batch_parity(sess_full, ora_full):
    """A batch of 8 events of more than 100 000 hits each: the LS count pass hands its units
    out one at a time there (dense events), and every event of the batch equals the oracle."""
    evs = [S.make_event("highocc", 60 + i, n_tracks=7000) for i in range(8)]
    assert sum(e.n_hits for e in evs) >= 100_000 * len(evs)
    ids = sess_full.run_batch(evs)
    for i, (ev, rid) in enumerate(zip(evs, ids)):
        compare(sess_full, rid, oracle.run(ora_full, ev), ev, f"dense batch event {i}")
        sess_full.release(rid)


def _first_hits(ev, n):
    """The event's first n hits (no seeds): a valid event of exactly n hits."""
    return E.Event(ev.x[:n].copy(), ev.y[:n].copy(), ev.z[:n].copy(), ev.det[:n].copy(), ev.sim[:n].copy(), ev.tracks)


def test_large_scans_at_chunk_boundaries(built, full_geom, ora_full):
    """After a 32-event batch the pipeline's capacities send every scan of later runs to the
    single-pass large form (one block per 8192 elements): runs whose hit count is an exact
    multiple of 8192, one more, one less, a single hit and no hit all equal the oracle."""
    s = lst.Session(full_geom.modules, keep_objects=True)
    for rid in s.run_batch([S.make_event("pu200", 80 + i, with_pls=True) for i in range(32)]):
        s.release(rid)
    base = S.make_event("pu200", 120)
    for n in (3 * 8192, 3 * 8192 + 1, 3 * 8192 - 1, 1, 0):
        ev = _first_hits(base, n)
        rid = s.run_event(ev)
        compare(s, rid, oracle.run(ora_full, ev), ev, f"{n} hits")
        s.release(rid)
    s.close()


def test_seed_item_scan_in_large_form(built, full_geom, ora_full):
    """A batch of more than 262 144 pixel seeds scans its pT3 items per seed in the large
    single-pass form too; sampled events equal the oracle."""
    evs = [S.make_event("pu200", 200 + i, with_pls=True) for i in range(104)]
    assert sum(e.n_pls for e in evs) > 262_144
    s = lst.Session(full_geom.modules, keep_objects=True)
    ids = s.run_batch(evs)
    for i in (0, 51, 103):
        compare(s, ids[i], oracle.run(ora_full, evs[i]), evs[i], f"seed-heavy batch event {i}")
    s.close()


def test_bench_workload_sampled_parity(sess_full, ora_full):
    # the benchmark's batch (PU200-like events with pixel seeds), 3 events checked in full
    evs = [S.make_event("pu200", i, with_pls=True) for i in range(16)]
    ids = sess_full.run_batch(evs)
    for i in (0, 7, 15):
        compare(sess_full, ids[i], oracle.run(ora_full, evs[i]), evs[i], f"bench event {i}")
    # the candidate tally behind the LS roofline: every LS is a tested pair, and no MD is
    # tested against more MDs than the batch holds
    st = sess_full.stats()
    assert st["n_ls"] <= st["ls_candidates"] <= st["n_md"] * st["n_md"]
    assert st["ls_candidates"] > 20 * st["n_ls"]  # the cuts reject almost every pair


def test_batched_barrel_workload(sess_barrel, ora_barrel):
    evs = [S.make_event("batched", i) for i in range(8)]  # 500-6000 tracks each
    ids = sess_barrel.run_batch(evs)
    for i in (0, 3, 7):
        compare(sess_barrel, ids[i], oracle.run(ora_barrel, evs[i]), evs[i], f"batched {i}")


def test_edge_cases(sess_full, ora_full, full_geom):
    z = np.zeros(0, np.float32)
    empty = E.Event(z, z, z, np.zeros(0, np.uint32), np.zeros(0, np.int32), np.zeros(0, E.TRACK_DTYPE))
    compare(sess_full, sess_full.run_event(empty), oracle.run(ora_full, empty), empty, "empty")
    one = S.make_event("pu200", 5, n_tracks=1)
    compare(sess_full, sess_full.run_event(one), oracle.run(ora_full, one), one, "one track")
    seeds_only = S.make_event("pu200", 6, n_tracks=200, with_pls=True)
    seeds_only = E.Event(z, z, z, np.zeros(0, np.uint32), np.zeros(0, np.int32), seeds_only.tracks,
                         seeds_only.pls, seeds_only.pls_sim)
    r = sess_full.run_event(seeds_only)
    compare(sess_full, r, oracle.run(ora_full, seeds_only), seeds_only, "seeds only")
    assert np.all(sess_full.candidates(r)["type"] == lst.TC_PLS)


def test_bad_input_is_rejected_and_context_survives(sess_full, ora_full):
    ev = S.make_event("pu200", 7, n_tracks=100)
    bad = E.Event(ev.x.copy(), ev.y, ev.z, ev.det.copy(), ev.sim, ev.tracks)
    bad.det[3] = 2 * len(S.geometry(False).modules)  # module id out of range
    with pytest.raises(lst.LstError) as e:
        sess_full.run_event(bad)
    assert e.value.status == -2
    nan = E.Event(ev.x.copy(), ev.y, ev.z, ev.det, ev.sim, ev.tracks)
    nan.x[5] = np.nan
    with pytest.raises(lst.LstError) as e:
        sess_full.run_event(nan)
    assert e.value.status == -2
    compare(sess_full, sess_full.run_event(ev), oracle.run(ora_full, ev), ev, "after errors")


def test_buffer_too_small_and_release(sess_full):
    ev = S.make_event("pu200", 8, n_tracks=200)
    rid = sess_full.run_event(ev)
    L = lst.load_library()
    import ctypes as C
    n = C.c_uint32()
    assert L.lst_get_candidates(sess_full.ctx, rid, None, 0, C.byref(n)) == 0 and n.value > 1
    buf = np.zeros(1, lst.TC_DTYPE)
    assert L.lst_get_candidates(sess_full.ctx, rid, buf.ctypes.data, 1, C.byref(n)) == -8
    sess_full.release(rid)
    assert L.lst_get_candidates(sess_full.ctx, rid, None, 0, C.byref(n)) == -9


def test_overflow_rerun_keeps_results(built, full_geom, ora_full):
    # 80 lower + 80 upper hits at almost one point of one module: 6400 MDs from 160 hits,
    # far beyond the sizing estimate -> the run must grow its buffers and re-run
    sess = lst.Session(full_geom.modules, keep_objects=True)
    m = 1000
    mod = full_geom.modules[m]
    r0 = float(mod["surf"])
    phi = 0.5 * (np.arctan2(mod["e0y"], mod["e0x"]) + np.arctan2(mod["e1y"], mod["e1x"]))
    rng = np.random.default_rng(0)
    n = 80
    rr = np.concatenate([np.full(n, r0), np.full(n, r0 + float(mod["gap"]))])
    ph = phi + rng.normal(0, 1e-5, 2 * n)
    z0 = 0.5 * (mod["emin"] + mod["emax"]) + rng.normal(0, 0.01, 2 * n)
    zz = z0 * rr / r0  # both sensors on lines through the beam spot
    ev = E.Event((rr * np.cos(ph)).astype(np.float32), (rr * np.sin(ph)).astype(np.float32), zz.astype(np.float32),
                 np.concatenate([np.full(n, 2 * m), np.full(n, 2 * m + 1)]).astype(np.uint32),
                 np.full(2 * n, -1, np.int32), np.zeros(0, E.TRACK_DTYPE))
    ora = oracle.run(ora_full, ev)
    assert len(ora["md"]) > 3000
    compare(sess, sess.run_event(ev), ora, ev, "overflow")
    assert sess.stats()["reruns"] >= 1
    sess.close()


def test_launch_configuration_invariance(built, full_geom):
    ev = S.make_event("pu200", 9, n_tracks=1500, with_pls=True)
    ref = None
    for bs, bps in ((64, 2), (128, 8), (256, 4), (512, 2)):
        s = lst.Session(full_geom.modules, block_size=bs, blocks_per_sm=bps)
        tc = s.candidates(s.run_event(ev)).tobytes()
        s.close()
        if ref is None:
            ref = tc
        assert tc == ref, (bs, bps)


def test_ls_without_stored_partner_lists(built, full_geom, ora_full):
    # ls_list_cap 1 (no shared-memory list) sends every module to the per-MD LS join, which
    # stores no partner lists, so the fill pass joins every anchor again; 4 mixes both paths
    ev = S.make_event("pu200", 13, n_tracks=1500, with_pls=True)
    ora = oracle.run(ora_full, ev)
    for cap in (1, 4):
        s = lst.Session(full_geom.modules, keep_objects=True, ls_list_cap=cap)
        compare(s, s.run_event(ev), ora, ev, f"ls_list_cap {cap}")
        s.close()


def test_long_neighbour_lists_at_every_list_cap(built, full_geom, ora_full):
    # high occupancy (12000 tracks): 15123 of 75703 anchors have more than 512 neighbour MDs
    # and 248 more than 1024, so a 512-entry list sends many modules to the per-MD join, a
    # 1024-entry list a few and a 2048-entry list none; all equal the oracle
    ev = S.make_event("highocc", 0)
    ora = oracle.run(ora_full, ev)
    for cap in (512, 1024, 2048):
        s = lst.Session(full_geom.modules, keep_objects=True, ls_list_cap=cap)
        compare(s, s.run_event(ev), ora, ev, f"highocc ls_list_cap {cap}")
        s.close()
    # the library's choice: the first run overflows the 512-entry start list, later runs
    # use a list that holds the longest one (1152)
    s = lst.Session(full_geom.modules, keep_objects=True)
    for run in range(2):
        compare(s, s.run_event(ev), ora, ev, f"highocc default list cap, run {run}")
    s.close()


def test_long_neighbour_lists_with_tilted_modules(built, tilted_geom, ora_tilted):
    # with tilted inner-barrel modules half of the high-occupancy pairs sit in lists of
    # 512-1520 MDs: the first run at the default cap joins those modules per MD, the second
    # stages them (a 1536-entry list); both equal the oracle
    ev = S.make_event("highocc", 1, realistic=True)
    ora = oracle.run(ora_tilted, ev)
    s = lst.Session(tilted_geom.modules, keep_objects=True)
    for run in range(2):
        compare(s, s.run_event(ev), ora, ev, f"tilted highocc, run {run}")
    s.close()


def test_pls_with_many_first_anchor_mds(built, full_geom, ora_full):
    # one exact 5 GeV track plus 11 extra hits on each sensor of its first-layer module,
    # within 20 um of its crossing: 144 MDs there all pass the pLS's first-anchor window
    # (more than the 64 kept per pLS), so pT3 phase 2 takes the fallback over every T3 of
    # the candidate modules, with more than 32 candidates per item
    rng = np.random.default_rng(5)
    t = E.random_tracks(rng, 1, pt_lo=5.0, pt_hi=5.0001, eta_max=0.3)
    ev = E.event_from_tracks(full_geom, t, 3, exact=True, with_pls=True, fake_pls_frac=0.0, shuffle=False)
    _, _, mod, sen, x, y, z = E.track_crossings(full_geom, t)
    r = np.hypot(x, y)
    xs, ys, zs, ds = [ev.x], [ev.y], [ev.z], [ev.det]
    for i in np.argsort(r)[:2]:
        phi = np.arctan2(y[i], x[i]) + rng.normal(0, 0.002 / r[i], 11)
        xs.append((r[i] * np.cos(phi)).astype(np.float32))
        ys.append((r[i] * np.sin(phi)).astype(np.float32))
        zs.append((z[i] + rng.normal(0, 0.002, 11)).astype(np.float32))
        ds.append(np.full(11, 2 * mod[i] + sen[i], np.uint32))
    ev = E.Event(np.concatenate(xs), np.concatenate(ys), np.concatenate(zs), np.concatenate(ds),
                 np.concatenate([ev.sim, np.full(22, -1, np.int32)]), ev.tracks, ev.pls)
    ora = oracle.run(ora_full, ev)
    assert (ora["md"][:, 0] == mod[np.argmin(r)]).sum() >= 144 and len(ora["pt3"]) > 64
    s = lst.Session(full_geom.modules, keep_objects=True)
    compare(s, s.run_event(ev), ora, ev, "dense first layer")
    s.close()


def test_track_metrics_from_batched_candidates(built, full_geom, ora_full):
    # the Sec. 3 metrics of a batch's candidates (split per event by the batch counts) equal
    # those of the oracle's candidates
    from paper_2407_18231_gb300 import validation as V
    evs = [S.make_event("pu200", 20 + i, n_tracks=1200, with_pls=True) for i in range(3)]
    s = lst.Session(full_geom.modules)
    ids = s.run_batch(evs)
    tcs, counts = s.candidates_batch(ids)
    offs = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    for k, ev in enumerate(evs):
        r = oracle.run(ora_full, ev)
        tc_o = np.zeros(len(r["tc_type"]), lst.TC_DTYPE)
        tc_o["ot"] = r["tc_ot"]
        tc_o["pix"] = r["tc_pix"]
        got = V.event_counts(tcs[offs[k]:offs[k + 1]], ev.sim, ev.pls_sim, len(ev.tracks))
        exp = V.event_counts(tc_o, ev.sim, ev.pls_sim, len(ev.tracks))
        assert {a: b for a, b in got.items() if a != "matched_per_sim"} == \
            {a: b for a, b in exp.items() if a != "matched_per_sim"}
        assert np.array_equal(got["matched_per_sim"], exp["matched_per_sim"])
    s.close()


def test_graph_and_eager_launches_agree(built, full_geom, ora_full):
    # the per-event path replays the context's graph; use_graph = 2 launches stream-ordered
    ev = S.make_event("pu200", 11, n_tracks=1200, with_pls=True)
    out = []
    for g in (0, 2):
        s = lst.Session(full_geom.modules, keep_objects=True, use_graph=g)
        rid = s.run_event(ev)
        compare(s, rid, oracle.run(ora_full, ev), ev, f"use_graph={g}")
        out.append(s.candidates(rid).tobytes())
        s.close()
    assert out[0] == out[1]


def test_candidates_batch_matches_per_result(built, full_geom):
    evs = [S.make_event("pu200", 20 + i, n_tracks=400 * (i + 1), with_pls=True) for i in range(5)]
    s = lst.Session(full_geom.modules)
    ids = s.run_batch(evs)
    tcs, counts = s.candidates_batch(ids)
    per = [s.candidates(i) for i in ids]
    assert list(counts) == [len(p) for p in per]
    assert tcs.tobytes() == b"".join(p.tobytes() for p in per)
    s.release(ids[2])
    with pytest.raises(lst.LstError) as e:
        s.candidates_batch(ids)
    assert e.value.status == -9  # NOT_FOUND
    s.close()


def test_async_batches_match_run_batch(built, full_geom):
    groups = [[S.make_event("pu200", 40 + 4 * g + i, n_tracks=600 + 200 * i, with_pls=True) for i in range(4)]
              for g in range(3)]
    s = lst.Session(full_geom.modules)
    ref = []
    for evs in groups:
        ids = s.run_batch(evs)
        ref.append([s.candidates(i).tobytes() for i in ids])
        for i in ids:
            s.release(i)
    ta = s.submit_batch(groups[0])
    tb = s.submit_batch(groups[1])
    with pytest.raises(lst.LstError) as e:
        s.submit_batch(groups[2])  # both slots in flight
    assert e.value.status == -1
    ids_b = s.collect_batch(tb)  # out of order: b waits for a on the device
    ids_a = s.collect_batch(ta)
    assert [s.candidates(i).tobytes() for i in ids_a] == ref[0]
    assert [s.candidates(i).tobytes() for i in ids_b] == ref[1]
    with pytest.raises(lst.LstError) as e:
        s.collect_batch(ta)  # already collected
    assert e.value.status == -9
    ids_c = s.collect_batch(s.submit_batch(groups[2]))
    assert [s.candidates(i).tobytes() for i in ids_c] == ref[2]
    s.close()


def test_repeat_runs_identical(sess_full):
    ev = S.make_event("pu200", 10, with_pls=True)
    a = sess_full.candidates(sess_full.run_event(ev)).tobytes()
    for _ in range(3):
        assert sess_full.candidates(sess_full.run_event(ev)).tobytes() == a


def test_device_resident_batch(built, full_geom):
    torch = pytest.importorskip("torch")
    evs = [S.make_event("pu200", 11 + i, n_tracks=800, with_pls=True) for i in range(4)]
    s = lst.Session(full_geom.modules)
    ref = [s.candidates(r) for r in s.run_batch(evs)]
    dev = torch.device("cuda:0")
    cat = lambda k: torch.from_numpy(np.concatenate([getattr(e, k) for e in evs])).to(dev)  # noqa: E731
    x, y, zz = cat("x"), cat("y"), cat("z")
    det = torch.from_numpy(np.concatenate([e.det for e in evs]).view(np.int32)).to(dev)
    pls = torch.from_numpy(np.concatenate([e.pls for e in evs]).view(np.uint8)).to(dev)
    hoff = torch.tensor(np.concatenate([[0], np.cumsum([e.n_hits for e in evs])]).astype(np.int32), device=dev)
    poff = torch.tensor(np.concatenate([[0], np.cumsum([e.n_pls for e in evs])]).astype(np.int32), device=dev)
    b = lst.lst_batch_dev(len(evs), int(hoff[-1]), int(poff[-1]), 0, x.data_ptr(), y.data_ptr(), zz.data_ptr(),
                          det.data_ptr(), hoff.data_ptr(), pls.data_ptr(), poff.data_ptr())
    s.run_batch_device(b)
    ntc, ids = s.batch_finish(len(evs), timeout_ms=60000, keep_results=True)
    for i in range(len(evs)):
        assert ntc[i] == len(ref[i])
        assert s.candidates(ids[i]).tobytes() == ref[i].tobytes()
    s.close()


def test_serving_results_equal_alone(built, full_geom):
    evs = [S.make_event("serving", i, n_tracks=1500 + 300 * i, with_pls=True) for i in range(12)]
    s = lst.Session(full_geom.modules)
    alone = [s.candidates(s.run_event(e)).tobytes() for e in evs]
    arrival = np.cumsum(np.full(len(evs), 2e-4))
    for share in (False, True):  # one batch on the device at a time, or all slots at once
        lat, ntc, ids, wall = s.serve_replay(evs, arrival, n_slots=3, max_batch=4, keep_results=True,
                                             share_device=share)
        for i in range(len(evs)):
            assert s.candidates(ids[i]).tobytes() == alone[i], (share, i)
            assert lat[i] > 0
    s.close()


def test_serving_under_a_memory_budget(built, full_geom):
    """A budget that leaves each slot room for only a few events: batches stay below
    max_batch, the peak device memory stays within the budget, results are unchanged."""
    evs = [S.make_event("serving", i, n_tracks=1500 + 300 * i, with_pls=True) for i in range(16)]
    s = lst.Session(full_geom.modules)
    alone = [s.candidates(s.run_event(e)).tobytes() for e in evs]
    arrival = np.zeros(len(evs))  # all waiting at once: unbounded, every batch would be full
    lat, ntc, ids, wall = s.serve_replay(evs, arrival, n_slots=2, max_batch=8, keep_results=True)
    st = s.stats()
    assert st["served_max_batch"] == 8
    base = st["device_bytes"]
    per_slot_full = (st["served_peak_bytes"] - base) / 2
    budget = int(base + 2 * 0.4 * per_slot_full)
    for share in (False, True):
        lat, ntc, ids, wall = s.serve_replay(evs, arrival, n_slots=2, max_batch=8, keep_results=True,
                                             memory_budget=budget, share_device=share)
        st = s.stats()
        assert 1 <= st["served_max_batch"] < 8, st
        assert st["served_batches"] > 2
        assert st["served_peak_bytes"] <= budget, (st["served_peak_bytes"], budget)
        for i in range(len(evs)):
            assert s.candidates(ids[i]).tobytes() == alone[i], (share, i)
    s.close()


def test_serving_event_beyond_the_budget(built, full_geom):
    """An event that alone needs more than a slot's share fails with LST_ERR_BUDGET; the
    context keeps working."""
    evs = [S.make_event("serving", 40 + i, n_tracks=3000, with_pls=True) for i in range(3)]
    s = lst.Session(full_geom.modules)
    ref = s.candidates(s.run_event(evs[0])).tobytes()
    budget = int(s.stats()["device_bytes"] + (8 << 20))
    with pytest.raises(lst.LstError) as e:
        s.serve_replay(evs, np.zeros(3), n_slots=2, max_batch=4, memory_budget=budget)
    assert e.value.status == -5
    assert s.candidates(s.run_event(evs[0])).tobytes() == ref
    lat, ntc, ids, wall = s.serve_replay(evs, np.zeros(3), n_slots=2, max_batch=4, keep_results=True)
    assert s.candidates(ids[0]).tobytes() == ref
    s.close()


# ---------------------------------------------------------------- tilted inner-barrel modules
@pytest.fixture(scope="module")
def sess_tilted(built, tilted_geom):
    return lst.Session(tilted_geom.modules, keep_objects=True)


def test_tilted_pu200_parity(sess_tilted, ora_tilted):
    """A PU200-like event with seeds in the geometry with tilted inner-barrel modules."""
    ev = S.make_event("pu200", 11, with_pls=True, realistic=True)
    compare(sess_tilted, sess_tilted.run_event(ev), oracle.run(ora_tilted, ev), ev, "tilted pu200")


def test_tilted_highocc_parity(sess_tilted, ora_tilted):
    """The high-occupancy event (12000 tracks, 30 % noise, seeds) with tilted modules."""
    ev = S.make_event("highocc", 1, realistic=True)
    compare(sess_tilted, sess_tilted.run_event(ev), oracle.run(ora_tilted, ev), ev, "tilted highocc")


def test_tilted_batch_parity(sess_tilted, ora_tilted):
    """Tilted-geometry events of uneven size in one batch, each equal to the oracle."""
    evs = [S.make_event("pu200", 12 + i, n_tracks=n, with_pls=True, realistic=True)
           for i, n in enumerate((300, 2500, 900))]
    ids = sess_tilted.run_batch(evs)
    for i, (rid, ev) in enumerate(zip(ids, evs)):
        compare(sess_tilted, rid, oracle.run(ora_tilted, ev), ev, f"tilted batch {i}")


# ---------------------------------------------------------------- LST as a seeder
def test_endcap_2s_parity(built, ec2s_geom, ora_ec2s):
    """The geometry whose outer endcap rings are 2S modules: per event and in a batch, every
    object list equals the oracle (events of up to 1000 tracks -- the half-strip radial
    tolerance multiplies the T3 and T5 combinatorics, 23 k T5s at 1000 tracks)."""
    s = lst.Session(ec2s_geom.modules, keep_objects=True)
    evs = [S.make_event("pu200", 90 + i, n_tracks=n, with_pls=True, endcap_2s=True)
           for i, n in enumerate((400, 800, 1000))]
    refs = [oracle.run(ora_ec2s, ev) for ev in evs]
    assert len(refs[2]["t5"]) > 10_000
    for i, (ev, ref) in enumerate(zip(evs, refs)):
        rid = s.run_event(ev)
        compare(s, rid, ref, ev, f"2S event {i}")
        s.release(rid)
    for i, (ev, ref, rid) in enumerate(zip(evs, refs, s.run_batch(evs))):
        compare(s, rid, ref, ev, f"2S batch event {i}")
    s.close()


def test_triplet_seeds_parity_and_seeder_output(sess_full, ora_full):
    """Events whose pixel seeds are 20 % triplets: every list equals the oracle's, and
    lst_get_seeds returns exactly the unlinked seeds (pLS candidates), quads only or quads
    and triplets (Sec. 2, Table 1)."""
    evs = [S.make_event("pu200", 30 + i, n_tracks=n, with_pls=True, triplet_frac=0.2)
           for i, n in enumerate((4000, 1200))]
    ids = sess_full.run_batch(evs)
    for rid, ev in zip(ids, evs):
        ora = oracle.run(ora_full, ev)
        compare(sess_full, rid, ora, ev, "triplet seeds")
        nh = np.where(ev.pls["n_hits"] == 3, 3, 4)
        assert (nh == 3).sum() > 50
        unlinked = np.nonzero(ora["pls_tc"])[0]
        for mode, want in ((lst.SEEDS_QUADS, unlinked[nh[unlinked] == 4]), (lst.SEEDS_QUADS_TRIPLETS, unlinked)):
            seeds = sess_full.seeds(rid, mode)
            assert np.array_equal(seeds["pls"], want)
            assert np.array_equal(seeds["n_pix"], nh[want])
            for s_ in seeds:
                assert list(s_["pix"][: s_["n_pix"]]) == [4 * s_["pls"] + k for k in range(s_["n_pix"])]


def test_bad_seed_hit_count_is_rejected(sess_full):
    ev = S.make_event("pu200", 33, n_tracks=300, with_pls=True)
    ev.pls["n_hits"][5] = 2
    with pytest.raises(lst.LstError) as e:
        sess_full.run_event(ev)
    assert e.value.status == -2
    ev.pls["n_hits"][5] = 4
    assert len(sess_full.candidates(sess_full.run_event(ev))) > 0
