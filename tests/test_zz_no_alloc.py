"""lst_run_event_static: the allocation-free entry point, called through the C ABI.

Callers that may not allocate device memory while running (a framework whose pool
allocator owns the GPU, a latency-critical loop, a plug-in that must not allocate after
start-up) use this variant; its intermediate lists live in one static device array.  Its
track candidates must equal lst_run_event's bit for bit, on two calls in a row (the shared
array keeps the previous call's contents, so whatever must start at zero is reset).
This file is collected last so that a failure here leaves every other test already run.
"""
import ctypes as C

import numpy as np
import pytest

import lst_synth as S
import paper_2407_18231_gb300 as lst

pytestmark = pytest.mark.gpu


def _device_event(torch, ev, dev):
    x = torch.from_numpy(ev.x.copy()).to(dev)
    y = torch.from_numpy(ev.y.copy()).to(dev)
    z = torch.from_numpy(ev.z.copy()).to(dev)
    det = torch.from_numpy(ev.det.view(np.int32).copy()).to(dev)
    pls = torch.from_numpy(np.ascontiguousarray(ev.pls).view(np.uint8).copy()).to(dev)
    hoff = torch.tensor([0, ev.n_hits], dtype=torch.int32, device=dev)
    poff = torch.tensor([0, ev.n_pls], dtype=torch.int32, device=dev)
    desc = lst.lst_batch_dev(1, ev.n_hits, ev.n_pls, ev.n_hits, x.data_ptr(), y.data_ptr(), z.data_ptr(),
                             det.data_ptr(), hoff.data_ptr(), pls.data_ptr(), poff.data_ptr())
    return desc, (x, y, z, det, pls, hoff, poff)


def _free_device_bytes():
    torch = pytest.importorskip("torch")
    free, _ = torch.cuda.mem_get_info(0)
    return free


def test_static_entry_point_matches_run_event():
    torch = pytest.importorskip("torch")
    lst.build()
    L = lst.load_library()
    dev = torch.device("cuda:0")
    geom = S.geometry(False)
    sess = lst.Session(geom.modules)
    events = [S.make_event("pu200", 21, n_tracks=250, with_pls=True),
              S.make_event("pu200", 22, n_tracks=180, with_pls=True)]
    cap = 4096
    out = torch.zeros(cap * lst.TC_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    refs = [sess.candidates(sess.run_event(ev)) for ev in events]
    descs = [_device_event(torch, ev, dev) for ev in events]
    torch.cuda.synchronize()
    # from here on only the allocation-free entry point runs: device memory must not move,
    # its first call on this device included (the context prepared it at creation)
    free0 = _free_device_bytes()
    for ev, ref, (desc, keep) in zip(events, refs, descs):
        assert ev.n_hits <= 8192 and ev.n_pls <= 512
        assert len(ref) > 10
        for call in range(2):  # two calls in a row on the same shared scratch
            n = C.c_uint32(0)
            s = L.lst_run_event_static(sess.ctx, C.byref(desc), out.data_ptr(), cap, C.byref(n), None)
            assert s == 0, L.lst_last_error(sess.ctx)
            assert n.value == len(ref)
            got = np.frombuffer(out[: n.value * lst.TC_DTYPE.itemsize].cpu().numpy().tobytes(), lst.TC_DTYPE)
            assert got.tobytes() == ref.tobytes(), f"call {call}"
            assert _free_device_bytes() == free0, f"device memory changed on call {call}"
    sess.close()


def test_static_entry_point_matches_the_oracle():
    """The allocation-free path against the CPU oracle directly, field by field."""
    torch = pytest.importorskip("torch")
    import oracle
    L = lst.load_library()
    dev = torch.device("cuda:0")
    geom = S.geometry(False)
    sess = lst.Session(geom.modules)
    ev = S.make_event("pu200", 25, n_tracks=220, with_pls=True)
    ora = oracle.run(oracle.Geometry(geom.modules), ev)
    desc, keep = _device_event(torch, ev, dev)
    cap = 4096
    out = torch.zeros(cap * lst.TC_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    n = C.c_uint32(0)
    assert L.lst_run_event_static(sess.ctx, C.byref(desc), out.data_ptr(), cap, C.byref(n), None) == 0
    tc = np.frombuffer(out[: n.value * lst.TC_DTYPE.itemsize].cpu().numpy().tobytes(), lst.TC_DTYPE)
    assert len(tc) == len(ora["tc_type"]) > 10
    assert np.array_equal(tc["type"], ora["tc_type"])
    assert np.array_equal(tc["obj"], ora["tc_obj"])
    assert np.array_equal(tc["pls"], ora["tc_pls"])
    assert np.array_equal(tc["ot"], ora["tc_ot"])
    assert np.array_equal(tc["pix"], ora["tc_pix"])
    assert tc["pt"].tobytes() == ora["tc_pt"].tobytes()
    assert tc["score"].tobytes() == ora["tc_score"].tobytes()
    sess.close()


def test_static_entry_point_rejects_oversize():
    torch = pytest.importorskip("torch")
    L = lst.load_library()
    dev = torch.device("cuda:0")
    sess = lst.Session(S.geometry(False).modules)
    ev = S.make_event("pu200", 23, n_tracks=700)  # > 8192 hits
    assert ev.n_hits > 8192
    desc, keep = _device_event(torch, ev, dev)
    n = C.c_uint32(0)
    out = torch.zeros(16 * lst.TC_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    s = L.lst_run_event_static(sess.ctx, C.byref(desc), out.data_ptr(), 16, C.byref(n), None)
    assert s == -5  # LST_ERR_BUDGET
    assert b"exceeds the static scratch" in L.lst_last_error(sess.ctx)
    # the context still works afterwards
    small = S.make_event("pu200", 24, n_tracks=120, with_pls=True)
    ref = sess.candidates(sess.run_event(small))
    desc, keep = _device_event(torch, small, dev)
    out = torch.zeros(2048 * lst.TC_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    assert L.lst_run_event_static(sess.ctx, C.byref(desc), out.data_ptr(), 2048, C.byref(n), None) == 0
    got = np.frombuffer(out[: n.value * lst.TC_DTYPE.itemsize].cpu().numpy().tobytes(), lst.TC_DTYPE)
    assert got.tobytes() == ref.tobytes()
    sess.close()


def test_static_entry_point_follows_the_t5_selection():
    """With the learned T5 selection set on the context the allocation-free path runs it too
    (oracle with the same weights), and after it is cleared, the cuts again."""
    torch = pytest.importorskip("torch")
    import oracle
    L = lst.load_library()
    dev = torch.device("cuda:0")
    geom = S.geometry(False)
    sess = lst.Session(geom.modules)
    w = lst.load_t5_mlp()
    og = oracle.Geometry(geom.modules)
    ev = S.make_event("pu200", 26, n_tracks=260, with_pls=True)
    desc, keep = _device_event(torch, ev, dev)
    cap = 4096
    out = torch.zeros(cap * lst.TC_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    for weights in (w, None):
        sess.set_t5_selection(weights)
        oracle.set_t5_mlp(og, weights)
        ora = oracle.run(og, ev)
        n = C.c_uint32(0)
        assert L.lst_run_event_static(sess.ctx, C.byref(desc), out.data_ptr(), cap, C.byref(n), None) == 0
        tc = np.frombuffer(out[: n.value * lst.TC_DTYPE.itemsize].cpu().numpy().tobytes(), lst.TC_DTYPE)
        assert len(tc) == len(ora["tc_type"]) > 10
        assert np.array_equal(tc["type"], ora["tc_type"]) and np.array_equal(tc["obj"], ora["tc_obj"])
        assert np.array_equal(tc["ot"], ora["tc_ot"]) and np.array_equal(tc["pix"], ora["tc_pix"])
        assert tc["score"].tobytes() == ora["tc_score"].tobytes()
    sess.close()


def test_scan_run_tags_start_again(monkeypatch):
    """The single-pass scans tag their chunk states with a 30-bit run number; when the tags
    would repeat, the states are cleared and the numbering starts again.  The test hook
    starts the tags two runs before that point: four runs of the pipeline and four calls of
    the allocation-free entry point across it all equal the oracle."""
    torch = pytest.importorskip("torch")
    import oracle
    L = lst.load_library()
    dev = torch.device("cuda:0")
    geom = S.geometry(False)
    monkeypatch.setenv("LST_TEST_SCAN_EPOCH", str(0x3FFFFFFD))
    sess = lst.Session(geom.modules)
    monkeypatch.delenv("LST_TEST_SCAN_EPOCH")
    ev = S.make_event("pu200", 26, n_tracks=220, with_pls=True)
    ora = oracle.run(oracle.Geometry(geom.modules), ev)
    for i in range(4):
        rid = sess.run_event(ev)
        tc = sess.candidates(rid)
        sess.release(rid)
        assert np.array_equal(tc["ot"], ora["tc_ot"]) and tc["score"].tobytes() == ora["tc_score"].tobytes(), i
    desc, keep = _device_event(torch, ev, dev)
    cap = 4096
    out = torch.zeros(cap * lst.TC_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    for i in range(4):
        n = C.c_uint32(0)
        assert L.lst_run_event_static(sess.ctx, C.byref(desc), out.data_ptr(), cap, C.byref(n), None) == 0
        tc = np.frombuffer(out[: n.value * lst.TC_DTYPE.itemsize].cpu().numpy().tobytes(), lst.TC_DTYPE)
        assert np.array_equal(tc["ot"], ora["tc_ot"]) and tc["score"].tobytes() == ora["tc_score"].tobytes(), i
    sess.close()
