"""GB300 Line Segment Tracking: Python binding of liblst.so (C ABI in include/lst.h).

The functions below carry the C names and only marshal arguments; every step of the chain
runs in the library's CUDA kernels.  There is no CPU fallback: if the library is missing or
no GPU is present the calls raise.

    import paper_2407_18231_gb300 as lst
    lst.build()                       # nvcc, sm_103a, in-tree
    s = lst.Session(modules)          # lst_load_geometry + lst_build_connection_map
    tcs = s.run_event(event)          # lst_run_event -> numpy structured array of lst_tc
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from .build import LIB_PATH, build  # noqa: F401

LST_OK = 0
STATUS = {
    0: "LST_OK", -1: "LST_ERR_INVALID_ARG", -2: "LST_ERR_BAD_INPUT", -3: "LST_ERR_NO_MAP", -4: "LST_ERR_OOM",
    -5: "LST_ERR_BUDGET", -6: "LST_ERR_CUDA", -7: "LST_ERR_TIMEOUT", -8: "LST_ERR_BUFFER_TOO_SMALL",
    -9: "LST_ERR_NOT_FOUND",
}
TC_PT5, TC_PT3, TC_T5, TC_PLS = 0, 1, 2, 3
OBJ_MD, OBJ_LS, OBJ_T3, OBJ_T5, OBJ_PT3, OBJ_PT5, OBJ_PLS = range(7)
NONE = 0xFFFFFFFF

TC_DTYPE = np.dtype([("type", np.uint8), ("n_ot", np.uint8), ("n_pix", np.uint8), ("pad", np.uint8),
                     ("obj", np.uint32), ("pls", np.uint32), ("ot", np.uint32, (10,)), ("pix", np.uint32, (4,)),
                     ("pt", np.float32), ("score", np.float32)])
assert TC_DTYPE.itemsize == 76
SEEDS_QUADS, SEEDS_QUADS_TRIPLETS = 0, 1
SEED_DTYPE = np.dtype([("pls", np.uint32), ("n_pix", np.uint32), ("pix", np.uint32, (4,))])
OBJ_DTYPES = {
    OBJ_MD: np.dtype([("module", np.uint32), ("lo", np.uint32), ("up", np.uint32)]),
    OBJ_LS: np.dtype([("md", np.uint32, (2,))]),
    OBJ_T3: np.dtype([("md", np.uint32, (3,))]),
    OBJ_T5: np.dtype([("md", np.uint32, (5,)), ("score", np.float32), ("kfull", np.float32), ("alive", np.uint32)]),
    OBJ_PT3: np.dtype([("pls", np.uint32), ("obj", np.uint32), ("score", np.float32), ("alive", np.uint32)]),
    OBJ_PT5: np.dtype([("pls", np.uint32), ("obj", np.uint32), ("score", np.float32), ("alive", np.uint32)]),
    OBJ_PLS: np.dtype([("n_cand", np.uint32), ("cand", np.uint32, (36,)), ("is_tc", np.uint32)]),
}


class LstError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class lst_event(C.Structure):
    _fields_ = [("n_hits", C.c_uint32), ("x", C.c_void_p), ("y", C.c_void_p), ("z", C.c_void_p),
                ("det", C.c_void_p), ("n_pls", C.c_uint32), ("pls", C.c_void_p)]


class lst_batch_dev(C.Structure):
    _fields_ = [("n_events", C.c_uint32), ("n_hits", C.c_uint32), ("n_pls", C.c_uint32),
                ("max_event_hits", C.c_uint32), ("x", C.c_void_p), ("y", C.c_void_p), ("z", C.c_void_p),
                ("det", C.c_void_p), ("hit_off", C.c_void_p), ("pls", C.c_void_p), ("pls_off", C.c_void_p)]


class lst_config(C.Structure):
    _fields_ = [("device", C.c_int32), ("keep_objects", C.c_uint32), ("use_graph", C.c_uint32),
                ("block_size", C.c_uint32), ("blocks_per_sm", C.c_uint32), ("profile", C.c_uint32),
                ("ls_list_cap", C.c_uint32), ("reserved", C.c_uint32 * 9)]


class lst_profile_entry(C.Structure):
    _fields_ = [("name", C.c_char * 24), ("launches", C.c_uint32), ("ms", C.c_float)]


class lst_stats(C.Structure):
    _fields_ = [(n, C.c_uint32) for n in ("n_events", "n_hits", "n_pls", "n_md", "n_ls", "n_t3", "n_t5", "n_pt3",
                                          "n_pt5", "n_tc", "reruns", "kernels")] + [("device_bytes", C.c_uint64),
                                                                           ("ls_candidates", C.c_uint64),
                                                                           ("served_batches", C.c_uint32),
                                                                           ("served_max_batch", C.c_uint32),
                                                                           ("served_peak_bytes", C.c_uint64),
                                                                           ("map_edges", C.c_uint64)]


class lst_serve_config(C.Structure):
    _fields_ = [("n_slots", C.c_uint32), ("max_batch", C.c_uint32), ("memory_budget", C.c_uint64),
                ("share_device", C.c_uint32), ("reserved", C.c_uint32 * 7)]


EXPORTS = [
    "lst_load_geometry", "lst_build_connection_map", "lst_run_event", "lst_run_batch", "lst_run_batch_device",
    "lst_batch_finish", "lst_get_candidates", "lst_get_objects", "lst_release_result", "lst_destroy",
    "lst_last_error", "lst_status_string", "lst_get_stats", "lst_get_profile", "lst_serve_replay",
    "lst_run_event_static", "lst_set_tuning", "lst_get_candidates_batch", "lst_submit_batch", "lst_collect_batch",
    "lst_get_seeds", "lst_set_t5_selection",
]

T5_MLP_PARAMS = 433  # LST_T5_MLP_PARAMS
T5_MLP_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data", "t5_mlp_pu200.json")


def load_t5_mlp(path: str = T5_MLP_PATH) -> np.ndarray:
    """Weights of the learned T5 selection (LST_T5_MLP_PARAMS float32, lst.h order) from a
    JSON file; the default is the network the package ships, trained on synthetic PU200-like
    events."""
    import json
    with open(path) as f:
        w = np.array(json.load(f)["weights"], np.float32)
    if w.size != T5_MLP_PARAMS:
        raise ValueError(f"{path}: {w.size} weights, expected {T5_MLP_PARAMS}")
    return w

_lib = None
_lock = threading.Lock()


def load_library(path: str = LIB_PATH):
    """Load liblst.so (built in-tree by ``build()``); raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"liblst.so not found at {path}; run paper_2407_18231_gb300.build() first")
        L = C.CDLL(path)
        P, u32, i32 = C.c_void_p, C.c_uint32, C.c_int32
        sig = {
            "lst_load_geometry": (i32, [P, u32, P, C.POINTER(P)]),
            "lst_build_connection_map": (i32, [P]),
            "lst_run_event": (i32, [P, P, C.POINTER(C.c_uint64)]),
            "lst_run_batch": (i32, [P, P, u32, P]),
            "lst_run_batch_device": (i32, [P, P, P]),
            "lst_batch_finish": (i32, [P, u32, P, P]),
            "lst_get_candidates": (i32, [P, C.c_uint64, P, u32, C.POINTER(u32)]),
            "lst_get_objects": (i32, [P, C.c_uint64, i32, P, u32, C.POINTER(u32)]),
            "lst_release_result": (i32, [P, C.c_uint64]),
            "lst_destroy": (None, [P]),
            "lst_last_error": (C.c_char_p, [P]),
            "lst_status_string": (C.c_char_p, [i32]),
            "lst_get_stats": (i32, [P, P]),
            "lst_get_profile": (i32, [P, P, u32, C.POINTER(u32)]),
            "lst_serve_replay": (i32, [P, P, P, P, u32, P, P, P, P]),
            "lst_run_event_static": (i32, [P, P, P, u32, C.POINTER(u32), P]),
            "lst_set_tuning": (i32, [P, P]),
            "lst_get_candidates_batch": (i32, [P, P, u32, P, C.c_uint64, P, C.POINTER(C.c_uint64)]),
            "lst_submit_batch": (i32, [P, P, u32, C.POINTER(C.c_uint64)]),
            "lst_collect_batch": (i32, [P, C.c_uint64, u32, P, P]),
            "lst_get_seeds": (i32, [P, C.c_uint64, i32, P, u32, C.POINTER(u32)]),
            "lst_set_t5_selection": (i32, [P, P, u32]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
        return L


def _check(ctx, s):
    if s != LST_OK:
        msg = load_library().lst_last_error(ctx).decode() if ctx else ""
        raise LstError(s, msg)


def _event_struct(ev, keep) -> lst_event:
    x = np.ascontiguousarray(ev.x, np.float32); y = np.ascontiguousarray(ev.y, np.float32)
    z = np.ascontiguousarray(ev.z, np.float32); det = np.ascontiguousarray(ev.det, np.uint32)
    pls = np.ascontiguousarray(ev.pls) if getattr(ev, "pls", None) is not None else np.zeros(0, np.uint8)
    keep.extend([x, y, z, det, pls])
    n_pls = int(len(pls)) if pls.dtype.itemsize == 80 else 0
    return lst_event(len(x), x.ctypes.data, y.ctypes.data, z.ctypes.data, det.ctypes.data, n_pls,
                     pls.ctypes.data if n_pls else None)


class Session:
    """One context: geometry + connection map resident on the device."""

    def __init__(self, modules: np.ndarray, *, device: int = 0, keep_objects: bool = False, use_graph: int = 0,
                 block_size: int = 0, blocks_per_sm: int = 0, profile: bool = False, ls_list_cap: int = 0):
        L = load_library()
        self._mods = np.ascontiguousarray(modules)
        self._tickets = {}
        assert self._mods.dtype.itemsize == 48
        cfg = lst_config(device, int(keep_objects), use_graph, block_size, blocks_per_sm, int(profile), ls_list_cap)
        h = C.c_void_p()
        s = L.lst_load_geometry(self._mods.ctypes.data, len(self._mods), C.byref(cfg), C.byref(h))
        if s != LST_OK:
            raise LstError(s, "lst_load_geometry failed")
        self.ctx = h.value
        _check(self.ctx, L.lst_build_connection_map(self.ctx))

    def close(self):
        if getattr(self, "ctx", None):
            load_library().lst_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- runs ----
    def run_event(self, ev):
        keep = []
        e = _event_struct(ev, keep)
        rid = C.c_uint64()
        _check(self.ctx, load_library().lst_run_event(self.ctx, C.byref(e), C.byref(rid)))
        return rid.value

    def run_batch(self, events):
        keep = []
        arr = (lst_event * len(events))(*[_event_struct(ev, keep) for ev in events])
        ids = (C.c_uint64 * len(events))()
        _check(self.ctx, load_library().lst_run_batch(self.ctx, arr, len(events), ids))
        return list(ids)

    def submit_batch(self, events) -> int:
        """Start a batch on one of the two slots; returns a ticket for collect_batch."""
        keep = []
        arr = (lst_event * len(events))(*[_event_struct(ev, keep) for ev in events])
        t = C.c_uint64()
        _check(self.ctx, load_library().lst_submit_batch(self.ctx, arr, len(events), C.byref(t)))
        self._tickets[t.value] = len(events)
        return t.value

    def collect_batch(self, ticket: int, timeout_ms: int = 0):
        """Wait for a submitted batch; returns its result ids (one per event)."""
        n = self._tickets.get(ticket, 1)
        ids = (C.c_uint64 * n)()
        _check(self.ctx, load_library().lst_collect_batch(self.ctx, ticket, timeout_ms, None, ids))
        self._tickets.pop(ticket, None)
        return list(ids)

    def run_batch_device(self, batch: lst_batch_dev, stream=None):
        _check(self.ctx, load_library().lst_run_batch_device(self.ctx, C.byref(batch), stream))

    def batch_finish(self, n_events: int, timeout_ms: int = 0, keep_results: bool = False):
        ntc = np.zeros(n_events, np.uint32)
        ids = (C.c_uint64 * n_events)() if keep_results else None
        _check(self.ctx, load_library().lst_batch_finish(self.ctx, timeout_ms, ntc.ctypes.data,
                                                         ids if keep_results else None))
        return ntc, (list(ids) if keep_results else None)

    # ---- results ----
    def candidates(self, rid: int) -> np.ndarray:
        L = load_library()
        n = C.c_uint32()
        _check(self.ctx, L.lst_get_candidates(self.ctx, rid, None, 0, C.byref(n)))
        out = np.zeros(n.value, TC_DTYPE)
        _check(self.ctx, L.lst_get_candidates(self.ctx, rid, out.ctypes.data, n.value, C.byref(n)))
        return out

    def seeds(self, rid: int, mode: int = SEEDS_QUADS) -> np.ndarray:
        """The seeds LST left unlinked (lst_get_seeds): quads, or quads and triplets."""
        L = load_library()
        n = C.c_uint32()
        _check(self.ctx, L.lst_get_seeds(self.ctx, rid, mode, None, 0, C.byref(n)))
        out = np.zeros(n.value, SEED_DTYPE)
        _check(self.ctx, L.lst_get_seeds(self.ctx, rid, mode, out.ctypes.data, n.value, C.byref(n)))
        return out

    def candidates_batch(self, rids) -> tuple[np.ndarray, np.ndarray]:
        """All candidates of several results in one call: (records back to back, counts)."""
        L = load_library()
        n = len(rids)
        ids = (C.c_uint64 * n)(*rids)
        counts = np.zeros(n, np.uint32)
        total = C.c_uint64()
        _check(self.ctx, L.lst_get_candidates_batch(self.ctx, ids, n, None, 0, counts.ctypes.data, C.byref(total)))
        out = np.empty(total.value, TC_DTYPE)
        _check(self.ctx, L.lst_get_candidates_batch(self.ctx, ids, n, out.ctypes.data, total.value,
                                                    counts.ctypes.data, C.byref(total)))
        return out, counts

    def objects(self, rid: int, kind: int) -> np.ndarray:
        L = load_library()
        n = C.c_uint32()
        _check(self.ctx, L.lst_get_objects(self.ctx, rid, kind, None, 0, C.byref(n)))
        out = np.zeros(n.value, OBJ_DTYPES[kind])
        _check(self.ctx, L.lst_get_objects(self.ctx, rid, kind, out.ctypes.data, n.value, C.byref(n)))
        return out

    def release(self, rid: int):
        _check(self.ctx, load_library().lst_release_result(self.ctx, rid))

    def stats(self) -> dict:
        st = lst_stats()
        _check(self.ctx, load_library().lst_get_stats(self.ctx, C.byref(st)))
        return {f: getattr(st, f) for f, _ in lst_stats._fields_}

    def set_tuning(self, block_size: int = 0, blocks_per_sm: int = 0, ls_list_cap: int = 0):
        cfg = lst_config(0, 0, 0, block_size, blocks_per_sm, 0, ls_list_cap)
        _check(self.ctx, load_library().lst_set_tuning(self.ctx, C.byref(cfg)))

    def set_t5_selection(self, weights=None):
        """Learned T5 selection with these LST_T5_MLP_PARAMS weights (lst_set_t5_selection),
        or the curvature cuts when ``weights`` is None."""
        L = load_library()
        if weights is None:
            _check(self.ctx, L.lst_set_t5_selection(self.ctx, None, 0))
            return
        w = np.ascontiguousarray(np.asarray(weights, np.float32).ravel())
        _check(self.ctx, L.lst_set_t5_selection(self.ctx, w.ctypes.data, w.size))

    def profile(self) -> dict:
        """Per-kernel {name: (launches, ms)} of the last run (profile mode)."""
        L = load_library()
        n = C.c_uint32()
        _check(self.ctx, L.lst_get_profile(self.ctx, None, 0, C.byref(n)))
        buf = (lst_profile_entry * max(n.value, 1))()
        _check(self.ctx, L.lst_get_profile(self.ctx, buf, n.value, C.byref(n)))
        return {buf[i].name.decode(): (buf[i].launches, buf[i].ms) for i in range(n.value)}

    def serve_replay(self, events, arrival_s, *, n_slots=4, max_batch=16, memory_budget=0, keep_results=False,
                     share_device=False):
        n = len(events)
        keep = []
        arr = (lst_event * n)(*[_event_struct(ev, keep) for ev in events])
        arrival = np.ascontiguousarray(arrival_s, np.float64)
        lat = np.zeros(n, np.float64)
        ntc = np.zeros(n, np.uint32)
        ids = (C.c_uint64 * n)() if keep_results else None
        wall = C.c_double()
        cfg = lst_serve_config(n_slots, max_batch, memory_budget, int(share_device))
        _check(self.ctx, load_library().lst_serve_replay(self.ctx, C.byref(cfg), arr, arrival.ctypes.data, n,
                                                         lat.ctypes.data, ntc.ctypes.data, ids, C.byref(wall)))
        return lat, ntc, (list(ids) if keep_results else None), wall.value
