"""Python access to the CPU oracle -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may import
this package.  The CUDA library never uses it.  ``build()`` compiles ``lst_oracle.c`` with
gcc into ``oracle/_build/liblst_oracle.so`` (FP32, no contraction, no fast math).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "liblst_oracle.so")
SRC = os.path.join(HERE, "lst_oracle.c")
CFLAGS = ["-O2", "-std=c99", "-D_GNU_SOURCE", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
          "-shared"]

_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the oracle (no-op when the library is newer than its sources)."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    srcs = [SRC, os.path.join(HERE, "lst_oracle.h")]
    if (not force and os.path.exists(LIB_PATH)
            and os.path.getmtime(LIB_PATH) >= max(os.path.getmtime(s) for s in srcs)):
        return LIB_PATH
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    subprocess.run(["gcc", *CFLAGS, "-o", tmp, SRC, "-lm", "-lpthread"], check=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


class _Event(C.Structure):
    _fields_ = [("n_hits", C.c_uint32), ("x", C.c_void_p), ("y", C.c_void_p), ("z", C.c_void_p),
                ("det", C.c_void_p), ("n_pls", C.c_uint32), ("pls", C.c_void_p)]


_P = C.c_void_p


class _Result(C.Structure):
    _fields_ = [
        ("n_md", C.c_uint32), ("md_module", _P), ("md_lo", _P), ("md_up", _P),
        ("n_ls", C.c_uint32), ("ls_md", _P),
        ("n_t3", C.c_uint32), ("t3_md", _P),
        ("n_t5", C.c_uint32), ("t5_md", _P), ("t5_score", _P), ("t5_kfull", _P),
        ("n_pt3", C.c_uint32), ("pt3_pls", _P), ("pt3_obj", _P), ("pt3_score", _P),
        ("n_pt5", C.c_uint32), ("pt5_pls", _P), ("pt5_obj", _P), ("pt5_score", _P),
        ("pls_cand_n", _P), ("pls_cand", _P),
        ("alive_pt5", _P), ("alive_pt3", _P), ("alive_t5", _P), ("pls_tc", _P),
        ("n_tc", C.c_uint32),
        ("tc_type", _P), ("tc_obj", _P), ("tc_pls", _P), ("tc_ot", _P), ("tc_pix", _P),
        ("tc_pt", _P), ("tc_score", _P),
        ("n_tests", C.c_uint64 * 7),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            # LST_ORACLE_LIB: a separately built copy of the oracle (the mutation test builds
            # copies with one planted mistake each and runs the pins against them)
            path = os.environ.get("LST_ORACLE_LIB")
            if not path:
                build()
                path = LIB_PATH
            L = C.CDLL(path)
            L.ora_geom_create.restype = C.c_void_p
            L.ora_geom_create.argtypes = [C.c_void_p, C.c_uint32]
            L.ora_geom_destroy.argtypes = [C.c_void_p]
            L.ora_geom_map.restype = C.c_uint32
            L.ora_geom_map.argtypes = [C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p)]
            L.ora_run.restype = C.c_int
            L.ora_run.argtypes = [C.c_void_p, C.POINTER(_Event), C.c_int, C.POINTER(_Result)]
            L.ora_result_free.argtypes = [C.POINTER(_Result)]
            L.ora_run_many.restype = C.c_int
            L.ora_run_many.argtypes = [C.c_void_p, C.POINTER(_Event), C.c_uint32, C.c_int,
                                       C.POINTER(_Result)]
            L.ora_arc_len.restype = C.c_float
            L.ora_arc_len.argtypes = [C.c_float, C.c_float]
            L.ora_sincos.argtypes = [C.c_float, C.POINTER(C.c_float), C.POINTER(C.c_float)]
            L.ora_md_test.restype = C.c_int
            L.ora_md_test.argtypes = [C.c_void_p, C.c_uint32, C.POINTER(C.c_float), C.POINTER(C.c_float)]
            F3 = C.POINTER(C.c_float)
            L.ora_ls_eval.restype = C.c_uint32
            L.ora_ls_eval.argtypes = [C.c_void_p, C.c_uint32, C.c_uint32, F3, F3, F3, F3]
            L.ora_t3_eval.restype = C.c_uint32
            L.ora_t3_eval.argtypes = [C.c_void_p, C.POINTER(C.c_uint32), F3, F3, F3, F3]
            L.ora_t5_eval.restype = C.c_uint32
            L.ora_t5_eval.argtypes = [C.c_void_p, C.POINTER(C.c_uint32), F3, F3, F3]
            L.ora_pls_eval.restype = C.c_uint32
            L.ora_pls_eval.argtypes = [C.c_void_p, C.c_void_p, C.c_uint32, F3, F3]
            L.ora_pt5_eval.restype = C.c_uint32
            L.ora_pt5_eval.argtypes = [C.c_void_p, C.c_void_p, C.POINTER(C.c_uint32), F3]
            L.ora_geom_set_t5_mlp.restype = C.c_int
            L.ora_geom_set_t5_mlp.argtypes = [C.c_void_p, F3, C.c_uint32]
            L.ora_t5_features.restype = C.c_uint32
            L.ora_t5_features.argtypes = [C.c_void_p, C.POINTER(C.c_uint32), F3, F3]
            L.ora_t5_logit.restype = C.c_float
            L.ora_t5_logit.argtypes = [F3, F3]
            _lib = L
    return _lib


def _arr(ptr, n, dtype):
    if n == 0 or not ptr:
        return np.zeros(n, dtype)
    buf = (C.c_char * (n * np.dtype(dtype).itemsize)).from_address(ptr)
    return np.frombuffer(buf, dtype=dtype, count=n).copy()


class Geometry:
    """Oracle-side geometry: module table + derived constants + its own connection map."""

    def __init__(self, modules: np.ndarray):
        self._mods = np.ascontiguousarray(modules)
        self._h = lib().ora_geom_create(self._mods.ctypes.data, len(self._mods))
        if not self._h:
            raise ValueError("oracle rejected the module table")
        self.n_modules = len(self._mods)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.ora_geom_destroy(h)
            self._h = None

    def connection_map(self):
        ro, co = C.c_void_p(), C.c_void_p()
        ne = lib().ora_geom_map(self._h, C.byref(ro), C.byref(co))
        return _arr(ro.value, self.n_modules + 1, np.uint32), _arr(co.value, ne, np.uint32)


def _event_struct(ev, keep):
    x = np.ascontiguousarray(ev.x, np.float32); y = np.ascontiguousarray(ev.y, np.float32)
    z = np.ascontiguousarray(ev.z, np.float32); det = np.ascontiguousarray(ev.det, np.uint32)
    pls = np.ascontiguousarray(ev.pls)
    keep.extend([x, y, z, det, pls])
    return _Event(len(x), x.ctypes.data, y.ctypes.data, z.ctypes.data, det.ctypes.data,
                  len(pls), pls.ctypes.data if len(pls) else None)


def _convert(r: _Result, n_pls: int) -> dict:
    o = {
        "md": np.stack([_arr(r.md_module, r.n_md, np.uint32), _arr(r.md_lo, r.n_md, np.uint32),
                        _arr(r.md_up, r.n_md, np.uint32)], axis=1),
        "ls": _arr(r.ls_md, 2 * r.n_ls, np.uint32).reshape(-1, 2),
        "t3": _arr(r.t3_md, 3 * r.n_t3, np.uint32).reshape(-1, 3),
        "t5": _arr(r.t5_md, 5 * r.n_t5, np.uint32).reshape(-1, 5),
        "t5_score": _arr(r.t5_score, r.n_t5, np.float32),
        "t5_kfull": _arr(r.t5_kfull, r.n_t5, np.float32),
        "pt3": np.stack([_arr(r.pt3_pls, r.n_pt3, np.uint32), _arr(r.pt3_obj, r.n_pt3, np.uint32)], axis=1),
        "pt3_score": _arr(r.pt3_score, r.n_pt3, np.float32),
        "pt5": np.stack([_arr(r.pt5_pls, r.n_pt5, np.uint32), _arr(r.pt5_obj, r.n_pt5, np.uint32)], axis=1),
        "pt5_score": _arr(r.pt5_score, r.n_pt5, np.float32),
        "pls_cand_n": _arr(r.pls_cand_n, n_pls, np.uint32),
        "pls_cand": _arr(r.pls_cand, 36 * n_pls, np.uint32).reshape(-1, 36),
        "alive_pt5": _arr(r.alive_pt5, r.n_pt5, np.uint8),
        "alive_pt3": _arr(r.alive_pt3, r.n_pt3, np.uint8),
        "alive_t5": _arr(r.alive_t5, r.n_t5, np.uint8),
        "pls_tc": _arr(r.pls_tc, n_pls, np.uint8),
        "tc_type": _arr(r.tc_type, r.n_tc, np.uint8),
        "tc_obj": _arr(r.tc_obj, r.n_tc, np.uint32),
        "tc_pls": _arr(r.tc_pls, r.n_tc, np.uint32),
        "tc_ot": _arr(r.tc_ot, 10 * r.n_tc, np.uint32).reshape(-1, 10),
        "tc_pix": _arr(r.tc_pix, 4 * r.n_tc, np.uint32).reshape(-1, 4),
        "tc_pt": _arr(r.tc_pt, r.n_tc, np.float32),
        "tc_score": _arr(r.tc_score, r.n_tc, np.float32),
        "n_tests": np.array(list(r.n_tests), np.uint64),
    }
    return o


def run(geom: Geometry, ev, brute_ls: bool = False) -> dict:
    """Whole chain on one event; returns numpy arrays keyed by object kind."""
    keep = []
    e = _event_struct(ev, keep)
    r = _Result()
    rc = lib().ora_run(geom._h, C.byref(e), int(brute_ls), C.byref(r))
    if rc != 0:
        raise ValueError("oracle rejected the event")
    try:
        return _convert(r, ev.n_pls)
    finally:
        lib().ora_result_free(C.byref(r))


def run_many(geom: Geometry, events, n_threads: int = 1, convert: bool = True):
    """Events in parallel on ``n_threads`` host threads (results per event)."""
    keep = []
    arr = (_Event * len(events))(*[_event_struct(ev, keep) for ev in events])
    res = (_Result * len(events))()
    rc = lib().ora_run_many(geom._h, arr, len(events), int(n_threads), res)
    try:
        if rc != 0:
            raise ValueError("oracle rejected an event")
        return [(_convert(res[i], events[i].n_pls) if convert else None) for i in range(len(events))]
    finally:
        for i in range(len(events)):
            lib().ora_result_free(C.byref(res[i]))


def arc_len(chord: float, R: float) -> float:
    return float(lib().ora_arc_len(chord, R))


def sincos(a: float):
    s, c = C.c_float(), C.c_float()
    lib().ora_sincos(a, C.byref(s), C.byref(c))
    return float(s.value), float(c.value)


def md_test(geom: Geometry, module: int, a, b) -> bool:
    fa = (C.c_float * 3)(*a)
    fb = (C.c_float * 3)(*b)
    return bool(lib().ora_md_test(geom._h, module, fa, fb))


# ---- predicate-level decisions (bit masks; see lst_oracle.h) ----
LS_BEND, LS_RZ, LS_EXIT, LS_DIR_IN, LS_DIR_OUT = 1, 2, 4, 8, 16
T3_RZ, T3_MIDDIR, T3_RADIUS = 1, 2, 4
T5_INOUT, T5_BRFULL, T5_RADIUS, T5_RZ = 1, 2, 4, 8
PLS_RPHI, PLS_RZ = 1, 2
PT5_WINDOWS, PT5_CURV = 1, 2


def _f3(v):
    return (C.c_float * 3)(*[float(np.float32(x)) for x in v])


def ls_eval(geom: Geometry, A: int, B: int, a, au, b, bu) -> int:
    return int(lib().ora_ls_eval(geom._h, A, B, _f3(a), _f3(au), _f3(b), _f3(bu)))


def t3_eval(geom: Geometry, mods, a, b, bu, c) -> int:
    m = (C.c_uint32 * 3)(*map(int, mods))
    return int(lib().ora_t3_eval(geom._h, m, _f3(a), _f3(b), _f3(bu), _f3(c)))


def t5_eval(geom: Geometry, mods, pts):
    """(mask, score, k_full) of five anchors (x, y, z) on modules ``mods``."""
    m = (C.c_uint32 * 5)(*map(int, mods))
    p = (C.c_float * 15)(*np.asarray(pts, np.float32).ravel().tolist())
    sc, kf = C.c_float(), C.c_float()
    mask = lib().ora_t5_eval(geom._h, m, p, C.byref(sc), C.byref(kf))
    return int(mask), np.float32(sc.value), np.float32(kf.value)


T5_NF, T5_NH = 8, 16
T5_NPARAM = T5_NH * T5_NF + T5_NH + T5_NH * T5_NH + T5_NH + T5_NH + 1


def set_t5_mlp(geom: Geometry, weights) -> None:
    """Learned T5 selection on ``geom`` (T5_NPARAM float32 weights), or None for the cuts."""
    if weights is None:
        lib().ora_geom_set_t5_mlp(geom._h, None, 0)
        return
    w = np.ascontiguousarray(np.asarray(weights, np.float32).ravel())
    if lib().ora_geom_set_t5_mlp(geom._h, w.ctypes.data_as(C.POINTER(C.c_float)), w.size) != 0:
        raise ValueError("bad T5 network weights")


def t5_features(geom: Geometry, mods, pts) -> np.ndarray:
    """The T5_NF network inputs of five anchors (x, y, z) on modules ``mods``."""
    m = (C.c_uint32 * 5)(*map(int, mods))
    p = (C.c_float * 15)(*np.asarray(pts, np.float32).ravel().tolist())
    f = (C.c_float * T5_NF)()
    if not lib().ora_t5_features(geom._h, m, p, f):
        raise ValueError("module id out of range")
    return np.array(f[:], np.float32)


def t5_logit(weights, f) -> np.float32:
    """Network output z for inputs f (the candidate passes when z > 0)."""
    w = np.ascontiguousarray(np.asarray(weights, np.float32).ravel())
    x = np.ascontiguousarray(np.asarray(f, np.float32).ravel())
    assert w.size == T5_NPARAM and x.size == T5_NF
    return np.float32(lib().ora_t5_logit(w.ctypes.data_as(C.POINTER(C.c_float)),
                                         x.ctypes.data_as(C.POINTER(C.c_float))))


def pls_eval(geom: Geometry, pls, module: int, x):
    """(mask, normalised squared residual) of one anchor against one pLS record."""
    rec = np.ascontiguousarray(np.asarray(pls).reshape(1))
    sc = C.c_float()
    mask = lib().ora_pls_eval(geom._h, rec.ctypes.data, int(module), _f3(x), C.byref(sc))
    return int(mask), np.float32(sc.value)


def pt5_eval(geom: Geometry, pls, mods, pts) -> int:
    rec = np.ascontiguousarray(np.asarray(pls).reshape(1))
    m = (C.c_uint32 * 5)(*map(int, mods))
    p = (C.c_float * 15)(*np.asarray(pts, np.float32).ravel().tolist())
    return int(lib().ora_pt5_eval(geom._h, rec.ctypes.data, m, p))
