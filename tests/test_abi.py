"""CPU checks of the C ABI boundary: the library builds, loads without a GPU, and exports
every entry point include/lst.h declares; the binding's records match the header sizes."""
import ctypes as C
import os
import re

import numpy as np

import paper_2407_18231_gb300 as lst

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lst.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lst_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("lst_load_geometry", "lst_build_connection_map", "lst_run_event", "lst_run_batch",
                     "lst_get_candidates"):
        assert required in names
    assert set(names) == set(lst.EXPORTS)


def test_library_exports_every_symbol():
    path = lst.build()
    lib = C.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_status_strings_without_gpu():
    L = lst.load_library()
    assert L.lst_status_string(0) == b"ok"
    assert L.lst_status_string(-8) == b"buffer too small"
    # null arguments are rejected before any CUDA call
    assert L.lst_load_geometry(None, 0, None, None) == -1
    assert L.lst_run_event(None, None, None) == -1
    assert L.lst_destroy(None) is None


def test_record_sizes_match_header():
    import lst_synth as S
    assert S.MODULE_DTYPE.itemsize == 48
    assert S.PLS_DTYPE.itemsize == 80
    assert lst.TC_DTYPE.itemsize == 76
    assert C.sizeof(lst.lst_event) == 4 + 4 + 8 * 4 + 8 + 8  # padded like the C struct
    assert C.sizeof(lst.lst_config) == 16 * 4
    assert lst.OBJ_DTYPES[lst.OBJ_PLS].itemsize == 38 * 4
    assert np.dtype(lst.OBJ_DTYPES[lst.OBJ_T5]).itemsize == 32


def test_t5_network_sizes_agree():
    """lst.h's network constants, the binding's, the oracle's and the shipped weights agree."""
    import oracle
    text = open(HEADER).read()
    c = {k: int(v) for k, v in re.findall(r"#define (LST_T5_MLP_[A-Z]+) (\d+)", text)}
    nf, nh = c["LST_T5_MLP_INPUTS"], c["LST_T5_MLP_HIDDEN"]
    assert c["LST_T5_MLP_PARAMS"] == nh * nf + nh + nh * nh + nh + nh + 1
    assert (nf, nh, c["LST_T5_MLP_PARAMS"]) == (oracle.T5_NF, oracle.T5_NH, oracle.T5_NPARAM)
    assert lst.T5_MLP_PARAMS == c["LST_T5_MLP_PARAMS"] == lst.load_t5_mlp().size
    assert lst.load_library().lst_set_t5_selection(None, None, 0) == -1  # null context, no CUDA call
