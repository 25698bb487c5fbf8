"""The C-ABI library builds, loads without a GPU, and exports every symbol
include/wtvis.h declares. Host-only entry points are exercised here; compute
entry points are only called in the GPU tests."""
import ctypes as C
import os
import re

import pytest

import paper_1909_03956_gb300 as wt

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    src = open(os.path.join(ROOT, "include", "wtvis.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"^\s*(?:int|void|const char\*)\s+(\w+)\s*\(", src, flags=re.M))
    return names


def test_library_loads_and_exports_every_declared_symbol():
    L = wt.load()
    declared = _declared_symbols()
    assert declared, "no declarations parsed"
    assert declared == set(wt.EXPORTS)
    for name in declared:
        assert hasattr(L, name), name


def test_recommended_J_matches_table1_rule():
    mas = 3.141592653589793 / (180 * 3600 * 1000)
    assert [wt.wt_recommended_J(x * mas) for x in (1300, 200, 150, 12, 15, 3)] == [20, 23, 23, 27, 26, 29]
    with pytest.raises(wt.WtError):
        wt.wt_recommended_J(-1.0)


def test_last_error_is_a_string():
    assert isinstance(wt.wt_last_error(), str)


def test_host_argument_checks_need_no_gpu():
    L = wt.load()
    h = C.c_void_p()
    # J outside 1..30 and negative sizes are rejected on the host
    assert L.wt_build_tree(None, None, None, 0, 0.0, 0.0, 0, C.byref(h), None) == wt.WT_ERR_RANGE
    assert L.wt_build_tree(None, None, None, -1, 0.0, 0.0, 8, C.byref(h), None) == wt.WT_ERR_ARG
    assert L.wt_predict_vis(None, None, 0, None, 0, 1, 0, None) == wt.WT_ERR_ARG
    assert L.dft_predict_vis(None, None, None, 0, None, 0, None, 0, 3, None) == wt.WT_ERR_ARG
    assert L.subtract_model(None, None, None, -5, 0, None) == wt.WT_ERR_ARG


def test_host_argument_checks_of_the_imaging_and_cross_reference_entries():
    L = wt.load()
    h = C.c_void_p()
    # image size, pixel size and level are checked before any device call
    assert L.wt_xref_table(0, 1e-4, 0.0, 0.5, 10, None, None) == wt.WT_ERR_ARG
    assert L.wt_xref_table(64, -1.0, 0.0, 0.5, 10, None, None) == wt.WT_ERR_RANGE
    assert L.wt_xref_table(64, 1e-4, 0.0, 0.5, 31, None, None) == wt.WT_ERR_RANGE
    assert L.wt_build_tree_xref(None, 64, None, None, 1, 0.0, 0.5, 0, C.byref(h), None) == wt.WT_ERR_RANGE
    assert L.wt_build_tree_xref(None, 64, None, None, -1, 0.0, 0.5, 10, C.byref(h), None) == wt.WT_ERR_ARG
    assert L.wt_hogbom(None, None, 31, C.c_float(0.1), C.c_float(0.0), 10, None, None, None, None) == wt.WT_ERR_ARG
    assert L.wt_hogbom(None, None, 32, C.c_float(1.5), C.c_float(0.0), 10, None, None, None, None) == wt.WT_ERR_RANGE
    assert L.wt_selftest_grid_barrier(0, None) == wt.WT_ERR_ARG
    # the double-float mode is known to the mode checks (a null tree is the error here)
    assert L.wt_predict_vis(None, None, 0, None, wt.WT_FP64_DF, 1, 2, None) == wt.WT_ERR_ARG


def test_host_checks_of_the_tensor_core_mode():
    L = wt.load()
    assert wt.WT_MIXED_TC == 5
    # an unknown mode is rejected before any device call; WT_MIXED_TC passes
    # the mode check and, with nothing to read, stops at the missing device
    # (or, on a machine with one, has nothing to do)
    assert L.dft_predict_vis(None, None, None, 0, None, 0, None, 6, 1, None) == wt.WT_ERR_ARG
    assert L.dft_predict_vis(None, None, None, 0, None, 0, None, wt.WT_MIXED_TC, 1, None) in (wt.WT_ERR_CUDA,
                                                                                              wt.WT_OK)
    # the no-allocation direct sum refuses it: its fixed array holds no tensor-core operand
    assert L.dft_predict_vis_noalloc(None, None, None, 0, None, 0, None, wt.WT_MIXED_TC, 1, None,
                                     None) == wt.WT_ERR_ARG
    assert "bad mode" in L.wt_last_error().decode()
    # a negative size is still the first thing checked
    assert L.subtract_model(None, None, None, -1, wt.WT_MIXED_TC, None) == wt.WT_ERR_ARG
