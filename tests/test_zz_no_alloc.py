"""dft_predict_vis_noalloc: the direct sum for callers that cannot allocate
device memory while they run (a fixed, pre-reserved device budget; a host
framework that owns every allocation). It must give what dft_predict_vis
gives, call after call, without allocating.

This file is collected last on purpose, so that a run stopping at the first
failure has already run every other test. It passes alone in a fresh
process (the first call then does the per-device set-up) and after the rest
of the suite.
"""
import ctypes as C

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
wt = pytest.importorskip("paper_1909_03956_gb300")

pytestmark = pytest.mark.gpu

TOL = {wt.WT_FP64: 1e-10, wt.WT_MIXED: 1e-6}     # of sum |C|, as in the parity tests


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _noalloc(l, m, f, uvw, mode, out, status=None):
    L = wt.load()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = L.dft_predict_vis_noalloc(_ptr(l), _ptr(m), _ptr(f), l.numel(), _ptr(uvw), uvw.shape[0], _ptr(out),
                                   int(mode), 1, _ptr(status), stream)
    assert rc == wt.WT_OK, L.wt_last_error().decode()
    return out


@pytest.mark.parametrize("mode", [wt.WT_FP64, wt.WT_MIXED])
def test_noalloc_matches_dft_predict_vis_on_two_calls_in_a_row(mode):
    # First call: 5 000 components (ten shared-memory chunks); second call:
    # 100 components, so a stale record from the first call would show.
    big = synth.medium(n_t=2)
    small = synth.small()
    ctype = torch.complex128 if mode == wt.WT_FP64 else torch.complex64
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    for w, uvw_np in ((big, big.uvw[::3]), (small, small.uvw)):
        l, m, f, uvw = _dev(w.l), _dev(w.m), _dev(w.flux), _dev(uvw_np)
        got = torch.empty(uvw.shape[0], dtype=ctype, device="cuda")
        _noalloc(l, m, f, uvw, mode, got, status)
        ref = wt.dft_predict_vis(l, m, f, uvw, mode=mode)
        torch.cuda.synchronize()
        err = (got - ref).abs().max().item() / float(np.abs(w.flux).sum())
        assert err <= TOL[mode], err
    assert int(status.item()) == 0


def test_noalloc_allocates_nothing_after_setup():
    w = synth.small()
    l, m, f, uvw = _dev(w.l), _dev(w.m), _dev(w.flux), _dev(w.uvw)
    out = torch.empty(uvw.shape[0], dtype=torch.complex128, device="cuda")
    _noalloc(l, m, f, uvw, wt.WT_FP64, out)          # set-up happens here at the latest
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        _noalloc(l, m, f, uvw, wt.WT_FP64, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_rejects_too_many_components_before_launch():
    L = wt.load()
    n = wt.WT_NOALLOC_MAX_COMPONENTS + 1
    rc = L.dft_predict_vis_noalloc(None, None, None, n, None, 0, None, 0, 1, None, None)
    assert rc == wt.WT_ERR_RANGE
    assert "capacity" in L.wt_last_error().decode()


def test_noalloc_reports_bad_component_in_caller_status():
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    l, m, f = _dev([0.01, 1.5]), _dev([0.0, 0.0]), _dev([1.0, 1.0])
    uvw = _dev(np.ones((4, 3)))
    out = torch.empty(4, dtype=torch.complex128, device="cuda")
    _noalloc(l, m, f, uvw, wt.WT_FP64, out, status)
    torch.cuda.synchronize()
    assert int(status.item()) == wt.WT_ERR_RANGE
