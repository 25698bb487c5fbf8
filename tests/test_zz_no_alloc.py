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
import math
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle as O
import synth

torch = pytest.importorskip("torch")
wt = pytest.importorskip("paper_1909_03956_gb300")

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
MODES = [wt.WT_FP64, wt.WT_FP64_DF, wt.WT_MIXED, wt.WT_MIXED_FAST]
TOL = {wt.WT_FP64: 1e-10, wt.WT_MIXED: 1e-6, wt.WT_MIXED_FAST: 1e-6}     # of sum |C|, as in the parity tests


def _tol(mode, w, uvw):
    """The parity tests' bar; for the double-float form the float64 bar or,
    where phases reach beyond about 500 turns, the one its 48-bit arithmetic
    implies (2 pi 2^-45 max |B.s|)."""
    if mode != wt.WT_FP64_DF:
        return TOL[mode]
    r2 = w.l ** 2 + w.m ** 2
    d = np.abs(np.stack([w.l, w.m, -r2 / (1 + np.sqrt(1 - r2))], axis=1))
    return max(1e-10, 2 * math.pi * 2.0 ** -45 * float(np.max(np.abs(uvw) @ d.T)))


def _ctype(mode):
    return torch.complex128 if mode in (wt.WT_FP64, wt.WT_FP64_DF) else torch.complex64


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


@pytest.mark.parametrize("mode", MODES)
def test_noalloc_matches_dft_predict_vis_on_two_calls_in_a_row(mode):
    # First call: 5 000 components (ten shared-memory chunks); second call:
    # 100 components, so a stale record from the first call would show.
    # Each call is held to the bar against dft_predict_vis and, independently
    # of the allocating path, against the oracle's Eq. 12.
    big = synth.medium(n_t=2)
    small = synth.small()
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    for w, uvw_np in ((big, big.uvw[::3]), (small, small.uvw)):
        l, m, f, uvw = _dev(w.l), _dev(w.m), _dev(w.flux), _dev(uvw_np)
        got = torch.empty(uvw.shape[0], dtype=_ctype(mode), device="cuda")
        _noalloc(l, m, f, uvw, mode, got, status)
        ref = wt.dft_predict_vis(l, m, f, uvw, mode=mode)
        torch.cuda.synchronize()
        S = float(np.abs(w.flux).sum())
        tol = _tol(mode, w, uvw_np)
        err = (got - ref).abs().max().item() / S
        assert err <= tol, err
        orc = O.dft(w.l, w.m, w.flux, uvw_np, threads=os.cpu_count() or 1)
        err_o = float(np.max(np.abs(got.cpu().numpy() - orc))) / S
        assert err_o <= tol, err_o
    assert int(status.item()) == 0


@pytest.mark.parametrize("mode", [wt.WT_FP64, wt.WT_MIXED])
def test_noalloc_at_its_full_capacity(mode):
    # exactly WT_NOALLOC_MAX_COMPONENTS components: the pack fills the whole
    # fixed array and the last staging copy reads it up to its last byte
    rng = np.random.default_rng(91)
    n = wt.WT_NOALLOC_MAX_COMPONENTS
    l, m, f = synth.components_uniform(n, 2.0, rng)
    uvw_np = synth.small().uvw[:700]
    dl, dm, df, duvw = _dev(l), _dev(m), _dev(f), _dev(uvw_np)
    got = torch.empty(uvw_np.shape[0], dtype=_ctype(mode), device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    _noalloc(dl, dm, df, duvw, mode, got, status)
    ref = wt.dft_predict_vis(dl, dm, df, duvw, mode=mode)
    torch.cuda.synchronize()
    S = float(np.abs(f).sum())
    assert (got - ref).abs().max().item() / S <= TOL[mode]
    idx = np.arange(0, uvw_np.shape[0], 7)
    orc = O.dft(l, m, f, uvw_np[idx], threads=os.cpu_count() or 1)
    assert float(np.max(np.abs(got.cpu().numpy()[idx] - orc))) / S <= TOL[mode]
    assert int(status.item()) == 0


@pytest.mark.parametrize("mode", MODES)
def test_noalloc_allocates_nothing_after_setup(mode):
    # with no status word the kernels report into the library's own sink
    w = synth.small()
    l, m, f, uvw = _dev(w.l), _dev(w.m), _dev(w.flux), _dev(w.uvw)
    out = torch.empty(uvw.shape[0], dtype=_ctype(mode), device="cuda")
    _noalloc(l, m, f, uvw, mode, out)          # set-up happens here at the latest
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        _noalloc(l, m, f, uvw, mode, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_rejects_a_bad_mode_before_launch():
    L = wt.load()
    rc = L.dft_predict_vis_noalloc(None, None, None, 0, None, 0, None, 7, 1, None, None)
    assert rc == wt.WT_ERR_ARG and "mode" in L.wt_last_error().decode()


def test_noalloc_after_a_context_reset():
    # The fixed array's device address and the status word are looked up
    # again in a new context: the library's own self-test resets the device
    # (cudaDeviceReset) between two calls, so it runs in a fresh process that
    # holds nothing else on the GPU.
    code = ("import sys; sys.path.insert(0, %r); import paper_1909_03956_gb300 as wt; L = wt.load(); "
            "rc = L.wt_selftest_context_reset(); print(rc, L.wt_last_error().decode())" % ROOT)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.split()[0] == "0", r.stdout


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
