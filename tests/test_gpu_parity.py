"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bars (see the oracle's readings R1-R9):
  * tree keys, topology, lambda, gamma, merged fluxes: bit-exact;
    leaf pixel centres: within a few ulp (they go through sin/cos);
  * WT_FP64 visibilities: max |dV| <= 1e-10 * sum |C| (relative to the peak
    amplitude, the zero-spacing visibility);
  * WT_MIXED visibilities: max |dV| <= 1e-6 * sum |C|;
  * WT_FP64_DF visibilities: the float64 bar, or where phases reach beyond
    about 500 turns the bar its 48-bit arithmetic implies (df_bar).
"""
import math

import numpy as np
import pytest

import oracle as O
import synth

torch = pytest.importorskip("torch")
wt = pytest.importorskip("paper_1909_03956_gb300")

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOLMIX = 1e-6


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def peak(flux):
    return float(np.abs(flux).sum())


def gpu_tree(w, J):
    return wt.wt_build_tree(dev(w.l), dev(w.m), dev(w.flux), w.ra0, w.dec0, J)


def assert_margins_clear(w, J, thresh=1e-9):
    # Every component must sit clearly inside its pixel for a bit-exact key
    # comparison (the GPU's atan2 may differ from libm's in the last ulp).
    _, mg = O.map_components(w.l, w.m, w.ra0, w.dec0, J)
    assert mg.min() > thresh, "component within %g of a pixel edge; choose another seed" % thresh


def compare_trees(w, J):
    assert_margins_clear(w, J)
    t = gpu_tree(w, J)
    g = t.export()
    o = O.Tree(w.l, w.m, w.flux, w.ra0, w.dec0, J).export()
    assert g["n_nodes"] == len(o["key"])
    assert np.array_equal(g["level_offsets"], o["level_offsets"])
    assert np.array_equal(g["key"], o["key"])
    assert np.array_equal(g["child_mask"], o["child_mask"])
    assert np.array_equal(g["first_child"], o["first_child"])
    assert np.array_equal(g["leaf_flux"], o["leaf_flux"])
    assert np.array_equal(g["lam"], o["lam"])
    assert np.array_equal(g["gamma"], o["gamma"])
    # pixel centres go through sin/cos: a few ulp of the unit vector
    assert np.max(np.abs(g["leaf_dir"] - o["leaf_dir"])) < 1e-15
    rel = np.abs(g["leaf_dir"][:, 2] - o["leaf_dir"][:, 2]) / np.maximum(np.abs(o["leaf_dir"][:, 2]), 1e-300)
    assert rel.max() < 1e-12
    return t


# ---------------------------------------------------------------- tree build

@pytest.mark.parametrize("J", [1, 2, 5, 8, 12, 16, 20, 25, 30])
def test_tree_bit_exact_small(J):
    compare_trees(synth.small(), J)


@pytest.mark.parametrize("J", [8, 10, 12, 14])
def test_tree_bit_exact_medium(J):
    compare_trees(synth.medium(n_t=2), J)


def test_tree_bit_exact_mixed_sign_and_duplicates():
    w = synth.small()
    rng = np.random.default_rng(21)
    f = w.flux * np.where(rng.random(len(w.flux)) < 0.5, -1.0, 1.0)
    l = np.concatenate([w.l, w.l[:30]])          # exact duplicates: same pixel
    m = np.concatenate([w.m, w.m[:30]])
    f = np.concatenate([f, -f[:30]])             # some pixels cancel to zero
    w2 = synth.Workload("dup", w.uvw, l, m, f, 10)
    compare_trees(w2, 10)


def test_tree_large_component_list():
    # 50 000 components (the learned-response workload's list), several sort
    # tiles and many chunks of records.
    w = synth.learned(n_t=2)
    compare_trees(w, 12)


def test_tree_empty():
    t = wt.wt_build_tree(dev(np.zeros(0)), dev(np.zeros(0)), dev(np.zeros(0)), 1.0, 0.5, 8)
    inf = t.info()
    assert inf["n_nodes"] == 0 and inf["n_leaves"] == 0
    v = wt.wt_predict_vis(t, dev(np.ones((5, 3))))
    assert torch.all(v == 0)


# ---------------------------------------------------------------- wavelet

def df_bar(w, J, uvw):
    """Error bar of the double-float form (WT_FP64_DF): its inputs and phase
    carry 48 significant bits, so a term's phase can be off by a few times
    2^-48 |B.s| turns (eight roundings' worth: 2^-45 (|u s_u| + |v s_v| +
    |w (s_w - 1)|)), 32 times the float64 form's; summed over the terms and
    relative to sum |C|: 2 pi 2^-45 max |B.s|. Never below the float64
    form's bar, which it meets wherever |B.s| stays below about 500 turns."""
    d = np.abs(O.Tree(w.l, w.m, w.flux, w.ra0, w.dec0, J).export()["leaf_dir"])
    T = float(np.max(np.abs(np.asarray(uvw)) @ d.T)) if len(d) else 0.0
    return max(TOL64, 2 * math.pi * 2.0 ** -45 * T)


def _wavelet_case(w, J, uvw, mode, which=wt.WT_SUM_EQ17, sign=1):
    t = gpu_tree(w, J)
    v = wt.wt_predict_vis(t, dev(uvw), mode=mode, which=which, sign=sign).cpu().numpy()
    ot = O.Tree(w.l, w.m, w.flux, w.ra0, w.dec0, J)
    ref = ot.vis_eq16(uvw, sign) if which == wt.WT_SUM_EQ16 else ot.vis_eq17(uvw, sign)
    return np.max(np.abs(v - ref)) / peak(w.flux)


@pytest.mark.parametrize("J", [1, 3, 8, 12, 20])
def test_wavelet_fp64_small_all_vis(J):
    w = synth.small()
    assert _wavelet_case(w, J, w.uvw, wt.WT_FP64) <= TOL64


@pytest.mark.parametrize("J", [8, 12, 14])
def test_wavelet_fp64_medium(J):
    # J = 14 has thousands of nodes: the records stream through shared
    # memory in many chunks.
    w = synth.medium(n_t=6)
    uvw = w.uvw[::3]
    assert _wavelet_case(w, J, uvw, wt.WT_FP64) <= TOL64


@pytest.mark.parametrize("J", [8, 12, 14])
def test_wavelet_mixed_medium(J):
    w = synth.medium(n_t=6)
    uvw = w.uvw[::3]
    assert _wavelet_case(w, J, uvw, wt.WT_MIXED) <= TOLMIX


@pytest.mark.parametrize("mode,tol", [(wt.WT_FP64, TOL64), (wt.WT_MIXED, TOLMIX)])
def test_wavelet_eq16(mode, tol):
    w = synth.medium(n_t=6)
    assert _wavelet_case(w, 12, w.uvw[::5], mode, which=wt.WT_SUM_EQ16) <= tol


@pytest.mark.parametrize("mode,tol", [(wt.WT_FP64, TOL64), (wt.WT_MIXED, TOLMIX)])
def test_wavelet_sign_minus(mode, tol):
    w = synth.small()
    assert _wavelet_case(w, 10, w.uvw[:777], mode, sign=-1) <= tol


@pytest.mark.parametrize("n", [1, 31, 255, 257, 1000])
def test_wavelet_ragged_tiles(n):
    w = synth.small()
    assert _wavelet_case(w, 12, w.uvw[:n], wt.WT_FP64) <= TOL64
    assert _wavelet_case(w, 12, w.uvw[:n], wt.WT_MIXED) <= TOLMIX


def test_wavelet_zero_vis():
    w = synth.small()
    t = gpu_tree(w, 8)
    out = wt.wt_predict_vis(t, dev(np.zeros((0, 3))))
    assert out.numel() == 0


def test_wavelet_deep_tree_spaced_components():
    # Distinct components far apart: every leaf has its own chain of
    # ancestors (the tree of the paper's run-time study, Sec. 3.6.1).
    w = synth.medium_fixed(40, n_t=4)
    for J in (16, 25):
        assert _wavelet_case(w, J, w.uvw[::4], wt.WT_FP64) <= TOL64
        assert _wavelet_case(w, J, w.uvw[::4], wt.WT_MIXED) <= TOLMIX


# ---------------------------------------------------------------- direct sum

def _dft_case(w, uvw, mode, sign=1):
    v = wt.dft_predict_vis(dev(w.l), dev(w.m), dev(w.flux), dev(uvw), mode=mode, sign=sign).cpu().numpy()
    ref = O.dft(w.l, w.m, w.flux, uvw, sign)
    return np.max(np.abs(v - ref)) / peak(w.flux)


def dft_df_bar(w, uvw):
    """The double-float form's bar for the direct sum (see df_bar), with the
    components' (l, m, n - 1) in place of the pixel centres."""
    r2 = w.l ** 2 + w.m ** 2
    d = np.abs(np.stack([w.l, w.m, -r2 / (1 + np.sqrt(1 - r2))], axis=1))
    T = float(np.max(np.abs(np.asarray(uvw)) @ d.T))
    return max(TOL64, 2 * math.pi * 2.0 ** -45 * T)


def test_dft_df_small_all_vis_and_sign():
    w = synth.small()
    assert _dft_case(w, w.uvw, wt.WT_FP64_DF) <= dft_df_bar(w, w.uvw)
    assert _dft_case(w, w.uvw[:333], wt.WT_FP64_DF, sign=-1) <= dft_df_bar(w, w.uvw[:333])


def test_dft_df_medium_many_chunks_and_agreement_with_fp64():
    w = synth.medium(n_t=2)
    uvw = w.uvw[::4]
    assert _dft_case(w, uvw, wt.WT_FP64_DF) <= dft_df_bar(w, uvw)
    a = wt.dft_predict_vis(dev(w.l), dev(w.m), dev(w.flux), dev(uvw), mode=wt.WT_FP64).cpu().numpy()
    b = wt.dft_predict_vis(dev(w.l), dev(w.m), dev(w.flux), dev(uvw), mode=wt.WT_FP64_DF).cpu().numpy()
    assert np.max(np.abs(a - b)) / peak(w.flux) <= 1e-11


def test_dft_fp64_small_all_vis():
    w = synth.small()
    assert _dft_case(w, w.uvw, wt.WT_FP64) <= TOL64


def test_dft_mixed_small_all_vis():
    w = synth.small()
    assert _dft_case(w, w.uvw, wt.WT_MIXED) <= TOLMIX


@pytest.mark.parametrize("mode,tol", [(wt.WT_FP64, TOL64), (wt.WT_MIXED, TOLMIX)])
def test_dft_medium_many_chunks(mode, tol):
    # 5 000 components: ten shared-memory chunks per sweep.
    w = synth.medium(n_t=2)
    assert _dft_case(w, w.uvw[::4], mode) <= tol


@pytest.mark.parametrize("mode,tol", [(wt.WT_FP64, TOL64), (wt.WT_MIXED, TOLMIX)])
def test_dft_sign_and_ragged(mode, tol):
    w = synth.small()
    assert _dft_case(w, w.uvw[:333], mode, sign=-1) <= tol


def test_dft_empty_components():
    v = wt.dft_predict_vis(dev(np.zeros(0)), dev(np.zeros(0)), dev(np.zeros(0)), dev(np.ones((7, 3))))
    assert torch.all(v == 0)


def test_dft_point_source_phase_centre_exact():
    rng = np.random.default_rng(3)
    uvw = rng.uniform(-3e4, 3e4, (1000, 3))
    v = wt.dft_predict_vis(dev([0.0]), dev([0.0]), dev([0.37]), dev(uvw)).cpu().numpy()
    assert np.all(v.real == 0.37) and np.all(v.imag == 0.0)


# ---------------------------------------------------------------- subtract

@pytest.mark.parametrize("mode", [wt.WT_FP64, wt.WT_MIXED])
@pytest.mark.parametrize("n", [1, 2, 3, 1001, 100000])
def test_subtract(mode, n):
    rng = np.random.default_rng(n)
    a = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    ct = np.complex128 if mode == wt.WT_FP64 else np.complex64
    a, b = a.astype(ct), b.astype(ct)
    r = wt.subtract_model(dev(a), dev(b), mode=mode).cpu().numpy()
    assert np.array_equal(r, a - b)
    x = dev(a)
    wt.subtract_model(x, dev(b), mode=mode, out=x)          # in place
    assert np.array_equal(x.cpu().numpy(), a - b)


def test_subtract_unaligned_complex64_view():
    n = 1001
    a = (np.arange(n + 1) + 1j).astype(np.complex64)
    b = (np.arange(n + 1) * 0.5).astype(np.complex64)
    A, B = dev(a)[1:], dev(b)[1:]
    r = wt.subtract_model(A, B, mode=wt.WT_MIXED).cpu().numpy()
    assert np.array_equal(r, a[1:] - b[1:])


# ---------------------------------------------------------------- errors

def test_component_outside_unit_disc_is_reported():
    l = np.array([0.1, 1.2])
    m = np.array([0.0, 0.0])
    f = np.array([1.0, 1.0])
    wt.wt_device_status()
    t = wt.wt_build_tree(dev(l), dev(m), dev(f), 1.0, 0.5, 8)
    with pytest.raises(wt.WtError) as e:
        wt.wt_device_status()
    assert e.value.status == wt.WT_ERR_RANGE
    t.close()
    wt.wt_device_status()   # cleared


def test_host_pointer_rejected_before_launch():
    import ctypes as C
    L = wt.load()
    host = np.zeros(3 * 10)
    out = torch.empty(10, dtype=torch.complex128, device="cuda")
    rc = L.dft_predict_vis(C.c_void_p(out.data_ptr()), C.c_void_p(out.data_ptr()), C.c_void_p(out.data_ptr()), 1,
                           host.ctypes.data_as(C.c_void_p), 10, C.c_void_p(out.data_ptr()), 0, 1, None)
    assert rc == wt.WT_ERR_ARG


def test_buffer_too_small_rejected_before_launch():
    uvw = torch.zeros((10, 3), dtype=torch.float64, device="cuda")
    out = torch.empty(5, dtype=torch.complex128, device="cuda")
    import ctypes as C
    L = wt.load()
    z = torch.zeros(1, dtype=torch.float64, device="cuda")
    # claim 10**9 visibilities: far beyond the allocations
    rc = L.dft_predict_vis(C.c_void_p(z.data_ptr()), C.c_void_p(z.data_ptr()), C.c_void_p(z.data_ptr()), 1,
                           C.c_void_p(uvw.data_ptr()), 10 ** 9, C.c_void_p(out.data_ptr()), 0, 1, None)
    assert rc == wt.WT_ERR_ARG


def test_misaligned_buffers_rejected_before_launch():
    # complex128 outputs need 16-byte alignment, float64 inputs 8: a pointer
    # off by 8 (or 4) bytes is an argument error, returned before any launch
    import ctypes as C
    L = wt.load()
    w = synth.small()
    t = gpu_tree(w, 8)
    n = 64
    uvw = dev(w.uvw[:n + 1])
    out = torch.empty(n + 1, dtype=torch.complex128, device="cuda")
    z = dev(np.zeros(2))
    base = out.data_ptr()
    rc = L.wt_predict_vis(t.h, C.c_void_p(uvw.data_ptr()), n, C.c_void_p(base + 8), wt.WT_FP64, 1,
                          wt.WT_SUM_EQ17, None)
    assert rc == wt.WT_ERR_ARG and "aligned" in L.wt_last_error().decode()
    rc = L.wt_predict_vis(t.h, C.c_void_p(uvw.data_ptr() + 4), n, C.c_void_p(base), wt.WT_FP64, 1,
                          wt.WT_SUM_EQ17, None)
    assert rc == wt.WT_ERR_ARG and "aligned" in L.wt_last_error().decode()
    rc = L.dft_predict_vis(C.c_void_p(z.data_ptr()), C.c_void_p(z.data_ptr()), C.c_void_p(z.data_ptr()), 1,
                           C.c_void_p(uvw.data_ptr()), n, C.c_void_p(base + 8), wt.WT_FP64_DF, 1, None)
    assert rc == wt.WT_ERR_ARG and "aligned" in L.wt_last_error().decode()
    # a complex64 output needs only 8 bytes
    out32 = torch.empty(n + 1, dtype=torch.complex64, device="cuda")
    rc = L.wt_predict_vis(t.h, C.c_void_p(uvw.data_ptr()), n, C.c_void_p(out32.data_ptr() + 8), wt.WT_MIXED, 1,
                          wt.WT_SUM_EQ17, None)
    assert rc == wt.WT_OK
    torch.cuda.synchronize()
    ot = O.Tree(w.l, w.m, w.flux, w.ra0, w.dec0, 8)
    assert np.max(np.abs(out32.cpu().numpy()[1:] - ot.vis_eq17(w.uvw[:n]))) <= TOLMIX * peak(w.flux)


def test_tree_on_wrong_mode_rejected():
    w = synth.small()
    t = gpu_tree(w, 8)
    with pytest.raises(wt.WtError):
        wt.wt_predict_vis(t, dev(w.uvw[:4]), mode=7)


# ---------------------------------------------------------------- launch shapes

@pytest.mark.parametrize("variant", range(8))
@pytest.mark.parametrize("mode,tol", [(wt.WT_FP64, TOL64), (wt.WT_MIXED, TOLMIX), (wt.WT_MIXED_FAST, TOLMIX)])
def test_wavelet_every_launch_shape(variant, mode, tol, monkeypatch):
    # Each (threads per CTA, visibilities per thread) shape the autotuner may
    # pick gives the oracle's answer, on a ragged count of visibilities.
    monkeypatch.setenv("WT_WAVELET_VARIANT", str(variant))
    w = synth.medium(n_t=4)
    uvw = w.uvw[::7][:1111]
    assert _wavelet_case(w, 13, uvw, mode) <= tol
    assert _wavelet_case(w, 13, uvw, mode, which=wt.WT_SUM_EQ16) <= tol
    assert _wavelet_case(w, 13, uvw, mode, which=wt.WT_SUM_EQ17_REGROUPED) <= tol


@pytest.mark.parametrize("variant", range(8))
def test_wavelet_df_every_launch_shape(variant, monkeypatch):
    # the double-float form in every launch shape, on a ragged count
    monkeypatch.setenv("WT_WAVELET_VARIANT", str(variant))
    w = synth.medium(n_t=4)
    uvw = w.uvw[::7][:1111]
    assert _wavelet_case(w, 13, uvw, wt.WT_FP64_DF, which=wt.WT_SUM_EQ17_REGROUPED) <= df_bar(w, 13, uvw)
    assert _wavelet_case(w, 13, uvw, wt.WT_FP64_DF, which=wt.WT_SUM_EQ16) <= df_bar(w, 13, uvw)


def test_wavelet_df_subtract_and_default_sum():
    # the binding picks the regrouped sum for the double-float form, and its
    # complex128 output subtracts under its own mode
    w = synth.small()
    t = gpu_tree(w, 10)
    uvw = dev(w.uvw[:500])
    v = wt.wt_predict_vis(t, uvw, mode=wt.WT_FP64_DF)
    assert v.dtype == torch.complex128
    r = wt.subtract_model(v, v, mode=wt.WT_FP64_DF)
    assert torch.all(r == 0)


def test_wavelet_df_explicit_sum_refused():
    w = synth.small()
    t = gpu_tree(w, 8)
    with pytest.raises(wt.WtError) as e:
        wt.wt_predict_vis(t, dev(w.uvw[:10]), mode=wt.WT_FP64_DF, which=wt.WT_SUM_EQ17)
    assert e.value.status == wt.WT_ERR_UNSUPPORTED


@pytest.mark.parametrize("J", [1, 8, 12, 20])
def test_wavelet_df_eq16(J):
    # the level-J sum in double-float, against the oracle's Eq. 16
    w = synth.small()
    uvw = w.uvw[::3]
    assert _wavelet_case(w, J, uvw, wt.WT_FP64_DF, which=wt.WT_SUM_EQ16) <= df_bar(w, J, uvw)
    assert _wavelet_case(w, J, uvw[:777], wt.WT_FP64_DF, which=wt.WT_SUM_EQ16, sign=-1) <= df_bar(w, J, uvw)


def test_wavelet_df_agrees_with_the_float64_form_far_below_the_bar():
    # float64-class: against the float64 kernel the double-float form
    # differs by the phase tail's float32 rounding (about 1e-11 turns at a
    # thousand turns), far below the 1e-10 bar both meet
    w = synth.medium(n_t=6)
    uvw = w.uvw[::3]
    t = gpu_tree(w, 12)
    a = wt.wt_predict_vis(t, dev(uvw), mode=wt.WT_FP64, which=wt.WT_SUM_EQ17_REGROUPED).cpu().numpy()
    b = wt.wt_predict_vis(t, dev(uvw), mode=wt.WT_FP64_DF, which=wt.WT_SUM_EQ17_REGROUPED).cpu().numpy()
    assert np.max(np.abs(a - b)) / peak(w.flux) <= 1e-11


# ---------------------------------------------------------------- regrouped Eq. 17

@pytest.mark.parametrize("J", [1, 2, 3, 4, 8, 12, 20])
@pytest.mark.parametrize("mode,tol", [(wt.WT_FP64, TOL64), (wt.WT_FP64_DF, TOL64), (wt.WT_MIXED, TOLMIX)])
def test_wavelet_regrouped_small(J, mode, tol):
    # V = sum_n w_n eta_n with w from the parents' gammas: the same terms as
    # Eq. 17, checked against the oracle's literal Eq. 17.
    w = synth.small()
    if mode == wt.WT_FP64_DF:
        tol = df_bar(w, J, w.uvw[::3])
    assert _wavelet_case(w, J, w.uvw[::3], mode, which=wt.WT_SUM_EQ17_REGROUPED) <= tol


@pytest.mark.parametrize("J", [10, 14])
@pytest.mark.parametrize("mode,tol", [(wt.WT_FP64, TOL64), (wt.WT_FP64_DF, TOL64), (wt.WT_MIXED, TOLMIX)])
def test_wavelet_regrouped_medium_and_sign(J, mode, tol):
    w = synth.medium(n_t=6)
    if mode == wt.WT_FP64_DF:
        tol = df_bar(w, J, w.uvw)
    assert _wavelet_case(w, J, w.uvw[::3], mode, which=wt.WT_SUM_EQ17_REGROUPED) <= tol
    assert _wavelet_case(w, J, w.uvw[:999], mode, which=wt.WT_SUM_EQ17_REGROUPED, sign=-1) <= tol


@pytest.mark.parametrize("mode,which,tol", [(wt.WT_FP64, wt.WT_SUM_EQ17, TOL64),
                                           (wt.WT_FP64, wt.WT_SUM_EQ17_REGROUPED, TOL64),
                                           (wt.WT_FP64_DF, wt.WT_SUM_EQ17_REGROUPED, TOL64),
                                           (wt.WT_MIXED, wt.WT_SUM_EQ17, TOLMIX),
                                           (wt.WT_MIXED_FAST, wt.WT_SUM_EQ17_REGROUPED, TOLMIX)])
def test_wavelet_deepest_tree_J30(mode, which, tol):
    # the largest J the int64 keys hold: level-29 HEALPix pixels (Nside 2^29),
    # 29 stack levels, every form's launch shapes at their shared-memory limit
    w = synth.medium_fixed(20, n_t=2)
    if mode == wt.WT_FP64_DF:
        tol = df_bar(w, 30, w.uvw[::5])
    assert _wavelet_case(w, 30, w.uvw[::5], mode, which=which) <= tol


def test_wavelet_regrouped_deep_and_mixed_sign():
    w = synth.medium_fixed(40, n_t=4)
    for J in (16, 25):
        assert _wavelet_case(w, J, w.uvw[::4], wt.WT_FP64, which=wt.WT_SUM_EQ17_REGROUPED) <= TOL64
        assert _wavelet_case(w, J, w.uvw[::4], wt.WT_FP64_DF, which=wt.WT_SUM_EQ17_REGROUPED) <= df_bar(w, J, w.uvw[::4])
        assert _wavelet_case(w, J, w.uvw[::4], wt.WT_MIXED, which=wt.WT_SUM_EQ17_REGROUPED) <= TOLMIX
    rng = np.random.default_rng(31)
    s = synth.small()
    f = s.flux * np.where(rng.random(len(s.flux)) < 0.5, -1.0, 1.0)
    w2 = synth.Workload("mixed-sign", s.uvw, s.l, s.m, f, 11)
    assert _wavelet_case(w2, 11, s.uvw[::5], wt.WT_FP64, which=wt.WT_SUM_EQ17_REGROUPED) <= TOL64
    assert _wavelet_case(w2, 11, s.uvw[::5], wt.WT_FP64_DF, which=wt.WT_SUM_EQ17_REGROUPED) <= df_bar(w2, 11, s.uvw[::5])


# ---------------------------------------------------------------- one launch against pieces

@pytest.mark.parametrize("n_extra", [0, 777])
@pytest.mark.parametrize("mode", [wt.WT_MIXED_FAST, wt.WT_FP64])
def test_wavelet_one_launch_equals_pieces(mode, n_extra, monkeypatch):
    # With the launch shape pinned, predicting a batch of several waves of
    # CTAs in one call gives, bit for bit, what calls over pieces of it give
    # (each visibility's arithmetic is its own, wherever its tile runs); a
    # consumer on the caller's stream sees the whole result without a
    # synchronisation; the visibilities at the cut match the oracle.
    monkeypatch.setenv("WT_WAVELET_VARIANT", "2")
    w = synth.medium(J=10)
    n = (1 << 19) + n_extra
    uvw = dev(w.uvw[:n])
    t = gpu_tree(w, 10)
    which = wt.WT_SUM_EQ17_REGROUPED
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        v = wt.wt_predict_vis(t, uvw, mode=mode, which=which)
        seen = v.clone()
    torch.cuda.synchronize()
    q = 1 << 18
    parts = [wt.wt_predict_vis(t, uvw[a:b], mode=mode, which=which) for a, b in ((0, q), (q, n))]
    whole = torch.cat(parts).cpu().numpy()
    assert np.array_equal(v.cpu().numpy(), whole)
    assert np.array_equal(seen.cpu().numpy(), whole)
    idx = np.array([0, q - 2, q - 1, q, q + 1, n - 1])
    ref = O.Tree(w.l, w.m, w.flux, w.ra0, w.dec0, 10).vis_eq17(w.uvw[idx])
    assert np.max(np.abs(whole[idx] - ref)) / peak(w.flux) <= (TOL64 if mode == wt.WT_FP64 else TOLMIX)


# ---------------------------------------------------------------- failure detection

def test_bounded_wait_times_out_and_reports():
    # A wait on a phase nothing completes gives up after its poll limit and
    # reports WT_ERR_TIMEOUT; the context stays usable afterwards.
    wt.wt_device_status()
    wt.wt_selftest_bounded_wait(500)
    with pytest.raises(wt.WtError) as e:
        wt.wt_device_status()
    assert e.value.status == wt.WT_ERR_TIMEOUT
    wt.wt_device_status()                     # cleared
    w = synth.small()
    assert _dft_case(w, w.uvw[:100], wt.WT_FP64) <= TOL64


# ---------------------------------------------------------------- fast mixed form

@pytest.mark.parametrize("J", [1, 8, 12, 14])
def test_wavelet_mixed_fast(J):
    # sin/cos from the special-function unit: the same 1e-6 bar.
    w = synth.medium(n_t=6)
    uvw = w.uvw[::3]
    for which in (wt.WT_SUM_EQ17, wt.WT_SUM_EQ16, wt.WT_SUM_EQ17_REGROUPED):
        assert _wavelet_case(w, J, uvw, wt.WT_MIXED_FAST, which=which) <= TOLMIX
    assert _wavelet_case(w, J, uvw[:500], wt.WT_MIXED_FAST, sign=-1) <= TOLMIX


def test_wavelet_mixed_fast_single_component_worst_case():
    # One component: no averaging over terms, so the per-term error bound
    # of the fast form is what shows.
    rng = np.random.default_rng(41)
    uvw = rng.uniform(-3e4, 3e4, (20000, 3))
    w = synth.Workload("one", uvw, np.array([0.0123]), np.array([-0.0071]), np.array([1.0]), 14)
    assert _wavelet_case(w, 14, uvw, wt.WT_MIXED_FAST) <= TOLMIX
    assert _dft_case(w, uvw, wt.WT_MIXED_FAST) <= TOLMIX


def test_dft_mixed_fast():
    w = synth.medium(n_t=2)
    assert _dft_case(w, w.uvw[::4], wt.WT_MIXED_FAST) <= TOLMIX
    s = synth.small()
    assert _dft_case(s, s.uvw[:333], wt.WT_MIXED_FAST, sign=-1) <= TOLMIX


# ---------------------------------------------------------------- cross-reference table (Sec. 3.5)

@pytest.mark.parametrize("J", [8, 12, 18])
def test_xref_table_matches_the_oracle(J):
    n, dl = 96, 2.0e-5
    g = wt.wt_xref_table(n, dl, synth.RA0, synth.DEC0, J).cpu().numpy()
    o, margin = O.xref_table(n, dl, synth.RA0, synth.DEC0, J)
    # the GPU's atan2 may differ from libm's in the last ulp: pixels within
    # 1e-9 of a sphere-pixel edge (a row on the phase centre's meridian
    # here) are left out
    clear = margin > 1e-9
    assert clear.mean() > 0.95
    assert np.array_equal(g[clear], o[clear])
    # corners outside the unit disc
    g2 = wt.wt_xref_table(8, 0.3, synth.RA0, synth.DEC0, J).cpu().numpy()
    assert g2[0, 0] == -1 and g2[4, 4] >= 0


def test_tree_from_xref_equals_tree_from_pixel_centres():
    # components at image pixels (repeats merge), mapped through the table,
    # give bit for bit the tree of the pixel centres' (l, m)
    n, dl, J = 128, 2.0e-5, 16
    rng = np.random.default_rng(5)
    pix = rng.integers(0, n * n, 400).astype(np.int32)
    pix[:20] = pix[20:40]
    flux = rng.uniform(0.1, 1.0, 400)
    l = (pix % n - n // 2).astype(np.float64) * dl
    m = (pix // n - n // 2).astype(np.float64) * dl
    table = wt.wt_xref_table(n, dl, synth.RA0, synth.DEC0, J)
    tx = wt.wt_build_tree_xref(table, dev(pix), dev(flux), synth.RA0, synth.DEC0, J).export()
    tl = wt.wt_build_tree(dev(l), dev(m), dev(flux), synth.RA0, synth.DEC0, J).export()
    for k in tl:
        assert np.array_equal(np.asarray(tx[k]), np.asarray(tl[k])), k


def test_tree_from_xref_bad_pixel_is_reported():
    n, J = 16, 10
    table = wt.wt_xref_table(n, 1e-4, synth.RA0, synth.DEC0, J)
    wt.wt_device_status()
    t = wt.wt_build_tree_xref(table, dev(np.array([3, n * n + 5], np.int32)), dev(np.ones(2)),
                              synth.RA0, synth.DEC0, J)
    with pytest.raises(wt.WtError) as e:
        wt.wt_device_status()
    assert e.value.status == wt.WT_ERR_RANGE
    t.close()
    wt.wt_device_status()
