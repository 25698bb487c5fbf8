"""Parity at the full workload sizes, in the launch configuration the bench
times (autotuned shapes, the same entry points), on strided samples of the
outputs that the oracle computes one by one.

Workloads: medium (1 008 000 visibilities, 5 000 components, J = 12, and
J = 8, 14); isolated components (140, J = 20 and 25);
mixed (2 032 000 visibilities at 1.3 GHz, 20 000 components, J = 12);
learned-response array and the large array (15 993 600 visibilities, 50 000
components, J = 12; the large one's Eq. 16 and truncation on the tensor cores);
batched (64 channels x 2 032 000 visibilities, uneven trees).
"""
import numpy as np
import pytest

import oracle as O
import synth

torch = pytest.importorskip("torch")
wt = pytest.importorskip("paper_1909_03956_gb300")

pytestmark = pytest.mark.gpu

TOL = {wt.WT_FP64: 1e-10, wt.WT_FP64_DF: 1e-10, wt.WT_MIXED: 1e-6, wt.WT_MIXED_FAST: 1e-6}


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def _sample(n, k=300):
    return np.unique(np.concatenate([np.arange(0, n, max(1, n // k)), [n - 1]]))


@pytest.mark.parametrize("mode,which", [(m, w) for m in (wt.WT_MIXED_FAST, wt.WT_MIXED, wt.WT_FP64)
                                        for w in (wt.WT_SUM_EQ17_REGROUPED, wt.WT_SUM_EQ17)]
                         + [(wt.WT_FP64_DF, wt.WT_SUM_EQ17_REGROUPED)])
def test_medium_full_size(mode, which):
    # the bench's step uses the regrouped sum in the fast form, autotuned shape
    w = synth.medium(J=12)
    t = wt.wt_build_tree(dev(w.l), dev(w.m), dev(w.flux), w.ra0, w.dec0, w.J)
    v = wt.wt_predict_vis(t, dev(w.uvw), mode=mode, which=which).cpu().numpy()
    idx = _sample(w.n_vis)
    ref = O.Tree(w.l, w.m, w.flux, w.ra0, w.dec0, w.J).vis_eq17(w.uvw[idx])
    assert np.max(np.abs(v[idx] - ref)) / np.abs(w.flux).sum() <= TOL[mode]


@pytest.mark.parametrize("J", [8, 14])
def test_medium_full_size_regrouped_fast_other_depths(J):
    # the ends of the bench's J sweep, in the bench's form
    w = synth.medium(J=J)
    t = wt.wt_build_tree(dev(w.l), dev(w.m), dev(w.flux), w.ra0, w.dec0, w.J)
    v = wt.wt_predict_vis(t, dev(w.uvw), mode=wt.WT_MIXED_FAST, which=wt.WT_SUM_EQ17_REGROUPED).cpu().numpy()
    idx = _sample(w.n_vis, 150)
    ref = O.Tree(w.l, w.m, w.flux, w.ra0, w.dec0, w.J).vis_eq17(w.uvw[idx])
    assert np.max(np.abs(v[idx] - ref)) / np.abs(w.flux).sum() <= 1e-6


@pytest.mark.parametrize("J", [20, 25])
def test_isolated_components_deep_tree_regrouped_fast(J):
    # deep, sparse trees (every component alone in its pixel: chains of
    # single-child nodes), the paper's wide-field regime
    w = synth.medium_fixed(140, J=J)
    t = wt.wt_build_tree(dev(w.l), dev(w.m), dev(w.flux), w.ra0, w.dec0, w.J)
    v = wt.wt_predict_vis(t, dev(w.uvw), mode=wt.WT_MIXED_FAST, which=wt.WT_SUM_EQ17_REGROUPED).cpu().numpy()
    idx = _sample(w.n_vis, 150)
    ref = O.Tree(w.l, w.m, w.flux, w.ra0, w.dec0, w.J).vis_eq17(w.uvw[idx])
    assert np.max(np.abs(v[idx] - ref)) / np.abs(w.flux).sum() <= 1e-6


def test_mixed_config_full_size_wavelet_and_direct():
    w = synth.mixed()
    uvw = w.uvw
    t = wt.wt_build_tree(dev(w.l), dev(w.m), dev(w.flux), w.ra0, w.dec0, w.J)
    vw = wt.wt_predict_vis(t, dev(uvw), mode=wt.WT_MIXED).cpu().numpy()
    vr = wt.wt_predict_vis(t, dev(uvw), mode=wt.WT_MIXED_FAST, which=wt.WT_SUM_EQ17_REGROUPED).cpu().numpy()
    vd = wt.dft_predict_vis(dev(w.l), dev(w.m), dev(w.flux), dev(uvw), mode=wt.WT_MIXED).cpu().numpy()
    idx = _sample(w.n_vis, 200)
    S = np.abs(w.flux).sum()
    ref = O.Tree(w.l, w.m, w.flux, w.ra0, w.dec0, w.J).vis_eq17(uvw[idx])
    assert np.max(np.abs(vw[idx] - ref)) / S <= 1e-6
    assert np.max(np.abs(vr[idx] - ref)) / S <= 1e-6
    ref_d = O.dft(w.l, w.m, w.flux, uvw[idx])
    assert np.max(np.abs(vd[idx] - ref_d)) / S <= 1e-6
    # the direct sum with its phases on the tensor cores, as the bench times it
    vt = wt.dft_predict_vis(dev(w.l), dev(w.m), dev(w.flux), dev(uvw), mode=wt.WT_MIXED_TC).cpu().numpy()
    assert np.max(np.abs(vt[idx] - ref_d)) / S <= 1e-6


def test_large_array_full_size_eq16_and_truncation_on_the_tensor_cores():
    # 15 993 600 visibilities, 50 000 components, J = 12: Eq. 16 over the
    # 1 663 leaves and the truncation at level 11 (522 nodes), both on the
    # tensor cores, on a strided sample against the oracle
    w = synth.large()
    t = wt.wt_build_tree(dev(w.l), dev(w.m), dev(w.flux), w.ra0, w.dec0, w.J)
    u = dev(w.uvw)
    v16 = wt.wt_predict_vis(t, u, mode=wt.WT_MIXED_TC, which=wt.WT_SUM_EQ16).cpu().numpy()
    v11 = wt.wt_predict_vis_truncated(t, 11, u).cpu().numpy()
    t.close()
    idx = _sample(w.n_vis, 200)
    S = np.abs(w.flux).sum()
    ot = O.Tree(w.l, w.m, w.flux, w.ra0, w.dec0, w.J)
    assert np.max(np.abs(v16[idx] - ot.vis_eq16(w.uvw[idx]))) / S <= 1e-6
    assert np.max(np.abs(v11[idx] - ot.vis_truncated(11, w.uvw[idx], kind="snapped"))) / S <= 1e-6


@pytest.mark.parametrize("mode,which", [(wt.WT_MIXED, wt.WT_SUM_EQ17),
                                        (wt.WT_MIXED_FAST, wt.WT_SUM_EQ17_REGROUPED)])
def test_learned_array_full_size_mixed(mode, which):
    w = synth.learned()
    t = wt.wt_build_tree(dev(w.l), dev(w.m), dev(w.flux), w.ra0, w.dec0, w.J)
    v = wt.wt_predict_vis(t, dev(w.uvw), mode=mode, which=which).cpu().numpy()
    idx = _sample(w.n_vis, 200)
    ref = O.Tree(w.l, w.m, w.flux, w.ra0, w.dec0, w.J).vis_eq17(w.uvw[idx])
    assert np.max(np.abs(v[idx] - ref)) / np.abs(w.flux).sum() <= 1e-6


def test_batched_full_size():
    w = synth.batched()
    chans = w.extra["channels"]
    uvw_m = w.extra["uvw_m"]
    trees = [wt.wt_build_tree(dev(c["l"]), dev(c["m"]), dev(c["flux"]), w.ra0, w.dec0, c["J"]) for c in chans]
    v = wt.wt_predict_vis_batched(trees, [c["freq"] for c in chans], dev(uvw_m), mode=wt.WT_MIXED_FAST)
    idx = _sample(uvw_m.shape[0], 40)
    got = v.cpu().numpy()[:, idx]
    for c, ch in enumerate(chans):
        ref = O.Tree(ch["l"], ch["m"], ch["flux"], w.ra0, w.dec0, ch["J"]).vis_eq17(
            uvw_m[idx] * (ch["freq"] / synth.C_LIGHT))
        assert np.max(np.abs(got[c] - ref)) / np.abs(ch["flux"]).sum() <= 1e-6, c
