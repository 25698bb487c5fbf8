"""Parity at the full workload sizes, in the launch configuration the bench
times (autotuned shapes, the same entry points), on strided samples of the
outputs that the oracle computes one by one.

Workloads: medium (1 008 000 visibilities, 5 000 components, J = 12);
mixed (2 032 000 visibilities at 1.3 GHz, 20 000 components, J = 12);
learned-response array (15 993 600 visibilities, 50 000 components, J = 12);
batched (64 channels x 2 032 000 visibilities, uneven trees).
"""
import numpy as np
import pytest

import oracle as O
import synth

torch = pytest.importorskip("torch")
wt = pytest.importorskip("paper_1909_03956_gb300")

pytestmark = pytest.mark.gpu

TOL = {wt.WT_FP64: 1e-10, wt.WT_MIXED: 1e-6, wt.WT_MIXED_FAST: 1e-6}


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def _sample(n, k=300):
    return np.unique(np.concatenate([np.arange(0, n, max(1, n // k)), [n - 1]]))


@pytest.mark.parametrize("mode", [wt.WT_MIXED_FAST, wt.WT_MIXED, wt.WT_FP64])
def test_medium_full_size(mode):
    w = synth.medium(J=12)
    t = wt.wt_build_tree(dev(w.l), dev(w.m), dev(w.flux), w.ra0, w.dec0, w.J)
    v = wt.wt_predict_vis(t, dev(w.uvw), mode=mode).cpu().numpy()
    idx = _sample(w.n_vis)
    ref = O.Tree(w.l, w.m, w.flux, w.ra0, w.dec0, w.J).vis_eq17(w.uvw[idx])
    assert np.max(np.abs(v[idx] - ref)) / np.abs(w.flux).sum() <= TOL[mode]


def test_mixed_config_full_size_wavelet_and_direct():
    w = synth.mixed()
    uvw = w.uvw
    t = wt.wt_build_tree(dev(w.l), dev(w.m), dev(w.flux), w.ra0, w.dec0, w.J)
    vw = wt.wt_predict_vis(t, dev(uvw), mode=wt.WT_MIXED).cpu().numpy()
    vd = wt.dft_predict_vis(dev(w.l), dev(w.m), dev(w.flux), dev(uvw), mode=wt.WT_MIXED).cpu().numpy()
    idx = _sample(w.n_vis, 200)
    S = np.abs(w.flux).sum()
    assert np.max(np.abs(vw[idx] - O.Tree(w.l, w.m, w.flux, w.ra0, w.dec0, w.J).vis_eq17(uvw[idx]))) / S <= 1e-6
    assert np.max(np.abs(vd[idx] - O.dft(w.l, w.m, w.flux, uvw[idx]))) / S <= 1e-6


def test_learned_array_full_size_mixed():
    w = synth.learned()
    t = wt.wt_build_tree(dev(w.l), dev(w.m), dev(w.flux), w.ra0, w.dec0, w.J)
    v = wt.wt_predict_vis(t, dev(w.uvw), mode=wt.WT_MIXED).cpu().numpy()
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
