"""wt_predict_vis_batched: many channels, uneven trees, one persistent
graph-captured launch -- against the oracle, channel by channel.

The oracle evaluates Eq. 17 on each channel's own tree with the baselines
scaled to that channel's wavelength, u_lambda = u_m f_c / c.
"""
import numpy as np
import pytest

import oracle as O
import synth

torch = pytest.importorskip("torch")
wt = pytest.importorskip("paper_1909_03956_gb300")

pytestmark = pytest.mark.gpu

C_LIGHT = 299792458.0
TOL = {wt.WT_FP64: 1e-10, wt.WT_MIXED: 1e-6, wt.WT_MIXED_FAST: 1e-6}


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def _channels(n_ch, seed=5):
    rng = np.random.default_rng(seed)
    chans = []
    for c in range(n_ch):
        n = int(10 ** rng.uniform(1.0, 3.3))          # uneven: 10 .. 2000 components
        J = int(rng.integers(6, 14))
        l, m, f = synth.components_blobs(5, max(1, n // 5), 2.0, rng)
        chans.append(dict(l=l, m=m, flux=f, J=J, freq=float(rng.uniform(1.0e9, 1.8e9))))
    return chans


def _uvw_m(n, seed=6):
    rng = np.random.default_rng(seed)
    return rng.uniform(-4000.0, 4000.0, (n, 3)) * np.array([1.0, 1.0, 0.05])


def _oracle(chans, uvw_m, sign=1):
    out = []
    for ch in chans:
        t = O.Tree(ch["l"], ch["m"], ch["flux"], synth.RA0, synth.DEC0, ch["J"])
        out.append(t.vis_eq17(uvw_m * (ch["freq"] / C_LIGHT), sign))
    return out


def _gpu_trees(chans):
    return [wt.wt_build_tree(dev(c["l"]), dev(c["m"]), dev(c["flux"]), synth.RA0, synth.DEC0, c["J"]) for c in chans]


def _df_bar(ch, uvw):
    """The double-float form's bar (see the single-tree parity tests): the
    float64 bar, or 2 pi 2^-45 max |B.s| where phases reach beyond about
    500 turns."""
    d = np.abs(O.Tree(ch["l"], ch["m"], ch["flux"], synth.RA0, synth.DEC0, ch["J"]).export()["leaf_dir"])
    return max(TOL[wt.WT_FP64], 2 * np.pi * 2.0 ** -45 * float(np.max(np.abs(uvw) @ d.T)))


@pytest.mark.parametrize("mode", [wt.WT_FP64, wt.WT_FP64_DF, wt.WT_MIXED, wt.WT_MIXED_FAST])
def test_batched_matches_oracle_per_channel(mode):
    chans = _channels(9)
    uvw_m = _uvw_m(3001)                       # ragged against every tile size
    trees = _gpu_trees(chans)
    v = wt.wt_predict_vis_batched(trees, [c["freq"] for c in chans], dev(uvw_m), mode=mode).cpu().numpy()
    ref = _oracle(chans, uvw_m)
    for c, ch in enumerate(chans):
        err = np.max(np.abs(v[c] - ref[c])) / np.abs(ch["flux"]).sum()
        bar = _df_bar(ch, uvw_m * (ch["freq"] / C_LIGHT)) if mode == wt.WT_FP64_DF else TOL[mode]
        assert err <= bar, (c, err)


@pytest.mark.parametrize("shape", range(6))
@pytest.mark.parametrize("mode", [wt.WT_MIXED, wt.WT_MIXED_FAST])
def test_batched_every_launch_shape(shape, mode, monkeypatch):
    # each (threads per CTA, visibilities per thread) shape the batched
    # autotuner may pick gives the oracle's answer on a ragged batch
    monkeypatch.setenv("WT_BATCH_SHAPE", str(shape))
    chans = _channels(4, seed=21 + shape)
    uvw_m = _uvw_m(2999, seed=22)
    trees = _gpu_trees(chans)
    v = wt.wt_predict_vis_batched(trees, [c["freq"] for c in chans], dev(uvw_m), mode=mode).cpu().numpy()
    ref = _oracle(chans, uvw_m)
    for c, ch in enumerate(chans):
        assert np.max(np.abs(v[c] - ref[c])) / np.abs(ch["flux"]).sum() <= TOL[mode], c
    for t in trees:
        t.close()


@pytest.mark.parametrize("mode", [wt.WT_FP64, wt.WT_MIXED_FAST])
def test_batched_persistent_queue_matches_oracle(mode, monkeypatch):
    # the persistent work queue (a fixed grid taking items from an atomic
    # counter), forced on a small batch
    monkeypatch.setenv("WT_BATCH_QUEUE", "1")
    chans = _channels(6, seed=31)
    uvw_m = _uvw_m(4097, seed=32)
    trees = _gpu_trees(chans)
    v = wt.wt_predict_vis_batched(trees, [c["freq"] for c in chans], dev(uvw_m), mode=mode).cpu().numpy()
    ref = _oracle(chans, uvw_m)
    for c, ch in enumerate(chans):
        assert np.max(np.abs(v[c] - ref[c])) / np.abs(ch["flux"]).sum() <= TOL[mode], c
    for t in trees:
        t.close()


def test_batched_double_float_equals_single_channel_calls():
    chans = _channels(5, seed=12)
    uvw_m = _uvw_m(2048, seed=13)
    trees = _gpu_trees(chans)
    freqs = [c["freq"] for c in chans]
    v = wt.wt_predict_vis_batched(trees, freqs, dev(uvw_m), mode=wt.WT_FP64_DF, sign=-1).cpu().numpy()
    for c, ch in enumerate(chans):
        u = dev(uvw_m * (ch["freq"] / C_LIGHT))
        s = wt.wt_predict_vis(trees[c], u, mode=wt.WT_FP64_DF, sign=-1).cpu().numpy()
        assert np.max(np.abs(v[c] - s)) <= 1e-12 * np.abs(ch["flux"]).sum()


def test_batched_equals_single_channel_calls_and_sign():
    chans = _channels(5, seed=9)
    uvw_m = _uvw_m(2048, seed=10)
    trees = _gpu_trees(chans)
    freqs = [c["freq"] for c in chans]
    for sign in (1, -1):
        v = wt.wt_predict_vis_batched(trees, freqs, dev(uvw_m), mode=wt.WT_FP64, sign=sign).cpu().numpy()
        for c, ch in enumerate(chans):
            u = dev(uvw_m * (ch["freq"] / C_LIGHT))
            s = wt.wt_predict_vis(trees[c], u, mode=wt.WT_FP64, sign=sign).cpu().numpy()
            assert np.max(np.abs(v[c] - s)) <= 1e-12 * np.abs(ch["flux"]).sum()


def test_batched_graph_replay_sees_new_inputs_and_new_buffers():
    chans = _channels(4, seed=11)
    trees = _gpu_trees(chans)
    freqs = [c["freq"] for c in chans]
    uvw = dev(_uvw_m(1500, seed=12))
    out = torch.empty((4, 1500), dtype=torch.complex64, device="cuda")
    wt.wt_predict_vis_batched(trees, freqs, uvw, mode=wt.WT_MIXED, out=out)
    # same buffers, new contents: the replayed graph reads them
    new = _uvw_m(1500, seed=13)
    uvw.copy_(dev(new))
    wt.wt_predict_vis_batched(trees, freqs, uvw, mode=wt.WT_MIXED, out=out)
    ref = _oracle(chans, new)
    got = out.cpu().numpy()
    for c, ch in enumerate(chans):
        assert np.max(np.abs(got[c] - ref[c])) / np.abs(ch["flux"]).sum() <= TOL[wt.WT_MIXED]
    # other buffers and another size: a new capture
    new2 = _uvw_m(777, seed=14)
    got2 = wt.wt_predict_vis_batched(trees, freqs, dev(new2), mode=wt.WT_MIXED).cpu().numpy()
    ref2 = _oracle(chans, new2)
    for c, ch in enumerate(chans):
        assert np.max(np.abs(got2[c] - ref2[c])) / np.abs(ch["flux"]).sum() <= TOL[wt.WT_MIXED]


def test_batched_after_freeing_a_tree():
    chans = _channels(3, seed=15)
    trees = _gpu_trees(chans)
    freqs = [c["freq"] for c in chans]
    uvw_m = _uvw_m(600, seed=16)
    wt.wt_predict_vis_batched(trees, freqs, dev(uvw_m), mode=wt.WT_FP64)
    trees[1].close()                            # drops the plan that used it
    trees[1] = wt.wt_build_tree(dev(chans[1]["l"]), dev(chans[1]["m"]), dev(chans[1]["flux"]), synth.RA0,
                                synth.DEC0, chans[1]["J"])
    v = wt.wt_predict_vis_batched(trees, freqs, dev(uvw_m), mode=wt.WT_FP64).cpu().numpy()
    ref = _oracle(chans, uvw_m)
    for c, ch in enumerate(chans):
        assert np.max(np.abs(v[c] - ref[c])) / np.abs(ch["flux"]).sum() <= TOL[wt.WT_FP64]


def test_batched_rejects_bad_arguments():
    chans = _channels(2, seed=17)
    trees = _gpu_trees(chans)
    uvw = dev(_uvw_m(10))
    with pytest.raises(wt.WtError):
        wt.wt_predict_vis_batched(trees, [1e9, -1.0], uvw)
    with pytest.raises(ValueError):
        wt.wt_predict_vis_batched(trees, [1e9], uvw)
