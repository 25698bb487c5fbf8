"""Checkpoint and resume on the GPU.

* a tree exported (wt_tree_export) and imported again from its leaves
  (wt_tree_import) is the same tree bit for bit -- keys, topology, lambda,
  gamma, pixel centres -- and predicts the same visibilities bit for bit;
* a training run of the response network cut into two ranges, with the
  optimiser state saved and restored into a fresh network in between, ends
  with the same parameters, bit for bit, as the run done in one go (and two
  runs done in one go agree with each other).
"""
import numpy as np
import pytest

import oracle as O
import synth

torch = pytest.importorskip("torch")
wt = pytest.importorskip("paper_1909_03956_gb300")

pytestmark = pytest.mark.gpu


def dev(a, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    return t.to(dtype) if dtype is not None else t


def _skies():
    w = synth.medium(n_t=2)
    yield w, 12
    s = synth.small()
    # duplicated components and mixed-sign fluxes (a zero-sum leaf among them)
    l = np.concatenate([s.l, s.l[:10]])
    m = np.concatenate([s.m, s.m[:10]])
    f = np.concatenate([s.flux, -s.flux[:10]])
    yield synth.Workload("dup", s.uvw, l, m, f, 9), 9


@pytest.mark.parametrize("case", [0, 1])
def test_tree_export_import_round_trip(case):
    w, J = list(_skies())[case]
    t = wt.wt_build_tree(dev(w.l), dev(w.m), dev(w.flux), w.ra0, w.dec0, J)
    a = t.export()
    nl = a["n_leaves"]
    t2 = wt.wt_tree_import(a["key"][-nl:], a["leaf_flux"], w.ra0, w.dec0, J)
    b = t2.export()
    for k in ("key", "child_mask", "first_child", "lam", "gamma", "leaf_dir", "leaf_flux", "level_offsets"):
        assert np.array_equal(a[k], b[k]), k
    uvw = dev(w.uvw[:3000])
    for mode, which in ((wt.WT_MIXED_FAST, wt.WT_SUM_EQ17_REGROUPED), (wt.WT_FP64, wt.WT_SUM_EQ17),
                        (wt.WT_FP64_DF, wt.WT_SUM_EQ17_REGROUPED)):
        va = wt.wt_predict_vis(t, uvw, mode=mode, which=which).cpu().numpy()
        vb = wt.wt_predict_vis(t2, uvw, mode=mode, which=which).cpu().numpy()
        assert np.array_equal(va, vb)
    # and the oracle's tree agrees with the imported one as with the original
    o = O.Tree(w.l, w.m, w.flux, w.ra0, w.dec0, J).export()
    assert np.array_equal(o["key"], b["key"]) and np.array_equal(o["lam"], b["lam"])
    t.close()
    t2.close()


def test_tree_import_rejects_bad_leaves():
    with pytest.raises(wt.WtError):
        wt.wt_tree_import([5, 3], [1.0, 1.0], synth.RA0, synth.DEC0, 4)          # not ascending
    with pytest.raises(wt.WtError):
        wt.wt_tree_import([12 * 4 ** 3], [1.0], synth.RA0, synth.DEC0, 4)        # not a level-4 pixel
    with pytest.raises(wt.WtError):
        wt.wt_tree_import([1], [np.nan], synth.RA0, synth.DEC0, 4)


def _data(level, n=50000, seed=3):
    rng = np.random.default_rng(seed)
    pool = synth.medium(n_t=20).uvw
    uvw = pool[rng.integers(0, len(pool), n)]
    tgt = O.pixel_response(level, 3, synth.RA0, synth.DEC0, uvw)
    return dev(uvw), dev(np.stack([tgt.real, tgt.imag], axis=1), torch.float32)


def test_training_resumes_bit_identically():
    level, total, cut = 12, 120, 47
    uvw, tgt = _data(level)
    kw = dict(batch=4096, lr=3e-3)
    a = wt.Mlp(level, synth.RA0, synth.DEC0, depth=3, x_max=1e30, seed=3)
    a.train_range(uvw, tgt, 0, total, total, **kw)
    a2 = wt.Mlp(level, synth.RA0, synth.DEC0, depth=3, x_max=1e30, seed=3)
    a2.train(uvw, tgt, total, **kw)
    b = wt.Mlp(level, synth.RA0, synth.DEC0, depth=3, x_max=1e30, seed=3)
    b.train_range(uvw, tgt, 0, cut, total, **kw)
    state = b.get_state()
    assert state[3] == cut
    c = wt.Mlp(level, synth.RA0, synth.DEC0, depth=3, x_max=1e30, seed=99)   # another start, overwritten
    c.set_state(*state)
    c.train_range(uvw, tgt, cut, total - cut, total, **kw)
    pa, pa2, pc = a.get_params(), a2.get_params(), c.get_params()
    assert np.array_equal(pa, pa2)
    assert np.array_equal(pa, pc)
    assert np.array_equal(a.get_state()[1], c.get_state()[1]) and np.array_equal(a.get_state()[2], c.get_state()[2])
    ya, yc = a.eval(uvw[:1000]).cpu().numpy(), c.eval(uvw[:1000]).cpu().numpy()
    assert np.array_equal(ya, yc)
    for m in (a, a2, b, c):
        m.close()
