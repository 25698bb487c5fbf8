"""The direct sum (Eq. 12) with its phase contraction on the tensor cores
(WT_MIXED_TC): exact float16 slices of the baselines and of the component
coordinates, summed by tcgen05.mma into three FP32 accumulators and
recombined modulo 1 in float32. Held to the mixed forms' bar (1e-6 of
sum |C|) against the oracle's Eq. 12 on the synthetic workloads, across
stage and chunk boundaries, ragged tiles, both signs, the degenerate skies,
and tiles beyond the tensor-core range (left to the exact pass).
"""
import numpy as np
import pytest

import oracle as O
import synth

torch = pytest.importorskip("torch")
wt = pytest.importorskip("paper_1909_03956_gb300")

pytestmark = pytest.mark.gpu

TOLMIX = 1e-6


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def predict(l, m, f, uvw, mode=wt.WT_MIXED_TC, sign=1):
    return wt.dft_predict_vis(dev(l), dev(m), dev(f), dev(uvw), mode=mode, sign=sign).cpu().numpy()


def rel_err(l, m, f, uvw, sign=1):
    v = predict(l, m, f, uvw, sign=sign)
    return float(np.max(np.abs(v - O.dft(l, m, f, uvw, sign))) / np.abs(f).sum())


def sky(n, half_width_rad, rng):
    return (rng.uniform(-half_width_rad, half_width_rad, n), rng.uniform(-half_width_rad, half_width_rad, n),
            10.0 ** rng.uniform(-3, 0, n))


def test_small_workload_every_visibility_both_signs():
    w = synth.small()
    assert rel_err(w.l, w.m, w.flux, w.uvw) <= TOLMIX
    assert rel_err(w.l, w.m, w.flux, w.uvw, sign=-1) <= TOLMIX


def test_medium_workload_sample():
    # 5 000 clustered components (40 stages of 128) against a strided sample
    # of the medium array's visibilities, ragged at both ends
    w = synth.medium()
    uvw = w.uvw[::97][:12345]
    assert rel_err(w.l, w.m, w.flux, uvw) <= TOLMIX


@pytest.mark.parametrize("n_comp", [1, 31, 32, 33, 127, 128, 129, 257, 1000])
def test_chunk_and_stage_boundaries(n_comp):
    rng = np.random.default_rng(900 + n_comp)
    l, m, f = sky(n_comp, 0.03, rng)
    uvw = rng.uniform(-4e4, 4e4, (1000, 3))   # 7 full tiles and a ragged one
    assert rel_err(l, m, f, uvw) <= TOLMIX


def test_matches_the_fast_mixed_form():
    # same terms, same sin/cos unit: the two forms differ by their phases'
    # last roundings only
    rng = np.random.default_rng(910)
    l, m, f = sky(3000, 0.02, rng)
    uvw = rng.uniform(-3e4, 3e4, (5000, 3))
    a = predict(l, m, f, uvw)
    b = predict(l, m, f, uvw, mode=wt.WT_MIXED_FAST)
    assert np.max(np.abs(a - b)) / f.sum() <= TOLMIX


def test_single_component_worst_case():
    # one component: no averaging over terms, the per-term bound must hold
    rng = np.random.default_rng(911)
    l, m, f = np.array([0.0123]), np.array([-0.0071]), np.array([1.0])
    for scale in (3e3, 3e5):
        uvw = rng.uniform(-scale, scale, (20000, 3))
        assert rel_err(l, m, f, uvw) <= TOLMIX
        assert rel_err(l, m, f, uvw, sign=-1) <= TOLMIX


def test_degenerate_skies():
    rng = np.random.default_rng(912)
    uvw = rng.uniform(-5e4, 5e4, (700, 3))
    # every component at the phase centre: each coordinate's bound is 0 and
    # V = sum of the fluxes on every baseline
    f = 10.0 ** rng.uniform(-3, 0, 40)
    z = np.zeros(40)
    v = predict(z, z, f, uvw)
    assert np.max(np.abs(v - f.sum())) / f.sum() <= TOLMIX
    # components on the l axis only (m and n - 1 bounds from l alone)
    l = rng.uniform(-0.01, 0.01, 40)
    assert rel_err(l, z, f, uvw) <= TOLMIX
    # zero baselines: V = sum of the fluxes
    l, m, f = sky(60, 0.05, rng)
    v = predict(l, m, f, np.zeros((300, 3)))
    assert np.max(np.abs(v - f.sum())) / f.sum() <= TOLMIX
    # no components: every visibility 0
    e = np.zeros(0)
    v = predict(e, e, e, uvw)
    assert np.array_equal(v, np.zeros(len(uvw), dtype=v.dtype))


def test_tiles_beyond_the_tensor_core_range():
    # long baselines in one visibility of every 500: the 128-visibility tiles
    # that hold one exceed 2^14 turns per coordinate and take the exact pass
    rng = np.random.default_rng(913)
    l, m, f = sky(200, 0.3, rng)
    uvw = rng.uniform(-2e3, 2e3, (6000, 3))
    uvw[::500] = rng.uniform(5e4, 8e4, (len(uvw[::500]), 3)) * rng.choice([-1.0, 1.0], (len(uvw[::500]), 3))
    assert rel_err(l, m, f, uvw) <= TOLMIX
    assert rel_err(l, m, f, uvw, sign=-1) <= TOLMIX


def test_repeatable_and_status_clear():
    rng = np.random.default_rng(914)
    l, m, f = sky(500, 0.02, rng)
    uvw = rng.uniform(-3e4, 3e4, (2000, 3))
    a = predict(l, m, f, uvw)
    b = predict(l, m, f, uvw)
    assert np.array_equal(a, b)
    wt.wt_device_status()   # raises on a recorded device-side error


# ---------------------------------------------------------------- Eq. 16

def eq16_err(w, J, uvw, sign=1):
    """Eq. 16 in the tensor-core form against the oracle's Eq. 16 (the leaves'
    pixel centres with their merged fluxes), relative to sum |C|."""
    t = wt.wt_build_tree(dev(w.l), dev(w.m), dev(w.flux), w.ra0, w.dec0, J)
    try:
        v = wt.wt_predict_vis(t, dev(uvw), mode=wt.WT_MIXED_TC, which=wt.WT_SUM_EQ16, sign=sign).cpu().numpy()
    finally:
        t.close()
    ref = O.Tree(w.l, w.m, w.flux, w.ra0, w.dec0, J).vis_eq16(uvw, sign)
    return float(np.max(np.abs(v - ref)) / np.abs(w.flux).sum())


@pytest.mark.parametrize("J", [1, 6, 12, 18])
def test_eq16_small_workload(J):
    w = synth.small()
    assert eq16_err(w, J, w.uvw) <= TOLMIX
    assert eq16_err(w, J, w.uvw[:999], sign=-1) <= TOLMIX


def test_eq16_medium_workload():
    # 1 115 leaves at J = 12 (9 stages of 128, the last one ragged)
    w = synth.medium(n_t=6)
    assert eq16_err(w, 12, w.uvw[::3]) <= TOLMIX


def test_eq16_matches_the_fast_form_and_other_sums_are_refused():
    w = synth.medium(n_t=4)
    t = wt.wt_build_tree(dev(w.l), dev(w.m), dev(w.flux), w.ra0, w.dec0, 12)
    try:
        u = dev(w.uvw)
        a = wt.wt_predict_vis(t, u, mode=wt.WT_MIXED_TC, which=wt.WT_SUM_EQ16).cpu().numpy()
        b = wt.wt_predict_vis(t, u, mode=wt.WT_MIXED_FAST, which=wt.WT_SUM_EQ16).cpu().numpy()
        assert np.max(np.abs(a - b)) / np.abs(w.flux).sum() <= TOLMIX
        for which in (wt.WT_SUM_EQ17, wt.WT_SUM_EQ17_REGROUPED):
            with pytest.raises(wt.WtError) as e:
                wt.wt_predict_vis(t, u, mode=wt.WT_MIXED_TC, which=which)
            assert e.value.status == wt.WT_ERR_UNSUPPORTED
    finally:
        t.close()


def test_eq16_empty_tree_and_long_baselines():
    rng = np.random.default_rng(915)
    e = np.zeros(0)
    t = wt.wt_build_tree(dev(e), dev(e), dev(e), synth.RA0, synth.DEC0, 10)
    try:
        v = wt.wt_predict_vis(t, dev(rng.uniform(-1e4, 1e4, (300, 3))), mode=wt.WT_MIXED_TC,
                              which=wt.WT_SUM_EQ16).cpu().numpy()
        assert np.array_equal(v, np.zeros(300, dtype=v.dtype))
    finally:
        t.close()
    # a wide field and baselines beyond the tensor-core range in some tiles
    w = synth.small()
    uvw = w.uvw.copy()
    uvw[::300] *= 400.0
    assert eq16_err(w, 14, uvw) <= TOLMIX


# ------------------------------------------------- truncated and thresholded

def test_large_level_of_truncation_and_thresholding():
    # level 11 of the medium sky's J = 12 tree has 409 nodes, above
    # WT_TRUNCATED_TC_MIN_NODES: the truncated and the thresholded (j0 = 11)
    # predictors sum it on the tensor cores
    from oracle import threshold as T
    J, j0 = 12, 11
    w = synth.medium(n_t=3)
    uvw = w.uvw[::7][:2000]
    t = wt.wt_build_tree(dev(w.l), dev(w.m), dev(w.flux), w.ra0, w.dec0, J)
    try:
        assert t.info()["per_level"][j0 - 1] >= wt.WT_TRUNCATED_TC_MIN_NODES
        tol = TOLMIX * np.abs(w.flux).sum()
        tr = O.Tree(w.l, w.m, w.flux, w.ra0, w.dec0, J)
        got = wt.wt_predict_vis_truncated(t, j0, dev(uvw)).cpu().numpy()
        assert np.max(np.abs(got - tr.vis_truncated(j0, uvw, kind="snapped"))) <= tol
        base, G, S = T.full_response_terms(tr.export(), J, j0, uvw, w.ra0, w.dec0, d_leaf=1, reading="snapped")
        tau = float(np.median(np.abs(G)))
        th = wt.wt_predict_vis_thresholded(t, j0, tau, dev(uvw), response=wt.WT_RESPONSE_SNAPPED).cpu().numpy()
        assert np.max(np.abs(th - T.thresholded_vis_tau(base, G, S, tau))) <= tol
        # nothing kept below j0: the truncated tree, bit for bit
        none = wt.wt_predict_vis_thresholded(t, j0, np.inf, dev(uvw), response=wt.WT_RESPONSE_SNAPPED).cpu().numpy()
        assert np.array_equal(none, got)
    finally:
        t.close()


# ---------------------------------------------------------------- major cycle

def test_clean_with_the_tensor_core_direct_sum_matches_the_oracle():
    # one major cycle of wt_clean with the direct-sum predictor in WT_MIXED_TC
    # (and its subtraction, complex64) against the imaging oracle's cycle
    from oracle import imaging as I
    n = 64
    w = synth.small()
    uvw = w.uvw * np.array([1.0, 1.0, 0.0])
    dl = 0.45 / np.max(np.abs(uvw[:, :2]))
    src = [(n // 2 + 6, n // 2 - 4, 1.0), (n // 2 - 9, n // 2 + 5, 0.6)]
    l = np.array([(x - n // 2) * dl for x, y, _ in src])
    m = np.array([(y - n // 2) * dl for x, y, _ in src])
    f = np.array([s[2] for s in src])
    obs = O.dft(l, m, f, uvw)
    pix, flux, resid, img = wt.wt_clean(dev(uvw), dev(obs.astype(np.complex64)), n, dl, synth.RA0, synth.DEC0, 12,
                                        predictor=wt.WT_PREDICT_DIRECT, mode=wt.WT_MIXED_TC, gain=0.2,
                                        minor_iter=20, n_major=1)
    pix_o, flux_o, resid_o, img_o = I.major_cycles(uvw, obs, n, dl, 0.2, 20, 0.0, 1,
                                                   lambda a, b, c, d: O.dft(a, b, c, d))
    assert np.array_equal(pix.cpu().numpy(), pix_o.astype(np.int32))
    assert np.allclose(flux.cpu().numpy(), flux_o, rtol=1e-4)
    assert np.max(np.abs(resid.cpu().numpy() - resid_o)) <= 1e-4 * np.max(np.abs(obs))
    # the tree predictor has no tensor-core form of its regrouped sum
    with pytest.raises(wt.WtError):
        wt.wt_clean(dev(uvw), dev(obs.astype(np.complex64)), n, dl, synth.RA0, synth.DEC0, 12,
                    predictor=wt.WT_PREDICT_TREE, mode=wt.WT_MIXED_TC, minor_iter=5, n_major=1)
