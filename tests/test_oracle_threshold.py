"""Hard thresholding of Eq. 17's wavelet coefficients (oracle/threshold.py,
reading T1), pinned and measured on the CPU."""
import math

import numpy as np

import oracle as O
import synth
from oracle import threshold as T


def _terms(w, J, uvw):
    tr = O.Tree(w.l, w.m, w.flux, w.ra0, w.dec0, J)
    return tr, T.eq17_terms(tr.export(), J, uvw)


def test_all_coefficients_kept_is_the_oracles_eq17():
    # the numpy evaluation against the C oracle's recursion: two codes, one sum
    w = synth.small()
    uvw = w.uvw[::40]
    tr, (base, G, S) = _terms(w, 10, uvw)
    v = T.thresholded_vis(base, G, S, len(G))
    assert np.max(np.abs(v - tr.vis_eq17(uvw))) <= 1e-12 * np.abs(w.flux).sum()


def test_single_component_closed_forms():
    # one component: all coefficients give its own plane wave at the pixel
    # centre (Eq. 16); none give the level-1 term alone, Phi eta_J / 4^(J-1)
    w = synth.small()
    one = synth.Workload("one", w.uvw, w.l[:1], w.m[:1], np.array([2.5]), 9)
    uvw = w.uvw[::50]
    tr, (base, G, S) = _terms(one, 9, uvw)
    s = tr.export()["leaf_dir"][0]
    wave = 2.5 * np.exp(2j * np.pi * (uvw @ s))
    assert np.allclose(T.thresholded_vis(base, G, S, len(G)), wave, rtol=0, atol=1e-12)
    assert np.allclose(T.thresholded_vis(base, G, S, 0), wave / 4.0 ** 8, rtol=0, atol=1e-14)


def test_keep_largest_order_and_ties():
    G = np.array([0.5, -2.0, 0.5, 1.0, -0.5])
    assert T.keep_largest(G, 2).tolist() == [1, 3]
    assert T.keep_largest(G, 3).tolist() == [0, 1, 3]       # ties: the lower index first


def test_thresholding_does_not_compress_a_clean_component_sky():
    # The measured reading behind leaving thresholding out of the GPU path:
    # on the medium sky (5 000 components, J = 12) keeping half of the
    # coefficients leaves errors above 1e-3 of sum |C|, and even 99 % leave
    # more than the mixed forms' 1e-6 bar; each component needs its own chain
    # of fine-level coefficients. (The leaf plane waves, 88 % of the work,
    # would be needed for any K anyway: every eta comes from them.)
    w = synth.medium(n_t=2)
    uvw = w.uvw[::len(w.uvw) // 150][:150]
    tr, (base, G, S) = _terms(w, 12, uvw)
    ref = tr.vis_eq17(uvw)
    Sg = np.abs(w.flux).sum()
    err = {f: np.max(np.abs(T.thresholded_vis(base, G, S, int(round(f * len(G)))) - ref)) / Sg
           for f in (0.01, 0.5, 0.99)}
    assert err[0.01] > 0.1
    assert err[0.5] > 1e-3
    assert err[0.99] > 1e-6
    assert math.isfinite(err[0.99])


def test_planted_mistakes_fail_the_oracle_equality(monkeypatch):
    # each plausible mistake planted in the numpy evaluation (a sign flipped
    # in a butterfly row, the area of the wrong level, a dropped area factor)
    # breaks the equality with the C oracle's Eq. 17 (the first pin above)
    w = synth.small()
    uvw = w.uvw[::40]
    tr = O.Tree(w.l, w.m, w.flux, w.ra0, w.dec0, 10)
    ref = tr.vis_eq17(uvw)
    Sg = np.abs(w.flux).sum()
    area = T.area
    H_flip = T._H.copy()
    H_flip[1] = -H_flip[1]
    plants = {"butterfly row sign": ("_H", H_flip),
              "area of level j + 1": ("area", lambda j: area(j + 1)),
              "no area factor at level 1": ("area", lambda j: 1.0 if j == 1 else area(j))}
    for kind, (attr, value) in plants.items():
        with monkeypatch.context() as mp:
            mp.setattr(T, attr, value)
            base, G, S = T.eq17_terms(tr.export(), 10, uvw)
        v = T.thresholded_vis(base, G, S, len(G))
        assert np.max(np.abs(v - ref)) > 1e-6 * Sg, kind


# ---------------------------------------------------------------- reading T2

def _t2(w, J, j0, uvw, d_leaf=2, reading="pixel"):
    tr = O.Tree(w.l, w.m, w.flux, w.ra0, w.dec0, J)
    return tr, T.full_response_terms(tr.export(), J, j0, uvw, w.ra0, w.dec0, d_leaf=d_leaf, reading=reading)


def test_t2_every_coefficient_kept_is_the_level_J_image():
    # with the responses on one common finest level, a pixel's response is
    # the mean of its children's: all coefficients kept give the level-J
    # image with each pixel's flux spread over it (the truncated tree at J,
    # each pixel's own response)
    w = synth.small()
    J, j0, dl = 10, 6, 2
    uvw = w.uvw[::200]
    tr, (base, G, S) = _t2(w, J, j0, uvw, dl)
    ref = tr.vis_truncated(J, uvw, kind="pixel", depth=dl)
    assert np.max(np.abs(T.thresholded_vis(base, G, S, len(G)) - ref)) <= 1e-12 * np.abs(w.flux).sum()


def test_t2_no_coefficient_kept_is_the_tree_truncated_at_j0():
    w = synth.small()
    J, j0, dl = 10, 7, 2
    uvw = w.uvw[::200]
    tr, (base, G, S) = _t2(w, J, j0, uvw, dl)
    ref = tr.vis_truncated(j0, uvw, kind="pixel", depth=J + dl - j0)
    assert np.max(np.abs(T.thresholded_vis(base, G, S, 0) - ref)) <= 1e-12 * np.abs(w.flux).sum()


def test_t2_every_reading_keeps_the_total_flux_at_zero_baseline():
    w = synth.small()
    z = np.zeros((2, 3))
    for reading in ("pixel", "level", "snapped"):
        _, (base, G, S) = _t2(w, 9, 6, z, 2, reading)
        for K in (0, len(G) // 3, len(G)):
            assert np.max(np.abs(T.thresholded_vis(base, G, S, K) - w.flux.sum())) <= 1e-12 * w.flux.sum()


def test_t2_threshold_by_value_is_the_largest_by_count():
    w = synth.small()
    _, (base, G, S) = _t2(w, 9, 6, w.uvw[::300], 2, "level")
    tau = float(np.median(np.abs(G)))
    K = int(np.sum(np.abs(G) >= tau))
    assert np.array_equal(T.keep_at_least(G, tau), T.keep_largest(G, K)) or \
        len(set(np.abs(G[T.keep_at_least(G, tau)]))) < K          # ties at tau are the only way they differ
    assert np.max(np.abs(T.thresholded_vis_tau(base, G, S, tau) - T.thresholded_vis(base, G, S, K))) < 1e-12


def test_t2_planted_butterfly_sign_breaks_the_level_J_identity(monkeypatch):
    w = synth.small()
    J, j0, dl = 10, 6, 2
    uvw = w.uvw[::200]
    tr = O.Tree(w.l, w.m, w.flux, w.ra0, w.dec0, J)
    ref = tr.vis_truncated(J, uvw, kind="pixel", depth=dl)
    H_flip = T._H.copy()
    H_flip[2] = -H_flip[2]
    monkeypatch.setattr(T, "_H", H_flip)
    base, G, S = T.full_response_terms(tr.export(), J, j0, uvw, w.ra0, w.dec0, d_leaf=dl)
    assert np.max(np.abs(T.thresholded_vis(base, G, S, len(G)) - ref)) > 1e-6 * np.abs(w.flux).sum()


def test_t2_compresses_the_large_sky_against_the_true_visibilities():
    # The measured reading behind the GPU path for thresholding: with
    # full-pixel responses a few dozen coarse pixels predict the large sky
    # (50 000 components in 20 blobs) closer to its true visibilities
    # (Eq. 12 at the true positions) than the centre-snapped level-J sum
    # over all 1 663 leaves; adding the largest coefficients converges to
    # the level-J image.
    w = synth.learned(n_t=2)
    J, j0, dl = 12, 9, 2
    uvw = w.uvw[::len(w.uvw) // 100][:100]
    tr, (base, G, S) = _t2(w, J, j0, uvw, dl)
    v_true = O.dft(w.l, w.m, w.flux, uvw, threads=4)
    Sg = np.abs(w.flux).sum()
    rms = lambda v: float(np.sqrt(np.mean(np.abs(v - v_true) ** 2)) / Sg)
    e_leaves = rms(tr.vis_eq16(uvw))
    assert rms(T.thresholded_vis(base, G, S, 0)) < e_leaves
    full = T.thresholded_vis(base, G, S, len(G))
    d = [float(np.max(np.abs(T.thresholded_vis(base, G, S, int(f * len(G))) - full)) / Sg) for f in (0.1, 0.5)]
    assert d[1] < d[0] < 0.1
