"""Pins for the oracle's coefficient tree and wavelet predictors
(Sec. 3.2-3.5, Eqs. 9, 10, 11, 16, 17 of arXiv:1909.03956)."""
import math

import numpy as np
import pytest

import oracle as O
import synth

EPS = np.finfo(np.float64).eps


def _tree(w, J):
    return O.Tree(w.l, w.m, w.flux, w.ra0, w.dec0, J)


@pytest.mark.parametrize("J", [1, 2, 5, 8, 12, 16, 20])
def test_eq17_equals_eq16(J):
    # The multiresolution sum equals the level-J sum: the Hadamard rows of
    # Eq. 10 plus (1,1,1,1) are orthogonal, so the per-node identity
    # A_j lambda eta + sum_m gamma sigma = A_{j+1} sum_c lambda_c eta_c holds.
    w = synth.small()
    t = _tree(w, J)
    uvw = w.uvw[::97]
    v17, v16 = t.vis_eq17(uvw), t.vis_eq16(uvw)
    S = np.abs(w.flux).sum()
    assert np.max(np.abs(v17 - v16)) <= 8 * t.n_nodes * EPS * S


def test_eq17_equals_eq16_mixed_sign_fluxes():
    rng = np.random.default_rng(11)
    w = synth.small()
    f = w.flux * np.where(rng.random(len(w.flux)) < 0.4, -1.0, 1.0)
    t = O.Tree(w.l, w.m, f, w.ra0, w.dec0, 10)
    uvw = w.uvw[::211]
    S = np.abs(f).sum()
    assert np.max(np.abs(t.vis_eq17(uvw) - t.vis_eq16(uvw))) <= 8 * t.n_nodes * EPS * S


@pytest.mark.parametrize("J", [6, 10, 14])
def test_eq16_is_direct_sum_at_pixel_centres(J):
    # Eq. 16 = Eq. 12 with each component moved to its pixel centre and the
    # fluxes of a pixel merged (Sec. 3.3, "distinct" components).
    w = synth.small()
    t = _tree(w, J)
    e = t.export()
    uvw = w.uvw[::53]
    ld = e["leaf_dir"]
    vd = O.dft(ld[:, 0], ld[:, 1], e["leaf_flux"], uvw)
    S = np.abs(w.flux).sum()
    assert np.max(np.abs(t.vis_eq16(uvw) - vd)) < 1e-13 * S


def test_error_against_true_positions_is_bounded_and_shrinks():
    # |V_tree - V_true| <= 2 pi sum_i |C_i| |B| d_i, d_i the distance between a
    # component and its pixel centre; the error halves per level (Sec. 3.3).
    w = synth.small()
    uvw = w.uvw[::31]
    vt = O.dft(w.l, w.m, w.flux, uvw)
    errs = []
    for J in (12, 14, 16, 18):
        t = _tree(w, J)
        e = t.export()
        k, _ = O.map_components(w.l, w.m, w.ra0, w.dec0, J)
        keys = e["key"][-t.n_leaves:]
        idx = np.searchsorted(keys, k)
        ld = e["leaf_dir"][idx]
        n_true = np.sqrt(1 - w.l ** 2 - w.m ** 2)
        dvec = np.stack([w.l - ld[:, 0], w.m - ld[:, 1], (n_true - 1) - ld[:, 2]], axis=1)
        d = np.linalg.norm(dvec, axis=1)
        bound = 2 * np.pi * np.linalg.norm(uvw, axis=1) * np.sum(np.abs(w.flux) * d)
        err = np.abs(t.vis_eq17(uvw) - vt)
        assert np.all(err <= bound * (1 + 1e-9) + 1e-12)
        errs.append(err.max())
    for a, b in zip(errs, errs[1:]):
        assert b < 0.75 * a


def test_bfs_structure_invariants():
    w = synth.medium(n_t=2)
    J = 12
    t = _tree(w, J)
    e = t.export()
    offs = e["level_offsets"]
    key, mask, first = e["key"], e["child_mask"], e["first_child"]
    assert offs[-1] == t.n_nodes and t.per_level[-1] == t.n_leaves
    assert t.per_level[0] <= 12
    for j in range(1, J + 1):
        kk = key[offs[j - 1]:offs[j]]
        assert np.all(np.diff(kk) > 0)
        assert np.all(kk < 12 * 4 ** (j - 1))
    for i in range(offs[J - 1]):
        kids = [c for c in range(4) if mask[i] >> c & 1]
        assert kids, "internal node without children"
        for r, c in enumerate(kids):
            ch = first[i] + r
            assert key[ch] == 4 * key[i] + c
    assert np.all(first[offs[J - 1]:] == -1) and np.all(mask[offs[J - 1]:] == 0)
    # the leaves are exactly the distinct level-J pixels of the components
    k, _ = O.map_components(w.l, w.m, w.ra0, w.dec0, J)
    assert np.array_equal(np.unique(k), key[offs[J - 1]:])
    # Phi_k: the summed fluxes, each pixel's components added in input order
    for leaf, kk in enumerate(key[offs[J - 1]:offs[J - 1] + 50]):
        s = 0.0
        for f in w.flux[k == kk]:
            s += f
        assert e["leaf_flux"][leaf] == s


@pytest.mark.parametrize("J", [3, 5, 6])
def test_brute_force_dense_grid(J):
    # Dense transform over every pixel of every level (zeros included):
    # the tree's lambda and gamma equal the dense ones bit for bit at the
    # tree's nodes; nonzero counts per level equal the tree's node counts
    # (positive fluxes); dense Eq. 17 equals the tree's Eq. 17.
    w = synth.small()
    t = _tree(w, J)
    e = t.export()
    lams, gams = O.dense_coeffs(w.l, w.m, w.flux, w.ra0, w.dec0, J)
    offs = e["level_offsets"]
    for j in range(1, J + 1):
        keys = e["key"][offs[j - 1]:offs[j]]
        assert np.count_nonzero(lams[j - 1]) == t.per_level[j - 1]
        assert np.array_equal(lams[j - 1][keys], e["lam"][offs[j - 1]:offs[j]])
        if j < J:
            assert np.array_equal(gams[j - 1][keys], e["gamma"][offs[j - 1]:offs[j]])
    uvw = w.uvw[::997]
    vd = O.dense_vis_eq17(w.l, w.m, w.flux, w.ra0, w.dec0, J, uvw)
    S = np.abs(w.flux).sum()
    assert np.max(np.abs(vd - t.vis_eq17(uvw))) < 1e-13 * S


def test_nonzero_count_brute_force_J9():
    # The number of nonzero coefficients per level from a dense scan at J = 9
    # (786 432 level-9 pixels) equals the tree's nodes per level.
    w = synth.medium(n_t=2)
    J = 9
    t = _tree(w, J)
    lams, _ = O.dense_coeffs(w.l, w.m, w.flux, w.ra0, w.dec0, J)
    assert [np.count_nonzero(x) for x in lams] == list(t.per_level)


def test_synthesis_reconstructs_leaf_coefficients():
    # Eq. 11 (the inverse of Eqs. 9/10) rebuilds lambda_J from lambda_1 and
    # the gammas, top-down, to within a few rounding errors per level (the
    # sqrt(A_j) factors of Eq. 10 and of the inverse do not cancel exactly).
    rng = np.random.default_rng(12)
    w = synth.small()
    f = rng.integers(1, 64, len(w.l)).astype(np.float64) / 64.0
    for J in (4, 8, 12):
        t = O.Tree(w.l, w.m, f, w.ra0, w.dec0, J)
        e = t.export()
        lamJ = e["lam"][-t.n_leaves:]
        rec = t.synthesis()
        rel = np.abs(rec - lamJ) / np.abs(lamJ)
        assert rel.max() < 8 * J * EPS
    t = O.Tree(w.l, w.m, w.flux, w.ra0, w.dec0, 12)
    e = t.export()
    lamJ = e["lam"][-t.n_leaves:]
    assert np.max(np.abs(t.synthesis() - lamJ)) / np.abs(lamJ).max() < 64 * EPS


def test_point_source_on_pixel_centre_at_phase_centre():
    # Phase centre placed on a level-J pixel centre: a component at l = m = 0
    # lies in that pixel at its centre, so V = C for every baseline (Eq. 16).
    J = 14
    k0 = 5 * 4 ** 13 + 123456
    z, st, phi = O.pix2ang_nest(J - 1, k0)
    ra0, dec0 = phi, math.asin(z)
    t = O.Tree([0.0], [0.0], [0.7], ra0, dec0, J)
    e = t.export()
    assert e["key"][-1] == k0
    rng = np.random.default_rng(13)
    uvw = rng.uniform(-2e4, 2e4, (200, 3))
    v = t.vis_eq17(uvw)
    assert np.max(np.abs(v - 0.7)) < 1e-9


def test_single_component_generic_position_closed_form():
    # One component anywhere: V = C exp(i 2 pi B.(s_k - P)) with s_k the
    # centre of its level-J pixel (Eq. 16 with a single term).
    J = 10
    t = O.Tree([0.004], [-0.002], [1.5], 1.0, 0.5, J)
    k, _ = O.map_components([0.004], [-0.002], 1.0, 0.5, J)
    d = O.pixel_dir_uvw(J, int(k[0]), 1.0, 0.5)
    rng = np.random.default_rng(14)
    uvw = rng.uniform(-5e3, 5e3, (100, 3))
    ref = 1.5 * np.exp(1j * 2 * np.pi * (uvw @ d))
    assert np.max(np.abs(t.vis_eq17(uvw) - ref)) < 1e-10


def test_node_with_zero_flux_sum_is_kept():
    # Reading: a pixel is a node when a component maps there, even if the
    # fluxes cancel.
    t = O.Tree([0.001, 0.001], [0.002, 0.002], [0.5, -0.5], 1.0, 0.5, 8)
    assert t.n_leaves == 1 and t.n_nodes == 8
    e = t.export()
    assert e["lam"][-1] == 0.0


def test_empty_component_list():
    t = O.Tree([], [], [], 1.0, 0.5, 8)
    assert t.n_nodes == 0
    v = t.vis_eq17(np.ones((3, 3)))
    assert np.all(v == 0)
