"""Randomised properties of the oracle (hypothesis; CPU only): for random
component lists, baselines, phase centres and levels, what the mathematics
fixes must hold -- Eq. 17 equals Eq. 16 on the same tree, Eq. 16 at pixel
centres equals the direct sum Eq. 12 at those centres, the direct sum is
Hermitian and linear in the fluxes, and merging duplicates changes nothing."""
import numpy as np
import pytest

import oracle as O

hyp = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

EPS = np.finfo(np.float64).eps


def _inputs(seed, n_comp, n_vis, field):
    rng = np.random.default_rng(seed)
    l = rng.uniform(-field, field, n_comp)
    m = rng.uniform(-field, field, n_comp)
    f = rng.uniform(-1.0, 1.0, n_comp)
    uvw = rng.uniform(-3000.0, 3000.0, (n_vis, 3)) * np.array([1.0, 1.0, 0.2])
    return l, m, f, uvw


common = settings(max_examples=25, deadline=None)


@common
@given(seed=st.integers(0, 2 ** 31 - 1), n_comp=st.integers(1, 40), J=st.integers(1, 16),
       ra0=st.floats(0.0, 6.28), dec0=st.floats(-1.4, 1.4))
def test_eq17_equals_eq16_on_random_trees(seed, n_comp, J, ra0, dec0):
    l, m, f, uvw = _inputs(seed, n_comp, 12, 0.02)
    t = O.Tree(l, m, f, ra0, dec0, J)
    S = np.abs(f).sum()
    assert np.max(np.abs(t.vis_eq17(uvw) - t.vis_eq16(uvw))) <= 8 * t.n_nodes * EPS * S * 16


@common
@given(seed=st.integers(0, 2 ** 31 - 1), n_comp=st.integers(1, 30), J=st.integers(4, 20))
def test_eq16_is_the_direct_sum_at_pixel_centres(seed, n_comp, J):
    # Eq. 16 sums each leaf's merged flux times the plane wave at its pixel
    # centre: the direct sum over the leaves at their centres
    l, m, f, uvw = _inputs(seed, n_comp, 10, 0.02)
    ra0, dec0 = 1.0, 0.5
    t = O.Tree(l, m, f, ra0, dec0, J)
    e = t.export()
    d = e["leaf_dir"]                       # (s_u, s_v, s_w - 1) of each leaf centre
    V = (np.exp(2j * np.pi * (uvw @ d.T)) * e["leaf_flux"]).sum(axis=1)
    S = np.abs(f).sum()
    assert np.max(np.abs(t.vis_eq16(uvw) - V)) <= 1e-12 * max(S, 1e-300) + 1e-14


@common
@given(seed=st.integers(0, 2 ** 31 - 1), n_comp=st.integers(1, 30), a=st.floats(-3.0, 3.0))
def test_direct_sum_hermitian_and_linear(seed, n_comp, a):
    l, m, f, uvw = _inputs(seed, n_comp, 16, 0.05)
    V = O.dft(l, m, f, uvw)
    S = np.abs(f).sum()
    assert np.max(np.abs(O.dft(l, m, f, -uvw) - np.conj(V))) <= 1e-13 * S
    assert np.max(np.abs(O.dft(l, m, f, uvw, sign=-1) - np.conj(V))) <= 1e-13 * S
    assert np.max(np.abs(O.dft(l, m, a * f, uvw) - a * V)) <= 1e-13 * S * max(1.0, abs(a))


@common
@given(seed=st.integers(0, 2 ** 31 - 1), n_comp=st.integers(1, 20), J=st.integers(2, 14))
def test_duplicated_components_merge(seed, n_comp, J):
    # listing every component twice at half its flux gives the same leaves
    # (same keys, summed flux) and the same visibilities
    l, m, f, uvw = _inputs(seed, n_comp, 8, 0.02)
    t1 = O.Tree(l, m, f, 1.0, 0.5, J)
    t2 = O.Tree(np.concatenate([l, l]), np.concatenate([m, m]), np.concatenate([f, f]) / 2, 1.0, 0.5, J)
    e1, e2 = t1.export(), t2.export()
    assert np.array_equal(e1["key"], e2["key"])
    assert np.allclose(e1["leaf_flux"], e2["leaf_flux"], rtol=0, atol=4 * EPS * np.abs(f).sum())
    S = np.abs(f).sum()
    assert np.max(np.abs(t1.vis_eq17(uvw) - t2.vis_eq17(uvw))) <= 1e-12 * S
