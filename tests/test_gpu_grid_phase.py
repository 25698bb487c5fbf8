"""Eq. 17 (regrouped and explicit) and Eq. 16 in the mixed forms run in two passes: the grid pass
forms each leaf phase with its three head products rounded onto a common
grid (exact float32 sums, valid while every head of the tile's visibilities
stays below 2^14 turns), and the exact pass takes the tiles that do not fit,
with error-free sums. These GPU tests hold both passes, and tiles of either
kind side by side, to the mixed forms' bar against the oracle's Eq. 17 and
Eq. 16.
"""
import numpy as np
import pytest

import oracle as O
import synth

torch = pytest.importorskip("torch")
wt = pytest.importorskip("paper_1909_03956_gb300")

pytestmark = pytest.mark.gpu

TOLMIX = 1e-6
MIXED = [wt.WT_MIXED, wt.WT_MIXED_FAST]
GRID_LIMIT_TURNS = 2.0 ** 14   # bound below 2^(kGridMaxK - 1) turns (less a 2^-10 margin): the grid pass


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def phase_bound(w, J, uvw):
    """sum_c |B_c| max_leaves |s_c| per visibility: the bound the kernel tests."""
    d = np.abs(O.Tree(w.l, w.m, w.flux, w.ra0, w.dec0, J).export()["leaf_dir"]).max(axis=0)
    return np.abs(uvw) @ d


def rel_err(w, J, uvw, mode, sign=1, which=wt.WT_SUM_EQ17_REGROUPED):
    t = wt.wt_build_tree(dev(w.l), dev(w.m), dev(w.flux), w.ra0, w.dec0, J)
    v = wt.wt_predict_vis(t, dev(uvw), mode=mode, which=which, sign=sign).cpu().numpy()
    ot = O.Tree(w.l, w.m, w.flux, w.ra0, w.dec0, J)
    ref = ot.vis_eq16(uvw, sign) if which == wt.WT_SUM_EQ16 else ot.vis_eq17(uvw, sign)
    t.close()
    return float(np.max(np.abs(v - ref)) / np.abs(w.flux).sum())


SUMS = [wt.WT_SUM_EQ17_REGROUPED, wt.WT_SUM_EQ17, wt.WT_SUM_EQ16]


def long_baselines(n, lo, hi, rng):
    """Baselines with |u|, |v|, |w| in [lo, hi] and random signs."""
    return rng.uniform(lo, hi, (n, 3)) * rng.choice([-1.0, 1.0], (n, 3))


def wide_sky(n, half_width_rad, rng):
    l = rng.uniform(-half_width_rad, half_width_rad, n)
    m = rng.uniform(-half_width_rad, half_width_rad, n)
    return l, m, 10.0 ** rng.uniform(-3, 0, n)


@pytest.mark.parametrize("which", SUMS)
@pytest.mark.parametrize("mode", MIXED)
def test_every_tile_in_the_exact_pass(mode, which):
    # 20 deg field and baselines to 6e4 wavelengths: heads of ~10^4 turns
    rng = np.random.default_rng(71)
    l, m, f = wide_sky(300, 0.35, rng)
    uvw = long_baselines(3000, 5e4, 7e4, rng)
    w = synth.Workload("wide", uvw, l, m, f, 10)
    assert phase_bound(w, 10, uvw).min() > 1.1 * GRID_LIMIT_TURNS
    assert rel_err(w, 10, uvw, mode, which=which) <= TOLMIX
    assert rel_err(w, 10, uvw[:1001], mode, sign=-1, which=which) <= TOLMIX


@pytest.mark.parametrize("which", SUMS)
@pytest.mark.parametrize("mode", MIXED)
def test_grid_and_exact_tiles_side_by_side(mode, which):
    # short baselines everywhere except one visibility in every 700: tiles
    # of 256 that hold one go to the exact pass, the others stay on the grid
    rng = np.random.default_rng(72)
    l, m, f = wide_sky(200, 0.2, rng)
    uvw = rng.uniform(-2e3, 2e3, (9000, 3))
    uvw[::700] = long_baselines(len(uvw[::700]), 5e4, 8e4, rng)
    w = synth.Workload("mixed_tiles", uvw, l, m, f, 11)
    pb = phase_bound(w, 11, uvw)
    assert pb[::700].min() > 1.1 * GRID_LIMIT_TURNS and np.delete(pb, np.s_[::700]).max() < GRID_LIMIT_TURNS / 2
    assert rel_err(w, 11, uvw, mode, which=which) <= TOLMIX


@pytest.mark.parametrize("which", SUMS)
@pytest.mark.parametrize("mode", MIXED)
def test_grid_pass_just_below_its_limit(mode, which):
    # heads up to just under 2^14 turns: the coarsest grid the pass uses
    rng = np.random.default_rng(73)
    l, m, f = wide_sky(150, 0.1, rng)
    uvw = rng.uniform(-1, 1, (4000, 3))
    w = synth.Workload("edge", uvw, l, m, f, 12)
    pb = phase_bound(w, 12, uvw)
    uvw *= (0.97 * GRID_LIMIT_TURNS / pb)[:, None]
    assert phase_bound(w, 12, uvw).max() < GRID_LIMIT_TURNS
    assert rel_err(w, 12, uvw, mode, which=which) <= TOLMIX


def test_single_component_worst_case_both_passes():
    # one component, no averaging over terms: the per-term bound of the fast
    # form must hold on the grid (heads of ~10^3 turns) and in the exact
    # pass (~10^5 turns)
    rng = np.random.default_rng(74)
    for scale in (3e4, 3e6):
        uvw = rng.uniform(-scale, scale, (20000, 3))
        w = synth.Workload("one", uvw, np.array([0.0123]), np.array([-0.0071]), np.array([1.0]), 14)
        for mode in MIXED:
            for which in SUMS:
                assert rel_err(w, 14, uvw, mode, which=which) <= TOLMIX


def test_zero_and_tiny_baselines():
    # B = 0 gives V = sum of the fluxes; tiny phases sit on the finest grid
    w = synth.small()
    uvw = np.zeros((600, 3))
    uvw[300:] = np.random.default_rng(75).uniform(-1e-3, 1e-3, (300, 3))
    for mode in MIXED:
        assert rel_err(w, 9, uvw, mode) <= TOLMIX


@pytest.mark.parametrize("mode", MIXED)
def test_batched_channels_in_both_passes(mode):
    # one channel's tree spans a 20 deg field (its tiles take the exact pass
    # at the high frequencies), the other's a 1 deg field (the grid pass)
    rng = np.random.default_rng(76)
    uvw_m = rng.uniform(-9e3, 9e3, (5000, 3))
    freqs = [1.0e9, 1.9e9]
    skies = [wide_sky(120, 0.35, rng), wide_sky(120, 0.01, rng)]
    trees = [wt.wt_build_tree(dev(l), dev(m), dev(f), synth.RA0, synth.DEC0, 11) for l, m, f in skies]
    out = wt.wt_predict_vis_batched(trees, freqs, dev(uvw_m), mode=mode)
    got = out.cpu().numpy()
    for c, ((l, m, f), fr) in enumerate(zip(skies, freqs)):
        uvw = uvw_m * (fr / synth.C_LIGHT)
        ref = O.Tree(l, m, f, synth.RA0, synth.DEC0, 11).vis_eq17(uvw)
        assert np.max(np.abs(got[c] - ref)) / np.abs(f).sum() <= TOLMIX
    w0 = synth.Workload("w0", uvw_m * (freqs[1] / synth.C_LIGHT), *skies[0], 11)
    assert phase_bound(w0, 11, w0.uvw).max() > 1.1 * GRID_LIMIT_TURNS
    for t in trees:
        t.close()
