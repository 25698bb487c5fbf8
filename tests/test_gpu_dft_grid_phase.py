"""The direct sum (Eq. 12) in the mixed forms runs in two passes, as the
regrouped wavelet sum does: the grid pass forms each term's phase with its
three head products rounded onto a common grid per visibility (exact float32
sums, valid while every head of the tile's visibilities, bounded by the
components' largest |l|, |m|, |n - 1| reduced when they are packed, stays
below 2^14 turns), and the exact pass takes the tiles that do not fit, with
error-free sums. These GPU tests hold both passes, and tiles of either kind
side by side, to the mixed forms' bar (1e-6 of sum |C|) against the
oracle's Eq. 12, through dft_predict_vis and dft_predict_vis_noalloc.
"""
import ctypes as C

import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")
wt = pytest.importorskip("paper_1909_03956_gb300")

pytestmark = pytest.mark.gpu

TOLMIX = 1e-6
MIXED = [wt.WT_MIXED, wt.WT_MIXED_FAST]
GRID_LIMIT_TURNS = 2.0 ** 14


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def phase_bound(l, m, uvw):
    """sum_c |B_c| max_components |s_c| per visibility: the bound the grid pass tests."""
    r2 = l * l + m * m
    s = np.abs(np.stack([l, m, -r2 / (1 + np.sqrt(1 - r2))], axis=1)).max(axis=0)
    return np.abs(uvw) @ s


def sky(n, half_width_rad, rng):
    return (rng.uniform(-half_width_rad, half_width_rad, n), rng.uniform(-half_width_rad, half_width_rad, n),
            10.0 ** rng.uniform(-3, 0, n))


def long_baselines(n, lo, hi, rng):
    return rng.uniform(lo, hi, (n, 3)) * rng.choice([-1.0, 1.0], (n, 3))


def rel_err(l, m, f, uvw, mode, sign=1):
    v = wt.dft_predict_vis(dev(l), dev(m), dev(f), dev(uvw), mode=mode, sign=sign).cpu().numpy()
    return float(np.max(np.abs(v - O.dft(l, m, f, uvw, sign))) / np.abs(f).sum())


def noalloc_err(l, m, f, uvw, mode):
    L = wt.load()
    out = torch.empty(len(uvw), dtype=torch.complex64, device="cuda")
    dl, dm, df, du = dev(l), dev(m), dev(f), dev(uvw)
    p = lambda t: C.c_void_p(t.data_ptr())
    rc = L.dft_predict_vis_noalloc(p(dl), p(dm), p(df), len(l), p(du), len(uvw), p(out), int(mode), 1, None,
                                   C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == wt.WT_OK, L.wt_last_error().decode()
    return float(np.max(np.abs(out.cpu().numpy() - O.dft(l, m, f, uvw))) / np.abs(f).sum())


@pytest.mark.parametrize("mode", MIXED)
def test_every_tile_in_the_exact_pass(mode):
    # a 20 deg field and baselines to 7e4 wavelengths: heads of ~10^4 turns
    rng = np.random.default_rng(81)
    l, m, f = sky(300, 0.35, rng)
    uvw = long_baselines(3000, 5e4, 7e4, rng)
    assert phase_bound(l, m, uvw).min() > 1.1 * GRID_LIMIT_TURNS
    assert rel_err(l, m, f, uvw, mode) <= TOLMIX
    assert rel_err(l, m, f, uvw[:1001], mode, sign=-1) <= TOLMIX


@pytest.mark.parametrize("mode", MIXED)
def test_grid_and_exact_tiles_side_by_side(mode):
    # short baselines except one visibility in every 700: the tiles of 512
    # that hold one take the exact pass, the others stay on the grid
    rng = np.random.default_rng(82)
    l, m, f = sky(200, 0.2, rng)
    uvw = rng.uniform(-2e3, 2e3, (9000, 3))
    uvw[::700] = long_baselines(len(uvw[::700]), 5e4, 8e4, rng)
    pb = phase_bound(l, m, uvw)
    assert pb[::700].min() > 1.1 * GRID_LIMIT_TURNS and np.delete(pb, np.s_[::700]).max() < GRID_LIMIT_TURNS / 2
    assert rel_err(l, m, f, uvw, mode) <= TOLMIX
    assert noalloc_err(l, m, f, uvw, mode) <= TOLMIX


@pytest.mark.parametrize("mode", MIXED)
def test_grid_pass_just_below_its_limit(mode):
    # heads up to just under 2^14 turns: the coarsest grid the pass uses
    rng = np.random.default_rng(83)
    l, m, f = sky(150, 0.1, rng)
    uvw = rng.uniform(-1, 1, (4000, 3))
    uvw *= (0.97 * GRID_LIMIT_TURNS / phase_bound(l, m, uvw))[:, None]
    assert phase_bound(l, m, uvw).max() < GRID_LIMIT_TURNS
    assert rel_err(l, m, f, uvw, mode) <= TOLMIX


def test_single_component_worst_case_both_passes():
    # one component, no averaging over terms: the per-term bound must hold
    # on the grid (heads of ~10^3 turns) and in the exact pass (~10^5)
    rng = np.random.default_rng(84)
    l, m, f = np.array([0.0123]), np.array([-0.0071]), np.array([1.0])
    for scale in (3e4, 3e6):
        uvw = rng.uniform(-scale, scale, (20000, 3))
        for mode in MIXED:
            assert rel_err(l, m, f, uvw, mode) <= TOLMIX


def test_zero_tiny_baselines_and_no_components():
    # B = 0 gives V = sum of the fluxes; tiny phases sit on the finest grid;
    # with no component every visibility is 0 (the bounds stay 0)
    rng = np.random.default_rng(85)
    l, m, f = sky(50, 0.05, rng)
    uvw = np.zeros((1200, 3))
    uvw[600:] = rng.uniform(-1e-3, 1e-3, (600, 3))
    for mode in MIXED:
        assert rel_err(l, m, f, uvw, mode) <= TOLMIX
        e = np.zeros(0)
        v = wt.dft_predict_vis(dev(e), dev(e), dev(e), dev(uvw), mode=mode).cpu().numpy()
        assert np.array_equal(v, np.zeros(len(uvw), dtype=v.dtype))
