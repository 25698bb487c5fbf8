"""Pins for the oracle's truncated-tree prediction and per-pixel responses
(reading R12, the use of the learned response: an addition to
arXiv:1909.03956).

The truncated tree keeps the level-jt nodes with the flux of their pixels,
F_k = A_jt lambda_jt,k, and predicts sum_k F_k exp(i 2 pi B.(c_k - P)) R_k(B)
with R_k = 1 (centre-snapped), the phase-centre pixel's response R_jt (what
the network learns) or each pixel's own response R_jt,k. The pins tie each
reading to the direct sum of Eq. 12, itself pinned by closed forms.
"""
import numpy as np
import pytest

import oracle as O
import synth

RA0, DEC0 = synth.RA0, synth.DEC0


def _subpixel_sky(j, k, D, flux=1.0):
    """Components at the centres of all 4^D level-(j + D) descendants of
    pixel k at level j, each of the same flux."""
    sub = np.array([O.pixel_dir_uvw(j + D, (k << (2 * D)) + i, RA0, DEC0) for i in range(4 ** D)])
    return sub[:, 0].copy(), sub[:, 1].copy(), np.full(4 ** D, flux)


def _phase_centre_pixel(j):
    k, _ = O.map_components([0.0], [0.0], RA0, DEC0, j)
    return int(k[0])


def test_truncated_at_level_J_is_eq16():
    w = synth.small()
    t = O.Tree(w.l, w.m, w.flux, w.ra0, w.dec0, 9)
    uvw = w.uvw[::40]
    S = np.abs(w.flux).sum()
    assert np.max(np.abs(t.vis_truncated(9, uvw) - t.vis_eq16(uvw))) <= 1e-13 * S


def test_pixel_response_of_the_phase_centre_pixel_is_the_level_response():
    rng = np.random.default_rng(11)
    uvw = rng.uniform(-5000, 5000, (40, 3))
    j = 10
    assert np.array_equal(O.pixel_response_of(j, _phase_centre_pixel(j), 3, RA0, DEC0, uvw),
                          O.pixel_response(j, 3, RA0, DEC0, uvw))


@pytest.mark.parametrize("offset_pixels", [5, -37])
def test_pixel_response_of_any_pixel_is_the_direct_sum_over_its_descendants(offset_pixels):
    # unit fluxes at every descendant centre, summed by Eq. 12 and
    # demodulated by the plane wave at the pixel's centre, divided by 4^D
    j, D = 9, 3
    k = _phase_centre_pixel(j) + offset_pixels
    l, m, f = _subpixel_sky(j, k, D)
    c = O.pixel_dir_uvw(j, k, RA0, DEC0)
    rng = np.random.default_rng(12)
    uvw = rng.uniform(-3000, 3000, (60, 3))
    ref = O.dft(l, m, f, uvw) / 4 ** D / np.exp(1j * 2 * np.pi * (uvw @ c))
    assert np.max(np.abs(O.pixel_response_of(j, k, D, RA0, DEC0, uvw) - ref)) < 1e-11


@pytest.mark.parametrize("kind", ["level", "pixel"])
def test_fully_populated_phase_centre_pixel_is_eq12(kind):
    # A level-jt pixel whose every level-J sub-pixel centre holds the same
    # flux: truncating at jt with responses of depth J - jt loses nothing,
    # so both response readings equal the direct sum over the components.
    jt, D = 8, 3
    J = jt + D
    l, m, f = _subpixel_sky(jt, _phase_centre_pixel(jt), D, flux=0.25)
    t = O.Tree(l, m, f, RA0, DEC0, J)
    assert t.per_level[jt - 1] == 1
    rng = np.random.default_rng(13)
    uvw = rng.uniform(-8000, 8000, (80, 3))
    v = t.vis_truncated(jt, uvw, kind=kind, depth=D)
    ref = O.dft(l, m, f, uvw)
    assert np.max(np.abs(v - ref)) <= 1e-11 * f.sum()
    assert np.max(np.abs(t.vis_truncated(jt, uvw, kind=kind, depth=D, sign=-1) - np.conj(ref))) <= 1e-11 * f.sum()


def test_fully_populated_pixel_away_from_the_centre():
    # the pixel's own response reproduces Eq. 12 there; the phase-centre
    # pixel's response (the learned form's single response per level) does
    # not quite: the pixels differ in shape across the field
    jt, D = 8, 3
    k = _phase_centre_pixel(jt) + 9
    l, m, f = _subpixel_sky(jt, k, D)
    t = O.Tree(l, m, f, RA0, DEC0, jt + D)
    rng = np.random.default_rng(14)
    uvw = rng.uniform(-8000, 8000, (80, 3))
    ref = O.dft(l, m, f, uvw)
    assert np.max(np.abs(t.vis_truncated(jt, uvw, kind="pixel", depth=D) - ref)) <= 1e-11 * f.sum()
    assert np.max(np.abs(t.vis_truncated(jt, uvw, kind="level", depth=D) - ref)) > 1e-6 * f.sum()


def test_every_reading_gives_the_total_flux_at_zero_baseline():
    w = synth.medium(n_t=2)
    t = O.Tree(w.l, w.m, w.flux, w.ra0, w.dec0, 12)
    z = np.zeros((3, 3))
    for kind in ("snapped", "level", "pixel"):
        for jt in (6, 9, 12):
            assert np.max(np.abs(t.vis_truncated(jt, z, kind=kind, depth=2) - w.flux.sum())) <= 1e-12 * w.flux.sum()
