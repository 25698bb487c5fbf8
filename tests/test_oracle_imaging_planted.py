"""The imaging oracle's pins catch plausible mistakes: each case below plants
one mistake in a copy of an oracle function (gridding, the transform, the
normalisation, Hogbom's maximum rule or gain, the major cycle's component
list) and checks that at least one of the pins in test_oracle_imaging.py
then fails. The unplanted oracle passes them all (that file)."""
import numpy as np
import pytest

from oracle import imaging as I

import test_oracle_imaging as P

PINS = [P.test_single_visibility_lands_in_its_cell_and_mirror, P.test_fft_image_equals_the_double_sum,
        P.test_point_source_at_phase_centre_and_beam_peak, P.test_off_centre_point_source_is_the_shifted_beam,
        P.test_hogbom_on_a_pure_beam_follows_the_gain, P.test_hogbom_threshold_and_maximum_value,
        P.test_major_cycles_recover_point_sources_with_the_direct_sum,
        P.test_exact_image_of_a_source_is_its_flux_at_its_pixel_for_any_w,
        P.test_exact_image_at_w_zero_on_cell_centres_is_the_fft_image]

_grid_nn, _image_from_grid, _hogbom, _major_cycles = I.grid_nn, I.image_from_grid, I.hogbom, I.major_cycles
_exact = I.dirty_image_exact


def _exact_variant(uvw, vis, n, dl, ix, iy, w_sign=-1.0, m_sign=1.0):
    # the direct sum with the w term's sign or the m axis changed
    uvw = np.asarray(uvw, dtype=np.float64)
    ix, iy = np.atleast_1d(ix), np.atleast_1d(iy)
    l, m = (ix - n // 2) * dl, (iy - n // 2) * dl * m_sign
    r2 = l * l + m * m
    nm1 = -r2 / (1.0 + np.sqrt(1.0 - r2))
    ph = np.outer(uvw[:, 0], l) + np.outer(uvw[:, 1], m) - w_sign * np.outer(uvw[:, 2], nm1)
    return (np.asarray(vis)[:, None] * np.exp(-2j * np.pi * ph)).real.sum(axis=0) / len(uvw)


def exact_without_w(uvw, vis, n, dl, ix, iy):
    u0 = np.array(uvw, dtype=np.float64, copy=True)
    u0[:, 2] = 0.0
    return _exact(u0, vis, n, dl, ix, iy)


def _plain_grid(uvw, vis, n, dl, conj):
    G = np.zeros((n, n), dtype=np.complex128)
    W = 0
    for (u, v, _), V in zip(np.asarray(uvw, dtype=np.float64), np.asarray(vis, dtype=np.complex128)):
        ru, rv = np.rint(u * n * dl), np.rint(v * n * dl)
        if not (-n // 2 < ru < n // 2 and -n // 2 < rv < n // 2):
            continue
        G[int(rv) + n // 2, int(ru) + n // 2] += V
        G[n // 2 - int(rv), n // 2 - int(ru)] += np.conj(V) if conj else V
        W += 2
    return G, W


def image_half_normalised(G, W):
    return _image_from_grid(G, W) * 2.0


def image_wrong_sign(G, W):
    if W == 0:
        return np.zeros(G.shape)
    F = np.fft.fftshift(np.fft.ifft2(np.fft.ifftshift(G))) * G.size
    return F.real / W


def hogbom_by_magnitude(image, psf, gain, max_iter, threshold):
    img = np.array(image, dtype=np.float32, copy=True)
    flip = img.flat[int(np.argmax(np.abs(img)))] < 0
    if flip:
        img = -img
    res, pix, flux = _hogbom(img, psf, gain, max_iter, threshold)
    return (-res if flip else res), pix, (-flux if flip else flux)


def hogbom_without_gain(image, psf, gain, max_iter, threshold):
    return _hogbom(image, psf, 1.0, max_iter, threshold)


def major_cycles_latest_only(uvw, vis_obs, n, dl, gain, minor_iter, threshold, n_major, predict):
    # the model from the latest cycle's components only, not every one so far
    psf = I.dirty_beam(uvw, n, dl)
    resid = np.asarray(vis_obs, dtype=np.complex128).copy()
    pix_all, flux_all = [], []
    for _ in range(n_major):
        dirty = I.dirty_image(uvw, resid, n, dl)
        _, pix, flux = I.hogbom(dirty, psf, gain, minor_iter, threshold)
        if len(pix) == 0:
            break
        pix_all.extend(pix.tolist())
        flux_all.extend(flux.tolist())
        l, m = I.pixel_lm(pix, n, dl)
        resid = np.asarray(vis_obs) - predict(l, m, np.asarray(flux, dtype=np.float64), uvw)
    return np.array(pix_all), np.array(flux_all, dtype=np.float32), resid, I.dirty_image(uvw, resid, n, dl)


PLANTS = {
    "mirror cell without the conjugate": ("grid_nn", lambda u, v, n, dl: _plain_grid(u, v, n, dl, conj=False)),
    "image normalised by W / 2": ("image_from_grid", image_half_normalised),
    "inverse transform (wrong sign of the exponent)": ("image_from_grid", image_wrong_sign),
    "largest magnitude instead of largest value": ("hogbom", hogbom_by_magnitude),
    "component flux without the loop gain": ("hogbom", hogbom_without_gain),
    "model from the latest cycle only": ("major_cycles", major_cycles_latest_only),
    "exact image without the w term": ("dirty_image_exact", exact_without_w),
    "exact image with the w term's sign flipped": ("dirty_image_exact",
                                                   lambda *a: _exact_variant(*a, w_sign=1.0)),
    "exact image with the m axis mirrored": ("dirty_image_exact", lambda *a: _exact_variant(*a, m_sign=-1.0)),
}


@pytest.mark.parametrize("plant", sorted(PLANTS))
def test_a_planted_mistake_fails_a_pin(plant, monkeypatch):
    name, fn = PLANTS[plant]
    monkeypatch.setattr(I, name, fn)
    failed = []
    for pin in PINS:
        try:
            pin()
        except AssertionError:
            failed.append(pin.__name__)
    assert failed, "no pin caught: " + plant
