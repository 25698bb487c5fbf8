"""Pins of the imaging oracle (gridding, FFT, Hogbom, major cycles) against
what the definitions fix: single-cell gridding, the FFT against the double
sum it stands for, closed forms for point sources and for cleaning a pure
beam, the threshold, and recovery of point sources through full major
cycles with the direct sum (Eq. 12) as the prediction."""
import numpy as np
import pytest

import oracle as O
from oracle import imaging as I


def _on_grid_uvw(n, dl, count, seed):
    # baselines exactly on cell centres (and w = 0)
    rng = np.random.default_rng(seed)
    du = 1.0 / (n * dl)
    k = rng.integers(-n // 2 + 1, n // 2, (count, 2))
    return np.column_stack([k[:, 0] * du, k[:, 1] * du, np.zeros(count)])


def test_single_visibility_lands_in_its_cell_and_mirror():
    n, dl = 16, 1e-3
    du = 1.0 / (n * dl)
    uvw = np.array([[3 * du, -2 * du, 5.0]])
    G, W = I.grid_nn(uvw, np.array([2.0 + 1.0j]), n, dl)
    assert W == 2
    assert G[n // 2 - 2, n // 2 + 3] == 2.0 + 1.0j          # [iv][iu]
    assert G[n // 2 + 2, n // 2 - 3] == 2.0 - 1.0j          # the mirrored cell holds the conjugate
    assert np.count_nonzero(G) == 2
    # a cell outside the grid leaves the visibility out
    G, W = I.grid_nn(np.array([[(n // 2) * du, 0.0, 0.0]]), np.array([1.0 + 0j]), n, dl)
    assert W == 0 and not G.any()


def test_fft_image_equals_the_double_sum():
    n, dl = 16, 2e-3
    rng = np.random.default_rng(3)
    uvw = rng.uniform(-0.45, 0.45, (40, 3)) / dl
    vis = rng.standard_normal(40) + 1j * rng.standard_normal(40)
    G, W = I.grid_nn(uvw, vis, n, dl)
    a = I.image_from_grid(G, W)
    b = I.image_from_grid_direct(G, W, dl)
    assert np.max(np.abs(a - b)) < 1e-12 * np.max(np.abs(b))


def test_point_source_at_phase_centre_and_beam_peak():
    n, dl = 32, 1e-3
    uvw = _on_grid_uvw(n, dl, 200, 4)
    C = 1.7
    img = I.dirty_image(uvw, np.full(len(uvw), C, dtype=np.complex128), n, dl)
    assert img[n // 2, n // 2] == pytest.approx(C, rel=1e-13)
    assert np.argmax(img) == (n // 2) * n + n // 2
    psf = I.dirty_beam(uvw, n, dl)
    assert psf[n // 2, n // 2] == pytest.approx(1.0, rel=1e-13)
    assert np.max(psf) == pytest.approx(1.0, rel=1e-13)
    # the beam of real-valued unit visibilities with their conjugates is symmetric
    assert np.allclose(psf[1:, 1:], psf[1:, 1:][::-1, ::-1], atol=1e-12)


def test_off_centre_point_source_is_the_shifted_beam():
    # uv on cell centres: the image of a source at pixel offset (dx, dy) is
    # C times the beam rolled by (dy, dx) (the shift theorem on the grid)
    n, dl = 32, 1e-3
    uvw = _on_grid_uvw(n, dl, 300, 5)
    dx, dy, C = 5, -3, 0.8
    l0, m0 = dx * dl, dy * dl
    vis = O.dft(np.array([l0]), np.array([m0]), np.array([C]), uvw * np.array([1, 1, 0]))
    img = I.dirty_image(uvw, vis, n, dl)
    psf = I.dirty_beam(uvw, n, dl)
    # the direct sum includes n - 1 for w = 0: no effect; the 2-D image has the
    # source exactly at (n/2 + dy, n/2 + dx)
    assert np.max(np.abs(img - C * np.roll(psf, (dy, dx), axis=(0, 1)))) < 1e-12
    assert np.argmax(img) == (n // 2 + dy) * n + (n // 2 + dx)


def test_hogbom_on_a_pure_beam_follows_the_gain():
    n, dl = 32, 1e-3
    psf = I.dirty_beam(_on_grid_uvw(n, dl, 300, 6), n, dl).astype(np.float32)
    A, g, dx, dy = np.float32(2.5), 0.1, 4, 7
    img = A * np.roll(psf, (dy, dx), axis=(0, 1))
    # keep the image free of wrapped beam: zero where the roll wrapped around
    img[:dy, :] = 0
    img[:, :dx] = 0
    p0 = (n // 2 + dy) * n + (n // 2 + dx)
    res, pix, flux = I.hogbom(img, psf, g, 10, 0.0)
    assert np.all(pix == p0)
    # component k has flux g A (1 - g)^k, the residual peak A (1 - g)^10
    k = np.arange(10)
    assert np.allclose(flux, g * A * (1 - g) ** k, rtol=2e-6)
    assert res.flat[p0] == pytest.approx(A * (1 - g) ** 10, rel=2e-6)
    assert flux.sum() == pytest.approx(A * (1 - (1 - g) ** 10), rel=2e-6)


def test_hogbom_threshold_and_maximum_value():
    n = 16
    psf = np.zeros((n, n), dtype=np.float32)
    psf[n // 2, n // 2] = 1.0                         # a delta beam: one component per pixel
    img = np.zeros((n, n), dtype=np.float32)
    img[3, 4], img[9, 9], img[12, 1] = 1.0, -5.0, 0.5
    res, pix, flux = I.hogbom(img, psf, 1.0, 10, 0.6)
    # the largest value, not the largest magnitude: the negative pixel stays
    assert pix.tolist() == [3 * n + 4]
    assert flux.tolist() == [1.0]
    assert res[9, 9] == -5.0 and res[12, 1] == 0.5 and res[3, 4] == 0.0


def test_major_cycles_recover_point_sources_with_the_direct_sum():
    # two sources on pixel positions, baselines of a synthetic array (not on
    # cell centres), three major cycles of the direct sum
    import synth
    w = synth.small()
    n = 64
    # pixel size such that every baseline falls inside the grid (|u| < 0.45 / dl)
    dl = 0.45 / np.max(np.abs(w.uvw[:, :2]))
    src_px = [(n // 2 + 6, n // 2 - 4, 1.0), (n // 2 - 9, n // 2 + 5, 0.6)]
    l = np.array([(x - n // 2) * dl for x, y, f in src_px])
    m = np.array([(y - n // 2) * dl for x, y, f in src_px])
    f = np.array([s[2] for s in src_px])
    uvw = w.uvw * np.array([1.0, 1.0, 0.0])
    obs = O.dft(l, m, f, uvw)

    def predict(lc, mc, fc, b):
        return O.dft(lc, mc, fc, b)

    pix, flux, resid, img = I.major_cycles(uvw, obs, n, dl, 0.2, 60, 0.0, 3, predict)
    want = {y * n + x: fl for x, y, fl in src_px}
    tot = {}
    for p, fl in zip(pix, flux):
        tot[p] = tot.get(p, 0.0) + float(fl)
    main = sorted(tot, key=lambda p: -tot[p])[:2]
    assert set(main) == set(want)
    for p in want:
        assert tot[p] == pytest.approx(want[p], rel=0.05)
    assert np.sqrt(np.mean(np.abs(resid) ** 2)) < 0.05 * np.sqrt(np.mean(np.abs(obs) ** 2))


# ---------------------------------------------------------------- reading I5
# The w-corrected dirty image by direct summation: pinned by its closed
# forms and, at w = 0 on cell centres, by the FFT image of I1-I3.

def _source_vis(uvw, l0, m0, flux=1.0):
    nm1 = -(l0 * l0 + m0 * m0) / (1.0 + np.sqrt(1.0 - l0 * l0 - m0 * m0))
    return flux * np.exp(2j * np.pi * (uvw @ np.array([l0, m0, nm1])))


def test_exact_image_of_a_source_is_its_flux_at_its_pixel_for_any_w():
    # a wide field and large w: the exact image peaks at the source with
    # exactly its flux; dropping the w term (the plain 2-D image) does not
    n, dl = 256, 2e-3
    rng = np.random.default_rng(61)
    uvw = rng.uniform(-60, 60, (3000, 3)) * np.array([1.0, 1.0, 8.0])
    ix0, iy0 = n // 2 + 90, n // 2 - 70
    l0, m0 = (ix0 - n // 2) * dl, (iy0 - n // 2) * dl
    v = _source_vis(uvw, l0, m0, 2.5)
    assert abs(I.dirty_image_exact(uvw, v, n, dl, ix0, iy0)[0] - 2.5) < 1e-12
    # the neighbourhood is below the peak
    around = I.dirty_image_exact(uvw, v, n, dl, [ix0 + 1, ix0 - 1, ix0], [iy0, iy0, iy0 + 1])
    assert np.all(around < 2.5)
    # with w set to zero in the image (but not in the data) the peak is lost
    u0 = uvw.copy()
    u0[:, 2] = 0.0
    assert I.dirty_image_exact(u0, v, n, dl, ix0, iy0)[0] < 2.0
    # at the phase centre a source of flux C gives C for any w
    assert abs(I.dirty_image_exact(uvw, np.full(len(uvw), 0.7 + 0j), n, dl, n // 2, n // 2)[0] - 0.7) < 1e-12


def test_exact_image_at_w_zero_on_cell_centres_is_the_fft_image():
    n, dl = 32, 5e-3
    uvw = _on_grid_uvw(n, dl, 400, seed=62)
    rng = np.random.default_rng(63)
    vis = rng.normal(size=400) + 1j * rng.normal(size=400)
    ref = I.dirty_image(uvw, vis, n, dl)
    iy, ix = np.mgrid[0:n, 0:n]
    got = I.dirty_image_exact(uvw, vis, n, dl, ix.ravel(), iy.ravel()).reshape(n, n)
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))
