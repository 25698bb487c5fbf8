"""The imaging half of the major cycle on the GPU against the imaging oracle:
dirty image and beam (float32 FFT against the float64 definition), Hogbom
clean bit for bit against the float32 oracle (same argmax decisions, same
roundings), and whole major cycles with the direct sum and with the tree."""
import numpy as np
import pytest

import oracle as O
import synth
from oracle import imaging as I

torch = pytest.importorskip("torch")
wt = pytest.importorskip("paper_1909_03956_gb300")

pytestmark = pytest.mark.gpu


def dev(a, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    return t.to(dtype) if dtype is not None else t


def _array(n):
    w = synth.small()
    uvw = w.uvw * np.array([1.0, 1.0, 0.0])
    dl = 0.45 / np.max(np.abs(uvw[:, :2]))
    return uvw, dl


@pytest.mark.parametrize("n", [64, 256])
def test_dirty_image_and_beam_match_the_oracle(n):
    uvw, dl = _array(n)
    rng = np.random.default_rng(n)
    vis = (rng.standard_normal(len(uvw)) + 1j * rng.standard_normal(len(uvw))).astype(np.complex64)
    img = wt.wt_dirty_image(dev(uvw), dev(vis), n, dl).cpu().numpy()
    ref = I.dirty_image(uvw, vis.astype(np.complex128), n, dl)
    assert np.max(np.abs(img - ref)) <= 2e-5 * np.max(np.abs(ref))
    beam = wt.wt_dirty_image(dev(uvw), None, n, dl).cpu().numpy()
    rb = I.dirty_beam(uvw, n, dl)
    assert np.max(np.abs(beam - rb)) <= 2e-5
    assert beam[n // 2, n // 2] == pytest.approx(1.0, abs=1e-5)


def test_dirty_image_edge_cases():
    uvw, dl = _array(32)
    # no visibilities: a zero image; odd n: refused
    img = wt.wt_dirty_image(dev(uvw[:0].copy()), dev(np.zeros(0, np.complex64)), 32, dl).cpu().numpy()
    assert not img.any()
    with pytest.raises(wt.WtError):
        wt.wt_dirty_image(dev(uvw), None, 31, dl)
    # every baseline outside the grid (pixel far too large): nothing gridded
    img = wt.wt_dirty_image(dev(uvw), None, 32, 1.0).cpu().numpy()
    assert not img.any()


SCHEDULES = ["persistent", "launches"]


@pytest.fixture(params=SCHEDULES)
def schedule(request, monkeypatch):
    # the whole clean in one cooperative launch (the default where the rows
    # fit in shared memory) or one launch per iteration
    if request.param == "launches":
        monkeypatch.setenv("WT_HOGBOM", "launches")
    else:
        monkeypatch.delenv("WT_HOGBOM", raising=False)
    return request.param


@pytest.mark.parametrize("n,iters,gain,thr", [(64, 300, 0.1, 0.0), (128, 500, 0.2, 0.05), (64, 50, 1.0, 0.3),
                                              (66, 120, 0.3, 0.0), (1024, 40, 0.1, 0.0)])
def test_hogbom_bit_exact_against_the_float32_oracle(n, iters, gain, thr, schedule):
    # n = 66 takes the one-pixel-per-step path (n not a multiple of 4); at
    # n = 1024 every CTA holds several rows
    uvw, dl = _array(n)
    rng = np.random.default_rng(7)
    k = 6
    l = rng.integers(-n // 4, n // 4, k) * dl
    m = rng.integers(-n // 4, n // 4, k) * dl
    f = rng.uniform(0.2, 1.0, k)
    vis = O.dft(l, m, f, uvw)
    dirty = I.dirty_image(uvw, vis, n, dl).astype(np.float32)
    psf = I.dirty_beam(uvw, n, dl).astype(np.float32)
    res_o, pix_o, flux_o = I.hogbom(dirty, psf, gain, iters, thr)
    img = dev(dirty)
    pix, flux = wt.wt_hogbom(img, dev(psf), gain, iters, thr)
    assert np.array_equal(pix.cpu().numpy(), pix_o.astype(np.int32))
    assert np.array_equal(flux.cpu().numpy(), flux_o)
    assert np.array_equal(img.cpu().numpy(), res_o)


def test_hogbom_maximum_value_rule_and_zero_iterations(schedule):
    n = 16
    psf = np.zeros((n, n), np.float32)
    psf[n // 2, n // 2] = 1.0
    img = np.zeros((n, n), np.float32)
    img[3, 4], img[9, 9], img[12, 1] = 1.0, -5.0, 0.5
    t = dev(img)
    pix, flux = wt.wt_hogbom(t, dev(psf), 1.0, 10, 0.6)
    assert pix.cpu().tolist() == [3 * n + 4] and flux.cpu().tolist() == [1.0]
    out = t.cpu().numpy()
    assert out[9, 9] == -5.0 and out[12, 1] == 0.5 and out[3, 4] == 0.0
    pix, flux = wt.wt_hogbom(dev(img), dev(psf), 0.5, 0)
    assert pix.numel() == 0


def test_hogbom_image_without_a_comparable_value(schedule):
    # an all-NaN image has no maximum: no component, the image untouched
    n = 16
    psf = np.zeros((n, n), np.float32)
    psf[n // 2, n // 2] = 1.0
    t = dev(np.full((n, n), np.nan, np.float32))
    wt.wt_device_status()
    pix, flux = wt.wt_hogbom(t, dev(psf), 0.5, 5)
    wt.wt_device_status()
    assert pix.numel() == 0
    assert np.isnan(t.cpu().numpy()).all()


def _two_sources(n):
    uvw, dl = _array(n)
    src = [(n // 2 + 6, n // 2 - 4, 1.0), (n // 2 - 9, n // 2 + 5, 0.6)]
    l = np.array([(x - n // 2) * dl for x, y, _ in src])
    m = np.array([(y - n // 2) * dl for x, y, _ in src])
    f = np.array([s[2] for s in src])
    return uvw, dl, src, l, m, f


@pytest.mark.parametrize("predictor", [wt.WT_PREDICT_DIRECT, wt.WT_PREDICT_TREE])
def test_clean_recovers_point_sources(predictor, schedule):
    n = 64
    uvw, dl, src, l, m, f = _two_sources(n)
    obs = O.dft(l, m, f, uvw).astype(np.complex64)
    # the tree places each component at the centre of its level-J sphere
    # pixel: two levels finer than the Table 1 rule keeps that offset below
    # dl/8; flux that lands next to a source is counted with it
    J = wt.wt_recommended_J(dl) + 2
    pix, flux, resid, img = wt.wt_clean(dev(uvw), dev(obs), n, dl, synth.RA0, synth.DEC0, J, predictor=predictor,
                                        mode=wt.WT_MIXED, gain=0.2, minor_iter=60, n_major=3)
    pix, flux = pix.cpu().numpy(), flux.cpu().numpy()
    tot = {}
    for p, fl in zip(pix, flux):
        tot[int(p)] = tot.get(int(p), 0.0) + float(fl)
    want = {y * n + x: fl for x, y, fl in src}
    assert set(sorted(tot, key=lambda p: -tot[p])[:2]) == set(want)
    for x, y, fl in src:
        near = sum(v for p, v in tot.items() if abs(p % n - x) <= 1 and abs(p // n - y) <= 1)
        assert near == pytest.approx(fl, rel=0.05)
    r = resid.cpu().numpy()
    assert np.sqrt(np.mean(np.abs(r) ** 2)) < 0.05 * np.sqrt(np.mean(np.abs(obs) ** 2))
    # the returned image is the dirty image of the returned residuals
    ref_img = I.dirty_image(uvw, r.astype(np.complex128), n, dl)
    assert np.max(np.abs(img.cpu().numpy() - ref_img)) <= 2e-5 * max(1e-3, np.max(np.abs(ref_img)))


def test_clean_matches_the_oracle_cycle_by_cycle_with_the_direct_sum():
    # one major cycle: the first dirty image and its components agree with the
    # oracle (the dirty images differ by float32 rounding only, far below the
    # gaps between the peaks of this sky)
    n = 64
    uvw, dl, src, l, m, f = _two_sources(n)
    obs = O.dft(l, m, f, uvw)
    pix, flux, resid, img = wt.wt_clean(dev(uvw), dev(obs.astype(np.complex64)), n, dl, synth.RA0, synth.DEC0, 12,
                                        predictor=wt.WT_PREDICT_DIRECT, mode=wt.WT_MIXED, gain=0.2, minor_iter=20,
                                        n_major=1)
    pix_o, flux_o, resid_o, img_o = I.major_cycles(uvw, obs, n, dl, 0.2, 20, 0.0, 1,
                                                   lambda a, b, c, d: O.dft(a, b, c, d))
    assert np.array_equal(pix.cpu().numpy(), pix_o.astype(np.int32))
    assert np.allclose(flux.cpu().numpy(), flux_o, rtol=1e-4)
    assert np.max(np.abs(resid.cpu().numpy() - resid_o)) <= 1e-4 * np.max(np.abs(obs))


def test_hogbom_grid_barrier_times_out_and_reports():
    # the persistent clean's grid barrier, made never to open, gives up after
    # its poll limit and reports WT_ERR_TIMEOUT; the context stays usable
    wt.wt_device_status()
    wt.wt_selftest_grid_barrier(500)
    with pytest.raises(wt.WtError) as e:
        wt.wt_device_status()
    assert e.value.status == wt.WT_ERR_TIMEOUT
    wt.wt_device_status()
    n = 16
    psf = np.zeros((n, n), np.float32)
    psf[n // 2, n // 2] = 1.0
    img = np.zeros((n, n), np.float32)
    img[5, 7] = 2.0
    pix, flux = wt.wt_hogbom(dev(img), dev(psf), 0.5, 3)
    assert pix.cpu().tolist() == [5 * n + 7] * 3
    assert flux.cpu().tolist() == [1.0, 0.5, 0.25]
