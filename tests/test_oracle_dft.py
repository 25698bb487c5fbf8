"""Pins for the oracle's direct sum (Eq. 12 of arXiv:1909.03956).

Each test checks the oracle against something other than itself: closed
forms, symmetries, a library FFT, or a higher-precision evaluation.
"""
import math

import numpy as np
import pytest

import oracle as O
import synth


def test_point_source_at_phase_centre_is_constant():
    # Eq. 12 with C at l = m = 0: B.(C - P) = 0 for every baseline, V = C.
    rng = np.random.default_rng(1)
    uvw = rng.uniform(-3e4, 3e4, (500, 3))
    v = O.dft([0.0], [0.0], [0.37], uvw)
    assert np.all(v.real == 0.37) and np.all(v.imag == 0.0)


def test_symmetric_pair_closed_form():
    # Two equal fluxes at (+l0, 0) and (-l0, 0):
    # V = 2 C cos(2 pi u l0) exp(i 2 pi w (n0 - 1)).
    rng = np.random.default_rng(2)
    uvw = rng.uniform(-2e4, 2e4, (300, 3))
    l0, C = 0.013, 0.8
    v = O.dft([l0, -l0], [0.0, 0.0], [C, C], uvw)
    n0 = math.sqrt(1 - l0 * l0)
    ref = 2 * C * np.cos(2 * np.pi * uvw[:, 0] * l0) * np.exp(1j * 2 * np.pi * uvw[:, 2] * (n0 - 1))
    assert np.max(np.abs(v - ref)) < 1e-11 * 2 * C


def test_two_component_modulus_closed_form():
    # |C1 e^{i a} + C2 e^{i b}|^2 = C1^2 + C2^2 + 2 C1 C2 cos(a - b), with
    # a - b = 2 pi B.(C1 - C2) computed from the geometry directly.
    rng = np.random.default_rng(3)
    uvw = rng.uniform(-1e4, 1e4, (400, 3))
    (l1, m1), (l2, m2) = (0.01, -0.004), (-0.007, 0.012)
    c1, c2 = 1.3, 0.45
    v = O.dft([l1, l2], [m1, m2], [c1, c2], uvw)
    n1, n2 = math.sqrt(1 - l1 * l1 - m1 * m1), math.sqrt(1 - l2 * l2 - m2 * m2)
    d = uvw[:, 0] * (l1 - l2) + uvw[:, 1] * (m1 - m2) + uvw[:, 2] * (n1 - n2)
    ref = c1 * c1 + c2 * c2 + 2 * c1 * c2 * np.cos(2 * np.pi * d)
    assert np.max(np.abs(np.abs(v) ** 2 - ref)) < 1e-10


def test_hermitian_and_sign_conjugation():
    # Real fluxes: V(-B) = conj V(B); sign = -1 is the complex conjugate.
    w = synth.small()
    uvw = w.uvw[:300]
    v = O.dft(w.l, w.m, w.flux, uvw)
    vneg = O.dft(w.l, w.m, w.flux, -uvw)
    vconj = O.dft(w.l, w.m, w.flux, uvw, sign=-1)
    S = np.abs(w.flux).sum()
    assert np.max(np.abs(vneg - np.conj(v))) < 1e-13 * S
    assert np.max(np.abs(vconj - np.conj(v))) == 0.0


def test_w_zero_reduces_to_2d_fft():
    # Eq. 2 (w = 0): components on the grid l = p/N, m = q/N and integer
    # (u, v) give V(u, v) = sum_pq I[p, q] exp(+i 2 pi (u p + v q) / N), which
    # numpy computes as N^2 * ifft2 (for small |l|, |m| < 1 the n term vanishes
    # only through w = 0).
    N = 8
    rng = np.random.default_rng(4)
    img = rng.uniform(0, 1, (N, N))
    # direction cosines must satisfy l^2 + m^2 < 1: use p/N - 1/2 shifted grid
    ps = np.arange(N)
    L, M = np.meshgrid((ps - N // 2) / (4.0 * N), (ps - N // 2) / (4.0 * N), indexing="ij")
    # scale u by 4 so that u * l = (u' / N) (p - N/2) with integer u'
    us, vs = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    uvw = np.stack([4.0 * us.ravel(), 4.0 * vs.ravel(), np.zeros(N * N)], axis=1)
    v = O.dft(L.ravel(), M.ravel(), img.ravel(), uvw)
    shift = np.exp(-1j * 2 * np.pi * (us + vs) * (N // 2) / N)
    ref = (N * N * np.fft.ifft2(img)) * shift
    assert np.max(np.abs(v - ref.ravel())) < 1e-12 * img.sum()


def test_fp64_against_long_double():
    # The FP64 sum agrees with the long-double evaluation of the same
    # definition to ~1e-14 of the peak amplitude sum |C|.
    w = synth.small()
    uvw = w.uvw[::40]
    v = O.dft(w.l, w.m, w.flux, uvw)
    vl = O.dft(w.l, w.m, w.flux, uvw, long_double=True)
    assert np.max(np.abs(v - vl)) / np.abs(w.flux).sum() < 2e-14


def test_subtract():
    a = np.array([1 + 2j, -3 + 0.5j])
    b = np.array([0.5 - 1j, 1 + 1j])
    assert np.all(O.subtract(a, b) == a - b)


def test_rejects_bad_sign():
    with pytest.raises(ValueError):
        O.dft([0.0], [0.0], [1.0], np.zeros((1, 3)), sign=2)


def test_threaded_evaluation_is_bitwise_single_threaded():
    """The all-core CPU baseline splits the visibilities over OpenMP threads;
    each visibility is computed by the unchanged single-threaded routine, so
    the results must be identical bit for bit (Eq. 12 and Eq. 17)."""
    w = synth.small()
    uvw = w.uvw[:997]
    one = O.dft(w.l, w.m, w.flux, uvw)
    for th in (2, 3, 8):
        assert np.array_equal(O.dft(w.l, w.m, w.flux, uvw, threads=th), one)
    t = O.Tree(w.l, w.m, w.flux, w.ra0, w.dec0, 9)
    one = t.vis_eq17(uvw)
    for th in (2, 5):
        assert np.array_equal(t.vis_eq17(uvw, threads=th), one)
