"""Pins for the oracle's learned-response pieces (an addition to
arXiv:1909.03956): the exact per-level pixel response and the FP64 network
forward/backward pass."""
import math

import numpy as np
import pytest

import oracle as O
import synth

RA0, DEC0 = synth.RA0, synth.DEC0


def test_pixel_response_at_zero_baseline_is_one():
    r = O.pixel_response(10, 3, RA0, DEC0, np.zeros((3, 3)))
    assert np.all(r == 1.0)


def test_pixel_response_is_the_direct_sum_over_subpixel_centres():
    # A unit flux at every level-(j+D) sub-pixel centre, summed by Eq. 12
    # (itself pinned by closed forms), divided by N and by the plane wave at
    # the level-j centre, is R_j(B).
    j, D = 11, 3
    k, _ = O.map_components([0.0], [0.0], RA0, DEC0, j)
    c = O.pixel_dir_uvw(j, int(k[0]), RA0, DEC0)
    sub = np.array([O.pixel_dir_uvw(j + D, (int(k[0]) << (2 * D)) + i, RA0, DEC0) for i in range(4 ** D)])
    rng = np.random.default_rng(1)
    uvw = rng.uniform(-4000, 4000, (50, 3))
    v = O.dft(sub[:, 0], sub[:, 1], np.ones(4 ** D), uvw)
    ref = v / 4 ** D / np.exp(1j * 2 * np.pi * (uvw @ c))
    r = O.pixel_response(j, D, RA0, DEC0, uvw)
    assert np.max(np.abs(r - ref)) < 1e-11


def test_pixel_response_symmetries_and_bound():
    rng = np.random.default_rng(2)
    uvw = rng.uniform(-20000, 20000, (200, 3))
    r = O.pixel_response(12, 3, RA0, DEC0, uvw)
    assert np.max(np.abs(r)) <= 1.0 + 1e-12
    assert np.max(np.abs(O.pixel_response(12, 3, RA0, DEC0, -uvw) - np.conj(r))) < 1e-13
    assert np.max(np.abs(O.pixel_response(12, 3, RA0, DEC0, uvw, sign=-1) - np.conj(r))) < 1e-15


def test_pixel_response_converges_with_depth_and_decays():
    # Finer sub-pixel grids approach the pixel average: differences shrink
    # by about 4 per extra level (midpoint rule, second order).
    j = 12
    dt = O.level_pixel_size(j)
    rng = np.random.default_rng(3)
    uvw = rng.uniform(-1.5 / dt, 1.5 / dt, (100, 3))
    r = [O.pixel_response(j, D, RA0, DEC0, uvw) for D in (2, 3, 4, 5)]
    d = [np.max(np.abs(r[i + 1] - r[i])) for i in range(3)]
    assert d[1] < 0.4 * d[0] and d[2] < 0.4 * d[1]
    # baselines much longer than 1 / pixel size see a strongly damped response
    far = np.array([[20 / dt, 17 / dt, 0.0], [-25 / dt, 9 / dt, 0.0]])
    assert np.max(np.abs(O.pixel_response(j, 5, RA0, DEC0, far))) < 0.05


def _random_params(rng, scale=0.5):
    return rng.standard_normal(O.mlp_n_params()) * scale


def test_mlp_forward_closed_form():
    # One path through the network: W1[0,0] = a, W2[0,0] = b, W3[0,0] = c,
    # b3 = (d0, d1), all else zero: y0 = c silu(b silu(a x0)) + d0, y1 = d1.
    silu = lambda z: z / (1 + math.exp(-z))
    j = 9
    p = np.zeros(O.mlp_n_params())
    W1, b1, W2, b2, W3, b3 = O.mlp_split(p)
    W1[0, 0], W2[0, 0], W3[0, 0] = 0.7, -1.3, 2.1
    b3[:] = [0.25, -0.5]
    uvw = np.array([[1000.0, -200.0, 30.0], [-4000.0, 10.0, 0.0]])
    y = O.mlp_forward(p, j, uvw)
    for q in range(2):
        x0 = uvw[q, 0] * O.level_pixel_size(j)
        assert abs(y[q, 0] - (2.1 * silu(-1.3 * silu(0.7 * x0)) + 0.25)) < 1e-14
        assert y[q, 1] == -0.5
    # an off-diagonal path pins the orientation of every matrix: input v into
    # hidden unit 3, into second-layer unit 5, into output 1
    p = np.zeros(O.mlp_n_params())
    W1, b1, W2, b2, W3, b3 = O.mlp_split(p)
    W1[3, 1], W2[5, 3], W3[1, 5] = 0.9, 1.1, -0.8
    y = O.mlp_forward(p, j, uvw)
    for q in range(2):
        x1 = uvw[q, 1] * O.level_pixel_size(j)
        assert y[q, 0] == 0.0
        assert abs(y[q, 1] - (-0.8 * silu(1.1 * silu(0.9 * x1)))) < 1e-14


def test_mlp_gradient_matches_finite_differences():
    rng = np.random.default_rng(4)
    p = _random_params(rng)
    j = 12
    dt = O.level_pixel_size(j)
    uvw = rng.uniform(-2 / dt, 2 / dt, (16, 3))
    tgt = rng.standard_normal((16, 2))
    loss, g = O.mlp_loss_grad(p, j, uvw, tgt)
    idx = rng.choice(len(p), 60, replace=False)
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (O.mlp_loss_grad(pp, j, uvw, tgt)[0] - O.mlp_loss_grad(pm, j, uvw, tgt)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])
    y = O.mlp_forward(p, j, uvw)
    assert abs(loss - np.mean(np.sum((y - tgt) ** 2, axis=1))) < 1e-12
