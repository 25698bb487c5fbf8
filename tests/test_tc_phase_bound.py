"""The error bound of the tensor-core phase (WT_MIXED_TC), checked on the CPU.

The tensor-core form writes each phase t = u l + v m + w (n - 1) (turns) as
products of exact 11-bit slices: the terms' coordinates in four slices below
a per-call exponent q_c, the baselines in five (balanced base-2048 digits of
x 2^(q_c + 44)), summed into three accumulators of scales 2^-11, 2^-22 and
2^-33 (slice pairs i + j = 1, 2 and 3-4; i + j = 0 is an integer and drops
out). This test carries out that arithmetic in exact integers and float32
exactly as stated, and checks against the float64 phase modulo 1:

* every slice fits float16 exactly (|digit| <= 1024, |a_0| <= 16) and the
  first two accumulators stay below 2^24, so the tensor cores sum them
  exactly whatever their order;
* the recombined phase is within 2^-29 turns of the true one modulo 1 on
  the synthetic workloads' components and baselines, and on a single
  component at the edge of the range (phases near 2^14 turns per
  coordinate).

It pins the numerical design, not the kernel; the kernel's results are held
to the oracle by the GPU tests.
"""
import math

import numpy as np

import synth


def _exponent(bound):
    """q with |s| < 1024 2^q for |s| <= bound (bound raised by 2^-20)."""
    if not bound > 0:
        return -200
    return math.frexp(bound * (1.0 + 2.0 ** -20))[1] - 1 - 9


def _term_slices(s, q):
    """Four slices of s 2^-q: rint of the remainder, then times 2^11."""
    y = np.ldexp(s, -q)
    out = []
    for _ in range(4):
        r = np.rint(y)
        out.append(r)
        y = (y - r) * 2048.0
    return np.array(out)


def _baseline_slices(x, q):
    """Five balanced base-2048 digits of rint(x 2^(q + 44)), most significant first."""
    Y = np.rint(np.ldexp(x, q + 44)).astype(np.int64)
    digits = []
    for _ in range(4):
        d = ((Y + 1024) & 2047) - 1024
        digits.append(d)
        Y = (Y - d) >> 11
    digits.append(Y)
    return np.array(digits[::-1], dtype=np.float64)


def _tc_phase(l, m, uvw):
    """The recombined phase modulo 1 (float32 steps as the kernel takes them)
    and the float64 phase modulo 1, for every (visibility, component)."""
    r2 = l * l + m * m
    s = np.stack([l, m, -r2 / (1.0 + np.sqrt(1.0 - r2))])                 # [3, C]
    bounds = np.abs(s.astype(np.float32)).max(axis=1)
    q = [_exponent(float(b)) for b in bounds]
    b = np.stack([_term_slices(s[c], q[c]) for c in range(3)])              # [3, 4, C]
    a = np.stack([_baseline_slices(uvw[:, c], q[c]) for c in range(3)])     # [3, 5, V]
    assert np.abs(b).max() <= 1024 and np.abs(a[:, 1:]).max() <= 1024 and np.abs(a[:, 0]).max() <= 16

    def pair(i, j):
        return np.einsum("cv,cm->vm", a[:, i], b[:, j])                     # exact: integers < 2^53

    acc1 = pair(0, 1) + pair(1, 0)
    acc2 = pair(0, 2) + pair(1, 1) + pair(2, 0)
    acc3 = pair(0, 3) + pair(1, 2) + pair(2, 1) + pair(3, 0) + 2.0 ** -11 * (
        pair(1, 3) + pair(2, 2) + pair(3, 1) + pair(4, 0))
    assert np.abs(acc1).max() < 2 ** 24 and np.abs(acc2).max() < 2 ** 24
    f32 = np.float32
    A1, A2, A3 = acc1.astype(f32), acc2.astype(f32), acc3.astype(f32)
    M = f32(12582912.0)
    y = (A1 * f32(2.0 ** -11) + M).astype(f32)
    f1 = (A1.astype(np.float64) * 2.0 ** -11 - (y - M).astype(np.float64)).astype(f32)
    h = (A2.astype(np.float64) * 2.0 ** -22 + f1.astype(np.float64)).astype(f32)
    # the kernel's h is exact: check it
    assert np.array_equal(h.astype(np.float64), A2.astype(np.float64) * 2.0 ** -22 + f1.astype(np.float64))
    hp = (h - ((h + M) - M)).astype(f32)
    t = hp.astype(np.float64) + A3.astype(np.float64) * 2.0 ** -33
    ph = uvw @ s
    return t, ph - np.rint(ph)


def _max_err(l, m, uvw):
    t, ref = _tc_phase(l, m, uvw)
    d = t - ref
    return float(np.max(np.abs(d - np.rint(d))))


def test_phase_bound_on_the_synthetic_workloads():
    for w in (synth.small(), synth.medium(), synth.large()):
        idx = np.linspace(0, w.n_vis - 1, 1500).astype(int)
        cidx = np.linspace(0, len(w.l) - 1, min(len(w.l), 1500)).astype(int)
        assert _max_err(w.l[cidx], w.m[cidx], w.uvw[idx]) <= 2.0 ** -29
        assert _max_err(w.l[cidx], w.m[cidx], -w.uvw[idx]) <= 2.0 ** -29   # the other sign


def test_phase_bound_at_the_edge_of_the_range():
    # one component; baselines scaled so that |x| 2^q approaches 16 (phases
    # near 2^14 turns per coordinate, the tile condition's limit)
    l, m = np.array([0.0123]), np.array([-0.0071])
    rng = np.random.default_rng(5)
    r2 = l * l + m * m
    s = np.abs(np.stack([l, m, -r2 / (1.0 + np.sqrt(1.0 - r2))])[:, 0])
    q = [_exponent(float(np.float32(v))) for v in s]
    lim = np.array([16.0 * 2.0 ** -qc for qc in q]) * 0.999
    uvw = rng.uniform(-1.0, 1.0, (4000, 3)) * lim
    assert _max_err(l, m, uvw) <= 2.0 ** -29
