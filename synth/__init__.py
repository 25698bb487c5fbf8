"""Seeded synthetic workloads for model-visibility prediction.

This module only draws inputs: antenna layouts, baseline coordinates and
clean-component lists. It holds none of the prediction arithmetic and is the
one module that both the CPU oracle's tests and the CUDA path's tests and
benchmark import.

Stand-ins for the paper's data. The paper measures on a simulated VLA-C
measurement set and on JVLA observations of NGC 628 (Sec. 3.3, 3.6); neither
is available, so every workload here is synthetic:

* antennas uniform in a disc of the given diameter on a flat local
  east-north-up plane (up = 0), site latitude 34.0784 deg (a VLA-like site);
* phase centre RA 12h, Dec 45 deg (the simulation of Sec. 3.3);
* hour angles evenly spaced over -1h .. +1h;
* baselines (u, v, w) from the standard east-north-up -> equatorial ->
  (hour angle, declination) rotation, one polarisation, no autocorrelations;
* components with direction cosines (l, m) uniform in a square field centred
  on the phase centre, or in Gaussian blobs of per-axis width 0.05 deg;
* fluxes log-uniform between 1 mJy and 1 Jy.

Randomness comes from numpy's PCG64 generator (``numpy.random.default_rng``),
which gives the same stream on every platform.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

C_LIGHT = 299792458.0
SITE_LAT_DEG = 34.0784
RA0 = math.pi                 # 12h
DEC0 = math.radians(45.0)


def antenna_disc(n_ant, diameter_m, rng):
    """East/north/up positions (metres) uniform in a disc."""
    r = 0.5 * diameter_m * np.sqrt(rng.random(n_ant))
    th = 2.0 * np.pi * rng.random(n_ant)
    return np.stack([r * np.cos(th), r * np.sin(th), np.zeros(n_ant)], axis=1)


def baselines_xyz(enu, lat_rad):
    """Equatorial baseline vectors (metres) of every antenna pair i < j."""
    sl, cl = math.sin(lat_rad), math.cos(lat_rad)
    e, n, u = enu[:, 0], enu[:, 1], enu[:, 2]
    X = -sl * n + cl * u
    Y = e
    Z = cl * n + sl * u
    xyz = np.stack([X, Y, Z], axis=1)
    i, j = np.triu_indices(len(enu), k=1)
    return xyz[j] - xyz[i]


def uvw_metres(bxyz, hour_angles, dec_rad):
    """(u, v, w) in metres for every (time, baseline), time-major."""
    sd, cd = math.sin(dec_rad), math.cos(dec_rad)
    out = []
    for H in hour_angles:
        sh, ch = math.sin(H), math.cos(H)
        X, Y, Z = bxyz[:, 0], bxyz[:, 1], bxyz[:, 2]
        u = sh * X + ch * Y
        v = -sd * ch * X + sd * sh * Y + cd * Z
        w = cd * ch * X - cd * sh * Y + sd * Z
        out.append(np.stack([u, v, w], axis=1))
    return np.concatenate(out, axis=0)


def log_uniform_flux(n, rng, lo=-3.0, hi=0.0):
    return 10.0 ** rng.uniform(lo, hi, n)


def components_uniform(n, field_deg, rng):
    half = math.radians(field_deg) / 2.0
    l = rng.uniform(-half, half, n)
    m = rng.uniform(-half, half, n)
    return l, m, log_uniform_flux(n, rng)


def components_blobs(n_blobs, per_blob, field_deg, rng, width_deg=0.05):
    half = math.radians(field_deg) / 2.0
    cl = rng.uniform(-half, half, n_blobs)
    cm = rng.uniform(-half, half, n_blobs)
    sig = math.radians(width_deg)
    l = (cl[:, None] + sig * rng.standard_normal((n_blobs, per_blob))).ravel()
    m = (cm[:, None] + sig * rng.standard_normal((n_blobs, per_blob))).ravel()
    return l, m, log_uniform_flux(n_blobs * per_blob, rng)


def components_spaced(n, field_deg, min_sep_deg, rng):
    """n components at least min_sep apart (rejection sampling)."""
    half = math.radians(field_deg) / 2.0
    sep = math.radians(min_sep_deg)
    pts = []
    while len(pts) < n:
        p = rng.uniform(-half, half, 2)
        if all((p[0] - q[0]) ** 2 + (p[1] - q[1]) ** 2 >= sep * sep for q in pts):
            pts.append(p)
    pts = np.array(pts)
    return pts[:, 0].copy(), pts[:, 1].copy(), log_uniform_flux(n, rng)


@dataclass
class Workload:
    name: str
    uvw: np.ndarray            # [n_vis, 3] wavelengths (first channel)
    l: np.ndarray
    m: np.ndarray
    flux: np.ndarray
    J: int
    ra0: float = RA0
    dec0: float = DEC0
    freq_hz: float = 1.4e9
    extra: dict = field(default_factory=dict)

    @property
    def n_vis(self):
        return self.uvw.shape[0]

    @property
    def n_comp(self):
        return len(self.l)


def _array_uvw(n_ant, diameter_m, n_t, freq_hz, rng):
    enu = antenna_disc(n_ant, diameter_m, rng)
    b = baselines_xyz(enu, math.radians(SITE_LAT_DEG))
    ha = np.linspace(-math.pi / 12.0, math.pi / 12.0, n_t)
    uvw_m = uvw_metres(b, ha, DEC0)
    return uvw_m, uvw_m * (freq_hz / C_LIGHT)


def small(seed=1909, J=8):
    """32 antennas in a 2 km disc, 20 hour angles, 1.4 GHz (9 920 vis);
    100 components uniform in a 1 deg field."""
    rng = np.random.default_rng(seed)
    _, uvw = _array_uvw(32, 2000.0, 20, 1.4e9, rng)
    l, m, f = components_uniform(100, 1.0, rng)
    return Workload("small_32ant_9920vis_100comp", uvw, l, m, f, J)


def medium(seed=1910, J=12, n_t=500):
    """64 antennas in a 5 km disc, 500 hour angles (1 008 000 vis);
    5 000 components in 20 Gaussian blobs inside a 2 deg field."""
    rng = np.random.default_rng(seed)
    _, uvw = _array_uvw(64, 5000.0, n_t, 1.4e9, rng)
    l, m, f = components_blobs(20, 250, 2.0, rng)
    return Workload("medium_64ant_%dvis_5000comp" % uvw.shape[0], uvw, l, m, f, J)


def medium_fixed(n_distinct, seed=1915, J=12, n_t=500):
    """Medium array with n_distinct components spaced >= 1 deg apart in a
    40 deg field, so every component stays in its own pixel at every J >= 8."""
    rng = np.random.default_rng(seed)
    _, uvw = _array_uvw(64, 5000.0, n_t, 1.4e9, rng)
    l, m, f = components_spaced(n_distinct, 40.0, 1.0, rng)
    return Workload("medium_fixed_%dcomp" % n_distinct, uvw, l, m, f, J)


def mixed(seed=1911, J=12, n_t=250, freqs=(1.3e9, 1.5e9)):
    """128 antennas in a 10 km disc, 250 times, two channels (2 032 000 vis
    each); 20 000 components in 20 blobs inside a 2 deg field."""
    rng = np.random.default_rng(seed)
    uvw_m, _ = _array_uvw(128, 10000.0, n_t, freqs[0], rng)
    l, m, f = components_blobs(20, 1000, 2.0, rng)
    w = Workload("mixed_128ant_%dvis_x%dch_20000comp" % (uvw_m.shape[0], len(freqs)),
                 uvw_m * (freqs[0] / C_LIGHT), l, m, f, J, freq_hz=freqs[0])
    w.extra["uvw_m"] = uvw_m
    w.extra["freqs"] = np.array(freqs)
    return w


def batched(seed=1912, n_ch=64, n_t=250):
    """128 antennas in a 10 km disc, 64 channels over 1.0-1.8 GHz; per channel
    an independent component list of log-uniform size 100..20 000 and a level
    J drawn from 10..13."""
    rng = np.random.default_rng(seed)
    uvw_m, _ = _array_uvw(128, 10000.0, n_t, 1.0e9, rng)
    freqs = np.linspace(1.0e9, 1.8e9, n_ch)
    chans = []
    for c in range(n_ch):
        n = int(round(10.0 ** rng.uniform(2.0, math.log10(2.0e4))))
        J = int(rng.integers(10, 14))
        n_blobs = 20
        per = max(1, n // n_blobs)
        l, m, f = components_blobs(n_blobs, per, 2.0, rng)
        chans.append(dict(l=l, m=m, flux=f, J=J, freq=freqs[c]))
    w = Workload("batched_128ant_%dvis_x%dch" % (uvw_m.shape[0], n_ch),
                 uvw_m * (freqs[0] / C_LIGHT), chans[0]["l"], chans[0]["m"], chans[0]["flux"],
                 chans[0]["J"], freq_hz=freqs[0])
    w.extra["uvw_m"] = uvw_m
    w.extra["channels"] = chans
    return w


def large(seed=1913, J=12, n_t=490, shard=(0, 1)):
    """The largest single-GPU workload: 256 antennas in a 10 km disc, 490
    times (15 993 600 vis), 1.4 GHz; 50 000 components in 20 blobs inside a
    2 deg field.

    shard = (rank, world) with world > 1 describes one batch of world * n_t
    hour angles over the same -1h .. +1h track, of which this rank takes the
    rank-th contiguous block of n_t (visibilities are time-major, so a
    contiguous range of the batch); the array and the sky are the same for
    every rank. (0, 1) is the workload above."""
    rank, world = shard
    if not (0 <= rank < world):
        raise ValueError("shard rank outside 0..world-1")
    rng = np.random.default_rng(seed)
    enu = antenna_disc(256, 10000.0, rng)
    b = baselines_xyz(enu, math.radians(SITE_LAT_DEG))
    ha = np.linspace(-math.pi / 12.0, math.pi / 12.0, n_t * world)[rank * n_t:(rank + 1) * n_t]
    uvw = uvw_metres(b, ha, DEC0) * (1.4e9 / C_LIGHT)
    l, m, f = components_blobs(20, 2500, 2.0, rng)
    tag = "" if world == 1 else "_shard%dof%d" % (rank, world)
    return Workload("large_256ant_%dvis_50000comp%s" % (uvw.shape[0], tag), uvw, l, m, f, J)


def learned(seed=1913, J=12, n_t=490):
    """The learned-response workload: the same sky and array as large()."""
    return large(seed=seed, J=J, n_t=n_t)


def paper_context(n_distinct=140, seed=1914, J=20, n_t=3600):
    """27 antennas (351 baselines) in a 3.4 km disc, 3 600 one-second dumps
    over one hour (1 263 600 vis); n_distinct spaced components."""
    rng = np.random.default_rng(seed)
    enu = antenna_disc(27, 3400.0, rng)
    b = baselines_xyz(enu, math.radians(SITE_LAT_DEG))
    ha = np.linspace(-math.pi / 24.0, math.pi / 24.0, n_t)
    uvw = uvw_metres(b, ha, DEC0) * (1.4e9 / C_LIGHT)
    l, m, f = components_spaced(n_distinct, 2.0, 0.05, rng)
    return Workload("paper_27ant_%dvis_%dcomp" % (uvw.shape[0], n_distinct), uvw, l, m, f, J)


def random_uvw(n, scale, rng):
    return rng.uniform(-scale, scale, (n, 3))
