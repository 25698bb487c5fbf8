"""Pins for the oracle's frames and pixelisation (Sec. 3.2, 3.4, Eq. 18).

The pixelisation is the HEALPix nested geometry of Gorski et al. (2005),
which Sec. 3.2 adopts: 12 equal base pixels, each split into four equal
children per level, children numbered 4k .. 4k + 3.
"""
import math
import os

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    out = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            out.append([c.strip() for c in line.split("|")])
    return out


# ---------------------------------------------------------------- Eq. 18

@pytest.mark.parametrize("ra0,dec0", [(math.pi, math.radians(45)), (0.3, -0.7), (5.9, 1.2)])
def test_rotation_maps_phase_centre_east_north(ra0, dec0):
    R = O.rotation(ra0, dec0)
    # P = [0, 0, 1] goes to RA ra0, Dec dec0 in xyz (x to RA 6h, y to NCP, z to RA 0h)
    p = R @ np.array([0, 0, 1.0])
    assert np.allclose(p, [math.cos(dec0) * math.sin(ra0), math.sin(dec0),
                           math.cos(dec0) * math.cos(ra0)], atol=1e-15)
    # u points east (increasing RA), v north (increasing Dec), Sec. 3.4
    east = np.array([math.cos(ra0), 0.0, -math.sin(ra0)])
    north = np.array([-math.sin(dec0) * math.sin(ra0), math.cos(dec0), -math.sin(dec0) * math.cos(ra0)])
    assert np.allclose(R @ np.array([1.0, 0, 0]), east, atol=1e-15)
    assert np.allclose(R @ np.array([0, 1.0, 0]), north, atol=1e-15)
    assert np.allclose(R.T @ R, np.eye(3), atol=1e-15)
    assert abs(np.linalg.det(R) - 1) < 1e-14


# ---------------------------------------------------------------- pixels

def test_golden_nested_points():
    for order, z, phi, pix in _rows("healpix_nest_points.txt"):
        k, _ = O.ang2pix_nest(int(order), float(z), float(phi))
        assert k == int(pix), (order, z, phi, k, pix)


def test_base_pixel_centres():
    # Gorski et al. 2005: base-pixel centres at z in {2/3, 0, -2/3}.
    for f in range(12):
        z, st, phi = O.pix2ang_nest(0, f)
        row, col = divmod(f, 4)
        zref = [2.0 / 3.0, 0.0, -2.0 / 3.0][row]
        phiref = (col + 0.5) * math.pi / 2 if row != 1 else col * math.pi / 2
        assert abs(z - zref) < 1e-15 and abs(phi - phiref) < 1e-15
        assert abs(st - math.sqrt(1 - zref * zref)) < 1e-15


def test_pixel_counts_and_area():
    # N_j = 12 * 4^(j-1) (Sec. 3.2) and A_j N_j = 4 pi.
    for J, printed, _ in _rows("pixel_counts.txt"):
        J, printed = int(J), float(printed)
        NJ = O.pixels_at_level(J)
        if J == 26:
            assert abs(NJ / 1.35e16 - 1) < 0.01
            assert abs(O.pixels_at_level(27) / printed - 1) < 0.01
        else:
            assert abs(NJ / printed - 1) < 0.02
    for j in range(1, 31):
        A = (math.pi / 3.0) * 4.0 ** (1 - j)
        assert abs(A * O.pixels_at_level(j) - 4 * math.pi) < 1e-12


@pytest.mark.parametrize("order", [0, 1, 2, 3, 4, 5])
def test_round_trip_every_pixel(order):
    n = 12 * 4 ** order
    for k in range(n):
        z, st, phi = O.pix2ang_nest(order, k)
        assert abs(st * st + z * z - 1) < 1e-14
        kk, mg = O.ang2pix_nest(order, z, phi)
        assert kk == k
        assert mg > 0.2          # the centre lies well inside its pixel


def _random_sphere(n, rng):
    z = rng.uniform(-1, 1, n)
    phi = rng.uniform(0, 2 * math.pi, n)
    return z, phi


def test_nested_parent_is_shifted_child():
    # Sec. 3.5: k_j = k_J >> 2 (J - j) -- the parent of a pixel holds the point.
    rng = np.random.default_rng(5)
    z, phi = _random_sphere(20000, rng)
    for i in range(len(z)):
        order = 1 + (i % 22)
        k, _ = O.ang2pix_nest(order, z[i], phi[i])
        kp, _ = O.ang2pix_nest(order - 1, z[i], phi[i])
        assert k >> 2 == kp


def test_equal_area_monte_carlo():
    # Sec. 3.2: the pixels at a level have equal area. Uniform points on the
    # sphere fall into the 192 order-2 pixels with equal probability.
    rng = np.random.default_rng(6)
    n = 192 * 400
    z, phi = _random_sphere(n, rng)
    counts = np.zeros(192)
    for i in range(n):
        counts[O.ang2pix_nest(2, z[i], phi[i])[0]] += 1
    e = n / 192
    chi2 = np.sum((counts - e) ** 2 / e)
    # 191 degrees of freedom: mean 191, sd ~19.5; 300 is > 5 sd
    assert chi2 < 300, chi2
    assert np.all(np.abs(counts - e) < 6 * math.sqrt(e))


def test_point_lies_near_its_pixel_centre():
    # A point is within one pixel size of its pixel's centre, and the four
    # children of a pixel have centres within one parent pixel size.
    rng = np.random.default_rng(7)
    z, phi = _random_sphere(3000, rng)
    for i in range(len(z)):
        order = i % 12
        size = math.sqrt(4 * math.pi / (12 * 4 ** order))
        k, _ = O.ang2pix_nest(order, z[i], phi[i])
        zc, stc, phc = O.pix2ang_nest(order, k)
        st = math.sqrt(1 - z[i] ** 2)
        a = np.array([st * math.cos(phi[i]), st * math.sin(phi[i]), z[i]])
        b = np.array([stc * math.cos(phc), stc * math.sin(phc), zc])
        ang = math.acos(min(1.0, float(a @ b)))
        assert ang < 1.2 * size, (order, ang, size)


def test_pixel_dir_uvw_of_phase_centre_pixel():
    # The pixel centre returned in the uvw frame is a unit vector: check
    # s_u^2 + s_v^2 + s_w^2 = 1 using s_w = 1 + (s_w - 1).
    for J in (1, 5, 12, 20):
        for k in (0, 7, 12 * 4 ** (J - 1) - 1):
            d = O.pixel_dir_uvw(J, k, math.pi, math.radians(45))
            sw = 1 + d[2]
            assert abs(d[0] ** 2 + d[1] ** 2 + sw ** 2 - 1) < 1e-14


def test_recommended_J_table1():
    # Table 1 (Sec. 3.3): all six rows.
    mas = math.pi / (180 * 3600 * 1000)
    for name, res, J, wres in _rows("table1_recommended_J.txt"):
        assert O.recommended_J(float(res) * mas) == int(J), name
        dJ = 2.0 ** (1 - int(J)) * math.sqrt(math.pi / 3) / mas
        # the printed wavelet resolution is the rounded Delta theta_J
        assert abs(dJ / float(wres) - 1) < 0.03, (name, dJ)


# ---------------------------------------------------------------- cross-reference table (Sec. 3.5)

@pytest.mark.parametrize("ra0,dec0", [(0.3, 0.9), (4.0, -0.4), (2.0, 1.45)])
@pytest.mark.parametrize("J", [6, 12, 20])
def test_xref_phase_centre_pixel_is_the_phase_centre_direction(ra0, dec0, J):
    # image pixel (n/2, n/2) is l = m = 0, the phase centre itself: its sphere
    # pixel is that of (RA, Dec) = (ra0, dec0), found here straight from the
    # spherical coordinates (z = sin dec, phi = RA) without the rotation
    n, dl = 16, 1e-4
    table, margin = O.xref_table(n, dl, ra0, dec0, J)
    k, mg = O.ang2pix_nest(J - 1, math.sin(dec0), ra0 % (2 * math.pi))
    assert min(mg, margin[n // 2, n // 2]) > 1e-6    # clear of every edge: the keys must agree
    assert table[n // 2, n // 2] == k


def test_xref_levels_nest():
    # the table at level J, shifted by 2 (J - j) bits, is the table at level j
    # (k_j = k_J >> 2 (J - j)) wherever neither pixel edge is within reach
    n, dl, ra0, dec0 = 48, 3e-3, 1.1, 0.6
    tJ, mJ = O.xref_table(n, dl, ra0, dec0, 14)
    for j in (3, 8, 11):
        tj, mj = O.xref_table(n, dl, ra0, dec0, j)
        ok = (mJ > 1e-9) & (mj > 1e-9)
        assert ok.mean() > 0.99
        assert np.array_equal(tJ[ok] >> (2 * (14 - j)), tj[ok])


def test_xref_outside_the_unit_disc_and_pixel_sharing():
    # corners beyond l^2 + m^2 = 1 are -1; with pixels much smaller than the
    # sphere pixels, neighbouring image pixels share a sphere pixel
    table, _ = O.xref_table(8, 0.3, 0.5, 0.2, 8)
    assert table[0, 0] == -1 and table[7, 7] == -1 and table[4, 4] >= 0
    fine, _ = O.xref_table(32, 1e-6, 0.5, 0.2, 8)
    assert len(np.unique(fine)) <= 4


def _ring_scheme_centres(nside):
    """Every pixel centre (z, phi) from the RING-scheme formulas of Gorski et
    al. (2005), Sec. 4: ring i = 1 .. 4 nside - 1 from the north; in the
    polar caps (i < nside, and mirrored in the south) 4i pixels at
    z = 1 - i^2 / (3 nside^2), phi = (pi / 2i)(j - 1/2); in the equatorial
    belt (nside <= i <= 3 nside) 4 nside pixels at z = 4/3 - 2i / (3 nside),
    phi = (pi / 2 nside)(j - s/2), s = (i - nside + 1) mod 2."""
    out = []
    for i in range(1, 4 * nside):
        ii = i if i < 2 * nside else 4 * nside - i        # distance in rings from the nearer pole
        if ii < nside:
            z = 1.0 - ii * ii / (3.0 * nside * nside)
            z = z if i < 2 * nside else -z
            out += [(z, math.pi / (2 * ii) * (j - 0.5)) for j in range(1, 4 * ii + 1)]
        else:
            z = 4.0 / 3.0 - 2.0 * i / (3.0 * nside)
            s = (i - nside + 1) % 2
            out += [(z, math.pi / (2 * nside) * (j - s / 2.0)) for j in range(1, 4 * nside + 1)]
    out = np.array(out)
    out[:, 1] %= 2 * math.pi          # phi = 2 pi (j = 4 nside, s = 0) is phi = 0
    return out


@pytest.mark.parametrize("order", [3, 4])
def test_nested_pixel_centres_are_the_ring_scheme_centres(order):
    # The oracle's nested pix2ang over all 12 4^order pixels gives exactly
    # the set of centres the ring-scheme formulas give: a second derivation
    # of the geometry, independent of the nested recipe.
    nside = 1 << order
    ring = _ring_scheme_centres(nside)
    assert len(ring) == 12 * nside * nside
    nest = np.array([O.pix2ang_nest(order, k)[0::2] for k in range(12 * nside * nside)])
    key = lambda a: np.lexsort((np.round(a[:, 1], 9), np.round(a[:, 0], 9)))
    a, b = ring[key(ring)], nest[key(nest)]
    assert np.max(np.abs(a - b)) < 1e-12


@pytest.mark.parametrize("order", [3, 5, 6])
def test_points_near_ring_scheme_centres_map_to_those_pixels(order):
    # a point a thousandth of a pixel from a ring-scheme centre lies in that
    # pixel: ang2pix_nest must return the pixel whose centre it is
    nside = 1 << order
    ring = _ring_scheme_centres(nside)
    rng = np.random.default_rng(order)
    pick = ring[rng.choice(len(ring), 400, replace=False)]
    step = 1e-3 * math.sqrt(4 * math.pi / (12 * nside * nside))
    for z, phi in pick:
        zz = float(np.clip(z + step * rng.uniform(-1, 1) * math.sqrt(max(1 - z * z, 1e-12)), -1, 1))
        pp = (phi + step * rng.uniform(-1, 1) / math.sqrt(max(1 - z * z, 1e-12))) % (2 * math.pi)
        k, _ = O.ang2pix_nest(order, zz, pp)
        zc, _, pc = O.pix2ang_nest(order, k)
        assert abs(zc - z) < 1e-12 and abs((pc - phi + math.pi) % (2 * math.pi) - math.pi) < 1e-12
