"""Plain FP64 CPU oracle for arXiv:1909.03956 (model-visibility prediction).

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package. The CUDA library never imports, links or calls it, and the two share
no code: the oracle is ``oracle.c`` (plain C, double precision, built with
``-ffp-contract=off``), wrapped here with ctypes and numpy.

Every function cites the section or equation of the paper it evaluates; the
readings taken where the paper is silent are listed at the top of
``oracle.c`` (R1-R9).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_SOURCES = ["oracle.c", "oracle_mlp.c"]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, -O2, no FMA contraction)."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES if os.path.exists(os.path.join(_HERE, s))]
    newest = max(os.path.getmtime(s) for s in srcs + [os.path.join(_HERE, "oracle.h")])
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-fopenmp",
           "-Wall", "-o", tmp] + srcs + ["-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _declare(_lib)
    return _lib


_d = C.POINTER(C.c_double)
_i64 = C.POINTER(C.c_int64)
_i32 = C.POINTER(C.c_int32)
_u8 = C.POINTER(C.c_uint8)


def _declare(L):
    L.orc_dft.argtypes = [C.c_int64, _d, _d, _d, C.c_int64, _d, C.c_int, _d]
    L.orc_dft_ld.argtypes = L.orc_dft.argtypes
    L.orc_rotation.argtypes = [C.c_double, C.c_double, _d]
    L.orc_rotation.restype = None
    L.orc_ang2pix_nest.argtypes = [C.c_int, C.c_double, C.c_double, _d]
    L.orc_ang2pix_nest.restype = C.c_int64
    L.orc_pix2ang_nest.argtypes = [C.c_int, C.c_int64, _d, _d, _d]
    L.orc_pix2ang_nest.restype = None
    L.orc_pixel_dir_uvw.argtypes = [C.c_int, C.c_int64, C.c_double, C.c_double, _d]
    L.orc_pixel_dir_uvw.restype = None
    L.orc_map_components.argtypes = [C.c_int64, _d, _d, C.c_double, C.c_double, C.c_int, _i64, _d]
    L.orc_tree_build.argtypes = [C.c_int64, _d, _d, _d, C.c_double, C.c_double, C.c_int]
    L.orc_tree_build.restype = C.c_void_p
    L.orc_tree_free.argtypes = [C.c_void_p]
    L.orc_tree_free.restype = None
    L.orc_tree_sizes.argtypes = [C.c_void_p, _i64, _i64, _i64]
    L.orc_tree_export.argtypes = [C.c_void_p, _i64, _u8, _i32, _d, _d, _d, _d]
    L.orc_tree_vis_eq17.argtypes = [C.c_void_p, C.c_int64, _d, C.c_int, _d]
    L.orc_tree_vis_truncated.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int64, _d, C.c_int, _d]
    L.orc_tree_vis_eq17_mt.argtypes = [C.c_void_p, C.c_int64, _d, C.c_int, _d, C.c_int]
    L.orc_dft_mt.argtypes = [C.c_int64, _d, _d, _d, C.c_int64, _d, C.c_int, _d, C.c_int]
    L.orc_tree_vis_eq16.argtypes = [C.c_void_p, C.c_int64, _d, C.c_int, _d]
    L.orc_tree_synthesis.argtypes = [C.c_void_p, _d]
    L.orc_dense_coeffs.argtypes = [C.c_int, C.c_int64, _d, _d, _d, C.c_double, C.c_double, _d, _d]
    L.orc_dense_vis_eq17.argtypes = [C.c_int, C.c_int64, _d, _d, _d, C.c_double, C.c_double,
                                     C.c_int64, _d, C.c_int, _d]
    L.orc_recommended_J.argtypes = [C.c_double]
    L.orc_subtract.argtypes = [C.c_int64, _d, _d, _d]
    if hasattr(L, "orc_mlp_forward"):
        _declare_mlp(L)


def _declare_mlp(L):
    L.orc_pixel_response.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_int64, _d, C.c_int, _d]
    L.orc_pixel_response_of.argtypes = [C.c_int, C.c_int64, C.c_int, C.c_double, C.c_double, C.c_int64, _d, C.c_int,
                                        _d]
    L.orc_level_pixel_size.argtypes = [C.c_int]
    L.orc_level_pixel_size.restype = C.c_double
    L.orc_mlp_n_params.restype = C.c_int
    L.orc_mlp_forward.argtypes = [_d, C.c_int, C.c_int64, _d, _d]
    L.orc_mlp_loss_grad.argtypes = [_d, C.c_int, C.c_int64, _d, _d, _d, _d]


def _p(a, t=_d):
    return a.ctypes.data_as(t)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(rc, what):
    if rc != 0:
        raise ValueError("oracle %s failed with status %d" % (what, rc))


def _as_complex(buf):
    return buf[0::2] + 1j * buf[1::2]


# ---------------------------------------------------------------------------
# Eq. 12: direct sum
# ---------------------------------------------------------------------------

def dft(l, m, flux, uvw, sign=1, long_double=False, threads=1):
    """Eq. 12: V_n = sum_m C_m exp(sign i 2 pi (u l + v m + w (n - 1))).
    threads > 1 splits the visibilities over that many OpenMP threads
    (identical results)."""
    l, m, flux, uvw = _f64(l), _f64(m), _f64(flux), _f64(uvw).reshape(-1, 3)
    nv = uvw.shape[0]
    out = np.zeros(2 * nv)
    if threads > 1 and not long_double:
        _check(lib().orc_dft_mt(len(l), _p(l), _p(m), _p(flux), nv, _p(uvw), sign, _p(out), threads), "dft")
        return _as_complex(out)
    fn = lib().orc_dft_ld if long_double else lib().orc_dft
    _check(fn(len(l), _p(l), _p(m), _p(flux), nv, _p(uvw), sign, _p(out)), "dft")
    return _as_complex(out)


# ---------------------------------------------------------------------------
# Sec. 3.2 / 3.4: frames and pixels
# ---------------------------------------------------------------------------

def rotation(ra0, dec0):
    """Eq. 18: R_uvw->xyz = R_y(ra0) R_x(-dec0), row-major 3x3."""
    R = np.zeros(9)
    lib().orc_rotation(ra0, dec0, _p(R))
    return R.reshape(3, 3)


def ang2pix_nest(order, z, phi):
    """Nested pixel index at HEALPix order ``order`` (= level - 1) and the
    distance of the point to the nearest pixel edge in pixel-grid units."""
    mg = C.c_double(0.0)
    k = lib().orc_ang2pix_nest(order, float(z), float(phi), C.byref(mg))
    return int(k), mg.value


def pix2ang_nest(order, pix):
    z, st, ph = C.c_double(), C.c_double(), C.c_double()
    lib().orc_pix2ang_nest(order, int(pix), C.byref(z), C.byref(st), C.byref(ph))
    return z.value, st.value, ph.value


def pixel_dir_uvw(J, k, ra0, dec0):
    out = np.zeros(3)
    lib().orc_pixel_dir_uvw(J, int(k), ra0, dec0, _p(out))
    return out


def map_components(l, m, ra0, dec0, J):
    """Sec. 3.5 cross-reference: level-J pixel of each component and its
    margin to the nearest pixel edge (pixel-grid units)."""
    l, m = _f64(l), _f64(m)
    n = len(l)
    k = np.zeros(n, dtype=np.int64)
    mg = np.zeros(n)
    _check(lib().orc_map_components(n, _p(l), _p(m), ra0, dec0, J, _p(k, _i64), _p(mg)),
           "map_components")
    return k, mg


def xref_table(n, dl, ra0, dec0, J):
    """Sec. 3.5: the cross-reference table built before cleaning, image pixel
    -> level-J sphere pixel. Pixel (ix, iy) of an n x n image sits at
    l = (ix - n/2) dl, m = (iy - n/2) dl (the imaging geometry); the table is
    indexed [iy][ix], -1 where l^2 + m^2 >= 1. Returns the table and each
    pixel's margin to the nearest sphere-pixel edge (inf outside the disc)."""
    ax = (np.arange(n) - n // 2).astype(np.float64) * dl
    m, l = np.meshgrid(ax, ax, indexing="ij")
    inside = l * l + m * m < 1.0
    table = np.full((n, n), -1, dtype=np.int64)
    margin = np.full((n, n), np.inf)
    if inside.any():
        k, mg = map_components(l[inside], m[inside], ra0, dec0, J)
        table[inside] = k
        margin[inside] = mg
    return table, margin


# ---------------------------------------------------------------------------
# Sec. 3.5: the coefficient tree
# ---------------------------------------------------------------------------

class Tree:
    """Pointer tree of Sec. 3.5 built node by node as components arrive."""

    def __init__(self, l, m, flux, ra0, dec0, J):
        l, m, flux = _f64(l), _f64(m), _f64(flux)
        self._keep = (l, m, flux)
        self.J = J
        self.h = lib().orc_tree_build(len(l), _p(l), _p(m), _p(flux), ra0, dec0, J)
        if not self.h:
            raise ValueError("oracle tree build failed")
        nl, nn = C.c_int64(), C.c_int64()
        per = np.zeros(J, dtype=np.int64)
        lib().orc_tree_sizes(self.h, C.byref(nl), C.byref(nn), _p(per, _i64))
        self.n_leaves, self.n_nodes, self.per_level = nl.value, nn.value, per

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_tree_free(self.h)
            self.h = None

    def export(self):
        """Breadth-first arrays, nodes in (level, key) order."""
        T, NL = self.n_nodes, self.n_leaves
        key = np.zeros(T, dtype=np.int64)
        mask = np.zeros(T, dtype=np.uint8)
        first = np.zeros(T, dtype=np.int32)
        lam = np.zeros(T)
        gam = np.zeros((T, 3))
        ldir = np.zeros((NL, 3))
        lflux = np.zeros(NL)
        _check(lib().orc_tree_export(self.h, _p(key, _i64), _p(mask, _u8), _p(first, _i32),
                                     _p(lam), _p(gam), _p(ldir), _p(lflux)), "tree_export")
        offs = np.concatenate([[0], np.cumsum(self.per_level)])
        return dict(key=key, child_mask=mask, first_child=first, lam=lam, gamma=gam,
                    leaf_dir=ldir, leaf_flux=lflux, level_offsets=offs)

    def vis_eq17(self, uvw, sign=1, threads=1):
        """Eq. 17 per visibility; threads > 1 splits the visibilities over
        that many OpenMP threads (identical results)."""
        uvw = _f64(uvw).reshape(-1, 3)
        out = np.zeros(2 * uvw.shape[0])
        if threads > 1:
            _check(lib().orc_tree_vis_eq17_mt(self.h, uvw.shape[0], _p(uvw), sign, _p(out), threads), "eq17")
        else:
            _check(lib().orc_tree_vis_eq17(self.h, uvw.shape[0], _p(uvw), sign, _p(out)), "eq17")
        return _as_complex(out)

    def vis_eq16(self, uvw, sign=1):
        uvw = _f64(uvw).reshape(-1, 3)
        out = np.zeros(2 * uvw.shape[0])
        _check(lib().orc_tree_vis_eq16(self.h, uvw.shape[0], _p(uvw), sign, _p(out)), "eq16")
        return _as_complex(out)

    def vis_truncated(self, jt, uvw, kind="snapped", depth=4, sign=1):
        """The tree truncated at level jt (reading R12): sum over the level-jt
        nodes of F_k exp(sign i 2 pi B.(c_k - P)) R_k(B), F_k = A_jt lambda_jt;
        kind "snapped" R_k = 1, "level" R_k = the phase-centre pixel's
        response R_jt(B), "pixel" R_k = each pixel's own response (depth D
        quadrature)."""
        kinds = {"snapped": 0, "level": 1, "pixel": 2}
        uvw = _f64(uvw).reshape(-1, 3)
        out = np.zeros(2 * uvw.shape[0])
        _check(lib().orc_tree_vis_truncated(self.h, jt, kinds[kind], depth, uvw.shape[0], _p(uvw), sign, _p(out)),
               "truncated")
        return _as_complex(out)

    def synthesis(self):
        out = np.zeros(self.n_leaves)
        _check(lib().orc_tree_synthesis(self.h, _p(out)), "synthesis")
        return out


def pixels_at_level(j):
    return 12 * 4 ** (j - 1)


def dense_coeffs(l, m, flux, ra0, dec0, J):
    """Brute force: dense lambda_j (list per level) and gamma_j (j < J)."""
    l, m, flux = _f64(l), _f64(m), _f64(flux)
    tot = sum(pixels_at_level(j) for j in range(1, J + 1))
    gtot = sum(pixels_at_level(j) for j in range(1, J))
    lam = np.zeros(tot)
    gam = np.zeros(3 * max(gtot, 1))
    _check(lib().orc_dense_coeffs(J, len(l), _p(l), _p(m), _p(flux), ra0, dec0, _p(lam), _p(gam)),
           "dense_coeffs")
    lams, gams, o, g = [], [], 0, 0
    for j in range(1, J + 1):
        n = pixels_at_level(j)
        lams.append(lam[o:o + n])
        o += n
        if j < J:
            gams.append(gam[3 * g:3 * (g + n)].reshape(n, 3))
            g += n
    return lams, gams


def dense_vis_eq17(l, m, flux, ra0, dec0, J, uvw, sign=1):
    l, m, flux, uvw = _f64(l), _f64(m), _f64(flux), _f64(uvw).reshape(-1, 3)
    out = np.zeros(2 * uvw.shape[0])
    _check(lib().orc_dense_vis_eq17(J, len(l), _p(l), _p(m), _p(flux), ra0, dec0,
                                    uvw.shape[0], _p(uvw), sign, _p(out)), "dense_eq17")
    return _as_complex(out)


# ---------------------------------------------------------------------------
# Learned response (an addition, not in the paper): readings R10, R11 of
# oracle_mlp.c
# ---------------------------------------------------------------------------

MLP_HIDDEN = 64


def pixel_response(j, D, ra0, dec0, uvw, sign=1):
    """Exact R_j(B): mean of exp(sign i 2 pi B.(s_i - c_j)) over the 4^D
    level-(j+D) sub-pixel centres of the level-j pixel holding the phase
    centre (float64, OpenMP over samples)."""
    uvw = _f64(uvw).reshape(-1, 3)
    out = np.zeros(2 * uvw.shape[0])
    _check(lib().orc_pixel_response(j, D, ra0, dec0, uvw.shape[0], _p(uvw), sign, _p(out)), "pixel_response")
    return _as_complex(out)


def pixel_response_of(j, k, D, ra0, dec0, uvw, sign=1):
    """Exact R_j,k(B) of any level-j pixel k: mean of exp(sign i 2 pi B.(s_i -
    c_j,k)) over the centres of its 4^D descendants D levels down."""
    uvw = _f64(uvw).reshape(-1, 3)
    out = np.zeros(2 * uvw.shape[0])
    _check(lib().orc_pixel_response_of(j, int(k), D, ra0, dec0, uvw.shape[0], _p(uvw), sign, _p(out)),
           "pixel_response_of")
    return _as_complex(out)


def level_pixel_size(j):
    return float(lib().orc_level_pixel_size(j))


def mlp_n_params():
    return int(lib().orc_mlp_n_params())


def mlp_split(params):
    """Views W1[64,3], b1, W2[64,64], b2, W3[2,64], b3 of a flat vector."""
    h = MLP_HIDDEN
    o = np.cumsum([0, 3 * h, h, h * h, h, 2 * h, 2])
    p = np.asarray(params)
    return (p[o[0]:o[1]].reshape(h, 3), p[o[1]:o[2]], p[o[2]:o[3]].reshape(h, h), p[o[3]:o[4]],
            p[o[4]:o[5]].reshape(2, h), p[o[5]:o[6]])


def mlp_forward(params, level, uvw):
    params = _f64(params)
    uvw = _f64(uvw).reshape(-1, 3)
    y = np.zeros(2 * uvw.shape[0])
    _check(lib().orc_mlp_forward(_p(params), level, uvw.shape[0], _p(uvw), _p(y)), "mlp_forward")
    return y.reshape(-1, 2)


def mlp_loss_grad(params, level, uvw, target):
    """Mean squared error (both outputs) and its gradient (float64)."""
    params = _f64(params)
    uvw = _f64(uvw).reshape(-1, 3)
    target = _f64(target).reshape(-1, 2)
    g = np.zeros_like(params)
    loss = C.c_double()
    _check(lib().orc_mlp_loss_grad(_p(params), level, uvw.shape[0], _p(uvw), _p(target), C.byref(loss), _p(g)),
           "mlp_loss_grad")
    return loss.value, g


def recommended_J(dtheta_rad):
    """Sec. 3.3 / Table 1: smallest J with Delta theta_J <= Delta theta / 2."""
    return int(lib().orc_recommended_J(float(dtheta_rad)))


def subtract(obs, model):
    """Sec. 2.2 major cycle step 2: V_resid = V - V_M."""
    o = np.ascontiguousarray(np.asarray(obs, dtype=np.complex128)).view(np.float64)
    mo = np.ascontiguousarray(np.asarray(model, dtype=np.complex128)).view(np.float64)
    out = np.zeros_like(o)
    _check(lib().orc_subtract(len(o) // 2, _p(o), _p(mo), _p(out)), "subtract")
    return _as_complex(out)
