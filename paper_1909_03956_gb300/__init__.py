"""GB300-native model-visibility prediction (arXiv:1909.03956).

A thin ctypes binding over ``libwtvis.so``, the C-ABI library declared in
``include/wtvis.h``. The functions here carry the same names as the C entry
points and only marshal arguments: torch tensors supply device memory and
the current CUDA stream; every step of the computation runs in the library's
CUDA kernels. There is no CPU fallback: if the library cannot be loaded, or
a call fails, an exception is raised.

Entry points (see include/wtvis.h for the contract of each):
    wt_build_tree     components -> sphere pixels -> coefficient tree (Sec. 3.5)
    wt_tree_info      tree sizes
    wt_tree_export    tree arrays, breadth-first, on the host
    wt_free_tree      release a tree
    wt_predict_vis    Eq. 17 (or Eq. 16) per visibility on the tree
    dft_predict_vis   Eq. 12, direct sum over the components
    subtract_model    V_resid = V - V_M (Sec. 2.2)
    wt_recommended_J  Table 1 rule (Sec. 3.3)
    wt_device_status  read and clear the device-side status word
    wt_dirty_image    gridding and FFT to the dirty image or beam (Sec. 2.2)
    wt_hogbom         Hogbom clean (Eqs. 4-5)
    wt_clean          Cotton-Schwab major cycles around the prediction
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

WT_OK, WT_ERR_ARG, WT_ERR_RANGE, WT_ERR_CUDA, WT_ERR_NOMEM, WT_ERR_TIMEOUT, WT_ERR_CORRUPT, WT_ERR_UNSUPPORTED = \
    0, -1, -2, -3, -4, -5, -6, -7
WT_FP64, WT_MIXED, WT_LEARNED, WT_MIXED_FAST, WT_FP64_DF, WT_MIXED_TC = 0, 1, 2, 3, 4, 5
WT_SUM_EQ17, WT_SUM_EQ16, WT_SUM_EQ17_REGROUPED = 0, 1, 2
WT_PREDICT_TREE, WT_PREDICT_DIRECT = 0, 1
WT_RESPONSE_SNAPPED, WT_RESPONSE_LEARNED, WT_RESPONSE_EXACT = 0, 1, 2

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libwtvis.so")

# Every symbol include/wtvis.h declares.
EXPORTS = [
    "wt_build_tree", "wt_tree_info", "wt_tree_export", "wt_free_tree", "wt_predict_vis",
    "dft_predict_vis", "subtract_model", "wt_recommended_J", "wt_device_status", "wt_last_error",
    "dft_predict_vis_noalloc", "wt_predict_vis_batched",
    "wt_mlp_create", "wt_mlp_free", "wt_mlp_get_params", "wt_mlp_set_params", "wt_response_exact",
    "wt_mlp_loss_grad", "wt_mlp_train", "wt_mlp_eval", "wt_predict_vis_learned",
    "wt_selftest_bounded_wait", "wt_selftest_grid_barrier", "wt_dirty_image", "wt_hogbom", "wt_clean",
    "wt_xref_table", "wt_build_tree_xref", "wt_measure_pipe_rates",
    "wt_selftest_context_reset", "wt_predict_vis_truncated",
    "wt_predict_vis_thresholded", "wt_tree_import", "wt_mlp_get_state", "wt_mlp_set_state", "wt_mlp_train_range",
    "wt_dirty_image_w",
]
MLP_N_PARAMS = 4546
WT_NOALLOC_MAX_COMPONENTS = 65536
WT_TRUNCATED_TC_MIN_NODES = 160


class WtError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s (status %d)" % (msg, status))
        self.status = status


_lib = None


def load(build_if_missing=True):
    """Load libwtvis.so (building it with nvcc when absent or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        from . import build as _b
        _b.build()
    if not os.path.exists(LIB_PATH):
        raise ImportError("libwtvis.so is not built (%s); run paper_1909_03956_gb300/build.py" % LIB_PATH)
    L = C.CDLL(LIB_PATH)
    _declare(L)
    _lib = L
    return L


def _declare(L):
    vp, d, i64 = C.c_void_p, C.c_double, C.c_int64
    L.wt_build_tree.argtypes = [vp, vp, vp, i64, d, d, C.c_int, C.POINTER(vp), vp]
    L.wt_xref_table.argtypes = [C.c_int, d, d, d, C.c_int, vp, vp]
    L.wt_build_tree_xref.argtypes = [vp, C.c_int, vp, vp, i64, d, d, C.c_int, C.POINTER(vp), vp]
    L.wt_tree_info.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(i64), C.POINTER(i64), vp]
    L.wt_tree_export.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
    L.wt_free_tree.argtypes = [vp]
    L.wt_free_tree.restype = None
    L.wt_predict_vis.argtypes = [vp, vp, i64, vp, C.c_int, C.c_int, C.c_int, vp]
    L.dft_predict_vis.argtypes = [vp, vp, vp, i64, vp, i64, vp, C.c_int, C.c_int, vp]
    L.dft_predict_vis_noalloc.argtypes = [vp, vp, vp, i64, vp, i64, vp, C.c_int, C.c_int, vp, vp]
    L.subtract_model.argtypes = [vp, vp, vp, i64, C.c_int, vp]
    L.wt_predict_vis_batched.argtypes = [vp, vp, C.c_int, vp, i64, vp, C.c_int, C.c_int, vp]
    f = C.c_float
    L.wt_mlp_create.argtypes = [C.c_int, d, d, C.c_int, f, C.c_uint64, C.POINTER(vp)]
    L.wt_mlp_free.argtypes = [vp]
    L.wt_mlp_free.restype = None
    L.wt_mlp_get_params.argtypes = [vp, vp]
    L.wt_mlp_set_params.argtypes = [vp, vp]
    L.wt_response_exact.argtypes = [C.c_int, C.c_int, d, d, vp, i64, C.c_int, vp, vp]
    L.wt_mlp_loss_grad.argtypes = [vp, vp, vp, i64, vp, vp, vp]
    L.wt_mlp_train.argtypes = [vp, vp, vp, i64, C.c_int, C.c_int, f, vp, vp]
    L.wt_mlp_eval.argtypes = [vp, vp, i64, C.c_int, vp, vp]
    L.wt_predict_vis_learned.argtypes = [vp, vp, vp, i64, vp, C.c_int, vp]
    L.wt_mlp_train_range.argtypes = [vp, vp, vp, i64, i64, C.c_int, i64, C.c_int, f, vp, vp]
    L.wt_mlp_get_state.argtypes = [vp, vp, vp, vp, C.POINTER(C.c_int64)]
    L.wt_mlp_set_state.argtypes = [vp, vp, vp, vp, i64]
    L.wt_tree_import.argtypes = [vp, vp, i64, d, d, C.c_int, C.POINTER(C.c_void_p), vp]
    L.wt_predict_vis_truncated.argtypes = [vp, C.c_int, C.c_int, vp, C.c_int, vp, i64, vp, C.c_int, vp]
    L.wt_predict_vis_thresholded.argtypes = [vp, C.c_int, d, C.c_int, vp, C.c_int, vp, i64, vp, C.c_int, vp]
    L.wt_recommended_J.argtypes = [d]
    L.wt_device_status.argtypes = [vp]
    L.wt_selftest_bounded_wait.argtypes = [C.c_uint32, vp]
    L.wt_selftest_grid_barrier.argtypes = [C.c_uint32, vp]
    L.wt_measure_pipe_rates.argtypes = [C.POINTER(C.c_double), vp]
    L.wt_selftest_context_reset.argtypes = []
    L.wt_last_error.restype = C.c_char_p
    L.wt_dirty_image.argtypes = [vp, vp, i64, C.c_int, d, vp, vp]
    L.wt_dirty_image_w.argtypes = [vp, vp, i64, C.c_int, d, C.c_int, d, vp, vp]
    L.wt_hogbom.argtypes = [vp, vp, C.c_int, f, f, C.c_int, vp, vp, vp, vp]
    L.wt_clean.argtypes = [vp, vp, i64, C.c_int, d, d, d, C.c_int, C.c_int, C.c_int, f, f, C.c_int, C.c_int,
                           C.c_int, vp, vp, C.POINTER(C.c_int), vp, vp, vp]


def _check(rc):
    if rc != WT_OK:
        raise WtError(rc, load().wt_last_error().decode())
    return rc


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _dev(t, dtype):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError("expected dtype %s, got %s" % (dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


def _vis_dtype(mode):
    import torch
    return torch.complex128 if mode in (WT_FP64, WT_FP64_DF) else torch.complex64


# ---------------------------------------------------------------- tree

class Tree:
    """Owns a wt_tree handle (freed on close / garbage collection)."""

    def __init__(self, handle, J):
        self.h = handle
        self.J = J

    def close(self):
        if self.h:
            load().wt_free_tree(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        return wt_tree_info(self)

    def export(self):
        return wt_tree_export(self)


def wt_build_tree(l, m, flux, ra0, dec0, J, stream=None):
    """Build the coefficient tree of Sec. 3.5 from float64 CUDA tensors."""
    import torch
    n = l.numel()
    h = C.c_void_p()
    _check(load().wt_build_tree(_dev(l, torch.float64), _dev(m, torch.float64), _dev(flux, torch.float64), n,
                                float(ra0), float(dec0), int(J), C.byref(h), _stream(stream)))
    return Tree(h, int(J))


def wt_xref_table(n, dl, ra0, dec0, J, out=None, stream=None):
    """Cross-reference table (Sec. 3.5): k_J of every pixel of an n x n image
    of pixel size dl, as an int64 CUDA tensor [n, n] (-1 outside the unit
    disc)."""
    import torch
    if out is None:
        out = torch.empty((n, n), dtype=torch.int64, device="cuda")
    _check(load().wt_xref_table(int(n), float(dl), float(ra0), float(dec0), int(J), _dev(out, torch.int64),
                                _stream(stream)))
    return out


def wt_build_tree_xref(table, pix, flux, ra0, dec0, J, stream=None):
    """Tree of components at image pixels (int32 row-major indices) with
    float64 fluxes, their k_J read from a wt_xref_table table."""
    import torch
    n = table.shape[0]
    h = C.c_void_p()
    _check(load().wt_build_tree_xref(_dev(table, torch.int64), int(n), _dev(pix, torch.int32),
                                     _dev(flux, torch.float64), pix.numel(), float(ra0), float(dec0), int(J),
                                     C.byref(h), _stream(stream)))
    return Tree(h, int(J))


def wt_tree_info(tree):
    J = C.c_int()
    nl, nn = C.c_int64(), C.c_int64()
    per = np.zeros(tree.J, dtype=np.int64)
    _check(load().wt_tree_info(tree.h, C.byref(J), C.byref(nl), C.byref(nn), per.ctypes.data_as(C.c_void_p)))
    return dict(J=J.value, n_leaves=nl.value, n_nodes=nn.value, per_level=per)


def wt_tree_export(tree):
    inf = wt_tree_info(tree)
    T, NL = inf["n_nodes"], inf["n_leaves"]
    key = np.zeros(T, dtype=np.int64)
    mask = np.zeros(T, dtype=np.uint8)
    first = np.zeros(T, dtype=np.int32)
    lam = np.zeros(T)
    gam = np.zeros((T, 3))
    ldir = np.zeros((NL, 3))
    lflux = np.zeros(NL)
    p = lambda a: a.ctypes.data_as(C.c_void_p)
    _check(load().wt_tree_export(tree.h, p(key), p(mask), p(first), p(lam), p(gam), p(ldir), p(lflux)))
    offs = np.concatenate([[0], np.cumsum(inf["per_level"])])
    return dict(key=key, child_mask=mask, first_child=first, lam=lam, gamma=gam, leaf_dir=ldir,
                leaf_flux=lflux, level_offsets=offs, **inf)


def wt_tree_import(leaf_keys, leaf_flux, ra0, dec0, J, stream=None):
    """Rebuild a tree from its leaves (host arrays: the level-J keys and
    merged fluxes of wt_tree_export): bit for bit the exported tree."""
    k = np.ascontiguousarray(np.asarray(leaf_keys, dtype=np.int64))
    f = np.ascontiguousarray(np.asarray(leaf_flux, dtype=np.float64))
    if k.shape != f.shape:
        raise ValueError("leaf_keys and leaf_flux must have the same length")
    h = C.c_void_p()
    _check(load().wt_tree_import(k.ctypes.data_as(C.c_void_p), f.ctypes.data_as(C.c_void_p), k.size, float(ra0),
                                 float(dec0), int(J), C.byref(h), _stream(stream)))
    return Tree(h, int(J))


def wt_free_tree(tree):
    tree.close()


def wt_predict_vis(tree, uvw, mode=WT_FP64, sign=1, which=None, out=None, stream=None):
    """Model visibilities on the tree (Eq. 17, or Eq. 16 with which=WT_SUM_EQ16).
    which=None: the explicit Eq. 17, or the regrouped sum for WT_FP64_DF
    (which evaluates the regrouped Eq. 17 and Eq. 16)."""
    import torch
    if which is None:
        which = WT_SUM_EQ17_REGROUPED if mode == WT_FP64_DF else WT_SUM_EQ17
    n = uvw.shape[0]
    if out is None:
        out = torch.empty(n, dtype=_vis_dtype(mode), device=uvw.device)
    _check(load().wt_predict_vis(tree.h, _dev(uvw, torch.float64), n, _dev(out, _vis_dtype(mode)), int(mode),
                                 int(sign), int(which), _stream(stream)))
    return out


def wt_predict_vis_batched(trees, freq_hz, uvw_m, mode=WT_MIXED, sign=1, out=None, stream=None):
    """Eq. 17 for many channels in one persistent, graph-captured launch.
    trees: list of Tree; freq_hz: per-channel frequencies; uvw_m: [n_vis, 3]
    metres (CUDA float64). Returns [n_ch, n_vis] visibilities."""
    import torch
    n_ch, n = len(trees), uvw_m.shape[0]
    if out is None:
        out = torch.empty((n_ch, n), dtype=_vis_dtype(mode), device=uvw_m.device)
    handles = (C.c_void_p * n_ch)(*[t.h.value if isinstance(t.h, C.c_void_p) else t.h for t in trees])
    freqs = np.ascontiguousarray(np.asarray(freq_hz, dtype=np.float64))
    if freqs.shape != (n_ch,):
        raise ValueError("freq_hz must have one entry per tree")
    _check(load().wt_predict_vis_batched(C.cast(handles, C.c_void_p), freqs.ctypes.data_as(C.c_void_p), n_ch,
                                         _dev(uvw_m, torch.float64), n, _dev(out, _vis_dtype(mode)), int(mode),
                                         int(sign), _stream(stream)))
    return out


# ---------------------------------------------------------------- learned response

class Mlp:
    """Owns a wt_mlp handle: the per-level response network."""

    def __init__(self, level, ra0, dec0, depth=4, x_max=8.0, seed=0):
        h = C.c_void_p()
        _check(load().wt_mlp_create(int(level), float(ra0), float(dec0), int(depth), float(x_max), int(seed),
                                    C.byref(h)))
        self.h, self.level, self.depth, self.x_max = h, level, depth, x_max

    def close(self):
        if self.h:
            load().wt_mlp_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self):
        p = np.zeros(MLP_N_PARAMS, dtype=np.float32)
        _check(load().wt_mlp_get_params(self.h, p.ctypes.data_as(C.c_void_p)))
        return p

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        _check(load().wt_mlp_set_params(self.h, p.ctypes.data_as(C.c_void_p)))

    def loss_grad(self, uvw, target, stream=None):
        import torch
        loss = np.zeros(1, dtype=np.float32)
        g = np.zeros(MLP_N_PARAMS, dtype=np.float32)
        _check(load().wt_mlp_loss_grad(self.h, _dev(uvw, torch.float64), _dev(target, torch.float32), uvw.shape[0],
                                       loss.ctypes.data_as(C.c_void_p), g.ctypes.data_as(C.c_void_p),
                                       _stream(stream)))
        return float(loss[0]), g

    def train(self, uvw, target, steps, batch=8192, lr=3e-3, stream=None):
        import torch
        loss = np.zeros(1, dtype=np.float32)
        _check(load().wt_mlp_train(self.h, _dev(uvw, torch.float64), _dev(target, torch.float32), uvw.shape[0],
                                   int(steps), int(batch), float(lr), loss.ctypes.data_as(C.c_void_p),
                                   _stream(stream)))
        return float(loss[0])

    def train_range(self, uvw, target, step0, steps, total_steps, batch=8192, lr=3e-3, stream=None):
        """Steps step0 .. step0 + steps - 1 of a run of total_steps."""
        import torch
        loss = np.zeros(1, dtype=np.float32)
        _check(load().wt_mlp_train_range(self.h, _dev(uvw, torch.float64), _dev(target, torch.float32),
                                         uvw.shape[0], int(step0), int(steps), int(total_steps), int(batch),
                                         float(lr), loss.ctypes.data_as(C.c_void_p), _stream(stream)))
        return float(loss[0])

    def get_state(self):
        """(params, Adam first moments, second moments, step) as host arrays."""
        p, m1, m2 = (np.zeros(MLP_N_PARAMS, dtype=np.float32) for _ in range(3))
        st = C.c_int64()
        _check(load().wt_mlp_get_state(self.h, p.ctypes.data_as(C.c_void_p), m1.ctypes.data_as(C.c_void_p),
                                       m2.ctypes.data_as(C.c_void_p), C.byref(st)))
        return p, m1, m2, st.value

    def set_state(self, params, m1, m2, step):
        a = [np.ascontiguousarray(x, dtype=np.float32) for x in (params, m1, m2)]
        _check(load().wt_mlp_set_state(self.h, *[x.ctypes.data_as(C.c_void_p) for x in a], int(step)))

    def eval(self, uvw, sign=1, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty(uvw.shape[0], dtype=torch.complex64, device=uvw.device)
        _check(load().wt_mlp_eval(self.h, _dev(uvw, torch.float64), uvw.shape[0], int(sign),
                                  _dev(out, torch.complex64), _stream(stream)))
        return out


def wt_response_exact(level, depth, ra0, dec0, uvw, sign=1, out=None, stream=None):
    """Exact per-level pixel response R_j(B) (float64)."""
    import torch
    if out is None:
        out = torch.empty(uvw.shape[0], dtype=torch.complex128, device=uvw.device)
    _check(load().wt_response_exact(int(level), int(depth), float(ra0), float(dec0), _dev(uvw, torch.float64),
                                    uvw.shape[0], int(sign), _dev(out, torch.complex128), _stream(stream)))
    return out


def wt_predict_vis_learned(tree, mlp, uvw, sign=1, out=None, stream=None):
    """Learned form: the level-J sum with each leaf's full pixel response."""
    import torch
    if out is None:
        out = torch.empty(uvw.shape[0], dtype=torch.complex64, device=uvw.device)
    _check(load().wt_predict_vis_learned(tree.h, mlp.h, _dev(uvw, torch.float64), uvw.shape[0],
                                         _dev(out, torch.complex64), int(sign), _stream(stream)))
    return out


def wt_predict_vis_truncated(tree, level, uvw, response=WT_RESPONSE_SNAPPED, mlp=None, depth=4, sign=1, out=None,
                             stream=None):
    """The tree truncated at `level`: R(B) sum_k F_k exp(sign i 2 pi B.(c_k - P))
    over its level-`level` nodes, R = 1 (WT_RESPONSE_SNAPPED), the network
    `mlp` (WT_RESPONSE_LEARNED) or the exact response of depth `depth`
    (WT_RESPONSE_EXACT). complex64 out."""
    import torch
    if out is None:
        out = torch.empty(uvw.shape[0], dtype=torch.complex64, device=uvw.device)
    _check(load().wt_predict_vis_truncated(tree.h, int(level), int(response), mlp.h if mlp is not None else None,
                                           int(depth), _dev(uvw, torch.float64), uvw.shape[0],
                                           _dev(out, torch.complex64), int(sign), _stream(stream)))
    return out


def wt_predict_vis_thresholded(tree, j0, tau, uvw, response=WT_RESPONSE_SNAPPED, mlps=None, depth=4, sign=1,
                               out=None, stream=None):
    """Hard thresholding with full-pixel responses: the tree truncated at j0
    plus the coefficients of levels j0 .. J-1 with |gamma| >= tau, each
    through its node's four children; mlps = the networks of levels j0 .. J
    (WT_RESPONSE_LEARNED). complex64 out."""
    import torch
    if out is None:
        out = torch.empty(uvw.shape[0], dtype=torch.complex64, device=uvw.device)
    arr = None
    if mlps is not None:
        arr = (C.c_void_p * len(mlps))(*[m.h.value if isinstance(m.h, C.c_void_p) else m.h for m in mlps])
    _check(load().wt_predict_vis_thresholded(tree.h, int(j0), float(tau), int(response),
                                             C.cast(arr, C.c_void_p) if arr is not None else None, int(depth),
                                             _dev(uvw, torch.float64), uvw.shape[0], _dev(out, torch.complex64),
                                             int(sign), _stream(stream)))
    return out


def dft_predict_vis(l, m, flux, uvw, mode=WT_FP64, sign=1, out=None, stream=None):
    """Direct sum over the components (Eq. 12)."""
    import torch
    n = uvw.shape[0]
    if out is None:
        out = torch.empty(n, dtype=_vis_dtype(mode), device=uvw.device)
    _check(load().dft_predict_vis(_dev(l, torch.float64), _dev(m, torch.float64), _dev(flux, torch.float64),
                                  l.numel(), _dev(uvw, torch.float64), n, _dev(out, _vis_dtype(mode)), int(mode),
                                  int(sign), _stream(stream)))
    return out


def subtract_model(vis_obs, vis_model, mode=WT_FP64, out=None, stream=None):
    """V_resid = V - V_M (Sec. 2.2). out may be vis_obs (in place)."""
    dt = _vis_dtype(mode)
    if out is None:
        out = vis_obs.new_empty(vis_obs.shape)
    _check(load().subtract_model(_dev(vis_obs, dt), _dev(vis_model, dt), _dev(out, dt), vis_obs.numel(),
                                 int(mode), _stream(stream)))
    return out


def wt_recommended_J(dtheta_rad):
    rc = load().wt_recommended_J(float(dtheta_rad))
    if rc < 0:
        _check(rc)
    return rc


def wt_device_status(stream=None):
    return _check(load().wt_device_status(_stream(stream)))


def wt_selftest_bounded_wait(spin_limit=1000, stream=None):
    """Run the bounded-wait self-test kernel; the timeout shows up in
    wt_device_status() as WT_ERR_TIMEOUT."""
    return _check(load().wt_selftest_bounded_wait(int(spin_limit), _stream(stream)))


def wt_selftest_grid_barrier(spin_limit=1000, stream=None):
    """Run the grid-barrier self-test (a barrier that never opens); the
    timeout shows up in wt_device_status() as WT_ERR_TIMEOUT."""
    return _check(load().wt_selftest_grid_barrier(int(spin_limit), _stream(stream)))


def wt_measure_pipe_rates(stream=None):
    """Measured issue rates of the current device's pipes, per clock per SM:
    {"ffma", "ffma2_elems", "dfma", "mufu_sin", "mufu_tanh",
    "mufu_tanh_bf16x2_elems", "mufu_ex2"}."""
    out = (C.c_double * 7)()
    _check(load().wt_measure_pipe_rates(out, _stream(stream)))
    keys = ("ffma", "ffma2_elems", "dfma", "mufu_sin", "mufu_tanh", "mufu_tanh_bf16x2_elems", "mufu_ex2")
    return {k: out[i] for i, k in enumerate(keys)}


def wt_last_error():
    return load().wt_last_error().decode()


# ---------------------------------------------------------------- imaging

def wt_dirty_image(uvw, vis, n, dl, out=None, stream=None):
    """Dirty image (float32 [n][n]) of complex64 visibilities, or the dirty
    beam when vis is None (Sec. 2.2, major-cycle step 3)."""
    import torch
    if out is None:
        out = torch.empty((n, n), dtype=torch.float32, device=uvw.device)
    v = _dev(vis, torch.complex64) if vis is not None else C.c_void_p(0)
    _check(load().wt_dirty_image(_dev(uvw, torch.float64), v, uvw.shape[0], int(n), float(dl),
                                 _dev(out, torch.float32), _stream(stream)))
    return out


def wt_dirty_image_w(uvw, vis, n, dl, w_planes=128, w_max=0.0, out=None, stream=None):
    """w-corrected dirty image (float32 [n][n]) by w-projection gridding, or
    the dirty beam when vis is None (Sec. 3.6.2's wide-field imaging);
    w_max = 0 plans for the batch's own largest |w| (synchronises)."""
    import torch
    if out is None:
        out = torch.empty((n, n), dtype=torch.float32, device=uvw.device)
    v = _dev(vis, torch.complex64) if vis is not None else C.c_void_p(0)
    _check(load().wt_dirty_image_w(_dev(uvw, torch.float64), v, uvw.shape[0], int(n), float(dl), int(w_planes),
                                   float(w_max), _dev(out, torch.float32), _stream(stream)))
    return out


def wt_hogbom(image, psf, gain, max_iter, threshold=0.0, stream=None):
    """Hogbom clean of `image` (float32 [n][n], cleaned in place) with the
    beam `psf`; returns (pixels int32, fluxes float32) of the components."""
    import torch
    n = image.shape[0]
    pix = torch.empty(max(max_iter, 1), dtype=torch.int32, device=image.device)
    flux = torch.empty(max(max_iter, 1), dtype=torch.float32, device=image.device)
    cnt = torch.zeros(1, dtype=torch.int32, device=image.device)
    _check(load().wt_hogbom(_dev(image, torch.float32), _dev(psf, torch.float32), int(n), float(gain), float(threshold),
                            int(max_iter), _dev(pix, torch.int32), _dev(flux, torch.float32), _dev(cnt, torch.int32),
                            _stream(stream)))
    k = int(cnt.item())
    return pix[:k], flux[:k]


def wt_clean(uvw, vis_obs, n, dl, ra0, dec0, J, predictor=WT_PREDICT_TREE, mode=WT_MIXED_FAST, gain=0.1,
             threshold=0.0, minor_iter=100, n_major=3, w_planes=0, stream=None):
    """Cotton-Schwab major cycles with the tree (or direct-sum) prediction,
    imaging by nearest-cell gridding (w_planes = 0) or w-projection;
    returns (pixels, fluxes, residual visibilities, residual image)."""
    import torch
    n_vis = uvw.shape[0]
    cap = max(minor_iter * n_major, 1)
    pix = torch.empty(cap, dtype=torch.int32, device=uvw.device)
    flux = torch.empty(cap, dtype=torch.float32, device=uvw.device)
    resid = torch.empty(n_vis, dtype=torch.complex64, device=uvw.device)
    img = torch.empty((n, n), dtype=torch.float32, device=uvw.device)
    cnt = C.c_int(0)
    _check(load().wt_clean(_dev(uvw, torch.float64), _dev(vis_obs, torch.complex64), n_vis, int(n), float(dl),
                           float(ra0), float(dec0), int(J), int(predictor), int(mode), float(gain), float(threshold),
                           int(minor_iter), int(n_major), int(w_planes), _dev(pix, torch.int32),
                           _dev(flux, torch.float32),
                           C.byref(cnt), _dev(resid, torch.complex64), _dev(img, torch.float32), _stream(stream)))
    return pix[:cnt.value], flux[:cnt.value], resid, img
