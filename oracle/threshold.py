"""Hard thresholding of the wavelet coefficients in Eq. 17, on the CPU.

The paper's introduction (Sec. 1) describes the earlier wavelet method of
McEwen (2008), which keeps only the largest wavelet coefficients (a fixed
proportion, or by annealing) and reports accurate visibilities with under
one per cent of them. This module measures what that does to the paper's
own sum, Eq. 17, on the coefficient tree of a clean-component sky.

TEST INFRASTRUCTURE, like the rest of ``oracle/``: only ``tests/`` and
``bench.py``'s CPU legs may import it; the CUDA library never calls it.
numpy only, from the oracle's exported tree (``oracle.Tree.export``).

Reading T1 (the paper is silent on thresholding its own sum): keep the K
wavelet coefficients gamma^m_{j,k} of largest magnitude (ties: breadth-first
node order, then m), set the others to zero, and evaluate Eq. 17 with the
unchanged plane-wave coefficients: eta and sigma from the recursion over
every leaf (Eqs. 14, 16 and the Eq. 9 / Eq. 10 forms), the level-1 scaling
term A_1 sum_k lambda_1,k eta_1,k always kept.
"""
from __future__ import annotations

import math

import numpy as np

# rows H_1, H_2, H_3 of the Haar butterfly over child slots c = 0..3
_H = np.array([[1, -1, 1, -1], [1, 1, -1, -1], [1, -1, -1, 1]], dtype=np.float64)


def area(j):
    """A_j = 4 pi / N_j, N_j = 12 * 4^(j-1) pixels at level j."""
    return 4.0 * math.pi / (12.0 * 4.0 ** (j - 1))


def eq17_terms(tree, J, uvw, sign=1):
    """Eq. 17 split as V = base + S @ G for the visibilities ``uvw``:
    base = A_1 sum_k lambda_1,k eta_1,k, G = every gamma^m_{j,k} (breadth-
    first nodes of levels 1..J-1, m = 1..3, flattened), S = the matching
    sigma^m_{j,k} per visibility. ``tree`` is ``oracle.Tree(...).export()``."""
    uvw = np.asarray(uvw, dtype=np.float64).reshape(-1, 3)
    offs = tree["level_offsets"]
    mask, first = tree["child_mask"], tree["first_child"]
    n_nodes = int(offs[-1])
    eta = np.zeros((uvw.shape[0], n_nodes), dtype=np.complex128)
    # leaves (level J): the plane wave at the pixel centre, Eq. 14
    t = uvw @ tree["leaf_dir"].T
    eta[:, offs[J - 1]:offs[J]] = np.exp(sign * 2j * np.pi * t)
    sigma = np.zeros((uvw.shape[0], n_nodes, 3), dtype=np.complex128)
    for j in range(J - 1, 0, -1):
        q = math.sqrt(area(j)) / 4.0
        for i in range(int(offs[j - 1]), int(offs[j])):
            slots = [c for c in range(4) if mask[i] >> c & 1]
            kids = eta[:, first[i]:first[i] + len(slots)]
            eta[:, i] = kids.sum(axis=1) / 4.0                       # Eq. 9 form, absent child = 0
            sigma[:, i, :] = q * kids @ _H[:, slots].T               # Eq. 10 form
    base = area(1) * (eta[:, offs[0]:offs[1]] @ tree["lam"][offs[0]:offs[1]])
    internal = slice(int(offs[0]), int(offs[J - 1]))
    G = tree["gamma"][internal].reshape(-1)
    S = sigma[:, internal, :].reshape(uvw.shape[0], -1)
    return base, G, S


def keep_largest(G, K):
    """Indices of the K coefficients of largest |gamma| (ties: lower index)."""
    order = np.lexsort((np.arange(len(G)), -np.abs(G)))
    return np.sort(order[:K])


def thresholded_vis(base, G, S, K):
    """Eq. 17 with only the K largest |gamma| kept (reading T1)."""
    keep = keep_largest(G, K)
    return base + S[:, keep] @ G[keep]


# ---------------------------------------------------------------------------
# Reading T2: thresholding with full-pixel responses.
#
# McEwen (2008) keeps the largest wavelet coefficients with each one's
# response over the whole of its pixels. The Haar wavelets of Eq. 10 read as
# functions on the sphere, psi^m_j,k = A_j^-1/2 sum_c H_m[c] chi_j+1,c (chi
# the indicator of a child pixel; Eq. 11 synthesises the children from
# them), are orthonormal, so the K coefficients of largest |gamma| give the
# best K-term image, and the visibility of a kept coefficient is
#   gamma^m_j,k sigma^m_j,k,  sigma^m_j,k = (sqrt(A_j)/4) sum_c H_m[c] eta_j+1,c
# with eta_j,k = exp(sign i 2 pi B.(c_j,k - P)) R_j,k(B) the plane wave's mean
# over the pixel (its full-pixel response), for all four children, present
# in the tree or not: dropping a coefficient changes the image on every
# child. Every coefficient above a level j0 is kept: together with the level-1
# term they reproduce the level-j0 image, whose visibility is the tree
# truncated at j0 with full-pixel responses (oracle reading R12, kind
# "pixel"); the K largest |gamma| among levels j0 .. J - 1 are added to it.
# The responses are dense quadratures over one common finest level
# J + d_leaf, so that a pixel's response is exactly the mean of its four
# children's, and with every coefficient kept the sum is the visibility of
# the level-J image with each pixel's flux spread over it (kind "pixel" at
# level J).
# ---------------------------------------------------------------------------

def _eta_full(j, k, uvw, ra0, dec0, depth, sign, reading="pixel", cache=None):
    """eta_j,k = exp(sign i 2 pi B.(c_j,k - P)) R(B): R = the pixel's own
    response by quadrature (reading "pixel"), the response of the level-j
    pixel holding the phase centre (reading "level", the approximation the
    GPU makes: one response per level), or 1 (reading "snapped")."""
    import oracle as O
    c = O.pixel_dir_uvw(j, int(k), ra0, dec0)
    wave = np.exp(sign * 2j * np.pi * (uvw @ c))
    if reading == "snapped":
        return wave
    if reading == "level":
        if cache is not None and j in cache:
            return wave * cache[j]
        r = O.pixel_response(j, depth, ra0, dec0, uvw, sign)
        if cache is not None:
            cache[j] = r
        return wave * r
    return wave * O.pixel_response_of(j, int(k), depth, ra0, dec0, uvw, sign)


def full_response_terms(tree, J, j0, uvw, ra0, dec0, d_leaf=2, sign=1, reading="pixel"):
    """Reading T2 split as V = base + S @ G: base = the level-j0 image's
    visibility (sum over the level-j0 nodes of A_j0 lambda_j0,k eta_j0,k),
    G = gamma^m_j,k of the nodes of levels j0 .. J-1 (breadth-first, m =
    1..3, flattened), S = the matching sigma^m_j,k from the full-pixel
    responses of all four children. ``tree`` is ``oracle.Tree(...).export()``;
    ``reading`` chooses the response (see _eta_full)."""
    uvw = np.asarray(uvw, dtype=np.float64).reshape(-1, 3)
    offs = tree["level_offsets"]
    key, lam, gam = tree["key"], tree["lam"], tree["gamma"]
    Lq = J + d_leaf
    cache = {}
    base = np.zeros(uvw.shape[0], dtype=np.complex128)
    for i in range(int(offs[j0 - 1]), int(offs[j0])):
        base += area(j0) * lam[i] * _eta_full(j0, key[i], uvw, ra0, dec0, Lq - j0, sign, reading, cache)
    G, cols = [], []
    for j in range(j0, J):
        q = math.sqrt(area(j)) / 4.0
        for i in range(int(offs[j - 1]), int(offs[j])):
            kids = np.stack([_eta_full(j + 1, 4 * int(key[i]) + c, uvw, ra0, dec0, Lq - j - 1, sign, reading, cache)
                             for c in range(4)], axis=1)
            sig = q * kids @ _H.T                                    # the three sigma^m, Eq. 10 form
            for mm in range(3):
                G.append(gam[i, mm])
                cols.append(sig[:, mm])
    S = np.stack(cols, axis=1) if cols else np.zeros((uvw.shape[0], 0), dtype=np.complex128)
    return base, np.asarray(G, dtype=np.float64), S


def keep_at_least(G, tau):
    """Indices of the coefficients with |gamma| >= tau (hard thresholding by
    value)."""
    return np.nonzero(np.abs(G) >= tau)[0]


def thresholded_vis_tau(base, G, S, tau):
    """base + the coefficients with |gamma| >= tau."""
    keep = keep_at_least(G, tau)
    return base + S[:, keep] @ G[keep]
