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
