"""Brute-force combinatorial optima on small graphs (<= 16 vertices).

TEST INFRASTRUCTURE ONLY. These bound the SDP relaxations of Section 2.2 from
below (max cut, stability number, correlation-clustering integer optimum).
"""
from __future__ import annotations

import itertools

import numpy as np


def max_cut(weights: np.ndarray) -> float:
    """max over +-1 vectors of (1/2) sum_{i<j} w_ij (1 - x_i x_j) (Example "Maximum Cut")."""
    n = weights.shape[0]
    best = 0.0
    for mask in range(1 << (n - 1)):
        x = np.array([1.0 if (mask >> i) & 1 else -1.0 for i in range(n)])
        val = 0.25 * float(np.sum(weights * (1.0 - np.outer(x, x))))
        best = max(best, val)
    return best


def stability_number(adj: np.ndarray) -> int:
    """alpha(G): the largest vertex set without edges (Example "Maximum Stable Set")."""
    n = adj.shape[0]
    nbr = [int(sum(1 << j for j in range(n) if adj[i, j])) for i in range(n)]
    best = 0
    for mask in range(1 << n):
        ok = True
        m = mask
        while m:
            i = (m & -m).bit_length() - 1
            if nbr[i] & mask:
                ok = False
                break
            m &= m - 1
        if ok:
            best = max(best, bin(mask).count("1"))
    return best


def _partitions(n):
    # restricted growth strings enumerate set partitions
    a = [0] * n

    def rec(i, m):
        if i == n:
            yield list(a)
            return
        for v in range(m + 2):
            a[i] = v
            yield from rec(i + 1, max(m, v))

    if n == 0:
        yield []
        return
    a[0] = 0
    yield from rec(1, 0)


def cc_integer(c_plus: np.ndarray, c_minus: np.ndarray) -> float:
    """Example "Correlation Clustering": max over partitions of the agreement objective."""
    n = c_plus.shape[0]
    iu, ju = np.triu_indices(n, k=1)
    best = -np.inf
    for lab in _partitions(n):
        lab = np.array(lab)
        same = (lab[iu] == lab[ju]).astype(float)
        val = float(np.sum(c_plus[iu, ju] * same + c_minus[iu, ju] * (1.0 - same)))
        best = max(best, val)
    return best
