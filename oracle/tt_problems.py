"""O1 (assembly) -- the TT problem formulations of Section 4, built core-wise.

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import this module.

Operators act on the vec_TT index space (4 = 2 x 2 modes per core) and are
TT matrices with 4 x 4 mode cores; right-hand sides are TT vectors with mode 4;
C is a TT matrix with 2 x 2 modes.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import tt


@dataclass
class TTProblem:
    kind: str
    d: int
    C: list                 # TT matrix, 2 x 2 modes
    A_eq: list              # TT matrix, 4 x 4 modes
    B_eq: list              # TT vector, mode 4
    K_y: list               # TT matrix, 4 x 4 modes
    A_ineq: list | None = None
    B_ineq: list | None = None
    K_t: list | None = None
    ones_t: list | None = None  # 1_T: ones on the non-idle inequality positions (TT matrix 2 x 2)
    ineq_sign: float = 1.0
    q: int = 0
    lam0: float = 1.0
    lam0_ineq: float = 1e-3


def graph_tt(adj_or_weights: np.ndarray, eps_rel: float = 1e-13) -> list:
    """TT-matrix cores (2 x 2 modes) of a dense graph matrix by TT-SVD of its vec_TT form."""
    n = adj_or_weights.shape[0]
    d = int(round(np.log2(n)))
    cores = tt.tt_svd(tt.vec_tt_dense(np.asarray(adj_or_weights, dtype=np.float64), d), [4] * d, eps_rel=eps_rel)
    return tt.unvec_tt(cores)


def _ones_vec(d: int) -> list:
    return [np.ones((1, 2, 1)) for _ in range(d)]


def _vec_as_diag_mat(v: list) -> list:
    """diag_TT of a mode-2 TT vector: a 2 x 2 mode TT matrix."""
    return tt.diag_tt(v)


def maxcut(adj_tt: list, d: int) -> TTProblem:
    """Section 4.1: C = (diag_TT(A_G 1) - A_G) / 4, A_eq = diag_TT(vec_TT I), B_eq = vec_TT I,
    K_Y = diag_TT(vec_TT(J - I))."""
    deg = tt.matvec(adj_tt, _ones_vec(d))
    C = tt.add(_vec_as_diag_mat(deg), adj_tt, 0.25, -0.25)
    I = tt.identity(d)
    J = tt.ones_mat(d)
    return TTProblem(kind="maxcut", d=d, C=C, A_eq=tt.diag_tt(tt.vec_tt(I)), B_eq=tt.vec_tt(I),
                     K_y=tt.diag_tt(tt.vec_tt(tt.add(J, I, 1.0, -1.0))), lam0=1.0)


def theta(adj_tt: list, d: int) -> TTProblem:
    """Section 4.2: A_eq = diag_TT(vec_TT A_G) + vec_TT(E_11) vec_TT(I)^T, B_eq = vec_TT(E_11),
    K_Y = diag_TT(vec_TT(J - A_G - E_11)), C = J; trace stored in the first entry."""
    I = tt.identity(d)
    J = tt.ones_mat(d)
    E = tt.unit_mat([0] * d, [0] * d)
    part1 = tt.diag_tt(tt.vec_tt(adj_tt))
    part2 = tt.outer(tt.vec_tt(E), tt.vec_tt(I))
    K = tt.add(tt.add(J, adj_tt, 1.0, -1.0), E, 1.0, -1.0)
    return TTProblem(kind="theta", d=d, C=J, A_eq=tt.add(part1, part2), B_eq=tt.vec_tt(E),
                     K_y=tt.diag_tt(tt.vec_tt(K)), lam0=2.0)


def corr_clustering(c_plus_tt: list, c_minus_tt: list, adj_tt: list, d: int) -> TTProblem:
    """Section 4.3: C = C+ + diag_TT(C- 1) - C-, diag(X) = 1 as in Max-Cut,
    A_ineq = diag_TT(vec_TT A_G) with the lower-bound convention, B_ineq = 0,
    K_T = diag_TT(vec_TT(J - A_G))."""
    deg = tt.matvec(c_minus_tt, _ones_vec(d))
    C = tt.add(tt.add(c_plus_tt, _vec_as_diag_mat(deg)), c_minus_tt, 1.0, -1.0)
    I = tt.identity(d)
    J = tt.ones_mat(d)
    zero = [np.zeros((1, 4, 1)) for _ in range(d)]
    q = int(round(tt.inner(tt.vec_tt(adj_tt), tt.vec_tt(J))))
    return TTProblem(kind="cc", d=d, C=C, A_eq=tt.diag_tt(tt.vec_tt(I)), B_eq=tt.vec_tt(I),
                     K_y=tt.diag_tt(tt.vec_tt(tt.add(J, I, 1.0, -1.0))),
                     A_ineq=tt.diag_tt(tt.vec_tt(adj_tt)), B_ineq=zero,
                     K_t=tt.diag_tt(tt.vec_tt(tt.add(J, adj_tt, 1.0, -1.0))),
                     ones_t=[c.copy() for c in adj_tt], ineq_sign=1.0, q=q, lam0=2.0, lam0_ineq=1e-3)
