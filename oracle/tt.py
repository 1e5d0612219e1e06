"""O1 -- plain FP64 tensor-train algebra, written from the paper's definitions.

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import this module;
only tests, the smoke check and the benchmark's CPU-baseline leg use it.

Conventions (Section 2.3, Definitions "Tensor-Train", "TT Matrix"):

* a TT vector is a list of cores of shape (r_k, n_k, r_{k+1}), r_1 = r_{d+1} = 1;
* a TT matrix is a list of cores of shape (r_k, m_k, n_k, r_{k+1});
* full tensors use the big-endian multi-index order (alpha_1 most
  significant, Section 2.3 remark on vectorisation), i.e. numpy C order;
* vec(M) of a matrix is its row-major flattening (the worked example of
  Section 3.1 fixes this); vec_TT interleaves (alpha_k, beta_k) with alpha_k
  the more significant digit (Definition "TT Vectorisation").

Everything here is deliberately plain: einsum contractions (numpy picks the
pairwise evaluation order of each sum), numpy QR and SVD as library steps, no
blocking or fusion.
"""
from __future__ import annotations

import math

import numpy as np

# ----------------------------------------------------------------------------
# reconstruction (Definition "Tensor-Train", "TT Matrix")
# ----------------------------------------------------------------------------


def full_vec(cores: list[np.ndarray]) -> np.ndarray:
    """Dense vector of a TT vector, big-endian index order."""
    acc = np.ones((1, 1))
    for c in cores:
        r, n, r2 = c.shape
        acc = np.einsum("xa,aib->xib", acc, c).reshape(-1, r2)
    return acc[:, 0].copy()


def full_mat(cores: list[np.ndarray]) -> np.ndarray:
    """Dense matrix of a TT matrix: entry (alpha; beta) = A_1(a1,b1) ... A_d(ad,bd)."""
    acc = np.ones((1, 1, 1))
    for c in cores:
        r, m, n, r2 = c.shape
        acc = np.einsum("xya,aijb->xiyjb", acc, c)
        acc = acc.reshape(acc.shape[0] * m, acc.shape[2] * n, r2)
    return acc[:, :, 0].copy()


def ranks(cores: list[np.ndarray]) -> list[int]:
    return [int(c.shape[0]) for c in cores] + [int(cores[-1].shape[-1])]


# ----------------------------------------------------------------------------
# vec / vec_TT (Definition "TT Vectorisation" and its worked example)
# ----------------------------------------------------------------------------


def vec(m: np.ndarray) -> np.ndarray:
    """Standard row-major vectorisation of a matrix."""
    return np.asarray(m).reshape(-1).copy()


def vec_tt_permutation(d: int, n: int = 2) -> np.ndarray:
    """Index map p with vec_TT(M) = vec(M)[p] for an n^d x n^d matrix M.

    vec_TT position (alpha_1, beta_1, ..., alpha_d, beta_d) holds the entry at
    row (alpha_1..alpha_d), column (beta_1..beta_d).
    """
    size = n ** (2 * d)
    pos = np.arange(size)
    digits = []
    rem = pos
    for _ in range(2 * d):
        digits.append(rem % n)
        rem = rem // n
    digits = digits[::-1]  # most significant first: a1, b1, a2, b2, ...
    row = np.zeros(size, dtype=np.int64)
    col = np.zeros(size, dtype=np.int64)
    for k in range(d):
        row = row * n + digits[2 * k]
        col = col * n + digits[2 * k + 1]
    return row * (n**d) + col


def vec_tt_dense(m: np.ndarray, d: int, n: int = 2) -> np.ndarray:
    return vec(m)[vec_tt_permutation(d, n)]


def unvec_tt_dense(v: np.ndarray, d: int, n: int = 2) -> np.ndarray:
    out = np.zeros(n ** (2 * d))
    out[vec_tt_permutation(d, n)] = v
    return out.reshape(n**d, n**d)


def vec_tt(mat_cores: list[np.ndarray]) -> list[np.ndarray]:
    """vec_TT of a TT matrix: V_k(s, :, s') = vec(M_k(s, :, :, s'))."""
    return [c.reshape(c.shape[0], c.shape[1] * c.shape[2], c.shape[3]).copy() for c in mat_cores]


def unvec_tt(vec_cores: list[np.ndarray], n: int = 2) -> list[np.ndarray]:
    """Inverse of vec_tt for square n x n mode pairs."""
    return [c.reshape(c.shape[0], n, n, c.shape[2]).copy() for c in vec_cores]


# ----------------------------------------------------------------------------
# TT-SVD (Oseledets 2011, Algorithm 1) -- used to build TT forms from dense data
# ----------------------------------------------------------------------------


def tt_svd(full: np.ndarray, dims: list[int], eps_rel: float = 1e-14, cap: int | None = None) -> list[np.ndarray]:
    """TT decomposition of a dense tensor by sequential truncated SVDs.

    The per-unfolding threshold is eps_rel * ||full||_F / sqrt(d - 1)
    (Oseledets' split of the total error over the d - 1 bonds).
    """
    d = len(dims)
    t = np.asarray(full, dtype=np.float64).reshape(-1)
    nrm = np.linalg.norm(t)
    thr = eps_rel * nrm / math.sqrt(max(d - 1, 1))
    cores = []
    r = 1
    c = t.reshape(1, -1)
    for k in range(d - 1):
        c = c.reshape(r * dims[k], -1)
        u, s, vt = np.linalg.svd(c, full_matrices=False)
        keep = _truncation_rank(s, thr)
        if cap is not None:
            keep = min(keep, cap)
        cores.append(u[:, :keep].reshape(r, dims[k], keep))
        c = s[:keep, None] * vt[:keep]
        r = keep
    cores.append(c.reshape(r, dims[-1], 1))
    return cores


def _truncation_rank(s: np.ndarray, thr: float) -> int:
    """Smallest rank whose discarded tail energy is <= thr**2 (at least 1)."""
    tail = 0.0
    keep = len(s)
    # sum the tail from the smallest singular value upward
    for j in range(len(s) - 1, 0, -1):
        if tail + s[j] ** 2 <= thr**2:
            tail += s[j] ** 2
            keep = j
        else:
            break
    return max(keep, 1)


# ----------------------------------------------------------------------------
# core-wise constructions (Section 3.3 definitions)
# ----------------------------------------------------------------------------


def diag_tt(vec_cores: list[np.ndarray]) -> list[np.ndarray]:
    """Definition "TT Diagonalisation": M_k(s, :, :, s') = diag(V_k(s, :, s'))."""
    out = []
    for v in vec_cores:
        r, n, r2 = v.shape
        m = np.zeros((r, n, n, r2))
        for i in range(n):
            m[:, i, i, :] = v[:, i, :]
        out.append(m)
    return out


def kron(a: list[np.ndarray], b: list[np.ndarray]) -> list[np.ndarray]:
    """Definition "Kronecker product of TT matrices": C_k = A_k kron B_k.

    C_k[(sa, sb), (ia, ib), (ja, jb), (sa', sb')] = A_k[sa, ia, ja, sa'] B_k[sb, ib, jb, sb'].
    """
    out = []
    for ca, cb in zip(a, b):
        ra, ma, na, ra2 = ca.shape
        rb, mb, nb, rb2 = cb.shape
        c = np.einsum("aijb,xkly->axikjlby", ca, cb)
        out.append(c.reshape(ra * rb, ma * mb, na * nb, ra2 * rb2))
    return out


def matvec(a: list[np.ndarray], x: list[np.ndarray]) -> list[np.ndarray]:
    """TT matrix times TT vector: y_k[(p, a), i, (q, b)] = sum_j A_k[p, i, j, q] x_k[a, j, b]."""
    out = []
    for ca, cx in zip(a, x):
        p, m, n, q = ca.shape
        a_, n2, b_ = cx.shape
        assert n == n2
        y = np.einsum("pijq,ajb->paiqb", ca, cx)
        out.append(y.reshape(p * a_, m, q * b_))
    return out


def matmul(a: list[np.ndarray], b: list[np.ndarray]) -> list[np.ndarray]:
    """TT matrix product: C_k[(p, a), i, l, (q, b)] = sum_j A_k[p, i, j, q] B_k[a, j, l, b]."""
    out = []
    for ca, cb in zip(a, b):
        p, m, n, q = ca.shape
        a_, n2, l, b_ = cb.shape
        assert n == n2
        c = np.einsum("pijq,ajlb->pailqb", ca, cb)
        out.append(c.reshape(p * a_, m, l, q * b_))
    return out


def transpose(a: list[np.ndarray]) -> list[np.ndarray]:
    """TT matrix transpose: swap the row and column mode of every core."""
    return [c.transpose(0, 2, 1, 3).copy() for c in a]


def scale(cores: list[np.ndarray], alpha: float) -> list[np.ndarray]:
    out = [c.copy() for c in cores]
    out[0] = out[0] * alpha
    return out


def add(a: list[np.ndarray], b: list[np.ndarray], alpha: float = 1.0, beta: float = 1.0) -> list[np.ndarray]:
    """alpha * A + beta * B by block-diagonal core concatenation (ranks add)."""
    d = len(a)
    out = []
    for k in range(d):
        ca, cb = a[k], b[k]
        mode_shape = ca.shape[1:-1]
        assert mode_shape == cb.shape[1:-1]
        ra, ra2 = ca.shape[0], ca.shape[-1]
        rb, rb2 = cb.shape[0], cb.shape[-1]
        if d == 1:
            out.append(alpha * ca + beta * cb)
            continue
        if k == 0:
            c = np.zeros((1,) + mode_shape + (ra2 + rb2,))
            c[..., :ra2] = alpha * ca
            c[..., ra2:] = beta * cb
        elif k == d - 1:
            c = np.zeros((ra + rb,) + mode_shape + (1,))
            c[:ra] = ca
            c[ra:] = cb
        else:
            c = np.zeros((ra + rb,) + mode_shape + (ra2 + rb2,))
            c[:ra, ..., :ra2] = ca
            c[ra:, ..., ra2:] = cb
        out.append(c)
    return out


def hadamard(a: list[np.ndarray], b: list[np.ndarray]) -> list[np.ndarray]:
    """Element-wise product of two TT tensors with equal mode shapes (ranks multiply).

    For TT matrices this is the product that the Remark of Section 3.3 writes
    as vec_TT(M . N) = diag_TT(vec_TT(M)) vec_TT(N).
    """
    out = []
    for ca, cb in zip(a, b):
        ra, ra2 = ca.shape[0], ca.shape[-1]
        rb, rb2 = cb.shape[0], cb.shape[-1]
        mode = ca.shape[1:-1]
        c = ca.reshape(ra, 1, -1, ra2, 1) * cb.reshape(1, rb, -1, 1, rb2)
        out.append(c.reshape((ra * rb,) + mode + (ra2 * rb2,)))
    return out


def identity(d: int, n: int = 2) -> list[np.ndarray]:
    """The identity I = I_n kron ... kron I_n (TT rank 1, Section 4)."""
    return [np.eye(n).reshape(1, n, n, 1) for _ in range(d)]


def ones_mat(d: int, n: int = 2) -> list[np.ndarray]:
    """The all-ones matrix J = J_n kron ... kron J_n (TT rank 1, Section 4)."""
    return [np.ones((1, n, n, 1)) for _ in range(d)]


def unit_mat(alpha: list[int], beta: list[int], n: int = 2) -> list[np.ndarray]:
    """E_(alpha; beta) = E_{a1 b1} kron ... kron E_{ad bd} (TT rank 1, Section 4)."""
    out = []
    for a, b in zip(alpha, beta):
        c = np.zeros((1, n, n, 1))
        c[0, a, b, 0] = 1.0
        out.append(c)
    return out


def outer(u: list[np.ndarray], v: list[np.ndarray]) -> list[np.ndarray]:
    """TT matrix u v^T from TT vectors u, v: core [(pu, pv), i, j, (qu, qv)] = u[pu, i, qu] v[pv, j, qv]."""
    out = []
    for cu, cv in zip(u, v):
        c = np.einsum("aib,xjy->axijby", cu, cv)
        ru, nu, ru2 = cu.shape
        rv, nv, rv2 = cv.shape
        out.append(c.reshape(ru * rv, nu, nv, ru2 * rv2))
    return out


# ----------------------------------------------------------------------------
# inner products and norms
# ----------------------------------------------------------------------------


def inner(u: list[np.ndarray], v: list[np.ndarray]) -> float:
    """<u, v> over all entries by a left-to-right sweep of 2-TT environments."""
    phi = np.ones((1, 1))
    for cu, cv in zip(u, v):
        ru, ru2 = cu.shape[0], cu.shape[-1]
        rv, rv2 = cv.shape[0], cv.shape[-1]
        a = cu.reshape(ru, -1, ru2)
        b = cv.reshape(rv, -1, rv2)
        phi = np.einsum("ax,aib,xiy->by", phi, a, b, optimize=True)
    return float(phi[0, 0])


def norm(u: list[np.ndarray]) -> float:
    return math.sqrt(max(inner(u, u), 0.0))


# ----------------------------------------------------------------------------
# interface / frame matrices (Definitions "Interface Matrix", "Frame Matrix")
# ----------------------------------------------------------------------------


def interface_left(cores: list[np.ndarray], k: int) -> np.ndarray:
    """T^{<k} (k is 0-based: product of cores 0..k-1), shape (prod n_<k, r_k)."""
    acc = np.ones((1, 1))
    for c in cores[:k]:
        r, n, r2 = c.shape
        acc = np.einsum("xa,aib->xib", acc, c).reshape(-1, r2)
    return acc


def interface_right(cores: list[np.ndarray], k: int) -> np.ndarray:
    """T^{>k} (0-based: product of cores k+1..d-1), shape (prod n_>k, r_{k+1})."""
    acc = np.ones((1, 1))
    for c in reversed(cores[k + 1 :]):
        r, n, r2 = c.shape
        # rows: (alpha_{k+1}, ..., alpha_d) big-endian, so new digit is most significant
        acc = np.einsum("aib,yb->iya", c, acc).reshape(-1, r)
    return acc


def frame(cores: list[np.ndarray], k: int) -> np.ndarray:
    """T_{!=k} = T^{<k} kron I_{n_k} kron T^{>k}; vec(T) = T_{!=k} vec(T_k)."""
    n = cores[k].shape[1]
    return np.kron(np.kron(interface_left(cores, k), np.eye(n)), interface_right(cores, k))


# ----------------------------------------------------------------------------
# environments and local operators (Section 3.3, matrix-free local products)
# ----------------------------------------------------------------------------


# The local products are evaluated as the three successive matrix products the
# paper's cost statement for the matrix-free local product describes
# (Section 3.3): contract over the vector rank, then over (operator rank,
# mode), then over the frame rank and mode. Each step is one tensordot.


def env_left_step(phi: np.ndarray, u: np.ndarray, op: np.ndarray, v: np.ndarray) -> np.ndarray:
    """Phi'[b', q, b] = sum U[a', i, b'] Op[p, i, j, q] V[a, j, b] Phi[a', p, a]."""
    t1 = np.tensordot(phi, v, axes=([2], [0]))          # [a', p, j, b]
    t2 = np.tensordot(t1, op, axes=([1, 2], [0, 2]))     # [a', b, i, q]
    return np.tensordot(u, t2, axes=([0, 1], [0, 2])).transpose(0, 2, 1).copy()  # [b', q, b]


def env_right_step(psi: np.ndarray, u: np.ndarray, op: np.ndarray, v: np.ndarray) -> np.ndarray:
    """Psi'[a', p, a] = sum U[a', i, b'] Op[p, i, j, q] V[a, j, b] Psi[b', q, b]."""
    t1 = np.tensordot(v, psi, axes=([2], [2]))           # [a, j, b', q]
    t2 = np.tensordot(t1, op, axes=([1, 3], [2, 3]))     # [a, b', p, i]
    return np.tensordot(u, t2, axes=([1, 2], [3, 1])).transpose(0, 2, 1).copy()  # [a', p, a]


def envs_left(u: list[np.ndarray], op: list[np.ndarray], v: list[np.ndarray]) -> list[np.ndarray]:
    """Left environments Phi_0..Phi_d (Phi_k covers cores 0..k-1)."""
    out = [np.ones((1, 1, 1))]
    for k in range(len(u)):
        out.append(env_left_step(out[-1], u[k], op[k], v[k]))
    return out


def envs_right(u: list[np.ndarray], op: list[np.ndarray], v: list[np.ndarray]) -> list[np.ndarray]:
    """Right environments Psi_0..Psi_d (Psi_k covers cores k..d-1; Psi_d = 1)."""
    d = len(u)
    out = [None] * (d + 1)
    out[d] = np.ones((1, 1, 1))
    for k in range(d - 1, -1, -1):
        out[k] = env_right_step(out[k + 1], u[k], op[k], v[k])
    return out


def local_apply(phi: np.ndarray, op: np.ndarray, psi: np.ndarray, x: np.ndarray) -> np.ndarray:
    """y[a', i, b'] = sum Phi[a', p, a] Op[p, i, j, q] Psi[b', q, b] x[a, j, b]."""
    t1 = np.tensordot(phi, x, axes=([2], [0]))           # [a', p, j, b]
    t2 = np.tensordot(t1, op, axes=([1, 2], [0, 2]))     # [a', b, i, q]
    return np.tensordot(t2, psi, axes=([3, 1], [1, 2])).copy()  # [a', i, b']


def local_matrix(phi: np.ndarray, op: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """Dense projected operator, rows (a', i, b'), columns (a, j, b)."""
    t1 = np.tensordot(phi, op, axes=([1], [0]))          # [a', a, i, j, q]
    m = np.tensordot(t1, psi, axes=([4], [1]))           # [a', a, i, j, b', b]
    m = m.transpose(0, 2, 4, 1, 3, 5)
    s = m.shape
    return m.reshape(s[0] * s[1] * s[2], s[3] * s[4] * s[5]).copy()


def local_matrix_by_frame(u: list[np.ndarray], op: list[np.ndarray], v: list[np.ndarray], k: int) -> np.ndarray:
    """U_{!=k}^T Op V_{!=k} with the dense frames (small d only)."""
    return frame(u, k).T @ full_mat(op) @ frame(v, k)


def identity_op(d: int, n: int = 4) -> list[np.ndarray]:
    return [np.eye(n).reshape(1, n, n, 1) for _ in range(d)]


# ----------------------------------------------------------------------------
# orthogonalisation and rounding (TT rounding of Oseledets 2011)
# ----------------------------------------------------------------------------


def orth_right(cores: list[np.ndarray]) -> list[np.ndarray]:
    """Right-to-left QR sweep: cores 1..d-1 become right-orthonormal."""
    c = [x.copy() for x in cores]
    for k in range(len(c) - 1, 0, -1):
        r, n, r2 = c[k].shape
        mat = c[k].reshape(r, n * r2)
        q, rr = np.linalg.qr(mat.T)  # mat^T = q rr  ->  mat = rr^T q^T
        newr = q.shape[1]
        c[k] = q.T.reshape(newr, n, r2)
        c[k - 1] = np.einsum("aib,cb->aic", c[k - 1], rr)
    return c


def orth_left(cores: list[np.ndarray]) -> list[np.ndarray]:
    """Left-to-right QR sweep: cores 0..d-2 become left-orthonormal."""
    c = [x.copy() for x in cores]
    for k in range(len(c) - 1):
        r, n, r2 = c[k].shape
        q, rr = np.linalg.qr(c[k].reshape(r * n, r2))
        newr = q.shape[1]
        c[k] = q.reshape(r, n, newr)
        c[k + 1] = np.einsum("ab,bjc->ajc", rr, c[k + 1])
    return c


def tie_flag(tail: float, thr2: float) -> bool:
    """A bond whose tail energy lies within 4 ulp of the threshold is a tie."""
    return abs(tail - thr2) <= 4.0 * np.spacing(max(thr2, 1e-300))


def round_tt(cores: list[np.ndarray], delta: float, cap: int | None = None):
    """round_TT(T, delta) for a TT vector (use vec_tt for TT matrices).

    Right-to-left QR, then left-to-right truncated SVD. Bond k keeps the
    smallest rank whose discarded energy is <= (delta / sqrt(d - 1))^2, then at
    most `cap`. Returns (cores, zeta, ties) with zeta = sqrt(sum of all
    discarded sigma^2) = ||T - round(T)||_F and the per-bond tie flags.
    """
    d = len(cores)
    c = orth_right(cores)
    thr = delta / math.sqrt(max(d - 1, 1))
    thr2 = thr * thr
    zeta2 = 0.0
    ties = []
    for k in range(d - 1):
        r, n, r2 = c[k].shape
        u, s, vt = np.linalg.svd(c[k].reshape(r * n, r2), full_matrices=False)
        keep = _truncation_rank(s, thr)
        # tie detection on the tail at the chosen rank and at one more rank
        tail_keep = float(np.sum(s[keep:] ** 2))
        tail_less = float(np.sum(s[keep - 1 :] ** 2)) if keep > 1 else float("inf")
        ties.append(tie_flag(tail_keep, thr2) or tie_flag(tail_less, thr2))
        if cap is not None and keep > cap:
            keep = cap
        zeta2 += float(np.sum(s[keep:] ** 2))
        c[k] = u[:, :keep].reshape(r, n, keep)
        c[k + 1] = np.einsum("a,ab,bjc->ajc", s[:keep], vt[:keep], c[k + 1], optimize=True)
    return c, math.sqrt(zeta2), ties
