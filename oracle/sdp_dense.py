"""O2 / O3 -- dense FP64 SDP oracles.

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import this module.

O2 (result oracle): the standard-form SDPs of the three examples of Section 2.2
(Max-Cut relaxation, Lovasz theta, correlation clustering), built straight
from the graph, solved by a textbook dense infeasible primal-dual
path-following method: HKM direction, Mehrotra predictor-corrector, the
step-length rule of Theorem "Optimal Step Size" (Section 2.2), damping 0.95.

    primal  max <C, X>  s.t.  A(X) = b,  G(X) + s = g,  s >= 0,  X psd
    dual    min b.y + g.t  s.t.  A^T y + G^T t - Z = C,  Z psd,  t >= 0

Every constraint matrix is symmetric and stored as its list of nonzero
entries (rows, cols, vals), both triangles.

O3 (Newton oracle): the block Newton system of Section 3.3
(eq. tt-kkt-newton-system) assembled densely on the vec_TT index space from
dense operators, for the padded formulation of Sections 3.2 and 4.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import tt as _tt

# ----------------------------------------------------------------------------
# standard-form problems from graphs (Examples of Section 2.2)
# ----------------------------------------------------------------------------


@dataclass
class DenseSDP:
    C: np.ndarray
    eq: list = field(default_factory=list)  # list of (rows, cols, vals)
    b: np.ndarray = None
    ineq: list = field(default_factory=list)
    g: np.ndarray = None

    @property
    def n(self) -> int:
        return self.C.shape[0]


def _unit(u: int, v: int, scale: float = 1.0):
    if u == v:
        return (np.array([u]), np.array([u]), np.array([scale]))
    return (np.array([u, v]), np.array([v, u]), np.array([0.5 * scale, 0.5 * scale]))


def laplacian(w: np.ndarray) -> np.ndarray:
    return np.diag(w.sum(axis=1)) - w


def maxcut_sdp(weights: np.ndarray) -> DenseSDP:
    """Example "Maximum Cut": max <L/4, X>, diag(X) = 1, X psd."""
    n = weights.shape[0]
    return DenseSDP(C=laplacian(weights) / 4.0, eq=[_unit(i, i) for i in range(n)], b=np.ones(n),
                    ineq=[], g=np.zeros(0))


def theta_sdp(adj: np.ndarray) -> DenseSDP:
    """Example "Maximum Stable Set": max <J, X>, tr X = 1, X_ij = 0 on edges, X psd."""
    n = adj.shape[0]
    idx = np.arange(n)
    eq = [(idx, idx, np.ones(n))]
    b = [1.0]
    iu, ju = np.nonzero(np.triu(adj, k=1))
    for u, v in zip(iu, ju):
        eq.append(_unit(int(u), int(v)))
        b.append(0.0)
    return DenseSDP(C=np.ones((n, n)), eq=eq, b=np.array(b), ineq=[], g=np.zeros(0))


def cc_sdp(c_plus: np.ndarray, c_minus: np.ndarray, adj: np.ndarray) -> DenseSDP:
    """Example "Correlation Clustering": max <C+ + L-, X>, diag X = 1, X_uv >= 0 on E, X psd."""
    n = c_plus.shape[0]
    C = c_plus + laplacian(c_minus)
    eq = [_unit(i, i) for i in range(n)]
    ineq = []
    iu, ju = np.nonzero(np.triu(adj, k=1))
    for u, v in zip(iu, ju):
        ineq.append(_unit(int(u), int(v), scale=-1.0))  # -X_uv <= 0
    return DenseSDP(C=C, eq=eq, b=np.ones(n), ineq=ineq, g=np.zeros(len(ineq)))


# ----------------------------------------------------------------------------
# constraint algebra
# ----------------------------------------------------------------------------


def _stack(cons):
    if not cons:
        z = np.zeros(0, dtype=np.int64)
        return z, z, np.zeros(0), z
    rows = np.concatenate([c[0] for c in cons])
    cols = np.concatenate([c[1] for c in cons])
    vals = np.concatenate([c[2] for c in cons])
    ids = np.concatenate([np.full(len(c[0]), i) for i, c in enumerate(cons)])
    return rows, cols, vals, ids


def _apply(st, m, x):
    rows, cols, vals, ids = st
    out = np.zeros(m)
    np.add.at(out, ids, vals * x[rows, cols])
    return out


def _adjoint(st, n, y):
    rows, cols, vals, ids = st
    out = np.zeros((n, n))
    np.add.at(out, (rows, cols), vals * y[ids])
    return out


def _schur(st_a, ma, st_b, mb, X, Zi, chunk=256):
    """M[i, j] = <A_i, X B_j Zi> = sum over entries (a,b,al) of A_i, (c,e,be) of B_j of al be X[a,c] Zi[e,b]."""
    ra, ca, va, ia = st_a
    rb, cb, vb, ib = st_b
    out = np.zeros((ma, mb))
    for s in range(0, len(rb), chunk):
        sl = slice(s, s + chunk)
        k = X[ra[:, None], rb[None, sl]] * Zi[cb[None, sl], ca[:, None]]
        k *= va[:, None] * vb[None, sl]
        part = np.zeros((ma, k.shape[1]))
        np.add.at(part, ia, k)
        np.add.at(out.T, ib[sl], part.T)
    return out


def max_step(M: np.ndarray, dM: np.ndarray) -> float:
    """Theorem "Optimal Step Size": sup{a : M + a dM psd} via Cholesky of M."""
    L = np.linalg.cholesky(M)
    Li = np.linalg.inv(L)
    S = -Li @ dM @ Li.T
    lam = float(np.linalg.eigvalsh(0.5 * (S + S.T))[-1])
    return math.inf if lam <= 0 else 1.0 / lam


def _max_step_vec(v: np.ndarray, dv: np.ndarray) -> float:
    neg = dv < 0
    if not np.any(neg):
        return math.inf
    return float(np.min(-v[neg] / dv[neg]))


@dataclass
class DenseResult:
    pobj: float
    dobj: float
    X: np.ndarray
    y: np.ndarray
    t: np.ndarray
    Z: np.ndarray
    iters: int
    rel_gap: float
    rel_p: float
    rel_d: float
    history: list


def solve_dense(p: DenseSDP, tol: float = 1e-9, max_iter: int = 100, gamma: float = 0.95,
                x0: float = 1.0, z0: float | None = None) -> DenseResult:
    """Infeasible primal-dual path following, HKM direction, Mehrotra predictor-corrector."""
    n = p.n
    m, q = len(p.eq), len(p.ineq)
    sa, sg = _stack(p.eq), _stack(p.ineq)
    C, b, g = p.C, p.b, p.g
    if z0 is None:
        z0 = max(1.0, float(np.abs(C).sum(axis=1).max()))
    X = x0 * np.eye(n)
    Z = z0 * np.eye(n)
    y = np.zeros(m)
    t = np.ones(q)
    s = np.ones(q)
    hist = []
    nb, nc = np.linalg.norm(b), np.linalg.norm(C)
    for it in range(max_iter + 1):
        Zi = np.linalg.inv(Z)
        Zi = 0.5 * (Zi + Zi.T)
        Rd = _adjoint(sa, n, y) + _adjoint(sg, n, t) - Z - C
        rp = b - _apply(sa, m, X)
        rg = g - _apply(sg, q, X) - s
        mu = (np.sum(X * Z) + t @ s) / (n + q)
        pobj = float(np.sum(C * X))
        dobj = float(b @ y + g @ t)
        rel_gap = abs(pobj - dobj) / (1.0 + abs(pobj) + abs(dobj))
        rel_p = math.sqrt(rp @ rp + rg @ rg) / (1.0 + nb)
        rel_d = np.linalg.norm(Rd) / (1.0 + nc)
        hist.append((it, pobj, dobj, rel_gap, rel_p, rel_d, mu))
        if max(rel_gap, rel_p, rel_d) <= tol or it == max_iter:
            break
        Maa = _schur(sa, m, sa, m, X, Zi)
        if q:
            Mag = _schur(sa, m, sg, q, X, Zi)
            Mgg = _schur(sg, q, sg, q, X, Zi) + np.diag(s / t)
            M = np.block([[Maa, Mag], [Mag.T, Mgg]])
        else:
            M = Maa
        M = 0.5 * (M + M.T)
        # Cholesky of the Schur complement; near the optimum it can lose
        # definiteness in floating point, then an LU solve is used instead
        try:
            cho = np.linalg.cholesky(M)
            solve_m = lambda rhs: np.linalg.solve(cho.T, np.linalg.solve(cho, rhs))
        except np.linalg.LinAlgError:
            solve_m = lambda rhs: np.linalg.solve(M, rhs)

        def direction(sigma_mu, corr_x, corr_s):
            H = sigma_mu * Zi - X - 0.5 * (X @ Rd @ Zi + Zi @ Rd @ X) - corr_x
            rhs_a = _apply(sa, m, H) - rp
            parts = [rhs_a]
            if q:
                parts.append(_apply(sg, q, H) + (sigma_mu - t * s - corr_s) / t - rg)
            rhs = np.concatenate(parts)
            sol = solve_m(rhs)
            dy, dt = sol[:m], sol[m:]
            dZ = _adjoint(sa, n, dy) + _adjoint(sg, n, dt) + Rd
            dX = H - 0.5 * (X @ (dZ - Rd) @ Zi + Zi @ (dZ - Rd) @ X)
            dX = 0.5 * (dX + dX.T)
            ds = (sigma_mu - t * s - corr_s - s * dt) / t if q else np.zeros(0)
            return dX, dy, dt, dZ, ds

        def steps(dX, dt, dZ, ds):
            ap = min(max_step(X, dX), _max_step_vec(s, ds) if q else math.inf)
            ad = min(max_step(Z, dZ), _max_step_vec(t, dt) if q else math.inf)
            return min(1.0, gamma * ap), min(1.0, gamma * ad)

        # predictor (affine scaling, sigma = 0)
        dXa, dya, dta, dZa, dsa = direction(0.0, 0.0, 0.0 * t)
        apa, ada = steps(dXa, dta, dZa, dsa)
        mu_aff = (np.sum((X + apa * dXa) * (Z + ada * dZa)) + (t + ada * dta) @ (s + apa * dsa)) / (n + q)
        sigma = (mu_aff / mu) ** 3
        # corrector with the second-order terms
        corr_x = 0.5 * (dXa @ dZa @ Zi + Zi @ dZa @ dXa)
        corr_s = dta * dsa
        dX, dy, dt, dZ, ds = direction(sigma * mu, corr_x, corr_s)
        ap, ad = steps(dX, dt, dZ, ds)
        X = X + ap * dX
        s = s + ap * ds
        y = y + ad * dy
        t = t + ad * dt
        Z = Z + ad * dZ
        X = 0.5 * (X + X.T)
        Z = 0.5 * (Z + Z.T)
    return DenseResult(pobj, dobj, X, y, t, Z, it, rel_gap, rel_p, rel_d, hist)


# ----------------------------------------------------------------------------
# O3: the padded TT formulation written densely (Sections 3.2, 3.3, 4)
# ----------------------------------------------------------------------------


@dataclass
class PaddedProblem:
    """Dense operators on the vec_TT index space (size 4^d) of Section 3.1."""
    d: int
    C: np.ndarray          # N x N objective
    A_eq: np.ndarray       # 4^d x 4^d
    B_eq: np.ndarray       # 4^d
    K_y: np.ndarray        # 4^d x 4^d
    A_ineq: np.ndarray | None = None
    B_ineq: np.ndarray | None = None
    K_t: np.ndarray | None = None
    ineq_sign: float = 1.0  # +1: s = A_ineq vec X - B_ineq (lower bound, Section 4.3)
    q: int = 0

    @property
    def has_ineq(self) -> bool:
        return self.A_ineq is not None


def padded_maxcut(weights: np.ndarray) -> PaddedProblem:
    """Section 4.1 written densely: C = (diag(A 1) - A)/4, A_eq = diag(vec_TT I), K_Y = diag(vec_TT(J - I))."""
    n = weights.shape[0]
    d = int(round(math.log2(n)))
    I, J = np.eye(n), np.ones((n, n))
    return PaddedProblem(d=d, C=(np.diag(weights.sum(1)) - weights) / 4.0,
                         A_eq=np.diag(_tt.vec_tt_dense(I, d)), B_eq=_tt.vec_tt_dense(I, d),
                         K_y=np.diag(_tt.vec_tt_dense(J - I, d)))


def padded_theta(adj: np.ndarray) -> PaddedProblem:
    """Section 4.2 written densely (trace stored at the first entry)."""
    n = adj.shape[0]
    d = int(round(math.log2(n)))
    A = adj.astype(np.float64)
    I, J = np.eye(n), np.ones((n, n))
    E = np.zeros((n, n))
    E[0, 0] = 1.0
    e = _tt.vec_tt_dense(E, d)
    A_eq = np.diag(_tt.vec_tt_dense(A, d)) + np.outer(e, _tt.vec_tt_dense(I, d))
    return PaddedProblem(d=d, C=J.copy(), A_eq=A_eq, B_eq=e.copy(),
                         K_y=np.diag(_tt.vec_tt_dense(J - A - E, d)))


def padded_cc(c_plus: np.ndarray, c_minus: np.ndarray, adj: np.ndarray) -> PaddedProblem:
    """Section 4.3 written densely; lower-bound inequality convention."""
    n = c_plus.shape[0]
    d = int(round(math.log2(n)))
    A = adj.astype(np.float64)
    I, J = np.eye(n), np.ones((n, n))
    C = c_plus + np.diag(c_minus.sum(1)) - c_minus
    return PaddedProblem(d=d, C=C, A_eq=np.diag(_tt.vec_tt_dense(I, d)), B_eq=_tt.vec_tt_dense(I, d),
                         K_y=np.diag(_tt.vec_tt_dense(J - I, d)), A_ineq=np.diag(_tt.vec_tt_dense(A, d)),
                         B_ineq=np.zeros(4**d), K_t=np.diag(_tt.vec_tt_dense(J - A, d)), ineq_sign=1.0,
                         q=int(A.sum()))


def kron_left(M: np.ndarray, d: int) -> np.ndarray:
    """M kron I on vec_TT space: acts as vec_TT(X) -> vec_TT(M X)."""
    P = _tt.vec_tt_permutation(d)
    K = np.kron(M, np.eye(M.shape[0]))
    return K[np.ix_(P, P)]


def kron_right(M: np.ndarray, d: int) -> np.ndarray:
    """I kron M on vec_TT space: acts as vec_TT(X) -> vec_TT(X M^T)."""
    P = _tt.vec_tt_permutation(d)
    K = np.kron(np.eye(M.shape[0]), M)
    return K[np.ix_(P, P)]


def slack(p: PaddedProblem, X: np.ndarray) -> np.ndarray:
    """s_ineq(X) with the problem's sign convention (Section 3.3; Section 4.3 lower bound)."""
    v = p.A_ineq @ _tt.vec_tt_dense(X, p.d) - p.B_ineq
    return v if p.ineq_sign > 0 else -v


def mu_of(p: PaddedProblem, X, Z, T=None) -> float:
    """mu = (<Z, X> + <vec_TT T, s_ineq(X)>) / (n^d + q) (Section 3.3)."""
    N = X.shape[0]
    val = float(np.sum(Z * X))
    if p.has_ineq:
        val += float(_tt.vec_tt_dense(T, p.d) @ slack(p, X))
    return val / (N + p.q)


def newton_system(p: PaddedProblem, X, Y, Z, T=None, mu=None, direction="aho", sigma=1.0,
                  corr_xz=None):
    """Dense block operator K and residual R of eq. tt-kkt-newton-system.

    Unknown order: [vec_TT dX, vec_TT dY, (vec_TT dT,) vec_TT dZ]. With
    direction "xz" the complementarity row uses Z kron I, I kron X and
    R_c = vec(Z X) - sigma mu vec I (the XZ warm-up direction); with "aho" it
    uses L_Z = I kron Z + Z kron I, L_X = I kron X + X kron I and
    R_c = L_Z vec X - 2 sigma mu vec I. `corr_xz` (an N x N matrix) is added
    to R_c as vec_TT(corr_xz): the Mehrotra second-order term.
    """
    d = p.d
    N = X.shape[0]
    D = 4**d
    vt = lambda M: _tt.vec_tt_dense(M, d)
    I = np.eye(N)
    if mu is None:
        mu = mu_of(p, X, Z, T)
    if direction == "aho":
        LZ = kron_right(Z, d) + kron_left(Z, d)
        LX = kron_right(X, d) + kron_left(X, d)
        Rc = LZ @ vt(X) - 2.0 * sigma * mu * vt(I)
    else:
        LZ = kron_left(Z, d)
        LX = kron_right(X, d)
        Rc = vt(Z @ X) - sigma * mu * vt(I)
    if corr_xz is not None:
        Rc = Rc + vt(corr_xz)
    Id = np.eye(D)
    Zr = np.zeros((D, D))
    sgn = p.ineq_sign
    Rd = vt(Z) + vt(p.C) - p.A_eq.T @ vt(Y)
    Rp = p.B_eq - p.A_eq @ vt(X)
    if not p.has_ineq:
        K = np.block([[Zr, -p.A_eq.T, Id],
                      [-p.A_eq, p.K_y, Zr],
                      [LZ, Zr, LX]])
        R = np.concatenate([Rd, Rp, Rc])
        return K, R
    # sign convention of Section 4.3: with s = sgn (A_ineq vec X - B_ineq) the
    # stationarity residual carries + sgn A_ineq^T vec T and the complementarity
    # linearisation + sgn T A_ineq (sgn = +1: lower bounds, the paper's CC case)
    Tm = np.diag(vt(T))
    s = slack(p, X)
    Rd = Rd + sgn * p.A_ineq.T @ vt(T)
    ones_t = np.diag(p.K_t) == 0
    Rt = vt(T) * s - sigma * mu * ones_t.astype(float)
    Dq = np.diag(s)
    K = np.block([[Zr, -p.A_eq.T, sgn * p.A_ineq.T, Id],
                  [-p.A_eq, p.K_y, Zr, Zr],
                  [sgn * Tm @ p.A_ineq, Zr, Dq + p.K_t, Zr],
                  [LZ, Zr, Zr, LX]])
    R = np.concatenate([Rd, Rp, Rt, Rc])
    return K, R


def newton_solve(p: PaddedProblem, X, Y, Z, T=None, **kw):
    """Exact Newton direction of the padded system; returns (blocks as N x N matrices, K, R)."""
    K, R = newton_system(p, X, Y, Z, T, **kw)
    sol = np.linalg.solve(K, -R)
    D = 4**p.d
    nb = len(sol) // D
    blocks = [_tt.unvec_tt_dense(sol[i * D:(i + 1) * D], p.d) for i in range(nb)]
    return blocks, K, R
