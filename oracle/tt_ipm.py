"""O4 -- the tensor-train primal-dual IPM (Algorithm 1, Sections 3.3-3.5), FP64 numpy.

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import this module;
tests, the smoke check and the benchmark's CPU-baseline leg use it.

Steps in the paper's order:

* residuals R_d, R_p, [R_t], R_c of the tensorised KKT conditions (Section 3.3);
* mu = (<Z, X> + <vec T, s>) / (n^d + q) and the relative stopping rules of
  Section 3.5 ("Error Tracking and TT Rounding Tolerance");
* the Newton system eq. tt-kkt-newton-system, XZ direction for the first
  iterations then AHO (Section 3.5, "Mehrotra's Predictor-Corrector");
* its solution by block-AMEn: one frame W shared by the blocks
  (dX, dY, [dT], dZ), dZ eliminated locally, the reduced projected system
  eq. reduced_kkt_system solved at each core, the block index moved by an SVD
  step (Section 2.3, Definition "Block Tensor-Train" and the text after it);
* step lengths from extreme generalised Rayleigh quotients found by an
  alternating (one-site) TT eigen-solver (Section 3.4);
* the update of Algorithm 1 followed by TT rounding with the spectral shift
  of Corollary psdness_rounding.

Readings where the paper is silent (shared with the CUDA path, listed in the
design notes): Mehrotra sigma = (mu_aff / mu)^3 with the second-order term
added to R_c; step damping 0.95; AMEn enrichment by a random kick of
`kick` columns from a SplitMix64 counter stream; the local system is solved
densely; every block of an XZ direction is symmetrised (M <- (M + M^T) / 2).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import tt
from .tt_problems import TTProblem

# ----------------------------------------------------------------------------
# counter-based random numbers (SplitMix64, Steele, Lea & Flood 2014)
# ----------------------------------------------------------------------------

_M64 = (1 << 64) - 1


def splitmix64(x: int) -> int:
    z = (x + 0x9E3779B97F4A7C15) & _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def uniform_pm1(seed: int, counter: int, count: int) -> np.ndarray:
    """count values in [-1, 1): value j is splitmix64(seed ^ (counter + j) * golden) mapped by the top 53 bits."""
    out = np.empty(count)
    for j in range(count):
        x = splitmix64((seed ^ (((counter + j) * 0x9E3779B97F4A7C15) & _M64)) & _M64)
        out[j] = (x >> 11) * (2.0 / 9007199254740992.0) - 1.0
    return out


class Counter:
    def __init__(self, seed: int):
        self.seed = seed
        self.n = 0

    def draw(self, shape) -> np.ndarray:
        cnt = int(np.prod(shape))
        v = uniform_pm1(self.seed, self.n, cnt)
        self.n += cnt
        return v.reshape(shape)

    def fork(self) -> "Counter":
        """A counter seeded by the raw 64-bit value of this stream's next draw
        (one draw consumed): a sub-stream whose length does not move this one."""
        x = splitmix64((self.seed ^ ((self.n * 0x9E3779B97F4A7C15) & _M64)) & _M64)
        self.n += 1
        return Counter(x)


# ----------------------------------------------------------------------------
# operator terms on the vec_TT space (4 x 4 mode cores)
# ----------------------------------------------------------------------------


def op_kron_left(m: list) -> list:
    """M kron I: acts as vec_TT(X) -> vec_TT(M X) (Definition "Kronecker product of TT matrices")."""
    return tt.kron(m, tt.identity(len(m)))


def op_kron_right(m: list) -> list:
    """I kron M: acts as vec_TT(X) -> vec_TT(X M^T)."""
    return tt.kron(tt.identity(len(m)), m)


def op_identity(d: int) -> list:
    return tt.identity_op(d, 4)


def op_diagonal(op: list) -> list:
    """The diagonal of an operator that is diag_TT of a vector: that vector's
    cores, core [p][i][q] = op[p][i][i][q] (the off-diagonal mode entries must be 0)."""
    out = []
    for c in op:
        m = c.shape[1]
        off = c.copy()
        for i in range(m):
            off[:, i, i, :] = 0.0
        assert np.abs(off).max() <= 1e-14 * max(np.abs(c).max(), 1.0), "operator is not diagonal"
        out.append(np.ascontiguousarray(np.stack([c[:, i, i, :] for i in range(m)], axis=1)))
    return out


def _ones4(d: int) -> list:
    return [np.ones((1, 4, 1)) for _ in range(d)]


# ----------------------------------------------------------------------------
# environments of one (frame, operator, vector) triple
# ----------------------------------------------------------------------------


class Env:
    """Left/right environments of <W, Op V> with W the block frame.

    left[k] covers cores 0..k-1, right[k] covers cores k..d-1 (right[d] = 1).
    V is either the frame itself (vec=None) or a fixed TT vector.
    """

    def __init__(self, op: list, vec: list | None, d: int):
        self.op = op
        self.vec = vec
        self.left = [None] * (d + 1)
        self.right = [None] * (d + 1)
        self.left[0] = np.ones((1, 1, 1))
        self.right[d] = np.ones((1, 1, 1))

    def vcore(self, w: list, k: int) -> np.ndarray:
        return w[k] if self.vec is None else self.vec[k]

    def push_left(self, w: list, k: int):
        self.left[k + 1] = tt.env_left_step(self.left[k], w[k], self.op[k], self.vcore(w, k))

    def push_right(self, w: list, k: int):
        self.right[k] = tt.env_right_step(self.right[k + 1], w[k], self.op[k], self.vcore(w, k))

    def local_rhs(self, w: list, k: int) -> np.ndarray:
        """W_{!=k}^T Op vec(V) at core k (needs vec is not None)."""
        return tt.local_apply(self.left[k], self.op[k], self.right[k + 1], self.vec[k])

    def local_mat(self, k: int) -> np.ndarray:
        return tt.local_matrix(self.left[k], self.op[k], self.right[k + 1])


# ----------------------------------------------------------------------------
# the Newton system, block structure
# ----------------------------------------------------------------------------


@dataclass
class NewtonData:
    """Operators and right-hand-side terms of eq. tt-kkt-newton-system."""
    A_eq: list
    A_eqT: list
    K_y: list
    LZ: list            # list of op cores (terms summed)
    LX: list
    rhs_p: list         # list of (coef, op cores, vector cores)
    rhs_d: list
    rhs_c: list
    # inequality block (None without inequalities)
    TA: list | None = None
    D_K: list | None = None      # list of op cores: D_ineq terms + K_T
    A_ineqT: list | None = None
    rhs_t: list | None = None
    sgn: float = 1.0
    masks: tuple | None = None   # (P_Y, P_T) diagonals when dY, dT share one block dLambda

    @property
    def nblk(self) -> int:
        return 3 if self.TA is None else 4


def _envs(data: NewtonData, d: int):
    ops = {"A": Env(data.A_eq, None, d), "AT": Env(data.A_eqT, None, d), "K": Env(data.K_y, None, d),
           "LZ": [Env(o, None, d) for o in data.LZ], "LX": [Env(o, None, d) for o in data.LX]}
    rhs = {"p": [(c, Env(o, v, d)) for c, o, v in data.rhs_p],
           "d": [(c, Env(o, v, d)) for c, o, v in data.rhs_d],
           "c": [(c, Env(o, v, d)) for c, o, v in data.rhs_c]}
    if data.TA is not None:
        ops["TA"] = Env(data.TA, None, d)
        ops["DK"] = [Env(o, None, d) for o in data.D_K]
        ops["AiT"] = Env(data.A_ineqT, None, d)
        rhs["t"] = [(c, Env(o, v, d)) for c, o, v in data.rhs_t]
    return ops, rhs


def _all_envs(ops, rhs):
    out = [ops["A"], ops["AT"], ops["K"]] + ops["LZ"] + ops["LX"]
    if "TA" in ops:
        out += [ops["TA"], ops["AiT"]] + ops["DK"]
    for key in rhs:
        out += [e for _, e in rhs[key]]
    return out


def _local_system(ops, rhs, w, k, sgn):
    """Dense reduced projected system (eq. reduced_kkt_system) at core k.

    Returns (K_loc, b_loc, r_d) for unknowns [dX_k, dY_k, (dT_k)] and the
    projected dual residual used to recover dZ_k.
    """
    A = ops["A"].local_mat(k)
    AT = ops["AT"].local_mat(k)
    Ky = ops["K"].local_mat(k)
    LZ = sum(e.local_mat(k) for e in ops["LZ"])
    LX = sum(e.local_mat(k) for e in ops["LX"])
    r_p = sum(c * e.local_rhs(w, k) for c, e in rhs["p"]).reshape(-1)
    r_d = sum(c * e.local_rhs(w, k) for c, e in rhs["d"]).reshape(-1)
    r_c = sum(c * e.local_rhs(w, k) for c, e in rhs["c"]).reshape(-1)
    n = A.shape[0]
    Z0 = np.zeros((n, n))
    if "TA" not in ops:
        K = np.block([[-A, Ky], [LZ, LX @ AT]])
        b = np.concatenate([-r_p, -r_c + LX @ r_d])
        return K, b, r_d, (AT, None, n)
    TA = ops["TA"].local_mat(k)
    DK = sum(e.local_mat(k) for e in ops["DK"])
    AiT = ops["AiT"].local_mat(k)
    r_t = sum(c * e.local_rhs(w, k) for c, e in rhs["t"]).reshape(-1)
    K = np.block([[-A, Ky, Z0], [sgn * TA, Z0, DK], [LZ, LX @ AT, -sgn * LX @ AiT]])
    b = np.concatenate([-r_p, -r_t, -r_c + LX @ r_d])
    return K, b, r_d, (AT, AiT, n)


def _truncation_rank_rel(s: np.ndarray, tol_rel: float, cap: int) -> int:
    nrm2 = float(np.sum(s**2))
    thr2 = (tol_rel**2) * nrm2
    tail = 0.0
    keep = len(s)
    for j in range(len(s) - 1, 0, -1):
        if tail + s[j] ** 2 <= thr2:
            tail += s[j] ** 2
            keep = j
        else:
            break
    return max(1, min(keep, cap))


@dataclass
class BlockTT:
    """Block TT (Definition "Block Tensor-Train") with the block index at core `pos`."""
    cores: list          # cores[k] (r, 4, r') for k != pos
    block: np.ndarray    # (nblk, r_pos, 4, r_pos+1)
    pos: int

    def component(self, b: int) -> list:
        c = [x.copy() for x in self.cores]
        c[self.pos] = self.block[b].copy()
        return c


def _init_block(d: int, nblk: int, rk: int, rnd: Counter) -> BlockTT:
    ranks = [1] + [min(rk, 4 ** min(k, d - k)) for k in range(1, d)] + [1]
    cores = [rnd.draw((ranks[k], 4, ranks[k + 1])) for k in range(d)]
    cores = tt.orth_right(cores)
    block = np.zeros((nblk,) + cores[0].shape)
    return BlockTT(cores=cores, block=block, pos=0)


def amen_solve(data: NewtonData, d: int, w0: BlockTT | None, tol: float, cap: int, kick: int,
               max_sweeps: int, rnd: Counter):
    """Block-AMEn solve of the Newton system. Returns (BlockTT, info dict)."""
    nblk = data.nblk
    if w0 is None:
        w = _init_block(d, nblk, kick, rnd)
    else:
        w = BlockTT([c.copy() for c in w0.cores], w0.block.copy(), w0.pos)
    assert w.pos == 0
    ops, rhs = _envs(data, d)
    envs = _all_envs(ops, rhs)
    # frame cores: at the block position use block 0's shape (the frame excludes it)
    frame = [c.copy() for c in w.cores]
    for k in range(d - 1, 0, -1):
        for e in envs:
            e.push_right(frame, k)
    info = {"sweeps": 0, "max_change": None, "ranks": None}
    block = w.block
    for sweep in range(max_sweeps):
        forward = sweep % 2 == 0
        order = range(d) if forward else range(d - 1, -1, -1)
        max_change = 0.0
        for k in order:
            K, b, r_d, (AT, AiT, n) = _local_system(ops, rhs, frame, k, data.sgn)
            sol = np.linalg.solve(K, b)
            dX, dY = sol[:n], sol[n:2 * n]
            if data.TA is None:
                dZ = AT @ dY - r_d
                new = np.stack([dX, dY, dZ])
            else:
                dT = sol[2 * n:3 * n]
                dZ = AT @ dY - data.sgn * (AiT @ dT) - r_d
                new = np.stack([dX, dY, dT, dZ])
            shape = frame[k].shape
            new = new.reshape((nblk,) + shape)
            nrm = np.linalg.norm(new)
            if block.shape == new.shape:
                max_change = max(max_change, np.linalg.norm(new - block) / max(nrm, 1e-300))
            else:
                max_change = max(max_change, 1.0)
            last = (k == d - 1) if forward else (k == 0)
            if last:
                block = new
                frame[k] = new[0]
                break
            rl, m, rr = shape
            if forward:
                mat = new.transpose(1, 2, 0, 3).reshape(rl * m, nblk * rr)
                u, s, vt = np.linalg.svd(mat, full_matrices=False)
                keep = _truncation_rank_rel(s, tol / math.sqrt(d), cap)
                u = u[:, :keep]
                extra = min(kick, rl * m - keep, max(cap - keep, 0))
                if extra > 0:
                    u = np.linalg.qr(np.concatenate([u, rnd.draw((rl * m, extra))], axis=1))[0]
                coef = u.T @ mat  # (r', nblk * rr)
                frame[k] = u.reshape(rl, m, -1)
                coef = coef.reshape(-1, nblk, rr)
                nxt = frame[k + 1]
                block = np.einsum("xbc,cjy->bxjy", coef, nxt)
                frame[k + 1] = block[0]
                for e in envs:
                    e.push_left(frame, k)
            else:
                mat = new.transpose(0, 1, 2, 3).reshape(nblk * rl, m * rr)
                u, s, vt = np.linalg.svd(mat, full_matrices=False)
                keep = _truncation_rank_rel(s, tol / math.sqrt(d), cap)
                v = vt[:keep].T  # (m * rr, r')
                extra = min(kick, m * rr - keep, max(cap - keep, 0))
                if extra > 0:
                    v = np.linalg.qr(np.concatenate([v, rnd.draw((m * rr, extra))], axis=1))[0]
                coef = mat @ v  # (nblk * rl, r')
                frame[k] = v.T.reshape(-1, m, rr)
                coef = coef.reshape(nblk, rl, -1)
                prv = frame[k - 1]
                block = np.einsum("xja,bac->bxjc", prv, coef)
                frame[k - 1] = block[0]
                for e in envs:
                    e.push_right(frame, k)
        info["sweeps"] = sweep + 1
        info["max_change"] = max_change
        if sweep >= 1 and max_change < tol:
            break
    # the solution, exact, with the block index where the last sweep left it
    pos = d - 1 if (info["sweeps"] % 2 == 1) else 0
    sol = BlockTT(cores=[c.copy() for c in frame], block=block, pos=pos)
    sol.cores[pos] = block[0]
    info["ranks"] = tt.ranks(sol.cores)
    # the warm start of the next solve has its block index at core 0: moving it
    # there is a sweep of block moves, truncated like the sweeps' moves (the
    # frame would otherwise grow to nblk times its rank)
    warm = sol
    if pos == d - 1:
        cores = [c.copy() for c in frame]
        for k in range(d - 1, 0, -1):
            rl, m, rr = block.shape[1:]
            mat = block.reshape(nblk * rl, m * rr)
            u, sv, vt = np.linalg.svd(mat, full_matrices=False)
            keep = _truncation_rank_rel(sv, tol / math.sqrt(d), cap)
            cores[k] = vt[:keep].reshape(keep, m, rr)
            coef = (u[:, :keep] * sv[:keep]).reshape(nblk, rl, keep)
            block = np.einsum("xja,bac->bxjc", cores[k - 1], coef)
        cores[0] = block[0]
        warm = BlockTT(cores=cores, block=block, pos=0)
    return sol, warm, info


# ----------------------------------------------------------------------------
# step length: extreme generalised Rayleigh quotient by one-site ALS (Section 3.4)
# ----------------------------------------------------------------------------


def _sym(a):
    return 0.5 * (a + a.T)


def min_gen_eig(M: list, dM: list, e0: list | None, rnd: Counter, rank: int = 4, sweeps: int = 4):
    """min over TT vectors e of <e, dM e> / <e, M e> (M psd TT matrix), by alternating local eigenproblems.

    Returns (lambda_min, e). The local problem at core k is the projected
    generalised eigenproblem (E^T dM E, E^T M E), reduced by a Cholesky factor of E^T M E.
    """
    d = len(M)
    n = M[0].shape[1]
    if e0 is None:
        ranks = [1] + [min(rank, n ** min(k, d - k)) for k in range(1, d)] + [1]
        e = [rnd.draw((ranks[k], n, ranks[k + 1])) for k in range(d)]
    else:
        e = [c.copy() for c in e0]
    e = tt.orth_right(e)
    envM = Env(M, None, d)
    envD = Env(dM, None, d)
    for k in range(d - 1, 0, -1):
        envM.push_right(e, k)
        envD.push_right(e, k)
    lam = math.inf
    for sweep in range(sweeps):
        forward = sweep % 2 == 0
        order = range(d) if forward else range(d - 1, -1, -1)
        for k in order:
            Mk = _sym(envM.local_mat(k))
            Dk = _sym(envD.local_mat(k))
            L = _cholesky(Mk)
            Li = np.linalg.inv(L)
            S = _sym(Li @ Dk @ Li.T)
            w_, v_ = np.linalg.eigh(S)
            lam = float(w_[0])
            x = Li.T @ v_[:, 0]
            shape = e[k].shape
            last = (k == d - 1) if forward else (k == 0)
            if last:
                e[k] = x.reshape(shape)
                break
            rl, m, rr = shape
            if forward:
                mat = x.reshape(rl * m, rr)
                q, r = np.linalg.qr(np.concatenate([mat, rnd.draw((rl * m, max(0, min(rank, rl * m) - 1)))], axis=1)
                                    if rank > 1 else mat)
                keep = min(q.shape[1], rank)
                q = q[:, :keep]
                e[k] = q.reshape(rl, m, keep)
                coef = q.T @ mat
                e[k + 1] = np.einsum("ab,bjc->ajc", coef, e[k + 1])
                envM.push_left(e, k)
                envD.push_left(e, k)
            else:
                mat = x.reshape(rl, m * rr)
                q, r = np.linalg.qr(np.concatenate([mat.T, rnd.draw((m * rr, max(0, min(rank, m * rr) - 1)))], axis=1)
                                    if rank > 1 else mat.T)
                keep = min(q.shape[1], rank)
                q = q[:, :keep]
                e[k] = q.T.reshape(keep, m, rr)
                coef = mat @ q
                e[k - 1] = np.einsum("xja,ab->xjb", e[k - 1], coef)
                envM.push_right(e, k)
                envD.push_right(e, k)
    e = tt.orth_right(e)
    return lam, e


def merge_op_cores(op: list, k: int) -> np.ndarray:
    """Operator cores k and k+1 as one core with grouped modes [p][(i1 i2)][(j1 j2)][q]
    (the two-site operator of a DMRG step, Section 3.4)."""
    a, b = op[k], op[k + 1]
    R, m1, n1, _ = a.shape
    _, m2, n2, R2 = b.shape
    c = np.tensordot(a, b, axes=([3], [0]))  # p i1 j1 i2 j2 q
    return c.transpose(0, 1, 3, 2, 4, 5).reshape(R, m1 * m2, n1 * n2, R2)


class NotPositiveDefinite(ArithmeticError):
    """The iterate handed to the step-length eigenproblem is not positive definite (Section 3.4)."""


def _cholesky(Mk: np.ndarray) -> np.ndarray:
    try:
        return np.linalg.cholesky(Mk)
    except np.linalg.LinAlgError as e:
        raise NotPositiveDefinite("step length: the projected iterate is not positive definite") from e


def _local_gen_eig(Mk: np.ndarray, Dk: np.ndarray):
    """Smallest eigenpair of Dk x = lam Mk x (Mk spd) through the Cholesky reduction."""
    L = _cholesky(Mk)
    Li = np.linalg.inv(L)
    S = _sym(Li @ Dk @ Li.T)
    w_, v_ = np.linalg.eigh(S)
    return float(w_[0]), Li.T @ v_[:, 0]


def dmrg_keep(s: np.ndarray, tol: float, cap: int) -> int:
    """Smallest rank whose discarded tail energy is at most tol^2 of the total, in [1, cap]."""
    tot = float(np.sum(s * s))
    keep = len(s)
    tail = 0.0
    while keep > 1 and tail + s[keep - 1] ** 2 <= tol * tol * tot:
        tail += s[keep - 1] ** 2
        keep -= 1
    return max(1, min(keep, cap))


def min_gen_eig_dmrg(M: list, dM: list, e0: list | None, rnd: Counter, rank: int = 4, sweeps: int = 4,
                     tol: float = 1e-8, stall: float = 0.0):
    """min over TT vectors e of <e, dM e> / <e, M e> by two-site (DMRG) sweeps (Section 3.4).

    The unknown at bond (k, k+1) is the supercore of cores k and k+1; its
    projected generalised eigenproblem (with the merged operator cores) is
    solved by the Cholesky reduction, and the supercore is split by a truncated
    SVD (relative tolerance tol, at most `rank`). The orthonormal factor is then
    enriched with random columns up to `rank` (the kick) and re-orthonormalised
    by QR; the other factor is the projection of the supercore onto it.
    Returns (lambda_min, e).
    """
    d = len(M)
    if d < 2:
        return min_gen_eig(M, dM, e0, rnd, rank, sweeps)
    n = M[0].shape[1]
    if e0 is None:
        ranks = [1] + [min(rank, n ** min(k, d - k)) for k in range(1, d)] + [1]
        e = [rnd.draw((ranks[k], n, ranks[k + 1])) for k in range(d)]
    else:
        e = [c.copy() for c in e0]
    e = tt.orth_right(e)
    envM = Env(M, None, d)
    envD = Env(dM, None, d)
    for k in range(d - 1, 1, -1):
        envM.push_right(e, k)
        envD.push_right(e, k)
    Mm = [merge_op_cores(M, k) for k in range(d - 1)]
    Dm = [merge_op_cores(dM, k) for k in range(d - 1)]
    lam = math.inf
    for sweep in range(sweeps):
        # stop once the quotient of a full sweep has stalled (after two sweeps)
        if sweep >= 2 and stall > 0.0 and abs(lam - lam_prev) <= stall * abs(lam):
            break
        lam_prev = lam
        forward = sweep % 2 == 0
        bonds = range(d - 1) if forward else range(d - 2, -1, -1)
        for k in bonds:
            Mk = _sym(tt.local_matrix(envM.left[k], Mm[k], envM.right[k + 2]))
            Dk = _sym(tt.local_matrix(envD.left[k], Dm[k], envD.right[k + 2]))
            lam, x = _local_gen_eig(Mk, Dk)
            rl, rr = e[k].shape[0], e[k + 1].shape[2]
            mat = x.reshape(rl * n, n * rr)
            U, sv, Vt = np.linalg.svd(mat, full_matrices=False)
            keep = dmrg_keep(sv, tol, rank)
            if forward:
                left = U[:, :keep]
                extra = min(rank, rl * n, n * rr) - keep
                if extra > 0:
                    q, _ = np.linalg.qr(np.concatenate([left, rnd.draw((rl * n, extra))], axis=1))
                    left = q[:, :keep + extra]
                e[k] = left.reshape(rl, n, left.shape[1])
                e[k + 1] = (left.T @ mat).reshape(left.shape[1], n, rr)
                envM.push_left(e, k)
                envD.push_left(e, k)
            else:
                right = Vt[:keep].T  # (n rr) x keep, orthonormal columns
                extra = min(rank, rl * n, n * rr) - keep
                if extra > 0:
                    q, _ = np.linalg.qr(np.concatenate([right, rnd.draw((n * rr, extra))], axis=1))
                    right = q[:, :keep + extra]
                e[k + 1] = right.T.reshape(right.shape[1], n, rr)
                e[k] = (mat @ right).reshape(rl, n, right.shape[1])
                envM.push_right(e, k + 1)
                envD.push_right(e, k + 1)
    e = tt.orth_right(e)
    return lam, e


def step_from_lambda(lam: float) -> float:
    """Theorem "Optimal Step Size": alpha = -1/lambda_min(M^-1/2 dM M^-1/2) when negative, else unbounded."""
    return math.inf if lam >= 0 else -1.0 / lam


# ----------------------------------------------------------------------------
# the IPM
# ----------------------------------------------------------------------------


@dataclass
class Options:
    eps_gap: float = 1e-4
    rank_cap: int = 16
    xz_warmup: int = 3
    eta0: float = 1e-3
    eta_floor: float = 1e-4
    eta_C: float = 2.0
    damping: float = 0.95
    max_iters: int = 60
    max_sweeps: int = 4
    kick: int = 4
    seed: int = 1234
    eig_rank: int = 4
    eig_sweeps: int = 4
    eig_two_site: bool = True   # two-site DMRG sweeps (Section 3.4); False: one-site ALS
    eig_stall: float = 1e-9     # two-site sweeps stop once a sweep changes the quotient by less (relative)
    max_retries: int = 4        # damp-and-retry of an update that left the cone (Section 3.5)
    combined_multipliers: bool = True  # one block dLambda for dY and dT when their masks are disjoint (Section 3.5)
    # finishing phase (Section 3.5, "Relaxing the Positive Definiteness Barrier"): after
    # the relative criteria hold, iterate on with step lengths for M + nu I >= 0 until
    # ||R_p||_F, ||R_d||_F and the complementarity are below finish_tol (0: off)
    finish_tol: float = 0.0
    nu0: float = 1e-6
    nu_max: float = 1e-3
    fallback_step: float = 1e-3  # AHO -> XZ fallback below this step length (Section 3.5)


@dataclass
class IterInfo:
    it: int
    mu: float
    rel_p: float
    rel_d: float
    rel_gap: float
    pobj: float
    dobj: float
    alpha_p: float = 0.0
    alpha_d: float = 0.0
    direction: str = ""
    finishing: bool = False   # an iteration of the finishing phase
    accepted: bool = True     # its update reduced the merit (finishing phase)
    nu: float = 0.0           # barrier relaxation of its step lengths
    merit: float = 0.0        # merit of the iterate it started from (finishing phase)
    ranks_X: list = field(default_factory=list)
    ranks_Z: list = field(default_factory=list)
    ranks_W: list = field(default_factory=list)   # frame kept as the next solve's warm start
    sweeps: int = 0


def _round_psd(cores: list, delta: float, cap: int, shift: list | None):
    """TT rounding with the spectral shift of Corollary psdness_rounding.

    Rounds the vec_TT form at delta / (1 + ||S||_F), then adds zeta S. If the
    rank does not drop, the unrounded tensor is kept.
    """
    v = tt.vec_tt(cores)
    sn = tt.norm(tt.vec_tt(shift)) if shift is not None else 0.0
    rv, zeta, _ = tt.round_tt(v, delta / (1.0 + sn), cap)
    rounded = tt.unvec_tt(rv)
    if shift is not None and zeta > 0:
        rounded = tt.add(rounded, shift, 1.0, zeta)
    if max(tt.ranks(rounded)) >= max(tt.ranks(cores)) and max(tt.ranks(cores)) <= cap:
        return [c.copy() for c in cores], 0.0
    return rounded, zeta


def _sym_tt(m: list) -> list:
    return tt.add(m, tt.transpose(m), 0.5, 0.5)


class TTIPM:
    """State and iteration of the TT IPM on one problem."""

    def __init__(self, prob: TTProblem, opts: Options):
        self.p = prob
        self.o = opts
        d = prob.d
        self.d = d
        self.N = 2**d
        self.rnd = Counter(opts.seed)
        I = tt.identity(d)
        self.I = I
        lam = prob.lam0
        self.Z = tt.scale(I, lam)
        self.Y = [np.zeros((1, 2, 2, 1)) for _ in range(d)]
        self.T = None
        if prob.A_ineq is not None:
            # X = lam I + (alpha_p / 10) A_ineq(J), T = lam_ineq A_ineq(J) (Section 5.1)
            aJ = prob.ones_t
            lam_min, _ = self._gen_eig(I, aJ, None, 2, 6)
            alpha_p = lam * step_from_lambda(lam_min) if lam_min < 0 else lam
            self.X = tt.add(tt.scale(I, lam), aJ, 1.0, alpha_p / 10.0)
            self.T = tt.scale(aJ, prob.lam0_ineq)
        else:
            self.X = tt.scale(I, lam)
        self.eta = opts.eta0
        self.nB = tt.norm(prob.B_eq)
        self.nC = tt.norm(tt.vec_tt(prob.C))
        self.w = None
        self.eX = self.eZ = self.eT = self.eS = None
        self.history = []
        self.prev = None      # last update: iterate, direction, step lengths, rounding tolerances
        self.retries = 0
        self.nu = 0.0            # relaxation M + nu I >= 0 of the step lengths (finishing phase)
        self.finish_done = False
        self.fallbacks = 0

    # --- residuals and measures (Section 3.3, Section 3.5) ---
    def slack(self, X):
        """s_ineq(X) = A_ineq vec X - B_ineq (lower bound convention of Section 4.3), as a TT vector."""
        p = self.p
        return tt.add(tt.matvec(p.A_ineq, tt.vec_tt(X)), p.B_ineq, p.ineq_sign, -p.ineq_sign)

    def residual_d(self):
        p = self.p
        r = tt.add(tt.add(tt.vec_tt(self.Z), tt.vec_tt(p.C)), tt.matvec(tt.transpose(p.A_eq), tt.vec_tt(self.Y)), 1.0, -1.0)
        if self.T is not None:
            r = tt.add(r, tt.matvec(tt.transpose(p.A_ineq), tt.vec_tt(self.T)), 1.0, p.ineq_sign)
        return r

    def residual_p(self):
        p = self.p
        return tt.add(p.B_eq, tt.matvec(p.A_eq, tt.vec_tt(self.X)), 1.0, -1.0)

    def mu(self):
        val = tt.inner(tt.vec_tt(self.Z), tt.vec_tt(self.X))
        if self.T is not None:
            val += tt.inner(tt.vec_tt(self.T), self.slack(self.X))
        return val / (self.N + self.p.q)

    def measures(self):
        p = self.p
        rp = tt.norm(self.residual_p())
        rd = tt.norm(self.residual_d())
        comp = tt.inner(tt.vec_tt(self.Z), tt.vec_tt(self.X))
        if self.T is not None:
            comp += tt.inner(tt.vec_tt(self.T), self.slack(self.X))
        pobj = tt.inner(tt.vec_tt(p.C), tt.vec_tt(self.X))
        dobj = tt.inner(p.B_eq, tt.vec_tt(self.Y))
        if self.T is not None:
            dobj -= p.ineq_sign * tt.inner(p.B_ineq, tt.vec_tt(self.T))
        rel_p = rp / (1.0 + self.nB)
        rel_d = rd / (1.0 + self.nC)
        rel_gap = comp / ((self.N + p.q) * (1.0 + abs(pobj)))
        return rel_p, rel_d, rel_gap, pobj, dobj

    # --- the Newton system ---
    def newton_data(self, direction: str, sigma_mu: float, corr, zero_p: bool, zero_d: bool) -> NewtonData:
        p = self.p
        d = self.d
        X, Z = self.X, self.Z
        vI = tt.vec_tt(self.I)
        idop = op_identity(d)
        if direction == "aho":
            LZ = [op_kron_right(Z), op_kron_left(Z)]
            LX = [op_kron_right(X), op_kron_left(X)]
            rhs_c = [(1.0, op_kron_right(Z), tt.vec_tt(X)), (1.0, op_kron_left(Z), tt.vec_tt(X)),
                     (-2.0 * sigma_mu, idop, vI)]
        else:
            LZ = [op_kron_left(Z)]
            LX = [op_kron_right(X)]
            rhs_c = [(1.0, op_kron_left(Z), tt.vec_tt(X)), (-sigma_mu, idop, vI)]
        if corr is not None:
            dXa, dZa = corr[0], corr[1]
            if direction == "aho":
                # vec(dX dZ + dZ dX) = (I kron dZ^T) vec dX + (dZ kron I) vec dX
                rhs_c += [(1.0, op_kron_right(tt.transpose(dZa)), tt.vec_tt(dXa)),
                          (1.0, op_kron_left(dZa), tt.vec_tt(dXa))]
            else:
                rhs_c += [(1.0, op_kron_left(dZa), tt.vec_tt(dXa))]
        rhs_p = [] if zero_p else [(1.0, idop, p.B_eq), (-1.0, p.A_eq, tt.vec_tt(X))]
        rhs_d = [] if zero_d else [(1.0, idop, tt.vec_tt(Z)), (1.0, idop, tt.vec_tt(p.C)),
                                   (-1.0, tt.transpose(p.A_eq), tt.vec_tt(self.Y))]
        if not zero_d and self.T is not None:
            rhs_d.append((p.ineq_sign, tt.transpose(p.A_ineq), tt.vec_tt(self.T)))
        if not rhs_p:
            rhs_p = [(0.0, idop, vI)]
        if not rhs_d:
            rhs_d = [(0.0, idop, vI)]
        data = NewtonData(A_eq=p.A_eq, A_eqT=tt.transpose(p.A_eq), K_y=p.K_y, LZ=LZ, LX=LX,
                          rhs_p=rhs_p, rhs_d=rhs_d, rhs_c=rhs_c)
        if self.T is not None:
            vT = tt.vec_tt(self.T)
            vG = tt.vec_tt(p.ones_t)
            TA = tt.diag_tt(tt.hadamard(vT, vG))
            s = self.slack(X)
            data.TA = TA
            data.D_K = [tt.diag_tt(s), p.K_t]
            data.A_ineqT = tt.transpose(p.A_ineq)
            data.sgn = p.ineq_sign
            ones_t = tt.vec_tt(p.ones_t)
            # R_t = vec T . s - sigma mu vec 1_T  (+ dT_a . ds_a in the corrector)
            data.rhs_t = [(1.0, tt.diag_tt(vT), s), (-sigma_mu, idop, ones_t)]
            if corr is not None and len(corr) > 2:
                dTa, dsa = corr[2], corr[3]
                data.rhs_t.append((1.0, tt.diag_tt(tt.vec_tt(dTa)), dsa))
        return data

    def combine_multipliers(self, data: NewtonData) -> NewtonData:
        """Combined multiplier storage (Section 3.5, "Combined Multiplier Storage").

        With the non-idle masks P_Y = I - K_Y and P_T = I - K_T disjoint, dY and
        dT are kept in one block dLambda (dY = P_Y dLambda, dT = P_T dLambda).
        The multiplier rows become P_Y (p-row) + P_T (t-row):
            (-P_Y A_eq + sgn P_T T A_ineq) dX + (P_Y K_Y P_Y + P_T (D_ineq + K_T) P_T) dLambda
                = -(P_Y R_p + P_T R_t),
        the multiplier column of the dZ equation becomes A_eq^T P_Y - sgn A_ineq^T P_T,
        and the dX and dZ equations are otherwise unchanged. All operators here
        are diag_TT of vectors, so products are Hadamard products of their
        diagonals, and for 0/1 masks P D P = P D. Returns `data` itself when the
        masks overlap."""
        p, d = self.p, self.d
        one = _ones4(d)
        pY = tt.add(one, op_diagonal(p.K_y), 1.0, -1.0)
        pT = tt.add(one, op_diagonal(p.K_t), 1.0, -1.0)
        if abs(tt.inner(pY, pT)) > 1e-9:
            return data
        sg = data.sgn
        a_eq, a_in = op_diagonal(p.A_eq), op_diagonal(p.A_ineq)
        row = tt.add(tt.hadamard(pY, a_eq), tt.hadamard(pT, op_diagonal(data.TA)), 1.0, -sg)
        dk = op_diagonal(data.D_K[0])
        for o in data.D_K[1:]:
            dk = tt.add(dk, op_diagonal(o))
        lam = tt.add(tt.hadamard(pY, op_diagonal(p.K_y)), tt.hadamard(pT, dk))
        col = tt.add(tt.hadamard(pY, a_eq), tt.hadamard(pT, a_in), 1.0, -sg)
        rhs = [(c, tt.diag_tt(tt.hadamard(pY, op_diagonal(o))), v) for c, o, v in data.rhs_p]
        rhs += [(c, tt.diag_tt(tt.hadamard(pT, op_diagonal(o))), v) for c, o, v in data.rhs_t]
        return NewtonData(A_eq=tt.diag_tt(row), A_eqT=tt.diag_tt(col), K_y=tt.diag_tt(lam), LZ=data.LZ, LX=data.LX,
                          rhs_p=rhs, rhs_d=data.rhs_d, rhs_c=data.rhs_c, sgn=sg, masks=(pY, pT))

    def direction(self, direction, sigma_mu, corr, zero_p, zero_d):
        data = self.newton_data(direction, sigma_mu, corr, zero_p, zero_d)
        if data.TA is not None and self.o.combined_multipliers:
            data = self.combine_multipliers(data)
        w, warm, info = amen_solve(data, self.d, self.w, self.eta, self.o.rank_cap, self.o.kick,
                             self.o.max_sweeps, self.rnd)
        self.w = warm
        comps = [tt.unvec_tt(w.component(b)) for b in range(data.nblk)]
        if data.masks is not None:
            dX, dL, dZ = comps
            pY, pT = data.masks
            dY = tt.unvec_tt(tt.hadamard(tt.vec_tt(dL), pY))
            dT = tt.unvec_tt(tt.hadamard(tt.vec_tt(dL), pT))
        elif data.nblk == 3:
            dX, dY, dZ = comps
            dT = None
        else:
            dX, dY, dT, dZ = comps
        if direction == "xz":
            # the XZ linearisation is unsymmetric; every block is symmetrised so
            # that mirrored multipliers stay mirrored and dZ = A^T dY - ... - R_d holds
            dX, dY, dZ = _sym_tt(dX), _sym_tt(dY), _sym_tt(dZ)
            if dT is not None:
                dT = _sym_tt(dT)
        return dX, dY, dT, dZ, info

    def steps(self, dX, dT, dZ):
        a_p, self.eX = self._max_step(self.X, dX, self.eX)
        a_d, self.eZ = self._max_step(self.Z, dZ, self.eZ)
        if self.T is not None:
            # diagonal cases: slack and multiplier on the active mask
            ds = tt.matvec(self.p.A_ineq, tt.vec_tt(dX))
            s = self.slack(self.X)
            a_s, self.eS = self._max_step_diag(s, ds, self.eS)
            a_t, self.eT = self._max_step_diag(tt.vec_tt(self.T), tt.vec_tt(dT), self.eT)
            a_p, a_d = min(a_p, a_s), min(a_d, a_t)
        return min(1.0, self.o.damping * a_p), min(1.0, self.o.damping * a_d)

    def _gen_eig(self, M, dM, e0, rank, sweeps):
        # the eigensolver's random starts and kicks come from a sub-stream, so
        # how many sweeps it runs does not move the main stream
        sub = self.rnd.fork()
        if self.o.eig_two_site:
            return min_gen_eig_dmrg(M, dM, e0, sub, rank, sweeps, stall=self.o.eig_stall)
        return min_gen_eig(M, dM, e0, sub, rank, sweeps)

    def _max_step(self, M, dM, e0):
        if self.nu > 0.0:
            M = tt.add(M, self.I, 1.0, self.nu)
        lam, e = self._gen_eig(M, _sym_tt(dM), e0, self.o.eig_rank, self.o.eig_sweeps)
        return step_from_lambda(lam), e

    def _max_step_diag(self, v, dv, e0):
        # positivity of a TT vector restricted to the inequality mask: the
        # diagonal matrices diag_TT(v + mask_idle) and diag_TT(dv)
        p = self.p
        idle = tt.add(tt.vec_tt(tt.ones_mat(self.d)), tt.vec_tt(p.ones_t), 1.0, -1.0)
        M = tt.diag_tt(tt.add(v, idle))
        if self.nu > 0.0:
            M = tt.add(M, tt.diag_tt(tt.vec_tt(p.ones_t)), 1.0, self.nu)
        lam, e = self._gen_eig(M, tt.diag_tt(dv), e0, 1, self.o.eig_sweeps)
        return step_from_lambda(lam), e

    def _apply_update(self):
        """Algorithm 1's update from the stored iterate, direction and step lengths,
        rounded with the spectral shift (Corollary psdness_rounding)."""
        u, cap = self.prev, self.o.rank_cap
        self.X, _ = _round_psd(tt.add(u["X"], u["dX"], 1.0, u["ap"]), u["tol_p"], cap, self.I)
        self.Z, _ = _round_psd(tt.add(u["Z"], u["dZ"], 1.0, u["ad"]), u["tol_d"], cap, self.I)
        self.Y, _ = _round_psd(tt.add(u["Y"], u["dY"], 1.0, u["ad"]), u["tol_d"], cap, None)
        if u["T"] is not None:
            self.T, _ = _round_psd(tt.add(u["T"], u["dT"], 1.0, u["ad"]), u["tol_d"], cap, self.p.ones_t)

    def iterate(self, it: int) -> IterInfo | None:
        """One iteration; an update that the next step-length solve finds outside
        the cone is undone and repeated with both step lengths halved (the
        damp-and-retry safeguard of Section 3.5), at most max_retries times."""
        for attempt in range(self.o.max_retries + 1):
            try:
                return self._iterate_once(it)
            except NotPositiveDefinite:
                if self.prev is None or attempt == self.o.max_retries:
                    raise
                self.history.pop()
                self.prev["ap"] *= 0.5
                self.prev["ad"] *= 0.5
                self._apply_update()
                self.retries += 1
        raise AssertionError("unreachable")

    def _iterate_once(self, it: int) -> IterInfo | None:
        o, p = self.o, self.p
        rel_p, rel_d, rel_gap, pobj, dobj = self.measures()
        mu = self.mu()
        eps_p = eps_d = 2.0 * o.eps_gap
        eps_c = o.eps_gap / math.sqrt(self.d)
        info = IterInfo(it, mu, rel_p, rel_d, rel_gap, pobj, dobj)
        self.history.append(info)
        rel_ok = rel_p <= eps_p and rel_d <= eps_d and rel_gap <= eps_c
        if rel_ok and (o.finish_tol <= 0.0 or self.finish_done):
            return None
        if rel_ok:
            merit, done = self.finish_merit()
            if done:
                self.finish_done = True
                return None
            return self._finish_iteration(it, info, mu, merit)
        self.eta = max(min(self.eta, o.eta_C * mu), o.eta_floor)
        direction = "xz" if it < o.xz_warmup else "aho"
        zero_p = rel_p <= eps_p
        zero_d = rel_d <= eps_d
        dX, dY, dT, dZ, ap, ad, sweeps, amen_ok = self._mehrotra(direction, mu, zero_p, zero_d)
        if direction == "aho" and (min(ap, ad) < o.fallback_step or not amen_ok):
            # Section 3.5: an AHO solve that misses its target within the rank and
            # sweep budget, or whose admissible step is nearly zero, is redone
            # with the XZ direction for this iteration
            direction = "xz"
            self.fallbacks += 1
            dX, dY, dT, dZ, ap, ad, sweeps, amen_ok = self._mehrotra(direction, mu, zero_p, zero_d)
        info.alpha_p, info.alpha_d, info.direction, info.sweeps = ap, ad, direction, sweeps
        # update (Algorithm 1) and rounding with the spectral shift (Corollary psdness_rounding)
        tol_p = self.eta * (1.0 + self.nB) / 10.0
        tol_d = self.eta * (1.0 + self.nC) / 10.0
        self.prev = dict(X=self.X, Y=self.Y, T=self.T, Z=self.Z, dX=dX, dY=dY, dT=dT, dZ=dZ, ap=ap, ad=ad,
                         tol_p=tol_p, tol_d=tol_d)
        self._apply_update()
        info.ranks_X = tt.ranks(self.X)
        info.ranks_Z = tt.ranks(self.Z)
        info.ranks_W = tt.ranks(self.w.cores)
        return info

    def finish_merit(self):
        """Merit of the finishing phase and whether its absolute criteria hold:
        ||R_p||_F + ||R_d||_F + |<X, Z> + <vec T, s>| and each of the three
        below finish_tol (Section 3.5)."""
        rp = tt.norm(self.residual_p())
        rd = tt.norm(self.residual_d())
        comp = tt.inner(tt.vec_tt(self.Z), tt.vec_tt(self.X))
        if self.T is not None:
            comp += tt.inner(tt.vec_tt(self.T), self.slack(self.X))
        tol = self.o.finish_tol
        return rp + rd + abs(comp), (rp < tol and rd < tol and abs(comp) < tol)

    def _finish_iteration(self, it, info, mu, merit):
        """One iteration of the finishing phase: the Mehrotra direction without
        zeroed residual blocks, step lengths for the relaxed cone M + nu I >= 0,
        and the update kept only if the merit decreases while the relative
        criteria still hold; otherwise the previous iterate is retained and nu
        grows tenfold, up to nu_max (after which the phase ends)."""
        o = self.o
        if self.nu == 0.0:
            self.nu = o.nu0
        info.finishing, info.nu, info.merit = True, self.nu, merit
        self.eta = max(min(self.eta, o.eta_C * mu), o.eta_floor)
        direction = "xz" if it < o.xz_warmup else "aho"
        dX, dY, dT, dZ, ap, ad, sweeps, _ = self._mehrotra(direction, mu, False, False)
        info.alpha_p, info.alpha_d, info.direction, info.sweeps = ap, ad, direction, sweeps
        saved = (self.X, self.Y, self.T, self.Z)
        tol_p = self.eta * (1.0 + self.nB) / 10.0
        tol_d = self.eta * (1.0 + self.nC) / 10.0
        self.prev = dict(X=self.X, Y=self.Y, T=self.T, Z=self.Z, dX=dX, dY=dY, dT=dT, dZ=dZ, ap=ap, ad=ad,
                         tol_p=tol_p, tol_d=tol_d)
        self._apply_update()
        rel_p, rel_d, rel_gap, _, _ = self.measures()
        eps = 2.0 * o.eps_gap
        new_merit, _ = self.finish_merit()
        if rel_p <= eps and rel_d <= eps and rel_gap <= o.eps_gap / math.sqrt(self.d) and new_merit < merit:
            info.accepted = True
        else:
            info.accepted = False
            self.X, self.Y, self.T, self.Z = saved
            self.prev = None
            if self.nu >= o.nu_max:
                self.finish_done = True
            self.nu = min(10.0 * self.nu, o.nu_max)
        info.ranks_X = tt.ranks(self.X)
        info.ranks_Z = tt.ranks(self.Z)
        info.ranks_W = tt.ranks(self.w.cores)
        return info

    def _mehrotra(self, direction: str, mu: float, zero_p: bool, zero_d: bool):
        """Mehrotra predictor and corrector solves and their step lengths (Section 3.5).
        Returns the corrector direction, its step lengths, the AMEn sweeps of the
        corrector and whether both AMEn solves met their tolerance."""
        p = self.p
        # predictor
        dXa, dYa, dTa, dZa, pinfo = self.direction(direction, 0.0, None, zero_p, zero_d)
        ap, ad = self.steps(dXa, dTa, dZa)
        Xa = tt.add(self.X, dXa, 1.0, ap)
        Za = tt.add(self.Z, dZa, 1.0, ad)
        mu_aff = tt.inner(tt.vec_tt(Za), tt.vec_tt(Xa))
        if self.T is not None:
            Ta = tt.add(self.T, dTa, 1.0, ad)
            mu_aff += tt.inner(tt.vec_tt(Ta), self.slack(Xa))
        mu_aff /= (self.N + p.q)
        sigma = min(1.0, max(0.0, mu_aff / mu)) ** 3
        corr = (dXa, dZa)
        if self.T is not None:
            corr = (dXa, dZa, dTa, tt.matvec(p.A_ineq, tt.vec_tt(dXa)))
        dX, dY, dT, dZ, sinfo = self.direction(direction, sigma * mu, corr, zero_p, zero_d)
        ap, ad = self.steps(dX, dT, dZ)
        amen_ok = pinfo["max_change"] < self.eta and sinfo["max_change"] < self.eta
        return dX, dY, dT, dZ, ap, ad, sinfo["sweeps"], amen_ok

    def solve(self):
        for it in range(self.o.max_iters + 1):
            if self.iterate(it) is None:
                return True
        return False
