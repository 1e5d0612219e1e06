"""Seeded synthetic inputs for the tensor-train SDP interior-point method.

This module only draws graphs and weights. It holds none of the method's
arithmetic (no TT rounding, no operator assembly, no IPM step): both the
oracle and the CUDA path build everything else from what it returns, each
with its own code.

Workloads (all graphs on N = 2**d vertices, vertex u written big-endian in
d binary digits, digit 1 most significant, as in the paper's vectorisation
convention of Section 2.3):

* ``kron_patterns`` / ``maxcut_kron``: the Kronecker graph. For each of the d
  digits a symmetric 2x2 pattern B_k has entries p00, p01 = p10, p11 drawn
  U[0, 1] in that order and thresholded at 0.5 to {0, 1}. The adjacency is
  (B_1 kron ... kron B_d) with its diagonal zeroed; a draw without any edge is
  rejected and the next draw of the same stream is used.
* ``maxcut_kron_er``: the Kronecker graph OR-ed with an Erdos-Renyi graph
  (each unordered pair u < v independently with probability 2/N), every
  edge weighted U[0.5, 1.5], symmetric.
* ``theta_hypercube_kron``: the d-cube Q_d OR-ed with a Kronecker graph,
  accepted when the edge density lies in [0.8%, 1.5%].
* ``cc_signed``: complete signed graph. W = sign(M + M^T) off the diagonal
  (0 -> +1) for a rank-4 TT matrix M with N(0, 1) cores, then round(0.05 *
  N(N-1)/2) seeded pairs u < v have their sign flipped (mirrored).
* ``batch_maxcut``: many Kronecker Max-Cut instances with d drawn uniformly
  from a range.
* ``rank_controlled_graph``: the paper's instance family with a prescribed
  input TT rank r (Appendix A): a state in {0..r-1} is carried digit by digit;
  the first digit pair picks a state, every middle digit pair maps states to
  states (or drops them), the last digit pair names the state that makes the
  entry 1. Every choice is the same for the digit pairs (a, b) and (b, a), so
  the graph is undirected; on the middle digits' diagonal pairs (a, a) the
  states that diagonal paths can hold are dropped, so there are no loops.
  Draws whose TT rank is not exactly r, or without edges, are rejected.

Random streams come from numpy's Philox counter-based generator keyed by
(seed, stream id), so every workload is reproducible from its seed alone.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "rng",
    "kron_patterns",
    "kron_dense",
    "kron_adjacency_cores",
    "maxcut_kron",
    "rank_controlled_graph",
    "maxcut_kron_er",
    "theta_hypercube_kron",
    "cc_signed",
    "batch_maxcut",
    "random_tt",
    "random_tt_matrix",
]

# stream ids keep the draws of different workloads independent
_STREAM_KRON = 1
_STREAM_ER = 2
_STREAM_WEIGHT = 3
_STREAM_THETA = 4
_STREAM_CC = 5
_STREAM_CC_FLIP = 6
_STREAM_BATCH = 7
_STREAM_TT = 8
_STREAM_APPA = 9


def rng(seed: int, stream: int = 0) -> np.random.Generator:
    """Philox generator keyed by (seed, stream)."""
    return np.random.Generator(np.random.Philox(key=[int(seed) & (2**64 - 1), int(stream)]))


def _draw_patterns(g: np.random.Generator, d: int) -> np.ndarray:
    pats = np.zeros((d, 2, 2), dtype=np.int8)
    for k in range(d):
        p00, p01, p11 = g.uniform(0.0, 1.0, size=3)
        pats[k] = [[p00 > 0.5, p01 > 0.5], [p01 > 0.5, p11 > 0.5]]
    return pats


def kron_dense(pats: np.ndarray) -> np.ndarray:
    """Dense 0/1 adjacency (int8) of the Kronecker pattern graph, diagonal zeroed."""
    a = np.ones((1, 1), dtype=np.int8)
    for b in pats:
        a = np.kron(a, b.astype(np.int8))
    np.fill_diagonal(a, 0)
    return a


def _has_edge(pats: np.ndarray) -> bool:
    # an off-diagonal entry of the Kronecker product is 1 iff every pattern
    # has a 1 somewhere and at least one pattern has its off-diagonal 1
    if any(int(b.sum()) == 0 for b in pats):
        return False
    return any(int(b[0, 1]) == 1 for b in pats)


def kron_patterns(d: int, seed: int, stream: int = _STREAM_KRON) -> np.ndarray:
    """The d seeded 2x2 0/1 patterns of a Kronecker graph with at least one edge."""
    g = rng(seed, stream)
    while True:
        pats = _draw_patterns(g, d)
        if _has_edge(pats):
            return pats


def kron_adjacency_cores(pats: np.ndarray) -> list[np.ndarray]:
    """TT-matrix cores (r, 2, 2, r') of (kron_k B_k) - (kron_k diag(B_k)).

    The second term removes the diagonal of the first, so the result is the
    adjacency without self loops; its TT ranks are at most 2. The cores are
    the plain block construction of a sum of two Kronecker products.
    """
    d = len(pats)
    cores = []
    for k, b in enumerate(pats):
        bf = b.astype(np.float64)
        db = np.diag(np.diag(bf))
        if d == 1:
            cores.append((bf - db).reshape(1, 2, 2, 1))
        elif k == 0:
            c = np.zeros((1, 2, 2, 2))
            c[0, :, :, 0] = bf
            c[0, :, :, 1] = -db
            cores.append(c)
        elif k == d - 1:
            c = np.zeros((2, 2, 2, 1))
            c[0, :, :, 0] = bf
            c[1, :, :, 0] = db
            cores.append(c)
        else:
            c = np.zeros((2, 2, 2, 2))
            c[0, :, :, 0] = bf
            c[1, :, :, 1] = db
            cores.append(c)
    return cores


def maxcut_kron(d: int, seed: int) -> dict:
    """Unit-weight Max-Cut instance on a seeded Kronecker graph."""
    pats = kron_patterns(d, seed)
    adj = kron_dense(pats)
    return {
        "kind": "maxcut",
        "d": d,
        "seed": seed,
        "patterns": pats,
        "adjacency": adj,
        "weights": adj.astype(np.float64),
        "adjacency_cores": kron_adjacency_cores(pats),
    }


def maxcut_kron_er(d: int, seed: int, p_scale: float = 2.0) -> dict:
    """Kronecker graph OR Erdos-Renyi(p_scale / N), weights U[0.5, 1.5]."""
    n = 2**d
    pats = kron_patterns(d, seed)
    adj = kron_dense(pats).astype(bool)
    g = rng(seed, _STREAM_ER)
    er = np.triu(g.random((n, n)) < (p_scale / n), k=1)
    adj |= er | er.T
    np.fill_diagonal(adj, False)
    gw = rng(seed, _STREAM_WEIGHT)
    w = np.triu(gw.uniform(0.5, 1.5, size=(n, n)), k=1)
    w = w + w.T
    weights = np.where(adj, w, 0.0)
    return {
        "kind": "maxcut",
        "d": d,
        "seed": seed,
        "patterns": pats,
        "adjacency": adj.astype(np.int8),
        "weights": weights,
        "adjacency_cores": None,
    }


def hypercube_dense(d: int) -> np.ndarray:
    n = 2**d
    u = np.arange(n)
    x = u[:, None] ^ u[None, :]
    return ((x > 0) & ((x & (x - 1)) == 0)).astype(np.int8)


def theta_hypercube_kron(d: int, seed: int, lo: float = 0.008, hi: float = 0.015) -> dict:
    """Lovasz-theta instance: Q_d OR a Kronecker graph with density in [lo, hi]."""
    n = 2**d
    q = hypercube_dense(d).astype(bool)
    g_stream = 0
    while True:
        pats = kron_patterns(d, seed, stream=_STREAM_THETA * 1000 + g_stream)
        adj = q | kron_dense(pats).astype(bool)
        np.fill_diagonal(adj, False)
        dens = adj.sum() / (n * (n - 1))
        # below d = 10 the cube alone is denser than the window: take the first draw
        if lo <= dens <= hi or d < 6 or d / (n - 1) > hi:
            break
        g_stream += 1
    return {
        "kind": "theta",
        "d": d,
        "seed": seed,
        "patterns": pats,
        "adjacency": adj.astype(np.int8),
        "weights": adj.astype(np.float64),
        "adjacency_cores": None,
        "density": float(dens),
    }


def random_tt(dims: list[int], ranks: list[int], seed: int, stream: int = _STREAM_TT) -> list[np.ndarray]:
    """TT-vector cores (r_k, n_k, r_k+1) with N(0, 1) entries."""
    g = rng(seed, stream)
    return [g.standard_normal((ranks[k], dims[k], ranks[k + 1])) for k in range(len(dims))]


def random_tt_matrix(rows: list[int], cols: list[int], ranks: list[int], seed: int,
                     stream: int = _STREAM_TT) -> list[np.ndarray]:
    """TT-matrix cores (r_k, m_k, n_k, r_k+1) with N(0, 1) entries."""
    g = rng(seed, stream)
    return [g.standard_normal((ranks[k], rows[k], cols[k], ranks[k + 1])) for k in range(len(rows))]


def _tt_matrix_dense(cores: list[np.ndarray]) -> np.ndarray:
    # plain reconstruction used only to draw the sign pattern of cc_signed
    full = np.ones((1, 1, 1))
    for c in cores:
        r, m, n, r2 = c.shape
        full = np.einsum("xya,aijb->xiyjb", full, c)
        full = full.reshape(full.shape[0] * m, full.shape[2] * n, r2)
    return full[:, :, 0]


def cc_signed(d: int, seed: int, flip_frac: float = 0.05) -> dict:
    """Correlation-clustering instance on the complete signed graph."""
    n = 2**d
    ranks = [1] + [4] * (d - 1) + [1]
    m = _tt_matrix_dense(random_tt_matrix([2] * d, [2] * d, ranks, seed, stream=_STREAM_CC))
    s = m + m.T
    w = np.where(s >= 0.0, 1.0, -1.0)
    iu, ju = np.triu_indices(n, k=1)
    nflip = int(round(flip_frac * len(iu)))
    g = rng(seed, _STREAM_CC_FLIP)
    pick = g.choice(len(iu), size=nflip, replace=False)
    w[iu[pick], ju[pick]] *= -1.0
    w[ju[pick], iu[pick]] *= -1.0
    np.fill_diagonal(w, 0.0)
    adj = np.ones((n, n), dtype=np.int8)
    np.fill_diagonal(adj, 0)
    return {
        "kind": "cc",
        "d": d,
        "seed": seed,
        "adjacency": adj,
        "weights": w,
        "c_plus": np.where(w > 0, w, 0.0),
        "c_minus": np.where(w < 0, -w, 0.0),
        "adjacency_cores": None,
    }


def cc_signed_sub(d_full: int, d_sub: int, seed: int, flip_frac: float = 0.05) -> dict:
    """Principal sub-instance of the correlation-clustering instance of order
    d_full: the rows and columns whose d_full - d_sub most significant binary
    digits are 0 (the leading 2^d_sub x 2^d_sub block), a complete signed
    graph of order d_sub in the same vertex numbering."""
    full = cc_signed(d_full, seed, flip_frac)
    n = 2**d_sub
    w = full["weights"][:n, :n].copy()
    adj = np.ones((n, n), dtype=np.int8)
    np.fill_diagonal(adj, 0)
    return {
        "kind": "cc",
        "d": d_sub,
        "d_full": d_full,
        "seed": seed,
        "adjacency": adj,
        "weights": w,
        "c_plus": np.where(w > 0, w, 0.0),
        "c_minus": np.where(w < 0, -w, 0.0),
        "adjacency_cores": None,
    }


def batch_maxcut(count: int, seed: int, d_lo: int = 6, d_hi: int = 11) -> list[dict]:
    """`count` Kronecker Max-Cut instances with d ~ U{d_lo..d_hi}."""
    g = rng(seed, _STREAM_BATCH)
    ds = g.integers(d_lo, d_hi + 1, size=count)
    return [maxcut_kron(int(dd), seed * 100003 + i) for i, dd in enumerate(ds)]


def _tt_unfolding_ranks(adj: np.ndarray, d: int) -> list[int]:
    """Ranks of the unfoldings of the 2 x 2-mode TT matrix of adj (bond k splits
    the digit pairs 1..k from k+1..d), from the plain definition."""
    t = adj.reshape([2] * d + [2] * d)
    # interleave (row digit k, column digit k)
    order = [x for k in range(d) for x in (k, d + k)]
    t = np.transpose(t, order)
    out = []
    for k in range(1, d):
        out.append(int(np.linalg.matrix_rank(t.reshape(4 ** k, 4 ** (d - k)).astype(np.float64))))
    return out


def rank_controlled_graph(d: int, r: int, seed: int, stay: float = 0.5, max_draws: int = 500) -> dict:
    """Undirected graph without loops on 2**d vertices whose adjacency has TT
    rank exactly r (2 x 2 modes), drawn by the construction described in the
    module docstring. `stay` is the probability that a middle digit pair keeps
    a state unchanged (larger: denser graphs). Also returns the exact TT
    cores (bond dimension r) of the adjacency."""
    assert d >= 3 and r >= 1
    g = rng(seed, _STREAM_APPA)
    n = 2 ** d
    pairs = [(0, 0), (0, 1), (1, 1)]
    for _ in range(max_draws):
        first = np.zeros((2, 2), dtype=np.int64)
        last = np.zeros((2, 2), dtype=np.int64)
        maps = np.zeros((d - 2, 2, 2, r), dtype=np.int64)  # -1: the state is dropped
        for a, b in pairs:
            first[a, b] = first[b, a] = g.integers(r)
        reach = {int(first[0, 0]), int(first[1, 1])}  # states of diagonal paths
        for k in range(d - 2):
            for a, b in pairs:
                m = np.where(g.random(r) < stay, np.arange(r), g.integers(r, size=r))
                if a == b:
                    m[list(reach)] = -1
                maps[k, a, b] = maps[k, b, a] = m
            reach = set()  # every diagonal path is dropped at the first middle digit
        for a, b in pairs:
            last[a, b] = last[b, a] = g.integers(r)
        # entry (u, v): carry the state through the digits of u and v
        digits = (np.arange(n)[:, None] >> np.arange(d - 1, -1, -1)[None, :]) & 1  # (n, d), digit 1 first
        du = digits[:, None, :]
        dv = digits[None, :, :]
        state = np.broadcast_to(first[du[..., 0], dv[..., 0]], (n, n)).copy()
        for k in range(d - 2):
            mk = maps[k][du[..., k + 1], dv[..., k + 1]]  # (n, n, r)
            alive = state >= 0
            nxt = np.full_like(state, -1)
            idx = np.where(alive)
            nxt[idx] = mk[idx[0], idx[1], state[idx]]
            state = nxt
        adj = (state == last[du[..., d - 1], dv[..., d - 1]]).astype(np.int8)
        if adj.sum() == 0 or np.any(np.diag(adj)) or max(_tt_unfolding_ranks(adj, d)) != r:
            continue
        # exact TT cores (1 x 2 x 2 x r, r x 2 x 2 x r, r x 2 x 2 x 1)
        cores = []
        c = np.zeros((1, 2, 2, r))
        for a in range(2):
            for b in range(2):
                c[0, a, b, first[a, b]] = 1.0
        cores.append(c)
        for k in range(d - 2):
            c = np.zeros((r, 2, 2, r))
            for a in range(2):
                for b in range(2):
                    for i in range(r):
                        if maps[k, a, b, i] >= 0:
                            c[i, a, b, maps[k, a, b, i]] = 1.0
            cores.append(c)
        c = np.zeros((r, 2, 2, 1))
        for a in range(2):
            for b in range(2):
                c[last[a, b], a, b, 0] = 1.0
        cores.append(c)
        return {
            "kind": "maxcut",
            "d": d,
            "seed": seed,
            "r_in": r,
            "adjacency": adj,
            "weights": adj.astype(np.float64),
            "adjacency_cores": cores,
        }
    raise RuntimeError(f"no graph of TT rank {r} at d = {d} in {max_draws} draws")

