"""The remaining calls of the C ABI against the oracle: tt_sdp_round (TT rounding
plus the spectral shift of Section 3.4, Corollary psdness_rounding) on host
data, tt_sdp_create with a caller allocator, and tt_sdp_create_batch."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2509_11890_gb300 as tg  # noqa: E402
from oracle import sdp_dense as sd, tt, tt_problems as tp  # noqa: E402
from paper_2509_11890_gb300 import inputs  # noqa: E402


def _sum_of_random(d, ranks, seed):
    a = inputs.random_tt_matrix([2] * d, [2] * d, ranks, seed)
    b = inputs.random_tt_matrix([2] * d, [2] * d, ranks, seed + 1)
    # a + 0.5 a + 1e-3 b: rank-deficient unfoldings plus a small full-rank tail
    return tt.add(tt.add(a, a, 1.0, 0.5), b, 1.0, 1e-3)


def _shift(kind, d):
    I = tt.identity(d)
    if kind == 1:
        return I
    return tt.add(tt.ones_mat(d), I, 1.0, -1.0)


@pytest.mark.parametrize("psd_shift", [0, 1, 2])
@pytest.mark.parametrize("cap", [0, 6])
def test_round_sdp_matches_oracle_rounding_and_shift(psd_shift, cap):
    d = 6
    x = _sum_of_random(d, [1, 3, 5, 7, 5, 3, 1], 11)
    tol = 1e-2 * tt.norm(tt.vec_tt(x))
    got, zeta = tg.round_sdp(x, tol, cap, psd_shift)
    S = _shift(psd_shift, d) if psd_shift else None
    sn = tt.norm(tt.vec_tt(S)) if S is not None else 0.0
    rv, zeta_ref, ties = tt.round_tt(tt.vec_tt(x), tol / (1.0 + sn), cap or None)
    assert not any(ties)
    ref = tt.unvec_tt(rv)
    if S is not None and zeta_ref > 0:
        ref = tt.add(ref, S, 1.0, zeta_ref)
    # ranks are bookkeeping: bit-exact; zeta and the values in FP64
    assert tt.ranks(got) == tt.ranks(ref)
    assert math.isclose(zeta, zeta_ref, rel_tol=1e-9, abs_tol=1e-13)
    full_got, full_ref = tt.full_mat(got), tt.full_mat(ref)
    np.testing.assert_allclose(full_got, full_ref, rtol=0, atol=1e-11 * np.abs(full_ref).max())
    # the result differs from the input by zeta plus the shift: within tol when
    # the cap does not bind (Corollary psdness_rounding)
    err = np.linalg.norm(full_got - tt.full_mat(x))
    assert err <= zeta * (1.0 + sn) * (1 + 1e-9) + 1e-12 * tt.norm(tt.vec_tt(x))
    if not cap:
        assert err <= tol * (1 + 1e-9)
    if cap:
        extra = max(tt.ranks(S)) if (S is not None and zeta > 0) else 0
        assert max(tt.ranks(got)) <= cap + extra


def test_round_sdp_shift_keeps_psd():
    # a PSD matrix rounded hard stays PSD after the zeta I shift
    d = 5
    g = inputs.rng(3, 1)
    B = g.standard_normal((2 ** d, 6))
    M = B @ B.T + 1e-3 * np.eye(2 ** d)
    cores = tp.graph_tt(M, eps_rel=1e-14)
    tol = 0.05 * np.linalg.norm(M)
    got, zeta = tg.round_sdp(cores, tol, 4, 1)
    assert zeta > 0
    assert np.linalg.eigvalsh(tt.full_mat(got))[0] > -1e-9


def test_round_sdp_rejects_bad_arguments():
    x = _sum_of_random(4, [1, 2, 3, 2, 1], 3)
    with pytest.raises(tg.TTSDPError):
        tg.round_sdp(x, -1.0)
    with pytest.raises(tg.TTSDPError):
        tg.round_sdp(x, 1e-3, 0, 3)
    v = [c.reshape(c.shape[0], 4, c.shape[-1]) for c in x]
    with pytest.raises(tg.TTSDPError):
        tg.round_sdp(v, 1e-3, 0, 1)  # a shift needs a square TT matrix


def _parts(prob):
    return dict(C=prob.C, A_eq=prob.A_eq, B_eq=prob.B_eq, K_y=prob.K_y, A_ineq=prob.A_ineq, B_ineq=prob.B_ineq,
                K_t=prob.K_t, ones_t=prob.ones_t, ineq_sign=prob.ineq_sign, q=prob.q, lam0=prob.lam0,
                lam0_ineq=prob.lam0_ineq)


class _TorchAlloc:
    """Caller allocator backed by torch's caching allocator, counting blocks."""

    def __init__(self):
        self.live = {}
        self.allocs = 0

    def alloc(self, n, stream):
        p = torch.cuda.caching_allocator_alloc(max(int(n), 1), stream=int(stream or 0))
        self.live[p] = n
        self.allocs += 1
        return p

    def free(self, p, stream):
        self.live.pop(p)
        torch.cuda.caching_allocator_delete(p)


def test_create_with_caller_allocator_matches_default():
    d = 4
    inst = inputs.maxcut_kron(d, 2)
    prob = tp.maxcut(inst["adjacency_cores"], d)
    opts = tg.default_options(rank_cap=16, max_iters=40)
    ref = tg.Context.create(_parts(prob), opts).solve()
    ta = _TorchAlloc()
    al = tg.make_allocator(ta.alloc, ta.free)
    ctx = tg.Context.create(_parts(prob), opts, allocator=al)
    res = ctx.solve()
    assert res["status"] == 0, res
    assert ta.allocs > 100 and ta.live
    # same arithmetic, another allocator: the same iterates
    assert res["iters"] == ref["iters"]
    assert math.isclose(res["pobj"], ref["pobj"], rel_tol=1e-12)
    dense = sd.solve_dense(sd.maxcut_sdp(inst["weights"]))
    assert abs(res["pobj"] - dense.pobj) / (1 + abs(dense.pobj)) <= 2e-3
    ctx.close()
    torch.cuda.synchronize()
    assert not ta.live, len(ta.live)


def test_create_batch_solves_every_instance():
    insts = [inputs.maxcut_kron(d, 20 + d) for d in (3, 4, 5, 4)]
    parts = [_parts(tp.maxcut(i["adjacency_cores"], i["d"])) for i in insts]
    b = tg.Batch(parts, tg.default_options(rank_cap=16, max_iters=40))
    assert len(b) == 4
    res = b.solve()
    for inst, r in zip(insts, res):
        ref = sd.solve_dense(sd.maxcut_sdp(inst["weights"]))
        assert r["status"] == 0, r
        assert abs(r["pobj"] - ref.pobj) / (1 + abs(ref.pobj)) <= 2e-3
    X = tt.full_mat(b.member(2).iterate(0))
    np.testing.assert_allclose(np.diag(X), 1.0, atol=5e-3)
    with pytest.raises(IndexError):
        b.member(4)
    b.close()
