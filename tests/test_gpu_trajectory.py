"""FP64 GPU solves against the oracle TT-IPM (O4) at every iteration of a
complete solve: the objective to 1e-6 relative and the per-bond ranks of X, Z
and of the block-AMEn frame bit-exact (same algorithm, same parameters, same
SplitMix64 counter stream on both sides), and the final objective against the
dense optimum (O2)."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2509_11890_gb300 as tg  # noqa: E402
from oracle import sdp_dense as sd, tt, tt_ipm, tt_problems as tp  # noqa: E402
from paper_2509_11890_gb300 import inputs  # noqa: E402

OBJ_TOL = 1e-6


def _run_both(adj_cores, weights, d, cap, max_iters=30):
    prob = tp.maxcut(adj_cores, d)
    o4 = tt_ipm.TTIPM(prob, tt_ipm.Options(rank_cap=cap, max_iters=max_iters))
    ctx = tg.Context.maxcut(adj_cores, tg.default_options(rank_cap=cap, max_iters=max_iters))
    rows = []
    for it in range(max_iters + 1):
        info = ctx.newton_step()
        done = o4.iterate(it) is None
        h = o4.history[-1]
        rows.append((info, h, None if info["converged"] else (ctx.ranks(0), ctx.ranks(3), ctx.ranks(4))))
        assert bool(info["converged"]) == done, (it, info, h)
        if done:
            break
    return rows, ctx


@pytest.mark.parametrize("seed", [0, 1, 2, 3, 4])
def test_fp64_solve_follows_oracle_ipm_every_iteration(seed):
    # Max-Cut, Kronecker graph, unit weights, d = 6, rank cap 16
    d, cap = 6, 16
    inst = inputs.maxcut_kron(d, seed)
    rows, ctx = _run_both(inst["adjacency_cores"], inst["weights"], d, cap)
    for info, h, ranks in rows:
        it = info["iter"]
        assert math.isclose(info["pobj"], h.pobj, rel_tol=OBJ_TOL, abs_tol=1e-9), (it, info["pobj"], h.pobj)
        assert math.isclose(info["dobj"], h.dobj, rel_tol=OBJ_TOL, abs_tol=1e-9), (it, info["dobj"], h.dobj)
        # mu = <X, Z> / 2^d is a difference of nearly cancelling terms near the
        # optimum: compared relative to the objective's scale
        assert math.isclose(info["mu"], h.mu, rel_tol=OBJ_TOL, abs_tol=OBJ_TOL * 1e-2 * (1 + abs(h.pobj))), \
            (it, info["mu"], h.mu)
        if ranks is not None:
            assert ranks[0] == h.ranks_X, (it, ranks[0], h.ranks_X)
            assert ranks[1] == h.ranks_Z, (it, ranks[1], h.ranks_Z)
            assert ranks[2] == h.ranks_W, (it, ranks[2], h.ranks_W)
    last = rows[-1][0]
    assert last["converged"] == 1
    # the final objective against the dense optimum: within the certified
    # objective gap |pobj - dobj| / (1 + |pobj|) plus the residual terms
    ref = sd.solve_dense(sd.maxcut_sdp(inst["weights"]), tol=1e-10)
    err = abs(last["pobj"] - ref.pobj) / (1 + abs(ref.pobj))
    gap = abs(last["pobj"] - last["dobj"]) / (1 + abs(last["pobj"]))
    assert err <= gap + last["rel_p"] + last["rel_d"], (err, gap, last)
    X = tt.full_mat(ctx.iterate(0))
    assert np.linalg.eigvalsh(0.5 * (X + X.T))[0] > 0


def test_binding_rank_cap_is_the_method_not_the_gpu():
    # weights U[0.5, 1.5] on a Kronecker OR Erdos-Renyi graph at d = 5 with rank
    # cap 4: the cap binds (the objective's unfoldings have rank up to 16), and
    # the GPU follows the oracle's trajectory while neither can certify
    import bench
    d, cap = 5, 4
    inst = inputs.maxcut_kron_er(d, 0)
    adj = tp.graph_tt(inst["weights"], eps_rel=1e-13)
    assert max(tt.ranks(adj)) > cap
    lb = bench.dual_residual_lower_bound(inst["weights"], cap)
    assert not lb["certifiable"]
    rows, _ = _run_both(adj, inst["weights"], d, cap, max_iters=6)
    for info, h, ranks in rows:
        it = info["iter"]
        assert math.isclose(info["pobj"], h.pobj, rel_tol=OBJ_TOL, abs_tol=1e-9), (it, info["pobj"], h.pobj)
        assert math.isclose(info["rel_d"], h.rel_d, rel_tol=1e-5), (it, info["rel_d"], h.rel_d)
        # no iterate beats the Eckart-Young bound of the capped rank
        assert info["rel_d"] >= lb["rel_d_lower_bound"] * (1 - 1e-9)
        assert not info["converged"]


def test_theta_fp64_solve_follows_oracle_ipm_every_iteration():
    # Lovasz theta (Section 4.2: A_eq carries the trace row vec(E_11) vec(I)^T,
    # so the operator is not diagonal), d = 4, cap 16
    d, cap = 4, 16
    inst = inputs.theta_hypercube_kron(d, 0)
    a = tp.graph_tt(inst["adjacency"])
    o4 = tt_ipm.TTIPM(tp.theta(a, d), tt_ipm.Options(rank_cap=cap, max_iters=40))
    ctx = tg.Context.theta(a, tg.default_options(rank_cap=cap, max_iters=40))
    for it in range(41):
        info = ctx.newton_step()
        done = o4.iterate(it) is None
        h = o4.history[-1]
        assert math.isclose(info["pobj"], h.pobj, rel_tol=OBJ_TOL, abs_tol=1e-9), (it, info["pobj"], h.pobj)
        assert math.isclose(info["dobj"], h.dobj, rel_tol=OBJ_TOL, abs_tol=1e-9), (it, info["dobj"], h.dobj)
        assert bool(info["converged"]) == done, (it, info, h)
        if done:
            break
        assert ctx.ranks(0) == h.ranks_X and ctx.ranks(3) == h.ranks_Z, (it, ctx.ranks(0), h.ranks_X)
    assert info["converged"]
    ref = sd.solve_dense(sd.theta_sdp(inst["adjacency"]), tol=1e-10)
    assert abs(info["pobj"] - ref.pobj) / (1 + abs(ref.pobj)) <= 1e-3


def test_gmres_local_solves_at_real_ranks_reach_the_dense_optimum():
    # d = 8, cap 64, every local system of more than 512 unknowns on the
    # matrix-free GMRES path (restarted, FP64 forcing check); the result is
    # compared with the dense optimum
    d = 8
    inst = inputs.maxcut_kron(d, 3)
    ref = sd.solve_dense(sd.maxcut_sdp(inst["weights"]), tol=1e-10)
    ctx = tg.Context.maxcut(inst["adjacency_cores"], tg.default_options(rank_cap=64, max_iters=40,
                                                                         local_dense_max=512, time_limit=120.0))
    res = ctx.solve()
    assert res["status"] == 0, res
    info = ctx.newton_step()
    assert info["gmres_iters"] > 0
    err = abs(res["pobj"] - ref.pobj) / (1 + abs(ref.pobj))
    gap = abs(res["pobj"] - res["dobj"]) / (1 + abs(res["pobj"]))
    assert err <= gap + res["rel_p"] + res["rel_d"], (err, gap, res)
