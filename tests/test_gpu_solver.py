"""GPU parity of the full TT interior-point solver against the dense SDP optimum
(oracle O2) and the oracle TT-IPM (O4) on the same seeded instances."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2509_11890_gb300 as tg  # noqa: E402
from oracle import sdp_dense as sd, tt, tt_ipm, tt_problems as tp  # noqa: E402
from paper_2509_11890_gb300 import inputs  # noqa: E402


def _opts(**kw):
    base = dict(rank_cap=16, max_iters=40)
    base.update(kw)
    return tg.default_options(**base)


@pytest.mark.parametrize("d,seed", [(3, 0), (4, 2), (5, 1)])
def test_maxcut_reaches_dense_optimum(d, seed):
    inst = inputs.maxcut_kron(d, seed)
    ref = sd.solve_dense(sd.maxcut_sdp(inst["weights"]))
    ctx = tg.Context.maxcut(inst["adjacency_cores"], _opts())
    res = ctx.solve()
    assert res["status"] == 0, res
    assert abs(res["pobj"] - ref.pobj) / (1 + abs(ref.pobj)) <= 2e-3
    assert res["rel_gap"] <= 1e-4 / math.sqrt(d)
    X = tt.full_mat(ctx.iterate(0))
    assert np.linalg.eigvalsh(0.5 * (X + X.T))[0] > 0
    np.testing.assert_allclose(np.diag(X), 1.0, atol=5e-3)


def test_maxcut_trajectory_matches_oracle_ipm():
    # same algorithm, same counter stream: the first iterations agree closely
    d = 4
    inst = inputs.maxcut_kron(d, 3)
    prob = tp.maxcut(inst["adjacency_cores"], d)
    o4 = tt_ipm.TTIPM(prob, tt_ipm.Options(rank_cap=16, max_iters=40))
    ctx = tg.Context.maxcut(inst["adjacency_cores"], _opts())
    for it in range(3):
        info = ctx.newton_step()
        o4.iterate(it)
        h = o4.history[-1]
        assert math.isclose(info["pobj"], h.pobj, rel_tol=1e-6, abs_tol=1e-8), (it, info["pobj"], h.pobj)
        assert math.isclose(info["mu"], h.mu, rel_tol=1e-6), (it, info["mu"], h.mu)


def test_theta_reaches_dense_optimum():
    d = 3
    inst = inputs.theta_hypercube_kron(d, 0)
    ref = sd.solve_dense(sd.theta_sdp(inst["adjacency"]))
    a = tp.graph_tt(inst["adjacency"])
    ctx = tg.Context.theta(a, _opts(max_iters=60))
    res = ctx.solve()
    assert res["status"] == 0, res
    assert abs(res["pobj"] - ref.pobj) / (1 + abs(ref.pobj)) <= 5e-3


def test_cc_reaches_dense_optimum():
    d = 3
    inst = inputs.cc_signed(d, 1)
    ref = sd.solve_dense(sd.cc_sdp(inst["c_plus"], inst["c_minus"], inst["adjacency"]))
    ctx = tg.Context.cc(tp.graph_tt(inst["c_plus"]), tp.graph_tt(inst["c_minus"]), tp.graph_tt(inst["adjacency"]),
                        _opts(max_iters=60))
    res = ctx.solve()
    assert res["status"] == 0, res
    assert abs(res["pobj"] - ref.pobj) / (1 + abs(ref.pobj)) <= 5e-3


def test_maxcut_gmres_local_solver_matches_dense_path():
    # forcing every local system onto the matrix-free GMRES path gives the same optimum
    d = 4
    inst = inputs.maxcut_kron(d, 2)
    ref = sd.solve_dense(sd.maxcut_sdp(inst["weights"]))
    ctx = tg.Context.maxcut(inst["adjacency_cores"], _opts(local_dense_max=0))
    res = ctx.solve()
    assert res["status"] == 0, res
    assert abs(res["pobj"] - ref.pobj) / (1 + abs(ref.pobj)) <= 2e-3
    info = ctx.newton_step()
    assert info["gmres_iters"] > 0


@pytest.mark.parametrize("prec", [tg.FP32])
def test_maxcut_mixed_precision_reaches_optimum(prec):
    d = 4
    inst = inputs.maxcut_kron(d, 2)
    ref = sd.solve_dense(sd.maxcut_sdp(inst["weights"]))
    ctx = tg.Context.maxcut(inst["adjacency_cores"], _opts(precision=prec))
    res = ctx.solve()
    assert res["status"] == 0, res
    assert abs(res["pobj"] - ref.pobj) / (1 + abs(ref.pobj)) <= 2e-3


def test_tt_from_dense_matches_oracle_tt_svd():
    d = 6
    inst = inputs.maxcut_kron_er(d, 0)
    w = inst["weights"]
    cores = tg.tt_from_dense(torch.from_numpy(w).cuda(), eps_rel=1e-13)
    np.testing.assert_allclose(tt.full_mat(cores), w, atol=1e-10)
    ref = tp.graph_tt(w, eps_rel=1e-13)
    assert tt.ranks(cores) == tt.ranks(ref)


def test_concurrent_batch_matches_single_solves():
    insts = [inputs.maxcut_kron(d, 10 + d) for d in (3, 4, 5, 3, 4, 5)]
    ctxs = [tg.Context.maxcut(i["adjacency_cores"], _opts()) for i in insts]
    res = tg.solve_batch(ctxs, workers=3)
    for inst, r in zip(insts, res):
        ref = sd.solve_dense(sd.maxcut_sdp(inst["weights"]))
        assert r["status"] == 0, r
        assert abs(r["pobj"] - ref.pobj) / (1 + abs(ref.pobj)) <= 2e-3
        assert r["seconds"] > 0


@pytest.mark.parametrize("prec,dense_max", [(tg.FP64, 4096), (tg.MIXED_TF32, 4096), (tg.MIXED_TF32, 0)])
def test_forcing_check_reports_fp64_local_residuals(prec, dense_max):
    # row a11: every local solve's FP64 residual against the projected
    # operator is measured; the forcing condition ||E|| <= eta ||R|| holds
    # with eta <= eta0 = 1e-3 (LU refined to 1e-10, GMRES to eta/10)
    inst = inputs.maxcut_kron(4, 2)
    ctx = tg.Context.maxcut(inst["adjacency_cores"], _opts(precision=prec, local_dense_max=dense_max))
    for _ in range(4):
        info = ctx.newton_step()
        if info["converged"]:
            break
        assert 0.0 < info["forcing"] < 1e-3, info
        if dense_max > 0:
            assert info["forcing"] <= 1e-6, info
    assert info["forcing_corrections"] >= 0


def test_time_limit_stops_a_solve_and_keeps_the_last_iterate():
    inst = inputs.maxcut_kron(5, 1)
    ctx = tg.Context.maxcut(inst["adjacency_cores"], _opts(time_limit=1e-3))
    res = ctx.solve()
    assert res["status"] == 7, res          # TT_E_NO_CONVERGENCE: the limit passed
    X = tt.full_mat(ctx.iterate(0))         # the context is still usable
    assert np.all(np.isfinite(X))
    # without a limit the same context continues to the optimum
    ref = sd.solve_dense(sd.maxcut_sdp(inst["weights"]))
    ctx2 = tg.Context.maxcut(inst["adjacency_cores"], _opts())
    res2 = ctx2.solve()
    assert res2["status"] == 0 and abs(res2["pobj"] - ref.pobj) / (1 + abs(ref.pobj)) <= 2e-3


@pytest.mark.parametrize("d,r,seed", [(5, 2, 5), (6, 3, 6)])
def test_rank_controlled_maxcut_reaches_dense_optimum(d, r, seed):
    # the paper's instance family (Appendix A) with input TT rank r
    inst = inputs.rank_controlled_graph(d, r, seed)
    ref = sd.solve_dense(sd.maxcut_sdp(inst["weights"]))
    ctx = tg.Context.maxcut(inst["adjacency_cores"], _opts(rank_cap=32))
    res = ctx.solve()
    assert res["status"] == 0, res
    assert abs(res["pobj"] - ref.pobj) / (1 + abs(ref.pobj)) <= 2e-3
