"""Combined multiplier storage (Section 3.5, "Combined Multiplier Storage") on the
CUDA path: correlation clustering, whose multiplier masks (diagonal for Y,
off-diagonal for T) are disjoint, solved with one block dLambda against the
oracle TT-IPM (O4) with the same option, iteration by iteration, and against the
dense optimum (O2) in both storage forms."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2509_11890_gb300 as tg  # noqa: E402
from oracle import sdp_dense as sd, tt, tt_ipm, tt_problems as tp  # noqa: E402
from paper_2509_11890_gb300 import inputs  # noqa: E402


def _cc(d, seed):
    inst = inputs.cc_signed(d, seed)
    cores = [tp.graph_tt(inst[k]) for k in ("c_plus", "c_minus", "adjacency")]
    return inst, cores


# Correlation-clustering step lengths come from rank-1 eigensolver sweeps on
# diagonal operators (the slack and the multiplier T) whose spectra have exact
# ties (mirrored entries u, v and v, u); the GPU's local eigenvectors (FP32
# Jacobi, FP64 Rayleigh quotient) and the oracle's (LAPACK) then settle on
# step lengths that differ by up to about 1e-3 relative from the first
# iteration on, in either storage form. The trajectories are compared at that
# level; the optimum is compared with the dense oracle.
CC_TRAJ_TOL = 2e-3


@pytest.mark.parametrize("d,seed", [(3, 1), (3, 2)])
def test_combined_cc_follows_oracle_ipm(d, seed):
    inst, (cp, cm, ad) = _cc(d, seed)
    prob = tp.corr_clustering(cp, cm, ad, d)
    o4 = tt_ipm.TTIPM(prob, tt_ipm.Options(rank_cap=16, max_iters=60, combined_multipliers=True))
    ctx = tg.Context.cc(cp, cm, ad, tg.default_options(rank_cap=16, max_iters=60, combined_multipliers=1))
    for it in range(61):
        info = ctx.newton_step()
        done = o4.iterate(it) is None
        h = o4.history[-1]
        assert math.isclose(info["pobj"], h.pobj, rel_tol=CC_TRAJ_TOL), (it, info["pobj"], h.pobj)
        if done or info["converged"]:
            break
    for _ in range(60):
        if info["converged"]:
            break
        info = ctx.newton_step()
    assert info["converged"]
    ref = sd.solve_dense(sd.cc_sdp(inst["c_plus"], inst["c_minus"], inst["adjacency"]))
    assert abs(info["pobj"] - ref.pobj) / (1 + abs(ref.pobj)) <= 5e-3


def test_separate_and_combined_storage_reach_the_dense_optimum():
    d = 3
    inst, (cp, cm, ad) = _cc(d, 1)
    ref = sd.solve_dense(sd.cc_sdp(inst["c_plus"], inst["c_minus"], inst["adjacency"]))
    for combined in (0, 1):
        ctx = tg.Context.cc(cp, cm, ad, tg.default_options(rank_cap=16, max_iters=60,
                                                           combined_multipliers=combined))
        res = ctx.solve()
        assert res["status"] == 0, (combined, res)
        assert abs(res["pobj"] - ref.pobj) / (1 + abs(ref.pobj)) <= 5e-3
        T = tt.full_mat(ctx.iterate(2))
        n = 2 ** d
        assert np.all(T[~np.eye(n, dtype=bool)] > 0)
