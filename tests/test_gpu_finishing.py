"""The finishing phase of Section 3.5 ("Relaxing the Positive Definiteness
Barrier") on the CUDA path against the oracle TT-IPM (O4) with the same
options: the same iterations, the same accept / reject decisions and
relaxations, and the objective moved closer to the dense optimum (O2)."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2509_11890_gb300 as tg  # noqa: E402
from oracle import sdp_dense as sd, tt, tt_ipm, tt_problems as tp  # noqa: E402
from paper_2509_11890_gb300 import inputs  # noqa: E402


@pytest.mark.parametrize("d,seed", [(5, 1), (6, 0)])
def test_finishing_phase_follows_the_oracle(d, seed):
    inst = inputs.maxcut_kron(d, seed)
    prob = tp.maxcut(inst["adjacency_cores"], d)
    ref = sd.solve_dense(sd.maxcut_sdp(inst["weights"]), tol=1e-10).pobj
    o4 = tt_ipm.TTIPM(prob, tt_ipm.Options(rank_cap=16, max_iters=40, finish_tol=1e-3))
    ctx = tg.Context.maxcut(inst["adjacency_cores"], tg.default_options(rank_cap=16, max_iters=40, finish_tol=1e-3))
    nfin = 0
    for it in range(41):
        info = ctx.newton_step()
        done = o4.iterate(it) is None
        h = o4.history[-1]
        assert math.isclose(info["pobj"], h.pobj, rel_tol=1e-6, abs_tol=1e-9), (it, info["pobj"], h.pobj)
        assert bool(info["converged"]) == done, (it, info, h)
        if done:
            break
        assert bool(info["finishing"]) == h.finishing, (it, info["finishing"], h.finishing)
        if h.finishing:
            nfin += 1
            assert bool(info["accepted"]) == h.accepted and info["nu"] == h.nu
            # the merit sums absolute residual norms, which near the optimum are
            # small differences of large terms: compared on the objective's scale
            assert math.isclose(info["merit"], h.merit, rel_tol=1e-6, abs_tol=1e-6 * (1 + abs(h.pobj)))
    assert info["converged"] and nfin >= 1
    # the absolute criteria hold at the end and the objective is closer to p*
    plain = tg.Context.maxcut(inst["adjacency_cores"], tg.default_options(rank_cap=16, max_iters=40)).solve()
    e_plain = abs(plain["pobj"] - ref) / (1 + abs(ref))
    e_fin = abs(info["pobj"] - ref) / (1 + abs(ref))
    assert e_fin <= 0.1 * e_plain, (e_fin, e_plain)
    X = tt.full_mat(ctx.iterate(0))
    assert np.linalg.eigvalsh(0.5 * (X + X.T))[0] >= -1e-3
