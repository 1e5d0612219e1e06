"""The safeguards of Section 3.5 on the CUDA path against the oracle TT-IPM (O4):
damp-and-retry of an update planted past the boundary of the cone, and the
AHO -> XZ fallback when the AMEn sweep budget is too small to meet the
tolerance. Both sides run the same algorithm on the same counter stream, so
the counters must agree exactly and the objectives to 1e-6."""
import math

import numpy as np
import pytest
import scipy.linalg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2509_11890_gb300 as tg  # noqa: E402
from oracle import sdp_dense as sd, tt, tt_ipm, tt_problems as tp  # noqa: E402
from paper_2509_11890_gb300 import inputs  # noqa: E402


def test_damp_and_retry_repairs_a_planted_overlong_step():
    d, seed, cap = 4, 2, 16
    inst = inputs.maxcut_kron(d, seed)
    prob = tp.maxcut(inst["adjacency_cores"], d)
    ipm = tt_ipm.TTIPM(prob, tt_ipm.Options(rank_cap=cap, max_iters=40))
    ctx = tg.Context.maxcut(inst["adjacency_cores"], tg.default_options(rank_cap=cap, max_iters=40))
    assert ipm.iterate(0) is not None
    info = ctx.newton_step()
    assert math.isclose(info["alpha_p"], ipm.history[-1].alpha_p, rel_tol=1e-6)
    # a primal step three times past the boundary of the cone along dX
    lam = float(scipy.linalg.eigh(tt.full_mat(ipm.prev["dX"]), tt.full_mat(ipm.prev["X"]), eigvals_only=True)[0])
    assert lam < 0
    alpha = 3.0 * tt_ipm.step_from_lambda(lam)
    ipm.prev["ap"] = alpha
    ipm._apply_update()
    ctx.redo_update(alpha, -1.0)
    assert np.linalg.eigvalsh(tt.full_mat(ctx.iterate(0)))[0] < 0
    for it in range(1, 41):
        info = ctx.newton_step()
        done = ipm.iterate(it) is None
        h = ipm.history[-1]
        assert math.isclose(info["pobj"], h.pobj, rel_tol=1e-6, abs_tol=1e-9), (it, info["pobj"], h.pobj)
        assert info["damped_retries"] == ipm.retries, (it, info["damped_retries"], ipm.retries)
        assert bool(info["converged"]) == done
        if done:
            break
    assert info["converged"] and ipm.retries >= 1
    assert np.linalg.eigvalsh(tt.full_mat(ctx.iterate(0)))[0] > 0
    ref = sd.solve_dense(sd.maxcut_sdp(inst["weights"]))
    assert abs(info["pobj"] - ref.pobj) / (1 + abs(ref.pobj)) <= 2e-3


def test_aho_to_xz_fallback_fires_like_the_oracle():
    # one AMEn sweep per Newton solve cannot meet the tolerance once the warm
    # start stops matching: the AHO iterations after the warm-up fall back to XZ
    d, seed, cap = 4, 2, 16
    inst = inputs.maxcut_kron(d, seed)
    prob = tp.maxcut(inst["adjacency_cores"], d)
    ipm = tt_ipm.TTIPM(prob, tt_ipm.Options(rank_cap=cap, max_iters=12, max_sweeps=1))
    ctx = tg.Context.maxcut(inst["adjacency_cores"], tg.default_options(rank_cap=cap, max_iters=12, max_sweeps=1))
    for it in range(8):
        info = ctx.newton_step()
        done = ipm.iterate(it) is None
        h = ipm.history[-1]
        assert math.isclose(info["pobj"], h.pobj, rel_tol=1e-6, abs_tol=1e-9), (it, info["pobj"], h.pobj)
        assert info["xz_fallbacks"] == ipm.fallbacks, (it, info["xz_fallbacks"], ipm.fallbacks)
        if not done:
            assert info["direction"] == (1 if h.direction == "aho" else 0), (it, info["direction"], h.direction)
        if done:
            break
    assert ipm.fallbacks >= 1
