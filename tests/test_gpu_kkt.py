"""GPU parity of the block-elimination solve of the reduced projected Newton
system (Section 3.3, eq. reduced_kkt_system and the block elimination that
follows it: a Cholesky factor of the projected L_Z, an LU of the multipliers'
Schur complement) through tt_kkt_solve, against numpy's LU solve of the same
assembled system.

The systems have the block structure of the local systems of the AMEn sweep:
unknowns [dX; multipliers], equations [multiplier rows; complementarity rows],
with L_Z = W^T L_Z W symmetric positive definite up to rounding (a relative
asymmetry of 1e-12 is added, as the contractions leave one) and the coupling
block G = L_X A^T. Both solutions carry an error of at most about
cond(K) * eps * ||x||; the test allows 16 times that, element by element.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2509_11890_gb300 as tg  # noqa: E402
from oracle import sdp_dense as sd  # noqa: E402
from paper_2509_11890_gb300 import inputs  # noqa: E402

DEV = "cuda"
EPS = np.finfo(np.float64).eps


def _spd(g, n, lo, hi):
    q, _ = np.linalg.qr(g.standard_normal((n, n)))
    lam = np.exp(g.uniform(np.log(lo), np.log(hi), n))
    return (q * lam) @ q.T


def _system(n, ineq, seed, indefinite=False, spread=1e2):
    """K (N x N) and b with N = n (dX) + n or 2n (multipliers); the spectra of
    L_Z and L_X span [1 / spread, spread]."""
    g = inputs.rng(seed, n)
    LZ = _spd(g, n, 1.0 / spread, spread)
    if indefinite:
        LZ -= 2e-2 * np.eye(n) + np.diag(np.where(np.arange(n) % 3 == 0, 1.0, 0.0))
    LZ += 1e-12 * np.abs(LZ).max() * g.standard_normal((n, n))  # rounding-level asymmetry
    LX = _spd(g, n, 1.0 / spread, spread)
    A = g.standard_normal((n, n)) / np.sqrt(n)
    Ky = 0.1 * g.standard_normal((n, n)) / np.sqrt(n)
    if not ineq:
        E, F, G = -A, Ky, LX @ A.T
    else:
        TA = g.standard_normal((n, n)) / np.sqrt(n)
        AiT = g.standard_normal((n, n)) / np.sqrt(n)
        DK = np.diag(g.uniform(0.5, 2.0, n)) + 0.05 * g.standard_normal((n, n)) / np.sqrt(n)
        sgn = -1.0
        E = np.vstack([-A, sgn * TA])
        F = np.block([[Ky, np.zeros((n, n))], [np.zeros((n, n)), DK]])
        G = np.hstack([LX @ A.T, -sgn * LX @ AiT])
    K = np.block([[E, F], [LZ, G]])
    x = g.standard_normal(K.shape[0])
    return K, K @ x


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.mark.parametrize("n,ineq", [(1, False), (5, False), (32, False), (33, True), (100, False),
                                    (300, True), (700, False)])
@pytest.mark.parametrize("prec", [tg.FP64, tg.MIXED_TF32])
def test_kkt_block_solve_matches_lu(n, ineq, prec):
    # FP32 factors refine to 1e-10 only while cond(K) * 2^-24 is well below 1
    K, b = _system(n, ineq, 31, spread=1e2 if prec == tg.FP64 else 3.0)
    ref = np.linalg.solve(K, b)
    Kd, bd = _t(K), _t(b)
    tg.kkt_stats(reset=True)
    rho = tg.kkt_solve(Kd, bd, n, prec)
    block, fp32, fallback = tg.kkt_stats()
    assert (block, fallback) == (1, 0)
    if prec != tg.FP64:
        assert fp32 == 1
    got = bd.cpu().numpy()
    assert rho <= (1e-13 if prec == tg.FP64 else 1e-10), rho
    cond = np.linalg.cond(K)
    np.testing.assert_allclose(got, ref, rtol=0, atol=16 * cond * max(rho, EPS) * np.abs(ref).max())
    np.testing.assert_array_equal(Kd.cpu().numpy(), K)  # K is not modified


@pytest.mark.parametrize("prec", [tg.FP64, tg.MIXED_BF16])
def test_kkt_indefinite_lz_falls_back_to_lu(prec):
    n = 70
    K, b = _system(n, False, 5, indefinite=True, spread=3.0)
    assert np.linalg.eigvalsh(0.5 * (K[n:, :n] + K[n:, :n].T))[0] < 0
    ref = np.linalg.solve(K, b)
    bd = _t(b)
    tg.kkt_stats(reset=True)
    rho = tg.kkt_solve(_t(K), bd, n, prec)
    assert tg.kkt_stats() == (0, 0, 1)
    assert rho <= 1e-10
    np.testing.assert_allclose(bd.cpu().numpy(), ref, rtol=0,
                               atol=16 * np.linalg.cond(K) * max(rho, EPS) * np.abs(ref).max())


def test_kkt_solve_rejects_bad_block_sizes():
    K, b = _system(4, False, 1)
    for n_lz in (0, 8, -1):
        with pytest.raises(tg.TTSDPError):
            tg.kkt_solve(_t(K), _t(b), n_lz)


def test_fp32_factors_option_keeps_the_fp64_solve():
    # FP64 solves with FP32 factors refined to an FP64 residual of 1e-14
    # (the default) and with FP64 factors only: both certify, and both
    # objectives are as close to the dense optimum as the certified gap
    # allows (local solves that differ at 1e-14 can move a truncation rank of
    # the AMEn sweeps, so the trajectories agree to the solve's tolerance,
    # not to rounding)
    inst = inputs.maxcut_kron(5, 3)
    ref = sd.solve_dense(sd.maxcut_sdp(inst["weights"])).pobj
    res = {}
    for f32 in (1, 0):
        tg.kkt_stats(reset=True)
        ctx = tg.Context.maxcut(inst["adjacency_cores"], tg.default_options(rank_cap=16, max_iters=40,
                                                                            fp32_factors=f32))
        res[f32] = ctx.solve()
        block, fp32, _ = tg.kkt_stats(reset=True)
        ctx.close()
        assert block > 0
        assert (fp32 > 0) if f32 else (fp32 == 0)
        assert res[f32]["status"] == 0
    assert abs(res[0]["iters"] - res[1]["iters"]) <= 1
    for r in res.values():
        assert abs(r["pobj"] - ref) / (1 + abs(ref)) <= 2e-3
