"""The block elimination of the reduced projected Newton system (Section 3.3,
after eq. reduced_kkt_system), written out with numpy on random blocks of the
same structure and checked against the dense solve of the assembled system.

This pins the reading the CUDA path follows (tt_kkt_solve and the AMEn
dense local solves): without inequalities the paper's formulas are used as
printed (S = A L_Z^-1 L_X A^T + K_Y; S dY = A L_Z^-1 (L_X R_d - R_c) - R_p;
dZ = A^T dY - R_d; dX = -L_Z^-1 (R_c + L_X dZ)); with inequalities the exact
nested elimination (Phi first, then the multipliers' Schur complement), whose
last term carries the factors L_Z^-1 L_X A_ineq^T and L_Z^-1 L_X A_eq^T that
the printed S leaves out.
"""
import numpy as np
import pytest

from paper_2509_11890_gb300 import inputs


def _spd(g, n, lo, hi):
    q, _ = np.linalg.qr(g.standard_normal((n, n)))
    return (q * np.exp(g.uniform(np.log(lo), np.log(hi), n))) @ q.T


def _blocks(n, seed):
    g = inputs.rng(seed, 300 + n)
    LZ, LX = _spd(g, n, 0.1, 10.0), _spd(g, n, 0.1, 10.0)
    A = g.standard_normal((n, n)) / np.sqrt(n)
    Ky = 0.1 * g.standard_normal((n, n)) / np.sqrt(n)
    TA = g.standard_normal((n, n)) / np.sqrt(n)
    Ai = g.standard_normal((n, n)) / np.sqrt(n)
    D = np.diag(g.uniform(0.5, 2.0, n))
    Rp, Rt, Rc, Rd = (g.standard_normal(n) for _ in range(4))
    return LZ, LX, A, Ky, TA, Ai, D, Rp, Rt, Rc, Rd


@pytest.mark.parametrize("n", [3, 17, 40])
def test_paper_formulas_without_inequalities_solve_the_reduced_system(n):
    LZ, LX, A, Ky, _, _, _, Rp, _, Rc, Rd = _blocks(n, 1)
    # eq. reduced_kkt_system without the inequality block
    K = np.block([[-A, Ky], [LZ, LX @ A.T]])
    b = -np.concatenate([Rp, Rc - LX @ Rd])
    ref = np.linalg.solve(K, b)
    # the paper's elimination, as printed
    LZi = np.linalg.inv(LZ)
    S = A @ LZi @ LX @ A.T + Ky
    dY = np.linalg.solve(S, A @ LZi @ (LX @ Rd - Rc) - Rp)
    dZ = A.T @ dY - Rd
    dX = -LZi @ (Rc + LX @ dZ)
    np.testing.assert_allclose(np.concatenate([dX, dY]), ref, rtol=0, atol=1e-10 * np.abs(ref).max())
    # the Cholesky factor of L_Z is all the elimination needs of it
    L = np.linalg.cholesky(LZ)
    W, V = np.linalg.solve(L, (-A).T), np.linalg.solve(L, LX @ A.T)  # L^-1 E^T, L^-1 G
    np.testing.assert_allclose(Ky - W.T @ V, S, rtol=0, atol=1e-10 * np.abs(S).max())


@pytest.mark.parametrize("n", [3, 17, 40])
def test_nested_elimination_with_inequalities_solves_the_reduced_system(n):
    LZ, LX, A, Ky, TA, Ai, D, Rp, Rt, Rc, Rd = _blocks(n, 2)
    Gy, Gt = LX @ A.T, LX @ Ai.T
    Z0 = np.zeros((n, n))
    K = np.block([[-A, Ky, Z0], [-TA, Z0, D], [LZ, Gy, Gt]])
    b = -np.concatenate([Rp, Rt, Rc - LX @ Rd])
    ref = np.linalg.solve(K, b)
    bp, bt, bc = b[:n], b[n:2 * n], b[2 * n:]
    LZi = np.linalg.inv(LZ)
    # Phi (as printed), then the exact Schur complement of the multipliers
    Phi = TA @ LZi @ Gt + D
    S = A @ LZi @ Gy + Ky - A @ LZi @ Gt @ np.linalg.solve(Phi, TA @ LZi @ Gy)
    rt = bt + TA @ LZi @ bc
    dY = np.linalg.solve(S, bp + A @ LZi @ bc - A @ LZi @ Gt @ np.linalg.solve(Phi, rt))
    dT = np.linalg.solve(Phi, rt - TA @ LZi @ Gy @ dY)
    dX = LZi @ (bc - Gy @ dY - Gt @ dT)
    np.testing.assert_allclose(np.concatenate([dX, dY, dT]), ref, rtol=0, atol=1e-10 * np.abs(ref).max())
    # the single 2n x 2n Schur complement of the CUDA path gives the same
    # multipliers: (F - E L_Z^-1 G) dl = b_m - E L_Z^-1 b_c
    E = np.vstack([-A, -TA])
    F = np.block([[Ky, Z0], [Z0, D]])
    G = np.hstack([Gy, Gt])
    dl = np.linalg.solve(F - E @ LZi @ G, np.concatenate([bp, bt]) - E @ LZi @ bc)
    np.testing.assert_allclose(dl, np.concatenate([dY, dT]), rtol=0, atol=1e-10 * np.abs(ref).max())
    # the printed S, without those factors, is a different matrix
    S_printed = A @ LZi @ Gy + Ky - A @ np.linalg.solve(Phi, TA)
    assert np.abs(S_printed - S).max() > 1e-3 * np.abs(S).max()
