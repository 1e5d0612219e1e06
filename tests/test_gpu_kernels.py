"""GPU parity of the contraction, TT-arithmetic and rounding kernels against the oracle.

Every call goes through the C ABI (via the ctypes binding); expected values
come from the oracle only. Contractions are compared element by element: the
error of every output entry must stay below tol times the same contraction of
the operands' absolute values (the floating-point bound of a sum of
products, sum |terms|), with tol 1e-12 in FP64 and 1e-5 in FP32 (at most a
few times the unit roundoff times the longest chain of roundings).
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2509_11890_gb300 as tg  # noqa: E402
from oracle import tt  # noqa: E402
from paper_2509_11890_gb300 import inputs  # noqa: E402

DEV = "cuda"

# (rw, rw2, R, R2, rv, rv2, m, n): small, tile-spanning with ragged tails, boundary, 2x2 modes, bench-sized
SHAPES = [
    (1, 4, 1, 2, 1, 3, 4, 4),
    (3, 70, 5, 33, 2, 65, 4, 4),
    (17, 9, 7, 3, 66, 5, 4, 4),
    (5, 6, 3, 4, 7, 2, 2, 2),
    (16, 16, 32, 32, 16, 16, 4, 4),
    (64, 64, 128, 128, 64, 64, 4, 4),
]


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _rand(shape, seed):
    return inputs.rng(seed, 77).standard_normal(shape)


def _dims(s):
    return dict(zip(["rw", "rw2", "R", "R2", "rv", "rv2", "m", "n"], s))


def assert_bounded(got, ref, ref_abs, tol):
    """|got - ref| <= tol * ref_abs + tiny, element by element."""
    got = got.reshape(ref.shape)
    bound = tol * ref_abs + 1e-300
    bad = np.abs(got - ref) > bound
    assert not bad.any(), (int(bad.sum()), float(np.max(np.abs(got - ref) / bound)))


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("prec,tol", [(tg.FP64, 1e-12), (tg.FP32, 1e-5)])
def test_env_left_step(shape, prec, tol):
    rw, rw2, R, R2, rv, rv2, m, n = shape
    phi, u = _rand((rw, R, rv), 1), _rand((rw, m, rw2), 2)
    op, v = _rand((R, m, n, R2), 3), _rand((rv, n, rv2), 4)
    ref = tt.env_left_step(phi, u, op, v)
    ref_abs = tt.env_left_step(np.abs(phi), np.abs(u), np.abs(op), np.abs(v))
    out = torch.empty(rw2 * R2 * rv2, dtype=torch.float64, device=DEV)
    tg.env_left_step(_dims(shape), _t(phi), _t(u), _t(op), _t(v), out, prec)
    assert_bounded(out.cpu().numpy(), ref, ref_abs, tol)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("prec,tol", [(tg.FP64, 1e-12), (tg.FP32, 1e-5)])
def test_env_right_step(shape, prec, tol):
    rw, rw2, R, R2, rv, rv2, m, n = shape
    psi, u = _rand((rw2, R2, rv2), 5), _rand((rw, m, rw2), 6)
    op, v = _rand((R, m, n, R2), 7), _rand((rv, n, rv2), 8)
    ref = tt.env_right_step(psi, u, op, v)
    ref_abs = tt.env_right_step(np.abs(psi), np.abs(u), np.abs(op), np.abs(v))
    out = torch.empty(rw * R * rv, dtype=torch.float64, device=DEV)
    tg.env_right_step(_dims(shape), _t(psi), _t(u), _t(op), _t(v), out, prec)
    assert_bounded(out.cpu().numpy(), ref, ref_abs, tol)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("prec,tol", [(tg.FP64, 1e-12), (tg.FP32, 1e-5)])
def test_local_apply(shape, prec, tol):
    rw, rw2, R, R2, rv, rv2, m, n = shape
    phi, psi = _rand((rw, R, rv), 9), _rand((rw2, R2, rv2), 10)
    op, x = _rand((R, m, n, R2), 11), _rand((rv, n, rv2), 12)
    ref = tt.local_apply(phi, op, psi, x)
    ref_abs = tt.local_apply(np.abs(phi), np.abs(op), np.abs(psi), np.abs(x))
    y = torch.empty(rw * m * rw2, dtype=torch.float64, device=DEV)
    tg.local_apply(_dims(shape), _t(phi), _t(op), _t(psi), _t(x), y, prec)
    assert_bounded(y.cpu().numpy(), ref, ref_abs, tol)


@pytest.mark.parametrize("shape", SHAPES[:5])
def test_local_matrix(shape):
    rw, rw2, R, R2, rv, rv2, m, n = shape
    phi, psi = _rand((rw, R, rv), 13), _rand((rw2, R2, rv2), 14)
    op = _rand((R, m, n, R2), 15)
    ref = tt.local_matrix(phi, op, psi)
    ref_abs = tt.local_matrix(np.abs(phi), np.abs(op), np.abs(psi))
    out = torch.empty(ref.size, dtype=torch.float64, device=DEV)
    tg.local_matrix(_dims(shape), _t(phi), _t(op), _t(psi), out, tg.FP64)
    assert_bounded(out.cpu().numpy(), ref, ref_abs, 1e-12)


def _rtt(dims, rk, seed, mat=False):
    d = len(dims)
    ranks = [1] + [rk] * (d - 1) + [1]
    if mat:
        return inputs.random_tt_matrix(dims, dims, ranks, seed)
    return inputs.random_tt(dims, ranks, seed)


def test_hadamard_matvec_inner():
    a = _rtt([2] * 5, 3, 21, mat=True)
    b = _rtt([2] * 5, 4, 22, mat=True)
    got = tg.hadamard(tg.DevTT.from_cores(a), tg.DevTT.from_cores(b)).cores()
    ref = tt.hadamard(a, b)
    for g, r in zip(got, ref):
        np.testing.assert_allclose(g, r, rtol=0, atol=1e-13 * np.abs(r).max())
    op = inputs.random_tt_matrix([4] * 4, [4] * 4, [1, 2, 3, 2, 1], 23)
    v = _rtt([4] * 4, 3, 24)
    got = tg.matvec(tg.DevTT.from_cores(op), tg.DevTT.from_cores(v)).cores()
    np.testing.assert_allclose(tt.full_vec(got), tt.full_vec(tt.matvec(op, v)), rtol=1e-12,
                               atol=1e-12 * np.abs(tt.full_vec(tt.matvec(op, v))).max())
    u, w = _rtt([4] * 6, 5, 25), _rtt([4] * 6, 3, 26)
    val = tg.inner(tg.DevTT.from_cores(u), tg.DevTT.from_cores(w))
    assert math.isclose(val, tt.inner(u, w), rel_tol=1e-11, abs_tol=1e-11)


@pytest.mark.parametrize("d,rk,seed", [(5, 6, 30), (8, 12, 31), (10, 20, 32), (6, 48, 33), (7, 40, 34)])
def test_round_ranks_and_error(d, rk, seed):
    base = _rtt([4] * d, max(2, rk // 3), seed)
    noise = tt.scale(_rtt([4] * d, rk, seed + 100), 1e-6)
    s = tt.add(base, noise)
    nrm = tt.norm(s)
    delta = 1e-4 * nrm
    ref, zeta_ref, ties = tt.round_tt(s, delta)
    got, zeta = tg.round_tt(tg.DevTT.from_cores(s), delta)
    # ranks bit-exact on bonds that are not ties
    for k, (rg, rr) in enumerate(zip(got.ranks, tt.ranks(ref))):
        if 0 < k < d and not ties[k - 1]:
            assert rg == rr, (k, got.ranks, tt.ranks(ref))
    assert math.isclose(zeta, zeta_ref, rel_tol=1e-8, abs_tol=1e-13 * nrm)
    if d <= 8:
        np.testing.assert_allclose(tt.full_vec(got.cores()), tt.full_vec(ref), atol=1e-10 * nrm)
    else:
        # the rounded tensor differs from the input by exactly zeta
        diff = tt.add(got.cores(), s, 1.0, -1.0)
        assert math.isclose(tt.norm(diff), zeta, rel_tol=1e-6, abs_tol=1e-12 * nrm)


def test_round_cap_and_degenerate():
    s = tt.add(_rtt([4] * 6, 5, 40), _rtt([4] * 6, 4, 41))
    ref, zr, _ = tt.round_tt(s, 0.0, cap=3)
    got, zg = tg.round_tt(tg.DevTT.from_cores(s), 0.0, cap=3)
    assert got.ranks == tt.ranks(ref)
    assert math.isclose(zg, zr, rel_tol=1e-9)
    # d = 1 and rank-1 inputs round to themselves
    one = [inputs.rng(42).standard_normal((1, 4, 1))]
    g1, z1 = tg.round_tt(tg.DevTT.from_cores(one), 1e-3)
    np.testing.assert_allclose(g1.cores()[0], one[0], atol=1e-15)
    assert z1 == 0.0


@pytest.mark.parametrize("n", [1, 31, 33, 200, 1100, 2300])
@pytest.mark.parametrize("prec", [tg.FP64, tg.MIXED_TF32])
def test_dense_local_solve(n, prec):
    # tt_lu_solve against numpy's solve of the same system: one panel, ragged
    # panels, the one-CTA shared-memory panel and (n = 2300 in FP64) the
    # cluster panel
    g = inputs.rng(17, n)
    K = g.standard_normal((n, n)) + 2.0 * np.sqrt(n) * np.eye(n)
    x = g.standard_normal(n)
    b = K @ x
    Kd, bd = _t(K), _t(b)
    res = tg.lu_solve(Kd, bd, prec)
    ref = np.linalg.solve(K, b)
    np.testing.assert_allclose(bd.cpu().numpy(), ref, rtol=0, atol=1e-10 * np.abs(ref).max())
    assert res <= 1e-10
    np.testing.assert_array_equal(Kd.cpu().numpy(), K)  # K is not modified


def _stress_inputs():
    # unfoldings with at least 16 columns and twice as many rows, where the
    # FP64 tall-skinny QR (CholeskyQR2) and the SVD's first-order Jacobi
    # finish meet their fallback conditions
    d = 6
    x = _rtt([4] * d, 20, 50)
    yield "rank-deficient", tt.add(x, x, 1.0, 0.5), 1e-6          # exact duplicate columns
    c = [core.copy() for core in x]
    c[2][:, :, 0] *= 1e-9                                           # an ill-conditioned core
    yield "ill-conditioned", c, 1e-3
    rep = [core.copy() for core in x]
    u, _, vt = np.linalg.svd(rep[3].reshape(-1, rep[3].shape[-1]), full_matrices=False)
    rep[3] = (u @ vt).reshape(rep[3].shape)                         # all singular values equal
    yield "repeated singular values", rep, 1e-4


@pytest.mark.parametrize("case", [0, 1, 2])
def test_round_fallback_paths_match_oracle(case):
    name, s, rel = list(_stress_inputs())[case]
    nrm = tt.norm(s)
    ref, zeta_ref, ties = tt.round_tt(s, rel * nrm)
    got, zeta = tg.round_tt(tg.DevTT.from_cores(s), rel * nrm)
    for k, (rg, rr) in enumerate(zip(got.ranks, tt.ranks(ref))):
        if 0 < k < len(s) and not ties[k - 1]:
            assert rg == rr, (name, k, got.ranks, tt.ranks(ref))
    assert math.isclose(zeta, zeta_ref, rel_tol=1e-6, abs_tol=1e-12 * nrm), (name, zeta, zeta_ref)
    # the rounded tensor differs from the input by zeta (dense check: a TT
    # difference norm cannot resolve 1e-10 of the input's norm)
    err = np.linalg.norm(tt.full_vec(got.cores()) - tt.full_vec(s))
    assert math.isclose(err, zeta, rel_tol=1e-4, abs_tol=1e-12 * nrm), (name, err, zeta)
