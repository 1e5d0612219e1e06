"""Tensor-core (tcgen05, TF32 / BF16 inputs, FP32 accumulation) contractions against the oracle.

Tolerances follow from the input rounding: TF32 keeps 10 mantissa bits (unit
roundoff 2^-11), BF16 7 (2^-8); every term of the contraction is a product of
four rounded operands whose intermediate sums are rounded again between the
stages (at most six roundings of 2^-11 or 2^-8 on each term), so every output
entry stays within 5e-3 (TF32) or 3e-2 (BF16) of the exact value relative to
the same contraction of the operands' absolute values, element by element.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2509_11890_gb300 as tg  # noqa: E402
from oracle import tt  # noqa: E402
from paper_2509_11890_gb300 import inputs  # noqa: E402

SHAPES = [
    (3, 70, 5, 33, 2, 65, 4, 4),
    (17, 9, 7, 3, 66, 5, 4, 4),
    (16, 16, 32, 32, 16, 16, 4, 4),
    (64, 64, 128, 128, 64, 64, 4, 4),
    (33, 40, 65, 65, 33, 40, 4, 4),
]
TOL = {tg.MIXED_TF32: 5e-3, tg.MIXED_BF16: 3e-2}


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _rand(shape, seed):
    return inputs.rng(seed, 78).standard_normal(shape)


def _dims(s):
    return dict(zip(["rw", "rw2", "R", "R2", "rv", "rv2", "m", "n"], s))


def assert_bounded(got, ref, ref_abs, tol):
    """|got - ref| <= tol * ref_abs, element by element."""
    got = got.reshape(ref.shape)
    bound = tol * ref_abs + 1e-300
    bad = np.abs(got - ref) > bound
    assert not bad.any(), (int(bad.sum()), float(np.max(np.abs(got - ref) / bound)))


@pytest.mark.parametrize("prec", [tg.MIXED_TF32, tg.MIXED_BF16])
@pytest.mark.parametrize("shape", SHAPES)
def test_env_left_step_tensor_cores(shape, prec):
    rw, rw2, R, R2, rv, rv2, m, n = shape
    phi, u = _rand((rw, R, rv), 1), _rand((rw, m, rw2), 2)
    op, v = _rand((R, m, n, R2), 3), _rand((rv, n, rv2), 4)
    ref = tt.env_left_step(phi, u, op, v)
    ref_abs = tt.env_left_step(np.abs(phi), np.abs(u), np.abs(op), np.abs(v))
    out = torch.empty(rw2 * R2 * rv2, dtype=torch.float64, device="cuda")
    tg.env_left_step(_dims(shape), _t(phi), _t(u), _t(op), _t(v), out, prec)
    assert_bounded(out.cpu().numpy(), ref, ref_abs, TOL[prec])


@pytest.mark.parametrize("prec", [tg.MIXED_TF32, tg.MIXED_BF16])
@pytest.mark.parametrize("shape", SHAPES)
def test_env_right_step_tensor_cores(shape, prec):
    rw, rw2, R, R2, rv, rv2, m, n = shape
    psi, u = _rand((rw2, R2, rv2), 5), _rand((rw, m, rw2), 6)
    op, v = _rand((R, m, n, R2), 7), _rand((rv, n, rv2), 8)
    ref = tt.env_right_step(psi, u, op, v)
    ref_abs = tt.env_right_step(np.abs(psi), np.abs(u), np.abs(op), np.abs(v))
    out = torch.empty(rw * R * rv, dtype=torch.float64, device="cuda")
    tg.env_right_step(_dims(shape), _t(psi), _t(u), _t(op), _t(v), out, prec)
    assert_bounded(out.cpu().numpy(), ref, ref_abs, TOL[prec])


@pytest.mark.parametrize("prec", [tg.MIXED_TF32, tg.MIXED_BF16])
@pytest.mark.parametrize("shape", SHAPES)
def test_scaled_operands_keep_the_relative_error(shape, prec):
    # per-core norm scaling: operands far outside the FP32 range (1e-42 is
    # below its smallest normal number, 1e+35 times 1e+25 above its largest)
    # give the same relative error as unit-scaled ones
    rw, rw2, R, R2, rv, rv2, m, n = shape
    phi, u = _rand((rw, R, rv), 1) * 1e-42, _rand((rw, m, rw2), 2) * 1e25
    op, v = _rand((R, m, n, R2), 3) * 1e-3, _rand((rv, n, rv2), 4) * 1e35
    ref = tt.env_left_step(phi, u, op, v)
    ref_abs = tt.env_left_step(np.abs(phi), np.abs(u), np.abs(op), np.abs(v))
    out = torch.empty(rw2 * R2 * rv2, dtype=torch.float64, device="cuda")
    tg.env_left_step(_dims(shape), _t(phi), _t(u), _t(op), _t(v), out, prec)
    assert_bounded(out.cpu().numpy(), ref, ref_abs, TOL[prec])


@pytest.mark.parametrize("prec", [tg.MIXED_TF32, tg.MIXED_BF16])
@pytest.mark.parametrize("shape", SHAPES)
def test_local_apply_tensor_cores(shape, prec):
    rw, rw2, R, R2, rv, rv2, m, n = shape
    phi, psi = _rand((rw, R, rv), 9), _rand((rw2, R2, rv2), 10)
    op, x = _rand((R, m, n, R2), 11), _rand((rv, n, rv2), 12)
    ref = tt.local_apply(phi, op, psi, x)
    ref_abs = tt.local_apply(np.abs(phi), np.abs(op), np.abs(psi), np.abs(x))
    y = torch.empty(rw * m * rw2, dtype=torch.float64, device="cuda")
    tg.local_apply(_dims(shape), _t(phi), _t(op), _t(psi), _t(x), y, prec)
    assert_bounded(y.cpu().numpy(), ref, ref_abs, TOL[prec])


def test_solver_tf32_reaches_optimum():
    from oracle import sdp_dense as sd
    d = 4
    inst = inputs.maxcut_kron(d, 2)
    ref = sd.solve_dense(sd.maxcut_sdp(inst["weights"]))
    ctx = tg.Context.maxcut(inst["adjacency_cores"], tg.default_options(rank_cap=16, max_iters=40,
                                                                         precision=tg.MIXED_TF32))
    res = ctx.solve()
    assert res["status"] == 0, res
    assert abs(res["pobj"] - ref.pobj) / (1 + abs(ref.pobj)) <= 2e-3
