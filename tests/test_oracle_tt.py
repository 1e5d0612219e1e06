"""Pins for the oracle's TT algebra (O1) against definitions fixed outside it.

Each test compares the oracle with an independent construction: numpy's
Kronecker product, dense matrix algebra on reconstructed tensors, the
paper's printed worked example, or Eckart-Young optimality of the SVD.
"""
import math
import os

import numpy as np
import pytest

from oracle import tt
from paper_2509_11890_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_tt(dims, rk, seed):
    ranks = [1] + [rk] * (len(dims) - 1) + [1]
    return inputs.random_tt(dims, ranks, seed)


def _rand_ttm(d, rk, seed, m=2, n=2):
    ranks = [1] + [rk] * (d - 1) + [1]
    return inputs.random_tt_matrix([m] * d, [n] * d, ranks, seed)


def test_worked_example_vec_and_vec_tt():
    # Section 3.1 worked example, printed values (golden file)
    rows = [list(map(float, ln.split())) for ln in open(os.path.join(GOLDEN, "vec_tt_example.txt")) if not ln.startswith("#")]
    m = np.array([[1, 1, 2, 2], [1, 1, 2, 2], [3, 3, 4, 4], [3, 3, 4, 4]], dtype=float)
    assert np.array_equal(tt.vec(m), np.array(rows[1]))
    assert np.array_equal(tt.vec_tt_dense(m, 2), np.array(rows[2]))
    # the same through TT cores: M = [[1,2],[3,4]] kron J_2 has TT rank 1
    cores = [np.array([[1.0, 2.0], [3.0, 4.0]]).reshape(1, 2, 2, 1), np.ones((1, 2, 2, 1))]
    assert np.array_equal(tt.full_mat(cores), m)
    assert np.array_equal(tt.full_vec(tt.vec_tt(cores)), np.array(rows[2]))


def test_full_mat_matches_numpy_kron():
    g = inputs.rng(11)
    facs = [g.standard_normal((2, 3)) for _ in range(4)]
    cores = [f.reshape(1, 2, 3, 1) for f in facs]
    ref = facs[0]
    for f in facs[1:]:
        ref = np.kron(ref, f)
    np.testing.assert_allclose(tt.full_mat(cores), ref, rtol=0, atol=1e-14)


def test_full_vec_matches_numpy_kron_and_sums():
    g = inputs.rng(12)
    a = [g.standard_normal(3) for _ in range(5)]
    b = [g.standard_normal(3) for _ in range(5)]
    ref = a[0]
    ref2 = b[0]
    for x, y in zip(a[1:], b[1:]):
        ref = np.kron(ref, x)
        ref2 = np.kron(ref2, y)
    ca = [x.reshape(1, 3, 1) for x in a]
    cb = [y.reshape(1, 3, 1) for y in b]
    np.testing.assert_allclose(tt.full_vec(tt.add(ca, cb, 2.0, -0.5)), 2.0 * ref - 0.5 * ref2, atol=1e-13)


def test_tt_svd_reconstructs_and_finds_ranks():
    t = _rand_tt([2, 3, 2, 4, 2, 3], 3, seed=3)
    full = tt.full_vec(t)
    c = tt.tt_svd(full, [2, 3, 2, 4, 2, 3])
    np.testing.assert_allclose(tt.full_vec(c), full, atol=1e-12 * np.linalg.norm(full))
    assert max(tt.ranks(c)) <= 3
    # a Kronecker (rank-1) matrix has TT rank 1 in vec_TT form
    kr = [np.array([[1.0, 2.0], [0.5, -1.0]]).reshape(1, 2, 2, 1)] * 5
    dense = tt.full_mat(kr)
    c2 = tt.tt_svd(tt.vec_tt_dense(dense, 5), [4] * 5)
    assert tt.ranks(c2) == [1] * 6


def test_frame_identity_remark():
    # Remark after Definition "Frame Matrix": vec(T) = T_{!=k} vec(T_k)
    t = _rand_tt([2, 3, 4, 2, 3], 3, seed=5)
    full = tt.full_vec(t)
    for k in range(5):
        np.testing.assert_allclose(tt.frame(t, k) @ t[k].reshape(-1), full, atol=1e-12)


def test_vec_tt_permutation_matches_cores():
    a = _rand_ttm(4, 3, seed=6)
    dense = tt.full_mat(a)
    np.testing.assert_allclose(tt.full_vec(tt.vec_tt(a)), tt.vec_tt_dense(dense, 4), atol=1e-12)
    np.testing.assert_allclose(tt.unvec_tt_dense(tt.vec_tt_dense(dense, 4), 4), dense, atol=0)


def test_hadamard_remark_diag_tt():
    # Remark of Section 3.3: vec_TT(M . N) = diag_TT(vec_TT(M)) vec_TT(N)
    m = _rand_ttm(4, 2, seed=7)
    n = _rand_ttm(4, 3, seed=8)
    ref = tt.vec_tt_dense(tt.full_mat(m) * tt.full_mat(n), 4)
    via_diag = tt.full_vec(tt.matvec(tt.diag_tt(tt.vec_tt(m)), tt.vec_tt(n)))
    via_core = tt.full_vec(tt.vec_tt(tt.hadamard(m, n)))
    np.testing.assert_allclose(via_diag, ref, atol=1e-11)
    np.testing.assert_allclose(via_core, ref, atol=1e-11)
    # diag_TT of a vector is the dense diagonal matrix of that vector
    v = _rand_tt([4] * 3, 2, seed=9)
    np.testing.assert_allclose(tt.full_mat(tt.diag_tt(v)), np.diag(tt.full_vec(v)), atol=1e-12)


def test_kron_acts_as_a_x_bt():
    # (A kron B) vec_TT(X) = vec_TT(A X B^T) for the core-wise Kronecker product
    a = _rand_ttm(3, 2, seed=10)
    b = _rand_ttm(3, 2, seed=11)
    x = _rand_ttm(3, 3, seed=12)
    A, B, X = tt.full_mat(a), tt.full_mat(b), tt.full_mat(x)
    lhs = tt.full_mat(tt.kron(a, b)) @ tt.vec_tt_dense(X, 3)
    np.testing.assert_allclose(lhs, tt.vec_tt_dense(A @ X @ B.T, 3), atol=1e-10)
    # and with the standard vec it is numpy's Kronecker product
    perm = tt.vec_tt_permutation(3)
    K = np.kron(A, B)
    np.testing.assert_allclose(tt.full_mat(tt.kron(a, b))[np.ix_(np.argsort(perm), np.argsort(perm))], K, atol=1e-10)


def test_matmul_matvec_transpose():
    a = _rand_ttm(4, 2, seed=13)
    b = _rand_ttm(4, 3, seed=14)
    np.testing.assert_allclose(tt.full_mat(tt.matmul(a, b)), tt.full_mat(a) @ tt.full_mat(b), atol=1e-10)
    np.testing.assert_allclose(tt.full_mat(tt.transpose(a)), tt.full_mat(a).T, atol=0)
    x = _rand_tt([2] * 4, 2, seed=15)
    np.testing.assert_allclose(tt.full_vec(tt.matvec(a, x)), tt.full_mat(a) @ tt.full_vec(x), atol=1e-10)


def test_inner_and_norm():
    u = _rand_tt([4] * 5, 3, seed=16)
    v = _rand_tt([4] * 5, 2, seed=17)
    assert math.isclose(tt.inner(u, v), float(tt.full_vec(u) @ tt.full_vec(v)), rel_tol=1e-12, abs_tol=1e-10)
    assert math.isclose(tt.norm(u), float(np.linalg.norm(tt.full_vec(u))), rel_tol=1e-12)


def test_environments_equal_dense_frame_projection():
    # Section 3.3 local products: environments reproduce U_{!=k}^T Op V_{!=k}
    d = 4
    u = tt.orth_left(_rand_tt([4] * d, 3, seed=18))
    v = _rand_tt([4] * d, 2, seed=19)
    op = inputs.random_tt_matrix([4] * d, [4] * d, [1, 2, 3, 2, 1], seed=20)
    left = tt.envs_left(u, op, v)
    right = tt.envs_right(u, op, v)
    for k in range(d):
        dense = tt.local_matrix_by_frame(u, op, v, k)
        np.testing.assert_allclose(tt.local_matrix(left[k], op[k], right[k + 1]), dense, atol=1e-10)
        x = inputs.rng(21 + k).standard_normal(v[k].shape)
        np.testing.assert_allclose(tt.local_apply(left[k], op[k], right[k + 1], x).reshape(-1), dense @ x.reshape(-1), atol=1e-10)
    # the full chain contracts to <u, Op v>
    full = tt.full_vec(u) @ tt.full_mat(op) @ tt.full_vec(v)
    assert math.isclose(float(left[d][0, 0, 0]), float(full), rel_tol=1e-11, abs_tol=1e-11)
    assert math.isclose(float(right[0][0, 0, 0]), float(full), rel_tol=1e-11, abs_tol=1e-11)


def test_orthogonalisation():
    t = _rand_tt([4] * 5, 4, seed=22)
    full = tt.full_vec(t)
    r = tt.orth_right(t)
    l = tt.orth_left(t)
    np.testing.assert_allclose(tt.full_vec(r), full, atol=1e-10)
    np.testing.assert_allclose(tt.full_vec(l), full, atol=1e-10)
    for k in range(1, 5):
        m = r[k].reshape(r[k].shape[0], -1)
        np.testing.assert_allclose(m @ m.T, np.eye(m.shape[0]), atol=1e-12)
    for k in range(4):
        m = l[k].reshape(-1, l[k].shape[-1])
        np.testing.assert_allclose(m.T @ m, np.eye(m.shape[1]), atol=1e-12)


def test_rounding_error_and_eckart_young():
    # exact rank-2 tensor plus a small perturbation: rounding returns rank 2
    base = _rand_tt([4] * 5, 2, seed=23)
    noise = tt.scale(_rand_tt([4] * 5, 3, seed=24), 1e-7)
    s = tt.add(base, noise)
    full = tt.full_vec(s)
    nrm = np.linalg.norm(full)
    rounded, zeta, ties = tt.round_tt(s, 1e-4 * nrm)
    assert max(tt.ranks(rounded)) == 2
    err = np.linalg.norm(tt.full_vec(rounded) - full)
    assert math.isclose(zeta, err, rel_tol=1e-6, abs_tol=1e-12 * nrm)
    assert zeta <= 1e-4 * nrm
    assert not any(ties)
    # with no truncation possible the rounded tensor is exact
    r2, z2, _ = tt.round_tt(base, 1e-12)
    np.testing.assert_allclose(tt.full_vec(r2), tt.full_vec(base), atol=1e-10)
    # Eckart-Young at the first bond: error at fixed cap equals the SVD tail
    r3, z3, _ = tt.round_tt(s, 0.0, cap=1)
    mat = full.reshape(4, -1)
    sv = np.linalg.svd(mat, compute_uv=False)
    assert z3 >= math.sqrt(float(np.sum(sv[1:] ** 2))) * (1 - 1e-9)
    assert math.isclose(np.linalg.norm(tt.full_vec(r3) - full), z3, rel_tol=1e-8)


def test_rounding_cap_and_ranks_bound():
    t = _rand_tt([4] * 6, 5, seed=25)
    t2 = tt.add(t, _rand_tt([4] * 6, 4, seed=26))
    r, zeta, _ = tt.round_tt(t2, 0.0, cap=6)
    assert max(tt.ranks(r)) <= 6
    assert math.isclose(np.linalg.norm(tt.full_vec(r) - tt.full_vec(t2)), zeta, rel_tol=1e-8)


def test_identity_ones_unit():
    np.testing.assert_array_equal(tt.full_mat(tt.identity(3)), np.eye(8))
    np.testing.assert_array_equal(tt.full_mat(tt.ones_mat(3)), np.ones((8, 8)))
    e = tt.full_mat(tt.unit_mat([1, 0, 1], [0, 0, 1]))
    ref = np.zeros((8, 8))
    ref[5, 1] = 1
    np.testing.assert_array_equal(e, ref)
    u = _rand_tt([4] * 3, 2, seed=27)
    v = _rand_tt([4] * 3, 1, seed=28)
    np.testing.assert_allclose(tt.full_mat(tt.outer(u, v)), np.outer(tt.full_vec(u), tt.full_vec(v)), atol=1e-12)
