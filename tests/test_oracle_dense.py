"""Pins for the dense SDP oracle (O2) and the dense Newton oracle (O3).

O2 is checked against closed-form SDP values, brute-force combinatorial
bounds and duality invariants; O3 against the linearisation it claims to be
(a finite-difference check of the KKT residual map) and the dense step rule.
"""
import math

import numpy as np
import pytest

from oracle import brute, sdp_dense as sd, tt
from paper_2509_11890_gb300 import inputs


def _cycle(n):
    a = np.zeros((n, n))
    for i in range(n):
        a[i, (i + 1) % n] = a[(i + 1) % n, i] = 1
    return a


def _complete(n):
    return np.ones((n, n)) - np.eye(n)


def _hypercube(d):
    return inputs.hypercube_dense(d).astype(float)


def _solve(p, **kw):
    r = sd.solve_dense(p, **kw)
    assert max(r.rel_gap, r.rel_p, r.rel_d) <= 1e-8, (r.rel_gap, r.rel_p, r.rel_d)
    return r


@pytest.mark.parametrize("n", [4, 8, 16])
def test_maxcut_complete_graph(n):
    r = _solve(sd.maxcut_sdp(_complete(n)))
    assert math.isclose(r.pobj, n * n / 4.0, rel_tol=1e-7)


@pytest.mark.parametrize("n", [5, 7, 9])
def test_maxcut_odd_cycle(n):
    r = _solve(sd.maxcut_sdp(_cycle(n)))
    assert math.isclose(r.pobj, n / 2.0 * (1 + math.cos(math.pi / n)), rel_tol=1e-7)


@pytest.mark.parametrize("d", [3, 4])
def test_maxcut_hypercube_is_bipartite(d):
    a = _hypercube(d)
    r = _solve(sd.maxcut_sdp(a))
    assert math.isclose(r.pobj, a.sum() / 2.0, rel_tol=1e-7)


def test_maxcut_cayley_graph_eigen_bound():
    # A = sum_{s in S} kron_k sigma_x^{s_k}: SDP value = N lambda_max(L) / 4
    d = 4
    sx = np.array([[0.0, 1.0], [1.0, 0.0]])
    S = [(1, 0, 0, 1), (0, 1, 1, 0), (1, 1, 1, 0)]
    a = np.zeros((2**d, 2**d))
    for s in S:
        m = np.ones((1, 1))
        for bit in s:
            m = np.kron(m, sx if bit else np.eye(2))
        a += m
    L = sd.laplacian(a)
    r = _solve(sd.maxcut_sdp(a))
    assert math.isclose(r.pobj, 2**d * np.linalg.eigvalsh(L)[-1] / 4.0, rel_tol=1e-7)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_maxcut_brute_force_bounds(seed):
    g = inputs.rng(seed, 99)
    n = 10
    w = np.triu(g.uniform(0.5, 1.5, (n, n)) * (g.random((n, n)) < 0.5), 1)
    w = w + w.T
    r = _solve(sd.maxcut_sdp(w))
    mc = brute.max_cut(w)
    lam = np.linalg.eigvalsh(sd.laplacian(w))[-1]
    assert mc <= r.pobj * (1 + 1e-8)
    assert r.pobj <= n * lam / 4.0 * (1 + 1e-8)
    # the SDP relaxation of Goemans-Williamson is within 1/0.878 of the cut
    assert r.pobj <= mc / 0.87856 + 1e-6


def test_theta_closed_forms():
    assert math.isclose(_solve(sd.theta_sdp(_complete(6))).pobj, 1.0, rel_tol=1e-7)
    assert math.isclose(_solve(sd.theta_sdp(np.zeros((6, 6)))).pobj, 6.0, rel_tol=1e-7)
    assert math.isclose(_solve(sd.theta_sdp(_cycle(5))).pobj, math.sqrt(5.0), rel_tol=1e-7)
    c = math.cos(math.pi / 7)
    assert math.isclose(_solve(sd.theta_sdp(_cycle(7))).pobj, 7 * c / (1 + c), rel_tol=1e-7)
    assert math.isclose(_solve(sd.theta_sdp(_hypercube(3))).pobj, 4.0, rel_tol=1e-7)


def test_theta_vertex_transitive_product_and_stability_bound():
    # Lovasz 1979: theta(G) theta(complement G) = n for vertex-transitive G
    a = _hypercube(3)
    ac = _complete(8) - a
    t1 = _solve(sd.theta_sdp(a)).pobj
    t2 = _solve(sd.theta_sdp(ac)).pobj
    assert math.isclose(t1 * t2, 8.0, rel_tol=1e-6)
    g = inputs.rng(5, 98)
    n = 10
    adj = np.triu((g.random((n, n)) < 0.3).astype(float), 1)
    adj = adj + adj.T
    th = _solve(sd.theta_sdp(adj)).pobj
    assert brute.stability_number(adj.astype(int)) <= th * (1 + 1e-8)


def test_cc_closed_forms_and_brute_force():
    n = 6
    allpos = _complete(n)
    r = _solve(sd.cc_sdp(allpos, np.zeros((n, n)), _complete(n)))
    assert math.isclose(r.pobj, allpos.sum(), rel_tol=1e-7)
    r = _solve(sd.cc_sdp(np.zeros((n, n)), allpos, _complete(n)))
    assert math.isclose(r.pobj, np.trace(sd.laplacian(allpos)), rel_tol=1e-7)
    g = inputs.rng(3, 97)
    w = np.triu(np.where(g.random((n, n)) < 0.5, 1.0, -1.0), 1)
    w = w + w.T
    cp, cm = np.where(w > 0, w, 0), np.where(w < 0, -w, 0)
    r = _solve(sd.cc_sdp(cp, cm, _complete(n)))
    assert 2.0 * brute.cc_integer(cp, cm) <= r.pobj * (1 + 1e-8)
    # the optimum is entrywise nonnegative and psd with unit diagonal
    assert r.X.min() >= -1e-7
    np.testing.assert_allclose(np.diag(r.X), 1.0, atol=1e-7)


def test_duality_invariants():
    inst = inputs.maxcut_kron(5, 0)
    p = sd.maxcut_sdp(inst["weights"])
    r = _solve(p)
    # weak duality and complementarity at the optimum
    assert r.dobj >= r.pobj - 1e-6 * (1 + abs(r.pobj))
    assert abs(np.sum(r.X * r.Z)) <= 1e-6 * (1 + abs(r.pobj))
    assert np.linalg.eigvalsh(r.X)[0] >= -1e-8 and np.linalg.eigvalsh(r.Z)[0] >= -1e-8


def test_max_step_rule():
    # Theorem "Optimal Step Size" against bisection on the smallest eigenvalue
    g = inputs.rng(4, 96)
    a = g.standard_normal((6, 6))
    M = a @ a.T + 0.5 * np.eye(6)
    dM = g.standard_normal((6, 6))
    dM = dM + dM.T
    alpha = sd.max_step(M, dM)
    assert np.linalg.eigvalsh(M + 0.999999 * alpha * dM)[0] > 0
    assert np.linalg.eigvalsh(M + 1.000001 * alpha * dM)[0] < 0
    assert sd.max_step(M, np.eye(6)) == math.inf


def _spd(n, seed, scale=1.0):
    g = inputs.rng(seed, 95)
    a = g.standard_normal((n, n))
    return a @ a.T / n + scale * np.eye(n)


@pytest.mark.parametrize("direction", ["aho", "xz"])
def test_newton_system_is_the_linearisation(direction):
    # O3: K dU equals the directional derivative of the KKT residual map
    inst = inputs.maxcut_kron(3, 1)
    p = sd.padded_maxcut(inst["weights"])
    N = 8
    X, Z = _spd(N, 1), _spd(N, 2)
    Y = np.diag(inputs.rng(3, 94).standard_normal(N))
    mu = 0.3
    K, R = sd.newton_system(p, X, Y, Z, mu=mu, direction=direction)
    g = inputs.rng(7, 93)
    dX = g.standard_normal((N, N)); dX = dX + dX.T
    dY = np.diag(g.standard_normal(N))
    dZ = g.standard_normal((N, N)); dZ = dZ + dZ.T
    h = 1e-6
    _, Rp = sd.newton_system(p, X + h * dX, Y + h * dY, Z + h * dZ, mu=mu, direction=direction)
    _, Rm = sd.newton_system(p, X - h * dX, Y - h * dY, Z - h * dZ, mu=mu, direction=direction)
    fd = (Rp - Rm) / (2 * h)
    du = np.concatenate([tt.vec_tt_dense(m, 3) for m in (dX, dY, dZ)])
    np.testing.assert_allclose(K @ du, fd, atol=1e-6 * (1 + np.abs(fd).max()))


def test_newton_solution_satisfies_block_rows_dense():
    # the exact Newton direction of the padded system for Max-Cut keeps
    # diag(X + dX) = 1 and dY on the diagonal, and linearises XZ + ZX = 2 mu I
    inst = inputs.maxcut_kron(3, 2)
    p = sd.padded_maxcut(inst["weights"])
    N = 8
    X, Z = _spd(N, 3), _spd(N, 4)
    Y = np.zeros((N, N))
    (dX, dY, dZ), K, R = sd.newton_solve(p, X, Y, Z, mu=0.2, direction="aho")
    np.testing.assert_allclose(np.diag(X + dX), 1.0, atol=1e-10)
    np.testing.assert_allclose(dY - np.diag(np.diag(dY)), 0.0, atol=1e-10)
    lin = (X @ Z + Z @ X) + (dX @ Z + Z @ dX) + (X @ dZ + dZ @ X)
    np.testing.assert_allclose(lin, 2 * 0.2 * np.eye(N), atol=1e-9)
    np.testing.assert_allclose(dZ, dY - (Z + p.C - Y), atol=1e-10)


def test_padded_cc_newton_rows():
    n = 8
    w = inputs.cc_signed(3, 0)
    p = sd.padded_cc(w["c_plus"], w["c_minus"], w["adjacency"])
    X = np.eye(n) + 0.05 * (np.ones((n, n)) - np.eye(n))
    Z = 2.0 * np.eye(n)
    T = 1e-3 * (np.ones((n, n)) - np.eye(n))
    Y = np.zeros((n, n))
    (dX, dY, dT, dZ), K, R = sd.newton_solve(p, X, Y, Z, T, mu=0.1, direction="aho")
    # complementarity of the inequality block: (T + dT) s + T A dX = mu on edges (linearised)
    s = X * (1 - np.eye(n))
    lin = T * s + dT * s + T * (dX * (1 - np.eye(n)))
    off = ~np.eye(n, dtype=bool)
    np.testing.assert_allclose(lin[off], 0.1, atol=1e-9)
    np.testing.assert_allclose(np.diag(dT), 0.0, atol=1e-10)
