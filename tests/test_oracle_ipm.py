"""Pins for the oracle TT-IPM (O4) against the dense oracles O2 and O3."""
import math

import numpy as np
import pytest

from oracle import sdp_dense as sd, tt, tt_ipm, tt_problems as tp
from paper_2509_11890_gb300 import inputs


def _maxcut(d, seed):
    inst = inputs.maxcut_kron(d, seed)
    return inst, tp.maxcut(inst["adjacency_cores"], d)


def _state(ipm, seed):
    """A non-trivial interior point: perturb the initial X, Y, Z by low-rank symmetric TTs."""
    d = ipm.d
    g = [c * 0.05 for c in inputs.random_tt_matrix([2] * d, [2] * d, [1] + [2] * (d - 1) + [1], seed)]
    gs = tt.add(g, tt.transpose(g), 0.5, 0.5)
    ipm.X = tt.add(ipm.X, gs)
    ipm.Z = tt.add(ipm.Z, gs, 1.0, -0.5)
    ipm.Y = tt.hadamard(tt.identity(d), gs)


@pytest.mark.parametrize("direction", ["aho", "xz"])
def test_amen_direction_equals_dense_newton(direction):
    d = 3
    inst, prob = _maxcut(d, 0)
    o = tt_ipm.Options(rank_cap=64, kick=4, max_sweeps=8)
    ipm = tt_ipm.TTIPM(prob, o)
    _state(ipm, 5)
    ipm.eta = 1e-12
    mu = ipm.mu()
    X, Y, Z = (tt.full_mat(m) for m in (ipm.X, ipm.Y, ipm.Z))
    pad = sd.padded_maxcut(inst["weights"])
    (dX, dY, dZ), K, R = sd.newton_solve(pad, X, Y, Z, mu=mu, direction=direction, sigma=0.5)
    sig_mu = 0.5 * mu
    data = ipm.newton_data(direction, sig_mu, None, False, False)
    w, info = tt_ipm.amen_solve(data, d, None, 1e-12, 64, 4, 8, ipm.rnd)
    got = [tt.full_mat(tt.unvec_tt(w.component(b))) for b in range(3)]
    for a, b in zip(got, (dX, dY, dZ)):
        np.testing.assert_allclose(a, b, atol=1e-8 * (1 + np.abs(b).max()))
    # forcing condition of eq. forcing-condition, evaluated densely
    du = np.concatenate([tt.vec_tt_dense(m, d) for m in got])
    assert np.linalg.norm(K @ du + R) <= 1e-8 * np.linalg.norm(R)


def test_amen_truncated_direction_meets_forcing():
    d = 4
    inst, prob = _maxcut(d, 1)
    o = tt_ipm.Options(rank_cap=16, kick=2, max_sweeps=6)
    ipm = tt_ipm.TTIPM(prob, o)
    _state(ipm, 6)
    mu = ipm.mu()
    eta = 1e-3
    data = ipm.newton_data("aho", mu, None, False, False)
    w, info = tt_ipm.amen_solve(data, d, None, eta, 16, 2, 6, ipm.rnd)
    X, Y, Z = (tt.full_mat(m) for m in (ipm.X, ipm.Y, ipm.Z))
    K, R = sd.newton_system(sd.padded_maxcut(inst["weights"]), X, Y, Z, mu=mu, direction="aho", sigma=1.0)
    du = np.concatenate([tt.full_vec(w.component(b)) for b in range(3)])
    assert np.linalg.norm(K @ du + R) <= 10 * eta * np.linalg.norm(R)


@pytest.mark.parametrize("seed", [0, 1])
def test_als_step_length_matches_dense_rule(seed):
    d = 4
    g = inputs.random_tt_matrix([2] * d, [2] * d, [1, 2, 2, 2, 1], seed + 40)
    gs = tt.add(g, tt.transpose(g), 0.5, 0.5)
    shift = abs(np.linalg.eigvalsh(tt.full_mat(gs))[0]) + 1.0
    M = tt.add(tt.scale(tt.identity(d), shift), gs)
    h = inputs.random_tt_matrix([2] * d, [2] * d, [1, 2, 2, 2, 1], seed + 50)
    dM = tt.add(h, tt.transpose(h), 0.5, 0.5)
    Md, dMd = tt.full_mat(M), tt.full_mat(dM)
    assert np.linalg.eigvalsh(Md)[0] > 0
    ref = sd.max_step(Md, dMd)
    lam, e = tt_ipm.min_gen_eig(M, dM, None, tt_ipm.Counter(seed), rank=4, sweeps=8)
    # with rank 4 = full rank at the middle bond of d = 4 the ALS quotient is exact
    assert math.isclose(tt_ipm.step_from_lambda(lam), ref, rel_tol=1e-8)


def test_splitmix64_published_values():
    # first outputs of SplitMix64 seeded with 0 (reference values of the published generator)
    state = 0
    outs = []
    for _ in range(3):
        outs.append(tt_ipm.splitmix64(state))
        state = (state + 0x9E3779B97F4A7C15) & ((1 << 64) - 1)
    assert outs == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


@pytest.mark.parametrize("d,seed", [(3, 0), (4, 2)])
def test_ipm_maxcut_reaches_dense_optimum(d, seed):
    inst, prob = _maxcut(d, seed)
    ref = sd.solve_dense(sd.maxcut_sdp(inst["weights"]))
    ipm = tt_ipm.TTIPM(prob, tt_ipm.Options(rank_cap=16, max_iters=40))
    assert ipm.solve()
    h = ipm.history[-1]
    assert abs(h.pobj - ref.pobj) / (1 + abs(ref.pobj)) <= 2e-3
    assert h.rel_gap <= 1e-4 / math.sqrt(d)
    # X stays positive definite (dense check, Corollary psdness_rounding shift)
    assert np.linalg.eigvalsh(tt.full_mat(ipm.X))[0] > 0


def test_ipm_theta_reaches_dense_optimum():
    d = 3
    inst = inputs.theta_hypercube_kron(d, 0)
    prob = tp.theta(tp.graph_tt(inst["adjacency"]), d)
    ref = sd.solve_dense(sd.theta_sdp(inst["adjacency"]))
    ipm = tt_ipm.TTIPM(prob, tt_ipm.Options(rank_cap=16, max_iters=60))
    ok = ipm.solve()
    h = ipm.history[-1]
    assert ok, h
    assert abs(h.pobj - ref.pobj) / (1 + abs(ref.pobj)) <= 5e-3


def test_ipm_cc_reaches_dense_optimum():
    d = 3
    inst = inputs.cc_signed(d, 1)
    prob = tp.corr_clustering(tp.graph_tt(inst["c_plus"]), tp.graph_tt(inst["c_minus"]),
                              tp.graph_tt(inst["adjacency"]), d)
    ref = sd.solve_dense(sd.cc_sdp(inst["c_plus"], inst["c_minus"], inst["adjacency"]))
    ipm = tt_ipm.TTIPM(prob, tt_ipm.Options(rank_cap=16, max_iters=60))
    ok = ipm.solve()
    h = ipm.history[-1]
    assert ok, h
    assert abs(h.pobj - ref.pobj) / (1 + abs(ref.pobj)) <= 5e-3
