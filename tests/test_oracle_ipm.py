"""Pins for the oracle TT-IPM (O4) against the dense oracles O2 and O3."""
import math

import numpy as np
import scipy.linalg
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
    w, _, info = tt_ipm.amen_solve(data, d, None, 1e-12, 64, 4, 8, ipm.rnd)
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
    w, _, info = tt_ipm.amen_solve(data, d, None, eta, 16, 2, 6, ipm.rnd)
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


def _pd_pair(d, seed, rank=2):
    g = inputs.random_tt_matrix([2] * d, [2] * d, [1] + [rank] * (d - 1) + [1], seed + 40)
    gs = tt.add(g, tt.transpose(g), 0.5, 0.5)
    shift = abs(np.linalg.eigvalsh(tt.full_mat(gs))[0]) + 1.0
    M = tt.add(tt.scale(tt.identity(d), shift), gs)
    h = inputs.random_tt_matrix([2] * d, [2] * d, [1] + [rank] * (d - 1) + [1], seed + 50)
    dM = tt.add(h, tt.transpose(h), 0.5, 0.5)
    return M, dM


@pytest.mark.parametrize("k", [0, 1, 2])
def test_merged_operator_cores_define_the_same_matrix(k):
    d = 4
    M, _ = _pd_pair(d, 3)
    merged = M[:k] + [tt_ipm.merge_op_cores(M, k)] + M[k + 2:]
    np.testing.assert_allclose(tt.full_mat(merged), tt.full_mat(M), rtol=0, atol=1e-12)


@pytest.mark.parametrize("seed", [0, 1])
def test_dmrg_step_length_matches_dense_rule(seed):
    # rank 4 is full rank at every bond of d = 4: the two-site quotient is exact
    d = 4
    M, dM = _pd_pair(d, seed)
    ref = sd.max_step(tt.full_mat(M), tt.full_mat(dM))
    lam, e = tt_ipm.min_gen_eig_dmrg(M, dM, None, tt_ipm.Counter(seed), rank=4, sweeps=4)
    assert math.isclose(tt_ipm.step_from_lambda(lam), ref, rel_tol=1e-8)
    # the returned vector attains the returned quotient
    ev = tt.full_vec(e)
    Md, dMd = tt.full_mat(M), tt.full_mat(dM)
    assert math.isclose(ev @ dMd @ ev / (ev @ Md @ ev), lam, rel_tol=1e-8, abs_tol=1e-12)


@pytest.mark.parametrize("seed", [2, 3, 4])
def test_dmrg_finds_rank_one_extreme_eigenvector(seed):
    # M = I, dM = diag(v): the minimum quotient is min(v), attained at a unit
    # vector (TT rank one), found by two-site sweeps with rank 2
    d = 6
    v = inputs.random_tt([2] * d, [1] + [2] * (d - 1) + [1], seed)
    M = tt.identity(d)
    dM = tt.diag_tt(v)
    lam, e = tt_ipm.min_gen_eig_dmrg(M, dM, None, tt_ipm.Counter(seed), rank=2, sweeps=6)
    vmin = float(np.min(tt.full_vec(v)))
    assert math.isclose(lam, vmin, rel_tol=1e-8, abs_tol=1e-10)


def test_dmrg_quotient_bounds_the_dense_minimum_from_above():
    d = 6
    M, dM = _pd_pair(d, 7, rank=3)
    dense = float(scipy.linalg.eigh(tt.full_mat(dM), tt.full_mat(M), eigvals_only=True)[0])
    lam, _ = tt_ipm.min_gen_eig_dmrg(M, dM, None, tt_ipm.Counter(7), rank=2, sweeps=4)
    assert lam >= dense - 1e-10
    lam8, _ = tt_ipm.min_gen_eig_dmrg(M, dM, None, tt_ipm.Counter(7), rank=8, sweeps=4)
    assert lam8 >= dense - 1e-10 and lam8 <= lam + 1e-12
    assert math.isclose(lam8, dense, rel_tol=1e-6)


def test_dmrg_keep_rule():
    s = np.array([1.0, 1e-3, 1e-6, 1e-9])
    assert tt_ipm.dmrg_keep(s, 1e-8, 10) == 3
    assert tt_ipm.dmrg_keep(s, 1e-4, 10) == 2
    assert tt_ipm.dmrg_keep(s, 1e-8, 2) == 2
    assert tt_ipm.dmrg_keep(np.array([1.0]), 1e-8, 4) == 1


@pytest.mark.parametrize("two_site", [True, False])
def test_indefinite_iterate_raises(two_site):
    d = 4
    M, dM = _pd_pair(d, 0)
    Mneg = tt.add(M, tt.identity(d), 1.0, -100.0)
    fn = tt_ipm.min_gen_eig_dmrg if two_site else tt_ipm.min_gen_eig
    with pytest.raises(tt_ipm.NotPositiveDefinite):
        fn(Mneg, dM, None, tt_ipm.Counter(0), 4, 2)


def test_damp_and_retry_repairs_an_update_that_left_the_cone():
    # plant an overlong step after the first iteration: the next step-length
    # solve finds X outside the cone, the update is redone with halved steps
    # until X is positive definite again, and the solve still reaches the optimum
    d, seed = 4, 2
    inst, prob = _maxcut(d, seed)
    ref = sd.solve_dense(sd.maxcut_sdp(inst["weights"]))
    ipm = tt_ipm.TTIPM(prob, tt_ipm.Options(rank_cap=16, max_iters=40))
    assert ipm.iterate(0) is not None
    lam0 = np.linalg.eigvalsh(tt.full_mat(ipm.prev["dX"]))[0]
    assert lam0 < 0
    # a step three times past the boundary of the cone along dX
    ipm.prev["ap"] = 3.0 * tt_ipm.step_from_lambda(
        float(scipy.linalg.eigh(tt.full_mat(ipm.prev["dX"]), tt.full_mat(ipm.prev["X"]), eigvals_only=True)[0]))
    ipm._apply_update()
    assert np.linalg.eigvalsh(tt.full_mat(ipm.X))[0] < 0
    for it in range(1, 41):
        if ipm.iterate(it) is None:
            break
    assert ipm.retries >= 1
    assert np.linalg.eigvalsh(tt.full_mat(ipm.X))[0] > 0
    h = ipm.history[-1]
    assert abs(h.pobj - ref.pobj) / (1 + abs(ref.pobj)) <= 2e-3


def test_warm_start_frame_stays_within_the_rank_cap():
    # the solution is read where the last sweep ended; the warm start moved
    # back to core 0 is truncated like the sweeps' moves, so its frame keeps
    # the cap (an exact move would grow it to nblk times the rank)
    d, seed, cap = 5, 1, 4
    inst, prob = _maxcut(d, seed)
    # one sweep per solve: every sweep ends at core d-1, so every warm start is moved
    ipm = tt_ipm.TTIPM(prob, tt_ipm.Options(rank_cap=cap, max_iters=10, max_sweeps=1, kick=4))
    for it in range(3):
        ipm.iterate(it)
        assert ipm.w.pos == 0
        assert max(tt.ranks(ipm.w.cores)) <= cap, tt.ranks(ipm.w.cores)


@pytest.mark.parametrize("direction", ["aho", "xz"])
def test_combined_multiplier_direction_equals_dense_separate_newton(direction):
    # Section 3.5, "Combined Multiplier Storage": with disjoint masks the
    # direction found with one block dLambda (dY = P_Y dLambda, dT = P_T dLambda)
    # is the exact Newton direction of the separate padded system (O3)
    d = 3
    inst = inputs.cc_signed(d, 1)
    prob = tp.corr_clustering(tp.graph_tt(inst["c_plus"]), tp.graph_tt(inst["c_minus"]),
                              tp.graph_tt(inst["adjacency"]), d)
    ipm = tt_ipm.TTIPM(prob, tt_ipm.Options(rank_cap=64, kick=4, max_sweeps=8, combined_multipliers=True))
    _state(ipm, 7)
    ipm.eta = 1e-12
    mu = ipm.mu()
    X, Y, Z, T = (tt.full_mat(m) for m in (ipm.X, ipm.Y, ipm.Z, ipm.T))
    pad = sd.padded_cc(inst["c_plus"], inst["c_minus"], inst["adjacency"])
    blocks, K, R = sd.newton_solve(pad, X, Y, Z, T, mu=mu, direction=direction, sigma=0.5)
    data = ipm.combine_multipliers(ipm.newton_data(direction, 0.5 * mu, None, False, False))
    assert data.masks is not None and data.nblk == 3
    dX, dY, dT, dZ, info = ipm.direction(direction, 0.5 * mu, None, False, False)
    got = [tt.full_mat(m) for m in (dX, dY, dT, dZ)]
    if direction == "xz":
        # the XZ direction is symmetrised block by block (reading of Section 3.2)
        blocks = [0.5 * (b + b.T) for b in blocks]
    for a, b in zip(got, blocks):
        np.testing.assert_allclose(a, b, atol=1e-8 * (1 + np.abs(b).max()))
    # the multipliers live on their own masks
    n = 2 ** d
    assert np.abs(got[1][~np.eye(n, dtype=bool)]).max() <= 1e-12 * (1 + np.abs(got[1]).max())
    assert np.abs(np.diag(got[2])).max() <= 1e-12 * (1 + np.abs(got[2]).max())


def test_cc_separate_and_combined_multipliers_reach_the_same_optimum():
    d = 3
    inst = inputs.cc_signed(d, 1)
    prob = tp.corr_clustering(tp.graph_tt(inst["c_plus"]), tp.graph_tt(inst["c_minus"]),
                              tp.graph_tt(inst["adjacency"]), d)
    ref = sd.solve_dense(sd.cc_sdp(inst["c_plus"], inst["c_minus"], inst["adjacency"]))
    for combined in (False, True):
        ipm = tt_ipm.TTIPM(prob, tt_ipm.Options(rank_cap=16, max_iters=60, combined_multipliers=combined))
        assert ipm.solve()
        h = ipm.history[-1]
        assert abs(h.pobj - ref.pobj) / (1 + abs(ref.pobj)) <= 5e-3, (combined, h)


@pytest.mark.parametrize("d,seed", [(5, 1), (6, 0)])
def test_finishing_phase_reaches_the_absolute_criteria(d, seed):
    # Section 3.5, "Relaxing the Positive Definiteness Barrier": after the
    # relative criteria hold, iterations with step lengths for X + nu I >= 0
    # and merit-controlled acceptance reach ||R_p||, ||R_d||, <X, Z> < 1e-3 and
    # move the objective closer to the dense optimum
    inst, prob = _maxcut(d, seed)
    ref = sd.solve_dense(sd.maxcut_sdp(inst["weights"]), tol=1e-10).pobj
    plain = tt_ipm.TTIPM(prob, tt_ipm.Options(rank_cap=16, max_iters=40))
    assert plain.solve()
    fin = tt_ipm.TTIPM(prob, tt_ipm.Options(rank_cap=16, max_iters=40, finish_tol=1e-3))
    assert fin.solve()
    merit, done = fin.finish_merit()
    assert done and merit < 3e-3
    steps = [h for h in fin.history if h.finishing]
    assert steps and all(h.nu <= 1e-3 for h in steps)
    e_plain = abs(plain.history[-1].pobj - ref) / (1 + abs(ref))
    e_fin = abs(fin.history[-1].pobj - ref) / (1 + abs(ref))
    assert e_fin <= 0.1 * e_plain, (e_fin, e_plain)
    # the relaxed barrier allows eigenvalues down to -nu at most
    assert np.linalg.eigvalsh(tt.full_mat(fin.X))[0] >= -1e-3
    # the finishing phase never accepts an update that raises the merit
    merits = [h.merit for h in steps] + [merit]
    assert all(b <= a for a, b in zip(merits, merits[1:])), merits
