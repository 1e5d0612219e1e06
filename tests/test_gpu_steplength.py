"""Row a12 parity: the step-length eigenproblem min <e, dM e>/<e, M e> on the
GPU (tt_min_gen_eig, two-site DMRG and one-site ALS) against the dense
generalised eigenvalue and the oracle's sweeps."""
import math
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import paper_2509_11890_gb300 as tg  # noqa: E402
from oracle import sdp_dense as sd, tt, tt_ipm  # noqa: E402
from paper_2509_11890_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu


def _dev(cores):
    import torch
    ranks = [c.shape[0] for c in cores] + [1]
    flat = torch.from_numpy(np.concatenate([np.asarray(c, dtype=np.float64).ravel() for c in cores])).cuda()
    return tg.DevTT(ranks, cores[0].shape[1], cores[0].shape[2], flat)


def _pd_pair(d, seed, rank=2):
    g = inputs.random_tt_matrix([2] * d, [2] * d, [1] + [rank] * (d - 1) + [1], seed + 40)
    gs = tt.add(g, tt.transpose(g), 0.5, 0.5)
    shift = abs(np.linalg.eigvalsh(tt.full_mat(gs))[0]) + 1.0
    M = tt.add(tt.scale(tt.identity(d), shift), gs)
    h = inputs.random_tt_matrix([2] * d, [2] * d, [1] + [rank] * (d - 1) + [1], seed + 50)
    dM = tt.add(h, tt.transpose(h), 0.5, 0.5)
    return M, dM


@pytest.mark.parametrize("two_site", [True, False])
@pytest.mark.parametrize("seed", [0, 1])
def test_full_rank_quotient_equals_dense_step_rule(two_site, seed):
    d = 4
    M, dM = _pd_pair(d, seed)
    ref = sd.max_step(tt.full_mat(M), tt.full_mat(dM))
    lam = tg.min_gen_eig(_dev(M), _dev(dM), rank=4, sweeps=8 if not two_site else 4, two_site=two_site, seed=seed)
    assert math.isclose(tt_ipm.step_from_lambda(lam), ref, rel_tol=1e-8)


@pytest.mark.parametrize("d,seed", [(6, 2), (6, 3), (6, 4), (8, 2), (8, 3), (8, 4)])
def test_dmrg_rank_one_eigenvector(d, seed):
    # M = I, dM = diag(v): every local minimum of the quotient over unit
    # vectors is an entry of v; the sweeps stop at the oracle's entry (the
    # smallest one for these d = 6 draws, the second smallest for d = 8, seed 2)
    v = inputs.random_tt([2] * d, [1] + [2] * (d - 1) + [1], seed)
    M = tt.identity(d)
    dM = tt.diag_tt(v)
    lam = tg.min_gen_eig(_dev(M), _dev(dM), rank=2, sweeps=6, two_site=True, seed=seed)
    lam_o, _ = tt_ipm.min_gen_eig_dmrg(M, dM, None, tt_ipm.Counter(seed), rank=2, sweeps=6)
    assert math.isclose(lam, lam_o, rel_tol=1e-8, abs_tol=1e-10)
    entries = tt.full_vec(v)
    assert np.min(np.abs(entries - lam)) <= 1e-8 * max(1.0, abs(lam))
    if d == 6:
        assert math.isclose(lam, float(np.min(entries)), rel_tol=1e-8, abs_tol=1e-10)


@pytest.mark.parametrize("seed", [5, 6])
def test_dmrg_matches_oracle_sweeps_at_truncated_rank(seed):
    # same algorithm, same SplitMix64 stream: the quotient after the sweeps
    # agrees. The GPU takes each local eigenvector from an FP32 Jacobi SVD and
    # its eigenvalue as the FP64 Rayleigh quotient, so at a truncated rank the
    # sweeps follow the oracle's path to about 1e-7 and the quotients agree to
    # a few units in 1e-7
    d = 6
    M, dM = _pd_pair(d, seed, rank=3)
    lam_o, _ = tt_ipm.min_gen_eig_dmrg(M, dM, None, tt_ipm.Counter(seed), rank=3, sweeps=4)
    lam_g = tg.min_gen_eig(_dev(M), _dev(dM), rank=3, sweeps=4, two_site=True, seed=seed)
    assert math.isclose(lam_g, lam_o, rel_tol=1e-5, abs_tol=1e-10)
    lam_o1, _ = tt_ipm.min_gen_eig(M, dM, None, tt_ipm.Counter(seed), rank=3, sweeps=4)
    lam_g1 = tg.min_gen_eig(_dev(M), _dev(dM), rank=3, sweeps=4, two_site=False, seed=seed)
    assert math.isclose(lam_g1, lam_o1, rel_tol=1e-5, abs_tol=1e-10)


def test_indefinite_iterate_is_reported():
    # Section 3.4: an iterate that is not positive definite is detected in its projection
    d = 4
    M, dM = _pd_pair(d, 0)
    Mneg = tt.add(M, tt.identity(d), 1.0, -100.0)
    with pytest.raises(RuntimeError) as ei:
        tg.min_gen_eig(_dev(Mneg), _dev(dM), rank=4, sweeps=2)
    assert ei.value.status == 5  # TT_E_NOT_PD


def test_min_gen_eig_rejects_bad_arguments():
    M, dM = _pd_pair(3, 0)
    with pytest.raises(RuntimeError):
        tg.min_gen_eig(_dev(M), _dev(dM), rank=0)
