"""Pins for the oracle's TT problem assembly (row a1, Section 4).

The TT operators must equal the dense padded formulation written straight
from the graph, and meet the TT-rank statements of Section 4 exactly.
"""
import numpy as np
import pytest

from oracle import sdp_dense as sd, tt, tt_problems as tp
from paper_2509_11890_gb300 import inputs


def _dense_checks(prob, padded):
    d = prob.d
    np.testing.assert_allclose(tt.full_mat(prob.C), padded.C, atol=1e-12)
    np.testing.assert_allclose(tt.full_mat(prob.A_eq), padded.A_eq, atol=1e-12)
    np.testing.assert_allclose(tt.full_vec(prob.B_eq), padded.B_eq, atol=1e-12)
    np.testing.assert_allclose(tt.full_mat(prob.K_y), padded.K_y, atol=1e-12)
    if padded.has_ineq:
        np.testing.assert_allclose(tt.full_mat(prob.A_ineq), padded.A_ineq, atol=1e-12)
        np.testing.assert_allclose(tt.full_mat(prob.K_t), padded.K_t, atol=1e-12)


@pytest.mark.parametrize("d,seed", [(3, 0), (4, 1), (5, 2)])
def test_maxcut_assembly_and_ranks(d, seed):
    inst = inputs.maxcut_kron(d, seed)
    a = inst["adjacency_cores"]
    np.testing.assert_array_equal(tt.full_mat(a), inst["adjacency"].astype(float))
    prob = tp.maxcut(a, d)
    _dense_checks(prob, sd.padded_maxcut(inst["weights"]))
    # Section 4.1 rank statements
    ra = tt.ranks(a)
    assert all(rc <= 2 * r for rc, r in zip(tt.ranks(prob.C), ra))
    assert tt.ranks(prob.A_eq) == [1] * (d + 1)
    assert tt.ranks(prob.B_eq) == [1] * (d + 1)
    assert tt.ranks(prob.K_y) == [1] + [2] * (d - 1) + [1]


@pytest.mark.parametrize("d,seed", [(3, 0), (4, 3)])
def test_theta_assembly_and_ranks(d, seed):
    inst = inputs.theta_hypercube_kron(d, seed)
    a = tp.graph_tt(inst["adjacency"])
    prob = tp.theta(a, d)
    _dense_checks(prob, sd.padded_theta(inst["adjacency"]))
    ra = tt.ranks(a)
    assert all(r1 <= r + 1 for r1, r in zip(tt.ranks(prob.A_eq)[1:-1], ra[1:-1]))
    assert all(r1 <= r + 2 for r1, r in zip(tt.ranks(prob.K_y)[1:-1], ra[1:-1]))
    assert tt.ranks(prob.B_eq) == [1] * (d + 1)


@pytest.mark.parametrize("d", [3, 4])
def test_cc_assembly_and_ranks(d):
    inst = inputs.cc_signed(d, 0)
    cp, cm = tp.graph_tt(inst["c_plus"]), tp.graph_tt(inst["c_minus"])
    a = tp.graph_tt(inst["adjacency"])
    prob = tp.corr_clustering(cp, cm, a, d)
    _dense_checks(prob, sd.padded_cc(inst["c_plus"], inst["c_minus"], inst["adjacency"]))
    assert all(rc <= rp + 2 * rm for rc, rp, rm in zip(tt.ranks(prob.C), tt.ranks(cp), tt.ranks(cm)))
    assert all(r1 <= r for r1, r in zip(tt.ranks(prob.A_ineq), tt.ranks(a)))
    assert all(r1 <= 1 + r for r1, r in zip(tt.ranks(prob.K_t), tt.ranks(a)))
    assert prob.q == int(inst["adjacency"].sum())
    # the complete graph J - I has TT rank 2
    assert max(tt.ranks(a)) == 2
