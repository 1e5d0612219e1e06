"""The rank-controlled graph family (Appendix A): undirected, loop-free, binary,
TT rank exactly r, exact TT cores; the oracle TT-IPM certifies a small instance."""
import math
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from oracle import sdp_dense as sd, tt, tt_ipm, tt_problems as tp  # noqa: E402
from paper_2509_11890_gb300 import inputs  # noqa: E402


@pytest.mark.parametrize("d,r,seed", [(3, 1, 0), (4, 2, 1), (5, 3, 2), (6, 2, 3), (7, 4, 4)])
def test_graph_properties_and_exact_rank(d, r, seed):
    inst = inputs.rank_controlled_graph(d, r, seed)
    a = inst["adjacency"].astype(np.float64)
    assert a.shape == (2 ** d, 2 ** d)
    assert set(np.unique(a)) <= {0.0, 1.0} and a.sum() > 0
    np.testing.assert_array_equal(a, a.T)
    assert not np.any(np.diag(a))
    # TT ranks from the oracle's TT-SVD of the vec_TT form: exactly r at the largest bond
    cores = tt.tt_svd(tt.vec_tt_dense(a, d), [4] * d, eps_rel=1e-12)
    assert max(tt.ranks(cores)) == r
    # the returned cores are an exact TT of the adjacency
    np.testing.assert_array_equal(tt.full_mat(inst["adjacency_cores"]), a)


def test_draws_are_reproducible_and_seeds_differ():
    a = inputs.rank_controlled_graph(5, 2, 7)["adjacency"]
    b = inputs.rank_controlled_graph(5, 2, 7)["adjacency"]
    c = inputs.rank_controlled_graph(5, 2, 8)["adjacency"]
    np.testing.assert_array_equal(a, b)
    assert not np.array_equal(a, c)


def test_oracle_ipm_certifies_a_rank_controlled_maxcut():
    d, r = 4, 2
    inst = inputs.rank_controlled_graph(d, r, 5)
    ref = sd.solve_dense(sd.maxcut_sdp(inst["weights"]))
    ipm = tt_ipm.TTIPM(tp.maxcut(inst["adjacency_cores"], d), tt_ipm.Options(rank_cap=16, max_iters=40))
    assert ipm.solve()
    h = ipm.history[-1]
    assert abs(h.pobj - ref.pobj) / (1 + abs(ref.pobj)) <= 2e-3
    assert h.rel_gap <= 1e-4 / math.sqrt(d)
