"""Properties of the seeded synthetic inputs (no method arithmetic)."""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from paper_2509_11890_gb300 import inputs  # noqa: E402


def _undirected_loop_free(a):
    np.testing.assert_array_equal(a, a.T)
    assert not np.any(np.diag(a))


@pytest.mark.parametrize("d,seed", [(3, 0), (6, 1), (8, 2)])
def test_kronecker_graph_is_the_kron_of_its_patterns(d, seed):
    inst = inputs.maxcut_kron(d, seed)
    a = inst["adjacency"].astype(np.int64)
    _undirected_loop_free(a)
    full = np.ones((1, 1), dtype=np.int64)
    for p in inst["patterns"]:
        full = np.kron(full, p.astype(np.int64))
    np.fill_diagonal(full, 0)
    np.testing.assert_array_equal(a, full)
    assert a.sum() > 0


def test_kronecker_plus_er_weights():
    inst = inputs.maxcut_kron_er(8, 0)
    w = inst["weights"]
    _undirected_loop_free(w)
    nz = w[w != 0]
    assert nz.min() >= 0.5 and nz.max() <= 1.5
    kron = inputs.maxcut_kron(8, 0)["adjacency"]
    # every Kronecker edge is present (the ER graph is OR-ed in)
    assert np.all(w[kron.astype(bool)] > 0)


def test_theta_graph_contains_the_cube_and_meets_the_density_window():
    d = 10
    inst = inputs.theta_hypercube_kron(d, 0)
    a = inst["adjacency"].astype(bool)
    _undirected_loop_free(a)
    n = 2 ** d
    u = np.arange(n)
    for k in range(d):
        assert np.all(a[u, u ^ (1 << k)])         # Q_d edges
    dens = a.sum() / (n * (n - 1))
    assert 0.008 <= dens <= 0.015 and abs(dens - inst["density"]) < 1e-12


def test_signed_graph_is_complete_and_signed():
    inst = inputs.cc_signed(5, 0)
    w = inst["weights"]
    _undirected_loop_free(w)
    off = ~np.eye(len(w), dtype=bool)
    assert set(np.unique(w[off])) <= {-1.0, 1.0}
    np.testing.assert_array_equal(inst["c_plus"] - inst["c_minus"], w)
    assert np.all(inst["c_plus"] >= 0) and np.all(inst["c_minus"] >= 0)


def test_batch_orders_and_reproducibility():
    b1 = inputs.batch_maxcut(16, 3)
    b2 = inputs.batch_maxcut(16, 3)
    assert [i["d"] for i in b1] == [i["d"] for i in b2]
    assert all(6 <= i["d"] <= 11 for i in b1)
    for x, y in zip(b1, b2):
        np.testing.assert_array_equal(x["adjacency"], y["adjacency"])


def test_cc_sub_instance_is_the_leading_block_of_the_full_instance():
    full = inputs.cc_signed(9, 3)
    sub = inputs.cc_signed_sub(9, 6, 3)
    n = 2 ** 6
    np.testing.assert_array_equal(sub["weights"], full["weights"][:n, :n])
    w = sub["weights"]
    assert w.shape == (n, n) and np.array_equal(w, w.T) and np.all(np.diag(w) == 0)
    off = w[~np.eye(n, dtype=bool)]
    assert set(np.unique(off)) <= {-1.0, 1.0}
    np.testing.assert_array_equal(sub["c_plus"] - sub["c_minus"], w)
    assert sub["adjacency"].sum() == n * (n - 1)
