"""Pins of the planner oracle (Sec. 3.1 Eq. 1, Sec. 3.2 Eq. 2 and E_ac)."""
import math

import numpy as np
import pytest

from oracle import planner as PL


def test_paper_dense_example_160_vs_135():
    """Sec. 3.1: A_AP (4x5), M_{P.year>2020} (5x5), A_PT (5x3). (A_AP M) A_PT costs
    4*5*5 + 4*5*3 = 160 operations, A_AP (M A_PT) costs 5*5*3 + 4*5*3 = 135; the DP picks
    the second."""
    dims = [4, 5, 5, 3]
    cost, tree = PL.dense_plan(dims)
    assert cost == 135
    assert tree == (0, (1, 2))
    left = 4 * 5 * 5 + 4 * 5 * 3
    assert left == 160


def _tree_cost(tree, dims):
    """Brute-force dense cost of one parenthesisation."""
    if isinstance(tree, int):
        return 0, dims[tree], dims[tree + 1]
    cl, m, n = _tree_cost(tree[0], dims)
    cr, n2, l = _tree_cost(tree[1], dims)
    assert n == n2
    return cl + cr + m * n * l, m, l


@pytest.mark.parametrize("seed", range(20))
def test_dense_dp_equals_bruteforce_minimum(seed):
    rng = np.random.default_rng(seed)
    p = int(rng.integers(2, 8))
    dims = [int(x) for x in rng.integers(1, 60, p + 1)]
    cost, tree = PL.dense_plan(dims)
    costs = [_tree_cost(t, dims)[0] for t in PL.all_trees(0, p - 1)]
    assert len(costs) == math.comb(2 * (p - 1), p - 1) // p  # Catalan(p-1) trees
    assert cost == min(costs)
    assert _tree_cost(tree, dims)[0] == cost


def test_sparse_dp_reduces_to_dense_for_dense_inputs():
    """With every density 1, E_ac gives density 1 and Eq. 2 with (alpha, beta, gamma) =
    (0, 1, 0) is the operation count m*n*l of the dense cost."""
    rng = np.random.default_rng(5)
    for _ in range(20):
        p = int(rng.integers(2, 8))
        dims = [int(x) for x in rng.integers(1, 40, p + 1)]
        nnz = [dims[t] * dims[t + 1] for t in range(p)]
        c_sparse, t_sparse, *_ = PL.sparse_plan(dims, nnz, 0.0, 1.0, 0.0)
        c_dense, t_dense = PL.dense_plan(dims)
        assert c_sparse == pytest.approx(c_dense, rel=1e-12)
        assert t_sparse == t_dense


def test_eac_matches_monte_carlo():
    """E_ac is the expected density of a boolean product of uniform random matrices."""
    rng = np.random.default_rng(0)
    m, n, l = 300, 40, 300
    for rx, ry in ((0.05, 0.1), (0.2, 0.02), (0.01, 0.5)):
        X = rng.random((m, n)) < rx
        Y = rng.random((n, l)) < ry
        Z = (X.astype(np.int64) @ Y.astype(np.int64)) > 0
        emp = Z.mean()
        est = PL.eac_density(X.mean(), Y.mean(), n)
        sd = math.sqrt(est * (1 - est) / (m * l)) * 5 + 0.01 * est
        assert abs(emp - est) < sd, (rx, ry, emp, est)


def test_eq2_terms_match_counts():
    """N_op of Eq. 2 is the expected number of scalar products of Gustavson's method,
    sum_k nnz(X[:, k]) * nnz(Y[k, :]), for uniform random inputs."""
    rng = np.random.default_rng(1)
    m, n, l = 400, 80, 500
    X = rng.random((m, n)) < 0.03
    Y = rng.random((n, l)) < 0.05
    ops = int((X.sum(0) * Y.sum(1)).sum())
    rx, ry = X.mean(), Y.mean()
    rz = PL.eac_density(rx, ry, n)
    assert PL.sparse_cost(m, n, l, rx, ry, rz, 1, 0, 0) == pytest.approx(X.sum())
    assert PL.sparse_cost(m, n, l, rx, ry, rz, 0, 1, 0) == pytest.approx(ops, rel=0.05)
    assert PL.sparse_cost(m, n, l, rx, ry, rz, 0, 0, 1) == pytest.approx(m * l * rz)


def test_ties_take_smallest_split():
    cost, tree = PL.dense_plan([3, 3, 3, 3, 3])
    assert cost == 3 * 27
    assert tree == (0, (1, (2, 3)))
    C, D, S = PL.chain_dp([3, 3, 3, 3, 3], [1.0] * 4, PL.dense_product)
    assert S[0][3] == 0 and S[1][3] == 1 and S[0][2] == 0


def test_known_subchain_is_reused():
    """A cached sub-chain costs its retrieval (0) and carries its exact density."""
    dims = [1000, 10, 1000, 10, 1000]
    nnz = [5000, 5000, 5000, 5000]
    c0, t0, *_ = PL.sparse_plan(dims, nnz)
    c1, t1, C, D, S = PL.sparse_plan(dims, nnz, known={(1, 3): (0.0, 0.5)})
    assert c1 < c0
    assert t1 == (0, (1, 3, "known"))
    assert D[1][3] == 0.5


def test_fixed_density_changes_only_the_result_density():
    """A measured density replaces E_ac for that sub-chain: with the E_ac value itself the
    plan is unchanged; with a much denser measurement the DP avoids materialising it."""
    dims = [100, 100000, 100, 100000, 100]
    nnz = [5000, 5000, 5000, 5000]
    c0, t0, C0, D0, S0 = PL.sparse_plan(dims, nnz)
    c1, t1, C1, D1, S1 = PL.sparse_plan(dims, nnz, rho_fixed={(1, 2): D0[1][2]})
    assert c1 == pytest.approx(c0) and t1 == t0
    c2, t2, C2, D2, S2 = PL.sparse_plan(dims, nnz, rho_fixed={(1, 2): 0.9})
    assert D2[1][2] == 0.9
    assert C2[1][2] > C0[1][2]


def test_sampled_density_scaling():
    # every row sampled: the exact density
    assert PL.sampled_density(30, 10, 10, 10, 50) == pytest.approx(30 / 500)
    # 10 of 100 non-empty rows sampled in a 1000-row matrix
    assert PL.sampled_density(30, 10, 100, 1000, 50) == pytest.approx(300 / 50000)
    assert PL.sampled_density(0, 0, 10, 10, 10) == 0.0
