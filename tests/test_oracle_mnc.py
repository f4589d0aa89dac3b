"""Pins of the MNC sketch estimator and the DP over sketches (Sec. 3.2's comparison of
E_ac with MNC): hand-counted sketches, the cases where the estimate is exact (checked
against brute-force products), bounds, agreement with Monte Carlo on uniform inputs, a
skewed case where E_ac is off by the inner dimension, and the DP's reductions."""
import numpy as np
import pytest

from oracle import mnc as MNC
from oracle import planner as PL


def _nnz(A, B):
    return int(((np.asarray(A) != 0).astype(np.int64) @ (np.asarray(B) != 0).astype(np.int64) > 0).sum())


def _rand(rng, m, n, rho):
    return (rng.random((m, n)) < rho).astype(np.int8)


def test_sketch_counts_by_hand():
    A = np.array([[1, 0, 1, 0],
                  [0, 0, 1, 0],
                  [1, 1, 1, 0]])
    s = MNC.sketch_of_dense(A)
    np.testing.assert_array_equal(s.hr, [2, 1, 3])
    np.testing.assert_array_equal(s.hc, [2, 1, 3, 0])
    # columns with a single non-zero: only column 1 (in row 2)
    np.testing.assert_array_equal(s.her, [0, 0, 1])
    # rows with a single non-zero: only row 1 (in column 2)
    np.testing.assert_array_equal(s.hec, [0, 0, 1, 0])


@pytest.mark.parametrize("seed", range(5))
def test_csr_sketch_equals_dense_definition(seed):
    rng = np.random.default_rng(seed)
    A = _rand(rng, 40, 30, 0.07)
    rp = np.concatenate(([0], np.cumsum((A != 0).sum(1))))
    ci = np.nonzero(A)[1]
    a, b = MNC.sketch_of_csr(rp, ci, 30), MNC.sketch_of_dense(A)
    for f in ("hr", "hc", "her", "hec"):
        np.testing.assert_array_equal(getattr(a, f), getattr(b, f))


@pytest.mark.parametrize("seed", range(10))
def test_exact_when_rows_of_a_or_columns_of_b_are_single(seed):
    rng = np.random.default_rng(100 + seed)
    m, n, l = 30, 12, 25
    A = np.zeros((m, n), np.int8)
    A[np.arange(m), rng.integers(0, n, m)] = 1
    A[rng.random(m) < 0.3] = 0                       # some empty rows
    B = _rand(rng, n, l, 0.3)
    assert MNC.estimate(MNC.sketch_of_dense(A), MNC.sketch_of_dense(B)) == _nnz(A, B)
    # the mirror case: every column of B holds at most one non-zero
    A2 = _rand(rng, m, n, 0.3)
    B2 = np.zeros((n, l), np.int8)
    B2[rng.integers(0, n, l), np.arange(l)] = 1
    assert MNC.estimate(MNC.sketch_of_dense(A2), MNC.sketch_of_dense(B2)) == _nnz(A2, B2)


def test_extension_vectors_count_single_rows_and_columns_exactly():
    """A: row 0 single, row 1 double; B: column 0 single, column 1 double. The exact parts
    give 2 (row 0 of C) + 1 (C[1,0]); the remaining 1 x 1 block is covered with certainty."""
    A = np.array([[1, 0], [1, 1]])
    B = np.array([[1, 1], [0, 1]])
    assert MNC.estimate(MNC.sketch_of_dense(A), MNC.sketch_of_dense(B)) == pytest.approx(4.0)
    assert _nnz(A, B) == 4


def test_full_blocks_are_exact():
    for m, n, l in ((3, 2, 5), (7, 4, 1), (10, 10, 10)):
        A, B = np.ones((m, n)), np.ones((n, l))
        assert MNC.estimate(MNC.sketch_of_dense(A), MNC.sketch_of_dense(B)) == pytest.approx(m * l)


@pytest.mark.parametrize("seed", range(20))
def test_estimate_bounds(seed):
    rng = np.random.default_rng(200 + seed)
    m, n, l = (int(x) for x in rng.integers(2, 40, 3))
    A, B = _rand(rng, m, n, rng.random() * 0.4), _rand(rng, n, l, rng.random() * 0.4)
    a, b = MNC.sketch_of_dense(A), MNC.sketch_of_dense(B)
    est = MNC.estimate(a, b)
    products = float((a.hc * b.hr).sum())
    assert -1e-9 <= est <= min(products, m * l) + 1e-9
    if a.exact and b.exact and a.hr.max() > 1 and b.hc.max() > 1:
        exact_part = float((a.hec * b.hr).sum() + ((a.hc - a.hec) * b.her).sum())
        assert est >= exact_part - 1e-9
        assert exact_part <= _nnz(A, B)


def test_matches_monte_carlo_on_uniform_inputs():
    rng = np.random.default_rng(7)
    m, n, l = 300, 40, 300
    for rx, ry in ((0.05, 0.1), (0.2, 0.02), (0.01, 0.5)):
        A, B = _rand(rng, m, n, rx), _rand(rng, n, l, ry)
        est = MNC.estimate(MNC.sketch_of_dense(A), MNC.sketch_of_dense(B))
        assert est == pytest.approx(_nnz(A, B), rel=0.05), (rx, ry)


def test_skewed_case_exact_where_eac_is_off():
    """A's only non-empty column is 0 (a full column), B's only non-empty row is 0 with l0
    entries: nnz(AB) = m * l0. MNC sees that every row of A is single and is exact; E_ac,
    with uniform non-zeros assumed, gives about m * l0 / n."""
    m, n, l, l0 = 50, 40, 60, 30
    A = np.zeros((m, n)); A[:, 0] = 1
    B = np.zeros((n, l)); B[0, :l0] = 1
    assert MNC.estimate(MNC.sketch_of_dense(A), MNC.sketch_of_dense(B)) == m * l0 == _nnz(A, B)
    eac = m * l * PL.eac_density(A.mean(), B.mean(), n)
    assert eac < 0.1 * m * l0


def test_propagated_sketch_sums_to_the_estimate():
    rng = np.random.default_rng(9)
    A, B = _rand(rng, 30, 20, 0.2), _rand(rng, 20, 25, 0.2)
    a, b = MNC.sketch_of_dense(A), MNC.sketch_of_dense(B)
    s = MNC.estimate(a, b)
    c = MNC.propagate(a, b, s)
    assert c.hr.sum() == pytest.approx(s) and c.hc.sum() == pytest.approx(s)
    assert not c.exact
    # rows keep A's shape, columns B's
    nz = a.hr > 0
    np.testing.assert_allclose(c.hr[nz] / a.hr[nz], s / a.nnz)


def test_dp_reduces_to_dense_for_full_factors():
    """Full factors: every estimate is m*l (exact), so Eq. 2 with (0, 1, 0) is the dense
    operation count and the DP is the dense DP."""
    rng = np.random.default_rng(5)
    for _ in range(10):
        p = int(rng.integers(2, 6))
        dims = [int(x) for x in rng.integers(1, 12, p + 1)]
        leaves = [MNC.sketch_of_dense(np.ones((dims[t], dims[t + 1]))) for t in range(p)]
        c, tree, *_ = MNC.mnc_plan(dims, leaves, 0.0, 1.0, 0.0)
        cd, td = PL.dense_plan(dims)
        assert c == pytest.approx(cd, rel=1e-12)
        assert tree == td


def test_dp_single_product_cost_is_eq2_with_the_estimate():
    """With two factors the DP has one split; its cost is Eq. 2 with the MNC estimate."""
    rng = np.random.default_rng(11)
    A, B = _rand(rng, 20, 15, 0.2), _rand(rng, 15, 30, 0.1)
    a, b = MNC.sketch_of_dense(A), MNC.sketch_of_dense(B)
    c, tree, C, N, S = MNC.mnc_plan([20, 15, 30], [a, b], 1.0, 2.0, 3.0)
    z = MNC.estimate(a, b)
    want = PL.sparse_cost(20, 15, 30, A.mean(), B.mean(), z / 600.0, 1.0, 2.0, 3.0)
    assert c == pytest.approx(want) and N[0][1] == pytest.approx(z) and tree == (0, 1)


def test_known_subchain_is_reused():
    rng = np.random.default_rng(12)
    dims = [60, 8, 60, 8, 60]
    mats = [_rand(rng, dims[t], dims[t + 1], 0.2) for t in range(4)]
    leaves = [MNC.sketch_of_dense(x) for x in mats]
    c0, t0, *_ = MNC.mnc_plan(dims, leaves)
    c1, t1, C, N, S = MNC.mnc_plan(dims, leaves, known={(1, 3): (0.0, 123.0)})
    assert c1 < c0
    assert t1 == (0, (1, 3, "known"))
    assert N[1][3] == 123.0


def test_skew_changes_the_plan_toward_fewer_operations():
    """X0 (a full column, as above) X1 X2: MNC sees that X0 X1 is as large as m * l0 and
    prefers X0 (X1 X2); E_ac, which underestimates X0 X1 by the inner dimension, picks
    (X0 X1) X2. The true Gustavson operation count of MNC's plan is less than half."""
    m, n, l0, l, r = 100, 20, 5, 40, 400
    X0 = np.zeros((m, n)); X0[:, 0] = 1
    X1 = np.zeros((n, l)); X1[0, :l0] = 1
    X2 = (np.random.default_rng(13).random((l, r)) < 0.5).astype(np.int8)
    dims = [m, n, l, r]
    leaves = [MNC.sketch_of_dense(x) for x in (X0, X1, X2)]
    _, t_mnc, *_ = MNC.mnc_plan(dims, leaves, 0.0, 1.0, 0.0)
    nnz = [float((x != 0).sum()) for x in (X0, X1, X2)]
    _, t_eac, *_ = PL.sparse_plan(dims, nnz, 0.0, 1.0, 0.0)

    def ops(tree):
        """True Gustavson products of a plan: (matrix, operations)."""
        if isinstance(tree, int):
            return (np.asarray((X0, X1, X2)[tree]) != 0).astype(np.int64), 0
        (L, ol), (R, orr) = ops(tree[0]), ops(tree[1])
        prods = int(((L != 0).sum(0) * (R != 0).sum(1)).sum())
        return L @ R, ol + orr + prods

    assert t_mnc == (0, (1, 2)) and t_eac == ((0, 1), 2)
    assert ops(t_mnc)[1] < ops(t_eac)[1] / 2
