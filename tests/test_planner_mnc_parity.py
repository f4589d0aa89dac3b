"""The engine's C++ MNC planner (host-only entry point) against the MNC oracle: the same
exact leaf sketches in, the same splits, costs and estimated sizes out (up to rounding of
the density-map sum, taken as a product in the oracle and as a sum of logarithms in the
engine). Runs without a GPU."""
import numpy as np
import pytest

from oracle import mnc as MNC


def _leaf(rng, m, n, kind):
    """A random m x n pattern: uniform, skewed (Zipf-like degrees), or with many
    single-entry rows and columns (so every MNC case is reached)."""
    if kind == 0:
        A = rng.random((m, n)) < rng.uniform(0.02, 0.4)
    elif kind == 1:
        w = 1.0 / np.arange(1, n + 1) ** 1.2
        A = rng.random((m, n)) < np.minimum(1.0, rng.uniform(0.5, 3.0) * w[rng.permutation(n)])[None, :]
    else:
        A = np.zeros((m, n), bool)
        A[np.arange(m), rng.integers(0, n, m)] = True
        extra = rng.random((m, n)) < 0.05
        A |= extra & (rng.random(m) < 0.5)[:, None]
    return A.astype(np.int8)


def _check(dims, mats, known=None, ab=(1.0, 1.0, 1.0)):
    from paper_2201_04058_b300 import mp
    leaves = [MNC.sketch_of_dense(A) for A in mats]
    c, tree, C, N, S = MNC.mnc_plan(dims, leaves, *ab, known=known)
    sks = [(sk.hr, sk.hc, sk.her, sk.hec) for sk in leaves]
    split, cost, nnz = mp.mp_plan_chain_mnc(dims, sks, *ab, known=known)
    p = len(mats)
    for i in range(p):
        for j in range(i, p):
            assert split[i, j] == S[i][j], (i, j)
            assert cost[i, j] == pytest.approx(C[i][j], rel=1e-9, abs=1e-9), (i, j)
            assert nnz[i, j] == pytest.approx(N[i][j], rel=1e-9, abs=1e-9), (i, j)


@pytest.mark.parametrize("seed", range(40))
def test_mnc_planner_matches_oracle(seed):
    rng = np.random.default_rng(1000 + seed)
    p = int(rng.integers(1, 7))
    dims = [int(x) for x in rng.integers(2, 40, p + 1)]
    mats = [_leaf(rng, dims[t], dims[t + 1], int(rng.integers(0, 3))) for t in range(p)]
    ab = tuple(float(x) for x in rng.uniform(0.1, 3.0, 3))
    _check(dims, mats, ab=ab)


@pytest.mark.parametrize("seed", range(10))
def test_mnc_planner_with_known_subchains(seed):
    rng = np.random.default_rng(2000 + seed)
    p = int(rng.integers(3, 7))
    dims = [int(x) for x in rng.integers(2, 30, p + 1)]
    mats = [_leaf(rng, dims[t], dims[t + 1], int(rng.integers(0, 3))) for t in range(p)]
    i = int(rng.integers(0, p - 1))
    j = int(rng.integers(i + 1, p))
    known = {(i, j): (float(rng.uniform(0, 50)), float(rng.uniform(0, dims[i] * dims[j + 1])))}
    _check(dims, mats, known=known)


def test_skewed_chain_plan_through_engine():
    """The skewed chain of the oracle pins: the engine's MNC plan is X0 (X1 X2)."""
    from paper_2201_04058_b300 import mp
    m, n, l0, l, r = 100, 20, 5, 40, 400
    X0 = np.zeros((m, n)); X0[:, 0] = 1
    X1 = np.zeros((n, l)); X1[0, :l0] = 1
    X2 = (np.random.default_rng(13).random((l, r)) < 0.5).astype(np.int8)
    sks = []
    for A in (X0, X1, X2):
        sk = MNC.sketch_of_dense(A)
        sks.append((sk.hr, sk.hc, sk.her, sk.hec))
    split, cost, nnz = mp.mp_plan_chain_mnc([m, n, l, r], sks, 0.0, 1.0, 0.0)
    assert split[0, 2] == 0 and split[1, 2] == 1
    assert nnz[0, 1] == m * l0
