"""The engine's C++ chain planner against the oracle planner (Sec. 3.1 Eq. 1, Sec. 3.2
Eq. 2 and E_ac). Host-only entry point, so this runs without a GPU.

Where two splits cost the same up to rounding, both are optimal: the test compares the
optimal cost and checks that the engine's split is optimal under the oracle's costs."""
import numpy as np
import pytest

from oracle import planner as PL


def _tree_from_split(S, i, j):
    if i == j or S[i][j] < 0:
        return i if i == j else (i, j, "known")
    k = int(S[i][j])
    return (_tree_from_split(S, i, k), _tree_from_split(S, k + 1, j))


def test_paper_example_through_engine():
    from paper_2201_04058_b300 import mp
    split, cost = mp.mp_plan_chain([4, 5, 5, 3], [20, 25, 15], 0.0, 1.0, 0.0)
    assert cost[0, 2] == 135
    assert _tree_from_split(split, 0, 2) == (0, (1, 2))


@pytest.mark.parametrize("seed", range(40))
def test_engine_planner_matches_oracle(seed):
    from paper_2201_04058_b300 import mp
    rng = np.random.default_rng(seed)
    p = int(rng.integers(1, 9))
    dims = rng.integers(1, 5_000_000, p + 1).astype(np.float64)
    dens = 10.0 ** rng.uniform(-7, -1, p)
    nnz = np.maximum(1, np.floor(dims[:-1] * dims[1:] * dens))
    a, b, g = (float(x) for x in rng.uniform(0.1, 3.0, 3))
    known = None
    if p >= 3 and seed % 3 == 0:
        i = int(rng.integers(0, p - 1))
        j = int(rng.integers(i + 1, p))
        known = {(i, j): (float(rng.uniform(0, 1e6)), float(rng.uniform(0, 0.1)))}
    fixed = None
    if p >= 2 and seed % 2 == 1:
        i = int(rng.integers(0, p - 1))
        fixed = {(i, i + 1): float(10.0 ** rng.uniform(-6, -1))}
    c_o, t_o, C, D, S = PL.sparse_plan(list(dims), list(nnz), a, b, g, known, fixed)
    split, cost = mp.mp_plan_chain(dims, nnz, a, b, g, known, fixed)
    assert cost[0, p - 1] == pytest.approx(c_o, rel=1e-9)
    # the engine's split at every sub-chain is optimal under the oracle's recursion
    for ln in range(2, p + 1):
        for i in range(0, p - ln + 1):
            j = i + ln - 1
            if known and (i, j) in known:
                assert split[i, j] == -1
                continue
            k = int(split[i, j])
            prod = PL.sparse_product(a, b, g)
            c, _ = prod(dims[i], dims[k + 1], dims[j + 1], D[i][k], D[k + 1][j], (fixed or {}).get((i, j)))
            assert C[i][k] + C[k + 1][j] + c == pytest.approx(C[i][j], rel=1e-9)
