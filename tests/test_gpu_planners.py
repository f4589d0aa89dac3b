"""GPU: the plans themselves. The engine's planners, asked through mp_plan_query (plan
only, no product), against the oracle planners fed with the oracle's own masked leaves:
E_ac (Sec. 3.2, Eq. 1 with the Eq. 2 cost) on exact masked nnz, and MNC on exact count
sketches built on the GPU. Where two splits cost the same up to rounding (mirror-image
chains such as APTPA), either is optimal, so a differing split must tie under the
oracle's costs. Queries run with the MNC planner give the oracle's results."""
import numpy as np
import pytest

import gen
from oracle import chain as OC
from oracle import mnc as MNC
from oracle import planner as PL
from oracle.hin import OracleHIN

from test_gpu_parity import assert_same

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c1():
    h = gen.config1_hin()
    return h, OracleHIN(h)


@pytest.fixture(scope="module")
def c2_small(cuda_ok):
    h = gen.config2_hin(scale=0.01)
    return h, OracleHIN(h)


def _masked_leaves(ohin, q):
    """(dims, [(rp, ci, nrows, ncols)]) of diag(M_t) A_t diag(M_t+1) for every factor."""
    f, m = ohin.query(q)
    out = []
    for t, (rp, ci, nr, nc) in enumerate(f):
        rows = np.repeat(np.arange(nr), np.diff(rp))
        keep = np.ones(ci.size, bool)
        if m[t] is not None:
            keep &= m[t][rows].astype(bool)
        if m[t + 1] is not None:
            keep &= m[t + 1][ci].astype(bool)
        rp2 = np.zeros(nr + 1, np.int64)
        np.cumsum(np.bincount(rows[keep], minlength=nr), out=rp2[1:])
        out.append((rp2, ci[keep], nr, nc))
    dims = [f[0][2]] + [x[3] for x in f]
    return dims, out


def _check_splits(split, S, totals, p, what):
    for i in range(p):
        for j in range(i + 1, p):
            k_e, k_o = int(split[i, j]), S[i][j]
            if k_e != k_o:
                a, b = totals[(i, j, k_e)], totals[(i, j, k_o)]
                assert a == pytest.approx(b, rel=1e-9), (what, i, j, k_e, k_o, a, b)


def _queries(h, seed, n):
    return [q for q in gen.random_queries(h, seed, n, lengths=(3, 7))] + [gen.config1_query()]


def test_mnc_plans_match_oracle(c1, cuda_ok):
    from paper_2201_04058_b300 import mp
    h, o = c1
    e = mp.Engine(h, planner=mp.MP_PLAN_DP_MNC, policy=mp.MP_POLICY_NONE)
    try:
        for q in _queries(h, 21, 25) + gen.long_queries(5, 8):
            dims, leaves = _masked_leaves(o, q)
            sks = [MNC.sketch_of_csr(rp, ci, nc) for rp, ci, nr, nc in leaves]
            totals = {}
            c, tree, C, N, S = MNC.mnc_plan(dims, sks, totals=totals)
            split, nnz = e.plan(q)
            p = len(leaves)
            what = "".join(q["types"])
            for i in range(p):
                assert nnz[i, i] == pytest.approx(sks[i].nnz), what
            _check_splits(split, S, totals, p, what)
            if all(int(split[i, j]) == S[i][j] for i in range(p) for j in range(i + 1, p)):
                for i in range(p):
                    for j in range(i, p):
                        assert nnz[i, j] == pytest.approx(N[i][j], rel=1e-9, abs=1e-9), (what, i, j)
    finally:
        e.close()


def test_eac_plans_match_oracle(c1, cuda_ok):
    from paper_2201_04058_b300 import mp
    h, o = c1
    e = mp.Engine(h, planner=mp.MP_PLAN_DP, policy=mp.MP_POLICY_NONE)
    try:
        for q in _queries(h, 22, 25):
            dims, leaves = _masked_leaves(o, q)
            nnz = [float(ci.size) for rp, ci, nr, nc in leaves]
            p = len(leaves)
            C, D, S = PL.chain_dp(dims, [nnz[t] / (dims[t] * dims[t + 1]) for t in range(p)], PL.sparse_product())
            totals = {}
            for ln in range(2, p + 1):
                for i in range(p - ln + 1):
                    j = i + ln - 1
                    for k in range(i, j):
                        cost, _ = PL.sparse_product()(dims[i], dims[k + 1], dims[j + 1], D[i][k], D[k + 1][j])
                        totals[(i, j, k)] = C[i][k] + C[k + 1][j] + cost
            split, est = e.plan(q)
            _check_splits(split, S, totals, p, "".join(q["types"]))
            for i in range(p):
                assert est[i, i] == pytest.approx(nnz[i])
    finally:
        e.close()


def test_mnc_planner_results_match_oracle(c1, c2_small, cuda_ok):
    from paper_2201_04058_b300 import mp
    for (h, o), qs in ((c1, _queries(c1[0], 23, 12) + gen.long_queries(5, 4)),
                       (c2_small, gen.config2_queries(c2_small[0], seed=2, n_anchor_a=32, n_anchor_t=4))):
        e = mp.Engine(h, planner=mp.MP_PLAN_DP_MNC, policy=mp.MP_POLICY_ATRAPOS)
        try:
            for rnd in range(2):
                rc, res = e.run_batch(qs)
                assert rc == 0
                for q, g in zip(qs, res):
                    assert_same(g, OC.evaluate(o, q), ("mnc", rnd, "".join(q["types"])))
        finally:
            e.close()


def test_plan_query_leaves_cache_untouched(c1, cuda_ok):
    from paper_2201_04058_b300 import mp
    h, o = c1
    e = mp.Engine(h, planner=mp.MP_PLAN_DP_MNC, policy=mp.MP_POLICY_ATRAPOS)
    try:
        before = mp.mp_cache_stats(e.ctx)
        for q in _queries(h, 24, 5):
            e.plan(q)
        assert mp.mp_cache_stats(e.ctx) == before
        split, nnz = e.plan({"types": list("PA"), "constraints": []})
        assert split.shape == (1, 1) and split[0, 0] == -1 and nnz[0, 0] > 0
    finally:
        e.close()
