"""GPU parity at full size: the benchmark's workload (5 M papers, 4 M authors, 5 k venues,
50 k topics; twenty constrained queries) through the same calls the benchmark times.

The oracle cannot build every full result in seconds, so each result is checked
  * on sampled rows, which the oracle computes exactly (the query with its first position
    additionally restricted to the sampled rows: rows of A_m are independent);
  * on every row and every column through the invariants row_sum(A_m) = M_1 A_1 ... M_n 1
    and col_sum(A_m) = 1^T M_1 A_1 ... M_n, which the oracle evaluates as SpMV chains;
and the batched form (one DAG for all twenty queries) must equal the plain form."""
import numpy as np
import pytest

import gen
from oracle import chain as OC
from oracle.hin import OracleHIN

from test_gpu_parity import assert_same

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def full(cuda_ok):
    from paper_2201_04058_b300 import mp
    h = gen.config2_hin(seed=2)
    qs = gen.config2_queries(h, seed=2)
    eng = mp.Engine(h, policy=mp.MP_POLICY_NONE)
    res = [eng.run(q) for q in qs]
    yield h, qs, eng, res
    eng.close()


@pytest.fixture(scope="module")
def ohin(full):
    return OracleHIN(full[0])


def _row_sums(rp, val):
    out = np.zeros(len(rp) - 1, np.uint64)
    np.add.at(out, np.repeat(np.arange(len(rp) - 1), np.diff(rp)), val)
    return out


def test_sampled_rows_match_oracle(full, ohin):
    h, qs, eng, res = full
    rng = np.random.default_rng(11)
    for qi, (q, (rp, ci, val)) in enumerate(zip(qs, res)):
        nz = np.nonzero(np.diff(rp))[0]
        if nz.size == 0:
            continue
        # the heaviest row, the lightest non-empty row and a few at random
        sizes = np.diff(rp)[nz]
        pick = {int(nz[np.argmax(sizes)]), int(nz[np.argmin(sizes)])}
        pick |= set(int(x) for x in rng.choice(nz, size=min(4, nz.size), replace=False))
        rows = np.array(sorted(pick), np.uint32)
        qq = {"types": q["types"], "constraints": list(q["constraints"]) +
              [{"pos": 0, "prop": None, "op": "in", "set": rows}]}
        orp, oci, oval = OC.evaluate(ohin, qq)
        for r in rows:
            a, b = int(rp[r]), int(rp[r + 1])
            oa, ob = int(orp[r]), int(orp[r + 1])
            np.testing.assert_array_equal(ci[a:b], oci[oa:ob], err_msg=f"query {qi} row {r}")
            np.testing.assert_array_equal(val[a:b], oval[oa:ob], err_msg=f"query {qi} row {r}")


def test_row_and_column_sums_match_spmv_chains(full, ohin):
    h, qs, eng, res = full
    for qi, (q, (rp, ci, val)) in enumerate(zip(qs, res)):
        f, m = ohin.query(q)
        np.testing.assert_array_equal(_row_sums(rp, val), OC.rowsum(f, m), err_msg=f"query {qi} rows")
        cols = np.zeros(f[-1][3], np.uint64)
        np.add.at(cols, ci, val)
        np.testing.assert_array_equal(cols, OC.colsum(f, m), err_msg=f"query {qi} cols")
        # canonical CSR: strictly ascending columns within each row, no stored zeros
        d = np.diff(ci.astype(np.int64))
        if d.size:
            inner = np.ones(d.size, bool)
            b = rp[1:-1]
            b = b[(b > 0) & (b < ci.size)]
            inner[b - 1] = False  # the step from one row's last entry to the next row's first
            assert np.all(d[inner] > 0), f"query {qi}: columns not ascending"
        assert np.all(val > 0)


def test_batched_form_equals_plain(full):
    h, qs, eng, res = full
    rc, got = eng.run_batch(qs)
    assert rc == 0
    for q, g, w in zip(qs, got, res):
        assert_same(g, w, "".join(q["types"]))


def test_every_result_matches_oracle(full, ohin):
    """Every full-size result, element by element, against the oracle's whole CSR (about
    half a minute of single-threaded host time for the twenty queries)."""
    h, qs, eng, res = full
    for qi, (q, got) in enumerate(zip(qs, res)):
        assert_same(got, OC.evaluate(ohin, q), f"query {qi} {''.join(q['types'])}")
