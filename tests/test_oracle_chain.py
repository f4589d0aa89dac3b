"""Pins of the chain-product oracle against things other than itself.

* brute-force DFS enumeration of metapath instances (Def. 2, Def. 3) on tiny HINs;
* closed forms (n = 2, APA diagonal / co-authorship, PVP block structure);
* scipy.sparse int64 products on the 2,000-paper HIN;
* invariants: row/column sums from the SpMV chains, palindromic symmetry, every
  parenthesisation gives the same matrix, and overflow is reported, never wrapped.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import gen
from oracle import chain as OC
from oracle.hin import OracleHIN

from _brute import adjacency, check_canonical, csr_to_dict, enumerate_counts


def _tiny_cases(n_hins=12, n_queries=12):
    for seed in range(n_hins):
        h = gen.tiny_hin(seed, max_nodes=8 if seed % 3 else 12)
        qs = gen.random_queries(h, seed, n_queries, lengths=(2, 7), p_cons=0.4)
        yield seed, h, qs


@pytest.mark.parametrize("seed,hin,queries", list(_tiny_cases()))
def test_oracle_matches_bruteforce(seed, hin, queries):
    o = OracleHIN(hin)
    adj = adjacency(hin)
    for q in queries:
        rp, ci, val = OC.evaluate(o, q)
        n0, nl = hin["types"][q["types"][0]], hin["types"][q["types"][-1]]
        check_canonical(rp, ci, val, n0, nl)
        assert csr_to_dict(rp, ci, val) == enumerate_counts(hin, q, adj), q


def _compound_queries(hin, seed, n):
    """Queries whose positions carry one to three constraints at once, mixing every kind
    the boundary takes: a property range, a property equality, a property value set, an id
    window, an id equality and an id set."""
    g = np.random.default_rng(9000 + seed)
    out = []
    for _ in range(n):
        types = gen.schema_walk(g, gen.SCHOLARLY_STAR, int(g.integers(2, 7)))
        cons = []
        for i, t in enumerate(types):
            if g.random() < 0.4:
                continue
            nt = hin["types"][t]
            for _k in range(int(g.integers(1, 4))):
                kind = int(g.integers(6))
                if kind == 0:
                    lo = int(g.integers(1980, 2022))
                    cons.append({"pos": i, "prop": "year", "op": "range", "lo": lo, "hi": int(g.integers(lo, 2023))})
                elif kind == 1:
                    v = int(hin["props"][(t, "year")][int(g.integers(nt))])
                    cons.append({"pos": i, "prop": "year", "op": "eq", "lo": v})
                elif kind == 2:
                    vals = hin["props"][(t, "year")][g.integers(0, nt, size=int(g.integers(1, 4)))]
                    cons.append({"pos": i, "prop": "year", "op": "in", "set": np.unique(vals).astype(np.uint32)})
                elif kind == 3:
                    lo = int(g.integers(nt))
                    cons.append({"pos": i, "prop": None, "op": "range", "lo": lo, "hi": int(g.integers(lo, nt))})
                elif kind == 4:
                    cons.append({"pos": i, "prop": None, "op": "eq", "lo": int(g.integers(nt))})
                else:
                    ids = np.unique(g.integers(0, nt, size=int(g.integers(1, nt + 1)))).astype(np.uint32)
                    cons.append({"pos": i, "prop": None, "op": "in", "set": ids})
        out.append({"types": types, "constraints": cons})
    return out


@pytest.mark.parametrize("seed", range(8))
def test_oracle_matches_bruteforce_compound_constraints(seed):
    """Every constraint at a position must hold (Def. 3): the oracle's masks, ANDed over a
    position's constraints of all kinds, against the brute-force enumeration."""
    h = gen.tiny_hin(100 + seed, max_nodes=9)
    o = OracleHIN(h)
    adj = adjacency(h)
    nonempty = 0
    for q in _compound_queries(h, seed, 16):
        rp, ci, val = OC.evaluate(o, q)
        check_canonical(rp, ci, val, h["types"][q["types"][0]], h["types"][q["types"][-1]])
        want = enumerate_counts(h, q, adj)
        assert csr_to_dict(rp, ci, val) == want, q
        nonempty += bool(want)
    assert nonempty > 0  # the constraints leave some instances in some queries


def test_total_equals_instance_count():
    h = gen.tiny_hin(77, max_nodes=10)
    o = OracleHIN(h)
    for q in gen.random_queries(h, 77, 20, lengths=(3, 7), p_cons=0.3):
        rp, ci, val = OC.evaluate(o, q)
        assert int(val.sum()) == sum(enumerate_counts(h, q).values())


def _pairs(hin, a, b):
    for x, y, s, d in hin["relations"]:
        if (x, y) == (a, b):
            return set(zip(s.tolist(), d.tolist()))
        if (y, x) == (a, b):
            return set(zip(d.tolist(), s.tolist()))
    raise KeyError((a, b))


def test_length_two_is_masked_adjacency():
    h = gen.config1_hin()
    o = OracleHIN(h)
    year = h["props"][("P", "year")]
    q = {"types": ["P", "A"], "constraints": [{"pos": 0, "prop": "year", "op": "range", "lo": 2000, "hi": 2010},
                                              {"pos": 1, "prop": None, "op": "in", "set": np.arange(0, 1500, 3, dtype=np.uint32)}]}
    rp, ci, val = OC.evaluate(o, q)
    want = {(p, a): 1 for p, a in _pairs(h, "P", "A") if 2000 <= year[p] <= 2010 and a % 3 == 0}
    assert csr_to_dict(rp, ci, val) == want


def test_apa_closed_form():
    """APA[a, a] = number of (year-constrained) papers of a; APA[a, b] = number of papers
    a and b co-authored."""
    h = gen.config1_hin()
    o = OracleHIN(h)
    year = h["props"][("P", "year")]
    q = {"types": list("APA"), "constraints": [{"pos": 1, "prop": "year", "op": "range", "lo": 1995, "hi": 2015}]}
    got = csr_to_dict(*OC.evaluate(o, q))
    authors = {}
    for p, a in _pairs(h, "P", "A"):
        if 1995 <= year[p] <= 2015:
            authors.setdefault(p, set()).add(a)
    want = {}
    for p, al in authors.items():
        for a in al:
            for b in al:
                want[(a, b)] = want.get((a, b), 0) + 1
    assert got == want
    for (a, b), v in got.items():
        if a == b:
            assert v == sum(1 for al in authors.values() if a in al)


def test_pvp_block_diagonal():
    """Each paper has exactly one venue, so PVP is all-ones on venue blocks:
    nnz(PVP) = sum_v deg(v)^2 and every value is 1."""
    h = gen.config1_hin()
    o = OracleHIN(h)
    rp, ci, val = OC.evaluate(o, {"types": list("PVP"), "constraints": []})
    venue = {}
    for p, v in _pairs(h, "P", "V"):
        venue[p] = v
    deg = np.bincount(np.array(list(venue.values())), minlength=50)
    assert int(rp[-1]) == int((deg.astype(np.int64) ** 2).sum())
    assert np.all(val == 1)
    for p in range(0, 2000, 97):
        row = set(ci[rp[p]:rp[p + 1]].tolist())
        assert row == {q for q, v in venue.items() if v == venue.get(p, -1)}


def _scipy_adj(hin, a, b):
    pairs = _pairs(hin, a, b)
    r = np.array([x for x, _ in pairs], np.int64)
    c = np.array([y for _, y in pairs], np.int64)
    return sp.csr_matrix((np.ones(len(r), np.int64), (r, c)), shape=(hin["types"][a], hin["types"][b]))


def _scipy_mask(hin, t, cons):
    n = hin["types"][t]
    keep = np.ones(n, np.int64)
    for c in cons:
        v = np.arange(n) if c.get("prop") is None else hin["props"][(t, c["prop"])]
        if c["op"] == "range":
            keep &= ((v >= c["lo"]) & (v <= c["hi"])).astype(np.int64)
        elif c["op"] == "eq":
            keep &= (v == c["lo"]).astype(np.int64)
        else:
            keep &= np.isin(v, c["set"]).astype(np.int64)
    return sp.diags(keep, format="csr", dtype=np.int64)


def scipy_eval(hin, q):
    types = q["types"]
    R = _scipy_mask(hin, types[0], [c for c in q["constraints"] if c["pos"] == 0])
    for i in range(len(types) - 1):
        R = R @ _scipy_adj(hin, types[i], types[i + 1])
        R = R @ _scipy_mask(hin, types[i + 1], [c for c in q["constraints"] if c["pos"] == i + 1])
    R = sp.csr_matrix(R)
    R.eliminate_zeros()
    R.sort_indices()
    return R


def test_oracle_matches_scipy_on_2000_paper_hin():
    h = gen.config1_hin()
    o = OracleHIN(h)
    qs = [gen.config1_query()] + gen.random_queries(h, 5, 10, lengths=(3, 6), p_cons=0.3)
    for q in qs:
        rp, ci, val = OC.evaluate(o, q)
        R = scipy_eval(h, q)
        assert R.data.max(initial=0) < 2 ** 62
        np.testing.assert_array_equal(rp, R.indptr.astype(np.int64))
        np.testing.assert_array_equal(ci, R.indices.astype(np.int32))
        np.testing.assert_array_equal(val, R.data.astype(np.uint64))


def test_rowsum_colsum_chains_match_matrix():
    h = gen.config1_hin()
    o = OracleHIN(h)
    for q in [gen.config1_query()] + gen.random_queries(h, 9, 8, lengths=(2, 7), p_cons=0.4):
        f, m = o.query(q)
        rp, ci, val = OC.chain(f, m)
        rows = np.zeros(len(rp) - 1, np.uint64)
        np.add.at(rows, np.repeat(np.arange(len(rp) - 1), np.diff(rp)), val)
        np.testing.assert_array_equal(OC.rowsum(f, m), rows)
        cols = np.zeros(f[-1][3], np.uint64)
        np.add.at(cols, ci, val)
        np.testing.assert_array_equal(OC.colsum(f, m), cols)


def test_palindromic_query_is_symmetric():
    h = gen.config1_hin()
    o = OracleHIN(h)
    for name in ("APTPA", "APVPA", "TPAPT", "VPTPV", "APA"):
        q = {"types": list(name), "constraints": [c for c in gen._year_on_every(list(name), "P", 2000, 2015)]}
        rp, ci, val = OC.evaluate(o, q)
        M = sp.csr_matrix((val.astype(np.float64), ci, rp))
        assert (M != M.T).nnz == 0, name


def _eval_tree(tree, factors, masks):
    """Product of the sub-chain under `tree` with both end masks applied (masks are 0/1
    diagonals, so applying one twice changes nothing)."""
    if isinstance(tree, int):
        rp, ci, nr, nc = factors[tree]
        return OC.spgemm((np.arange(nr + 1, dtype=np.int64), np.arange(nr, dtype=np.int32), nr, nr),
                         (rp, ci, nr, nc), rmask=masks[tree], cmask=masks[tree + 1]) + (nr, nc)
    L = _eval_tree(tree[0], factors, masks)
    R = _eval_tree(tree[1], factors, masks)
    rp, ci, val = OC.spgemm((L[0], L[1], L[3], L[4], L[2]), (R[0], R[1], R[3], R[4], R[2]))
    return rp, ci, val, L[3], R[4]


def test_every_parenthesisation_gives_the_same_result():
    from oracle.planner import all_trees
    h = gen.config1_hin()
    o = OracleHIN(h)
    for q in gen.random_queries(h, 11, 6, lengths=(4, 6), p_cons=0.5):
        f, m = o.query(q)
        ref = OC.chain(f, m)
        for tree in all_trees(0, len(f) - 1):
            got = _eval_tree(tree, f, m)
            for a, b in zip(ref, got[:3]):
                np.testing.assert_array_equal(a, b)


def test_overflow_is_reported_not_wrapped():
    X = (np.array([0, 2], np.int64), np.array([0, 1], np.int32), 1, 2, np.array([2 ** 63, 2 ** 63], np.uint64))
    Y = (np.array([0, 1, 2], np.int64), np.array([0, 0], np.int32), 2, 1)
    with pytest.raises(OC.OracleOverflow):
        OC.spgemm(X, Y)
    X2 = (X[0], X[1], 1, 2, np.array([2 ** 62, 2 ** 62], np.uint64))
    rp, ci, val = OC.spgemm(X2, Y)
    assert int(val[0]) == 2 ** 63
    Y3 = (Y[0], Y[1], 2, 1, np.array([4, 1], np.uint64))
    with pytest.raises(OC.OracleOverflow):
        OC.spgemm(X2, Y3)


def test_empty_and_degenerate():
    h = gen.config1_hin()
    o = OracleHIN(h)
    q = {"types": list("APTPA"), "constraints": [{"pos": 2, "prop": None, "op": "in", "set": np.zeros(0, np.uint32)}]}
    rp, ci, val = OC.evaluate(o, q)
    assert rp.shape == (1501,) and rp[-1] == 0 and ci.size == 0
    q = {"types": list("APA"), "constraints": [{"pos": 1, "prop": "year", "op": "range", "lo": 3000, "hi": 4000}]}
    assert OC.evaluate(o, q)[0][-1] == 0
