"""Brute-force metapath instance enumeration for tiny HINs (test helper).

Works straight from the generator's edge lists and property arrays with Python sets and
loops, so it shares nothing with the oracle's CSR and mask code: an instance of a
metapath <o_1 ... o_n> (Def. 2) is a node sequence v_1..v_n with v_i of type o_i, each
consecutive pair linked by the relation between o_i and o_{i+1} (repeated edges count
once: the 0/1 adjacency of Def. 1), and each v_i meeting every constraint at position i
(Def. 3).
"""
from collections import defaultdict


def adjacency(hin):
    adj = defaultdict(lambda: defaultdict(set))
    for a, b, s, d in hin["relations"]:
        for x, y in zip(s.tolist(), d.tolist()):
            adj[(a, b)][x].add(y)
            adj[(b, a)][y].add(x)
    return adj


def passes(hin, node_type, v, cons):
    for c in cons:
        val = v if c.get("prop") is None else int(hin["props"][(node_type, c["prop"])][v])
        if c["op"] == "range" and not (int(c["lo"]) <= val <= int(c["hi"])):
            return False
        if c["op"] == "eq" and val != int(c["lo"]):
            return False
        if c["op"] == "in" and val not in set(int(x) for x in c["set"]):
            return False
    return True


def enumerate_counts(hin, query, adj=None):
    """{(u, v): number of instances} over all instances of the query."""
    adj = adj or adjacency(hin)
    types = query["types"]
    cons = [[c for c in query.get("constraints", []) if c["pos"] == i] for i in range(len(types))]
    counts = defaultdict(int)

    def dfs(i, start, v):
        if i == len(types) - 1:
            counts[(start, v)] += 1
            return
        for w in sorted(adj[(types[i], types[i + 1])].get(v, ())):
            if passes(hin, types[i + 1], w, cons[i + 1]):
                dfs(i + 1, start, w)

    for u in range(hin["types"][types[0]]):
        if passes(hin, types[0], u, cons[0]):
            dfs(0, u, u)
    return dict(counts)


def csr_to_dict(rp, ci, val):
    out = {}
    for i in range(len(rp) - 1):
        for p in range(int(rp[i]), int(rp[i + 1])):
            out[(i, int(ci[p]))] = int(val[p])
    return out


def check_canonical(rp, ci, val, nrows, ncols):
    """Canonical CSR: monotone row pointers, strictly ascending in-range columns per row,
    no stored zeros."""
    assert len(rp) == nrows + 1 and rp[0] == 0
    assert all(rp[i] <= rp[i + 1] for i in range(nrows))
    assert len(ci) == rp[-1] == len(val)
    for i in range(nrows):
        row = ci[rp[i]:rp[i + 1]]
        assert all(0 <= int(c) < ncols for c in row)
        assert all(int(row[t]) < int(row[t + 1]) for t in range(len(row) - 1))
    assert all(int(v) >= 1 for v in val)
