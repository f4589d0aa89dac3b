"""Typed 0/1 adjacency matrices and constraint masks for the oracle (test infrastructure).

Def. 1 (Sec. 2): for a relation r between node types o' and o'', A_r is the |o'| x |o''|
matrix with A_r[i, j] = 1 when node i of type o' is linked to node j of type o'', else 0.
Repeated edges collapse to a single 1. Relations are bidirectional (Sec. 1, and the HIN
tables of Sec. 4.1.1), so each generated relation yields A_r and its transpose.

Def. 3 and the constrained adjacency of Problem 1: a constraint on position i becomes
the 0/1 diagonal M_{c_i}; here it is a uint8 vector over the nodes of type o_i (1 =
satisfies every constraint at that position). A position without constraints has no
mask (the identity).
"""
import numpy as np


def csr_from_pairs(src, dst, n_rows, n_cols):
    """0/1 CSR (int64 row pointers, int32 columns ascending per row) of the edge list."""
    key = np.asarray(src, np.int64) * int(n_cols) + np.asarray(dst, np.int64)
    key = np.sort(key)
    if key.size:
        key = key[np.concatenate(([True], key[1:] != key[:-1]))]
    r = key // int(n_cols)
    c = (key % int(n_cols)).astype(np.int32)
    rp = np.zeros(int(n_rows) + 1, np.int64)
    np.cumsum(np.bincount(r, minlength=int(n_rows)), out=rp[1:])
    return rp, c


class OracleHIN:
    """All typed adjacency matrices of a generated HIN, in both directions."""

    def __init__(self, hin):
        self.types = dict(hin["types"])
        self.props = dict(hin["props"])
        self.rel = {}
        for a, b, s, d in hin["relations"]:
            na, nb = self.types[a], self.types[b]
            self.rel[(a, b)] = csr_from_pairs(s, d, na, nb)
            self.rel[(b, a)] = csr_from_pairs(d, s, nb, na)

    def mask(self, node_type, constraints):
        """uint8 mask of the nodes of `node_type` that satisfy every constraint, or
        None when there are no constraints."""
        if not constraints:
            return None
        n = self.types[node_type]
        ids = np.arange(n, dtype=np.int64)
        m = np.ones(n, dtype=bool)
        for c in constraints:
            v = ids if c.get("prop") is None else self.props[(node_type, c["prop"])].astype(np.int64)
            op = c["op"]
            if op == "range":
                m &= (v >= int(c["lo"])) & (v <= int(c["hi"]))
            elif op == "eq":
                m &= v == int(c["lo"])
            elif op == "in":
                m &= np.isin(v, np.asarray(c["set"], np.int64))
            else:
                raise ValueError(f"unknown constraint op {op!r}")
        return m.astype(np.uint8)

    def query(self, q):
        """(factors, masks) of a query: factors[t] = (rp, ci, n_rows, n_cols) of the
        relation from position t to t+1; masks[i] for position i (None = identity)."""
        types = q["types"]
        if len(types) < 2:
            raise ValueError("a metapath needs at least two node types")
        factors = []
        for t in range(len(types) - 1):
            a, b = types[t], types[t + 1]
            if (a, b) not in self.rel:
                raise ValueError(f"no relation {a}{b} in the schema")
            rp, ci = self.rel[(a, b)]
            factors.append((rp, ci, self.types[a], self.types[b]))
        masks = []
        for i, t in enumerate(types):
            masks.append(self.mask(t, [c for c in q.get("constraints", []) if c["pos"] == i]))
        return factors, masks
