"""Cache replacement policies for the oracle (test infrastructure only).

Sec. 3.4.2 and Alg. 1 (ATRAPOS-OTree): every cached entry e has a utility
h_e = f_e * c_e / s_e + l_e, with f its frequency, c its cost, s its size and l the value
of the inflation variable L when e was last inserted or hit (popularity-aware greedy
dual-size, PGDS). A request for an item p:
  * raises f_p (the frequency comes from the Overlap Tree, which counts occurrences);
  * on a hit, sets l_p = L and recomputes h_p;
  * on a miss, while p does not fit, sets L to the smallest utility in the cache, evicts
    an entry q with h_q = L and gives every cached entry e in q's subtree its cost back
    (c_e += c_q, h_e recomputed); then inserts p with l_p = L and takes p's cost off every
    cached entry in p's subtree (c_e -= c_p, clamped at 0, h_e recomputed).
"Subtree" follows the Overlap Tree: e is in p's subtree when p's sub-metapath is a proper
prefix of e's (same constraints on the shared positions), so e can be computed from p.
Items larger than 80 % of the capacity are never cached (Sec. 4.1.4).

PGDS is the same without the subtree cost adjustments; LRU evicts the least recently
requested entry. Ties between equal utilities go to the entry inserted or hit first.
"""
from __future__ import annotations


class CacheEntry:
    __slots__ = ("key", "f", "c", "s", "h", "l", "seq")

    def __init__(self, key, f, c, s, l, seq):
        self.key, self.f, self.c, self.s, self.l, self.seq = key, f, c, s, l, seq
        self.h = 0.0


def in_subtree(parent_key, child_key):
    """Keys are (types tuple, constraint key). child is in parent's subtree when parent's
    types are a proper prefix of child's and the constraints agree on the shared part."""
    from .otree import restrict_key
    pt, pk = parent_key
    ct, ck = child_key
    return len(pt) < len(ct) and tuple(ct[:len(pt)]) == tuple(pt) and restrict_key(ck, len(pt)) == pk


class Cache:
    def __init__(self, capacity, policy="atrapos", max_fraction=0.8):
        assert policy in ("atrapos", "pgds", "lru")
        self.capacity = float(capacity)
        self.policy = policy
        self.max_fraction = max_fraction
        self.L = 0.0
        self.entries = {}
        self.used = 0.0
        self.seq = 0
        self.evicted = []   # keys, in eviction order

    def _util(self, e):
        e.h = e.f * e.c / e.s + e.l

    def _tick(self):
        self.seq += 1
        return self.seq

    def request(self, key, f, c, s):
        """One request of item `key` with tree frequency f, cost c and size s (bytes).
        Returns "hit", "inserted" or "rejected"."""
        e = self.entries.get(key)
        if e is not None:
            e.f = f
            e.l = self.L
            e.seq = self._tick()
            self._util(e)
            return "hit"
        if s > self.max_fraction * self.capacity:
            return "rejected"
        while self.used + s > self.capacity and self.entries:
            q = self._victim()
            if self.policy != "lru":
                self.L = q.h
            del self.entries[q.key]
            self.used -= q.s
            self.evicted.append(q.key)
            if self.policy == "atrapos":
                for e2 in self.entries.values():
                    if in_subtree(q.key, e2.key):
                        e2.c += q.c
                        self._util(e2)
        p = CacheEntry(key, f, float(c), float(s), self.L, self._tick())
        self._util(p)
        self.entries[key] = p
        self.used += s
        if self.policy == "atrapos":
            for e2 in self.entries.values():
                if e2 is not p and in_subtree(key, e2.key):
                    e2.c = max(0.0, e2.c - p.c)
                    self._util(e2)
        return "inserted"

    def _victim(self):
        if self.policy == "lru":
            return min(self.entries.values(), key=lambda e: e.seq)
        return min(self.entries.values(), key=lambda e: (e.h, e.seq))
