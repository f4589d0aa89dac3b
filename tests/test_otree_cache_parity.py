"""The engine's Overlap Tree and cache policies (host code, replayed through the
host-only C entry points) against the oracle's on random workload traces."""
import itertools

import numpy as np
import pytest

from oracle.cache import Cache
from oracle.otree import OverlapTree, constraint_key


def _workload(seed, n=40, alphabet=4, lengths=(2, 7)):
    rng = np.random.default_rng(seed)
    qs, cons = [], []
    for _ in range(n):
        L = int(rng.integers(lengths[0], lengths[1] + 1))
        q = tuple(int(x) for x in rng.integers(0, alphabet, L))
        c = {}
        for i in range(L):
            if rng.random() < 0.25:
                c[i] = (f"p{int(rng.integers(0, 2))}in{int(rng.integers(0, 3))}",)
        qs.append(q)
        cons.append(c)
    return qs, cons


def _pos_keys(q, c):
    return ["&".join(c[i]) if i in c else "" for i in range(len(q))]


def _check_tree(qs, cons, construction):
    from paper_2201_04058_b300 import mp
    ot, et = OverlapTree(), mp.OTree(construction)
    for q, c in zip(qs, cons):
        ot.insert(q, c)
        et.insert(q, _pos_keys(q, c))
    nodes, leaves, ok = et.info()
    assert ok
    assert leaves == ot.n_leaves == sum(len(q) for q in qs)
    assert nodes == sum(1 for x in ot.nodes() if x is not ot.root)
    subs = {q[i:j] for q in qs for i in range(len(q)) for j in range(i + 1, len(q) + 1)}
    for s in sorted(subs):
        assert et.frequency(s) == ot.frequency(s), s
        keys = {constraint_key(c, k, len(s)) for q, c in zip(qs, cons)
                for k in range(len(q) - len(s) + 1) if q[k:k + len(s)] == s}
        for key in keys:
            assert et.frequency(s, key) == ot.frequency(s, key), (s, key)
    assert et.frequency((9, 9)) == 0


@pytest.mark.parametrize("construction", [0, 1])
@pytest.mark.parametrize("seed", range(12))
def test_tree_frequencies_match_oracle(seed, construction):
    """Both constructions of the engine's tree (the naive insertion of Sec. 3.3.2 and the
    on-line Ukkonen construction its footnote points to) against the oracle's tree."""
    qs, cons = _workload(seed)
    _check_tree(qs, cons, construction)


@pytest.mark.parametrize("seed", range(8))
def test_online_tree_on_repetitive_metapaths(seed):
    """Long metapaths over two or three symbols (runs like ABABAB and AAAA, where suffix
    links and walk-downs matter most), and repeated whole queries."""
    rng = np.random.default_rng(500 + seed)
    qs, cons = [], []
    for _ in range(30):
        L = int(rng.integers(1, 13))
        period = int(rng.integers(1, 4))
        base = rng.integers(0, 2 + seed % 2, period)
        q = tuple(int(base[i % period]) for i in range(L))
        if rng.random() < 0.2 and qs:
            q = qs[int(rng.integers(len(qs)))]
        c = {i: (f"p0in{int(rng.integers(0, 2))}",) for i in range(L) if rng.random() < 0.2}
        qs.append(q)
        cons.append(c)
    _check_tree(qs, cons, 1)


@pytest.mark.parametrize("policy,seed", list(itertools.product([0, 1, 2], range(10))))
def test_cache_decisions_match_oracle(policy, seed):
    """Same request trace -> same outcomes, evictions (in order), costs and utilities."""
    from paper_2201_04058_b300 import mp
    rng = np.random.default_rng(1000 + seed)
    name = {0: "atrapos", 1: "pgds", 2: "lru"}[policy]
    cap = float(rng.integers(50, 200))
    oc, ec = Cache(cap, name), mp.CacheSim(cap, policy)
    # items: prefixes and extensions of a few base strings so subtree relations occur
    bases = [tuple(int(x) for x in rng.integers(0, 3, int(rng.integers(3, 7)))) for _ in range(5)]
    items = set()
    for b in bases:
        for L in range(2, len(b) + 1):
            items.add((b[:L], ""))
            items.add((b[:L], "0:x" if rng.random() < 0.3 else ""))
    items = sorted(items)
    for step in range(120):
        t, k = items[int(rng.integers(len(items)))]
        f = int(rng.integers(1, 6))
        c = float(rng.integers(1, 100))
        s = float(rng.integers(1, 60))
        o1 = oc.request((t, k), f, c, s)
        o2 = ec.request(t, k, f, c, s)
        assert o1 == o2, (step, o1, o2)
    assert ec.evicted() == [mp.cache_item_id(t, k) for t, k in oc.evicted]
    L, used, n = ec.state()
    assert L == pytest.approx(oc.L) and used == pytest.approx(oc.used) and n == len(oc.entries)
    for (t, k), e in oc.entries.items():
        c, h = ec.entry(t, k)
        assert c == pytest.approx(e.c) and h == pytest.approx(e.h)
