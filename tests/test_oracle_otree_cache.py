"""Pins of the Overlap Tree and cache-policy oracles (Sec. 3.3, Sec. 3.4, Alg. 1).

Tree: the space bounds of Sec. 3.3.3 (lambda = sum |m_i| leaves, every internal node with
at least two children, at most 2*lambda - 1 nodes besides the root), f = 1 at leaves, and
every node's / every substring's frequency equal to a brute-force count of occurrences
(with and without constraint keys). Cache: hand traces of Alg. 1's utilities, inflation
and subtree cost subtract / reinstate, the 80 % rule, PGDS and LRU."""
import itertools

import numpy as np
import pytest

from oracle.cache import Cache, in_subtree
from oracle.otree import OverlapTree, constraint_key, is_terminator


def _brute_count(queries, s):
    s = tuple(s)
    return sum(1 for q in queries for k in range(len(q) - len(s) + 1) if tuple(q[k:k + len(s)]) == s)


def _random_workload(seed, n=30, alphabet="APVT", lengths=(2, 7)):
    rng = np.random.default_rng(seed)
    return [tuple(rng.choice(list(alphabet), size=int(rng.integers(lengths[0], lengths[1] + 1))))
            for _ in range(n)]


@pytest.mark.parametrize("seed", range(10))
def test_space_bounds_and_leaf_frequency(seed):
    qs = _random_workload(seed)
    t = OverlapTree()
    for q in qs:
        t.insert(q)
    lam = sum(len(q) for q in qs)
    leaves = list(t.leaves())
    assert len(leaves) == lam == t.n_leaves
    assert all(x.f == 1 for x in leaves)
    nodes = [x for x in t.nodes() if x is not t.root]
    assert len(nodes) <= 2 * lam - 1
    for x in nodes:
        if not x.is_leaf():
            assert len(x.children) >= 2


@pytest.mark.parametrize("seed", range(10))
def test_frequencies_equal_bruteforce_occurrences(seed):
    qs = _random_workload(100 + seed, n=25)
    t = OverlapTree()
    for q in qs:
        t.insert(q)
    for x in t.nodes():
        if x is t.root:
            continue
        s = x.string()
        if any(is_terminator(c) for c in s):
            assert x.f == 1
        else:
            assert x.f == _brute_count(qs, s), s
    subs = {q[i:j] for q in qs for i in range(len(q)) for j in range(i + 1, len(q) + 1)}
    for s in subs:
        assert t.frequency(s) == _brute_count(qs, s), s
    assert t.frequency(("X",)) == 0


def test_narrative_icpa_example():
    """Sec. 3.3.1 / 3.4: ICPA occurs in all three queries (f = 3); after a query with
    ICPALA arrives, ICPAL (seen twice, followed by different symbols) is an internal node
    in ICPA's subtree."""
    qs = ["ICPA", "TICPAL", "ICPAT"]
    t = OverlapTree()
    for q in qs:
        t.insert(tuple(q))
    n, exact = t.locate(tuple("ICPA"))
    assert exact and n.f == 3 and not n.is_leaf()
    t.insert(tuple("ICPALA"))
    n2, exact2 = t.locate(tuple("ICPAL"))
    assert exact2 and not n2.is_leaf() and n2.f == 2
    assert n2.parent is n
    assert t.frequency(tuple("ICPA")) == 4
    assert t.frequency(tuple("CPA")) == 4


def _window_key(cons, start, length):
    return constraint_key(cons, start, length)


@pytest.mark.parametrize("seed", range(6))
def test_constraint_index_frequencies(seed):
    rng = np.random.default_rng(seed)
    qs = _random_workload(200 + seed, n=20, alphabet="APV", lengths=(2, 6))
    cons = []
    for q in qs:
        c = {}
        for i in range(len(q)):
            if rng.random() < 0.3:
                c[i] = (f"year>={int(rng.integers(2000, 2003))}",)
        cons.append(c)
    t = OverlapTree()
    for q, c in zip(qs, cons):
        t.insert(q, c)
    for q in qs:
        for i, j in itertools.combinations(range(len(q) + 1), 2):
            s = q[i:j]
            keys = {_window_key(c, k, len(s)) for qq, c in zip(qs, cons)
                    for k in range(len(qq) - len(s) + 1) if qq[k:k + len(s)] == s}
            for key in keys:
                want = sum(1 for qq, c in zip(qs, cons) for k in range(len(qq) - len(s) + 1)
                           if qq[k:k + len(s)] == s and _window_key(c, k, len(s)) == key)
                assert t.frequency(s, key) == want, (s, key)


# ---------------------------------------------------------------- Alg. 1

def test_pgds_utilities_and_inflation_hand_trace():
    c = Cache(10, "pgds")
    assert c.request("a", 1, 8, 4) == "inserted"      # h = 8/4 + 0 = 2
    assert c.request("b", 1, 4, 4) == "inserted"      # h = 1
    assert c.request("c", 1, 12, 4) == "inserted"     # full: L = 1, evict b; h_c = 3 + 1
    assert c.evicted == ["b"] and c.L == 1
    assert c.entries["c"].h == 4 and c.entries["a"].h == 2
    assert c.request("a", 2, 8, 4) == "hit"           # l_a = L = 1: h = 2*8/4 + 1 = 5
    assert c.entries["a"].h == 5
    assert c.request("d", 1, 4, 4) == "inserted"      # evict c (h 4 < 5): L = 4, h_d = 1 + 4
    assert c.evicted == ["b", "c"] and c.L == 4 and c.entries["d"].h == 5
    assert set(c.entries) == {"a", "d"}


def test_eighty_percent_rule():
    c = Cache(10, "atrapos")
    assert c.request("big", 1, 100, 8.5) == "rejected"
    assert c.request("ok", 1, 100, 8.0) == "inserted"


def test_atrapos_subtree_cost_subtract_and_reinstate():
    """Sec. 3.4.2: caching ICPA makes cached ICPAL cheaper to recompute (its cost drops by
    ICPA's); evicting ICPA reinstates it."""
    icpal = (tuple("ICPAL"), "")
    icpa = (tuple("ICPA"), "")
    other = (tuple("VPV"), "")
    assert in_subtree(icpa, icpal) and not in_subtree(icpal, icpa)
    c = Cache(12, "atrapos")
    c.request(icpal, 2, 10, 4)           # h = 2*10/4 = 5
    c.request(icpa, 3, 6, 4)             # h = 3*6/4 = 4.5; ICPAL cost 10 - 6 = 4 -> h = 2
    assert c.entries[icpal].c == 4 and c.entries[icpal].h == 2
    c.request(other, 1, 40, 4)           # h = 10
    # next insertion must evict the smallest utility: ICPAL (h 2)
    c.request((tuple("TPT"), ""), 1, 40, 4)
    assert c.evicted == [icpal] and c.L == 2
    # evicting ICPA now gives nothing back (ICPAL is gone); re-add ICPAL, then evict ICPA
    c2 = Cache(8, "atrapos")
    c2.request(icpa, 1, 6, 4)            # h = 1.5
    c2.request(icpal, 5, 10, 4)          # cached after ICPA: cost kept as measured, h = 12.5
    c2.request(icpa, 1, 6, 4)            # hit
    c2.request((tuple("VPV"), ""), 1, 80, 4)   # evict ICPA (h 1.5): ICPAL gets +6 -> 16
    assert c2.evicted == [icpa]
    assert c2.entries[icpal].c == 16 and c2.entries[icpal].h == pytest.approx(5 * 16 / 4 + 0)


def test_subtree_respects_constraints():
    assert in_subtree((tuple("APT"), "1:y"), (tuple("APTP"), "1:y|3:y"))
    assert not in_subtree((tuple("APT"), "1:y"), (tuple("APTP"), "3:y"))
    assert not in_subtree((tuple("APT"), ""), (tuple("APT"), ""))


def test_lru_evicts_least_recently_requested():
    c = Cache(12, "lru")
    for k in "abc":
        c.request(k, 1, 1, 4)
    c.request("a", 1, 1, 4)
    c.request("d", 1, 1, 4)
    assert c.evicted == ["b"]
    c.request("e", 1, 1, 4)
    assert c.evicted == ["b", "c"]


def test_pgds_ignores_subtree():
    icpal = (tuple("ICPAL"), "")
    icpa = (tuple("ICPA"), "")
    c = Cache(12, "pgds")
    c.request(icpal, 2, 10, 4)
    c.request(icpa, 3, 6, 4)
    assert c.entries[icpal].c == 10


# ---------------------------------------------------------------- reductions and invariants

def _lru_evictions(trace, slots):
    """Textbook LRU over unit-size items: the evicted keys in order."""
    from collections import OrderedDict
    held, out = OrderedDict(), []
    for k in trace:
        if k in held:
            held.move_to_end(k)
            continue
        if len(held) == slots:
            out.append(held.popitem(last=False)[0])
        held[k] = True
    return out


@pytest.mark.parametrize("seed", range(6))
def test_greedy_dual_with_uniform_items_is_lru(seed):
    """With every frequency, cost and size equal, h = const + l and l only grows, so the
    smallest utility is the entry touched longest ago: PGDS and ATRAPOS (keys with no
    prefix relation) evict exactly as LRU does (the Greedy-Dual reduction to LRU)."""
    rng = np.random.default_rng(700 + seed)
    keys = [(tuple(f"K{i:02d}"), "") for i in range(12)]  # keys of one length: none a prefix of another
    trace = [keys[int(i)] for i in rng.integers(0, len(keys), size=300)]
    want = _lru_evictions(trace, 5)
    for policy in ("pgds", "atrapos", "lru"):
        c = Cache(5, policy, max_fraction=1.0)
        for k in trace:
            c.request(k, 1, 1, 1)
        assert c.evicted == want, policy


@pytest.mark.parametrize("seed", range(6))
def test_atrapos_without_subtrees_is_pgds(seed):
    """Alg. 1's subtree cost updates act only between keys where one is a proper prefix of
    the other; on keys of one length ATRAPOS and PGDS make the same choices."""
    rng = np.random.default_rng(800 + seed)
    keys = [(tuple(rng.choice(list("APVT"), size=3)), "") for _ in range(15)]
    a, p = Cache(40, "atrapos"), Cache(40, "pgds")
    for _ in range(400):
        k = keys[int(rng.integers(len(keys)))]
        f, cost, size = int(rng.integers(1, 6)), float(rng.integers(1, 50)), float(rng.integers(1, 12))
        assert a.request(k, f, cost, size) == p.request(k, f, cost, size)
    assert a.evicted == p.evicted and a.L == p.L


@pytest.mark.parametrize("policy", ["atrapos", "pgds", "lru"])
def test_capacity_and_accounting_invariants(policy):
    """After every request the bytes held equal the sum of the entries' sizes and never
    pass the capacity, and costs stay non-negative. Under PGDS the inflation L never
    decreases (every cached utility is at least the L it was set with); under ATRAPOS it can,
    since a cached sub-metapath lowers the costs, hence the utilities, of its subtree."""
    rng = np.random.default_rng(900)
    alphabet = list("APVT")
    keys = []
    for _ in range(40):
        n = int(rng.integers(2, 6))
        keys.append((tuple(rng.choice(alphabet, size=n)), ""))
    keys += [(k[0][:2], "") for k in keys[:10]]  # prefixes, so subtrees exist
    c = Cache(100, policy)
    last_L = 0.0
    for _ in range(1500):
        k = keys[int(rng.integers(len(keys)))]
        c.request(k, int(rng.integers(1, 9)), float(rng.integers(1, 100)), float(rng.integers(1, 40)))
        assert c.used == pytest.approx(sum(e.s for e in c.entries.values()))
        assert c.used <= c.capacity + 1e-9
        assert all(e.c >= 0 for e in c.entries.values())
        if policy == "pgds":
            assert c.L >= last_L
        last_L = c.L
