"""GPU: batches of queries through one product DAG, and the Overlap-Tree cache (Sec. 3.3,
3.4, Alg. 1) under every policy and budget, give the oracle's results bit for bit; each
query's result is the same alone and in the mix."""
import numpy as np
import pytest

import gen
from oracle import chain as OC
from oracle.hin import OracleHIN

from test_gpu_parity import assert_same

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c1():
    h = gen.config1_hin()
    return h, OracleHIN(h)


@pytest.fixture(scope="module")
def batch_queries(c1):
    qs = gen.batched_queries(seed=3, n=64, pool=20, anchor_p=0.5)
    return qs, [OC.evaluate(c1[1], q) for q in qs]


def _mp():
    from paper_2201_04058_b300 import mp
    return mp


@pytest.mark.parametrize("policy", [3, 0, 1, 2])
@pytest.mark.parametrize("budget", [8 << 30, 2 << 20])
def test_batch_matches_oracle_every_policy(c1, batch_queries, cuda_ok, policy, budget):
    mp = _mp()
    qs, want = batch_queries
    e = mp.Engine(c1[0], policy=policy, cache_bytes=budget)
    try:
        for rnd in range(2):  # the second round meets a warm cache
            rc, res = e.run_batch(qs)
            assert rc == 0
            for q, g, w in zip(qs, res, want):
                assert_same(g, w, (policy, budget, rnd, "".join(q["types"])))
        if policy != 3:
            st = mp.mp_cache_stats(e.ctx)
            assert st["inserts"] > 0 and st["hits"] > 0
            assert st["bytes"] <= budget
            if budget < (4 << 20):
                assert st["evictions"] > 0 or st["rejected"] > 0
    finally:
        e.close()


def test_each_result_same_alone_and_in_mix(c1, batch_queries, cuda_ok):
    mp = _mp()
    qs, want = batch_queries
    e = mp.Engine(c1[0], policy=mp.MP_POLICY_NONE)
    try:
        rc, mixed = e.run_batch(qs)
        assert rc == 0
        for q, g in zip(qs[:24], mixed[:24]):
            assert_same(e.run(q), g, "alone vs mix")
    finally:
        e.close()


def test_batch_shares_identical_products(c1, cuda_ok):
    mp = _mp()
    q = {"types": list("APTPA"), "constraints": gen._year_on_every(list("APTPA"), "P", 2000, 2015)}
    e = mp.Engine(c1[0], policy=mp.MP_POLICY_NONE)
    try:
        rc, tickets = e.submit_batch([q] * 4)
        assert rc == 0
        n = [mp.mp_result_stats(e.ctx, t)["n_products"] for t in tickets]
        assert n[0] >= 2 and sum(n[1:]) == 0  # the first query ran every product once
        first = e.fetch(tickets[0])
        for t in tickets:
            assert_same(e.fetch(t), first, "shared")
            e.release(t)
    finally:
        e.close()


def test_repeated_query_is_a_cache_hit(c1, cuda_ok):
    mp = _mp()
    q = gen.config1_query()
    want = OC.evaluate(c1[1], q)
    e = mp.Engine(c1[0], policy=mp.MP_POLICY_ATRAPOS)
    try:
        assert_same(e.run(q), want, "first")
        s1 = mp.mp_cache_stats(e.ctx)
        rc, t = e.submit(q)
        assert rc == 0
        assert mp.mp_result_stats(e.ctx, t)["n_products"] == 0
        assert_same(e.fetch(t), want, "cached")
        e.release(t)
        s2 = mp.mp_cache_stats(e.ctx)
        assert s2["hits"] > s1["hits"]
    finally:
        e.close()


def test_long_metapaths_with_squeezed_cache(c1, cuda_ok):
    """Long metapaths through venues and topics, with a budget far below the distinct
    intermediates, replayed with and without caching."""
    mp = _mp()
    qs = gen.long_queries(5, 16)
    want = [OC.evaluate(c1[1], q) for q in qs]
    for policy, budget in ((3, 1 << 30), (0, 6 << 20), (1, 6 << 20), (2, 6 << 20)):
        e = mp.Engine(c1[0], policy=policy, cache_bytes=budget)
        try:
            for rnd in range(2):
                for q, w in zip(qs, want):
                    assert_same(e.run(q), w, (policy, "".join(q["types"])))
        finally:
            e.close()


@pytest.mark.parametrize("insertion,policy", [(1, 2), (2, 2), (2, 0), (1, 1)])
def test_cache_baselines_match_oracle(c1, batch_queries, cuda_ok, insertion, policy):
    """Final-results-only + LRU (CBS1) and all-intermediates + LRU (CBS2), and the other
    combinations, change what is cached, never the results."""
    mp = _mp()
    qs, want = batch_queries
    e = mp.Engine(c1[0], policy=policy, insertion=insertion, cache_bytes=3 << 20)
    try:
        for rnd in range(2):
            rc, res = e.run_batch(qs)
            assert rc == 0
            for q, g, w in zip(qs, res, want):
                assert_same(g, w, (insertion, policy, rnd, "".join(q["types"])))
        st = mp.mp_cache_stats(e.ctx)
        assert st["inserts"] > 0
    finally:
        e.close()


@pytest.mark.parametrize("host_bytes", [256 << 20, 256 << 10])
def test_host_tier_results_and_reuse(c1, batch_queries, cuda_ok, host_bytes):
    """A device cache far too small for the batch's intermediates, every computed node
    offered (CBS2), and a second tier in host memory: evicted results go down, later plans
    copy some back instead of recomputing them, and every result stays the oracle's. A host
    tier smaller than the evicted results drops its least recently used entries."""
    mp = _mp()
    qs, want = batch_queries
    e = mp.Engine(c1[0], policy=mp.MP_POLICY_ATRAPOS, cache_bytes=2 << 20, host_tier_bytes=host_bytes,
                  insertion=mp.MP_INSERT_ALL)
    try:
        for rnd in range(3):
            rc, res = e.run_batch(qs)
            assert rc == 0
            for q, g, w in zip(qs, res, want):
                assert_same(g, w, ("host tier", host_bytes, rnd, "".join(q["types"])))
        st = mp.mp_host_tier_stats(e.ctx)
        assert st["stores"] > 0
        assert st["bytes"] <= host_bytes
        if host_bytes >= (256 << 20):
            assert st["loads"] > 0
        else:
            assert st["drops"] > 0 or st["entries"] == st["stores"]
    finally:
        e.close()
