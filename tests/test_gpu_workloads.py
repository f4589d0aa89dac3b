"""GPU parity on the benchmark's workloads, every query against the CPU oracle bit for bit:
  * the batched workload (256 queries drawn Zipf(1.1) from a pool of 500 templates, 75 %
    anchored on an entity of interest) as one batch, with and without the cache;
  * the stress workload (all 64 metapaths of length 7-9 through venues and topics) as one
    batch, and replayed one query at a time under a cache squeezed to force evictions;
  * the news-shaped serving workload (a scaled news HIN: articles, persons, organisations,
    locations, themes; session queries with an anchor entity and a date window on every
    article position) through the serving loop with Poisson arrivals."""
import time

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


def _mp():
    from paper_2201_04058_b300 import mp
    return mp


@pytest.mark.parametrize("policy", [3, 0])
def test_batched_workload_matches_oracle(c1, cuda_ok, policy):
    mp = _mp()
    h, o = c1
    qs = gen.batched_queries(seed=3, n=256, pool=500, anchor_p=0.75)
    want = [OC.evaluate(o, q) for q in qs]
    e = mp.Engine(h, policy=policy)
    try:
        for rnd in range(2):
            rc, res = e.run_batch(qs)
            assert rc == 0
            for i, (g, w) in enumerate(zip(res, want)):
                assert_same(g, w, ("batched", policy, rnd, i))
    finally:
        e.close()


def test_stress_workload_matches_oracle(c1, cuda_ok):
    mp = _mp()
    h, o = c1
    qs = gen.long_queries(5, 64)
    want = [OC.evaluate(o, q) for q in qs]
    e = mp.Engine(h, policy=mp.MP_POLICY_NONE)
    try:
        rc, res = e.run_batch(qs)
        assert rc == 0
        for i, (g, w) in enumerate(zip(res, want)):
            assert_same(g, w, ("stress batch", i))
    finally:
        e.close()
    for pol in (mp.MP_POLICY_ATRAPOS, mp.MP_POLICY_PGDS, mp.MP_POLICY_LRU):
        e = mp.Engine(h, policy=pol, cache_bytes=6 << 20)
        try:
            for rnd in range(2):
                for i, (q, w) in enumerate(zip(qs, want)):
                    assert_same(e.run(q), w, ("stress replay", pol, rnd, i))
            assert mp.mp_cache_stats(e.ctx)["evictions"] > 0
        finally:
            e.close()


@pytest.mark.parametrize("policy", [0, 3])
def test_news_serving_stream_matches_oracle(cuda_ok, policy):
    """A 20,000-article news HIN (1/500 of the benchmark's), 400 session queries with
    date windows and anchors, arriving as a Poisson process through the serving loop."""
    mp = _mp()
    h = gen.config4_hin(seed=4, scale=0.002)
    o = OracleHIN(h)
    qs, arrivals = gen.serving_stream(h, seed=4, n=400, rate_qps=4000.0)
    want = [OC.evaluate(o, q) for q in qs]
    e = mp.Engine(h, policy=policy, max_slots=32, hbm_budget_bytes=1 << 30)
    try:
        mp.mp_serve_start(e.ctx)
        tickets = []
        start = time.perf_counter()
        for q, at in zip(qs, arrivals):
            d = start + at - time.perf_counter()
            if d > 0:
                time.sleep(d)
            rc, t = e.submit(q)
            assert rc == mp.MP_OK
            tickets.append(t)
        for i, (t, w) in enumerate(zip(tickets, want)):
            assert mp.mp_wait(e.ctx, t) == mp.MP_OK
            assert_same(e.fetch(t), w, ("news serving", policy, i, "".join(qs[i]["types"])))
            e.release(t)
        assert mp.mp_serve_counters(e.ctx)["joined"] > 0
        mp.mp_serve_stop(e.ctx)
    finally:
        e.close()
