"""GPU: the serving loop (continuous batching). Queries submitted one by one with random
gaps join the product DAG while others are on the GPU; every result equals the CPU
oracle's bit for bit, and queries were admitted while others were in flight."""
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


@pytest.mark.parametrize("policy", [0, 3])
def test_stream_results_match_oracle(c1, cuda_ok, policy):
    from paper_2201_04058_b300 import mp
    h, o = c1
    qs = gen.batched_queries(seed=7, n=120, pool=25)
    want = [OC.evaluate(o, q) for q in qs]
    e = mp.Engine(h, policy=policy, max_slots=16, cache_bytes=8 << 20)
    try:
        mp.mp_serve_start(e.ctx)
        rng = np.random.default_rng(0)
        tickets = []
        for q in qs:
            rc, t = e.submit(q)
            assert rc == mp.MP_OK
            tickets.append(t)
            time.sleep(float(rng.exponential(0.0003)))
        for q, t, w in zip(qs, tickets, want):
            assert mp.mp_wait(e.ctx, t) == mp.MP_OK
            assert_same(e.fetch(t), w, "".join(q["types"]))
            assert mp.mp_result_latency(e.ctx, t) > 0
            mp.mp_release(e.ctx, t)
        st = mp.mp_serve_stats(e.ctx)
        assert st["queries"] == len(qs) and st["queued"] == 0
        assert st["batches"] < len(qs)  # some admission groups held several queries
        ct = mp.mp_serve_counters(e.ctx)
        assert ct["joined"] > 0  # queries joined work already on the GPU
        assert 1 < ct["max_inflight"] <= 16
        mp.mp_serve_stop(e.ctx)
        # after stopping, submission runs synchronously again
        assert_same(e.run(qs[0]), want[0], "after stop")
        # only cache entries stay charged to the budget once every result is released
        held = mp.mp_budget_stats(e.ctx)["held"]
        assert held == (mp.mp_cache_stats(e.ctx)["bytes"] if policy == 0 else 0)
    finally:
        e.close()


def test_stream_in_one_burst_overlaps(c1, cuda_ok):
    """A burst larger than the slots: later queries are admitted as earlier ones finish,
    beside the products of those still in flight; results exact, slots never exceeded."""
    from paper_2201_04058_b300 import mp
    h, o = c1
    qs = gen.long_queries(9, 24) + gen.batched_queries(seed=8, n=40, pool=30, anchor_p=0.5)
    e = mp.Engine(h, policy=mp.MP_POLICY_NONE, max_slots=6)
    try:
        mp.mp_serve_start(e.ctx)
        rc, ts = e.submit_batch(qs)
        assert rc == mp.MP_OK
        for q, t in zip(qs, ts):
            assert mp.mp_wait(e.ctx, t) == mp.MP_OK
            assert_same(e.fetch(t), OC.evaluate(o, q), "".join(q["types"]))
            e.release(t)
        ct = mp.mp_serve_counters(e.ctx)
        assert ct["max_inflight"] <= 6
        assert ct["joined"] > 0
        assert mp.mp_budget_stats(e.ctx)["held"] == 0
    finally:
        e.close()


def test_pending_ticket_is_not_readable(cuda_ok):
    from paper_2201_04058_b300 import mp
    h = gen.config1_hin()
    e = mp.Engine(h, policy=mp.MP_POLICY_NONE)
    try:
        mp.mp_serve_start(e.ctx)
        rc, ts = e.submit_batch(gen.long_queries(5, 8))
        assert rc == mp.MP_OK
        for t in ts:
            st = mp.mp_wait(e.ctx, t, 0)
            assert st in (mp.MP_OK, mp.MP_ERR_TIMEOUT)
        for t in ts:
            assert mp.mp_wait(e.ctx, t) == mp.MP_OK
            mp.mp_release(e.ctx, t)
    finally:
        e.close()
