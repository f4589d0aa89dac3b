"""GPU: the serving loop (continuous batching). Queries submitted one by one with random
gaps are served in rounds; each result equals the same query evaluated alone (bit for
bit), and rounds hold several queries."""
import time

import numpy as np
import pytest

import gen

from test_gpu_parity import assert_same

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("policy", [0, 3])
def test_stream_results_equal_alone(cuda_ok, policy):
    from paper_2201_04058_b300 import mp
    h = gen.config1_hin()
    qs = gen.batched_queries(seed=7, n=120, pool=25)
    alone = mp.Engine(h, policy=mp.MP_POLICY_NONE)
    try:
        want = [alone.run(q) for q in qs]
    finally:
        alone.close()
    e = mp.Engine(h, policy=policy, max_slots=16, hbm_budget_bytes=8 << 20)
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
        assert st["batches"] < len(qs)  # some rounds served several queries
        mp.mp_serve_stop(e.ctx)
        # after stopping, submission runs synchronously again
        assert_same(e.run(qs[0]), want[0], "after stop")
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
