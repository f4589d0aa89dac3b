"""GPU: the C-ABI boundary's memory contract. Device memory can come from the caller's
allocator (PyTorch's caching allocator through mp_config.alloc / .free) with results
bit for bit the oracle's and every buffer given back; the HBM byte budget is enforced
exactly: a product that cannot fit fails its query with MP_ERR_BUDGET, the cache yields
its entries to make room, and the bytes charged return to zero when results go."""
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


def test_torch_allocator_results_and_release(c1, cuda_ok):
    import torch
    mp = _mp()
    alloc = mp.TorchAllocator(0)
    stream = torch.cuda.Stream()
    e = mp.Engine(c1[0], allocator=alloc, cuda_stream=stream.cuda_stream, policy=mp.MP_POLICY_ATRAPOS)
    try:
        assert alloc.calls > 0 and alloc.live  # the HIN itself lives in torch's pool
        qs = [gen.config1_query()] + gen.random_queries(c1[0], 31, 12, lengths=(2, 7), p_cons=0.4)
        qs += gen.long_queries(5, 4)
        for rnd in range(2):  # the second round meets cache entries held in torch memory
            for q in qs:
                assert_same(e.run(q), OC.evaluate(c1[1], q), ("torch pool", rnd, "".join(q["types"])))
        rc, res = e.run_batch(qs)
        assert rc == 0
        for q, g in zip(qs, res):
            assert_same(g, OC.evaluate(c1[1], q), ("torch pool batch", "".join(q["types"])))
        # device copies into torch tensors through the same pool
        rc, t = e.submit(qs[0])
        rows, cols, nnz = mp.mp_result_info(e.ctx, t)
        d_rp = torch.empty(rows + 1, dtype=torch.int64, device="cuda:0")
        d_ci = torch.empty(nnz, dtype=torch.int32, device="cuda:0")
        d_val = torch.empty(nnz, dtype=torch.int64, device="cuda:0")
        mp.mp_result_copy(e.ctx, t, d_rp.data_ptr(), d_ci.data_ptr(), d_val.data_ptr(), on_device=True)
        torch.cuda.synchronize()
        want = OC.evaluate(c1[1], qs[0])
        assert np.array_equal(d_rp.cpu().numpy(), want[0])
        assert np.array_equal(d_ci.cpu().numpy(), want[1])
        assert np.array_equal(d_val.cpu().numpy().view(np.uint64), want[2])
        e.release(t)
    finally:
        e.close()
    assert not alloc.live, f"{len(alloc.live)} buffers not given back"


def test_budget_rejects_what_cannot_fit(c1, cuda_ok):
    """APTPA on the 2,000-paper HIN has a ~5 MB result: with a 1 MB budget and no cache
    it fails with MP_ERR_BUDGET, while a query with a small result still runs exactly."""
    mp = _mp()
    e = mp.Engine(c1[0], policy=mp.MP_POLICY_NONE, hbm_budget_bytes=1 << 20)
    try:
        rc, t = e.submit(gen.config1_query())
        assert rc == mp.MP_ERR_BUDGET
        assert mp.mp_wait(e.ctx, t) == mp.MP_ERR_BUDGET
        e.release(t)
        small = {"types": list("APA"), "constraints": [{"pos": 0, "prop": None, "op": "eq", "lo": 7}]}
        assert_same(e.run(small), OC.evaluate(c1[1], small), "small query under a small budget")
        assert mp.mp_budget_stats(e.ctx)["held"] == 0  # nothing charged once results are released
        # results held by tickets count: hold small results until the next one cannot fit
        held = []
        status = mp.MP_OK
        for a in range(0, 1500, 7):
            q = {"types": list("APTPA"), "constraints": [{"pos": 0, "prop": None, "op": "in",
                                                          "set": np.arange(a, a + 7, dtype=np.uint32)}]}
            rc, t = e.submit(q)
            held.append(t)
            if rc:
                status = rc
                break
        assert status == mp.MP_ERR_BUDGET
        assert mp.mp_budget_stats(e.ctx)["held"] <= 1 << 20
        for t in held:
            e.release(t)
        assert mp.mp_budget_stats(e.ctx)["held"] == 0
    finally:
        e.close()


def test_cache_yields_to_work(c1, cuda_ok):
    """A cache that fills the whole budget gives its entries up when a query needs the
    bytes: every query runs exactly, evictions are counted, and the budget is never passed.
    (The stress workload's intermediates total about 590 MB, the largest about 46 MB, so
    a 160 MB budget holds any one query's work but not every intermediate.)"""
    mp = _mp()
    budget = 160 << 20
    e = mp.Engine(c1[0], policy=mp.MP_POLICY_ATRAPOS, hbm_budget_bytes=budget, insertion=mp.MP_INSERT_ALL)
    try:
        qs = gen.long_queries(5, 32)
        for q in qs:
            assert_same(e.run(q), OC.evaluate(c1[1], q), "".join(q["types"]))
        st = mp.mp_cache_stats(e.ctx)
        assert st["evictions"] > 0 and st["bytes"] <= budget
        b = mp.mp_budget_stats(e.ctx)
        assert b["peak"] <= budget and b["held"] == st["bytes"]
    finally:
        e.close()
    # a budget twice one query's own working set: once cached results leave less room
    # than the next query needs, the cache must give some of them up
    q2 = gen.config1_query()
    probe = mp.Engine(c1[0], policy=mp.MP_POLICY_NONE, hbm_budget_bytes=0)
    try:
        probe.run(q2)
        need = mp.mp_budget_stats(probe.ctx)["peak"]
    finally:
        probe.close()
    budget = 2 * need
    e = mp.Engine(c1[0], policy=mp.MP_POLICY_ATRAPOS, hbm_budget_bytes=budget)
    try:
        for k in range(40):  # fill the cache with other APTPA results (year windows)
            lo = 1980 + k
            qk = {"types": list("APTPA"), "constraints": gen._year_on_every(list("APTPA"), "P", lo, lo + 12)}
            assert_same(e.run(qk), OC.evaluate(c1[1], qk), ("fill", k))
            if mp.mp_cache_stats(e.ctx)["bytes"] > budget - need:
                break
        assert mp.mp_cache_stats(e.ctx)["bytes"] > budget - need  # less room left than q2 needs
        before = mp.mp_cache_stats(e.ctx)["evictions"]
        assert_same(e.run(q2), OC.evaluate(c1[1], q2), "the cache yields")
        assert mp.mp_cache_stats(e.ctx)["evictions"] > before
        assert mp.mp_budget_stats(e.ctx)["peak"] <= budget
    finally:
        e.close()
