"""GPU: failures are made on the host and must come back as clean error codes -- device
allocations that fail (an injected allocator failure after N allocations), a result
beyond the size guard, a query released while it waits in the serving queue -- and the
HIN checkpoint (save, load into a fresh context) gives the same results."""
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


@pytest.mark.parametrize("policy", [3, 0])
def test_injected_allocation_failures(c1, cuda_ok, monkeypatch, policy):
    from paper_2201_04058_b300 import mp
    h, o = c1
    qs = [gen.config1_query()] + gen.long_queries(5, 2) + gen.random_queries(h, 3, 3, lengths=(2, 6))
    want = [OC.evaluate(o, q) for q in qs]
    seen_fail = seen_ok = False
    for k in (0, 1, 2, 3, 5, 8, 13, 21, 34, 55, 89, 144, 233, 10 ** 9):
        monkeypatch.setenv("MP_TUNING", f"fail_alloc_after_finalize={k}")
        e = mp.Engine(h, policy=policy)
        try:
            for q, w in zip(qs, want):
                rc, t = e.submit(q)
                assert rc in (mp.MP_OK, mp.MP_ERR_NOMEM), (k, rc)
                if rc == mp.MP_OK:
                    assert_same(e.fetch(t), w, ("alloc budget", k))
                    seen_ok = True
                else:
                    with pytest.raises(mp.MPError):
                        mp.mp_result_info(e.ctx, t)
                    seen_fail = True
                e.release(t)
        finally:
            e.close()
    assert seen_fail and seen_ok


def test_size_guard(c1, cuda_ok):
    from paper_2201_04058_b300 import mp
    h, o = c1
    e = mp.Engine(h, policy=mp.MP_POLICY_NONE, max_result_bytes=100_000)
    try:
        rc, t = e.submit(gen.config1_query())  # 441,873 entries * 12 bytes >> 100 kB
        assert rc == mp.MP_ERR_TOO_LARGE
        e.release(t)
        small = {"types": list("APA"), "constraints": [{"pos": 0, "prop": None, "op": "eq", "lo": 3}]}
        assert_same(e.run(small), OC.evaluate(o, small), "small result under the guard")
    finally:
        e.close()


@pytest.mark.parametrize("guard", ["size", "budget"])
def test_refused_product_beside_others(c1, cuda_ok, guard):
    """A one-product query whose result is refused (PAP, 1.5 M entries: beyond a 100 kB size
    guard and a 1 MB HBM budget) runs in the first wave beside the first products of small
    anchored queries that share no sub-chain with it. Its rows are binned for the numeric
    pass before the sizes are known; refusing it must leave the others exact."""
    from paper_2201_04058_b300 import mp
    h, o = c1
    kw = {"max_result_bytes": 100_000} if guard == "size" else {"hbm_budget_bytes": 1 << 20}
    e = mp.Engine(h, policy=mp.MP_POLICY_NONE, **kw)
    try:
        rng = np.random.default_rng(11)
        qs = []
        for t, n in (("APTPA", 1), ("APTPA", 3), ("PAP", 0), ("APTPA", 2), ("APVPA", 4)):
            cons = []
            if n:
                anchors = np.sort(rng.choice(1500, size=n, replace=False)).astype(np.uint32)
                cons = [{"pos": 0, "prop": None, "op": "in", "set": anchors}]
            qs.append({"types": list(t), "constraints": cons})
        qs.append({"types": list("APVPA"), "constraints": [{"pos": 0, "prop": None, "op": "eq", "lo": 5}]})
        refused = mp.MP_ERR_TOO_LARGE if guard == "size" else mp.MP_ERR_BUDGET
        for rnd in range(2):
            rc, res = e.run_batch(qs)
            assert res[2] == refused, (rnd, res[2])
            for i, (q, r) in enumerate(zip(qs, res)):
                if i != 2:
                    assert not isinstance(r, int), (rnd, i, r)
                    assert_same(r, OC.evaluate(o, q), (guard, rnd, i))
    finally:
        e.close()


def test_release_while_queued(c1, cuda_ok):
    from paper_2201_04058_b300 import mp
    h, _ = c1
    e = mp.Engine(h, policy=mp.MP_POLICY_NONE, max_slots=4)
    try:
        mp.mp_serve_start(e.ctx)
        rc, ts = e.submit_batch(gen.long_queries(5, 40))
        assert rc == mp.MP_OK
        for t in ts[10:]:
            mp.mp_release(e.ctx, t)  # most are still waiting or running: dropped cleanly
        for t in ts[:10]:
            assert mp.mp_wait(e.ctx, t) == mp.MP_OK
            mp.mp_release(e.ctx, t)
        mp.mp_serve_stop(e.ctx)
        assert mp.mp_serve_stats(e.ctx)["queued"] == 0
    finally:
        e.close()


def test_hin_checkpoint_round_trip(c1, cuda_ok, tmp_path):
    from paper_2201_04058_b300 import mp
    h, o = c1
    path = str(tmp_path / "hin.bin")
    e = mp.Engine(h, policy=mp.MP_POLICY_NONE)
    try:
        mp.mp_hin_save(e.ctx, path)
    finally:
        e.close()
    ctx = mp.mp_create(mp.mp_config_default())
    try:
        mp.mp_hin_load(ctx, path)
        mp.mp_finalize_hin(ctx)
        t = {n: mp.mp_type_id(ctx, n) for n in h["types"]}
        year = mp.mp_property_id(ctx, t["P"], "year")
        for q in [gen.config1_query()] + gen.random_queries(h, 21, 6, lengths=(2, 6), p_cons=0.0):
            buf = mp.make_query([t[x] for x in q["types"]], None, [])
            rc, tk = mp.mp_submit(ctx, buf)
            assert rc == mp.MP_OK
            rows, cols, nnz = mp.mp_result_info(ctx, tk)
            rp = np.empty(rows + 1, np.int64)
            ci = np.empty(nnz, np.int32)
            val = np.empty(nnz, np.uint64)
            mp.mp_result_copy(ctx, tk, rp, ci, val)
            mp.mp_release(ctx, tk)
            assert_same((rp, ci, val), OC.evaluate(o, q), "loaded HIN")
        qy = mp.make_query([t["A"], t["P"], t["A"]], None, [(1, year, mp.MP_OP_RANGE, 2000, 2010, None)])
        rc, tk = mp.mp_submit(ctx, qy)
        assert rc == mp.MP_OK
        mp.mp_release(ctx, tk)
    finally:
        mp.mp_destroy(ctx)
    ctx = mp.mp_create(mp.mp_config_default())
    try:
        with pytest.raises(mp.MPError):
            mp.mp_hin_load(ctx, str(tmp_path / "missing.bin"))
    finally:
        mp.mp_destroy(ctx)
