"""GPU parity: the engine's results, through the C ABI, equal the CPU oracle's bit for bit
(canonical CSR with exact uint64 counts) on seeded synthetic HINs, for every row-bin
class forced in turn, both planners, constraints of every kind, and the degenerate
cases (length-2 metapaths, masks that empty everything, overflow)."""
import numpy as np
import pytest

import gen
from oracle import chain as OC
from oracle.hin import OracleHIN

pytestmark = pytest.mark.gpu

BIN_CLASSES = [-1, 0, 1, 2, 3]  # auto, warp hash, block hash, dense smem, global scratch


def _mp():
    from paper_2201_04058_b300 import mp
    return mp


def assert_same(got, want, what=""):
    for name, g, w in zip(("row_ptr", "col", "val"), got, want):
        assert g.dtype == w.dtype, (what, name)
        assert g.shape == w.shape, (what, name, g.shape, w.shape)
        if not np.array_equal(g, w):
            bad = np.nonzero(g != w)[0][:5]
            raise AssertionError(f"{what}: {name} differs at {bad}: {g[bad]} vs {w[bad]}")


@pytest.fixture(scope="module")
def c1():
    h = gen.config1_hin()
    return h, OracleHIN(h)


@pytest.fixture(scope="module")
def c1_engines(c1, cuda_ok):
    mp = _mp()
    engines = {b: mp.Engine(c1[0], force_bin_class=b, policy=mp.MP_POLICY_NONE) for b in BIN_CLASSES}
    yield engines
    for e in engines.values():
        e.close()


@pytest.mark.parametrize("force", BIN_CLASSES)
def test_aptpa_2000_papers(c1, c1_engines, force):
    want = OC.evaluate(c1[1], gen.config1_query())
    assert_same(c1_engines[force].run(gen.config1_query()), want, f"APTPA bin {force}")


@pytest.mark.parametrize("force", BIN_CLASSES)
def test_random_constrained_queries(c1, c1_engines, force):
    qs = gen.random_queries(c1[0], 100 + max(force, 0), 25, lengths=(2, 7), p_cons=0.4)
    for q in qs:
        assert_same(c1_engines[force].run(q), OC.evaluate(c1[1], q), q["types"])


def test_forced_bins_are_used(c1, c1_engines):
    mp = _mp()
    q = gen.config1_query()
    # a forced class takes every row that fits it; larger rows go to the next class up
    # (the one-thread-per-row class, 11, only takes rows under automatic binning)
    allowed = {0: set(range(0, 11)), 1: set(range(6, 11)), 2: {9, 10}, 3: {10}}
    must = {0: set(range(0, 6)), 1: set(range(6, 9)), 2: {9}, 3: {10}}
    for force in allowed:
        e = c1_engines[force]
        rc, t = e.submit(q)
        assert rc == 0
        st = mp.mp_result_stats(e.ctx, t)
        e.release(t)
        for passname in ("sym_bins", "num_bins"):
            used = set(np.nonzero(st[passname])[0].tolist())
            assert used and used <= allowed[force], (force, passname, used)
            assert used & must[force], (force, passname, used)
        assert st["n_products"] >= 1 and st["products"] > 0


@pytest.mark.parametrize("seed", range(8))
def test_tiny_hins_every_bin(seed, cuda_ok):
    mp = _mp()
    h = gen.tiny_hin(seed, max_nodes=10)
    o = OracleHIN(h)
    qs = gen.random_queries(h, seed, 20, lengths=(2, 7), p_cons=0.5)
    for force in BIN_CLASSES:
        e = mp.Engine(h, force_bin_class=force, policy=mp.MP_POLICY_NONE)
        try:
            for q in qs:
                assert_same(e.run(q), OC.evaluate(o, q), (force, q["types"]))
        finally:
            e.close()


def test_planners_agree(c1, cuda_ok):
    mp = _mp()
    qs = gen.random_queries(c1[0], 7, 15, lengths=(4, 7), p_cons=0.3)
    e_dp = mp.Engine(c1[0], planner=mp.MP_PLAN_DP, policy=mp.MP_POLICY_NONE)
    e_lr = mp.Engine(c1[0], planner=mp.MP_PLAN_LEFT_TO_RIGHT, policy=mp.MP_POLICY_NONE)
    e_sp = mp.Engine(c1[0], planner=mp.MP_PLAN_DP_SAMPLED, policy=mp.MP_POLICY_NONE, sample_rows=64)
    try:
        for q in qs:
            want = OC.evaluate(c1[1], q)
            assert_same(e_dp.run(q), want, "dp")
            assert_same(e_lr.run(q), want, "left-to-right")
            assert_same(e_sp.run(q), want, "dp, sampled densities")
        rc, got = e_sp.run_batch(qs)
        assert rc == 0
        for q, g in zip(qs, got):
            assert_same(g, OC.evaluate(c1[1], q), "sampled, batch")
    finally:
        e_dp.close()
        e_lr.close()
        e_sp.close()


def test_long_metapaths_through_hubs(c1, c1_engines):
    for q in gen.long_queries(5, 6):
        assert_same(c1_engines[-1].run(q), OC.evaluate(c1[1], q), "".join(q["types"]))


def test_empty_results_and_length_two(c1, c1_engines):
    e = c1_engines[-1]
    qs = [
        {"types": list("APTPA"), "constraints": [{"pos": 2, "prop": None, "op": "in", "set": np.zeros(0, np.uint32)}]},
        {"types": list("APA"), "constraints": [{"pos": 1, "prop": "year", "op": "range", "lo": 3000, "hi": 4000}]},
        {"types": ["P", "A"], "constraints": [{"pos": 0, "prop": "year", "op": "range", "lo": 2000, "hi": 2010}]},
        {"types": ["A", "P"], "constraints": []},
        {"types": ["T", "P"], "constraints": [{"pos": 1, "prop": "year", "op": "in", "set": np.array([1990, 2001, 2020], np.uint32)}]},
    ]
    for q in qs:
        assert_same(e.run(q), OC.evaluate(c1[1], q), q["types"])


def test_unknown_relation_rejected(c1, c1_engines):
    mp = _mp()
    e = c1_engines[-1]
    with pytest.raises(mp.MPError) as ex:
        e.submit({"types": ["A", "V"], "constraints": []})
    assert ex.value.code == mp.MP_ERR_NOTFOUND


@pytest.mark.parametrize("tuning", ["", "glob_dense=0", "glob_dense=0,combine=0", "combine=0"])
def test_overflow_is_an_error_not_a_wrap(cuda_ok, tuning, monkeypatch):
    """A complete bipartite 100 x 100 relation: a metapath ABAB... of length n has
    100^(n-2) instances between every pair of end nodes; at n = 12 that is 10^20 > 2^64,
    so the count cannot be represented, while n = 11 (10^18) fits. Split rows run as
    dense rows (default) and as bitmap rows (glob_dense=0), with and without the
    shared-memory combining table; the last product of n = 12 is the one whose bound
    forces carry-checked additions."""
    mp = _mp()
    if tuning:
        monkeypatch.setenv("MP_TUNING", tuning)
    n = 100
    s = np.repeat(np.arange(n, dtype=np.uint32), n)
    d = np.tile(np.arange(n, dtype=np.uint32), n)
    h = {"types": {"A": n, "B": n}, "relations": [("A", "B", s, d)], "props": {}}
    q = {"types": list("ABABABABABAB"), "constraints": []}
    with pytest.raises(OC.OracleOverflow):
        OC.evaluate(OracleHIN(h), q)
    for force in (-1, 0, 1, 3):
        e = mp.Engine(h, force_bin_class=force, policy=mp.MP_POLICY_NONE)
        try:
            rc, t = e.submit(q)
            assert rc == mp.MP_ERR_OVERFLOW, force
            e.release(t)
            # one step shorter fits: 100^9 < 2^64
            q11 = {"types": list("ABABABABABA"), "constraints": []}
            rp, ci, val = e.run(q11)
            assert np.all(val == np.uint64(100 ** 9)) and rp[-1] == n * n
        finally:
            e.close()


@pytest.fixture(scope="module")
def c2_small(cuda_ok):
    h = gen.config2_hin(scale=0.01)
    return h, OracleHIN(h)


def test_scaled_scholarly_workload_sampled_planner(c2_small):
    mp = _mp()
    h, o = c2_small
    e = mp.Engine(h, planner=mp.MP_PLAN_DP_SAMPLED, policy=mp.MP_POLICY_NONE)
    try:
        for q in gen.config2_queries(h, seed=2, n_anchor_a=32, n_anchor_t=4):
            assert_same(e.run(q), OC.evaluate(o, q), ("sampled", "".join(q["types"])))
    finally:
        e.close()


@pytest.mark.parametrize("force", BIN_CLASSES)
def test_scaled_scholarly_workload(c2_small, force):
    """The twenty constrained queries of the scholarly workload on a 1 % HIN (50 k papers,
    40 k authors): output widths beyond the dense shared-memory limit, hub rows in the
    block-hash and global bins."""
    mp = _mp()
    h, o = c2_small
    e = mp.Engine(h, force_bin_class=force, policy=mp.MP_POLICY_NONE)
    try:
        for q in gen.config2_queries(h, seed=2, n_anchor_a=32, n_anchor_t=4):
            assert_same(e.run(q), OC.evaluate(o, q), (force, "".join(q["types"])))
    finally:
        e.close()


def test_copy_to_device_buffers(c1, c1_engines):
    import torch
    mp = _mp()
    e = c1_engines[-1]
    rc, t = e.submit(gen.config1_query())
    assert rc == 0
    rows, cols, nnz = mp.mp_result_info(e.ctx, t)
    rp = torch.empty(rows + 1, dtype=torch.int64, device="cuda")
    ci = torch.empty(nnz, dtype=torch.int32, device="cuda")
    val = torch.empty(nnz, dtype=torch.int64, device="cuda")
    mp.mp_result_copy(e.ctx, t, rp.data_ptr(), ci.data_ptr(), val.data_ptr(), on_device=True)
    e.release(t)
    want = OC.evaluate(c1[1], gen.config1_query())
    np.testing.assert_array_equal(rp.cpu().numpy(), want[0])
    np.testing.assert_array_equal(ci.cpu().numpy(), want[1])
    np.testing.assert_array_equal(val.cpu().numpy().view(np.uint64), want[2])


@pytest.mark.parametrize("lbs,combine,short_walk", [(1, 0, 0), (1, 1, 0), (0, 0, 0), (0, 0, 1), (0, 1, 0), (0, 1, 1)])
def test_split_row_kernel_variants(c1, c2_small, lbs, combine, short_walk, monkeypatch):
    """The split-row (GLOBAL) kernel's variants -- warp-level or block-staged product walk,
    shared-memory combining of hot outputs on or off, one-thread-per-entry walk of short Y
    rows on or off (staged walk) -- give identical results."""
    mp = _mp()
    monkeypatch.setenv("MP_TUNING", f"lbs={lbs},combine={combine},short_walk={short_walk}")
    for (h, o), qs in ((c1, gen.long_queries(5, 6) + [gen.config1_query()]),
                       (c2_small, gen.config2_queries(c2_small[0], seed=2, n_anchor_a=32, n_anchor_t=4))):
        e = mp.Engine(h, force_bin_class=mp.MP_BIN_GLOBAL, policy=mp.MP_POLICY_NONE)
        try:
            for q in qs:
                assert_same(e.run(q), OC.evaluate(o, q), (combine, short_walk, "".join(q["types"])))
        finally:
            e.close()


@pytest.mark.parametrize("combine,glob_dense,dense_scratch,occ", [
    (1, 0, 0, 4),            # dense rows off: every split row takes bitmap rounds
    (1, 1e-9, 0, 4),         # every split row takes a dense row
    (0, 1e-9, 0, 4),         # ... without the shared-memory combining table
    (1, 1e-9, 200000, 4),    # the dense scratch holds a few rows; the rest take bitmap rounds
    (1, 1e-9, 1, 4),         # no dense row fits: rows qualify, all take bitmap rounds
    (1, 0.5, 0, 4),          # half the default threshold
    (1, 1.0, 0, 4),          # the default threshold
    (1, 1e-9, 200000, 6),    # 6 resident blocks per SM (40 registers) for the adding kernels
    (0, 0, 0, 6),
])
@pytest.mark.parametrize("seg_walk", [0, 1])
def test_split_row_dense_rows(c1, c2_small, combine, glob_dense, dense_scratch, occ, seg_walk, monkeypatch):
    """Split rows that accumulate in a dense u64 row (one pass for size and values, a fill
    afterwards) give the oracle's results, alone and mixed with bitmap rows when the dense
    scratch runs out, one query at a time and as one batch. (The overflow test above runs
    its forced split rows through dense rows under the default threshold.)"""
    mp = _mp()
    tune = f"combine={combine},glob_dense={glob_dense},glob_occ={occ},lbs_occ={occ},seg_walk={seg_walk}"
    if dense_scratch:
        tune += f",dense_scratch={dense_scratch}"
    monkeypatch.setenv("MP_TUNING", tune)
    for (h, o), qs in ((c1, gen.long_queries(5, 6) + [gen.config1_query()]),
                       (c2_small, gen.config2_queries(c2_small[0], seed=2, n_anchor_a=32, n_anchor_t=4))):
        e = mp.Engine(h, force_bin_class=mp.MP_BIN_GLOBAL, policy=mp.MP_POLICY_NONE)
        try:
            for q in qs:
                assert_same(e.run(q), OC.evaluate(o, q), (tune, "".join(q["types"])))
            rc, res = e.run_batch(qs)
            assert rc == 0
            for q, g in zip(qs, res):
                assert_same(g, OC.evaluate(o, q), (tune, "batch", "".join(q["types"])))
        finally:
            e.close()


def test_async_copy_overlaps_next_query(c1, c1_engines):
    """Results copied with mp_result_copy_async while the next queries run equal the
    oracle's once mp_result_copy_wait returns; a ticket released right after its copy was
    queued does not disturb the copy (its memory is freed after the copy)."""
    mp = _mp()
    e = c1_engines[-1]
    qs = gen.long_queries(5, 3) + [gen.config1_query()]
    bufs, tks = [], []
    for q in qs:
        rc, t = e.submit(q)
        assert rc == 0
        rows, cols, nnz = mp.mp_result_info(e.ctx, t)
        b = (np.empty(rows + 1, np.int64), np.empty(nnz, np.int32), np.empty(nnz, np.uint64))
        mp.mp_result_copy_async(e.ctx, t, *b)
        bufs.append(b)
        tks.append(t)
    for q, t, b in zip(qs, tks, bufs):
        mp.mp_result_copy_wait(e.ctx, t)
        mp.mp_release(e.ctx, t)
        assert_same(b, OC.evaluate(c1[1], q), ("async", "".join(q["types"])))
    rc, t = e.submit(qs[0])
    rows, cols, nnz = mp.mp_result_info(e.ctx, t)
    b = (np.empty(rows + 1, np.int64), np.empty(nnz, np.int32), np.empty(nnz, np.uint64))
    mp.mp_result_copy_async(e.ctx, t, *b)
    mp.mp_release(e.ctx, t)
    rc2, t2 = e.submit(qs[1])  # reuses freed memory only after the copy above
    e.release(t2)
    import torch
    torch.cuda.synchronize()
    assert_same(b, OC.evaluate(c1[1], qs[0]), "released early")


@pytest.mark.parametrize("graphs", [0, 1])
def test_bin_passes_as_graphs(c1, graphs, monkeypatch):
    """The shared-memory bin passes replayed as CUDA graphs (one per wave shape, captured on
    the first wave of that shape) and launched directly give the oracle's results, for every
    forced bin class and for batches whose waves have many shapes, run twice so the second
    run replays every graph."""
    mp = _mp()
    monkeypatch.setenv("MP_TUNING", f"graphs={graphs}")
    h, o = c1
    qs = gen.random_queries(h, 31, 12, lengths=(3, 7)) + gen.long_queries(5, 3)
    want = [OC.evaluate(o, q) for q in qs]
    for force in BIN_CLASSES:
        e = mp.Engine(h, force_bin_class=force, policy=mp.MP_POLICY_NONE)
        try:
            for rnd in range(2):
                for q, w in zip(qs, want):
                    assert_same(e.run(q), w, (graphs, force, rnd, "".join(q["types"])))
                rc, res = e.run_batch(qs)
                assert rc == 0
                for q, g, w in zip(qs, res, want):
                    assert_same(g, w, (graphs, force, rnd, "batch", "".join(q["types"])))
            st = mp.mp_graph_stats(e.ctx)
            if graphs and force != mp.MP_BIN_GLOBAL:
                assert st["captures"] > 0 and st["replays"] > st["captures"], (force, st)
            elif not graphs:
                assert st == {"captures": 0, "replays": 0}, (force, st)
            # every row forced into the split-row bin leaves no shared-memory pass to capture
        finally:
            e.close()


@pytest.mark.parametrize("graphs", [0, 1])
def test_pooled_bin_pass(c1, graphs, monkeypatch):
    """The warp-hash and 2048-slot bins drained by one persistent launch per pass (a device
    work queue, largest tables first), directly and replayed as graphs, give the oracle's
    results for every forced bin class, alone and in batches, run twice."""
    mp = _mp()
    monkeypatch.setenv("MP_TUNING", f"pool=1,graphs={graphs}")
    h, o = c1
    qs = gen.random_queries(h, 41, 14, lengths=(2, 7)) + gen.long_queries(5, 3) + [gen.config1_query()]
    want = [OC.evaluate(o, q) for q in qs]
    for force in BIN_CLASSES:
        e = mp.Engine(h, force_bin_class=force, policy=mp.MP_POLICY_NONE)
        try:
            for rnd in range(2):
                for q, w in zip(qs, want):
                    assert_same(e.run(q), w, ("pool", graphs, force, rnd, "".join(q["types"])))
                rc, res = e.run_batch(qs)
                assert rc == 0
                for q, g, w in zip(qs, res, want):
                    assert_same(g, w, ("pool", graphs, force, rnd, "batch", "".join(q["types"])))
            names = set(mp.mp_kernel_stats(e.ctx)[0])
            if force in (-1, 0, 1):
                assert "sym_pool" in names and "num_pool" in names, names
        finally:
            e.close()


@pytest.mark.parametrize("glob_dense", [0, 1e-9])
def test_walk_kernel_stats(c1, glob_dense, monkeypatch):
    """The split-row walk kernels have counters of their own inside the split-row pass:
    their Gustavson products add up to the pass's (bitmap rows plus dense rows), their
    device time is part of the pass's, and their byte counts are positive."""
    mp = _mp()
    monkeypatch.setenv("MP_TUNING", f"glob_dense={glob_dense}")
    h, o = c1
    qs = gen.long_queries(5, 6) + [gen.config1_query()]
    e = mp.Engine(h, force_bin_class=mp.MP_BIN_GLOBAL, policy=mp.MP_POLICY_NONE)
    try:
        mp.mp_kernel_stats_reset(e.ctx)
        for q in qs:
            assert_same(e.run(q), OC.evaluate(o, q), ("walk stats", "".join(q["types"])))
        ks, _ = mp.mp_kernel_stats(e.ctx)
        walks = ["walk_dense"] if glob_dense else ["walk_sym", "walk_num"]
        for w in walks:
            assert w in ks and ks[w]["launches"] > 0 and ks[w]["bytes"] > 0, (w, ks.get(w))
        sym_walk = sum(ks[w]["products"] for w in ("walk_sym", "walk_dense") if w in ks)
        assert sym_walk == ks["sym_global"]["products"]
        assert sum(ks[w]["ms"] for w in ("walk_sym", "walk_dense") if w in ks) <= ks["sym_global"]["ms"]
        if not glob_dense:
            assert ks["walk_num"]["products"] == ks["num_global"]["products"]
            assert ks["walk_num"]["ms"] <= ks["num_global"]["ms"]
    finally:
        e.close()


@pytest.mark.parametrize("dsm_cols", [0, 24, 1 << 13])
@pytest.mark.parametrize("glob_dense", [1e-9, 1.0])
def test_dense_rows_in_shared_memory(c1, c2_small, dsm_cols, glob_dense, monkeypatch):
    """Dense split rows whose output is narrow enough add their counts in a shared-memory
    row per block and flush it to the dense row on every row change (dsm_cols = 8192, the
    default); with the variant off (0) or narrower than the outputs (24) they add straight
    into the global dense row. Same results as the oracle, alone and batched."""
    mp = _mp()
    tune = f"dsm_cols={dsm_cols},glob_dense={glob_dense}"
    monkeypatch.setenv("MP_TUNING", tune)
    for (h, o), qs in ((c1, gen.long_queries(5, 6) + [gen.config1_query()]),
                       (c2_small, gen.config2_queries(c2_small[0], seed=2, n_anchor_a=32, n_anchor_t=4))):
        e = mp.Engine(h, force_bin_class=mp.MP_BIN_GLOBAL, policy=mp.MP_POLICY_NONE)
        try:
            for q in qs:
                assert_same(e.run(q), OC.evaluate(o, q), (tune, "".join(q["types"])))
            rc, res = e.run_batch(qs)
            assert rc == 0
            for q, g in zip(qs, res):
                assert_same(g, OC.evaluate(o, q), (tune, "batch", "".join(q["types"])))
            ks, _ = mp.mp_kernel_stats(e.ctx)
            assert "walk_dense" in ks
        finally:
            e.close()


@pytest.mark.parametrize("graphs", [0, 1])
@pytest.mark.parametrize("lane_rows", [0, 1])
def test_lane_rows(c1, c2_small, graphs, lane_rows, monkeypatch):
    """Rows of at most 16 Gustavson products under automatic binning: one thread per row
    (merged by insertion into a sorted list) or, with the class off, the warp-hash bins;
    directly and replayed as graphs, alone and batched, the oracle's results. The class
    takes rows in both passes when on and none when off."""
    mp = _mp()
    monkeypatch.setenv("MP_TUNING", f"lane_rows={lane_rows},graphs={graphs}")
    for (h, o), qs in ((c1, gen.random_queries(c1[0], 43, 14, lengths=(2, 7), p_cons=0.4) + [gen.config1_query()]),
                       (c2_small, gen.config2_queries(c2_small[0], seed=2, n_anchor_a=32, n_anchor_t=4))):
        e = mp.Engine(h, policy=mp.MP_POLICY_NONE)
        try:
            lane = {"sym_bins": 0, "num_bins": 0}
            for rnd in range(2):
                for q in qs:
                    rc, t = e.submit(q)
                    assert rc == 0
                    st = mp.mp_result_stats(e.ctx, t)
                    for k in lane:
                        lane[k] += int(st[k][11])
                    assert_same(e.fetch(t), OC.evaluate(o, q), ("lane", lane_rows, graphs, rnd, "".join(q["types"])))
                    e.release(t)
                rc, res = e.run_batch(qs)
                assert rc == 0
                for q, g in zip(qs, res):
                    assert_same(g, OC.evaluate(o, q), ("lane batch", lane_rows, graphs, rnd, "".join(q["types"])))
            if lane_rows:
                assert lane["sym_bins"] > 0 and lane["num_bins"] > 0, lane
            else:
                assert lane == {"sym_bins": 0, "num_bins": 0}, lane
        finally:
            e.close()


@pytest.mark.parametrize("ew_max", [-1, 0, 4, 64, 1 << 20])
@pytest.mark.parametrize("glob_dense", [0, 1e-9, 1.0])
def test_split_rows_by_entries(c1, c2_small, ew_max, glob_dense, monkeypatch):
    """Split rows whose masked Y rows are all short (at most ew_max entries) are cut into
    work items of X entries, each entry's Y row looked up as it is walked; the others into
    items of products with per-entry offsets (ew_max = -1: every row). Bitmap rows, dense
    rows and a mix, alone and batched: the oracle's results."""
    mp = _mp()
    tune = f"ew_max={ew_max},glob_dense={glob_dense}"
    monkeypatch.setenv("MP_TUNING", tune)
    for (h, o), qs in ((c1, gen.long_queries(5, 6) + [gen.config1_query()] +
                        gen.random_queries(c1[0], 44, 8, lengths=(2, 6), p_cons=0.5)),
                       (c2_small, gen.config2_queries(c2_small[0], seed=2, n_anchor_a=32, n_anchor_t=4))):
        e = mp.Engine(h, force_bin_class=mp.MP_BIN_GLOBAL, policy=mp.MP_POLICY_NONE)
        try:
            for q in qs:
                assert_same(e.run(q), OC.evaluate(o, q), (tune, "".join(q["types"])))
            rc, res = e.run_batch(qs)
            assert rc == 0
            for q, g in zip(qs, res):
                assert_same(g, OC.evaluate(o, q), (tune, "batch", "".join(q["types"])))
        finally:
            e.close()


@pytest.mark.parametrize("row_lens", [0, 1])
def test_masked_row_lengths(c1, c2_small, row_lens, monkeypatch):
    """The row work reading precomputed masked Y-row lengths (products without a row mask
    whose X has at least as many entries as Y has rows) or the Y row pointers and the mask:
    same bins, same results as the oracle, with and without split rows."""
    mp = _mp()
    monkeypatch.setenv("MP_TUNING", f"row_lens={row_lens}")
    for (h, o), qs in ((c1, gen.long_queries(5, 6) + gen.random_queries(c1[0], 45, 10, lengths=(2, 6), p_cons=0.3)),
                       (c2_small, gen.config2_queries(c2_small[0], seed=2, n_anchor_a=32, n_anchor_t=4))):
        for force in (-1, mp.MP_BIN_GLOBAL):
            e = mp.Engine(h, force_bin_class=force, policy=mp.MP_POLICY_NONE)
            try:
                for q in qs:
                    assert_same(e.run(q), OC.evaluate(o, q), (row_lens, force, "".join(q["types"])))
            finally:
                e.close()


@pytest.mark.parametrize("compact", [0, 1])
@pytest.mark.parametrize("force", [-1, 3])
def test_masked_leaves_compacted(c1, c2_small, compact, force, monkeypatch):
    """Pattern leaves entering a product with the mask on their columns applied (X by the
    middle mask when X has no row mask, Y by the column mask; here every leaf qualifies),
    or with the masks applied entry by entry: the oracle's results, alone and batched."""
    mp = _mp()
    monkeypatch.setenv("MP_TUNING", f"compact={compact},compact_min=1")
    for (h, o), qs in ((c1, gen.long_queries(5, 6) + [gen.config1_query()] +
                        gen.random_queries(c1[0], 46, 12, lengths=(2, 7), p_cons=0.6)),
                       (c2_small, gen.config2_queries(c2_small[0], seed=2, n_anchor_a=32, n_anchor_t=4))):
        e = mp.Engine(h, force_bin_class=force, policy=mp.MP_POLICY_NONE)
        try:
            for q in qs:
                assert_same(e.run(q), OC.evaluate(o, q), (compact, force, "".join(q["types"])))
            rc, res = e.run_batch(qs)
            assert rc == 0
            for q, g in zip(qs, res):
                assert_same(g, OC.evaluate(o, q), (compact, force, "batch", "".join(q["types"])))
        finally:
            e.close()


@pytest.mark.parametrize("row_lists", [0, 1])
@pytest.mark.parametrize("force", [-1, 0, 1, 2, 3])
def test_row_lists(c1, c2_small, row_lists, force, monkeypatch):
    """Products whose left factor starts at a position constrained by a node-id set (or is
    the result of such a product) run over the listed rows only, the other rows' row
    pointers filled in afterwards; or over all rows. Every bin class, alone and batched,
    the oracle's results; the results of a list run feed later products."""
    mp = _mp()
    monkeypatch.setenv("MP_TUNING", f"row_lists={row_lists}")
    for (h, o), qs in ((c1, gen.batched_queries(seed=17, n=40, pool=30, anchor_p=0.9) + [gen.config1_query()]),
                       (c2_small, gen.config2_queries(c2_small[0], seed=2, n_anchor_a=32, n_anchor_t=4))):
        e = mp.Engine(h, force_bin_class=force, policy=mp.MP_POLICY_NONE)
        try:
            for q in qs:
                assert_same(e.run(q), OC.evaluate(o, q), (row_lists, force, "".join(q["types"])))
            rc, res = e.run_batch(qs)
            assert rc == 0
            for q, g in zip(qs, res):
                assert_same(g, OC.evaluate(o, q), (row_lists, force, "batch", "".join(q["types"])))
        finally:
            e.close()


@pytest.mark.parametrize("ech", [256, 1024, 8192])
def test_entry_split_item_sizes(c1, c2_small, ech, monkeypatch):
    """Rows cut by X entries into work items of several sizes (items of 256 entries put
    many items on every split row): the oracle's results."""
    mp = _mp()
    monkeypatch.setenv("MP_TUNING", f"ech={ech}")
    for (h, o), qs in ((c1, gen.long_queries(5, 6) + [gen.config1_query()]),
                       (c2_small, gen.config2_queries(c2_small[0], seed=2, n_anchor_a=32, n_anchor_t=4))):
        e = mp.Engine(h, force_bin_class=mp.MP_BIN_GLOBAL, policy=mp.MP_POLICY_NONE)
        try:
            for q in qs:
                assert_same(e.run(q), OC.evaluate(o, q), (ech, "".join(q["types"])))
        finally:
            e.close()
