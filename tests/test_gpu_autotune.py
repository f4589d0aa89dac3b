"""GPU: the autotuner picks bin thresholds and fits the Eq. 2 coefficients on a workload,
writes them to a file that a new context loads, and never changes a result."""
import json

import pytest

import gen
from oracle import chain as OC
from oracle.hin import OracleHIN

from test_gpu_parity import assert_same

pytestmark = pytest.mark.gpu


def test_autotune_persists_and_keeps_results(cuda_ok, tmp_path):
    from paper_2201_04058_b300 import mp
    h = gen.config1_hin()
    o = OracleHIN(h)
    qs = gen.batched_queries(seed=11, n=32, pool=12) + gen.long_queries(5, 4)
    want = [OC.evaluate(o, q) for q in qs]
    path = str(tmp_path / "tune.json")
    e = mp.Engine(h, policy=mp.MP_POLICY_ATRAPOS)
    try:
        best = mp.mp_autotune(e.ctx, [e.query(q) for q in qs], reps=1, out_path=path)
        assert best > 0
        for q, w in zip(qs, want):
            assert_same(e.run(q), w, "tuned")
    finally:
        e.close()
    d = json.load(open(path))
    # 9 threshold pairs, 4 kernel variants (one knob flipped at a time), and the re-timed
    # Eq. 2 fit when there is one
    assert len(d["candidates"]) in (13, 14)
    assert d["dense_min_u"] in (64, 256, 1024) and d["heavy"] in (16384, 65536, 262144)
    assert d["combine"] in (0, 1) and d["short_walk"] in (0, 1) and d["seg_walk"] in (0, 1)
    assert d["glob_occ"] in (4, 6)
    assert min(c["ms"] for c in d["candidates"]) == pytest.approx(d["best_ms"])
    assert d["alpha"] > 0 and d["beta"] > 0 and d["gamma"] > 0
    if not d["fitted"]:
        assert (d["alpha"], d["beta"], d["gamma"]) == (1.0, 1.0, 1.0)
    e2 = mp.Engine(h, policy=mp.MP_POLICY_NONE, tune_file=path)
    try:
        for q, w in zip(qs, want):
            assert_same(e2.run(q), w, "loaded")
    finally:
        e2.close()
    with pytest.raises(mp.MPError):
        mp.Engine(h, tune_file=str(tmp_path / "missing.json"))
