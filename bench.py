"""Benchmark of the metapath-query engine on one B300 (or N independent replicas).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl engine|reference]
                    [--workload scholarly|serving|batched|stress] [--scale S]
                    [--no-cpu-baseline] [--no-extra] [--serve-queries N]

Workload "scholarly" (the default and the headline): a seeded scholarly-shaped HIN with
5 M papers, 4 M authors, 5 k venues and 50 k topics (Zipf author/topic degrees, one venue
per paper, a uniform year per paper) and twenty constrained queries, four each of APA,
APVPA, APTPA, TPAPT and VPTPV with year in [2010, 2020] on every paper position; all but
APA are anchored on a seeded set of first-node entities. One step evaluates all twenty
queries, each planned by the Eq. 1 / Eq. 2 DP, through the engine's C ABI. The HIN stays
resident in HBM (ingestion is not query time, as in Sec. 4.1.4); L2 is flushed between
steps.

Prints one JSON line: queries/s (value), per-query latency p50/p99, the end-to-end rate
with results copied to pinned host memory, the batched form of the same step, the
dominant kernel's achieved bandwidth against the measured HBM peak, clocks sampled during
the timed region, the CPU oracle's rate on a bounded sample, and the number of kernel
launches. Unless --no-extra, the line also carries "configs": compact measurements of the
other workloads, each with its own clock record, dominant kernel and CPU oracle sample --
the 2,000-paper HIN's plain APTPA query, its batched workload (256 queries) and stress
workload (64 long metapaths, with cache replays), and the serving workload on the
10 M-article news HIN at four arrival rates relative to the plain path's saturation
(served with and without the cache, and the plain path, under the same arrivals).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "metapath queries/sec, p50/p99 latency; SpGEMM GB/s vs ~8 TB/s HBM"
UNIT = "queries/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="engine", choices=["engine", "reference"])
    ap.add_argument("--workload", default="scholarly", choices=["scholarly", "serving", "batched", "stress"])
    ap.add_argument("--pool", type=int, default=500, help="template pool of the batched workload")
    ap.add_argument("--anchor-p", type=float, default=0.75,
                    help="share of batched queries with a first-node entity of interest")
    ap.add_argument("--serve-queries", type=int, default=2000,
                    help="queries per arrival rate of the serving workload (a sample of its 100 k stream)")
    ap.add_argument("--no-extra", action="store_true",
                    help="the scholarly workload only (no summaries of the other configurations)")
    ap.add_argument("--serve-budget-gb", type=float, default=60.0)
    ap.add_argument("--scale", type=float, default=1.0)
    ap.add_argument("--planner", default="eac", choices=list(PLANNERS),
                    help="chain planner of the scholarly workload (Eq. 1 DP with E_ac, MNC sketches, "
                         "sampled rows, or left to right)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-queries", type=int, default=5)
    ap.add_argument("--kernel-probe", default=None, metavar="IDX",
                    help="comma list of scholarly query indices (or 'all'): run each once, plain form, on "
                         "a fresh engine and print the kernel counters of each (a small, fixed set of "
                         "launches for an ncu capture to compare with); no timing")
    return ap.parse_args()


# ---------------------------------------------------------------- distributed plumbing

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def dist_init(ws, backend):
    import torch.distributed as dist
    if ws > 1 and not dist.is_initialized():
        dist.init_process_group(backend)
    return dist


def reduce_max(x: float, ws: int, device=None) -> float:
    """Max of a float over ranks (identity at world size 1)."""
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------- workload

# planner name -> (mp_config.planner value, description)
PLANNERS = {"eac": (0, "Eq.1 DP, Eq.2 cost, E_ac"), "ltr": (1, "left to right"),
            "sampled": (2, "Eq.1 DP, Eq.2 cost, sampled-row densities"),
            "mnc": (3, "Eq.1 DP, Eq.2 cost, MNC count sketches")}

def workload(name, scale):
    import gen
    if name == "scholarly":
        hin = gen.config2_hin(seed=2, scale=scale)
        qs = gen.config2_queries(hin, seed=2)
        cfg = {"workload": "scholarly HIN, 20 constrained metapath queries (APA, APVPA, APTPA, TPAPT, VPTPV)",
               "papers": hin["types"]["P"], "authors": hin["types"]["A"], "venues": hin["types"]["V"],
               "topics": hin["types"]["T"], "queries_per_step": len(qs),
               "constraints": "year in [2010,2020] on every P; first-node id sets of 256 A / 16 T / 16 V",
               "planner": "Eq.1 DP, Eq.2 cost, E_ac", "cache": "off (plain one-query-at-a-time chain)",
               "l2": "flushed between steps (512 MB write)"}
        return hin, qs, cfg
    raise ValueError(name)


def query_bytes(q):
    """Host->device payload of one query: type ids, constraint records and id sets."""
    n = 4 * len(q["types"]) + 40 * len(q["constraints"])
    for c in q["constraints"]:
        if c.get("set") is not None:
            n += 4 * len(c["set"])
    return n


# ---------------------------------------------------------------- clocks

class Clocks:
    """nvidia-smi samples every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=5)

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- peaks / traffic

def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6400.0, "fallback"


def kernel_source_hash():
    """Hash of the split-row walk kernel's source (the k_glob_lbs template, from its template
    line to its closing brace, and the device helpers it uses): the committed DRAM traffic
    of that kernel holds only while this is unchanged."""
    csrc = os.path.join(ROOT, "paper_2201_04058_b300", "csrc")
    with open(os.path.join(csrc, "wave.cu")) as fh:
        src = fh.read()
    head = src.index("__global__ void __launch_bounds__(GNT, OCC) k_glob_lbs(")
    start = src.rindex("template <int MODE", 0, head)
    depth, i = 0, src.index("{", head)
    while True:
        depth += {"{": 1, "}": -1}.get(src[i], 0)
        i += 1
        if depth == 0:
            break
    h = hashlib.sha256(src[start:i].encode())
    with open(os.path.join(csrc, "common.cuh"), "rb") as fh:
        h.update(fh.read())
    return h.hexdigest()[:16]


def dominant_kernel(kstats):
    """The single kernel with the most device time. The "*_global" entries time a whole
    split-row pass (set-up, walk and rank kernels together) and the "stage_*" entries other
    groups of kernels, so they are reported but not chosen; the walk kernels inside the
    split-row passes are ("walk_sym", "walk_num", "walk_dense")."""
    single = {k: v for k, v in (kstats or {}).items()
              if not k.endswith("_global") and not k.startswith("stage_") and v["ms"] > 0}
    return max(single.items(), key=lambda kv: kv[1]["ms"]) if single else None


def ncu_traffic(kernel_name):
    """DRAM bytes per launch of the kernel from the committed ncu summary, or None when
    the summary is absent or the kernel source changed since it was taken."""
    p = os.path.join(ROOT, "profiles", "roofline_traffic.txt")
    try:
        with open(p) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    if d.get("source_hash") != kernel_source_hash():
        return None
    k = d.get("kernels", {}).get(kernel_name)
    return None if k is None else k.get("dram_bytes_per_launch")


# ---------------------------------------------------------------- CPU oracle leg

def cpu_oracle_rate(hin, qs, n_sample):
    """The CPU oracle as it stands (single-threaded C) on the first n_sample queries."""
    from oracle import chain as OC
    from oracle.hin import OracleHIN
    o = OracleHIN(hin)
    sample = qs[:n_sample]
    t0 = time.perf_counter()
    for q in sample:
        OC.evaluate(o, q)
    dt = time.perf_counter() - t0
    return {"value": len(sample) / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {len(sample)} of the {len(qs)} queries (one per template), single thread, "
                      f"{dt:.1f} s"}


def run_reference(args, ws, rank):
    """--impl reference: the oracle on the host cores, one query per step, cycling
    through the workload's queries."""
    if rank != 0:
        return
    hin, qs, cfg = workload(args.workload, args.scale)
    from oracle import chain as OC
    from oracle.hin import OracleHIN
    o = OracleHIN(hin)
    for i in range(args.warmup):
        OC.evaluate(o, qs[i % len(qs)])
    lat = []
    t0 = time.perf_counter()
    for i in range(args.steps):
        t = time.perf_counter()
        OC.evaluate(o, qs[(args.warmup + i) % len(qs)])
        lat.append(time.perf_counter() - t)
    dt = time.perf_counter() - t0
    v = args.steps / dt
    out = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "u64", "data": "synthetic", "config": dict(cfg, queries_per_step=1), "impl": "reference",
           "p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": "one query per step, cycling through the workload, single thread"},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------- engine leg

def run_engine(args, ws, rank, local):
    import torch
    from paper_2201_04058_b300 import mp

    torch.cuda.set_device(local)
    dist_init(ws, "nccl")
    dev = torch.device("cuda", local)
    hin, qs, cfg = workload(args.workload, args.scale)
    planner, cfg["planner"] = PLANNERS[args.planner]
    stream = torch.cuda.Stream(device=dev)
    eng = mp.Engine(hin, device=local, cuda_stream=stream.cuda_stream, policy=mp.MP_POLICY_NONE, planner=planner)
    bufs = [eng.query(q) for q in qs]
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    def step(copy_out=None):
        lat = []
        for b in bufs:
            rc, t = mp.mp_submit(eng.ctx, b)
            if rc != mp.MP_OK:
                raise mp.MPError(rc, "query")
            lat.append(mp.mp_result_time(eng.ctx, t))
            if copy_out is not None:
                copy_out(t)
            mp.mp_release(eng.ctx, t)
        return lat

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        # planning cost alone: every query of a step planned (sketches, sums, DP) without
        # running its products
        t0 = time.perf_counter()
        for b in bufs:
            mp.mp_plan_query(eng.ctx, b)
        plan_ms = 1e3 * (time.perf_counter() - t0) / len(bufs)

        # device-timed steps, L2 flushed between them
        mp.mp_kernel_stats_reset(eng.ctx)
        _, l0 = mp.mp_kernel_stats(eng.ctx)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        lat = []
        barrier(ws)
        torch.cuda.synchronize()
        with Clocks(local) as clk:
            for k in range(args.steps):
                flush.zero_()
                ev[k][0].record(stream)
                lat += step()
                ev[k][1].record(stream)
            torch.cuda.synchronize()
        barrier(ws)
        kstats, l1 = mp.mp_kernel_stats(eng.ctx)
        step_ms = [a.elapsed_time(b) for a, b in ev]
        total_s = reduce_max(sum(step_ms) / 1e3, ws, dev)

        # end to end: every result copied back to pinned host memory, asynchronously, so
        # query i's result travels while query i+1 runs; a step ends when all have landed
        d2h = [0]
        sizes = []
        for b in bufs:
            rc, t = mp.mp_submit(eng.ctx, b)
            rows, cols, nnz = mp.mp_result_info(eng.ctx, t)
            sizes.append((rows + 1) * 8 + nnz * 12)
            mp.mp_release(eng.ctx, t)
        offs = np.concatenate(([0], np.cumsum([(x + 255) // 256 * 256 for x in sizes])))
        pinned = torch.empty(int(offs[-1]), dtype=torch.uint8, pin_memory=True)

        def e2e_step():
            tks = []
            for i, b in enumerate(bufs):
                rc, t = mp.mp_submit(eng.ctx, b)
                if rc != mp.MP_OK:
                    raise mp.MPError(rc, "query")
                rows, cols, nnz = mp.mp_result_info(eng.ctx, t)
                base = pinned.data_ptr() + int(offs[i])
                mp.mp_result_copy_async(eng.ctx, t, base, base + (rows + 1) * 8, base + (rows + 1) * 8 + nnz * 4)
                d2h[0] += (rows + 1) * 8 + nnz * 12
                tks.append(t)
            for t in tks:
                mp.mp_result_copy_wait(eng.ctx, t)
                mp.mp_release(eng.ctx, t)

        e2e_steps = max(1, min(args.steps, 5))
        barrier(ws)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            flush.zero_()
            e2e_step()
        torch.cuda.synchronize()
        e2e_s = reduce_max(time.perf_counter() - t0, ws, dev)

        # batched form: the same queries as one workload per step (identical sub-chains run
        # once, every ready product of a plan level in one wave), cache off
        bev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        for _ in range(2):
            rc, tks = mp.mp_submit_batch(eng.ctx, bufs)
            for t in tks:
                mp.mp_release(eng.ctx, t)
        torch.cuda.synchronize()
        bprod = 0
        for k in range(args.steps):
            flush.zero_()
            bev[k][0].record(stream)
            rc, tks = mp.mp_submit_batch(eng.ctx, bufs)
            if rc != mp.MP_OK:
                raise mp.MPError(rc, "batch")
            for t in tks:
                bprod += mp.mp_result_stats(eng.ctx, t)["n_products"]
                mp.mp_release(eng.ctx, t)
            bev[k][1].record(stream)
        torch.cuda.synchronize()
        bstep_ms = [a.elapsed_time(b) for a, b in bev]
        btotal_s = reduce_max(sum(bstep_ms) / 1e3, ws, dev)

    n_q = len(qs)
    value = ws * n_q * args.steps / total_s
    # with all of a step's queries arriving together, a query's latency in the plain form
    # is the time until its own result (the queries before it run first); in the batched
    # form every query completes with the batch
    plain_arrival_lat = []
    for k in range(args.steps):
        acc = 0.0
        for x in lat[k * n_q:(k + 1) * n_q]:
            acc += x
            plain_arrival_lat.append(acc)
    batched = {"value": ws * n_q * args.steps / btotal_s, "unit": UNIT, "ms_per_step": 1e3 * btotal_s / args.steps,
               "speedup_vs_plain": total_s / btotal_s, "products_per_step": bprod / args.steps,
               "latency_p50_ms": float(np.percentile(bstep_ms, 50)), "latency_p99_ms": float(np.percentile(bstep_ms, 99)),
               "plain_latency_same_arrivals_p50_ms": float(np.percentile(plain_arrival_lat, 50)),
               "plain_latency_same_arrivals_p99_ms": float(np.percentile(plain_arrival_lat, 99)),
               "form": "mp_submit_batch of the step's queries: shared sub-chains once, one wave per plan level"}
    peak, peak_kind = measured_peak()
    dom = dominant_kernel(kstats)
    roofline = None
    if dom:
        name, k = dom
        ach = k["bytes"] / (k["ms"] / 1e3) / 1e9
        traffic = ncu_traffic(name)
        roofline = {"bound": "hbm", "kernel": name, "achieved": ach, "peak": peak, "unit": "GB/s",
                    "frac": ach / peak, "peak_source": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                    "traffic": traffic, "launches": k["launches"], "ms_per_launch": k["ms"] / k["launches"],
                    "algorithmic_bytes_per_launch": k["bytes"] / k["launches"],
                    "share_of_step": k["ms"] / sum(step_ms)}
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "u64", "data": "synthetic (seeded generator; no dataset)",
           "config": dict(cfg, parallelism=f"replicas x{ws}" if ws > 1 else "single GPU"),
           "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
           "plan_ms_per_query": plan_ms,
           "e2e": {"value": ws * n_q * e2e_steps / e2e_s, "unit": UNIT,
                   "h2d_bytes_per_step": sum(query_bytes(q) for q in qs),
                   "d2h_bytes_per_step": d2h[0] // e2e_steps},
           "batched": batched, "roofline": roofline, "clocks": clk.summary(), "gpu_launches": int(l1 - l0),
           "graphs": mp.mp_graph_stats(eng.ctx),
           "kernels": {k: {"launches": v["launches"], "ms": round(v["ms"], 3),
                           "GBps": round(v["bytes"] / max(v["ms"], 1e-9) / 1e6, 1),
                           "Gproducts_per_s": round(v["products"] / max(v["ms"], 1e-9) / 1e6, 2)}
                       for k, v in kstats.items()}}
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_oracle_rate(hin, qs, args.cpu_sample_queries)
    eng.close()
    if rank == 0 and not args.no_extra and args.scale == 1.0:
        # the other configurations, each with its own clocks, roofline and CPU oracle sample
        del hin
        out["configs"] = {
            "1_plain": leg_plain_config1(mp, local, peak, peak_kind),
            "3_batched": leg_small(mp, local, "batched", peak, peak_kind),
            "5_stress": leg_small(mp, local, "stress", peak, peak_kind),
            "4_serving": leg_serving(mp, local, peak, peak_kind, n=args.serve_queries),
        }
    if rank == 0:
        print(json.dumps(out), flush=True)


# ---------------------------------------------------------------- the other configurations
#
# Each leg below returns a compact summary (queries/s, p50/p99, a clock record sampled in
# its timed region, the dominant kernel's bandwidth and the CPU oracle on a bounded sample)
# that the default run folds into its JSON line under "configs"; --workload serving,
# batched or stress prints one leg's full line instead.

def _roofline(mp, ctx, peak, peak_kind, note):
    ks, _ = mp.mp_kernel_stats(ctx)
    dom = dominant_kernel(ks)
    if not dom:
        return None
    name, k = dom
    if k["ms"] <= 0:
        return None
    ach = k["bytes"] / (k["ms"] / 1e3) / 1e9
    return {"bound": "hbm", "kernel": name, "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "peak_source": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)", "traffic": None,
            "note": note}


def _pct(xs, q):
    return float(np.percentile(xs, q)) if len(xs) else None


def _oracle_sample(hin, qs, budget_s=6.0, max_q=None):
    """The CPU oracle as it stands on the first queries of a workload, until budget_s of
    host time is spent; returns (queries/s, the sample's description)."""
    from oracle import chain as OC
    from oracle.hin import OracleHIN
    o = OracleHIN(hin)
    n = 0
    t0 = time.perf_counter()
    for q in qs[:max_q or len(qs)]:
        OC.evaluate(o, q)
        n += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {n} of the {len(qs)} queries, single thread, {dt:.1f} s"}


def _plain_pass(mp, eng, bufs):
    """One query at a time, all queries ready at once: per-query wall latency from the
    start (the queries before it run first) and products run."""
    lat, prods = [], 0
    t0 = time.perf_counter()
    for b in bufs:
        rc, t = mp.mp_submit(eng.ctx, b)
        if rc != mp.MP_OK:
            raise mp.MPError(rc, "query")
        prods += mp.mp_result_stats(eng.ctx, t)["n_products"]
        mp.mp_release(eng.ctx, t)
        lat.append(time.perf_counter() - t0)
    return time.perf_counter() - t0, lat, prods


def _batch_pass(mp, eng, bufs):
    prods = 0
    t0 = time.perf_counter()
    rc, ts = mp.mp_submit_batch(eng.ctx, bufs)
    if rc != mp.MP_OK:
        raise mp.MPError(rc, "batch")
    for t in ts:
        prods += mp.mp_result_stats(eng.ctx, t)["n_products"]
        mp.mp_release(eng.ctx, t)
    return time.perf_counter() - t0, prods


def leg_plain_config1(mp, local, peak, peak_kind, reps=300):
    """The 2,000-paper HIN, one unconstrained APTPA query at a time (1500 x 1500 result)."""
    import torch
    import gen
    hin = gen.config1_hin()
    q = gen.config1_query()
    e = mp.Engine(hin, device=local, policy=mp.MP_POLICY_NONE)
    b = e.query(q)
    for _ in range(10):
        _, t = mp.mp_submit(e.ctx, b)
        mp.mp_release(e.ctx, t)
    torch.cuda.synchronize()
    mp.mp_kernel_stats_reset(e.ctx)
    lat = []
    with Clocks(local) as clk:
        t0 = time.perf_counter()
        for _ in range(reps):
            t1 = time.perf_counter()
            rc, t = mp.mp_submit(e.ctx, b)
            if rc != mp.MP_OK:
                raise mp.MPError(rc, "APTPA")
            mp.mp_release(e.ctx, t)
            lat.append(1e3 * (time.perf_counter() - t1))
        dt = time.perf_counter() - t0
    roof = _roofline(mp, e.ctx, peak, peak_kind, "2,000-paper HIN: the working set sits in L2")
    e.close()
    return {"workload": "2,000-paper scholarly HIN, unconstrained APTPA, one query at a time",
            "qps": reps / dt, "p50_ms": _pct(lat, 50), "p99_ms": _pct(lat, 99), "clocks": clk.summary(),
            "roofline": roof, "cpu_baseline": _oracle_sample(hin, [q] * 50, budget_s=3.0)}


def leg_small(mp, local, which, peak, peak_kind, reps=3, pool=500, anchor_p=0.75, full=False):
    """Batched workload (256 Zipf-drawn queries) or stress workload (64 long metapaths) on
    the 2,000-paper HIN: the plain one-at-a-time chain vs one batch (shared sub-chains
    once, one wave per level), autotuned, and replays through the Overlap-Tree cache."""
    import torch
    import gen
    hin = gen.config1_hin()
    if which == "batched":
        qs = gen.batched_queries(seed=3, n=256, pool=pool, anchor_p=anchor_p)
        name = (f"batched: 256 queries of length 3-7, Zipf(1.1) over a pool of {pool} templates, "
                f"{anchor_p:.0%} anchored on one of 16 entities, 2,000-paper HIN")
    else:
        qs = gen.long_queries(5, 64)
        name = "stress: 64 metapaths of length 7-9 through venues and topics, 2,000-paper HIN"
    plain = mp.Engine(hin, device=local, policy=mp.MP_POLICY_NONE)
    bufs = [plain.query(q) for q in qs]
    _plain_pass(mp, plain, bufs)
    _batch_pass(mp, plain, bufs)
    torch.cuda.synchronize()
    mp.mp_kernel_stats_reset(plain.ctx)
    p_s, b_s, p_lat, b_lat = [], [], [], []
    with Clocks(local) as clk:
        for _ in range(reps):
            dt, lat, p_prod = _plain_pass(mp, plain, bufs)
            p_s.append(dt)
            p_lat += lat
        for _ in range(reps):
            dt, b_prod = _batch_pass(mp, plain, bufs)
            b_s.append(dt)
            b_lat += [dt] * len(bufs)  # every query of a batch completes with the batch
    roof = _roofline(mp, plain.ctx, peak, peak_kind, "2,000-paper HIN: the working set sits in L2")
    tune = os.path.join(tempfile.mkdtemp(prefix="mp_tune_"), f"tune_{which}.json")
    mp.mp_autotune(plain.ctx, bufs, reps=2, out_path=tune)
    bt = min(_batch_pass(mp, plain, bufs)[0] for _ in range(reps))
    plain.close()
    n = len(qs)
    out = {"workload": name, "queries": n,
           "plain": {"qps": n / float(np.median(p_s)), "p50_ms": 1e3 * _pct(p_lat, 50),
                     "p99_ms": 1e3 * _pct(p_lat, 99), "products": p_prod},
           "batched": {"qps": n / float(np.median(b_s)), "p50_ms": 1e3 * _pct(b_lat, 50),
                       "p99_ms": 1e3 * _pct(b_lat, 99), "products": b_prod,
                       "duplicate_product_fraction": 1.0 - b_prod / max(p_prod, 1)},
           "batched_autotuned_qps": n / bt, "latency": "all queries arrive together; plain: time to each "
                                                       "query's own result, batched: the batch's time",
           "clocks": clk.summary(), "roofline": roof,
           "cpu_baseline": _oracle_sample(hin, qs, budget_s=4.0)}
    # replays through the cache: the first pass fills it, later passes reuse it
    budgets = {"8GB": 8 << 30}
    if which == "stress":
        # 25 % of the bytes of all distinct intermediates forces evictions
        e = mp.Engine(hin, device=local, policy=mp.MP_POLICY_ATRAPOS, insertion=mp.MP_INSERT_ALL,
                      cache_bytes=1 << 40, hbm_budget_bytes=1 << 40)
        rc, ts = mp.mp_submit_batch(e.ctx, [e.query(q) for q in qs])
        for t in ts:
            mp.mp_release(e.ctx, t)
        budgets["25pct"] = max(1 << 20, mp.mp_cache_stats(e.ctx)["bytes"] // 4)
        e.close()
    replays = {}
    pols = (mp.MP_POLICY_ATRAPOS, mp.MP_POLICY_PGDS, mp.MP_POLICY_LRU) if full or which == "stress" else \
        (mp.MP_POLICY_ATRAPOS,)
    for label, budget in budgets.items():
        for pol in pols:
            e = mp.Engine(hin, device=local, policy=pol, cache_bytes=int(budget))
            eb = [e.query(q) for q in qs]
            cold_s, _ = _batch_pass(mp, e, eb)
            warm = [_batch_pass(mp, e, eb) for _ in range(reps)]
            replays[f"{label}/{['atrapos', 'pgds', 'lru'][pol]}"] = {
                "first_pass_qps": n / cold_s, "replay_qps": n / float(np.median([w[0] for w in warm])),
                "replay_products": warm[-1][1], "cache": mp.mp_cache_stats(e.ctx) if full else None}
            e.close()
        if label == "25pct" and full:
            # the same budget with a second tier in host memory as large as everything
            e = mp.Engine(hin, device=local, policy=mp.MP_POLICY_ATRAPOS, cache_bytes=int(budget),
                          host_tier_bytes=int(4 * budget))
            eb = [e.query(q) for q in qs]
            cold_s, _ = _batch_pass(mp, e, eb)
            warm = [_batch_pass(mp, e, eb) for _ in range(reps)]
            replays[f"{label}/atrapos+host_tier"] = {
                "first_pass_qps": n / cold_s, "replay_qps": n / float(np.median([w[0] for w in warm])),
                "replay_products": warm[-1][1], "cache": mp.mp_cache_stats(e.ctx),
                "host_tier": mp.mp_host_tier_stats(e.ctx)}
            e.close()
    out["cached_replays"] = replays
    if full:
        out["batched_autotuned"] = {"qps": n / bt, "tune": json.load(open(tune))}
    return out


def leg_serving(mp, local, peak, peak_kind, scale=1.0, n=2000, loads=(0.5, 0.8, 1.0, 1.5), budget_gb=60.0):
    """News-shaped HIN (10 M articles, 2 M persons, 1 M organisations, 200 k locations, 20 k
    themes) and the session query stream of Sec. 4.1.2 arriving as a Poisson process at
    several rates relative to the plain path's saturation: the serving loop (continuous
    batching) with and without the Overlap-Tree cache against the plain one-query-at-a-time
    chain under the same arrivals. A seeded sample of n queries of the 100 k stream."""
    import torch
    import gen
    t_setup = time.perf_counter()
    hin = gen.config4_hin(seed=4, scale=scale)
    stream_q, _ = gen.serving_stream(hin, seed=4, n=100_000)
    qs = stream_q[:n]
    path = os.path.join(tempfile.mkdtemp(prefix="mp_news_"), "news.hin")
    budget = int(budget_gb * (1 << 30))
    plain = mp.Engine(hin, device=local, policy=mp.MP_POLICY_NONE, max_slots=1, hbm_budget_bytes=budget)
    plain.save(path)
    names = {"types": hin["types"], "props": {k: None for k in hin["props"]}}
    del hin
    bufs = [plain.query(q) for q in qs]
    for b in bufs[:20]:
        _, t = mp.mp_submit(plain.ctx, b)
        mp.mp_release(plain.ctx, t)
    torch.cuda.synchronize()
    n_sat = min(len(bufs), 500)
    t0 = time.perf_counter()
    for b in bufs[:n_sat]:
        _, t = mp.mp_submit(plain.ctx, b)
        mp.mp_release(plain.ctx, t)
    sat = n_sat / (time.perf_counter() - t0)
    setup_s = time.perf_counter() - t_setup

    def serve(eng, arrivals):
        qb = [eng.query(q) for q in qs]
        mp.mp_serve_start(eng.ctx)
        tickets, done = [], []

        def finish(t, i):
            st = mp.mp_wait(eng.ctx, t)
            if st != mp.MP_OK:
                raise mp.MPError(st, f"served query {i}")
            ms = mp.mp_result_latency(eng.ctx, t)
            mp.mp_release(eng.ctx, t)
            return ms

        start = time.perf_counter()
        for i, (b, at) in enumerate(zip(qb, arrivals)):
            d = start + at - time.perf_counter()
            if d > 0:
                time.sleep(d)
            _, t = mp.mp_submit(eng.ctx, b)
            tickets.append((t, i))
            # a client that got its result lets it go (results held by tickets count against
            # the budget): release the finished ones as the stream goes on
            while tickets and mp.mp_wait(eng.ctx, tickets[0][0], 0) != mp.MP_ERR_TIMEOUT:
                done.append(finish(*tickets.pop(0)))
        lat = done + [finish(t, i) for t, i in tickets]
        end = time.perf_counter()
        ct = mp.mp_serve_counters(eng.ctx)
        mp.mp_serve_stop(eng.ctx)
        return {"qps": len(qs) / (end - start), "p50_ms": _pct(lat, 50), "p99_ms": _pct(lat, 99),
                "joined": ct["joined"], "max_inflight": ct["max_inflight"]}

    rates = {}
    for load in loads:
        rate = load * sat
        arrivals = np.cumsum(gen.stream(4, 950, int(load * 100)).exponential(1.0 / rate, len(qs)))
        # every arm starts from a fresh context at every rate (the same cold planner memos;
        # the cache arm's entries never carry over from the previous rate)
        one = mp.Engine(names, device=local, load_path=path, policy=mp.MP_POLICY_NONE, max_slots=1,
                        hbm_budget_bytes=budget)
        nocache = mp.Engine(names, device=local, load_path=path, policy=mp.MP_POLICY_NONE, max_slots=64,
                            hbm_budget_bytes=budget)
        cached = mp.Engine(names, device=local, load_path=path, policy=mp.MP_POLICY_ATRAPOS, max_slots=64,
                           hbm_budget_bytes=budget)
        with Clocks(local) as clk:
            arms = {"plain": serve(one, arrivals), "served_no_cache": serve(nocache, arrivals),
                    "served_cache": serve(cached, arrivals)}
        arms["served_cache"]["cache_hits"] = mp.mp_cache_stats(cached.ctx)["hits"]
        for e in (one, nocache, cached):
            e.close()
        rates[f"{load:g}x"] = dict(arms, arrival_qps=rate, clocks=clk.summary())
    plain.close()
    try:
        os.remove(path)
    except OSError:
        pass
    return {"workload": "serving: news HIN, session query stream (anchor entity, date window on every "
                        "article position), Poisson arrivals",
            "articles": names["types"]["R"], "persons": names["types"]["E"], "orgs": names["types"]["O"],
            "locations": names["types"]["L"], "themes": names["types"]["H"],
            "queries_per_rate": len(qs), "sample": f"first {len(qs)} queries of the seeded 100,000-query stream",
            "plain_saturation_qps": sat, "cache": f"ATRAPOS-OTree, {budget_gb:g} GB budget", "max_slots": 64,
            "rates": rates, "setup_s": setup_s,
            "cpu_baseline": None, "cpu_baseline_note": "not run: the oracle would first build the CSR of "
                                                       "180 M edges in numpy (minutes of host time)"}


def run_leg(args, local):
    """--workload serving | batched | stress: one leg's full JSON line."""
    from paper_2201_04058_b300 import mp
    import torch
    torch.cuda.set_device(local)
    peak, kind = measured_peak()
    if args.workload == "serving":
        d = leg_serving(mp, local, peak, kind, scale=args.scale, n=args.serve_queries,
                        budget_gb=args.serve_budget_gb)
        head = d["rates"].get("1.5x") or list(d["rates"].values())[-1]
        value, p99 = head["served_cache"]["qps"], head["served_cache"]["p99_ms"]
        cfg = {"workload": d["workload"], "queries": d["queries_per_rate"]}
    else:
        d = leg_small(mp, local, args.workload, peak, kind, reps=max(1, args.steps), pool=args.pool,
                      anchor_p=args.anchor_p, full=True)
        value, p99 = d["batched"]["qps"], d["batched"]["p99_ms"]
        cfg = {"workload": d["workload"], "queries_per_step": d["queries"]}
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": 1,
           "ms_per_step": 1e3 / value, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "u64", "data": "synthetic (seeded generator; no dataset)", "config": cfg, "p99_ms": p99,
           "clocks": d.get("clocks") or head.get("clocks"), "roofline": d.get("roofline"),
           "cpu_baseline": d.get("cpu_baseline"), "detail": d}
    print(json.dumps(out), flush=True)


def run_kernel_probe(args, local):
    """--kernel-probe: the chosen scholarly queries, each run once in the plain form on a
    fresh engine (no warm-up, nothing cached), with the engine's per-kernel counters printed
    for each: launches, algorithmic bytes and Gustavson products. A profiler capture of the
    same command sees exactly these launches, so its DRAM bytes compare with the bytes here
    launch for launch."""
    import torch
    from paper_2201_04058_b300 import mp
    torch.cuda.set_device(local)
    hin, qs, cfg = workload(args.workload, args.scale)
    idx = list(range(len(qs))) if args.kernel_probe == "all" else [int(x) for x in args.kernel_probe.split(",")]
    eng = mp.Engine(hin, device=local, policy=mp.MP_POLICY_NONE, planner=PLANNERS[args.planner][0])
    per = []
    for i in idx:
        mp.mp_kernel_stats_reset(eng.ctx)
        rc, t = mp.mp_submit(eng.ctx, eng.query(qs[i]))
        if rc != mp.MP_OK:
            raise mp.MPError(rc, "query")
        mp.mp_release(eng.ctx, t)
        ks, _ = mp.mp_kernel_stats(eng.ctx)
        per.append({"query": i, "types": "".join(qs[i]["types"]),
                    "kernels": {k: {"launches": v["launches"], "bytes": v["bytes"], "products": v["products"],
                                    "ms": v["ms"]} for k, v in ks.items()}})
    eng.close()
    print(json.dumps({"kernel_probe": per, "config": dict(cfg, scale=args.scale)}), flush=True)


def main():
    args = parse()
    ws, rank, local = dist_env()
    if args.kernel_probe is not None:
        if rank == 0:
            run_kernel_probe(args, local)
        return
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    if args.workload in ("serving", "batched", "stress"):
        if rank == 0:
            run_leg(args, local)
        return
    run_engine(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
