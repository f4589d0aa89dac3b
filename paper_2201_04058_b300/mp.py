"""ctypes binding of include/mp.h (argument marshalling only).

Every function below calls the C entry point of the same name in ``_lib/libmp.so``;
all work happens in that library's CUDA kernels. ``Engine`` is a convenience wrapper
that loads a generated HIN and turns query dicts into ``mp_query`` structs.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libmp.so")

MP_OK = 0
MP_ERR_ARG, MP_ERR_STATE, MP_ERR_BUDGET, MP_ERR_TOO_LARGE, MP_ERR_OVERFLOW = -1, -2, -3, -4, -5
MP_ERR_TIMEOUT, MP_ERR_CUDA, MP_ERR_NOMEM, MP_ERR_NOTFOUND, MP_ERR_INTERNAL = -6, -7, -8, -9, -10
MP_POLICY_ATRAPOS, MP_POLICY_PGDS, MP_POLICY_LRU, MP_POLICY_NONE = 0, 1, 2, 3
MP_PLAN_DP, MP_PLAN_LEFT_TO_RIGHT, MP_PLAN_DP_SAMPLED, MP_PLAN_DP_MNC = 0, 1, 2, 3
MP_INSERT_OTREE, MP_INSERT_FINAL, MP_INSERT_ALL = 0, 1, 2
MP_BIN_AUTO, MP_BIN_WARP_HASH, MP_BIN_BLOCK_HASH, MP_BIN_DENSE, MP_BIN_GLOBAL = -1, 0, 1, 2, 3
MP_OP_RANGE, MP_OP_EQ, MP_OP_IN = 0, 1, 2
NBINS = 12  # warp hash x6, block hash x3, dense, global, lane

EXPORTS = [
    "mp_config_default", "mp_create", "mp_destroy", "mp_add_node_type", "mp_add_property_i32",
    "mp_add_relation", "mp_finalize_hin", "mp_type_id", "mp_property_id", "mp_relation_id",
    "mp_submit", "mp_submit_batch", "mp_wait", "mp_result_info", "mp_result_copy", "mp_release",
    "mp_result_time", "mp_strerror", "mp_result_stats", "mp_plan_chain", "mp_kernel_stats",
    "mp_kernel_stats_reset", "mp_otree_create", "mp_otree_create_ex", "mp_otree_destroy", "mp_otree_insert", "mp_otree_frequency",
    "mp_otree_info", "mp_cachesim_create", "mp_cachesim_destroy", "mp_cachesim_request", "mp_cachesim_entry",
    "mp_cachesim_evicted", "mp_cachesim_state", "mp_cache_stats", "mp_row_product_noalloc",
    "mp_serve_start", "mp_serve_stop", "mp_serve_stats", "mp_result_latency", "mp_autotune", "mp_hin_save",
    "mp_hin_load", "mp_plan_chain_mnc", "mp_plan_query", "mp_host_tier_stats", "mp_result_copy_async",
    "mp_result_copy_wait", "mp_graph_stats", "mp_serve_counters", "mp_budget_stats",
]


class mp_config(C.Structure):
    _fields_ = [("device", C.c_int32), ("hbm_budget_bytes", C.c_uint64), ("max_slots", C.c_uint32),
                ("policy", C.c_int32), ("planner", C.c_int32), ("cuda_stream", C.c_void_p),
                ("alpha", C.c_double), ("beta", C.c_double), ("gamma", C.c_double),
                ("force_bin_class", C.c_int32), ("max_result_bytes", C.c_uint64),
                ("scratch_bytes", C.c_uint64), ("sample_rows", C.c_uint32), ("seed", C.c_uint64),
                ("insertion", C.c_int32), ("tune_file", C.c_char_p), ("host_tier_bytes", C.c_uint64),
                ("cache_bytes", C.c_uint64), ("otree_construction", C.c_int32),
                ("alloc", C.c_void_p), ("free", C.c_void_p), ("alloc_user", C.c_void_p)]


# mp_config.alloc / .free
ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class TorchAllocator:
    """mp_config.alloc / .free backed by PyTorch's CUDA caching allocator, so the engine's
    device buffers come from the same pool as the caller's tensors. Keep the object alive
    as long as the context that uses it. Counts the live allocations it made."""

    def __init__(self, device: int = 0):
        import torch
        self.torch = torch
        self.device = device
        self.live = {}
        self.calls = 0

        def _alloc(nbytes, stream, user):
            try:
                p = self.torch.cuda.caching_allocator_alloc(int(nbytes), self.device, int(stream or 0))
            except RuntimeError:
                return None
            self.live[p] = int(nbytes)
            self.calls += 1
            return p

        def _free(ptr, stream, user):
            if ptr:
                self.live.pop(int(ptr), None)
                self.torch.cuda.caching_allocator_delete(int(ptr))

        self.alloc_fn = ALLOC_FN(_alloc)
        self.free_fn = FREE_FN(_free)

    def install(self, cfg):
        cfg.alloc = C.cast(self.alloc_fn, C.c_void_p)
        cfg.free = C.cast(self.free_fn, C.c_void_p)
        cfg.alloc_user = None


class mp_constraint(C.Structure):
    _fields_ = [("pos", C.c_int32), ("prop", C.c_int32), ("op", C.c_int32), ("lo", C.c_int64),
                ("hi", C.c_int64), ("set", C.c_void_p), ("set_len", C.c_uint32)]


class mp_query(C.Structure):
    _fields_ = [("n_types", C.c_uint32), ("types", C.c_void_p), ("rels", C.c_void_p),
                ("n_constraints", C.c_uint32), ("c", C.c_void_p)]


class mp_kernel_stat(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_uint64), ("ms", C.c_double), ("bytes", C.c_double),
                ("products", C.c_double)]


class MPError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} ({code})")


_lib = None


def lib():
    """The loaded engine library. Raises if it has not been built: there is no fallback."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"engine library missing: {LIB_PATH} (run paper_2201_04058_b300/build.py)")
        L = C.CDLL(LIB_PATH)
        P, I32, U32, U64 = C.POINTER, C.c_int32, C.c_uint32, C.c_uint64
        sig = {
            "mp_config_default": (None, [P(mp_config)]),
            "mp_create": (C.c_int, [P(mp_config), P(C.c_void_p)]),
            "mp_destroy": (None, [C.c_void_p]),
            "mp_add_node_type": (C.c_int, [C.c_void_p, C.c_char_p, U32, P(I32)]),
            "mp_add_property_i32": (C.c_int, [C.c_void_p, I32, C.c_char_p, C.c_void_p]),
            "mp_add_relation": (C.c_int, [C.c_void_p, I32, I32, U64, C.c_void_p, C.c_void_p, P(I32)]),
            "mp_finalize_hin": (C.c_int, [C.c_void_p]),
            "mp_type_id": (C.c_int, [C.c_void_p, C.c_char_p, P(I32)]),
            "mp_property_id": (C.c_int, [C.c_void_p, I32, C.c_char_p, P(I32)]),
            "mp_relation_id": (C.c_int, [C.c_void_p, I32, I32, P(I32)]),
            "mp_submit": (C.c_int, [C.c_void_p, P(mp_query), P(U64)]),
            "mp_plan_query": (C.c_int, [C.c_void_p, P(mp_query), U32, C.c_void_p, C.c_void_p, P(U32)]),
            "mp_submit_batch": (C.c_int, [C.c_void_p, U32, P(mp_query), P(U64)]),
            "mp_wait": (C.c_int, [C.c_void_p, U64, U32]),
            "mp_result_info": (C.c_int, [C.c_void_p, U64, P(U32), P(U32), P(U64)]),
            "mp_result_copy": (C.c_int, [C.c_void_p, U64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
            "mp_release": (C.c_int, [C.c_void_p, U64]),
            "mp_result_copy_async": (C.c_int, [C.c_void_p, U64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
            "mp_result_copy_wait": (C.c_int, [C.c_void_p, U64]),
            "mp_result_time": (C.c_int, [C.c_void_p, U64, P(C.c_double)]),
            "mp_strerror": (C.c_char_p, [C.c_int]),
            "mp_result_stats": (C.c_int, [C.c_void_p, U64, P(U64), C.c_void_p, C.c_void_p, P(U32)]),
            "mp_kernel_stats": (C.c_int, [C.c_void_p, C.c_void_p, U32, P(U32), P(U64)]),
            "mp_kernel_stats_reset": (C.c_int, [C.c_void_p]),
            "mp_cache_stats": (C.c_int, [C.c_void_p] + [P(U64)] * 7),
            "mp_host_tier_stats": (C.c_int, [C.c_void_p] + [P(U64)] * 5),
            "mp_graph_stats": (C.c_int, [C.c_void_p, P(U64), P(U64)]),
            "mp_hin_save": (C.c_int, [C.c_void_p, C.c_char_p]),
            "mp_hin_load": (C.c_int, [C.c_void_p, C.c_char_p]),
            "mp_autotune": (C.c_int, [C.c_void_p, U32, P(mp_query), U32, C.c_char_p, P(C.c_double)]),
            "mp_serve_start": (C.c_int, [C.c_void_p]),
            "mp_serve_stop": (C.c_int, [C.c_void_p]),
            "mp_serve_stats": (C.c_int, [C.c_void_p, P(U64), P(U64), P(U64)]),
            "mp_serve_counters": (C.c_int, [C.c_void_p, P(U64), P(U64), P(U64)]),
            "mp_budget_stats": (C.c_int, [C.c_void_p, P(U64), P(U64)]),
            "mp_result_latency": (C.c_int, [C.c_void_p, U64, P(C.c_double)]),
            "mp_row_product_noalloc": (C.c_int, [I32, C.c_void_p, U64, C.c_void_p, C.c_void_p, C.c_void_p,
                                                 C.c_void_p, C.c_void_p, U32, C.c_void_p, C.c_void_p, U64,
                                                 C.c_void_p, C.c_void_p, P(U64)]),
            "mp_otree_create": (C.c_int, [P(C.c_void_p)]),
            "mp_otree_create_ex": (C.c_int, [I32, P(C.c_void_p)]),
            "mp_otree_destroy": (None, [C.c_void_p]),
            "mp_otree_insert": (C.c_int, [C.c_void_p, U32, C.c_void_p, C.c_void_p]),
            "mp_otree_frequency": (C.c_int, [C.c_void_p, U32, C.c_void_p, C.c_char_p, P(U64)]),
            "mp_otree_info": (C.c_int, [C.c_void_p, P(U64), P(U64), P(I32)]),
            "mp_cachesim_create": (C.c_int, [C.c_double, I32, P(C.c_void_p)]),
            "mp_cachesim_destroy": (None, [C.c_void_p]),
            "mp_cachesim_request": (C.c_int, [C.c_void_p, U32, C.c_void_p, C.c_char_p, C.c_double, C.c_double,
                                              C.c_double, P(I32)]),
            "mp_cachesim_entry": (C.c_int, [C.c_void_p, U32, C.c_void_p, C.c_char_p, P(C.c_double),
                                            P(C.c_double), P(I32)]),
            "mp_cachesim_evicted": (C.c_int, [C.c_void_p, U32, C.c_char_p, U32, P(U32)]),
            "mp_cachesim_state": (C.c_int, [C.c_void_p, P(C.c_double), P(C.c_double), P(U32)]),
            "mp_plan_chain": (C.c_int, [U32, C.c_void_p, C.c_void_p, C.c_double, C.c_double, C.c_double,
                                        C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
            "mp_plan_chain_mnc": (C.c_int, [U32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                            C.c_double, C.c_double, C.c_double, C.c_void_p, C.c_void_p,
                                            C.c_void_p, C.c_void_p, C.c_void_p]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def strerror(code: int) -> str:
    return lib().mp_strerror(code).decode()


def _ck(rc, what):
    if rc != MP_OK:
        raise MPError(rc, what)
    return rc


def _ptr(a):
    return None if a is None else C.c_void_p(a.ctypes.data)


# ---- same-name wrappers of the C entry points --------------------------------------

def mp_config_default() -> mp_config:
    c = mp_config()
    lib().mp_config_default(C.byref(c))
    return c


def mp_create(cfg: mp_config | None = None):
    h = C.c_void_p()
    _ck(lib().mp_create(C.byref(cfg) if cfg is not None else None, C.byref(h)), "mp_create")
    return h


def mp_destroy(ctx):
    lib().mp_destroy(ctx)


def mp_add_node_type(ctx, name: str, count: int) -> int:
    t = C.c_int32()
    _ck(lib().mp_add_node_type(ctx, name.encode(), int(count), C.byref(t)), "mp_add_node_type")
    return t.value


def mp_add_property_i32(ctx, type_id: int, prop: str, values):
    v = np.ascontiguousarray(values, np.int32)
    _ck(lib().mp_add_property_i32(ctx, type_id, prop.encode(), _ptr(v)), "mp_add_property_i32")


def mp_add_relation(ctx, src_type: int, dst_type: int, src, dst) -> int:
    s = np.ascontiguousarray(src, np.uint32)
    d = np.ascontiguousarray(dst, np.uint32)
    if s.shape != d.shape:
        raise ValueError("src and dst differ in length")
    r = C.c_int32()
    _ck(lib().mp_add_relation(ctx, src_type, dst_type, s.size, _ptr(s), _ptr(d), C.byref(r)), "mp_add_relation")
    return r.value


def mp_finalize_hin(ctx):
    _ck(lib().mp_finalize_hin(ctx), "mp_finalize_hin")


def mp_hin_save(ctx, path: str):
    _ck(lib().mp_hin_save(ctx, path.encode()), "mp_hin_save")


def mp_hin_load(ctx, path: str):
    _ck(lib().mp_hin_load(ctx, path.encode()), "mp_hin_load")


def mp_type_id(ctx, name: str) -> int:
    t = C.c_int32()
    _ck(lib().mp_type_id(ctx, name.encode(), C.byref(t)), "mp_type_id")
    return t.value


def mp_property_id(ctx, type_id: int, prop: str) -> int:
    p = C.c_int32()
    _ck(lib().mp_property_id(ctx, type_id, prop.encode(), C.byref(p)), "mp_property_id")
    return p.value


def mp_relation_id(ctx, src_type: int, dst_type: int) -> int:
    r = C.c_int32()
    _ck(lib().mp_relation_id(ctx, src_type, dst_type, C.byref(r)), "mp_relation_id")
    return r.value


class _QueryBuf:
    """Keeps the ctypes arrays of one mp_query alive."""

    def __init__(self, types, rels, cons):
        self.types = np.ascontiguousarray(types, np.int32)
        self.rels = None if rels is None else np.ascontiguousarray(rels, np.int32)
        self.sets = []
        arr = (mp_constraint * max(1, len(cons)))()
        for i, (pos, prop, op, lo, hi, st) in enumerate(cons):
            sv = None
            if st is not None:
                sv = np.ascontiguousarray(st, np.uint32)
                self.sets.append(sv)
            arr[i] = mp_constraint(pos, prop, op, lo, hi, None if sv is None else sv.ctypes.data,
                                   0 if sv is None else sv.size)
        self.cons = arr
        self.q = mp_query(self.types.size, self.types.ctypes.data,
                          None if self.rels is None else self.rels.ctypes.data, len(cons), C.addressof(arr))


def make_query(types, rels=None, constraints=()):
    """constraints: iterable of (pos, prop_id or -1, op, lo, hi, set or None)."""
    return _QueryBuf(types, rels, list(constraints))


def mp_plan_query(ctx, query: _QueryBuf):
    """(split p x p int32, estimated sizes p x p float64) of the context's planner for one
    query, without running it."""
    p = C.c_uint32()
    rc = lib().mp_plan_query(ctx, C.byref(query.q), 0, None, None, C.byref(p))
    if rc not in (MP_OK, MP_ERR_ARG) or p.value == 0:
        _ck(rc, "mp_plan_query")
    n = p.value
    split = np.zeros((n, n), np.int32)
    nnz = np.zeros((n, n), np.float64)
    _ck(lib().mp_plan_query(ctx, C.byref(query.q), n * n, _ptr(split), _ptr(nnz), C.byref(p)), "mp_plan_query")
    return split, nnz


def mp_submit(ctx, query: _QueryBuf) -> tuple[int, int]:
    """Returns (status, ticket); the ticket is valid even when the status is an error."""
    t = C.c_uint64()
    rc = lib().mp_submit(ctx, C.byref(query.q), C.byref(t))
    if rc in (MP_ERR_ARG, MP_ERR_STATE, MP_ERR_NOTFOUND) and t.value == 0:
        raise MPError(rc, "mp_submit")
    return rc, t.value


def mp_submit_batch(ctx, queries) -> tuple[int, list[int]]:
    n = len(queries)
    arr = (mp_query * max(1, n))(*[q.q for q in queries])
    tk = (C.c_uint64 * max(1, n))()
    rc = lib().mp_submit_batch(ctx, n, arr, tk)
    if rc in (MP_ERR_ARG, MP_ERR_STATE, MP_ERR_NOTFOUND) and n and tk[0] == 0:
        raise MPError(rc, "mp_submit_batch")
    return rc, [int(tk[i]) for i in range(n)]


def mp_wait(ctx, ticket: int, timeout_ms: int = 0xFFFFFFFF) -> int:
    return lib().mp_wait(ctx, ticket, timeout_ms)


def mp_autotune(ctx, queries, reps=2, out_path=None):
    """Tune bin thresholds and fit Eq. 2 on a workload; returns the best time per run (ms)."""
    n = len(queries)
    arr = (mp_query * max(1, n))(*[q.q for q in queries])
    best = C.c_double()
    _ck(lib().mp_autotune(ctx, n, arr, int(reps), None if out_path is None else out_path.encode(), C.byref(best)),
        "mp_autotune")
    return best.value


def mp_serve_start(ctx):
    _ck(lib().mp_serve_start(ctx), "mp_serve_start")


def mp_serve_stop(ctx):
    _ck(lib().mp_serve_stop(ctx), "mp_serve_stop")


def mp_serve_stats(ctx):
    b, q, w = C.c_uint64(), C.c_uint64(), C.c_uint64()
    _ck(lib().mp_serve_stats(ctx, C.byref(b), C.byref(q), C.byref(w)), "mp_serve_stats")
    return {"batches": b.value, "queries": q.value, "queued": w.value}


def mp_serve_counters(ctx):
    w, j, m = C.c_uint64(), C.c_uint64(), C.c_uint64()
    _ck(lib().mp_serve_counters(ctx, C.byref(w), C.byref(j), C.byref(m)), "mp_serve_counters")
    return {"waves": w.value, "joined": j.value, "max_inflight": m.value}


def mp_budget_stats(ctx):
    h, p = C.c_uint64(), C.c_uint64()
    _ck(lib().mp_budget_stats(ctx, C.byref(h), C.byref(p)), "mp_budget_stats")
    return {"held": h.value, "peak": p.value}


def mp_result_latency(ctx, ticket: int) -> float:
    ms = C.c_double()
    _ck(lib().mp_result_latency(ctx, ticket, C.byref(ms)), "mp_result_latency")
    return ms.value


def mp_result_info(ctx, ticket: int):
    r, c, z = C.c_uint32(), C.c_uint32(), C.c_uint64()
    _ck(lib().mp_result_info(ctx, ticket, C.byref(r), C.byref(c), C.byref(z)), "mp_result_info")
    return r.value, c.value, z.value


def mp_result_copy(ctx, ticket: int, row_ptr=None, col=None, val=None, on_device: bool = False):
    """Copy into caller buffers: numpy arrays (host) or integer device addresses."""
    def addr(a):
        if a is None:
            return None
        if isinstance(a, int):
            return C.c_void_p(a)
        return C.c_void_p(a.ctypes.data)
    _ck(lib().mp_result_copy(ctx, ticket, addr(row_ptr), addr(col), addr(val), 1 if on_device else 0),
        "mp_result_copy")


def mp_result_copy_async(ctx, ticket: int, row_ptr=None, col=None, val=None, on_device: bool = False):
    """Queue the copy and return; the buffers (integer addresses, or arrays kept alive by
    the caller) must not be read before mp_result_copy_wait."""
    def addr(a):
        if a is None:
            return None
        if isinstance(a, int):
            return C.c_void_p(a)
        return C.c_void_p(a.ctypes.data)
    _ck(lib().mp_result_copy_async(ctx, ticket, addr(row_ptr), addr(col), addr(val), 1 if on_device else 0),
        "mp_result_copy_async")


def mp_result_copy_wait(ctx, ticket: int):
    _ck(lib().mp_result_copy_wait(ctx, ticket), "mp_result_copy_wait")


def mp_release(ctx, ticket: int):
    _ck(lib().mp_release(ctx, ticket), "mp_release")


def mp_result_time(ctx, ticket: int) -> float:
    ms = C.c_double()
    _ck(lib().mp_result_time(ctx, ticket, C.byref(ms)), "mp_result_time")
    return ms.value


def mp_result_stats(ctx, ticket: int):
    prod, npr = C.c_uint64(), C.c_uint32()
    sb = np.zeros(NBINS, np.uint32)
    nb = np.zeros(NBINS, np.uint32)
    _ck(lib().mp_result_stats(ctx, ticket, C.byref(prod), _ptr(sb), _ptr(nb), C.byref(npr)), "mp_result_stats")
    return {"products": prod.value, "sym_bins": sb, "num_bins": nb, "n_products": npr.value}


def mp_plan_chain(dims, nnz, alpha=1.0, beta=1.0, gamma=1.0, known=None, rho_fixed=None):
    """Splits (p x p int32) and costs (p x p float64) of the C++ planner. known maps
    (i, j) -> (cost, density); rho_fixed maps (i, j) -> measured result density."""
    dims = np.ascontiguousarray(dims, np.float64)
    nnz = np.ascontiguousarray(nnz, np.float64)
    p = nnz.size
    kc = kr = None
    if known:
        kc = np.full((p, p), np.nan)
        kr = np.full((p, p), np.nan)
        for (i, j), (c, r) in known.items():
            kc[i, j], kr[i, j] = c, r
    rf = None
    if rho_fixed:
        rf = np.full((p, p), np.nan)
        for (i, j), r in rho_fixed.items():
            rf[i, j] = r
    split = np.zeros((p, p), np.int32)
    cost = np.zeros((p, p), np.float64)
    _ck(lib().mp_plan_chain(p, _ptr(dims), _ptr(nnz), alpha, beta, gamma, _ptr(kc), _ptr(kr), _ptr(rf),
                            _ptr(split), _ptr(cost)), "mp_plan_chain")
    return split, cost


def mp_plan_chain_mnc(dims, sketches, alpha=1.0, beta=1.0, gamma=1.0, known=None):
    """Splits (p x p int32), costs and estimated sizes (p x p float64) of the C++ MNC
    planner. sketches[t] = (hr, hc, her, hec) count vectors of leaf factor t; known maps
    (i, j) -> (cost, nnz)."""
    dims = np.ascontiguousarray(dims, np.float64)
    p = len(sketches)
    vecs = [[np.ascontiguousarray(v, np.uint32) for v in sk] for sk in sketches]
    arrs = []
    for f in range(4):
        a = (C.c_void_p * p)(*[vecs[t][f].ctypes.data for t in range(p)])
        arrs.append(a)
    kc = kz = None
    if known:
        kc = np.full((p, p), np.nan)
        kz = np.full((p, p), np.nan)
        for (i, j), (c, z) in known.items():
            kc[i, j], kz[i, j] = c, z
    split = np.zeros((p, p), np.int32)
    cost = np.zeros((p, p), np.float64)
    nnz = np.zeros((p, p), np.float64)
    _ck(lib().mp_plan_chain_mnc(p, _ptr(dims), *arrs, alpha, beta, gamma, _ptr(kc), _ptr(kz), _ptr(split),
                                _ptr(cost), _ptr(nnz)), "mp_plan_chain_mnc")
    return split, cost, nnz


def mp_kernel_stats(ctx):
    """({name: {"launches", "ms", "bytes", "products"}}, total kernel launches of the library)."""
    arr = (mp_kernel_stat * 64)()
    n, launches = C.c_uint32(), C.c_uint64()
    _ck(lib().mp_kernel_stats(ctx, arr, 64, C.byref(n), C.byref(launches)), "mp_kernel_stats")
    return ({arr[i].name.decode(): {"launches": arr[i].launches, "ms": arr[i].ms, "bytes": arr[i].bytes,
                                    "products": arr[i].products} for i in range(n.value)}, launches.value)


def mp_cache_stats(ctx):
    v = [C.c_uint64() for _ in range(7)]
    _ck(lib().mp_cache_stats(ctx, *[C.byref(x) for x in v]), "mp_cache_stats")
    return dict(zip(("requests", "hits", "inserts", "rejected", "evictions", "bytes", "entries"),
                    (x.value for x in v)))


def mp_host_tier_stats(ctx):
    v = [C.c_uint64() for _ in range(5)]
    _ck(lib().mp_host_tier_stats(ctx, *[C.byref(x) for x in v]), "mp_host_tier_stats")
    return dict(zip(("stores", "loads", "drops", "bytes", "entries"), (x.value for x in v)))


def mp_graph_stats(ctx):
    c, r = C.c_uint64(), C.c_uint64()
    _ck(lib().mp_graph_stats(ctx, C.byref(c), C.byref(r)), "mp_graph_stats")
    return {"captures": c.value, "replays": r.value}


def mp_kernel_stats_reset(ctx):
    _ck(lib().mp_kernel_stats_reset(ctx), "mp_kernel_stats_reset")


MP_OTREE_NAIVE, MP_OTREE_ONLINE = 0, 1


class OTree:
    """Host-only Overlap Tree replay (mp_otree_*), built by the naive insertion or on-line
    (Ukkonen)."""

    def __init__(self, construction: int = MP_OTREE_NAIVE):
        self.h = C.c_void_p()
        _ck(lib().mp_otree_create_ex(int(construction), C.byref(self.h)), "mp_otree_create_ex")

    def insert(self, types, pos_keys=None):
        t = np.ascontiguousarray(types, np.int32)
        keys = None
        if pos_keys is not None:
            keys = (C.c_char_p * t.size)(*[(k or "").encode() for k in pos_keys])
        _ck(lib().mp_otree_insert(self.h, t.size, _ptr(t), keys), "mp_otree_insert")

    def frequency(self, s, key=None):
        t = np.ascontiguousarray(s, np.int32)
        f = C.c_uint64()
        _ck(lib().mp_otree_frequency(self.h, t.size, _ptr(t), None if key is None else key.encode(), C.byref(f)),
            "mp_otree_frequency")
        return f.value

    def info(self):
        n, l, ok = C.c_uint64(), C.c_uint64(), C.c_int32()
        _ck(lib().mp_otree_info(self.h, C.byref(n), C.byref(l), C.byref(ok)), "mp_otree_info")
        return n.value, l.value, bool(ok.value)

    def __del__(self):
        try:
            lib().mp_otree_destroy(self.h)
        except Exception:
            pass


class CacheSim:
    """Host-only cache-policy replay (mp_cachesim_*)."""

    def __init__(self, capacity, policy):
        self.h = C.c_void_p()
        _ck(lib().mp_cachesim_create(float(capacity), int(policy), C.byref(self.h)), "mp_cachesim_create")

    def request(self, types, key, f, cost, size):
        t = np.ascontiguousarray(types, np.int32)
        out = C.c_int32()
        _ck(lib().mp_cachesim_request(self.h, t.size, _ptr(t), key.encode(), float(f), float(cost), float(size),
                                      C.byref(out)), "mp_cachesim_request")
        return ("hit", "inserted", "rejected")[out.value]

    def entry(self, types, key):
        t = np.ascontiguousarray(types, np.int32)
        c, h, pr = C.c_double(), C.c_double(), C.c_int32()
        _ck(lib().mp_cachesim_entry(self.h, t.size, _ptr(t), key.encode(), C.byref(c), C.byref(h), C.byref(pr)),
            "mp_cachesim_entry")
        return (c.value, h.value) if pr.value else None

    def evicted(self):
        n = C.c_uint32()
        _ck(lib().mp_cachesim_evicted(self.h, 0, None, 0, C.byref(n)), "mp_cachesim_evicted")
        out = []
        buf = C.create_string_buffer(1 << 16)
        for i in range(n.value):
            _ck(lib().mp_cachesim_evicted(self.h, i, buf, len(buf), None), "mp_cachesim_evicted")
            out.append(buf.value.decode())
        return out

    def state(self):
        L, used, items = C.c_double(), C.c_double(), C.c_uint32()
        _ck(lib().mp_cachesim_state(self.h, C.byref(L), C.byref(used), C.byref(items)), "mp_cachesim_state")
        return L.value, used.value, items.value

    def __del__(self):
        try:
            lib().mp_cachesim_destroy(self.h)
        except Exception:
            pass


def cache_item_id(types, key):
    """The engine's id string of a cached item (types + constraint key)."""
    return "".join(f"{int(t)}," for t in types) + "#" + key


def mp_row_product_noalloc(device, stream, x_len, x_ci, x_val, y_rp, y_ci, y_val, y_cols, km, cm, out_cap,
                           out_ci, out_val):
    """One product row into caller-owned device buffers, allocating nothing. Pointer
    arguments are integer device addresses (0 for NULL). Returns (status, nnz)."""
    nnz = C.c_uint64()
    v = lambda x: C.c_void_p(x) if x else None
    rc = lib().mp_row_product_noalloc(int(device), v(stream), int(x_len), v(x_ci), v(x_val), v(y_rp), v(y_ci),
                                      v(y_val), int(y_cols), v(km), v(cm), int(out_cap), v(out_ci), v(out_val),
                                      C.byref(nnz))
    return rc, nnz.value


# ---- convenience wrapper -------------------------------------------------------------

_OPS = {"range": MP_OP_RANGE, "eq": MP_OP_EQ, "in": MP_OP_IN}


class Engine:
    """One context with a HIN loaded from a generator dict (see the ``gen`` module)."""

    def __init__(self, hin, allocator=None, load_path=None, **cfg_fields):
        """hin: a generator dict (types, relations, props); with load_path, the HIN comes
        from a file mp_hin_save wrote instead (hin then only names its types and props)."""
        self.cfg = mp_config_default()
        for k, v in cfg_fields.items():
            setattr(self.cfg, k, v.encode() if isinstance(v, str) else v)
        self.allocator = allocator  # e.g. TorchAllocator: kept alive with the context
        if allocator is not None:
            allocator.install(self.cfg)
        self.ctx = mp_create(self.cfg)
        self.type_id = {}
        self.prop_id = {}
        if load_path is not None:
            mp_hin_load(self.ctx, load_path)
            mp_finalize_hin(self.ctx)
            for name in hin["types"]:
                self.type_id[name] = mp_type_id(self.ctx, name)
        else:
            for name, n in hin["types"].items():
                self.type_id[name] = mp_add_node_type(self.ctx, name, n)
            for (t, p), vals in hin["props"].items():
                mp_add_property_i32(self.ctx, self.type_id[t], p, vals)
            for a, b, s, d in hin["relations"]:
                mp_add_relation(self.ctx, self.type_id[a], self.type_id[b], s, d)
            mp_finalize_hin(self.ctx)
        for (t, p) in hin["props"]:
            self.prop_id[(t, p)] = mp_property_id(self.ctx, self.type_id[t], p)

    def save(self, path):
        mp_hin_save(self.ctx, path)

    def query(self, q):
        cons = []
        for c in q.get("constraints", []):
            t = q["types"][c["pos"]]
            prop = -1 if c.get("prop") is None else self.prop_id[(t, c["prop"])]
            op = _OPS[c["op"]]
            lo = int(c.get("lo", 0))
            hi = int(c.get("hi", lo))
            st = c.get("set") if op == MP_OP_IN else None
            if op == MP_OP_IN and st is None:
                st = np.zeros(0, np.uint32)
            cons.append((int(c["pos"]), prop, op, lo, hi, st))
        return make_query([self.type_id[t] for t in q["types"]], None, cons)

    def submit(self, q):
        return mp_submit(self.ctx, self.query(q))

    def plan(self, q):
        """The planner's (split, estimated sizes) for q; no product runs."""
        return mp_plan_query(self.ctx, self.query(q))

    def submit_batch(self, qs):
        return mp_submit_batch(self.ctx, [self.query(q) for q in qs])

    def fetch(self, ticket):
        rows, cols, nnz = mp_result_info(self.ctx, ticket)
        rp = np.empty(rows + 1, np.int64)
        ci = np.empty(nnz, np.int32)
        val = np.empty(nnz, np.uint64)
        mp_result_copy(self.ctx, ticket, rp, ci, val)
        return rp, ci, val

    def run_batch(self, qs):
        """Submit a batch, fetch every result (or the error code) and release the tickets."""
        rc, tickets = self.submit_batch(qs)
        out = []
        for t in tickets:
            st = mp_wait(self.ctx, t)
            out.append(self.fetch(t) if st == MP_OK else st)
            mp_release(self.ctx, t)
        return rc, out

    def run(self, q):
        """Submit, fetch and release one query; raises MPError on a query error."""
        rc, t = self.submit(q)
        try:
            _ck(rc, "query")
            return self.fetch(t)
        finally:
            mp_release(self.ctx, t)

    def release(self, ticket):
        mp_release(self.ctx, ticket)

    def close(self):
        if self.ctx:
            mp_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
