/*
 * mp.h -- C ABI of the B300 metapath-query engine.
 *
 * The engine evaluates metapath queries over a heterogeneous information network (HIN)
 * as chains of typed sparse adjacency products in CSR form with exact uint64 path
 * counts. Every call below follows the paper's statement of the problem:
 *
 *   - a HIN is a set of typed nodes and typed edges; each edge type r between node types
 *     o' and o'' is a |o'| x |o''| 0/1 adjacency matrix A_r (Sec. 2, Def. 1);
 *   - a metapath <o_1 ... o_n> has length n (number of node types, Def. 2) and a
 *     constrained metapath adds per-node property constraints (Def. 3);
 *   - a query returns every pair <v_o, v_d> joined by at least one instance, with the
 *     number of instances (Problem 1): the non-zeros of
 *         A_m = M_1 A_{o1 o2} M_2 A_{o2 o3} ... A_{o(n-1) o(n)} M_n,
 *     M_i being the 0/1 diagonal of the nodes of type o_i that meet the constraints at
 *     position i (the constrained adjacency M_c * A of Sec. 2);
 *   - a workload is a sequence of such queries (Problem 2), served with the chain-order
 *     planner of Sec. 3.1-3.2 (Eq. 1, Eq. 2) and the Overlap-Tree cache of Sec. 3.3-3.4.
 *
 * Conventions
 *   - Every call returns an int: MP_OK (0) or a negative MP_ERR_* code; no call throws
 *     or aborts across the ABI. mp_strerror() names a code.
 *   - Ownership: the library copies every input array before the call returns. Result
 *     buffers are allocated by the CALLER, sized from mp_result_info(). Tickets stay
 *     valid until mp_release().
 *   - Results are canonical CSR: int64 row pointers (rows+1 entries, empty rows kept),
 *     int32 column ids strictly ascending within a row, uint64 counts >= 1, no stored
 *     zeros. A count that does not fit in 64 bits is reported as MP_ERR_OVERFLOW on the
 *     query's ticket, never wrapped.
 *   - Threads: calls on one context are serialised by an internal lock.
 *   - Device: one GPU per context (mp_config.device). Device pointers passed in or out
 *     belong to that device.
 */
#ifndef MP_H_
#define MP_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MP_OK 0
#define MP_ERR_ARG (-1)       /* malformed argument */
#define MP_ERR_STATE (-2)     /* call not valid in the context's current state */
#define MP_ERR_BUDGET (-3)    /* the HBM byte budget cannot hold the work */
#define MP_ERR_TOO_LARGE (-4) /* result or intermediate beyond the size guard */
#define MP_ERR_OVERFLOW (-5)  /* a path count exceeds 2^64 - 1 */
#define MP_ERR_TIMEOUT (-6)   /* mp_wait timed out, or a bounded device wait gave up */
#define MP_ERR_CUDA (-7)      /* a CUDA runtime call failed */
#define MP_ERR_NOMEM (-8)     /* host or device allocation failed */
#define MP_ERR_NOTFOUND (-9)  /* unknown ticket, type, property or relation */
#define MP_ERR_INTERNAL (-10) /* a device-side consistency check failed */

/* cache replacement policies (Sec. 3.4.2) */
#define MP_POLICY_ATRAPOS 0 /* Alg. 1: PGDS utility + Overlap-Tree cost dependencies */
#define MP_POLICY_PGDS 1    /* popularity-aware greedy dual-size */
#define MP_POLICY_LRU 2     /* least recently used */
#define MP_POLICY_NONE 3    /* no caching */

/* cache insertion policies (Sec. 3.4.1 and the baselines of Sec. 4.1.3) */
#define MP_INSERT_OTREE 0 /* the whole query + its longest sub-metapath seen at least twice */
#define MP_INSERT_FINAL 1 /* final query results only (with LRU: the CBS1 baseline) */
#define MP_INSERT_ALL 2   /* every computed result and intermediate (with LRU: CBS2) */

/* chain-order planners */
#define MP_PLAN_DP 0            /* Eq. 1 DP with the Eq. 2 cost and E_ac densities */
#define MP_PLAN_LEFT_TO_RIGHT 1 /* ((A1 A2) A3) ... */
#define MP_PLAN_DP_SAMPLED 2    /* Eq. 1 DP, densities from per-row nnz sampling */
#define MP_PLAN_DP_MNC 3        /* Eq. 1 DP, result sizes from MNC count sketches */

/* row-bin classes, for mp_config.force_bin_class (tests and the autotuner) */
#define MP_BIN_AUTO (-1)
#define MP_BIN_WARP_HASH 0  /* one warp per row, shared-memory hash table */
#define MP_BIN_BLOCK_HASH 1 /* one block per row, shared-memory hash table */
#define MP_BIN_DENSE 2      /* one block per row, dense shared-memory accumulator */
#define MP_BIN_GLOBAL 3     /* split rows: fixed-size work items over all blocks, a bitmap +
                               rank or a dense count row per row in global scratch */

/* Overlap-Tree constructions (Sec. 3.3.2); both give the same tree */
#define MP_OTREE_NAIVE 0  /* the suffix-by-suffix insertion of Sec. 3.3.2 */
#define MP_OTREE_ONLINE 1 /* Ukkonen's on-line construction (footnote of Sec. 3.3.2) */

typedef struct mp_ctx mp_ctx;
typedef uint64_t mp_ticket;

typedef struct {
    int32_t device;            /* CUDA device ordinal */
    uint64_t hbm_budget_bytes; /* HBM byte budget of the queries' data: results held by
                                  tickets, intermediates in flight and cache entries (the
                                  HIN and the transient product workspace are not counted;
                                  0 = no limit). Every product's exact result bytes are
                                  charged before its arrays are made; when they do not fit,
                                  the cache evicts its policy's victims first, and a product
                                  that still cannot fit fails its query with MP_ERR_BUDGET.
                                  The serving loop admits new queries only while the planned
                                  result bytes of those in flight are below it. */
    uint32_t max_slots;        /* queries in flight at once in the serving loop */
    int32_t policy;            /* MP_POLICY_* */
    int32_t planner;           /* MP_PLAN_* */
    void *cuda_stream;         /* cudaStream_t to launch on; NULL = the library's own */
    double alpha, beta, gamma; /* Eq. 2 coefficients */
    int32_t force_bin_class;   /* MP_BIN_AUTO, or force every non-empty row into a class
                                  (rows that cannot fit it go to the next larger one) */
    uint64_t max_result_bytes; /* size guard per product (0 = no guard) */
    uint64_t scratch_bytes;    /* cap on the global-accumulator scratch (0 = default) */
    uint32_t sample_rows;      /* rows sampled per product by MP_PLAN_DP_SAMPLED */
    uint64_t seed;             /* seed of the sampled-row choice */
    int32_t insertion;         /* MP_INSERT_* (used when policy != MP_POLICY_NONE) */
    const char *tune_file;     /* NULL, or a file written by mp_autotune to load at create */
    uint64_t host_tier_bytes;  /* second cache tier in pinned host memory for results the
                                  device cache evicts (0 = off); a later plan may copy one
                                  back instead of recomputing it */
    uint64_t cache_bytes;      /* capacity of the cache (the cache size of Sec. 3.4), within
                                  the budget; 0 = the whole hbm_budget_bytes */
    int32_t otree_construction; /* MP_OTREE_ONLINE (default) or MP_OTREE_NAIVE */
    /* Optional device allocator for every device buffer the context makes (HIN, masks,
     * results, intermediates, workspaces), e.g. PyTorch's caching allocator, so that one
     * pool serves the caller and the engine. alloc returns `bytes` of device memory on
     * the context's device, usable in the order of `stream` (the context's cudaStream_t),
     * or NULL when it cannot; free gives back a buffer alloc returned, in the order of
     * `stream`: work queued on `stream` before the call may still use it, and the buffer
     * may serve later allocations on that stream. Both are called from the thread that
     * runs the query (the caller's, or the serving loop's), never concurrently for one
     * context. Both NULL (the default): the CUDA stream-ordered pool. Setting one alone is
     * MP_ERR_ARG at mp_create. */
    void *(*alloc)(size_t bytes, void *stream, void *user);
    void (*free)(void *ptr, void *stream, void *user);
    void *alloc_user;          /* passed to alloc and free as `user` */
} mp_config;

/* Fill *cfg with defaults: device 0, 8 GiB budget (the cache may use all of it), 64 slots,
 * ATRAPOS policy, DP planner, alpha = beta = gamma = 1, automatic bins, no size guard,
 * on-line Overlap-Tree construction, the CUDA stream-ordered pool. */
void mp_config_default(mp_config *cfg);

/* Create a context on cfg->device. Errors: MP_ERR_ARG, MP_ERR_CUDA. */
int mp_create(const mp_config *cfg, mp_ctx **out);
void mp_destroy(mp_ctx *ctx);

/* ---- HIN ingestion (Sec. 2, Def. 1); ingestion time is not query time (Sec. 4.1.4) */

/* Declare a node type with `count` nodes (ids 0..count-1). */
int mp_add_node_type(mp_ctx *ctx, const char *name, uint32_t count, int32_t *type_id);

/* Attach an int32 property to every node of a type; `values` has `count` entries of
 * that type, host memory, copied. */
int mp_add_property_i32(mp_ctx *ctx, int32_t type_id, const char *prop, const int32_t *values);

/* Add the edge type src_type -> dst_type from n_edges host (src, dst) pairs, copied.
 * Repeated pairs collapse (0/1 adjacency). The reverse relation dst -> src is created
 * too and gets id (*rel_id ^ 1). Errors: MP_ERR_ARG for out-of-range ids. */
int mp_add_relation(mp_ctx *ctx, int32_t src_type, int32_t dst_type, uint64_t n_edges,
                    const uint32_t *src, const uint32_t *dst, int32_t *rel_id);

/* Build the device CSR of every relation and upload properties. No adds after this. */
int mp_finalize_hin(mp_ctx *ctx);

/* Save a finalised context's HIN (node types, properties, every relation's CSR in both
 * directions) to a binary file, and load one into a fresh context instead of the
 * mp_add_* calls; mp_finalize_hin then uploads it without rebuilding the CSRs.
 * Errors: MP_ERR_STATE (save before finalize, load into a non-empty context),
 * MP_ERR_NOTFOUND (no file), MP_ERR_ARG (unreadable or malformed file). */
int mp_hin_save(mp_ctx *ctx, const char *path);
int mp_hin_load(mp_ctx *ctx, const char *path);

/* Look-ups by name. */
int mp_type_id(mp_ctx *ctx, const char *name, int32_t *type_id);
int mp_property_id(mp_ctx *ctx, int32_t type_id, const char *prop, int32_t *prop_id);
/* Relation from src_type to dst_type (the first one added, for queries with rels=NULL). */
int mp_relation_id(mp_ctx *ctx, int32_t src_type, int32_t dst_type, int32_t *rel_id);

/* ---- queries (Sec. 2, Def. 2-3, Problem 1-2) */

#define MP_OP_RANGE 0 /* lo <= v <= hi */
#define MP_OP_EQ 1    /* v == lo */
#define MP_OP_IN 2    /* v in set[0..set_len) */

typedef struct {
    int32_t pos;          /* 0-based position in the metapath */
    int32_t prop;         /* property id from mp_property_id, or -1 for the node id */
    int32_t op;           /* MP_OP_* */
    int64_t lo, hi;
    const uint32_t *set;  /* host array for MP_OP_IN, copied */
    uint32_t set_len;
} mp_constraint;

typedef struct {
    uint32_t n_types;      /* metapath length n >= 2 */
    const int32_t *types;  /* n type ids */
    const int32_t *rels;   /* n-1 relation ids, or NULL: the relation of each type pair */
    uint32_t n_constraints;
    const mp_constraint *c;
} mp_query;

/* Evaluate one query. The query is copied; the result is held under *ticket until
 * mp_release. Query errors (MP_ERR_OVERFLOW, MP_ERR_TOO_LARGE, MP_ERR_BUDGET) are
 * returned here and by mp_wait for the ticket. */
int mp_submit(mp_ctx *ctx, const mp_query *q, mp_ticket *ticket);

/* Evaluate n queries as one workload: products shared by several queries run once;
 * all products that are ready at the same time run in one launch per pass. tickets[i]
 * receives the ticket of q[i]; the return value is MP_OK when every query succeeded,
 * else the first failing query's error (each ticket keeps its own status). */
int mp_submit_batch(mp_ctx *ctx, uint32_t n, const mp_query *q, mp_ticket *tickets);

/* Wait for a ticket's result: MP_OK, the query's own error, or MP_ERR_TIMEOUT when it is
 * not finished within timeout_ms (UINT32_MAX = no limit, 0 = poll). */
int mp_wait(mp_ctx *ctx, mp_ticket ticket, uint32_t timeout_ms);

/* ---- serving (Problem 2 as a live request stream)
 *
 * mp_serve_start starts a host thread that serves the workload as it arrives, with
 * continuous batching. Every turn it admits the queries that have arrived, while fewer
 * than mp_config.max_slots are in flight and the planned result bytes of those in flight
 * are below the HBM budget: their plans join one product DAG with the queries already in
 * flight (a sub-chain that is on its way or held is shared, a cached one is reused,
 * Sec. 3.4). It then runs one wave -- every product whose operands are ready, of any
 * query, in one set of launches -- and publishes every query whose result is complete.
 * A query that arrives while others are on the GPU therefore starts at the next wave,
 * beside their later products. While serving, mp_submit and mp_submit_batch only queue
 * the queries and return tickets at once; results are read after mp_wait.
 * mp_serve_stop finishes the queued work and stops the thread (mp_destroy stops it too).
 * Errors: MP_ERR_STATE (not finalised, already serving). */
int mp_serve_start(mp_ctx *ctx);
int mp_serve_stop(mp_ctx *ctx);
/* Admission groups (turns that admitted at least one query) and queries served so far,
 * and queries waiting for admission now. */
int mp_serve_stats(mp_ctx *ctx, uint64_t *batches, uint64_t *queries, uint64_t *queued);
/* Waves the serving loop has run, queries it admitted while other queries were in flight
 * (their products joined waves beside the in-flight ones), and the most queries in flight
 * at once. Any pointer may be NULL. */
int mp_serve_counters(mp_ctx *ctx, uint64_t *waves, uint64_t *joined, uint64_t *max_inflight);
/* Bytes charged to the HBM budget now (results held by tickets, intermediates in flight,
 * cache entries) and the most charged at once since mp_create. Any pointer may be NULL. */
int mp_budget_stats(mp_ctx *ctx, uint64_t *held, uint64_t *peak);
/* Host wall time in ms from a ticket's submission to its completion (MP_ERR_STATE while
 * it is still pending). */
int mp_result_latency(mp_ctx *ctx, mp_ticket ticket, double *ms);

/* Shape of a finished result (MP_ERR_STATE while pending). Any output pointer may be NULL. */
int mp_result_info(mp_ctx *ctx, mp_ticket ticket, uint32_t *rows, uint32_t *cols, uint64_t *nnz);

/* Copy a result into caller-owned buffers: row_ptr (rows+1), col (nnz), val (nnz).
 * on_device = 0: host pointers (pageable or pinned); 1: device pointers on the
 * context's device. Any of the three may be NULL to skip it. */
int mp_result_copy(mp_ctx *ctx, mp_ticket ticket, int64_t *row_ptr, int32_t *col, uint64_t *val,
                   int on_device);

/* Drop a ticket and its result. */
int mp_release(mp_ctx *ctx, mp_ticket ticket);

/* mp_result_copy without waiting: the copies are queued on the context's copy stream and
 * the call returns at once, so the next query can run while the result travels. The
 * destination buffers must stay valid, and must not be read, until mp_result_copy_wait
 * returns for the ticket (host buffers should be pinned for the copy to overlap); wait
 * before mp_release (a release first still frees the device memory only after the copy,
 * but leaves nothing to wait on). Errors as mp_result_copy. */
int mp_result_copy_async(mp_ctx *ctx, mp_ticket ticket, int64_t *row_ptr, int32_t *col, uint64_t *val,
                         int on_device);
/* Blocks until the ticket's last asynchronous copy has landed (MP_OK at once if none).
 * MP_ERR_NOTFOUND for an unknown or released ticket. */
int mp_result_copy_wait(mp_ctx *ctx, mp_ticket ticket);

/* Device time in milliseconds spent on the ticket's query (products it ran itself). */
int mp_result_time(mp_ctx *ctx, mp_ticket ticket, double *ms);

const char *mp_strerror(int code);

/* ---- autotuning
 *
 * Times the given workload (run `reps` times per candidate, cache bypassed) over a grid of
 * row-bin thresholds -- the smallest row sent to the dense shared-memory bin and the
 * product count above which a row is split over many blocks -- and keeps the fastest. It
 * then runs each query once and fits the Eq. 2 coefficients alpha, beta, gamma to the
 * measured product times by least squares (Sec. 3.2), and keeps the fit (costs then in
 * milliseconds) only if the workload re-timed with it is not slower. Split-row kernel
 * variants are swept too. The result applies to this context at once and, when
 * out_path is not NULL, is written there as JSON for mp_config.tune_file. *best_ms (may
 * be NULL) receives the best candidate's time per run. Results never change. */
int mp_autotune(mp_ctx *ctx, uint32_t n, const mp_query *q, uint32_t reps, const char *out_path,
                double *best_ms);

/* ---- diagnostics */

/* Work counters of a ticket's query: Gustavson scalar products summed over its sparse
 * products, rows per bin class in the symbolic and numeric passes (12 entries each:
 * warp-hash tables of 32..1024 slots, block-hash tables of 2048..8192 slots, dense
 * shared-memory, split rows in global scratch, and rows of at most 16 products taken one
 * per thread) and the number of sparse products it ran. Any output pointer may be NULL. */
int mp_result_stats(mp_ctx *ctx, mp_ticket ticket, uint64_t *products, uint32_t *sym_bins,
                    uint32_t *num_bins, uint32_t *n_products);

/* Cache counters since mp_create (Sec. 3.4): requests (look-ups that found an entry plus
 * insertion attempts), hits, inserts, rejections (80 % rule), evictions, bytes held and
 * entries held. Any pointer may be NULL. MP_ERR_STATE when the policy is MP_POLICY_NONE. */
int mp_cache_stats(mp_ctx *ctx, uint64_t *requests, uint64_t *hits, uint64_t *inserts, uint64_t *rejected,
                   uint64_t *evictions, uint64_t *bytes, uint64_t *entries);

/* CUDA graphs of the shared-memory bin passes since mp_create: graphs captured (one per
 * wave shape: pass, non-empty bins, dense-bin width class) and passes replayed from them.
 * Any pointer may be NULL. Both stay 0 unless the replay is turned on (MP_TUNING=graphs=1;
 * off by default: measured, it brought no gain). */
int mp_graph_stats(mp_ctx *ctx, uint64_t *captures, uint64_t *replays);

/* Host-tier counters since mp_create (mp_config.host_tier_bytes): results stored after a
 * device-cache eviction, results copied back instead of recomputed, entries dropped to make
 * room (least recently used first), bytes and entries held. Any pointer may be NULL.
 * MP_ERR_STATE when there is no cache or no host tier. */
int mp_host_tier_stats(mp_ctx *ctx, uint64_t *stores, uint64_t *loads, uint64_t *drops, uint64_t *bytes,
                       uint64_t *entries);

/* Per-kernel counters of the SpGEMM passes since the last reset: one entry per (pass,
 * bin) kernel that ran, named "sym_<bin>" / "num_<bin>" with <bin> one of w32, w64,
 * w128, w256, w512, w1024 (warp-hash tables), k2048, k4096, k8192 (block-hash tables),
 * dense, global, lane (rows of at most 16 products, one per thread), or pool (the persistent launch that drains the warp-hash and 2048-slot
 * bins when that mode is on; those bins then have no entries of their own). The "global"
 * entries time a whole split-row pass (set-up, product walk and rank kernels); the walk
 * kernels inside it have entries of their own: "walk_sym" (bitmap rows, counting),
 * "walk_num" (bitmap rows, adding counts) and "walk_dense" (rows with a dense count row).
 * "stage_rowwork", "stage_symbin", "stage_globsetup", "stage_rowptr" and "stage_numbin"
 * time the other stages of a wave (row work, symbolic binning, split-row set-up, wave row
 * pointers, numeric binning; several kernels each, host gaps between them included; no
 * bytes). By default only the split-row passes, their walks and the pooled bins are timed
 * (the events cost a few percent of a query); the environment variable MP_TUNING=prof=2,
 * read when the context is made, times every bin kernel and the stages as well, prof=0
 * nothing.
 * ms sums the device time between CUDA events recorded on the launch stream around each
 * launch; bytes sums the algorithmic bytes of the launches (X row pointers, X entries with
 * the two Y row pointers each looks up, one Y column id (and value, in the pass that adds
 * the counts: the numeric pass, or the symbolic pass for split rows with a dense count
 * row) per Gustavson product, 12 bytes per output entry; a walk counts 16 bytes per X
 * entry (its product offset and Y-row start), plus its value when it adds counts, and 8
 * per output count it adds). Up to cap entries are written; *n receives the number
 * written. *launches receives every kernel launch this library made in the process (all
 * kernels, not only the passes). */
typedef struct {
    char name[32];
    uint64_t launches;
    double ms;
    double bytes;
    double products;  /* Gustavson scalar products of the rows the launches processed */
} mp_kernel_stat;
int mp_kernel_stats(mp_ctx *ctx, mp_kernel_stat *out, uint32_t cap, uint32_t *n, uint64_t *launches);
int mp_kernel_stats_reset(mp_ctx *ctx);

/* ---- host-only replay of the Overlap Tree and the cache policies (no GPU needed)
 *
 * The same tree and policy code the engine runs, driven by a caller-given trace. Symbols
 * are node type ids (>= 0). pos_keys gives one constraint description per position of an
 * inserted metapath (NULL or "" = unconstrained); keys of sub-metapaths are the
 * descriptions of their positions, renumbered from 0, as "i:<desc>" joined by '|'. */
typedef struct mp_otree mp_otree;
/* A tree built by the naive insertion (mp_otree_create) or by the construction given
 * (mp_otree_create_ex: MP_OTREE_NAIVE or MP_OTREE_ONLINE, else MP_ERR_ARG). Both give the
 * same tree, frequencies and constraint entries; a tree keeps its construction. */
int mp_otree_create(mp_otree **out);
int mp_otree_create_ex(int32_t construction, mp_otree **out);
void mp_otree_destroy(mp_otree *t);
/* Insert a metapath and all its suffixes (Sec. 3.3.2). */
int mp_otree_insert(mp_otree *t, uint32_t n, const int32_t *types, const char *const *pos_keys);
/* Occurrences of the sub-metapath s (Sec. 3.3.1 f); key NULL = any constraints. */
int mp_otree_frequency(mp_otree *t, uint32_t n, const int32_t *s, const char *key, uint64_t *f);
/* Node count (without the root), leaf count and the Sec. 3.3.3 invariant check. */
int mp_otree_info(mp_otree *t, uint64_t *nodes, uint64_t *leaves, int32_t *invariants_ok);

typedef struct mp_cachesim mp_cachesim;
/* A cache of `capacity` bytes under MP_POLICY_ATRAPOS (Alg. 1), _PGDS or _LRU. */
int mp_cachesim_create(double capacity, int32_t policy, mp_cachesim **out);
void mp_cachesim_destroy(mp_cachesim *c);
/* One request (Alg. 1) of the item (types, key) with tree frequency f, cost and size;
 * *outcome = 0 hit, 1 inserted, 2 rejected (above 80 % of the capacity). */
int mp_cachesim_request(mp_cachesim *c, uint32_t n, const int32_t *types, const char *key, double f,
                        double cost, double size, int32_t *outcome);
/* Current cost and utility h of an item; *present = 0 when it is not cached. */
int mp_cachesim_entry(mp_cachesim *c, uint32_t n, const int32_t *types, const char *key, double *cost,
                      double *utility, int32_t *present);
/* The i-th evicted item id ("t0,t1,...,#key"); *n_total = evictions so far. buf may be
 * NULL to read only the count. */
int mp_cachesim_evicted(mp_cachesim *c, uint32_t i, char *buf, uint32_t cap, uint32_t *n_total);
/* Inflation value L, bytes used and items held. */
int mp_cachesim_state(mp_cachesim *c, double *L, double *used, uint32_t *items);

/* ---- one product row without device allocation
 *
 * The paper has no counterpart: this entry point exists for callers that cannot allocate
 * device memory when they need a result row -- a serving process whose free device
 * memory is already handed to its own pool, a latency-critical loop that cannot take the
 * device synchronisation cudaMalloc/cudaFree may cause, or a runtime that only allows
 * allocation at set-up. It computes one row
 *     c = (x restricted to the nodes in km) * Y * diag(cm)
 * with exact uint64 counts, columns ascending, into buffers the caller owns, and calls no
 * cudaMalloc, cudaFree or allocating library routine. Its working memory is a fixed
 * scratch array compiled into the library (a bitmap and a rank word per 32 columns for
 * up to 16,777,216 output columns, 4 MiB), which every GPU that loads the library holds
 * until the process exits.
 *
 *   device, cuda_stream  GPU ordinal and the cudaStream_t to run on (NULL = default).
 *   x_len, x_ci, x_val    the row x: x_len column ids (int32, device) and uint64 values
 *                         (device, or NULL for all ones).
 *   y_rp, y_ci, y_val     Y in CSR on the device: int64 row pointers, int32 column ids,
 *                         uint64 values or NULL (all ones). y_cols = Y's column count.
 *   km, cm                device bitmaps (bit j of word j/32) over Y's rows and columns,
 *                         or NULL for no mask.
 *   out_cap, out_ci, out_val  caller's device buffers for up to out_cap entries.
 *   out_nnz               host: the row's number of entries.
 * Preconditions: every x_ci entry is a row of Y (0 <= k < rows of Y, so y_rp[k + 1] can be
 * read) and km, when given, has a bit for it; every y_ci entry lies in [0, y_cols).
 * Returns MP_OK; MP_ERR_TOO_LARGE when y_cols exceeds 16,777,216 (nothing runs) or the
 * row has more than out_cap entries (*out_nnz then holds the size needed and the output
 * buffers are untouched); MP_ERR_OVERFLOW for a count above 2^64-1; MP_ERR_ARG for a NULL
 * required pointer, a negative x_ci entry or a y_ci entry outside [0, y_cols) (those ids
 * are checked on the device and never used as indexes); MP_ERR_STATE when cuda_stream is
 * being captured into a CUDA graph; MP_ERR_CUDA when one of its own launches or copies
 * fails (errors left by the caller's earlier work are neither reported nor cleared).
 * The call is synchronous: it waits for its stream twice, so it must not be made while
 * that stream is being captured. The first call on a device looks up the scratch array's
 * device address for that device. All calls share the one scratch array, whose contents
 * the next call overwrites: calls that overlap on the GPU (other threads or streams) race
 * and must be serialised by the caller. */
int mp_row_product_noalloc(int32_t device, void *cuda_stream, uint64_t x_len, const int32_t *x_ci,
                           const uint64_t *x_val, const int64_t *y_rp, const int32_t *y_ci,
                           const uint64_t *y_val, uint32_t y_cols, const uint32_t *km,
                           const uint32_t *cm, uint64_t out_cap, int32_t *out_ci, uint64_t *out_val,
                           uint64_t *out_nnz);

/* The chain planner alone (host only; Sec. 3.1 Eq. 1 with the Eq. 2 cost and E_ac
 * densities of Sec. 3.2). p factors; factor t is dims[t] x dims[t+1] with nnz[t]
 * non-zeros. known_cost / known_rho (p*p, row-major, NaN = unknown, both NULL = none)
 * give sub-chains (i, j) whose cost and density are known. rho_fixed (p*p, NaN = none,
 * or NULL) gives measured result densities (sampled rows) that replace E_ac for those
 * sub-chains while their cost still follows Eq. 2. split (p*p) receives the chosen split k
 * of every sub-chain (-1 for single factors and known sub-chains); cost (p*p, may be NULL)
 * the optimal costs. Ties keep the smallest k. */
int mp_plan_chain(uint32_t p, const double *dims, const double *nnz, double alpha, double beta,
                  double gamma, const double *known_cost, const double *known_rho, const double *rho_fixed,
                  int32_t *split, double *cost);

/* The plan the context's planner (mp_config.planner) makes for one query in the current
 * cache state, without running any product and without touching the Overlap Tree or the
 * cache (an "explain"). For a query of p factors, *p_out = p, split (p*p, row-major)
 * receives the chosen split k of every sub-chain (i, j) (-1 for single factors and known
 * sub-chains) and nnz (p*p) the planner's size estimate of every sub-chain result (exact
 * masked nnz on the diagonal). Either array may be NULL. MP_ERR_ARG when p*p > cap (p_out
 * is still set) or on a NULL ctx, query or p_out; a query's own error otherwise. Blocks
 * like a query run outside the serving loop. */
int mp_plan_query(mp_ctx *ctx, const mp_query *q, uint32_t cap, int32_t *split, double *nnz, uint32_t *p_out);

/* The MNC sketch planner alone (host only). Sec. 3.2 compares E_ac with MNC, which
 * estimates a product's size from count sketches of its operands: per leaf factor t
 * (dims[t] x dims[t+1]) hr[t] holds its row counts (dims[t] entries), hc[t] its column
 * counts (dims[t+1]), her[t] per row the entries whose column holds a single entry, and
 * hec[t] per column the entries whose row holds a single entry (all host arrays, read
 * only). The estimate of X Y: the product count when every row of X or every column of Y
 * holds at most one entry; for two leaves, the entries in single-entry rows of X and
 * single-entry columns of Y counted exactly plus the density map
 * p (1 - prod_t (1 - c[t] r[t] / p)) over the remaining p cells; otherwise the density
 * map over (non-empty rows of X) x (non-empty columns of Y). A product's sketch keeps its
 * left operand's row shape and its right operand's column shape, scaled to the estimate.
 * known_cost / known_nnz (p*p, NaN = unknown, both NULL = none): known sub-chains, which
 * enter with a uniform sketch of their size. split (p*p) receives the splits as in
 * mp_plan_chain; cost and nnz (p*p, may be NULL) the costs (Eq. 1 with the Eq. 2 cost)
 * and the estimated result sizes. MP_ERR_ARG when p is 0 or a required array is NULL.
 * (The engine's MP_PLAN_DP_MNC computes the same sketches and sums on the GPU.) */
int mp_plan_chain_mnc(uint32_t p, const double *dims, const uint32_t *const *hr, const uint32_t *const *hc,
                      const uint32_t *const *her, const uint32_t *const *hec, double alpha, double beta,
                      double gamma, const double *known_cost, const double *known_nnz, int32_t *split,
                      double *cost, double *nnz);

#ifdef __cplusplus
}
#endif
#endif /* MP_H_ */
