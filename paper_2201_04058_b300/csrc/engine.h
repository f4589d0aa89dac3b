// The context object behind the opaque mp_ctx handle of include/mp.h.
#pragma once
#include <cuda_runtime.h>

#include <array>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <string>
#include <unordered_map>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/mp.h"
#include "internal.h"
#include "otree.h"

// A device CSR shared by results, cache entries and in-flight products; freed (stream
// ordered) when the last holder lets go. Base relations are never owned. Its bytes stay
// charged to the context's HBM budget (held) while it lives.
struct DevMat {
    mp::Mat m;
    mp::Alloc *al = nullptr;
    cudaStream_t s = nullptr;
    std::atomic<int64_t> *held = nullptr;
    int64_t charged = 0;
    ~DevMat() {
        if (held) held->fetch_sub(charged);
        if (!al) return;
        if (m.rp) al->free(m.rp, s);
        if (m.ci) al->free(m.ci, s);
        if (m.val) al->free(m.val, s);
    }
};
using MatPtr = std::shared_ptr<DevMat>;

// A named NVTX range for the scope (a batch, its planning, each wave, the cache offers, a
// serving batch): visible on a profiler's timeline, free when no tool is attached.
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

struct mp_ctx {
    struct NodeType {
        std::string name;
        uint32_t count;
    };
    struct Prop {
        int32_t type = -1;
        std::string name;
        std::vector<int32_t> host;
        int32_t *dev = nullptr;
    };
    struct Rel {
        int32_t src = -1, dst = -1;
        std::vector<uint32_t> s, d;  // staged edges (forward relations only), dropped at finalize
        std::vector<int64_t> hrp;    // CSR read from a saved HIN (both directions), dropped at finalize
        std::vector<int32_t> hci;
        mp::Mat dev;                 // 0/1 CSR, val == nullptr
    };
    struct Constraint {
        int32_t prop = -1, op = 0;
        int64_t lo = 0, hi = 0;
        std::vector<uint32_t> set;
    };
    struct Query {
        std::vector<int32_t> types, rels;
        std::vector<std::vector<Constraint>> cons;  // per position
        std::vector<std::string> pos_keys;          // canonical constraint text per position
    };
    struct Result {
        int status = 0;
        bool done = true;         // false while queued or running in the serving loop
        MatPtr m;
        double ms = 0.0;
        double latency_ms = 0.0;  // submission to completion, host wall clock
        mp::Stats st;
        uint32_t n_products = 0;
        uint32_t cache_hits = 0;
        cudaEvent_t copy_ev = nullptr;  // recorded after an asynchronous copy's last chunk
    };
    struct CacheCounters {
        uint64_t requests = 0, hits = 0, inserts = 0, rejected = 0, evictions = 0;
    };

    mp_config cfg{};
    cudaStream_t stream = nullptr;
    cudaStream_t copy_stream = nullptr;  // result copies, so they never wait behind a batch
    bool own_stream = false;
    std::mutex mu;       // tickets and results
    std::mutex exec_mu;  // the executor and its state (masks, DAG, Overlap Tree, cache, pool)
    // serving loop (continuous batching)
    struct Pending {
        uint64_t ticket;
        Query q;
        std::chrono::steady_clock::time_point t0;
    };
    std::mutex qmu;
    std::condition_variable qcv;       // with qmu: work arrived or stop requested
    std::condition_variable done_cv;   // with mu: a ticket finished
    std::deque<Pending> queue;
    std::thread server;
    bool serving = false, stop_req = false;
    size_t inflight = 0;          // with qmu: queries admitted by the serving loop, not yet finished
    double inflight_bytes = 0.0;  // with qmu: their planned result bytes
    uint64_t batches = 0, batched_queries = 0;  // admission groups of the serving loop, queries served
    uint64_t serve_waves = 0;         // waves the serving loop ran
    uint64_t serve_joined = 0;        // queries admitted while others were in flight
    uint64_t serve_max_inflight = 0;  // most queries in flight at once
    void serve_loop();
    // nnz of masked base factors already counted: (relation, row key, column key) -> nnz
    std::unordered_map<std::string, double> leaf_memo;
    // MNC sketches of masked base factors already built (same key), least recently used
    // first out above a byte cap
    struct MncMemo {
        mp::MncSketchPtr sk;
        uint64_t seq = 0;
    };
    std::unordered_map<std::string, MncMemo> mnc_memo;
    size_t mnc_memo_bytes = 0;
    uint64_t mnc_memo_seq = 0;
    static constexpr size_t MNC_MEMO_CAP = 4ull << 30;
    // per-product samples (nnz(X), N_op, nnz(Z), ms) for the Eq. 2 fit of mp_autotune
    bool collect_fit = false;
    uint64_t fail_alloc_after = UINT64_MAX;  // test hook: allocations allowed after finalize
    std::vector<std::array<double, 4>> fit_samples;
    std::vector<NodeType> types;
    std::vector<Prop> props;
    std::vector<Rel> rels;
    bool finalized = false;
    std::unordered_map<uint64_t, Result> results;
    uint64_t next_ticket = 1;
    std::unique_ptr<mp::Alloc> alloc;
    mp::Tuning tun;
    mp::Prof prof;
    mp::WaveCache wcache;  // persistent wave workspace and the bin passes' CUDA graphs
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;

    mp::OverlapTree otree;
    std::unique_ptr<mp::CachePolicy> cache;  // null when cfg.policy == MP_POLICY_NONE
    CacheCounters cstats;
    // Second cache tier in pinned host memory (mp_config.host_tier_bytes): a result the
    // device cache evicts is copied down; a later plan may treat it as known at the cost of
    // copying it back, and then loads it instead of recomputing it. The tier is one pinned
    // arena (allocated at the first store) with a first-fit allocator; least recently used
    // entries leave when no free block fits.
    struct HostEntry {
        std::vector<int32_t> types;
        std::string key;
        mp::Mat shape;        // sizes and value bound (its pointers are unused)
        size_t off = 0;       // in the arena: row pointers | column ids | counts
        size_t bytes = 0;
        double c_ms = 0.0, c_ops = 0.0;  // recorded computation time and Eq. 2 cost
        uint64_t seq = 0;
    };
    struct HostTier {
        char *arena = nullptr;
        size_t cap = 0;
        std::map<size_t, size_t> free_blocks;  // offset -> size, coalesced
        std::unordered_map<std::string, HostEntry> items;
        size_t bytes = 0;
        uint64_t seq = 0, stores = 0, loads = 0, drops = 0;
        double h2d_gbs = 0.0;  // measured once when the arena is made
    } htier;
    bool htier_init();  // the pinned arena and the measured copy-back rate
    bool htier_reserve(size_t bytes, size_t *off);  // evicts LRU entries until a block fits
    void htier_release(size_t off, size_t bytes);
    void htier_store(const std::string &id, const MatPtr &m, const std::vector<int32_t> &types,
                     const std::string &key, double c_ms, double c_ops);
    MatPtr htier_load(const std::string &id);        // stream-ordered copy back, no sync
    double htier_cost(const std::string &id) const;  // Eq. 2 units, NaN when absent
    void htier_clear();

    int parse(const mp_query *q, Query &out);
    int build_masks(const Query &q, std::vector<uint32_t *> &masks, std::vector<int32_t *> *rows = nullptr,
                    std::vector<int64_t> *nrows = nullptr,
                    std::vector<std::shared_ptr<const int32_t>> *holds = nullptr);
    void free_masks(std::vector<uint32_t *> &masks);
    void free_row_lists(std::vector<int32_t *> &rows, std::vector<int64_t> &nrows);

    // ---- the executor: a product DAG that queries join as they are admitted (query.cu)
    //
    // A query in flight: its parsed form and masks (shared with the nodes it registered,
    // which may outlive it when later queries reuse them), its plan's root and cache
    // candidate, and the counters of its result.
    struct QState {
        mp_ctx *ctx = nullptr;
        Query q;
        std::vector<uint32_t *> masks;
        // per position whose one constraint is a node-id set: the ids, ascending, on the
        // device (a factor that starts there runs over these rows only), and their count
        std::vector<int32_t *> rows;
        std::vector<int64_t> nrows;
        std::vector<std::shared_ptr<const int32_t>> rows_hold;  // owners of rows (shared with results)
        ~QState();
    };
    struct Flight {
        int64_t id = -1;
        std::shared_ptr<QState> qs;
        int64_t root = -1, candidate = -1;
        std::vector<int64_t> keeps;  // nodes it keeps until it finishes: root, candidates
        int status = MP_OK;
        uint64_t ticket = 0;
        std::chrono::steady_clock::time_point t0;
        double est_bytes = 0.0;  // planned bytes of the results it computes
        Result r;
        bool finished = false;
    };
    // One sub-chain of some query's plan: factors i..j of the registering query
    // (positions i..j+1), split at k; children are node ids (-1 = the base factor).
    struct PNode {
        std::string id;
        std::vector<int32_t> types;
        std::string key;
        int64_t flight = -1;
        std::shared_ptr<QState> qs;
        int i = 0, j = 0, k = 0;
        int64_t left = -1, right = -1;
        MatPtr res;
        bool done = false;
        bool from_cache = false;
        bool from_host = false;   // copied back from the host tier (offered to the cache again)
        bool filter = false;      // length-2 query: diag(M_1) A diag(M_2)
        int consumers = 0;        // parents that have not run yet
        int keepers = 0;          // flights that offer it to the cache when they finish
        int status = MP_OK;
        double ms = 0.0;          // device time of this node's own product
        double subtree_ms = 0.0;  // of every product this node's computation needed
        double c_ops = 0.0;       // Eq. 2 with the product's actual counts
        double rho_est = 0.0;     // planner density estimate (for later queries)
        mp::Stats st;
    };
    struct Exec {
        std::unordered_map<int64_t, PNode> nodes;
        std::unordered_map<std::string, int64_t> by_id;  // sub-chains whose result is on its way or held
        std::map<int64_t, Flight> flights;               // admitted, not yet finished
        int64_t next_node = 0, next_flight = 0;
        double est_bytes = 0.0;                          // planned bytes of the flights
    } ex;
    // Plans the queries and joins their products to the DAG; returns the flight ids (in
    // order). A query that fails before planning gets a flight with its status.
    int admit(std::vector<Query> &qs, const std::vector<uint64_t> &tickets,
              const std::vector<std::chrono::steady_clock::time_point> &t0s, std::vector<int64_t> &ids);
    // One wave: every node whose operands are ready, in one set of launches.
    int run_wave();
    // Flights whose root is done: results, statistics, cache offers; moved to `done`.
    void finish_flights(std::vector<Flight> &done);
    // a node of the DAG; a missing id is a broken invariant of the executor, reported and
    // fatal (never a silently made empty node)
    PNode &node(int64_t id) {
        auto it = ex.nodes.find(id);
        if (it == ex.nodes.end()) {
            fprintf(stderr, "mp: internal error: product node %lld is gone\n", (long long)id);
            abort();
        }
        return it->second;
    }
    void release_node(int64_t id);  // drop a node nobody needs any more
    void abort_nodes(int rc);       // a failed wave: every node not run yet fails with rc
    // results of finished serving flights into their tickets (wakes mp_wait)
    void publish(std::vector<Flight> &done);
    int run_batch(std::vector<Query> &qs, std::vector<Result> &rs);

    // ---- the HBM byte budget (mp_config.hbm_budget_bytes): bytes of results and
    // intermediates alive (held by tickets, cache entries or the DAG); the cache yields
    std::atomic<int64_t> held{0};
    std::atomic<int64_t> held_peak{0};
    void note_held() {
        int64_t h = held.load(), p = held_peak.load();
        while (h > p && !held_peak.compare_exchange_weak(p, h)) {
        }
    }
    int reserve_bytes(int64_t bytes);    // MP_OK (charged) or MP_ERR_BUDGET
    void unreserve_bytes(int64_t bytes);
    bool evict_one();                    // the cache's victim, to make room for work
    // set by mp_plan_query: run_batch plans its first query, keeps the plan here and runs
    // no product (and leaves the Overlap Tree and the cache untouched)
    struct Explain {
        bool on = false;
        int p = 0;
        std::vector<int> split;
        std::vector<double> nnz;
    } explain;
    MatPtr wrap(const mp::Mat &m, bool charged = false);
    void free_mat(mp::Mat &m);
    void release_result(Result &r);
    void cache_clear();
};
