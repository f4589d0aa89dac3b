// Internal declarations shared by the engine's translation units (not part of the ABI).
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstddef>
#include <cstdint>
#include <memory>
#include <unordered_map>
#include <utility>
#include <vector>

namespace mp {

// Device view of a CSR matrix. val == nullptr means every stored entry is 1 (a 0/1
// adjacency matrix, Sec. 2 Def. 1); otherwise val holds uint64 path counts.
struct DCsr {
    const int64_t *rp = nullptr;
    const int32_t *ci = nullptr;
    const uint64_t *val = nullptr;
    int64_t nrows = 0, ncols = 0;
    int64_t nnz = 0;
    // rows that may be non-empty, ascending (null: any row may be); a product over this
    // matrix then runs over these rows only
    const int32_t *arows = nullptr;
    int64_t narows = 0;
};

// Row-bin classes. Warp-hash bins hold one row per warp in a shared-memory table of T
// slots (T = 32 << b); block-hash bins one row per block with T = 2048 << (b - 6);
// DENSE one row per block in a shared-memory array as wide as the output; GLOBAL rows are
// split over many blocks (global-memory accumulators); LANE rows (at most LANE_PROD
// Gustavson products) one row per thread, merged by insertion into a short sorted list.
enum Bin : int {
    B_W32 = 0, B_W64, B_W128, B_W256, B_W512, B_W1024,
    B_K2048, B_K4096, B_K8192,
    B_DENSE, B_GLOBAL, B_LANE, NBINS
};
static constexpr int LANE_PROD = 16;
static constexpr int LANE_X = 4;  // ... and at most this many X entries

// Device error bits (OR-ed into one status word per product).
enum : uint32_t {
    ERR_OVERFLOW = 1u,   // a count exceeds 2^64 - 1
    ERR_PROBE = 2u,      // a hash table ran out of slots (bin assignment bug)
    ERR_COUNT = 4u,      // numeric row size differs from the symbolic count
};

struct Tuning {
    int dense_max_cols = 8192;   // DENSE needs ncols * 8 bytes of shared memory
    int dense_min_u = 256;       // ... and a row bound of at least this many entries
    int force_class = -1;        // -1 auto, else MP_BIN_* class
    uint64_t heavy = 65536;      // rows with more Gustavson products go to GLOBAL
    uint64_t warp_prod = 4096;   // rows with more products skip the one-warp bins
    int combine = 1;             // split-row kernel: shared-memory combining of hot outputs
    int short_walk = 0;          // split-row kernel: one thread per X entry on short Y rows
    int seg_walk = 1;            // split-row kernel: one warp per segment on long Y rows
    int lbs = 1;                 // split-row kernel: warp-level product walk (0: block-staged walk)
    int lbs_occ = 6;             // resident blocks per SM of the warp-walk count-adding passes (6 or 4)
    int lane_rows = 1;           // rows of at most LANE_PROD products: one thread per row (0: warp-hash bins)
    int row_lists = 1;           // products over X's row list when it is short (0: over all rows)
    int compact = 1;             // large pattern leaves enter products with their column mask applied (0: off)
    int64_t compact_min = 1 << 20;  // ... when they hold at least this many entries
    int row_lens = 1;            // masked Y-row length arrays for products with X.nnz >= Y.nrows (0: off)
    int64_t ech = 4096;          // X entries per work item of a split row cut by entries
    int ew_max = 64;             // split rows whose masked Y rows hold at most this many entries are cut
                                 // into runs of X entries (-1: always runs of products)
    int dsm_cols = 8192;         // dense split rows this narrow add their counts in a shared-memory row (0: off)
    uint64_t scratch_cap = 4ull << 30;  // bitmap + rank bytes of the GLOBAL bin per round
    // GLOBAL rows with prod_i >= glob_dense * ncols accumulate their counts in a dense u64
    // row (one pass gives both the size and the values); 0 turns the dense rows off
    double glob_dense = 1.0;
    uint64_t dense_scratch_cap = 16ull << 30;  // bytes of dense rows (+ bitmap, rank) per wave
    int glob_occ = 6;  // resident blocks per SM of the count-adding split-row kernels (4 or 6)
    int graphs = 0;    // shared-memory bin passes replayed as CUDA graphs, one per wave shape
    int pool = 1;      // warp-hash and 2048-slot bins in one persistent launch per pass
    int sm_count = 148;
};

struct Stats {
    uint64_t products = 0;       // sum over rows of prod_i (Gustavson scalar products)
    uint64_t nnz = 0;
    uint32_t sym_bins[NBINS] = {};
    uint32_t num_bins[NBINS] = {};
    float ms = 0.f;
};

// Per-kernel counters of the two SpGEMM passes (index [pass][bin], pass 0 = symbolic,
// 1 = numeric): launches, device time from CUDA events around each launch, and the
// algorithmic bytes of the work the launch did (see spgemm.cu for the byte model).
struct KStat {
    uint64_t launches = 0;
    double ms = 0.0, bytes = 0.0, prods = 0.0;
};
struct Prof {
    // 0: no events; 1: the split-row passes, their walk kernels and the pooled bins; 2: also
    // every other bin kernel and the stages of each wave (more events on the stream)
    bool on = true;
    int level = 1;
    bool full() const { return on && level >= 2; }
    cudaEvent_t ev[2][NBINS][2] = {};
    KStat k[2][NBINS];
    // the pooled launch of the warp-hash and 2048-slot bins (Tuning::pool), per pass
    cudaEvent_t pev[2][2] = {};
    KStat pool[2];
    bool pool_ran[2] = {false, false};
    // the split-row product walk kernels alone: [0] symbolic (bitmap rows), [1] numeric,
    // [2] dense rows; events around each launch of a wave (up to WALK_EV per mode)
    static constexpr int WALK_EV = 16;
    cudaEvent_t wev[3][WALK_EV][2] = {};
    int wn[3] = {0, 0, 0};
    bool wmiss[3] = {false, false, false};
    double wlast[3][2] = {};  // pass 0's walk bytes and products of the current wave
    KStat walk[3];
    // the other stages of a wave, each a few kernels (device time between events around
    // them, host gaps included): [0] row work, [1] symbolic binning, [2] split-row set-up,
    // [3] wave row pointers, [4] numeric binning
    static constexpr int NSTAGE = 5;
    cudaEvent_t sev[NSTAGE][2] = {};
    bool srec[NSTAGE] = {};
    KStat stage[NSTAGE];
    bool init();
    void destroy();
};

// Kernel launches made by this library in this process.
extern std::atomic<uint64_t> g_launches;

// An owned device CSR result.
struct Mat {
    int64_t nrows = 0, ncols = 0, nnz = 0;
    int64_t *rp = nullptr;
    int32_t *ci = nullptr;
    uint64_t *val = nullptr;   // nullptr only for base relations
    uint64_t vmax = 1;         // upper bound on the values (1: 0/1 pattern; UINT64_MAX: none known)
    // ascending rows outside which every row is empty (or null), and its owner: a row list is
    // shared by every result that inherits it and freed when the last one goes
    const int32_t *arows = nullptr;
    int64_t narows = 0;
    std::shared_ptr<const int32_t> arows_hold;
    size_t bytes() const { return (size_t)(nrows + 1) * 8 + (size_t)nnz * 12; }
    DCsr view() const { return DCsr{rp, ci, val, nrows, ncols, nnz, arows, narows}; }
};

// Stream-ordered device allocation used for results and workspaces. fail_after (tests):
// after this many more successful allocations every allocation fails (UINT64_MAX = never).
struct Alloc {
    uint64_t fail_after = UINT64_MAX;
    virtual void *alloc(size_t bytes, cudaStream_t s) = 0;
    virtual void free(void *p, cudaStream_t s) = 0;
    virtual ~Alloc() = default;
};

// ---- masks: bit j of word j >> 5 set = node j passes
void mask_fill(uint32_t *m, int64_t n, bool ones, cudaStream_t s);
void fill_iota(int32_t *d, int64_t lo, int64_t n, cudaStream_t s);  // d[t] = lo + t, t < n
void mask_and_range(uint32_t *m, const int32_t *prop, int64_t n, int64_t lo, int64_t hi,
                    cudaStream_t s, bool assign = false);
void mask_and_set(uint32_t *m, uint32_t *tmp, const uint32_t *set, int64_t set_len, int64_t n,
                  cudaStream_t s);

// nnz of diag(rm) A diag(cm), added into *out (device). long_rows (A.nrows entries) and
// *n_long (zeroed) are device scratch for rows longer than 8192 entries.
// The same count when the row mask selects exactly the n listed rows (ascending ids).
void masked_nnz_list(const DCsr &A, const int32_t *rows, int64_t n, const uint32_t *cm, unsigned long long *out,
                     cudaStream_t s);
void masked_nnz(const DCsr &A, const uint32_t *rm, const uint32_t *cm, unsigned long long *out,
                uint32_t *long_rows, uint32_t *n_long, cudaStream_t s);

// One product of a wave: C = diag(rm) X diag(km) Y diag(cm) (masks may be nullptr).
struct WaveIn {
    DCsr X, Y;
    std::shared_ptr<const int32_t> xrows_hold;  // owner of X.arows, passed on to the result
    const uint32_t *rm = nullptr, *km = nullptr, *cm = nullptr;
    uint64_t ymax = 1;  // upper bound on Y's values (Mat::vmax of Y)
};
struct WaveOut {
    int status = 0;  // MP_OK, MP_ERR_OVERFLOW, MP_ERR_TOO_LARGE, ...
    Mat m;           // owned by the caller on success
    uint64_t products = 0;
    uint32_t sym_bins[NBINS] = {};
    uint32_t num_bins[NBINS] = {};
};
// Row sampling for the sampled-density planner: active rows (pass rm, non-empty) of A,
// and a bitmap of the active rows whose SplitMix64(seed, row) draw is below thr.
void active_rows(const DCsr &A, const uint32_t *rm, unsigned long long *out, cudaStream_t s);
void sample_rows(const DCsr &A, const uint32_t *rm, uint64_t seed, uint64_t thr, uint32_t *bm,
                 unsigned long long *count, cudaStream_t s);

// Run independent products together: one launch per bin and pass for the whole wave.
// symbolic_only: stop after the symbolic pass; out[p].m holds only nrows, ncols, nnz.
// Returns MP_OK or a wave-wide error (CUDA, out of memory); per-product errors are in
// out[p].status.
// Persistent state of the wave executor: one workspace laid out for a row and product
// capacity (so its addresses stay put from wave to wave), and the CUDA graphs of the
// shared-memory bin passes captured on it, one per wave shape (pass, set of non-empty bins,
// dense-bin width class, profiling on or off). Growing the workspace drops the graphs.
struct WaveCache {
    char *ws = nullptr;
    int64_t mcap = 0;
    int wcap = 0;
    std::unordered_map<uint64_t, cudaGraphExec_t> graphs;
    uint64_t captures = 0, replays = 0;
    bool broken = false;  // a capture failed: plain launches from then on
    // pinned staging of a wave's uploads (product descriptors, row offsets), so they never
    // wait for the stream (a copy from pageable memory does); reused wave after wave, which
    // synchronise before it is written again
    char *pinned = nullptr;
    size_t pinned_cap = 0;
    void *stage(const void *src, size_t bytes, size_t at);  // copies to pinned + at; null on failure
    // pinned host memory the device writes the host's read-backs into (see Readback)
    char *rb = nullptr;
    static constexpr size_t RB_BYTES = 1 << 20;
    void drop_graphs();
    void clear(Alloc &al, cudaStream_t s);
};

// Device-to-host read-backs of small records (bin tallies, sizes, status flags) that take no
// copy engine: at sync() one kernel writes every queued record into the wave cache's pinned
// host buffer, which the device addresses directly (unified addressing), and once the stream
// is idle the bytes move into their host destinations. The sources must not change on the
// stream between get() and sync(). A cudaMemcpyAsync to the host would queue on the copy
// engine behind whatever result copies other streams have in flight. Without a wave cache, or
// when a record does not fit what is left of the buffer, get() falls back to cudaMemcpyAsync.
class Readback {
  public:
    Readback(WaveCache *wc, cudaStream_t s) : wc_(wc), s_(s) {}
    bool get(void *dst, const void *src, size_t bytes);  // false: a CUDA call failed
    bool sync();                                         // false: the stream reported an error
  private:
    struct Part {
        void *dst;
        const void *src;
        size_t at, bytes;
    };
    WaveCache *wc_;
    cudaStream_t s_;
    std::vector<Part> parts_;
    size_t used_ = 0;
};

// The HBM byte budget as the wave executor sees it: each product's exact result bytes are
// reserved once its size is known and before its arrays are made; MP_ERR_BUDGET fails that
// product alone. A reservation of a product that then fails is returned.
struct Budget {
    virtual int reserve(int64_t bytes) = 0;
    virtual void unreserve(int64_t bytes) = 0;
    virtual ~Budget() = default;
};

int spgemm_wave(const std::vector<WaveIn> &in, Alloc &al, const Tuning &tun, cudaStream_t s,
                uint64_t max_result_bytes, std::vector<WaveOut> &out, Prof *prof, bool symbolic_only = false,
                WaveCache *wc = nullptr, Budget *bud = nullptr);

// C = diag(rm) A diag(cm) with every value 1 (a length-2 metapath). Returns MP_* code.
// B = A diag(m) for a pattern CSR A (rows unchanged, entries in order), into new device
// arrays the caller frees (*rp_out, *ci_out); out->nnz is A's (an upper bound).
int compact_cols(const DCsr &A, const uint32_t *m, Alloc &al, const Tuning &tun, cudaStream_t s, DCsr *out,
                 int64_t **rp_out, int32_t **ci_out);
// Adds the Gustavson products of diag(rm) X diag(km) Y (Y's column mask not applied) into
// the device counter *out (zeroed by the caller).
void raw_products(const DCsr &X, const uint32_t *rm, const uint32_t *km, const int64_t *yrp, const Tuning &tun,
                  cudaStream_t s, unsigned long long *out);
int filter(const DCsr &A, const uint32_t *rm, const uint32_t *cm, Alloc &al,
           const Tuning &tun, cudaStream_t s, Mat *out);

// Exclusive scan of n int64 values into out[0..n] (out[n] = total); in may equal out.
// MP_ERR_NOMEM (nothing launched) when its partial-sum workspace cannot be allocated.
int scan_i64(const int64_t *in, int64_t *out, int64_t n, Alloc &al, cudaStream_t s);

// Eq. 1 / Eq. 2 chain planner (planner.cpp).
struct PlanNode {
    int i, j;     // factor range
    int k;        // split (-1 for a leaf or a known sub-chain)
};
// Fills split[i*p + j]; known_cost / known_rho are p*p arrays, NaN where unknown.
// rho_fixed (p*p, NaN where none, or nullptr): measured result densities of sub-chains.
void plan_chain(int p, const double *dims, const double *nnz, double alpha, double beta,
                double gamma, const double *known_cost, const double *known_rho, const double *rho_fixed,
                int *split, double *cost_out, double *rho_out);

// MNC sketch planner (planner.cpp): Eq. 1 with the Eq. 2 cost, the result size of every
// product estimated from count sketches of its operands (MNC, the estimator Sec. 3.2
// compares E_ac with). Leaves carry exact sketches; a product's sketch keeps its left
// operand's row shape and its right operand's column shape, scaled to the estimate; a
// known sub-chain carries a uniform sketch of its exact size.
struct MncLeaf {     // summary of a leaf's exact sketch (row counts hr, column counts hc)
    double nnz;      // sum of hr
    double nzr, maxr, r2;  // rows with hr > 0, max hr, rows with hr >= 2
    double nzc, maxc, c2;  // the same over columns
};
struct MncPair {     // leaf k and leaf k+1 meeting over the node type at position k+1
    double dot;      // sum_t hc_k[t] hr_k+1[t] (Gustavson products of the leaf product)
    double known;    // sum hec_k hr_k+1 + sum (hc_k - hec_k) her_k+1 (exactly counted part)
    double ls_ext;   // sum_t log(1 - (hc_k - hec_k)[t] (hr_k+1 - her_k+1)[t] / p2), -inf if a
                     // term covers every cell, with p2 = r2_k * c2_k+1 (0 when p2 = 0)
};
// The density-map log-sum a DP level asks for: sum_t log(1 - x w[t]) over the inner type
// of pair `pair`, with w = hc_k hr_k+1 (MNC_W_PAIR), hc_k (MNC_W_COL) or hr_k+1 (MNC_W_ROW).
enum { MNC_W_PAIR = 0, MNC_W_COL = 1, MNC_W_ROW = 2 };
struct MncReq {
    int pair, kind;
    double x;
};
// Device side of the MNC planner (mnc.cu): exact sketches of masked leaf factors, the
// per-pair sums, and the log-sums a DP level asks for.
struct MncLeafIn {
    DCsr A, AT;                   // the factor and its transpose (the reverse relation)
    const uint32_t *rm, *cm;      // masks of its two end positions (nullptr = none)
};
// A leaf's exact sketch on the device (kept across batches by the context's memo).
struct MncSketch {
    Alloc *al = nullptr;
    cudaStream_t s = nullptr;
    uint32_t *hr = nullptr, *hc = nullptr, *her = nullptr, *hec = nullptr;
    unsigned long long raw[8] = {};  // row sum, non-zero, max, >= 2; the same over columns
    MncLeaf stat{};
    size_t bytes = 0;
    ~MncSketch() {
        if (!al) return;
        al->free(hr, s);
        al->free(hc, s);
        al->free(her, s);
        al->free(hec, s);
    }
};
using MncSketchPtr = std::shared_ptr<MncSketch>;

class MncDevice {
  public:
    MncDevice(Alloc &al, cudaStream_t s, int sm_count) : al_(al), s_(s), sms_(sm_count) {}
    ~MncDevice();
    // index of a leaf: with a sketch already built (from an earlier batch), or a new one
    // that prepare() builds
    int leaf(const MncLeafIn &in, MncSketchPtr known = nullptr);
    int pair(int a, int b);          // leaf a's columns meet leaf b's rows
    int prepare();                   // builds sketches and pair sums; one sync. MP_* code
    const MncLeaf &leaf_stat(int i) const { return lstat_[i]; }
    const MncPair &pair_stat(int i) const { return pstat_[i]; }
    MncSketchPtr sketch(int i) const { return leaves_[i].sk; }
    bool built(int i) const { return leaves_[i].build; }
    // ls[r] = sum_t log(1 - x w[t]) for requests whose .pair indexes pairs of this object
    int eval(const std::vector<MncReq> &req, std::vector<double> &ls);
  private:
    struct Leaf {
        MncLeafIn in;
        MncSketchPtr sk;
        bool build = true;
    };
    Alloc &al_;
    cudaStream_t s_;
    int sms_;
    std::vector<Leaf> leaves_;
    std::vector<std::pair<int, int>> pairs_;
    std::vector<MncLeaf> lstat_;
    std::vector<MncPair> pstat_;
    unsigned long long *sum_ = nullptr;  // 8 per leaf: row sum, nz, max, >= 2; column the same
    void *req_ = nullptr;                // device request buffer (and results)
    size_t req_cap_ = 0;
};

class MncPlan {
  public:
    MncPlan(int p, const double *dims, const MncLeaf *leaves, const MncPair *pairs, double alpha, double beta,
            double gamma, const double *known_cost, const double *known_nnz);
    // sub-chains of length len (2..p): first the log-sums they need (appended to out, in
    // an order resolve() expects back), then resolve() with those sums
    void requests(int len, std::vector<MncReq> &out);
    void resolve(int len, const double *ls);
    int p;
    std::vector<int> split;            // p*p, -1 for leaves and known sub-chains
    std::vector<double> cost, nnz;     // p*p
  private:
    struct Sk {
        double nnz;
        int ra, ca;      // row / column anchor leaf, -1 for a uniform sketch
        double fr, fc;   // scale of the anchor's counts (a uniform sketch: the value itself)
        bool exact;
    };
    struct Cand {
        int k;
        int need;        // index into the level's log-sums, -1 when none is needed
        double est_fixed, p3;
        double ls_const; // host log-sum of a uniform-by-uniform product
    };
    std::vector<double> dims_;
    const MncLeaf *leaves_;
    const MncPair *pairs_;
    double alpha_, beta_, gamma_;
    const double *known_cost_, *known_nnz_;
    std::vector<Sk> sk_;
    std::vector<std::vector<Cand>> cand_;  // per sub-chain of the current level
    size_t at(int i, int j) const { return (size_t)i * p + j; }
};

}  // namespace mp
