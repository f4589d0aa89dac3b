// Internal declarations shared by the engine's translation units (not part of the ABI).
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstddef>
#include <cstdint>
#include <vector>

namespace mp {

// Device view of a CSR matrix. val == nullptr means every stored entry is 1 (a 0/1
// adjacency matrix, Sec. 2 Def. 1); otherwise val holds uint64 path counts.
struct DCsr {
    const int64_t *rp = nullptr;
    const int32_t *ci = nullptr;
    const uint64_t *val = nullptr;
    int64_t nrows = 0, ncols = 0;
};

// Row-bin classes. Warp-hash bins hold one row per warp in a shared-memory table of T
// slots (T = 32 << b); block-hash bins one row per block with T = 2048 << (b - 6);
// DENSE one row per block in a shared-memory array as wide as the output; GLOBAL one
// row per block in a dense accumulator in global scratch.
enum Bin : int {
    B_W32 = 0, B_W64, B_W128, B_W256, B_W512, B_W1024,
    B_K2048, B_K4096, B_K8192,
    B_DENSE, B_GLOBAL, NBINS
};

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
    uint64_t scratch_cap = 4ull << 30;  // bitmap + rank bytes of the GLOBAL bin per round
    // GLOBAL rows with prod_i >= glob_dense * ncols accumulate their counts in a dense u64
    // row (one pass gives both the size and the values); 0 turns the dense rows off
    double glob_dense = 0.5;
    uint64_t dense_scratch_cap = 16ull << 30;  // bytes of dense rows (+ bitmap, rank) per wave
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
    double ms = 0.0, bytes = 0.0;
};
struct Prof {
    bool on = true;
    cudaEvent_t ev[2][NBINS][2] = {};
    KStat k[2][NBINS];
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
    size_t bytes() const { return (size_t)(nrows + 1) * 8 + (size_t)nnz * 12; }
    DCsr view() const { return DCsr{rp, ci, val, nrows, ncols}; }
};

// Stream-ordered device allocation used for results and workspaces.
struct Alloc {
    virtual void *alloc(size_t bytes, cudaStream_t s) = 0;
    virtual void free(void *p, cudaStream_t s) = 0;
    virtual ~Alloc() = default;
};

// ---- masks: bit j of word j >> 5 set = node j passes
void mask_fill(uint32_t *m, int64_t n, bool ones, cudaStream_t s);
void mask_and_range(uint32_t *m, const int32_t *prop, int64_t n, int64_t lo, int64_t hi,
                    cudaStream_t s);
void mask_and_set(uint32_t *m, uint32_t *tmp, const uint32_t *set, int64_t set_len, int64_t n,
                  cudaStream_t s);

// nnz of diag(rm) A diag(cm), added into *out (device). long_rows (A.nrows entries) and
// *n_long (zeroed) are device scratch for rows longer than 8192 entries.
void masked_nnz(const DCsr &A, const uint32_t *rm, const uint32_t *cm, unsigned long long *out,
                uint32_t *long_rows, uint32_t *n_long, cudaStream_t s);

// One product of a wave: C = diag(rm) X diag(km) Y diag(cm) (masks may be nullptr).
struct WaveIn {
    DCsr X, Y;
    const uint32_t *rm = nullptr, *km = nullptr, *cm = nullptr;
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
int spgemm_wave(const std::vector<WaveIn> &in, Alloc &al, const Tuning &tun, cudaStream_t s,
                uint64_t max_result_bytes, std::vector<WaveOut> &out, Prof *prof, bool symbolic_only = false);

// C = diag(rm) A diag(cm) with every value 1 (a length-2 metapath). Returns MP_* code.
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

}  // namespace mp
