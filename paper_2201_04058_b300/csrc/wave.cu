// Sparse x sparse products of the metapath chain on sm_103a, many products per launch.
//
// One product C = diag(rm) X diag(km) Y diag(cm) is the constrained-adjacency product of
// Sec. 2 (Problem 1 and the M_c * A that follows it) for one split of a chain: X and Y are
// base 0/1 adjacency matrices (Def. 1) or earlier uint64 results, and the masks are the 0/1
// diagonals M of Def. 3 stored as bitmaps. Counts are exact uint64; a count beyond 2^64 - 1
// raises ERR_OVERFLOW instead of wrapping.
//
// A wave is a set of independent products (every ready product of a batch of queries).
// Their rows are concatenated into one row space, so each step below is one launch per
// bin for the whole wave, however many products it holds:
//   1. row work:  prod_i = sum_{k in X_i, km[k]} nnz(Y_k), the Gustavson scalar products of
//                 row i (an upper bound of nnz(C_i)); rows are binned by it;
//   2. symbolic:  exact nnz(C_i) per bin: warp-per-row or block-per-row hash sets in shared
//                 memory, a dense shared-memory bitmap for narrow outputs, or, for heavy
//                 and wide rows, a per-row bitmap in global memory with the row's products
//                 cut into equal work items spread over all SMs;
//   3. scan:      row pointers of the whole wave (warp-shuffle block scans), rebased per
//                 product;
//   4. numeric:   rows re-binned by their exact nnz; accumulate (col -> count) with 64-bit
//                 shared-memory atomics (hash or dense), or straight into the output slots
//                 given by the bitmap ranks; rows leave in ascending column order (bitonic
//                 sort for hash bins, in-order sweeps otherwise).
// Every row's products are enumerated by a group of threads that scans the lengths of the
// Y rows it needs and walks the flattened product list with a stride of the group size,
// so consecutive threads read consecutive entries of a Y row.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include "common.cuh"

namespace mp {

std::atomic<uint64_t> g_launches{0};

bool Prof::init() {
    for (int p = 0; p < 2; p++) {
        for (int b = 0; b < NBINS; b++)
            for (int e = 0; e < 2; e++)
                if (cudaEventCreate(&ev[p][b][e]) != cudaSuccess) return false;
        for (int e = 0; e < 2; e++)
            if (cudaEventCreate(&pev[p][e]) != cudaSuccess) return false;
    }
    for (int m = 0; m < 3; m++)
        for (int k = 0; k < WALK_EV; k++)
            for (int e = 0; e < 2; e++)
                if (cudaEventCreate(&wev[m][k][e]) != cudaSuccess) return false;
    for (int t = 0; t < NSTAGE; t++)
        for (int e = 0; e < 2; e++)
            if (cudaEventCreate(&sev[t][e]) != cudaSuccess) return false;
    return true;
}

void Prof::destroy() {
    for (int p = 0; p < 2; p++) {
        for (int b = 0; b < NBINS; b++)
            for (int e = 0; e < 2; e++)
                if (ev[p][b][e]) cudaEventDestroy(ev[p][b][e]);
        for (int e = 0; e < 2; e++)
            if (pev[p][e]) cudaEventDestroy(pev[p][e]);
    }
    for (int m = 0; m < 3; m++)
        for (int k = 0; k < WALK_EV; k++)
            for (int e = 0; e < 2; e++)
                if (wev[m][k][e]) cudaEventDestroy(wev[m][k][e]);
    for (int t = 0; t < NSTAGE; t++)
        for (int e = 0; e < 2; e++)
            if (sev[t][e]) cudaEventDestroy(sev[t][e]);
}

// One product of a wave, as the kernels see it.
struct Prod {
    DCsr X, Y;
    const uint32_t *rm, *km, *cm;
    int64_t row0;   // first wave row of this product
    // X's rows the product runs over: arows[0..nwr) (ascending) when X comes with a row list
    // much shorter than its row count, else all nwr = X.nrows rows; rows off the list are
    // empty in the result
    const int32_t *arows;
    int64_t nwr;
    int64_t *rp;    // output row pointers (X.nrows + 1)
    int32_t *ci;    // output column ids (after the symbolic pass)
    uint64_t *val;  // output counts
    uint64_t ymax;  // upper bound on Y's values
    // masked Y-row lengths (ml[k] = |Y row k| when km passes k, else 0), made for a product
    // without a row mask whose X has at least as many entries as Y has rows, so the row work
    // gathers one 4-byte word per X entry instead of two row pointers and a mask word; null
    // otherwise
    const uint32_t *ml;
};

// Per-product counters kept on the device.
struct PStat {
    unsigned long long prods;
    long long nnz;
    unsigned long long xsmax;  // bits of the largest row sum of X (a non-negative double)
    uint32_t unsafe;           // some row's sum times ymax reaches 2^63: counts are checked
    uint32_t err;
    uint32_t sym_bins[NBINS];
    uint32_t nerr;  // set by the numeric binning (kept apart from err, which it reads)
    uint32_t num_bins[NBINS];
};

struct BinArgs {
    int dense_max_cols, dense_min_u, force;
    uint64_t heavy, warp_prod;
    double gdense;  // GLOBAL rows with prod_i >= gdense * (their output's width) take a dense row
    int lane;       // rows of at most LANE_PROD products take the one-thread-per-row bin (automatic bins only)
    int ew_max;     // GLOBAL rows whose masked Y rows are all this short are split by X entries (-1: none)
};

__device__ __forceinline__ bool lane_row(const BinArgs &ba, uint64_t prod_i, int64_t xe) {
    return ba.lane && ba.force < 0 && prod_i <= (uint64_t)LANE_PROD && xe <= LANE_X;
}

// A split row whose masked Y rows hold at most ew_max entries each: its work items are
// fixed runs of X entries (each entry's Y row found as it is walked) instead of fixed runs
// of products, so it needs no per-entry product offsets.
__host__ __device__ __forceinline__ bool entry_split(uint32_t ymax_i, int ew_max) {
    return (int64_t)ymax_i <= (int64_t)ew_max;
}
// algorithmic bytes per X entry of a split-row walk: its column id and Y row pointers when
// split by entries, its product offset and Y-row start otherwise
__device__ __forceinline__ unsigned long long walk_xbytes(bool ew) { return ew ? 20ull : 16ull; }

// A GLOBAL row that accumulates in a dense u64 row as wide as its output (ncols): its
// products are at least gdense times that width, so zeroing and scanning the dense row
// costs little next to them.
__device__ __forceinline__ bool glob_dense_row(double gdense, uint64_t prod_i, int64_t ncols) {
    return gdense > 0.0 && (double)prod_i >= gdense * (double)ncols;
}

// Per-bin tallies of one pass over the wave: rows, X entries, Gustavson products, output
// entries and the algorithmic bytes of the bin's kernel.
struct BinTally {
    uint32_t counts[NBINS];
    unsigned long long xent[NBINS], prods[NBINS], outn[NBINS], bytes[NBINS];
    uint32_t gdense;  // GLOBAL rows that qualify for a dense row
    unsigned long long gd_cols, gb_cols;  // widest output among them, and among the other GLOBAL rows
    // the split-row product walks alone ([0] bitmap rows' symbolic, [1] their numeric, [2]
    // dense rows): algorithmic bytes (per X entry its product offset, Y-row start and value
    // when the walk adds counts; per product the Y column id and value; per output entry the
    // count the numeric walk adds) and Gustavson products
    unsigned long long wbytes[3], wprods[3];
    unsigned long long gx_pw;  // X entries of the GLOBAL rows split by products (they need offsets)
};

static constexpr int64_t LONGX = 2048;   // X rows longer than this are summed by whole blocks
static constexpr int64_t LONGCH = 16384; // X entries per block of a long row
// Marks a GLOBAL row with a dense slot between the partition and the numeric binning.
static constexpr int8_t B_GDENSE = 100;

// The X row of wave row g of product P.
__device__ __forceinline__ int64_t xrow(const Prod &P, int64_t g) {
    const int64_t r = g - P.row0;
    return P.arows ? (int64_t)__ldg(P.arows + r) : r;
}

// ------------------------------------------------------------------ row work + bins

// Product of every wave row (binary search over the products' first rows).
__global__ void k_rowprod(const int64_t *row0s, int w, int64_t M, int32_t *rowprod) {
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < M; g += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = w - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(row0s + mid) <= g) lo = mid; else hi = mid - 1;
        }
        rowprod[g] = lo;
    }
}

// Over the X entries p = p0, p0 + st, ... < e of one row: the masked Y-row lengths (the row's
// Gustavson products) into s and the X values (1 for a pattern X) into x. Four entries are
// loaded before their Y row pointers are, so four dependent gathers are in flight.
__device__ __forceinline__ void row_sums(const Prod &P, int64_t p0, int64_t e, int64_t st, uint64_t &s,
                                         double &x, uint32_t &mx) {
    const int32_t *__restrict__ xci = P.X.ci;
    const uint64_t *__restrict__ xv = P.X.val;
    const int64_t *__restrict__ yrp = P.Y.rp;
    const uint32_t *__restrict__ km = P.km;
    int64_t p = p0;
    if (const uint32_t *__restrict__ ml = P.ml) {
        for (; p + 3 * st < e; p += 4 * st) {
            int32_t k[4];
            uint32_t l[4];
#pragma unroll
            for (int u = 0; u < 4; u++) k[u] = __ldg(xci + p + u * st);
#pragma unroll
            for (int u = 0; u < 4; u++) l[u] = __ldg(ml + k[u]);
#pragma unroll
            for (int u = 0; u < 4; u++) {
                s += l[u];
                mx = max(mx, l[u]);
                x += xv ? (double)__ldg(xv + p + u * st) : 1.0;
            }
        }
        for (; p < e; p += st) {
            const uint32_t l = __ldg(ml + __ldg(xci + p));
            s += l;
            mx = max(mx, l);
            x += xv ? (double)__ldg(xv + p) : 1.0;
        }
        return;
    }
    for (; p + 3 * st < e; p += 4 * st) {
        int32_t k[4];
        int64_t y0[4], y1[4];
#pragma unroll
        for (int u = 0; u < 4; u++) k[u] = __ldg(xci + p + u * st);
        // the row pointers regardless of the mask, so they load beside the mask words
#pragma unroll
        for (int u = 0; u < 4; u++) {
            y0[u] = __ldg(yrp + k[u]);
            y1[u] = __ldg(yrp + k[u] + 1);
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int64_t len = bit_of(km, (uint32_t)k[u]) ? y1[u] - y0[u] : 0;
            s += (uint64_t)len;
            mx = max(mx, (uint32_t)len);
            x += xv ? (double)__ldg(xv + p + u * st) : 1.0;
        }
    }
    for (; p < e; p += st) {
        const int32_t k = __ldg(xci + p);
        const int64_t y0 = __ldg(yrp + k), y1 = __ldg(yrp + k + 1);
        const int64_t len = bit_of(km, (uint32_t)k) ? y1 - y0 : 0;
        s += (uint64_t)len;
        mx = max(mx, (uint32_t)len);
        x += xv ? (double)__ldg(xv + p) : 1.0;
    }
}

// ml[k] = masked length of Y row k (0 where the middle mask km drops k), k < n.
__global__ void k_masked_len(const int64_t *__restrict__ yrp, const uint32_t *__restrict__ km, int64_t n,
                             uint32_t *__restrict__ ml) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        ml[k] = bit_of(km, (uint32_t)k) ? (uint32_t)min(__ldg(yrp + k + 1) - __ldg(yrp + k), (int64_t)UINT32_MAX) : 0u;
}

// prod_i of every wave row, with the row's X value sum and its longest masked Y row. Each
// lane takes one of 32 consecutive rows and sums rows of up to 16 entries itself; longer
// rows are queued: up to LONGX entries for k_rowwork_mid (one warp per row), beyond that
// for k_rowwork_long (several blocks per row).
static constexpr int64_t SHORTX = 16;  // X rows up to this long are summed by one lane

__global__ void k_rowwork(const Prod *prods, const int32_t *rowprod, int64_t M, uint64_t *prod, double *xsum,
                          uint32_t *ymx, uint32_t *long_rows, uint32_t *huge_rows, uint32_t *n_long,
                          uint32_t *n_huge, uint32_t *mid_rows, uint32_t *n_mid) {
    const int lane = threadIdx.x & 31;
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t g0 = w * 32; g0 < M; g0 += nwarps * 32) {
        const int64_t g = g0 + lane;
        int64_t b = 0, e = 0;
        const Prod *P = nullptr;
        if (g < M) {
            P = prods + rowprod[g];
            const int64_t i = xrow(*P, g);
            if (bit_of(P->rm, (uint32_t)i)) {
                b = P->X.rp[i];
                e = P->X.rp[i + 1];
            }
        }
        uint64_t s = 0;
        double xs = 0.0;  // the row's sum of X values: x_ik <= xs bounds every product and sum
        uint32_t mx = 0;
        if (e - b <= SHORTX && e > b) row_sums(*P, b, e, 1, s, xs, mx);
        if (e - b > LONGX && e - b <= LONGCH) long_rows[atomicAdd(n_long, 1u)] = (uint32_t)g;  // one block
        if (e - b > LONGCH) huge_rows[atomicAdd(n_huge, 1u)] = (uint32_t)g;                    // several

        const bool mid = e - b > SHORTX && e - b <= LONGX;
        const unsigned mm = __ballot_sync(FULL, mid);
        if (mm) {  // warp-aggregated append to the mid-row queue
            const int leader = __ffs(mm) - 1;
            uint32_t at = 0;
            if (lane == leader) at = atomicAdd(n_mid, (uint32_t)__popc(mm));
            at = __shfl_sync(FULL, at, leader);
            if (mid) mid_rows[at + __popc(mm & ((1u << lane) - 1u))] = (uint32_t)g;
        }
        if (g < M && e - b <= SHORTX) {
            prod[g] = s;
            xsum[g] = xs;
            ymx[g] = mx;
        } else if (g < M && e - b > LONGX) {
            prod[g] = 0;  // k_rowwork_long adds its blocks' sums
            xsum[g] = 0.0;
            ymx[g] = 0;
        }
    }
}

// The queued mid-length rows, one warp each (all warps of the grid in parallel), with four
// dependent gathers in flight per lane.
__global__ void k_rowwork_mid(const Prod *prods, const int32_t *rowprod, uint64_t *prod, double *xsum, uint32_t *ymx,
                              const uint32_t *mid_rows, const uint32_t *n_mid) {
    const int lane = threadIdx.x & 31;
    const uint32_t n = *n_mid;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < n; r += nwarps) {
        const uint32_t g = mid_rows[r];
        const Prod &P = prods[rowprod[g]];
        const int64_t i = xrow(P, g);
        uint64_t s = 0;
        double x = 0.0;
        uint32_t mx = 0;
        row_sums(P, P.X.rp[i] + lane, P.X.rp[i + 1], 32, s, x, mx);
        for (int d = 16; d; d >>= 1) {
            s += __shfl_xor_sync(FULL, s, d);
            x += __shfl_xor_sync(FULL, x, d);
        }
        mx = __reduce_max_sync(FULL, mx);
        if (lane == 0) {
            prod[g] = s;
            xsum[g] = x;
            ymx[g] = mx;
        }
    }
}

// The queued long rows: a row of up to LONGCH entries is summed by one block (the blocks
// take such rows in turn); a longer row is shared by ceil(len / LONGCH) consecutive blocks
// (modulo the grid) starting at a block that depends on the row, so those rows spread over
// the grid and a row only a few chunks long does not make every block stop at it.
__device__ __forceinline__ void block_row_sums(const Prod &P, int64_t p0, int64_t e, int64_t st, uint64_t &s,
                                               double &x, uint32_t &mx, unsigned long long *red, double *redx,
                                               uint32_t *redm) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    s = 0;
    x = 0.0;
    mx = 0;
    row_sums(P, p0, e, st, s, x, mx);
    for (int d = 16; d; d >>= 1) {
        s += __shfl_xor_sync(FULL, s, d);
        x += __shfl_xor_sync(FULL, x, d);
    }
    mx = __reduce_max_sync(FULL, mx);
    if (lane == 0) {
        red[wid] = s;
        redx[wid] = x;
        redm[wid] = mx;
    }
    __syncthreads();
    if (wid == 0) {
        const bool in = lane < (int)(blockDim.x >> 5);
        s = in ? red[lane] : 0;
        x = in ? redx[lane] : 0.0;
        mx = __reduce_max_sync(FULL, in ? redm[lane] : 0u);
        for (int d = 16; d; d >>= 1) {
            s += __shfl_xor_sync(FULL, s, d);
            x += __shfl_xor_sync(FULL, x, d);
        }
    }
    __syncthreads();  // red* are free again; the sums are valid in warp 0
}

__global__ void k_rowwork_long(const Prod *prods, const int32_t *rowprod, uint64_t *prod, double *xsum,
                               uint32_t *ymx, const uint32_t *long_rows, const uint32_t *huge_rows,
                               const uint32_t *n_long, const uint32_t *n_huge) {
    __shared__ unsigned long long red[32];
    __shared__ double redx[32];
    __shared__ uint32_t redm[32];
    const int64_t G = gridDim.x;
    uint64_t s;
    double x;
    uint32_t mx;
    const uint32_t n1 = *n_long;
    for (int64_t r = blockIdx.x; r < n1; r += G) {  // uniform over the block
        const uint32_t g = long_rows[r];
        const Prod &P = prods[rowprod[g]];
        const int64_t i = xrow(P, g);
        block_row_sums(P, P.X.rp[i] + threadIdx.x, P.X.rp[i + 1], (int64_t)blockDim.x, s, x, mx, red, redx, redm);
        if (threadIdx.x == 0) {
            prod[g] = s;
            xsum[g] = x;
            ymx[g] = mx;
        }
    }
    const uint32_t n2 = *n_huge;
    for (uint32_t r = 0; r < n2; r++) {
        const uint32_t g = huge_rows[r];
        const Prod &P = prods[rowprod[g]];
        const int64_t i = xrow(P, g);
        const int64_t b = P.X.rp[i], e = P.X.rp[i + 1];
        const int64_t nb = min(G, (e - b + LONGCH - 1) / LONGCH);
        const int64_t off = (blockIdx.x - ((int64_t)r * 37) % G + G) % G;  // this block's share
        if (off >= nb) continue;  // uniform over the block
        block_row_sums(P, b + off * (int64_t)blockDim.x + threadIdx.x, e, nb * (int64_t)blockDim.x, s, x, mx, red,
                       redx, redm);
        if (threadIdx.x == 0 && s) atomicAdd((unsigned long long *)(prod + g), s);
        if (threadIdx.x == 0 && x > 0.0) atomicAdd(xsum + g, x);
        if (threadIdx.x == 0 && mx) atomicMax(ymx + g, mx);
    }
}

// Adds v into counter[key] once per group of lanes holding the same key (warp-aggregated).
__device__ __forceinline__ void agg_add_u32(uint32_t *counter_base, int key, bool active, uint32_t v) {
    const unsigned peers = __match_any_sync(FULL, active ? key : -1);
    if (!active) return;
    const int leader = __ffs(peers) - 1;
    if ((int)(threadIdx.x & 31) == leader) atomicAdd(counter_base + key, v * (uint32_t)__popc(peers));
}

// Symbolic bin of every wave row from prod_i; rows without products get nnz_i = 0 and no
// bin. Tallies per bin (for the byte model) and per product (products, rows per bin).
__global__ void k_binassign(const Prod *prods, const int32_t *rowprod, const uint64_t *prod, const double *xsum,
                            const uint32_t *ymx, int64_t M, BinArgs ba, int8_t *bin, int64_t *nnz, BinTally *tally,
                            PStat *ps) {
    __shared__ uint32_t hc[NBINS], hd;
    __shared__ unsigned long long hx[NBINS], hp[NBINS], hb[NBINS];
    constexpr int NP = 8;  // products aggregated in shared memory per chunk of rows
    __shared__ unsigned long long sp[NP], sx[NP];
    if (threadIdx.x < NBINS) {
        hc[threadIdx.x] = 0;
        hx[threadIdx.x] = 0;
        hp[threadIdx.x] = 0;
        hb[threadIdx.x] = 0;
    }
    if (threadIdx.x == 0) hd = 0;
    __syncthreads();
    for (int64_t g0 = blockIdx.x * (int64_t)blockDim.x; g0 < M; g0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = g0 + threadIdx.x;
        const int pfirst = rowprod[g0];
        if (threadIdx.x < NP) {
            sp[threadIdx.x] = 0;
            sx[threadIdx.x] = 0;
        }
        __syncthreads();
        int b = -1, pi = 0;
        uint64_t s = 0;
        if (g < M) {
            pi = rowprod[g];
            const Prod &P = prods[pi];
            s = prod[g];
            if (s) {
                const int64_t i = xrow(P, g);
                const unsigned long long xe = (unsigned long long)(P.X.rp[i + 1] - P.X.rp[i]);
                b = lane_row(ba, s, (int64_t)xe) ? B_LANE
                                                 : bin_for(s, s, P.Y.ncols, ba.dense_max_cols, ba.dense_min_u, ba.heavy,
                                                           ba.warp_prod, ba.force);
                atomicAdd(&hc[b], 1u);
                if (b == B_GLOBAL) {
                    // dense-row and bitmap scratch are as wide as the widest output of each kind
                    const bool d = glob_dense_row(ba.gdense, s, P.Y.ncols);
                    if (d) atomicAdd(&hd, 1u);
                    atomicMax(d ? &tally->gd_cols : &tally->gb_cols, (unsigned long long)P.Y.ncols);
                    // the bitmap walk's bytes (a row that takes a dense slot moves them later)
                    const bool ew = entry_split(ymx[g], ba.ew_max);
                    if (!ew) atomicAdd(&tally->gx_pw, xe);
                    atomicAdd(&tally->wbytes[0], xe * walk_xbytes(ew) + (unsigned long long)s * 4ull);
                    atomicAdd(&tally->wprods[0], (unsigned long long)s);
                }
                atomicAdd(&hx[b], xe);
                atomicAdd(&hp[b], (unsigned long long)s);
                // symbolic bytes: X row pointers + nnz write, per X entry its column id and the
                // two Y row pointers, per product one Y column id
                atomicAdd(&hb[b], 24ull + xe * 20ull + (unsigned long long)s * 4ull);
                // a row whose X sum times Y's value bound reaches 2^63 may overflow: its
                // product's counts take the checked (carry-detecting) additions
                const double xs = xsum[g];
                if (xs * (double)P.ymax >= 9223372036854775808.0) atomicOr(&ps[pi].unsafe, 1u);
                const unsigned long long xb = (unsigned long long)__double_as_longlong(xs);
                if (pi - pfirst < NP) {
                    atomicAdd(&sp[pi - pfirst], (unsigned long long)s);
                    atomicMax(&sx[pi - pfirst], xb);
                } else {
                    atomicAdd(&ps[pi].prods, (unsigned long long)s);
                    atomicMax(&ps[pi].xsmax, xb);
                }
            } else {
                nnz[g] = 0;
            }
            bin[g] = (int8_t)b;
        }
        // rows per (product, bin), aggregated over lanes with the same pair
        agg_add_u32(&ps[0].sym_bins[0], pi * (int)(sizeof(PStat) / 4) + b, b >= 0, 1u);
        __syncthreads();
        if (threadIdx.x < NP && sp[threadIdx.x]) {
            atomicAdd(&ps[pfirst + threadIdx.x].prods, sp[threadIdx.x]);
            atomicMax(&ps[pfirst + threadIdx.x].xsmax, sx[threadIdx.x]);
        }
        __syncthreads();
    }
    __syncthreads();
    const int t = threadIdx.x;
    if (t < NBINS && hc[t]) {
        atomicAdd(tally->counts + t, hc[t]);
        atomicAdd(tally->xent + t, hx[t]);
        atomicAdd(tally->prods + t, hp[t]);
        atomicAdd(tally->bytes + t, hb[t]);
    }
    if (t == 0 && hd) atomicAdd(&tally->gdense, hd);
}

// Numeric bins (bin) from the exact row sizes (grp = wave row pointers) and the symbolic
// bins (sbin); rows the symbolic pass put in GLOBAL stay there (their bitmaps give the output
// positions). With ahead set it runs before the outputs are allocated.
__global__ void k_numbin(const Prod *prods, const int32_t *rowprod, const int64_t *grp, const uint64_t *prod,
                         const uint32_t *ymx, int64_t M, BinArgs ba, const int8_t *sbin, int8_t *bin, int ahead,
                         BinTally *tally, PStat *ps) {
    __shared__ uint32_t hc[NBINS];
    __shared__ unsigned long long hx[NBINS], hp[NBINS], ho[NBINS], hb[NBINS];
    if (threadIdx.x < NBINS) {
        hc[threadIdx.x] = 0;
        hx[threadIdx.x] = 0;
        hp[threadIdx.x] = 0;
        ho[threadIdx.x] = 0;
        hb[threadIdx.x] = 0;
    }
    __syncthreads();
    for (int64_t g0 = blockIdx.x * (int64_t)blockDim.x; g0 < M; g0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = g0 + threadIdx.x;
        int b = -1, pi = 0;
        if (g < M) {
            pi = rowprod[g];
            const Prod &P = prods[pi];
            // rows of failed products get no bin: ahead of the output allocation the failures
            // are the ones the earlier passes flagged, after it the products left without outputs
            const bool live = ahead ? ps[pi].err == 0 : P.ci != nullptr;
            const int64_t z = live ? grp[g + 1] - grp[g] : 0;
            const int sb = sbin[g];
            const bool dense = sb == B_GDENSE;
            if (z) {
                if (sb == B_GLOBAL || dense) {
                    b = B_GLOBAL;
                } else if (sb == B_LANE) {
                    b = B_LANE;  // z <= prod_i <= LANE_PROD
                } else {
                    b = bin_for(prod[g], (uint64_t)z, P.Y.ncols, ba.dense_max_cols, ba.dense_min_u, ~0ull, ba.warp_prod,
                                ba.force);
                    if (b == B_GLOBAL) atomicOr(&ps[pi].nerr, ERR_PROBE);  // cannot happen: nnz <= the bound
                }
                const int64_t i = xrow(P, g);
                const unsigned long long xe = (unsigned long long)(P.X.rp[i + 1] - P.X.rp[i]);
                const unsigned long long pr = prod[g];
                atomicAdd(&hc[b], 1u);
                atomicAdd(&hx[b], xe);
                if (!dense) atomicAdd(&hp[b], pr);  // a dense row's products ran in the symbolic pass
                atomicAdd(&ho[b], (unsigned long long)z);
                // numeric bytes: X and C row pointers, per X entry its column id (+ value) and
                // two Y row pointers, per product a Y column id (+ value), per output 12 bytes;
                // a dense row gathered in the symbolic pass only reads its counts and writes
                if (dense)
                    atomicAdd(&hb[b], 16ull + (unsigned long long)z * 20ull);
                else
                    atomicAdd(&hb[b], 32ull + xe * (20ull + (P.X.val ? 8ull : 0ull)) +
                                          pr * (4ull + (P.Y.val ? 8ull : 0ull)) + (unsigned long long)z * 12ull);
                if (b == B_GLOBAL && !dense) {
                    const bool ew = entry_split(ymx[g], ba.ew_max);
                    atomicAdd(&tally->wbytes[1], xe * (walk_xbytes(ew) + (P.X.val ? 8ull : 0ull)) +
                                                     pr * (4ull + (P.Y.val ? 8ull : 0ull)) + (unsigned long long)z * 8ull);
                    atomicAdd(&tally->wprods[1], pr);
                }
            }
            bin[g] = (int8_t)b;
        }
        agg_add_u32(&ps[0].num_bins[0], pi * (int)(sizeof(PStat) / 4) + b, b >= 0, 1u);
    }
    __syncthreads();
    const int t = threadIdx.x;
    if (t < NBINS && hc[t]) {
        atomicAdd(tally->counts + t, hc[t]);
        atomicAdd(tally->xent + t, hx[t]);
        atomicAdd(tally->prods + t, hp[t]);
        atomicAdd(tally->outn + t, ho[t]);
        atomicAdd(tally->bytes + t, hb[t]);
    }
}

// Rows grouped by bin: every block derives the bins' offsets from their counts (block 0
// also stores them, with the total, for the passes and the host); the cursors start at
// zero (the wave's tallies are zeroed when it begins).
__global__ void k_bin_fill(const int8_t *bin, int64_t n, const uint32_t *counts, uint32_t *offsets, uint32_t *cursors,
                           uint32_t *list) {
    __shared__ uint32_t s_off[NBINS];
    const int lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int b = 0; b < NBINS; b++) {
            s_off[b] = t;
            t += counts[b];
        }
        if (blockIdx.x == 0) {
            for (int b = 0; b < NBINS; b++) offsets[b] = s_off[b];
            offsets[NBINS] = t;
        }
    }
    __syncthreads();
    for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x; i0 < n; i0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = i0 + threadIdx.x;
        const int b = i < n ? bin[i] : -1;
        const unsigned peers = __match_any_sync(FULL, b);
        if (b >= 0) {
            const int leader = __ffs(peers) - 1;
            uint32_t base = 0;
            if (lane == leader) base = atomicAdd(cursors + b, (uint32_t)__popc(peers));
            base = __shfl_sync(peers, base, leader);
            const uint32_t rank = __popc(peers & ((1u << lane) - 1u));
            list[s_off[b] + base + rank] = (uint32_t)i;
        }
    }
}

// Per-product row pointers from the wave's: rp_p[i] = grp[row0 + i] - grp[row0], and each
// product's nnz. A product over a row list gets its row pointers from k_rp_expand.
__global__ void k_rebase(const Prod *prods, const int32_t *rowprod, const int64_t *grp, int64_t M, PStat *ps) {
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < M; g += (int64_t)gridDim.x * blockDim.x) {
        const int pi = rowprod[g];
        const Prod &P = prods[pi];
        const int64_t r = g - P.row0;
        const int64_t base = grp[P.row0];
        if (!P.arows) P.rp[r] = grp[g] - base;
        if (r == P.nwr - 1) {
            if (!P.arows) P.rp[r + 1] = grp[g + 1] - base;
            ps[pi].nnz = grp[g + 1] - base;
        }
    }
}

// Row pointers of the products over a row list (one launch for the wave: blockIdx.y is
// the product; the others return at once): row i's entries start where those of the first
// listed row at or after i start (the rows off the list are empty). A list of up to
// RP_SMEM rows is searched in shared memory.
static constexpr int RP_SMEM = 4096;

__global__ void __launch_bounds__(256) k_rp_expand(const Prod *prods, const int64_t *grp) {
    __shared__ int32_t s_rows[RP_SMEM];
    const Prod *P = prods + blockIdx.y;  // prods: the first product of this launch's range
    if (!P->arows) return;  // uniform over the block
    const int64_t n = P->X.nrows, na = P->nwr, row0 = P->row0;
    const int32_t *__restrict__ arows = P->arows;
    const int64_t base = grp[row0];
    const bool shared = na <= RP_SMEM;
    if (shared)
        for (int64_t a = threadIdx.x; a < na; a += blockDim.x) s_rows[a] = arows[a];
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= n; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = na;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            const int64_t v = shared ? (int64_t)s_rows[mid] : (int64_t)__ldg(arows + mid);
            if (v < i) lo = mid + 1; else hi = mid;
        }
        P->rp[i] = grp[row0 + lo] - base;
    }
}

// ------------------------------------------------------------------ shared-memory bins

struct PassArgs {
    const Prod *prods;
    const int32_t *rowprod;
    const uint32_t *list;
    const uint32_t *counts, *offsets;
    int64_t *nnz;    // symbolic: nnz per wave row; numeric: the wave row pointers
    PStat *ps;       // per-product error words live here
    unsigned *pool_head;  // work queue of the pooled pass (zeroed before its launch)
};

// The row a bin entry stands for.
struct RowRef {
    const Prod *P;
    int pi;
    int64_t g, i;
    __device__ __forceinline__ RowRef(const PassArgs &a, uint32_t entry) {
        g = entry;
        pi = a.rowprod[g];
        P = a.prods + pi;
        i = xrow(*P, g);
    }
    __device__ __forceinline__ uint32_t *err(const PassArgs &a) const { return &a.ps[pi].err; }
    // numeric: output offset of the row inside its product and its exact length
    __device__ __forceinline__ int64_t out_off(const PassArgs &a) const { return a.nnz[g] - a.nnz[P->row0]; }
    __device__ __forceinline__ int64_t out_len(const PassArgs &a) const { return a.nnz[g + 1] - a.nnz[g]; }
};

// LANE bin: one thread per row of at most LANE_PROD Gustavson products and LANE_X X
// entries. The thread walks its row's products (X entries passing the middle mask, their
// Y rows' entries passing the column mask) and merges each into a sorted list of distinct
// columns held in shared memory (slot-major, so the threads of a warp never share a bank):
// insertion from the back, adding the count when the column is already there. The symbolic pass stores the
// list's length, the numeric pass writes the list (already in column order).
static constexpr int LANE_NT = 128;  // threads per block of the LANE bin

template <bool NUM>
__global__ void __launch_bounds__(LANE_NT) k_lane_rows(PassArgs a, int bin) {
    __shared__ uint32_t s_key[LANE_PROD * LANE_NT];
    __shared__ unsigned long long s_val[NUM ? LANE_PROD * LANE_NT : 1];
    const uint32_t cnt = a.counts[bin], base = a.offsets[bin];
    const int tid = threadIdx.x;
    uint32_t *key = s_key + tid;
    unsigned long long *val = s_val + (NUM ? tid : 0);
    for (uint32_t r = blockIdx.x * LANE_NT + tid; r < cnt; r += gridDim.x * LANE_NT) {
        const RowRef R(a, a.list[base + r]);
        const Prod *P = R.P;
        uint32_t *err = R.err(a);
        const int32_t *__restrict__ yci = P->Y.ci;
        const uint64_t *__restrict__ yv = P->Y.val;
        const uint32_t *__restrict__ cm = P->cm;
        const int64_t xb = P->X.rp[R.i];
        const int nx = (int)min((int64_t)LANE_X, P->X.rp[R.i + 1] - xb);  // the bin holds rows of <= LANE_X
        // every entry's column, then every entry's Y row bounds: independent loads in flight
        uint32_t kk[LANE_X];
        int64_t y0[LANE_X], y1[LANE_X];
#pragma unroll
        for (int u = 0; u < LANE_X; u++) kk[u] = u < nx ? (uint32_t)__ldg(P->X.ci + xb + u) : 0u;
#pragma unroll
        for (int u = 0; u < LANE_X; u++) {
            y0[u] = y1[u] = 0;
            if (u < nx) {
                y0[u] = __ldg(P->Y.rp + kk[u]);
                y1[u] = __ldg(P->Y.rp + kk[u] + 1);
            }
        }
        int n = 0;
        auto insert = [&](uint32_t j, unsigned long long v) {
            int s = n - 1;  // the list is sorted: find j's place from the back
            while (s >= 0 && key[s * LANE_NT] > j) s--;
            if (s >= 0 && key[s * LANE_NT] == j) {
                if (NUM) {
                    const unsigned long long o = val[s * LANE_NT];
                    if (o + v < o) atomicOr(err, ERR_OVERFLOW);
                    val[s * LANE_NT] = o + v;
                }
                return;
            }
            if (n == LANE_PROD) {  // more products than the row work counted
                atomicOr(err, ERR_PROBE);
                return;
            }
            for (int t = n - 1; t > s; t--) {
                key[(t + 1) * LANE_NT] = key[t * LANE_NT];
                if (NUM) val[(t + 1) * LANE_NT] = val[t * LANE_NT];
            }
            key[(s + 1) * LANE_NT] = j;
            if (NUM) val[(s + 1) * LANE_NT] = v;
            n++;
        };
#pragma unroll
        for (int u = 0; u < LANE_X; u++) {
            if (u >= nx || !bit_of(P->km, kk[u])) continue;
            const uint64_t av = NUM && P->X.val ? __ldg(P->X.val + xb + u) : 1ull;
            for (int64_t q0 = y0[u]; q0 < y1[u]; q0 += 4) {  // four column loads in flight
                const int m = (int)min((int64_t)4, y1[u] - q0);
                uint32_t jj[4];
                uint64_t bv[4];
#pragma unroll
                for (int c = 0; c < 4; c++) {
                    jj[c] = c < m ? (uint32_t)__ldg(yci + q0 + c) : 0u;
                    bv[c] = NUM && yv && c < m ? __ldg(yv + q0 + c) : 1ull;
                }
#pragma unroll
                for (int c = 0; c < 4; c++) {
                    if (c >= m || !bit_of(cm, jj[c])) continue;
                    unsigned long long v = 1;
                    if (NUM) {
                        v = av * bv[c];
                        if (__umul64hi(av, bv[c])) atomicOr(err, ERR_OVERFLOW);
                    }
                    insert(jj[c], v);
                }
            }
        }
        if (!NUM) {
            a.nnz[R.g] = n;
        } else {
            const int64_t o = R.out_off(a), len = R.out_len(a);
            if (len != n) atomicOr(err, ERR_COUNT);
            const int m = (int)min((int64_t)n, len);
            for (int s = 0; s < m; s++) {
                P->ci[o + s] = (int32_t)key[s * LANE_NT];
                P->val[o + s] = val[s * LANE_NT];
            }
        }
    }
}

// One row of each shared-memory bin. The per-bin kernels below loop over their bin's rows
// with these; the pooled pass (k_bins_pool) calls them for the tiles it takes from a queue.

// Warp-hash symbolic: one warp counts the distinct columns of a row in a T-slot set.
template <int T>
__device__ __forceinline__ void sym_warp_row(const PassArgs &a, uint32_t entry, Stage *sg, uint32_t *keys, int lane) {
    const RowRef R(a, entry);
    const Prod P = *R.P;
    for (int s = lane; s < T; s += 32) keys[s] = EMPTY;
    __syncwarp();
    int c = 0;
    uint32_t *err = R.err(a);
    for_each_product<32, false>(P.X, P.Y, P.km, P.cm, P.X.rp[R.i], P.X.rp[R.i + 1], sg, nullptr, nullptr, lane, err,
                                [&](uint32_t j, uint64_t) { c += hset_insert(keys, T - 1, j, err); });
    for (int d = 16; d; d >>= 1) c += __shfl_xor_sync(FULL, c, d);
    if (lane == 0) a.nnz[R.g] = c;
    __syncwarp();
}

template <int T, int W>
__global__ void __launch_bounds__(W * 32) k_sym_warp(PassArgs a, int bin) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    Stage *sg = (Stage *)smem + wid * 32;
    uint32_t *keys = (uint32_t *)((Stage *)smem + W * 32) + wid * T;
    const uint32_t cnt = a.counts[bin], base = a.offsets[bin];
    for (uint32_t r = blockIdx.x * W + wid; r < cnt; r += gridDim.x * W) sym_warp_row<T>(a, a.list[base + r], sg, keys, lane);
}

// Warp-hash numeric: one warp sums a row's counts in a T-slot map, then compacts and sorts it.
template <int T>
__device__ __forceinline__ void num_warp_row(const PassArgs &a, uint32_t entry, Stage *sg, unsigned long long *vals,
                                             uint32_t *keys, int lane) {
    const RowRef R(a, entry);
    const Prod P = *R.P;
    uint32_t *err = R.err(a);
    for (int s = lane; s < T; s += 32) {
        keys[s] = EMPTY;
        vals[s] = 0;
    }
    __syncwarp();
    for_each_product<32, true>(P.X, P.Y, P.km, P.cm, P.X.rp[R.i], P.X.rp[R.i + 1], sg, nullptr, nullptr, lane, err,
                               [&](uint32_t j, uint64_t v) { hmap_add(keys, vals, T - 1, j, v, err); });
    __syncwarp();
    // compact occupied slots to the front (in place: writes never pass the read point)
    int n = 0;
    for (int s0 = 0; s0 < T; s0 += 32) {
        const uint32_t k = keys[s0 + lane];
        const unsigned long long v = vals[s0 + lane];
        const unsigned bal = __ballot_sync(FULL, k != EMPTY);
        const int pos = n + __popc(bal & ((1u << lane) - 1u));
        __syncwarp();
        if (k != EMPTY) {
            keys[pos] = k;
            vals[pos] = v;
        }
        n += __popc(bal);
        __syncwarp();
    }
    int Pn = 1;
    while (Pn < n) Pn <<= 1;
    for (int s = n + lane; s < Pn; s += 32) keys[s] = EMPTY;
    __syncwarp();
    bitonic<32>(keys, vals, Pn, lane);
    const int64_t o = R.out_off(a), len = R.out_len(a);
    if (lane == 0 && len != n) atomicOr(err, ERR_COUNT);
    const int m = (int)min((int64_t)n, len);
    for (int s = lane; s < m; s += 32) {
        P.ci[o + s] = (int32_t)keys[s];
        P.val[o + s] = vals[s];
    }
    __syncwarp();
}

template <int T, int W>
__global__ void __launch_bounds__(W * 32) k_num_warp(PassArgs a, int bin) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    Stage *sg = (Stage *)smem + wid * 32;
    unsigned long long *vals = (unsigned long long *)((Stage *)smem + W * 32) + wid * T;
    uint32_t *keys = (uint32_t *)((unsigned long long *)((Stage *)smem + W * 32) + W * T) + wid * T;
    const uint32_t cnt = a.counts[bin], base = a.offsets[bin];
    for (uint32_t r = blockIdx.x * W + wid; r < cnt; r += gridDim.x * W)
        num_warp_row<T>(a, a.list[base + r], sg, vals, keys, lane);
}

// Block-hash symbolic: one block counts the distinct columns of a row in a T-slot set.
template <int T, int NT>
__device__ __forceinline__ void sym_block_row(const PassArgs &a, uint32_t entry, Stage *sg, uint32_t *keys,
                                              int64_t *warp_sums, int64_t *gtot, int *cnt_s) {
    const RowRef R(a, entry);
    const Prod P = *R.P;
    uint32_t *err = R.err(a);
    for (int s = threadIdx.x; s < T; s += NT) keys[s] = EMPTY;
    if (threadIdx.x == 0) *cnt_s = 0;
    __syncthreads();
    int c = 0;
    for_each_product<NT, false>(P.X, P.Y, P.km, P.cm, P.X.rp[R.i], P.X.rp[R.i + 1], sg, gtot, warp_sums, threadIdx.x,
                                err, [&](uint32_t j, uint64_t) { c += hset_insert(keys, T - 1, j, err); });
    for (int d = 16; d; d >>= 1) c += __shfl_xor_sync(FULL, c, d);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(cnt_s, c);
    __syncthreads();
    if (threadIdx.x == 0) a.nnz[R.g] = *cnt_s;
    __syncthreads();
}

template <int T, int NT>
__global__ void __launch_bounds__(NT) k_sym_block(PassArgs a, int bin) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int64_t warp_sums[32];
    __shared__ int64_t gtot;
    __shared__ int cnt_s;
    Stage *sg = (Stage *)smem;
    uint32_t *keys = (uint32_t *)(sg + NT);
    const uint32_t cnt = a.counts[bin], base = a.offsets[bin];
    for (uint32_t r = blockIdx.x; r < cnt; r += gridDim.x)
        sym_block_row<T, NT>(a, a.list[base + r], sg, keys, warp_sums, &gtot, &cnt_s);
}

// Block-hash numeric: one block sums a row's counts in a T-slot map, compacts and sorts it.
template <int T, int NT>
__device__ __forceinline__ void num_block_row(const PassArgs &a, uint32_t entry, Stage *sg, unsigned long long *vals,
                                              uint32_t *keys, int64_t *warp_sums, int64_t *gtot) {
    constexpr int PER = T / NT;  // slots per thread in the compaction
    const RowRef R(a, entry);
    const Prod P = *R.P;
    uint32_t *err = R.err(a);
    for (int s = threadIdx.x; s < T; s += NT) {
        keys[s] = EMPTY;
        vals[s] = 0;
    }
    __syncthreads();
    for_each_product<NT, true>(P.X, P.Y, P.km, P.cm, P.X.rp[R.i], P.X.rp[R.i + 1], sg, gtot, warp_sums,
                               threadIdx.x, err,
                               [&](uint32_t j, uint64_t v) { hmap_add(keys, vals, T - 1, j, v, err); });
    __syncthreads();
    uint32_t k[PER];
    unsigned long long v[PER];
    int c = 0;
#pragma unroll
    for (int u = 0; u < PER; u++) {
        k[u] = keys[threadIdx.x * PER + u];
        v[u] = vals[threadIdx.x * PER + u];
        c += k[u] != EMPTY;
    }
    int64_t pos = block_excl_scan<NT>(c, warp_sums, gtot);
    const int n = (int)*gtot;
#pragma unroll
    for (int u = 0; u < PER; u++)
        if (k[u] != EMPTY) {
            keys[pos] = k[u];
            vals[pos] = v[u];
            pos++;
        }
    int Pn = 1;
    while (Pn < n) Pn <<= 1;
    __syncthreads();
    for (int s = n + threadIdx.x; s < Pn; s += NT) keys[s] = EMPTY;
    __syncthreads();
    bitonic<NT>(keys, vals, Pn, threadIdx.x);
    const int64_t o = R.out_off(a), len = R.out_len(a);
    if (threadIdx.x == 0 && len != n) atomicOr(err, ERR_COUNT);
    const int m = (int)min((int64_t)n, len);
    for (int s = threadIdx.x; s < m; s += NT) {
        P.ci[o + s] = (int32_t)keys[s];
        P.val[o + s] = vals[s];
    }
    __syncthreads();
}

template <int T, int NT>
__global__ void __launch_bounds__(NT) k_num_block(PassArgs a, int bin) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int64_t warp_sums[32];
    __shared__ int64_t gtot;
    Stage *sg = (Stage *)smem;
    unsigned long long *vals = (unsigned long long *)(sg + NT);
    uint32_t *keys = (uint32_t *)(vals + T);
    const uint32_t cnt = a.counts[bin], base = a.offsets[bin];
    for (uint32_t r = blockIdx.x; r < cnt; r += gridDim.x)
        num_block_row<T, NT>(a, a.list[base + r], sg, vals, keys, warp_sums, &gtot);
}

template <int NT>
__global__ void __launch_bounds__(NT) k_sym_dense(PassArgs a, int bin) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int64_t warp_sums[32];
    __shared__ int64_t gtot;
    __shared__ int cnt_s;
    Stage *sg = (Stage *)smem;
    uint32_t *bm = (uint32_t *)(sg + NT);
    const uint32_t cnt = a.counts[bin], base = a.offsets[bin];
    for (uint32_t r = blockIdx.x; r < cnt; r += gridDim.x) {
        const RowRef R(a, a.list[base + r]);
        const Prod P = *R.P;
        uint32_t *err = R.err(a);
        const int nw = (int)((P.Y.ncols + 31) >> 5);
        for (int s = threadIdx.x; s < nw; s += NT) bm[s] = 0;
        if (threadIdx.x == 0) cnt_s = 0;
        __syncthreads();
        int c = 0;
        for_each_product<NT, false>(P.X, P.Y, P.km, P.cm, P.X.rp[R.i], P.X.rp[R.i + 1], sg, &gtot, warp_sums,
                                    threadIdx.x, err, [&](uint32_t j, uint64_t) {
                                        const uint32_t m = 1u << (j & 31);
                                        c += (atomicOr(bm + (j >> 5), m) & m) == 0;
                                    });
        for (int d = 16; d; d >>= 1) c += __shfl_xor_sync(FULL, c, d);
        if ((threadIdx.x & 31) == 0 && c) atomicAdd(&cnt_s, c);
        __syncthreads();
        if (threadIdx.x == 0) a.nnz[R.g] = cnt_s;
        __syncthreads();
    }
}

template <int NT>
__global__ void __launch_bounds__(NT) k_num_dense(PassArgs a, int bin) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int64_t warp_sums[32];
    __shared__ int64_t gtot;
    Stage *sg = (Stage *)smem;
    unsigned long long *acc = (unsigned long long *)(sg + NT);
    const uint32_t cnt = a.counts[bin], base = a.offsets[bin];
    for (uint32_t r = blockIdx.x; r < cnt; r += gridDim.x) {
        const RowRef R(a, a.list[base + r]);
        const Prod P = *R.P;
        uint32_t *err = R.err(a);
        const int ncols = (int)P.Y.ncols;
        const int per = (ncols + NT - 1) / NT;
        for (int s = threadIdx.x; s < ncols; s += NT) acc[s] = 0;
        __syncthreads();
        for_each_product<NT, true>(P.X, P.Y, P.km, P.cm, P.X.rp[R.i], P.X.rp[R.i + 1], sg, &gtot, warp_sums,
                                   threadIdx.x, err, [&](uint32_t j, uint64_t v) {
                                       const unsigned long long old = atomicAdd(acc + j, (unsigned long long)v);
                                       if (old + v < old) atomicOr(err, ERR_OVERFLOW);
                                   });
        __syncthreads();
        // in-order sweep: thread t owns columns [t*per, t*per + per)
        const int c0 = threadIdx.x * per;
        const int c1 = min(ncols, c0 + per);
        int c = 0;
        for (int s = c0; s < c1; s++) c += acc[s] != 0;
        int64_t pos = block_excl_scan<NT>(c, warp_sums, &gtot);
        const int64_t o = R.out_off(a), len = R.out_len(a);
        if (threadIdx.x == 0 && len != gtot) atomicOr(err, ERR_COUNT);
        for (int s = c0; s < c1; s++) {
            const unsigned long long v = acc[s];
            if (v) {
                if (pos < len) {
                    P.ci[o + pos] = s;
                    P.val[o + pos] = v;
                }
                pos++;
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ pooled shared-memory pass

// One persistent launch for the warp-hash bins and the 2048-slot block-hash bin of a pass:
// its blocks (256 threads, as many as fit on the SMs) take tiles from a device queue --
// largest tables first -- until every row of those bins is done: a block-hash tile is one
// row for the whole block, a warp-hash tile one row per warp (8 warps, or 4 for the 512-
// and 1024-slot tables, whose shared memory then stays at the size of the per-bin kernel).
// It replaces up to seven launches per pass and lets the bins' rows share the SMs instead
// of running one bin after the other. The bins' row counts are read on the device, so one
// launch shape serves every wave (and a captured graph of it every replay).
static constexpr int POOL_BINS = 7;
__constant__ int8_t c_pool_order[POOL_BINS] = {B_K2048, B_W1024, B_W512, B_W256, B_W128, B_W64, B_W32};

__host__ __device__ __forceinline__ bool pool_bin(int b) { return b <= B_K2048; }
__host__ __device__ __forceinline__ int pool_warps(int b) { return b >= B_W512 ? 4 : 8; }
__host__ __device__ __forceinline__ int pool_rows_per_tile(int b) { return b == B_K2048 ? 1 : pool_warps(b); }
// shared memory a bin needs in the pooled kernel
__host__ __device__ __forceinline__ size_t pool_smem(int b, bool numeric) {
    const size_t stage = sizeof(Stage);
    if (b == B_K2048) return 256 * stage + (size_t)2048 * (numeric ? 12 : 4);
    const size_t T = (size_t)32 << b, W = (size_t)pool_warps(b);
    return W * 32 * stage + W * T * (numeric ? 12 : 4);
}

template <bool NUM>
__global__ void __launch_bounds__(256) k_bins_pool(PassArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int64_t warp_sums[32];
    __shared__ int64_t gtot;
    __shared__ int cnt_s;
    __shared__ uint32_t s_start[POOL_BINS + 1];
    __shared__ uint32_t s_tile;
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        uint32_t acc = 0;
        for (int k = 0; k < POOL_BINS; k++) {
            s_start[k] = acc;
            const int b = c_pool_order[k];
            const uint32_t rpt = (uint32_t)pool_rows_per_tile(b);
            acc += (a.counts[b] + rpt - 1) / rpt;
        }
        s_start[POOL_BINS] = acc;
    }
    __syncthreads();
    const uint32_t total = s_start[POOL_BINS];
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(a.pool_head, 1u);
        __syncthreads();
        const uint32_t t = s_tile;
        __syncthreads();  // every thread has the tile before thread 0 takes the next
        if (t >= total) break;
        int k = 0;
        while (t >= s_start[k + 1]) k++;
        const int b = c_pool_order[k];
        const uint32_t lt = t - s_start[k];
        const uint32_t cnt = a.counts[b], base = a.offsets[b];
        if (b == B_K2048) {
            Stage *sg = (Stage *)smem;
            if (!NUM) {
                sym_block_row<2048, 256>(a, a.list[base + lt], sg, (uint32_t *)(sg + 256), warp_sums, &gtot, &cnt_s);
            } else {
                unsigned long long *vals = (unsigned long long *)(sg + 256);
                num_block_row<2048, 256>(a, a.list[base + lt], sg, vals, (uint32_t *)(vals + 2048), warp_sums, &gtot);
            }
        } else {
            const int W = pool_warps(b);
            const uint32_t r = lt * (uint32_t)W + (uint32_t)wid;
            if (wid < W && r < cnt) {
                Stage *sg = (Stage *)smem + wid * 32;
                unsigned char *tab = (unsigned char *)((Stage *)smem + W * 32);
                switch (b) {
#define POOL_WARP(BIN, T)                                                                                   \
    case BIN:                                                                                               \
        if (!NUM)                                                                                           \
            sym_warp_row<T>(a, a.list[base + r], sg, (uint32_t *)tab + wid * T, lane);                       \
        else                                                                                                \
            num_warp_row<T>(a, a.list[base + r], sg, (unsigned long long *)tab + wid * T,                    \
                            (uint32_t *)((unsigned long long *)tab + W * T) + wid * T, lane);               \
        break;
                    POOL_WARP(B_W32, 32)
                    POOL_WARP(B_W64, 64)
                    POOL_WARP(B_W128, 128)
                    POOL_WARP(B_W256, 256)
                    POOL_WARP(B_W512, 512)
                    POOL_WARP(B_W1024, 1024)
#undef POOL_WARP
                    default:
                        break;
                }
            }
        }
        __syncthreads();  // the tables are reused by the next tile
    }
}

// ------------------------------------------------------------------ GLOBAL bin: split rows

// Heavy rows and rows too wide for a shared-memory table. Each row's Gustavson products,
// in the order of its X entries, are cut into work items of PCH products, and the items
// of all rows are spread over all blocks, so a few huge rows (or one hub Y row) still
// fill the GPU:
//   symbolic: every product sets bit j of the row's bitmap (1 bit per output column);
//             a rank pass turns the bitmap into rank[w] = set bits before word w, and the
//             row's nnz is the total;
//   numeric:  a fill pass writes each set bit's column id at its rank (so the row comes
//             out in ascending column order) and zeroes the value; then every product
//             adds its count straight into the output slot rank[w] + popc(bits below j).
// A bitmap word and its rank sit side by side (8 bytes per 32 output columns per row, slots
// of the widest product's size), so the numeric pass finds a slot with one load; rows are
// processed in rounds that fit the scratch cap (one round keeps the symbolic bitmaps for
// the numeric pass, several rounds rebuild them).
// Rows with at least glob_dense times as many products as the widest output instead add
// their counts into a dense u64 row in the symbolic pass; a scan of the dense row then
// gives the bitmap, the rank pass the size, and the numeric pass only copies the counts.
// Counts are added without carry checks (fire-and-forget atomics) when the product's row
// sums of X times the bound on Y's values stay below 2^63; otherwise every addition checks
// its carry and an overflow fails the product.
static constexpr int64_t PCH = 16384;  // Gustavson products per work item
// X entries per work item of a row split by entries (Tuning::ech, a multiple of 256): the
// grid works on about its block count of consecutive items at a time, so smaller items keep
// fewer rows' accumulators in use at once
static constexpr int GNT = 256;        // threads per GLOBAL block
static constexpr int RW = 8;           // bitmap words per thread in the rank pass
static constexpr int CSLOT = 1024;     // shared-memory combining slots per work item
static constexpr int SEG = 256;        // products per warp segment in the segment walk
static constexpr int SEGMIN = 32;      // mean products per staged X entry for the segment walk

struct GlobArgs {
    const uint32_t *list;     // wave rows of the GLOBAL bin, in symbolic order
    const int64_t *item_off;  // R+1 work-item offsets
    const int64_t *xbase;     // R+1 offsets of each row's X entries in xoff
    const int64_t *xoff;      // per X entry of a GLOBAL row: global product offset
    const int64_t *ys;        // per X entry of a GLOBAL row: its Y row's start
    const uint64_t *prod;     // prod_i per wave row
    const uint32_t *ymx;      // per wave row: its longest masked Y row (entry_split)
    int ew_max;
    int64_t ech;              // X entries per work item of a row split by entries
    int64_t items_ub;         // at least the pass's work items (no more blocks than this)
    int64_t r0, r1;           // rows of this round
    uint2 *bmr;               // (r1 - r0) slots of nw {bitmap word, rank} pairs
    int64_t nw;               // slot size (words)
    int short_walk;           // walk chunks of short Y rows one X entry per thread
    int seg_walk;             // walk chunks of long Y rows one warp per segment
    unsigned long long *dval; // dense rows: (r1 - r0) slots of dcols counts each
    int64_t dcols;
};

// Dense-row GLOBAL rows first: the rows that qualify go to the front of dst (in any order),
// the others to the back. cnt (two counters) starts at zero. The first nd front rows take
// dense slots: their bin is marked B_GDENSE until the numeric binning, and the symbolic
// pass's byte tally gains the X and Y values they read there.
__global__ void k_glob_split(const Prod *prods, const int32_t *rowprod, const uint32_t *src, int64_t R,
                             const uint64_t *prod, const uint32_t *ymx, int ew_max, double gdense, int64_t nd,
                             uint32_t *dst, uint32_t *cnt, int8_t *bin, BinTally *tally) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < R; r += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t gr = src[r];
        if (!glob_dense_row(gdense, prod[gr], prods[rowprod[gr]].Y.ncols)) {
            dst[R - 1 - atomicAdd(cnt + 1, 1u)] = gr;
            continue;
        }
        const uint32_t pos = atomicAdd(cnt, 1u);
        dst[pos] = gr;
        if ((int64_t)pos < nd) {
            bin[gr] = B_GDENSE;
            const Prod &P = prods[rowprod[gr]];
            const int64_t i = xrow(P, gr);
            const unsigned long long xe = (unsigned long long)(P.X.rp[i + 1] - P.X.rp[i]);
            const unsigned long long extra = xe * (P.X.val ? 8ull : 0ull) + prod[gr] * (P.Y.val ? 8ull : 0ull);
            if (extra) atomicAdd(tally->bytes + B_GLOBAL, extra);
            const unsigned long long sym = xe * walk_xbytes(entry_split(ymx[gr], ew_max)) + prod[gr] * 4ull;
            atomicAdd(&tally->wbytes[0], (unsigned long long)0 - sym);  // no longer a bitmap walk
            atomicAdd(&tally->wprods[0], (unsigned long long)0 - prod[gr]);
            atomicAdd(&tally->wbytes[2], sym + extra);
            atomicAdd(&tally->wprods[2], (unsigned long long)prod[gr]);
        }
    }
}

// Per GLOBAL row: its number of work items (ech X entries each for a row split by entries,
// PCH products otherwise) and how many product offsets it needs (its X entries, or none).
__global__ void k_glob_prep(PassArgs a, const uint32_t *list, int64_t R, const uint64_t *prod, const uint32_t *ymx,
                            int ew_max, int64_t ech, int64_t *xlen, int64_t *items) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < R; r += (int64_t)gridDim.x * blockDim.x) {
        const RowRef Rf(a, list[r]);
        const int64_t xe = Rf.P->X.rp[Rf.i + 1] - Rf.P->X.rp[Rf.i];
        if (entry_split(ymx[Rf.g], ew_max)) {
            xlen[r] = 0;
            items[r] = (xe + ech - 1) / ech;
        } else {
            xlen[r] = xe;
            items[r] = ((int64_t)prod[Rf.g] + PCH - 1) / PCH;
        }
    }
}

// The masked Y-row length of every X entry of every GLOBAL row split by products, as one
// flat array (row r's entries start at xbase[r]; rows split by entries have none); a
// device-wide exclusive scan then gives each entry's global product offset. Beside it, ys
// keeps each entry's Y-row start, so the product walks read both in order. A block takes
// XCH consecutive entries at a time: it finds the rows
// they belong to once (usually one or two) and keeps each row's pointers in shared memory.
static constexpr int64_t XCH = 2048;  // entries per block iteration
static constexpr int XSEG = 64;       // rows per iteration kept in shared memory

__global__ void __launch_bounds__(256) k_glob_xlen(PassArgs a, const uint32_t *list, int64_t R,
                                                   const int64_t *__restrict__ xbase, int64_t *__restrict__ xoff,
                                                   int64_t *__restrict__ ys) {
    struct Seg {
        const int32_t *xci;
        const int64_t *yrp;
        const uint32_t *km;
        int64_t e0;  // first entry of the row in the flat array, minus the row's start in X.ci
    };
    __shared__ Seg seg[XSEG];
    __shared__ int64_t s_lo[XSEG + 1];
    __shared__ int64_t s_r0;
    __shared__ int s_n;
    const int64_t xtot = xbase[R];
    for (int64_t c0 = blockIdx.x * XCH; c0 < xtot; c0 += (int64_t)gridDim.x * XCH) {
        const int64_t c1 = min(xtot, c0 + XCH);
        if (threadIdx.x == 0) {
            int64_t lo = 0, hi = R - 1;  // the row of entry c0: the last r with xbase[r] <= c0
            while (lo < hi) {
                const int64_t mid = (lo + hi + 1) >> 1;
                if (xbase[mid] <= c0) lo = mid; else hi = mid - 1;
            }
            int64_t r1 = lo;  // the row of entry c1 - 1
            hi = R - 1;
            while (r1 < hi) {
                const int64_t mid = (r1 + hi + 1) >> 1;
                if (xbase[mid] <= c1 - 1) r1 = mid; else hi = mid - 1;
            }
            s_r0 = lo;
            s_n = (int)min((int64_t)XSEG, r1 - lo + 1);
        }
        __syncthreads();
        const int64_t r0 = s_r0;
        const int n = s_n;
        if ((int)threadIdx.x < n) {
            const RowRef Rf(a, list[r0 + threadIdx.x]);
            const Prod *P = Rf.P;
            const int64_t xb = P->X.rp[Rf.i];
            const int64_t fb = xbase[r0 + threadIdx.x];
            seg[threadIdx.x] = Seg{P->X.ci, P->Y.rp, P->km, fb - xb};
            s_lo[threadIdx.x] = fb;
            if ((int)threadIdx.x == n - 1) s_lo[n] = xbase[r0 + n];
        }
        __syncthreads();
        for (int64_t e = c0 + threadIdx.x; e < c1; e += blockDim.x) {
            int64_t len = 0, y0 = 0;
            if (e < s_lo[n]) {  // within the rows kept in shared memory
                int l = 0, h = n - 1;
                while (l < h) {
                    const int mid = (l + h + 1) >> 1;
                    if (s_lo[mid] <= e) l = mid; else h = mid - 1;
                }
                const Seg &sg = seg[l];
                const int32_t k = __ldg(sg.xci + (e - sg.e0));
                y0 = __ldg(sg.yrp + k);
                if (bit_of(sg.km, (uint32_t)k)) len = __ldg(sg.yrp + k + 1) - y0;
            } else {  // more rows in this stretch than shared memory keeps: find the row
                int64_t lo = r0 + n, hi = R - 1;
                while (lo < hi) {
                    const int64_t mid = (lo + hi + 1) >> 1;
                    if (__ldg(xbase + mid) <= e) lo = mid; else hi = mid - 1;
                }
                const RowRef Rf(a, list[lo]);
                const Prod *P = Rf.P;
                const int32_t k = __ldg(P->X.ci + P->X.rp[Rf.i] + (e - xbase[lo]));
                y0 = __ldg(P->Y.rp + k);
                if (bit_of(P->km, (uint32_t)k)) len = __ldg(P->Y.rp + k + 1) - y0;
            }
            xoff[e] = len;
            ys[e] = y0;
        }
        __syncthreads();
    }
}

// One work item per block iteration: products [s0, s1) of one row. The X entries that hold
// them are staged GNT at a time with their product offsets (from xoff); consecutive
// threads take consecutive products, so a long Y row is read coalesced.
// MODE G_SYM sets the row's bitmap bits; G_NUM adds the counts into the output row at the
// positions the bitmap ranks give; G_DENSE adds the counts into the row's dense slot (the
// bitmap comes from a scan of the slot afterwards: every count is >= 1).
enum { G_SYM = 0, G_NUM = 1, G_DENSE = 2 };
template <int MODE, bool COMB, int OCC>
__global__ void __launch_bounds__(GNT, MODE != G_SYM ? OCC : 8) k_glob_set(PassArgs a, GlobArgs g) {
    constexpr bool NUM = MODE != G_SYM;
    __shared__ int64_t s_off[GNT + 1];
    __shared__ int64_t s_st[GNT];
    __shared__ uint64_t s_a[GNT];
    __shared__ int32_t s_seg[GNT];  // segment walk: first segment of each staged X entry
    __shared__ int64_t s_wsum[32], s_gtot;
    // combining table for the item's hot outputs: key = bitmap word (symbolic) or output
    // column (numeric); first come claims a slot, other keys go straight to global memory
    __shared__ uint32_t s_key[CSLOT];
    __shared__ unsigned long long s_acc[CSLOT];
    for (int x = threadIdx.x; x < CSLOT; x += GNT) {
        s_key[x] = EMPTY;
        s_acc[x] = 0;
    }
    __syncthreads();
    const int64_t t0 = g.item_off[g.r0], t1 = g.item_off[g.r1];
    for (int64_t t = t0 + blockIdx.x; t < t1; t += gridDim.x) {
        int64_t lo = g.r0, hi = g.r1 - 1;
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (g.item_off[mid] <= t) lo = mid; else hi = mid - 1;
        }
        const int64_t r = lo;
        const uint32_t gr = g.list[r];
        const int pi = a.rowprod[gr];
        const Prod *PP = a.prods + pi;
        uint64_t *const pval = PP->val;
        if (MODE == G_NUM && !pval) continue;  // the product failed before its numeric pass
        uint32_t *err = &a.ps[pi].err;
        const bool chk = a.ps[pi].unsafe != 0;  // uniform over the item
        const int64_t row = xrow(*PP, gr);
        const int32_t *__restrict__ xci = PP->X.ci;
        const uint64_t *__restrict__ xval = PP->X.val;
        const int64_t *__restrict__ yrp = PP->Y.rp;
        const int32_t *__restrict__ yci = PP->Y.ci;
        const uint64_t *__restrict__ yval = PP->Y.val;
        const uint32_t *__restrict__ cm = PP->cm;
        const int64_t xb = PP->X.rp[row], xe = PP->X.rp[row + 1];
        const int64_t *xo = g.xoff + g.xbase[r];
        // product offsets are global across the GLOBAL rows: this row's start at xo[0]
        const int64_t total = __ldg(xo) + (int64_t)g.prod[gr];
        const int64_t s0 = __ldg(xo) + (t - g.item_off[r]) * PCH;
        const int64_t s1 = min(total, s0 + PCH);
        // first X entry whose products reach s0: the last p with xo[p] <= s0
        int64_t plo = 0, phi = xe - xb - 1;
        while (plo < phi) {
            const int64_t mid = (plo + phi + 1) >> 1;
            if (__ldg(xo + mid) <= s0) plo = mid; else phi = mid - 1;
        }
        uint2 *bmr = g.bmr + (r - g.r0) * g.nw;
        unsigned long long *val = MODE == G_NUM    ? (unsigned long long *)pval + (a.nnz[gr] - a.nnz[PP->row0])
                                  : MODE == G_DENSE ? g.dval + (r - g.r0) * g.dcols
                                                    : nullptr;
        for (int64_t c0 = xb + plo; c0 < xe; c0 += GNT) {
            const int64_t base = __ldg(xo + (c0 - xb));
            if (base >= s1) break;  // uniform: every thread reads the same base
            const int64_t p = c0 + threadIdx.x;
            const int nent = (int)min((int64_t)GNT, xe - c0);
            if (threadIdx.x < nent) {
                const int32_t k = __ldg(xci + p);
                s_off[threadIdx.x] = __ldg(xo + (p - xb)) - base;
                s_st[threadIdx.x] = __ldg(yrp + k);
                s_a[threadIdx.x] = (NUM && xval) ? __ldg(xval + p) : 1ull;
            }
            if (threadIdx.x == 0) s_off[nent] = (c0 + nent < xe ? __ldg(xo + (c0 + nent - xb)) : total) - base;
            __syncthreads();
            const int64_t f0 = max(s0 - base, (int64_t)0), f1 = min(s1 - base, s_off[nent]);
            auto product = [&](int l, int64_t q) {
                const uint32_t j = (uint32_t)__ldg(yci + q);
                // the column mask first: a masked-out product costs one bit load, no atomic
                if (!bit_of(cm, j)) return;
                unsigned long long add;
                if (!NUM) {
                    add = 1ull << (j & 31);
                } else {
                    const uint64_t av = s_a[l];
                    const uint64_t bv = yval ? __ldg(yval + q) : 1ull;
                    add = av * bv;
                    if (chk && __umul64hi(av, bv)) atomicOr(err, ERR_OVERFLOW);
                }
                const uint32_t k = NUM ? j : (j >> 5);
                const uint32_t slot = (k * 0x9E3779B1u) >> (32 - 10);
                uint32_t cur = EMPTY - 1;
                if (COMB) {
                    cur = ((volatile uint32_t *)s_key)[slot];
                    if (cur == EMPTY) {
                        const uint32_t old = atomicCAS(s_key + slot, EMPTY, k);
                        cur = old == EMPTY ? k : old;
                    }
                }
                if (COMB && cur == k) {
                    if (!NUM) {
                        atomicOr((unsigned int *)&s_acc[slot], (unsigned int)add);
                    } else if (chk) {
                        const unsigned long long old = atomicAdd(s_acc + slot, add);
                        if (old + add < old) atomicOr(err, ERR_OVERFLOW);
                    } else {
                        atomicAdd(s_acc + slot, add);
                    }
                } else if (!NUM) {
                    atomicOr(&bmr[k].x, (uint32_t)add);
                } else {
                    unsigned long long *dst;
                    if (MODE == G_DENSE) {
                        dst = val + j;
                    } else {
                        const uint2 br = __ldg(bmr + (j >> 5));
                        dst = val + br.y + __popc(br.x & ((1u << (j & 31)) - 1u));
                    }
                    if (chk) {
                        const unsigned long long old = atomicAdd(dst, add);
                        if (old + add < old) atomicOr(err, ERR_OVERFLOW);
                    } else {
                        atomicAdd(dst, add);
                    }
                }
            };
            if (g.short_walk && s_off[nent] <= 8 * (int64_t)nent) {
                // short Y rows: each thread walks the products of its own X entry
                if ((int)threadIdx.x < nent) {
                    const int l = threadIdx.x;
                    const int64_t lo_f = max(s_off[l], f0), hi_f = min(s_off[l + 1], f1);
                    for (int64_t f = lo_f; f < hi_f; f++) product(l, s_st[l] + (f - s_off[l]));
                }
            } else if (g.seg_walk && s_off[nent] >= SEGMIN * (int64_t)nent) {
                // long Y rows: the X entries' products are cut into segments of up to SEG;
                // a warp takes a segment (its X entry found once per segment) and its lanes
                // read the Y row coalesced
                int cnt = 0;
                if ((int)threadIdx.x < nent) {
                    const int l = threadIdx.x;
                    const int64_t lo_f = max(s_off[l], f0), hi_f = min(s_off[l + 1], f1);
                    cnt = hi_f > lo_f ? (int)((hi_f - lo_f + SEG - 1) / SEG) : 0;
                }
                const int64_t ex = block_excl_scan<GNT>(cnt, s_wsum, &s_gtot);
                if ((int)threadIdx.x < nent) s_seg[threadIdx.x] = (int32_t)ex;
                __syncthreads();
                const int nseg = (int)s_gtot;
                const int lane = threadIdx.x & 31;
                for (int sg = threadIdx.x >> 5; sg < nseg; sg += GNT / 32) {
                    // the last entry whose first segment is at or before sg (it has segments)
                    int l = 0, h = nent - 1;
                    while (l < h) {
                        const int mid = (l + h + 1) >> 1;
                        if (s_seg[mid] <= sg) l = mid; else h = mid - 1;
                    }
                    const int64_t b0 = max(s_off[l], f0) + (int64_t)(sg - s_seg[l]) * SEG;
                    const int64_t b1 = min(b0 + SEG, min(s_off[l + 1], f1));
                    for (int64_t f = b0 + lane; f < b1; f += 32) product(l, s_st[l] + (f - s_off[l]));
                }
            } else {
                // long Y rows: consecutive threads take consecutive products (coalesced Y
                // reads); each finds its X entry by binary search in shared memory
                for (int64_t f = f0 + threadIdx.x; f < f1; f += GNT) {
                    int l = 0, h = nent - 1;
                    while (l < h) {
                        const int mid = (l + h + 1) >> 1;
                        if (s_off[mid] <= f) l = mid; else h = mid - 1;
                    }
                    product(l, s_st[l] + (f - s_off[l]));
                }
            }
            __syncthreads();
        }
        // flush the combining table into the row, reset it for the next item
        for (int x = threadIdx.x; COMB && x < CSLOT; x += GNT) {
            const uint32_t k = s_key[x];
            if (k == EMPTY) continue;
            if (!NUM) {
                atomicOr(&bmr[k].x, (uint32_t)s_acc[x]);
            } else {
                unsigned long long *dst;
                if (MODE == G_DENSE) {
                    dst = val + k;
                } else {
                    const uint2 br = __ldg(bmr + (k >> 5));
                    dst = val + br.y + __popc(br.x & ((1u << (k & 31)) - 1u));
                }
                const unsigned long long v = s_acc[x];
                if (chk) {
                    const unsigned long long old = atomicAdd(dst, v);
                    if (old + v < old) atomicOr(err, ERR_OVERFLOW);
                } else {
                    atomicAdd(dst, v);
                }
            }
            s_key[x] = EMPTY;
            s_acc[x] = 0;
        }
        __syncthreads();
    }
}

// The same split-row pass with a warp-level product walk (the default). Each of a block's
// warps takes a run of SUB consecutive products of the block's work item and finds the X
// entry holding the run's first product by a 32-way search over the row's product offsets.
// It then holds 32 X entries at a time in registers (Y row start, product offset, value)
// and walks their products 32 at a time: lane i takes product w + i and finds the entry
// that holds it by a 5-step shuffle search over the 32 lanes' offsets. Consecutive lanes
// read consecutive entries of a Y row (coalesced when Y rows are long), no lane idles when
// Y rows are short, and nothing is staged block-wide: the warps only meet to flush the
// combining table at the end of an item.
static constexpr int SUB = (int)(PCH / (GNT / 32));  // products per warp run
static constexpr unsigned LANE_RUN = 8;  // most products per entry for the lane-per-entry walk

//
// DSM (dense rows only, output no wider than the dynamic shared memory holds): the block keeps
// a whole dense count row in shared memory, takes a contiguous range of work items (so its
// items mostly belong to one row), adds every product there, and adds the row's non-zero
// counts to the global dense row when it moves to another row and at the end: one global
// atomic per touched column per block instead of one per product.
//
// EW: the launch takes only the work items of rows split by X entries (true) or only those
// of rows split by products (false); a wave with both kinds launches both variants.
template <int MODE, bool COMB, int OCC, bool DSM = false, bool EW = false>
__global__ void __launch_bounds__(GNT, OCC) k_glob_lbs(PassArgs a, GlobArgs g) {
    constexpr bool NUM = MODE != G_SYM;
    static_assert(!DSM || (MODE == G_DENSE && !COMB), "a shared-memory row replaces the combining table");
    __shared__ uint32_t s_key[COMB ? CSLOT : 1];
    __shared__ unsigned long long s_acc[COMB ? CSLOT : 1];
    extern __shared__ unsigned long long s_dense[];  // DSM: g.dcols counts
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int x = threadIdx.x; COMB && x < CSLOT; x += GNT) {
        s_key[x] = EMPTY;
        s_acc[x] = 0;
    }
    for (int64_t x = threadIdx.x; DSM && x < g.dcols; x += GNT) s_dense[x] = 0;
    __syncthreads();
    const int64_t t0 = g.item_off[g.r0], t1 = g.item_off[g.r1];
    int64_t ta = t0 + blockIdx.x, tb = t1, ts = gridDim.x;
    if (DSM) {
        const int64_t per = (t1 - t0 + gridDim.x - 1) / gridDim.x;
        ta = t0 + (int64_t)blockIdx.x * per;
        tb = min(t1, ta + per);
        ts = 1;
    }
    // DSM: the row whose counts the shared-memory row holds, and where they go
    int64_t d_r = -1, d_w = 0;
    unsigned long long *d_val = nullptr;
    uint32_t *d_err = nullptr;
    bool d_chk = false;
    auto d_flush = [&]() {  // all threads; the caller synchronises before and after
        for (int64_t x = threadIdx.x; x < d_w; x += GNT) {
            const unsigned long long v = s_dense[x];
            if (!v) continue;
            s_dense[x] = 0;
            if (d_chk) {
                const unsigned long long old = atomicAdd(d_val + x, v);
                if (old + v < old) atomicOr(d_err, ERR_OVERFLOW);
            } else {
                atomicAdd(d_val + x, v);
            }
        }
    };
    for (int64_t t = ta; t < tb; t += ts) {
        int64_t lo = g.r0, hi = g.r1 - 1;
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (g.item_off[mid] <= t) lo = mid; else hi = mid - 1;
        }
        const int64_t r = lo;
        const uint32_t gr = g.list[r];
        const int pi = a.rowprod[gr];
        const Prod *PP = a.prods + pi;
        uint64_t *const pval = PP->val;
        if (MODE == G_NUM && !pval) continue;  // the product failed before its numeric pass
        uint32_t *err = &a.ps[pi].err;
        const bool chk = a.ps[pi].unsafe != 0;  // uniform over the item
        const int64_t row = xrow(*PP, gr);
        const uint64_t *__restrict__ xval = PP->X.val;
        const int32_t *__restrict__ yci = PP->Y.ci;
        const uint64_t *__restrict__ yval = PP->Y.val;
        const uint32_t *__restrict__ cm = PP->cm;
        const int64_t xb = PP->X.rp[row], xlen = PP->X.rp[row + 1] - xb;
        if (entry_split(g.ymx[gr], g.ew_max) != EW) continue;  // the other variant's item (uniform)
        uint2 *bmr = g.bmr + (r - g.r0) * g.nw;
        unsigned long long *val = MODE == G_NUM    ? (unsigned long long *)pval + (a.nnz[gr] - a.nnz[PP->row0])
                                  : MODE == G_DENSE ? g.dval + (r - g.r0) * g.dcols
                                                    : nullptr;
        if (DSM && r != d_r) {  // uniform over the block (r follows from t)
            if (d_r >= 0) {
                d_flush();
                __syncthreads();
            }
            d_r = r;
            d_w = PP->Y.ncols;
            d_val = val;
            d_err = err;
            d_chk = chk;
        }
        // one scalar product x_ik * Y[k, j], its column j and Y value bv already loaded (the
        // callers issue several products' loads before applying any)
        auto apply = [&](uint64_t av, uint32_t j, uint64_t bv) {
            // the column mask first: a masked-out product costs one bit load, no atomic
            if (!bit_of(cm, j)) return;
            unsigned long long add;
            if (!NUM) {
                add = 1ull << (j & 31);
            } else {
                add = av * bv;
                if (chk && __umul64hi(av, bv)) atomicOr(err, ERR_OVERFLOW);
            }
            if (DSM) {
                if (chk) {
                    const unsigned long long old = atomicAdd(&s_dense[j], add);
                    if (old + add < old) atomicOr(err, ERR_OVERFLOW);
                } else {
                    atomicAdd(&s_dense[j], add);
                }
                return;
            }
            const uint32_t k = NUM ? j : (j >> 5);
            const uint32_t slot = (k * 0x9E3779B1u) >> (32 - 10);
            uint32_t cur = EMPTY - 1;
            if (COMB) {
                cur = ((volatile uint32_t *)s_key)[slot];
                if (cur == EMPTY) {
                    const uint32_t old = atomicCAS(s_key + slot, EMPTY, k);
                    cur = old == EMPTY ? k : old;
                }
            }
            if (COMB && cur == k) {
                if (!NUM) {
                    atomicOr((unsigned int *)&s_acc[slot], (unsigned int)add);
                } else if (chk) {
                    const unsigned long long old = atomicAdd(s_acc + slot, add);
                    if (old + add < old) atomicOr(err, ERR_OVERFLOW);
                } else {
                    atomicAdd(s_acc + slot, add);
                }
            } else if (!NUM) {
                atomicOr(&bmr[k].x, (uint32_t)add);
            } else {
                unsigned long long *dst;
                if (MODE == G_DENSE) {
                    dst = val + j;
                } else {
                    const uint2 br = __ldg(bmr + (j >> 5));
                    dst = val + br.y + __popc(br.x & ((1u << (j & 31)) - 1u));
                }
                if (chk) {
                    const unsigned long long old = atomicAdd(dst, add);
                    if (old + add < old) atomicOr(err, ERR_OVERFLOW);
                } else {
                    atomicAdd(dst, add);
                }
            }
        };
        auto yv = [&](int64_t q) -> uint64_t { return (NUM && yval) ? __ldg(yval + q) : 1ull; };
        auto product = [&](uint64_t av, int64_t q) { apply(av, (uint32_t)__ldg(yci + q), yv(q)); };
        // a lane's own run of n <= run products from Y position q0 (the lane-per-entry walk):
        // four column loads in flight per lane when Y is a pattern matrix
        auto lane_walk = [&](uint64_t av, int64_t q0, int n, int run) {
            if (NUM && yval) {  // valued Y (an earlier result): one product at a time
                for (int u = 0; u < run; u++)
                    if (u < n) product(av, q0 + u);
                return;
            }
            for (int u0 = 0; u0 < run; u0 += 4) {
                uint32_t jj[4];
#pragma unroll
                for (int u = 0; u < 4; u++)
                    if (u0 + u < n) jj[u] = (uint32_t)__ldg(yci + q0 + u0 + u);
#pragma unroll
                for (int u = 0; u < 4; u++)
                    if (u0 + u < n) apply(av, jj[u], 1ull);
            }
        };
        // the lane holding product fj of a group of 32 entries whose products start at offsets
        // off (ascending over the lanes) relative to window start w: the last lane whose
        // entry starts at or before fj = w + lane (a 5-step shuffle search)
        auto holder = [&](int64_t off, int64_t w) {
            const int rel = (int)max((int64_t)-1, min(off - w, (int64_t)32));
            int src = 0;
#pragma unroll
            for (int st = 16; st; st >>= 1) {
                const int v = __shfl_sync(FULL, rel, src + st);
                if (v <= lane) src += st;
            }
            return src;
        };
        if (EW) {
            // a row split by X entries: this warp's share of the item's entries, 32 at a time;
            // each lane looks up its entry's Y row, then the lanes walk their own short runs,
            // or the group's products in windows of 32 when some run is longer
            const int64_t e0 = (t - g.item_off[r]) * g.ech;
            const int64_t we0 = e0 + (int64_t)wid * (g.ech / (GNT / 32));
            const int64_t we1 = min(min(xlen, e0 + g.ech), we0 + g.ech / (GNT / 32));
            const int32_t *__restrict__ xci = PP->X.ci;
            const int64_t *__restrict__ yrp = PP->Y.rp;
            const uint32_t *__restrict__ km = PP->km;
            for (int64_t p = we0; p < we1; p += 32) {
                const int64_t e = p + lane;
                int64_t st = 0, len = 0;
                uint64_t av = 1;
                if (e < we1) {  // the row pointers load beside the mask word
                    const uint32_t k = (uint32_t)__ldg(xci + xb + e);
                    st = __ldg(yrp + k);
                    const int64_t y1 = __ldg(yrp + k + 1);
                    if (NUM && xval) av = __ldg(xval + xb + e);
                    if (bit_of(km, k)) len = y1 - st;
                }
                const unsigned run = __reduce_max_sync(FULL, (unsigned)len);
                if (run <= LANE_RUN) {
                    lane_walk(av, st, (int)len, (int)run);
                    continue;
                }
                int64_t x = len;  // inclusive scan of the run lengths over the lanes
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const int64_t y = __shfl_up_sync(FULL, x, d);
                    if (lane >= d) x += y;
                }
                const int64_t tot = __shfl_sync(FULL, x, 31), off = x - len, base = st - off;
                for (int64_t w = 0; w < tot; w += 32) {
                    const int src = holder(off, w);
                    const int64_t q = __shfl_sync(FULL, base, src) + w + lane;
                    const uint64_t ax = NUM ? __shfl_sync(FULL, av, src) : 1ull;
                    if (w + lane < tot) product(ax, q);
                }
            }
        }
        const int64_t *__restrict__ xo = g.xoff + g.xbase[r];
        const int64_t *__restrict__ ysr = g.ys + g.xbase[r];
        // product offsets are global across the GLOBAL rows split by products: this row's
        // start at xo[0]
        const int64_t total = EW ? 0 : __ldg(xo) + (int64_t)g.prod[gr];
        const int64_t s0 = EW ? 0 : __ldg(xo) + (t - g.item_off[r]) * PCH;
        const int64_t s1 = min(total, s0 + PCH);
        const int64_t ws0 = s0 + (int64_t)wid * SUB, ws1 = EW ? ws0 : min(s1, ws0 + SUB);
        if (ws0 < ws1) {
            // the last X entry p of the row with xo[p] <= ws0, 32 probes per step
            int64_t plo = 0, phi = xlen - 1;
            while (phi - plo >= 32) {
                const int64_t step = (phi - plo + 31) / 32;
                const int64_t probe = min(plo + (int64_t)lane * step, phi);
                const unsigned m = __ballot_sync(FULL, __ldg(xo + probe) <= ws0);
                const int kk = 31 - __clz(m);
                if (kk < 31) phi = min(plo + (int64_t)(kk + 1) * step, phi) - 1;
                plo = min(plo + (int64_t)kk * step, phi);
            }
            {
                const int64_t probe = plo + lane;
                const unsigned m = __ballot_sync(FULL, probe <= phi && __ldg(xo + min(probe, phi)) <= ws0);
                plo += 31 - __clz(m);
            }
            int64_t p = plo, f = ws0;
            while (f < ws1 && p < xlen) {
                const int64_t e = p + lane;
                const bool ok = e < xlen;
                const int64_t off = ok ? __ldg(xo + e) : total;
                int64_t base = 0;  // Y position of this entry's product f is base + f
                uint64_t av = 1;
                if (ok) {
                    base = __ldg(ysr + e) - off;
                    if (NUM && xval) av = __ldg(xval + xb + e);
                }
                int64_t gend = 0;  // first product after the 32 entries
                if (lane == 31) gend = e + 1 < xlen ? __ldg(xo + e + 1) : total;
                gend = __shfl_sync(FULL, gend, 31);
                const int64_t lim = min(ws1, gend);
                // short Y rows (papers to authors, topics or venues): when no entry has more
                // than LANE_RUN products in [f, lim), each lane walks its own entry's products
                // (no search); otherwise windows of 32 consecutive products
                int64_t nxt_e = __shfl_down_sync(FULL, off, 1);
                if (lane == 31) nxt_e = gend;
                const int64_t my_lo = max(off, f), my_hi = min(nxt_e, lim);
                const int my_n = my_hi > my_lo ? (int)min(my_hi - my_lo, (int64_t)1 << 20) : 0;
                const unsigned run = __reduce_max_sync(FULL, (unsigned)my_n);
                if (run <= LANE_RUN) {
                    lane_walk(av, base + my_lo, my_n, (int)run);
                    f = max(f, lim);
                    p += 32;
                    continue;
                }
                for (int64_t w = f; w < lim;) {
                    // the entry holding product w (the last lane whose entry starts at or
                    // before it) and where the next entry starts: while one entry holds the
                    // whole window (long Y rows), its lanes read its Y row with no search
                    const int cur = __popc(__ballot_sync(FULL, off <= w)) - 1;
                    int64_t nxt = __shfl_sync(FULL, off, min(cur + 1, 31));
                    if (cur == 31) nxt = gend;
                    const int64_t run_end = min(nxt, lim);
                    if (run_end >= w + 32) {  // uniform over the warp; at least one full window
                        const int64_t b = __shfl_sync(FULL, base, cur);
                        const uint64_t ax = NUM ? __shfl_sync(FULL, av, cur) : 1ull;
                        if (!(NUM && yval))
                            for (; w + 64 <= run_end; w += 64) {  // two windows' loads in flight
                                const uint32_t j0 = (uint32_t)__ldg(yci + b + w + lane);
                                const uint32_t j1 = (uint32_t)__ldg(yci + b + w + 32 + lane);
                                apply(ax, j0, 1ull);
                                apply(ax, j1, 1ull);
                            }
                        for (; w + 32 <= run_end; w += 32) product(ax, b + w + lane);
                        continue;
                    }
                    const int64_t fj = w + lane;
                    const int src = holder(off, w);
                    const int64_t q = __shfl_sync(FULL, base, src) + fj;
                    const uint64_t ax = NUM ? __shfl_sync(FULL, av, src) : 1ull;
                    if (fj < lim) product(ax, q);
                    w += 32;
                }
                f = max(f, lim);
                p += 32;
            }
        }
        __syncthreads();
        // flush the combining table into the row, reset it for the next item
        for (int x = threadIdx.x; COMB && x < CSLOT; x += GNT) {
            const uint32_t k = s_key[x];
            if (k == EMPTY) continue;
            if (!NUM) {
                atomicOr(&bmr[k].x, (uint32_t)s_acc[x]);
            } else {
                unsigned long long *dst;
                if (MODE == G_DENSE) {
                    dst = val + k;
                } else {
                    const uint2 br = __ldg(bmr + (k >> 5));
                    dst = val + br.y + __popc(br.x & ((1u << (k & 31)) - 1u));
                }
                const unsigned long long v = s_acc[x];
                if (chk) {
                    const unsigned long long old = atomicAdd(dst, v);
                    if (old + v < old) atomicOr(err, ERR_OVERFLOW);
                } else {
                    atomicAdd(dst, v);
                }
            }
            s_key[x] = EMPTY;
            s_acc[x] = 0;
        }
        __syncthreads();
    }
    if (DSM && d_r >= 0) d_flush();
}

// The rank pass in parallel over chunks of RCH words of every row slot (one block each), so a
// few very wide rows do not leave the GPU to a few blocks: (1) set bits per chunk, (2) one
// warp per row scans its chunks (the row's size), (3) each chunk writes its words' ranks.
static constexpr int64_t RCH = (int64_t)GNT * RW;  // words per chunk

__global__ void __launch_bounds__(GNT) k_glob_csum(GlobArgs g, int64_t nch, int64_t *csum) {
    __shared__ int64_t warp_sums[32];
    __shared__ int64_t gtot;
    const int64_t total = (g.r1 - g.r0) * nch;
    for (int64_t c = blockIdx.x; c < total; c += gridDim.x) {
        const int64_t slot = c / nch, w0 = (c - slot * nch) * RCH + (int64_t)threadIdx.x * RW;
        const uint2 *bmr = g.bmr + slot * g.nw;
        int cnt = 0;
#pragma unroll
        for (int u = 0; u < RW; u++) cnt += w0 + u < g.nw ? __popc(bmr[w0 + u].x) : 0;
        block_excl_scan<GNT>(cnt, warp_sums, &gtot);
        if (threadIdx.x == 0) csum[c] = gtot;
        __syncthreads();
    }
}

__global__ void k_glob_rowscan(PassArgs a, GlobArgs g, int64_t nch, int64_t *csum, int numeric) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < g.r1 - g.r0; r += nwarps) {
        int64_t *cs = csum + r * nch, carry = 0;
        for (int64_t c0 = 0; c0 < nch; c0 += 32) {
            const int64_t v = c0 + lane < nch ? cs[c0 + lane] : 0;
            int64_t x = v;
            for (int d = 1; d < 32; d <<= 1) {
                const int64_t y = __shfl_up_sync(FULL, x, d);
                if (lane >= d) x += y;
            }
            if (c0 + lane < nch) cs[c0 + lane] = carry + x - v;  // exclusive
            carry += __shfl_sync(FULL, x, 31);
        }
        if (lane == 0) {
            const RowRef Rf(a, g.list[g.r0 + r]);
            if (!numeric) a.nnz[Rf.g] = carry;
            else if (Rf.P->ci && Rf.out_len(a) != carry) atomicOr(Rf.err(a), ERR_COUNT);
        }
    }
}

__global__ void __launch_bounds__(GNT) k_glob_crank(GlobArgs g, int64_t nch, const int64_t *csum) {
    __shared__ int64_t warp_sums[32];
    __shared__ int64_t gtot;
    const int64_t total = (g.r1 - g.r0) * nch;
    for (int64_t c = blockIdx.x; c < total; c += gridDim.x) {
        const int64_t slot = c / nch, w0 = (c - slot * nch) * RCH + (int64_t)threadIdx.x * RW;
        uint2 *bmr = g.bmr + slot * g.nw;
        int cnt[RW];
        int sum = 0;
#pragma unroll
        for (int u = 0; u < RW; u++) {
            cnt[u] = w0 + u < g.nw ? __popc(bmr[w0 + u].x) : 0;
            sum += cnt[u];
        }
        int64_t ex = csum[c] + block_excl_scan<GNT>(sum, warp_sums, &gtot);
#pragma unroll
        for (int u = 0; u < RW; u++) {
            if (w0 + u < g.nw) bmr[w0 + u].y = (uint32_t)ex;
            ex += cnt[u];
        }
        __syncthreads();
    }
}

// One thread per bitmap word: the word's set bits become consecutive output entries.
__global__ void k_glob_fill(PassArgs a, GlobArgs g) {
    const int64_t total = (g.r1 - g.r0) * g.nw;
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < total; x += (int64_t)gridDim.x * blockDim.x) {
        const uint2 br = g.bmr[x];
        uint32_t word = br.x;
        if (!word) continue;
        const int64_t slot = x / g.nw, w = x - slot * g.nw;
        const RowRef Rf(a, g.list[g.r0 + slot]);
        int32_t *ci = Rf.P->ci;
        if (!ci) continue;
        // column ids in order; the counts were zeroed with the product's count array
        int64_t pos = Rf.out_off(a) + br.y;
        while (word) {
            const int b = __ffs(word) - 1;
            word &= word - 1;
            ci[pos++] = (int32_t)(w * 32 + b);
        }
    }
}

// Dense rows: one warp per bitmap word; lane i reads column 32w + i of the dense slot
// (coalesced) and the ballot of the non-zero counts is the word.
__global__ void k_glob_dscan(GlobArgs g) {
    const int lane = threadIdx.x & 31;
    const int64_t total = (g.r1 - g.r0) * g.nw;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t x = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; x < total; x += nwarps) {
        const int64_t slot = x / g.nw, w = x - slot * g.nw;
        const int64_t j = w * 32 + lane;
        const bool nz = j < g.dcols && g.dval[slot * g.dcols + j] != 0;
        const unsigned word = __ballot_sync(FULL, nz);
        if (lane == 0) g.bmr[x] = make_uint2(word, 0u);
    }
}

// Dense rows: one thread per bitmap word; the word's set bits become consecutive output
// entries with their counts from the dense slot.
__global__ void k_glob_dfill(PassArgs a, GlobArgs g) {
    const int64_t total = (g.r1 - g.r0) * g.nw;
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < total; x += (int64_t)gridDim.x * blockDim.x) {
        const uint2 br = g.bmr[x];
        uint32_t word = br.x;
        if (!word) continue;
        const int64_t slot = x / g.nw, w = x - slot * g.nw;
        const RowRef Rf(a, g.list[g.r0 + slot]);
        const Prod P = *Rf.P;
        if (!P.ci) continue;
        const unsigned long long *dv = g.dval + slot * g.dcols;
        int64_t pos = Rf.out_off(a) + br.y;
        while (word) {
            const int b = __ffs(word) - 1;
            word &= word - 1;
            const int64_t j = w * 32 + b;
            P.ci[pos] = (int32_t)j;
            P.val[pos] = dv[j];
            pos++;
        }
    }
}

// ------------------------------------------------------------------ launch helpers

// Set while a pass only prepares its kernels' shared-memory attributes (before a capture,
// where the attribute calls are kept out of the captured stream).
static thread_local bool g_attrs_only = false, g_capturing = false;

template <class K>
static void launch(K kern, unsigned grid, int nt, size_t smem, cudaStream_t s, const PassArgs &a, int bin) {
    if (smem > 48 * 1024 && !g_capturing)
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (!g_attrs_only) kl(kern, grid, nt, smem, s, a, bin);
}

static unsigned blocks_for(uint32_t rows_upper, int rows_per_block, int max_blocks) {
    const unsigned g = (unsigned)((rows_upper + rows_per_block - 1) / rows_per_block);
    return std::max(1u, std::min(g, (unsigned)max_blocks));
}

// Launch every non-empty shared-memory bin's kernel of one pass, each grid sized to its
// bin's rows (capped at a few blocks per SM; the kernels loop over their bin, reading its
// row count from the device), or at the cap for every bin when fixed_grid (a captured
// graph serves every wave of the same shape). With prof, CUDA events bracket each launch.
// GLOBAL runs separately (glob_pass). dense_cols is the widest output among the wave's
// products that fit the dense bin (it sizes the dense kernels' shared memory).
static void run_pass(int pass, const PassArgs &a, const uint32_t *host_counts, int64_t dense_cols, const Tuning &tun,
                     cudaStream_t s, Prof *prof, bool fixed_grid = false) {
    const bool numeric = pass == 1;
    const int sms = tun.sm_count;
    const size_t stage = sizeof(Stage);
    // the pooled kernel for the warp-hash and 2048-slot bins (tun.pool), sized to the largest
    // table among them that this pass uses
    bool pooled = false;
    if (tun.pool) {
        size_t smem = 0;
        for (int b = 0; b < B_GLOBAL; b++)
            if (pool_bin(b) && host_counts[b]) smem = std::max(smem, pool_smem(b, numeric));
        if (smem) {
            pooled = true;
            if (prof && prof->on) {
                prof->pool_ran[pass] = true;
                cudaEventRecordWithFlags(prof->pev[pass][0], s, g_capturing ? cudaEventRecordExternal : 0);
            }
            auto kern = numeric ? k_bins_pool<true> : k_bins_pool<false>;
            if (smem > 48 * 1024 && !g_capturing)
                cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            int per_sm = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem) != cudaSuccess || per_sm < 1) {
                cudaGetLastError();
                per_sm = 1;
            }
            // no more blocks than tiles (a few rows need not start every resident slot);
            // a captured pass keeps the full grid (its counts are only known on the device)
            uint64_t tiles = 0;
            for (int b = 0; b < B_GLOBAL; b++)
                if (pool_bin(b)) tiles += (host_counts[b] + pool_rows_per_tile(b) - 1) / pool_rows_per_tile(b);
            const uint64_t slots = (uint64_t)sms * per_sm;
            const unsigned grid = (unsigned)(fixed_grid ? slots : std::max<uint64_t>(1, std::min(slots, tiles)));
            if (!g_attrs_only) {
                cudaMemsetAsync(a.pool_head, 0, sizeof(unsigned), s);
                kl(kern, grid, 256, smem, s, a);
            }
            if (prof && prof->on)
                cudaEventRecordWithFlags(prof->pev[pass][1], s, g_capturing ? cudaEventRecordExternal : 0);
        }
    }
    if (host_counts[B_LANE]) {
        const uint32_t rows = fixed_grid ? (1u << 30) : host_counts[B_LANE];
        if (prof && prof->full())
            cudaEventRecordWithFlags(prof->ev[pass][B_LANE][0], s, g_capturing ? cudaEventRecordExternal : 0);
        const unsigned g = blocks_for(rows, LANE_NT, sms * 16);
        if (numeric) launch(k_lane_rows<true>, g, LANE_NT, 0, s, a, (int)B_LANE);
        else launch(k_lane_rows<false>, g, LANE_NT, 0, s, a, (int)B_LANE);
        if (prof && prof->full())
            cudaEventRecordWithFlags(prof->ev[pass][B_LANE][1], s, g_capturing ? cudaEventRecordExternal : 0);
    }
    for (int b = 0; b < B_GLOBAL; b++) {
        if (!host_counts[b]) continue;
        if (pooled && pool_bin(b)) continue;
        const uint32_t rows = fixed_grid ? (1u << 30) : host_counts[b];
        // inside a capture the records become event-record nodes, so replays time the bins
        if (prof && prof->full()) cudaEventRecordWithFlags(prof->ev[pass][b][0], s, g_capturing ? cudaEventRecordExternal : 0);
        switch (b) {
#define WARP_BIN(BIN, T, W)                                                                       \
    case BIN: {                                                                                   \
        const unsigned g = blocks_for(rows, W, sms * 8);                                          \
        if (numeric)                                                                              \
            launch(k_num_warp<T, W>, g, W * 32, W * 32 * stage + (size_t)W * T * 12, s, a, BIN); \
        else                                                                                      \
            launch(k_sym_warp<T, W>, g, W * 32, W * 32 * stage + (size_t)W * T * 4, s, a, BIN);  \
        break;                                                                                    \
    }
            WARP_BIN(B_W32, 32, 8)
            WARP_BIN(B_W64, 64, 8)
            WARP_BIN(B_W128, 128, 8)
            WARP_BIN(B_W256, 256, 8)
            WARP_BIN(B_W512, 512, 4)
            WARP_BIN(B_W1024, 1024, 4)
#undef WARP_BIN
#define BLOCK_BIN(BIN, T, NT)                                                          \
    case BIN: {                                                                        \
        const unsigned g = blocks_for(rows, 1, sms * 4);                               \
        if (numeric)                                                                   \
            launch(k_num_block<T, NT>, g, NT, NT * stage + (size_t)T * 12, s, a, BIN); \
        else                                                                           \
            launch(k_sym_block<T, NT>, g, NT, NT * stage + (size_t)T * 4, s, a, BIN);  \
        break;                                                                         \
    }
            BLOCK_BIN(B_K2048, 2048, 256)
            BLOCK_BIN(B_K4096, 4096, 512)
            BLOCK_BIN(B_K8192, 8192, 1024)
#undef BLOCK_BIN
            case B_DENSE: {
                const unsigned g = blocks_for(rows, 1, sms * 4);
                if (numeric)
                    launch(k_num_dense<256>, g, 256, 256 * stage + (size_t)dense_cols * 8, s, a, B_DENSE);
                else
                    launch(k_sym_dense<256>, g, 256, 256 * stage + (size_t)((dense_cols + 31) / 32) * 4, s, a,
                           B_DENSE);
                break;
            }
        }
        if (prof && prof->full()) cudaEventRecordWithFlags(prof->ev[pass][b][1], s, g_capturing ? cudaEventRecordExternal : 0);
    }
}

void WaveCache::drop_graphs() {
    for (auto &kv : graphs) cudaGraphExecDestroy(kv.second);
    graphs.clear();
}

void WaveCache::clear(Alloc &al, cudaStream_t s) {
    drop_graphs();
    if (ws) al.free(ws, s);
    ws = nullptr;
    mcap = 0;
    wcap = 0;
    if (pinned || rb) cudaStreamSynchronize(s);  // no upload may still read it, no read-back write it
    if (pinned) cudaFreeHost(pinned);
    if (rb) cudaFreeHost(rb);
    pinned = nullptr;
    pinned_cap = 0;
    rb = nullptr;
}

// Copies records into pinned host memory, one record per grid row (blockIdx.y): 16-byte
// words when both ends and the size allow, else bytes.
struct RbSegs {
    static constexpr int MAX = 8;
    const char *src[MAX];
    size_t at[MAX], n[MAX];
};
__global__ void k_readback(RbSegs g, char *__restrict__ dst_base) {
    const char *__restrict__ src = g.src[blockIdx.y];
    char *__restrict__ dst = dst_base + g.at[blockIdx.y];
    const size_t n = g.n[blockIdx.y];
    const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x, st = (size_t)gridDim.x * blockDim.x;
    if ((((uintptr_t)src | (uintptr_t)dst | n) & 15) == 0) {
        for (size_t i = t; i < n / 16; i += st) ((int4 *)dst)[i] = __ldg((const int4 *)src + i);
    } else {
        for (size_t i = t; i < n; i += st) dst[i] = src[i];
    }
}

bool Readback::get(void *dst, const void *src, size_t bytes) {
    if (!bytes) return true;
    if (wc_ && !wc_->rb && cudaMallocHost(&wc_->rb, WaveCache::RB_BYTES) != cudaSuccess) {
        cudaGetLastError();
        wc_->rb = nullptr;
    }
    if (!wc_ || !wc_->rb || used_ + bytes > WaveCache::RB_BYTES)
        return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s_) == cudaSuccess;
    // the copy itself is launched by sync(), with the other records, in one kernel
    parts_.push_back({dst, src, used_, bytes});
    used_ += (bytes + 255) / 256 * 256;
    return true;
}

bool Readback::sync() {
    bool ok = true;
    for (size_t p0 = 0; ok && p0 < parts_.size(); p0 += RbSegs::MAX) {
        RbSegs g{};
        size_t most = 0;
        const int k = (int)std::min<size_t>(RbSegs::MAX, parts_.size() - p0);
        for (int i = 0; i < k; i++) {
            const Part &p = parts_[p0 + i];
            g.src[i] = (const char *)p.src;
            g.at[i] = p.at;
            g.n[i] = p.bytes;
            most = std::max(most, p.bytes);
        }
        kl(k_readback, dim3((unsigned)std::min<size_t>((most + 4095) / 4096, 64), (unsigned)k), 256, 0, s_, g,
           wc_->rb);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            fprintf(stderr, "mp: read-back: %s\n", cudaGetErrorString(e));
            ok = false;
        }
    }
    const cudaError_t e = cudaStreamSynchronize(s_);
    if (e != cudaSuccess) {
        fprintf(stderr, "mp: sync: %s\n", cudaGetErrorString(e));
        ok = false;
    }
    if (ok)
        for (const Part &p : parts_) memcpy(p.dst, wc_->rb + p.at, p.bytes);
    parts_.clear();
    used_ = 0;
    return ok;
}

void *WaveCache::stage(const void *src, size_t bytes, size_t at) {
    if (at + bytes > pinned_cap) return nullptr;  // sized by the caller (reserve below)
    memcpy(pinned + at, src, bytes);
    return pinned + at;
}

// Room for a wave's uploads in the pinned staging buffer (grown by half again; the old one
// is freed only when the stream is idle, which it is between waves).
static bool stage_reserve(WaveCache *wc, size_t bytes, cudaStream_t s) {
    if (!wc) return false;
    if (bytes <= wc->pinned_cap) return true;
    const size_t cap = std::max(bytes, wc->pinned_cap + wc->pinned_cap / 2);
    char *p = nullptr;
    if (cudaMallocHost(&p, cap) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (wc->pinned) {
        cudaStreamSynchronize(s);
        cudaFreeHost(wc->pinned);
    }
    wc->pinned = p;
    wc->pinned_cap = cap;
    return true;
}

// One shared-memory bin pass through a CUDA graph: the wave's shape (pass, non-empty bins,
// dense width class, profiling) picks a graph captured once with fixed grids on the
// persistent workspace, so the launches and their arguments are the same for every wave
// of that shape; the kernels read their bins' row counts from the device. Falls back to
// plain launches if a capture fails.
static void run_pass_graph(int pass, const PassArgs &a, const uint32_t *host_counts, int64_t dense_cols,
                           const Tuning &tun, cudaStream_t s, Prof *prof, WaveCache &wc) {
    uint32_t mask = 0;
    for (int b = 0; b < NBINS; b++)
        if (b != B_GLOBAL && host_counts[b]) mask |= 1u << b;
    if (!mask) return;
    int64_t dcls = 0;
    if (mask & (1u << B_DENSE)) {
        dcls = 32;
        while (dcls < dense_cols) dcls <<= 1;
    }
    const bool timed = prof && prof->on;
    const uint64_t key = (uint64_t)pass | ((uint64_t)mask << 1) | ((uint64_t)dcls << 16) | ((uint64_t)timed << 62);
    auto it = wc.graphs.find(key);
    if (it == wc.graphs.end()) {
        g_attrs_only = true;  // shared-memory attributes outside the capture
        run_pass(pass, a, host_counts, dcls, tun, s, nullptr, true);
        g_attrs_only = false;
        cudaGraph_t g = nullptr;
        cudaGraphExec_t ex = nullptr;
        const uint64_t l0 = g_launches.load();
        cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        const char *step = "begin capture";
        if (e == cudaSuccess) {
            g_capturing = true;
            run_pass(pass, a, host_counts, dcls, tun, s, prof, true);
            g_capturing = false;
            e = cudaStreamEndCapture(s, &g);
            step = "end capture";
        }
        if (e == cudaSuccess) {
            e = cudaGraphInstantiate(&ex, g, 0);
            step = "instantiate";
        }
        if (g) cudaGraphDestroy(g);
        g_launches.fetch_sub(g_launches.load() - l0);  // replays are counted below
        if (e != cudaSuccess) {
            fprintf(stderr, "mp: bin-pass graph %s: %s; launching directly from now on\n", step,
                    cudaGetErrorString(e));
            cudaGetLastError();
            wc.broken = true;
            run_pass(pass, a, host_counts, dense_cols, tun, s, prof);
            return;
        }
        it = wc.graphs.emplace(key, ex).first;
        wc.captures++;
    }
    cudaGraphLaunch(it->second, s);
    g_launches.fetch_add((uint64_t)__builtin_popcount(mask), std::memory_order_relaxed);
    wc.replays++;
}

static void prof_collect(Prof *prof, int pass, const BinTally &t) {
    if (!prof || !prof->on) return;
    // the split-row walks of this pass: symbolic and dense after pass 0, numeric after pass 1
    // (and the symbolic walk again when pass 1 recounts bitmap rows it could not keep)
    for (int m = 0; m < 3; m++) {
        if (!prof->wn[m] || (pass == 0 && m == 1) || (pass == 1 && m == 2)) continue;
        if (prof->wmiss[m]) {  // some launches went untimed: this wave's walk is left out
            prof->wn[m] = 0;
            prof->wmiss[m] = false;
            continue;
        }
        double ms = 0.0;
        for (int k = 0; k < prof->wn[m]; k++) {
            float x = 0.f;
            if (cudaEventElapsedTime(&x, prof->wev[m][k][0], prof->wev[m][k][1]) == cudaSuccess) ms += x;
            else cudaGetLastError();
        }
        if (pass == 0) prof->wlast[m][0] = (double)t.wbytes[m], prof->wlast[m][1] = (double)t.wprods[m];
        const bool again = pass == 1 && m == 0;  // the recount walks pass 0's bytes once more
        KStat &w = prof->walk[m];
        w.launches += (uint64_t)prof->wn[m];
        w.ms += ms;
        w.bytes += again ? prof->wlast[0][0] : (double)t.wbytes[m];
        w.prods += again ? prof->wlast[0][1] : (double)t.wprods[m];
        prof->wn[m] = 0;
    }
    const bool pooled = prof->pool_ran[pass];
    prof->pool_ran[pass] = false;
    for (int b = 0; b < NBINS; b++) {
        if (!t.counts[b]) continue;
        if (b != B_GLOBAL && !prof->full() && !(pooled && pool_bin(b))) continue;  // not timed at this level
        if (pooled && pool_bin(b)) {  // timed as one launch below
            prof->pool[pass].bytes += (double)t.bytes[b];
            prof->pool[pass].prods += (double)t.prods[b];
            continue;
        }
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, prof->ev[pass][b][0], prof->ev[pass][b][1]) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        KStat &k = prof->k[pass][b];
        k.launches++;
        k.ms += ms;
        k.bytes += (double)t.bytes[b];
        k.prods += (double)t.prods[b];
    }
    if (pooled) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, prof->pev[pass][0], prof->pev[pass][1]) != cudaSuccess) {
            cudaGetLastError();
            return;
        }
        prof->pool[pass].launches++;
        prof->pool[pass].ms += ms;
    }
}

// Events around one stage of a wave (e = 0 start, 1 end); stage_collect adds the stages
// recorded since the last call once the wave has synchronised.
static inline void stage_mark(Prof *prof, int st, int e, cudaStream_t s) {
    if (!prof || !prof->full()) return;
    cudaEventRecord(prof->sev[st][e], s);
    if (e) prof->srec[st] = true;
}

static void stage_collect(Prof *prof) {
    if (!prof || !prof->full()) return;
    for (int st = 0; st < Prof::NSTAGE; st++) {
        if (!prof->srec[st]) continue;
        prof->srec[st] = false;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, prof->sev[st][0], prof->sev[st][1]) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        prof->stage[st].launches++;
        prof->stage[st].ms += ms;
    }
}

static inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// State of the GLOBAL bin of one wave across its two passes. Rows [0, nd) of list take
// dense slots (one pass in the symbolic phase, a fill in the numeric phase); rows
// [nd, R) take bitmap rounds.
struct Glob {
    int64_t R = 0, nw = 0, per_round = 0, rounds = 0, nd = 0, dcols = 0;
    int64_t nwd = 0;  // bitmap words per dense-row slot
    uint32_t *list = nullptr;  // the bin's rows, dense-row candidates first
    int64_t *item_off = nullptr, *xbase = nullptr, *xoff = nullptr, *ys = nullptr;
    const uint64_t *prod = nullptr;
    const uint32_t *ymx = nullptr;  // longest masked Y row per wave row
    int ew_max = -1;                // rows with ymx <= ew_max are split by X entries
    int64_t ech = 4096;             // ... into items of this many entries
    int64_t items_ub = 0;           // an upper bound on the work items of all its rows
    int kinds = 1;                  // bit 0: rows split by products present, bit 1: by entries
    uint2 *bmr = nullptr, *dbmr = nullptr;
    unsigned long long *dval = nullptr;
    int64_t *csum = nullptr;   // rank pass: per chunk of a row slot, its set bits, then its offset
    bool kept = false;         // bitmaps of a single round survive into the numeric pass
};

// The rank pass of rows [ga.r0, ga.r1): chunk sums, per-row scans (the rows' sizes, or the
// numeric pass's size check), chunk ranks.
static void glob_rank(const Glob &g, const PassArgs &a, const GlobArgs &ga, int numeric, unsigned grid,
                      cudaStream_t s) {
    const int64_t nch = (ga.nw + RCH - 1) / RCH;
    const int64_t chunks = (ga.r1 - ga.r0) * nch;
    const unsigned gc = (unsigned)std::max<int64_t>(1, std::min<int64_t>(chunks, (int64_t)grid * 2));
    kl(k_glob_csum, gc, GNT, 0, s, ga, nch, g.csum);
    kl(k_glob_rowscan, (unsigned)std::max<int64_t>(1, std::min<int64_t>(grid_for((ga.r1 - ga.r0) * 32, 256), grid)),
       256, 0, s, a, ga, nch, g.csum, numeric);
    kl(k_glob_crank, gc, GNT, 0, s, ga, nch, (const int64_t *)g.csum);
}

static void glob_release(Glob &g, Alloc &al, cudaStream_t s) {
    if (g.list) al.free(g.list, s);
    if (g.item_off) al.free(g.item_off, s);
    if (g.xbase) al.free(g.xbase, s);
    if (g.xoff) al.free(g.xoff, s);
    if (g.ys) al.free(g.ys, s);
    if (g.bmr) al.free(g.bmr, s);
    if (g.dbmr) al.free(g.dbmr, s);
    if (g.dval) al.free(g.dval, s);
    if (g.csum) al.free(g.csum, s);
    g = Glob{};
}

// The split-row kernel in the variant the tuning asks for: warp-level product walk (default)
// or block-staged walk, combining table on or off, and for the count-adding modes 4 or 6
// resident blocks per SM (64 or 40 registers a thread).
// One block per resident slot: the blocks loop over the work items.
// kinds: bit 0 when the GLOBAL rows include rows split by products, bit 1 rows split by X
// entries (the warp-level walk launches one variant for each kind present).
template <int MODE>
static void glob_set(const Tuning &tun, cudaStream_t s, const PassArgs &a, const GlobArgs &ga, int kinds) {
    const int occ = MODE == G_SYM ? 8 : tun.glob_occ >= 6 ? 6 : 4;
    const unsigned grid = (unsigned)(tun.sm_count * occ);
#define GLOB_SET_VARIANT(K)                                                       \
    if constexpr (MODE == G_SYM) {                                                \
        if (tun.combine) kl(K<MODE, true, 8>, grid, GNT, 0, s, a, ga);           \
        else kl(K<MODE, false, 8>, grid, GNT, 0, s, a, ga);                      \
    } else if (occ == 6) {                                                        \
        if (tun.combine) kl(K<MODE, true, 6>, grid, GNT, 0, s, a, ga);           \
        else kl(K<MODE, false, 6>, grid, GNT, 0, s, a, ga);                      \
    } else {                                                                      \
        if (tun.combine) kl(K<MODE, true, 4>, grid, GNT, 0, s, a, ga);           \
        else kl(K<MODE, false, 4>, grid, GNT, 0, s, a, ga);                      \
    }
    using KF = void (*)(PassArgs, GlobArgs);
    auto both = [&](KF k_pw, KF k_ew, unsigned grid, size_t sm) {
        if (kinds & 1) kl(k_pw, grid, GNT, sm, s, a, ga);
        if (kinds & 2) kl(k_ew, grid, GNT, sm, s, a, ga);
    };
    if constexpr (MODE == G_DENSE) {
        // dense rows narrow enough for a shared-memory row: as many blocks as fit per SM
        if (tun.lbs && tun.dsm_cols > 0 && ga.dcols > 0 && ga.dcols <= tun.dsm_cols) {
            const KF k0 = k_glob_lbs<G_DENSE, false, 6, true, false>, k1 = k_glob_lbs<G_DENSE, false, 6, true, true>;
            const size_t sm = (size_t)ga.dcols * 8;
            int nb = 0;
            if (cudaFuncSetAttribute(k0, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) == cudaSuccess &&
                cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) == cudaSuccess &&
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k0, GNT, sm) == cudaSuccess && nb > 0) {
                both(k0, k1, (unsigned)std::min<int64_t>((int64_t)tun.sm_count * nb, ga.items_ub), sm);
                return;
            }
            cudaGetLastError();  // no room: the global-row walk below
        }
    }
    if (tun.lbs) {
        // the bitmap pass at 6 blocks per SM (40 registers), the count-adding passes at
        // lbs_occ (4: 64 registers; 6 spills a few values of the shuffle walk)
        const int lo = MODE == G_SYM || tun.lbs_occ >= 6 ? 6 : 4;
        const unsigned g = (unsigned)std::min<int64_t>((int64_t)tun.sm_count * lo, ga.items_ub);
        if (lo == 6) {
            if (tun.combine) both(k_glob_lbs<MODE, true, 6, false, false>, k_glob_lbs<MODE, true, 6, false, true>, g, 0);
            else both(k_glob_lbs<MODE, false, 6, false, false>, k_glob_lbs<MODE, false, 6, false, true>, g, 0);
        } else {
            if (tun.combine) both(k_glob_lbs<MODE, true, 4, false, false>, k_glob_lbs<MODE, true, 4, false, true>, g, 0);
            else both(k_glob_lbs<MODE, false, 4, false, false>, k_glob_lbs<MODE, false, 4, false, true>, g, 0);
        }
    } else {
        GLOB_SET_VARIANT(k_glob_set)
    }
#undef GLOB_SET_VARIANT
}

// One pass of the GLOBAL bin (all rounds). pass 0 counts, pass 1 writes the rows.
// A split-row walk launch, bracketed by CUDA events when profiling (its own time, apart
// from the set-up and rank kernels of the pass).
template <int MODE>
static void glob_walk(const Tuning &tun, cudaStream_t s, const PassArgs &a, const GlobArgs &ga, int kinds, Prof *prof) {
    const int m = MODE == G_SYM ? 0 : MODE == G_NUM ? 1 : 2;
    const bool timed = prof && prof->on && prof->wn[m] < Prof::WALK_EV;
    if (prof && prof->on && !timed) prof->wmiss[m] = true;  // more rounds than events: no stat
    if (timed) cudaEventRecord(prof->wev[m][prof->wn[m]][0], s);
    glob_set<MODE>(tun, s, a, ga, kinds);
    if (timed) cudaEventRecord(prof->wev[m][prof->wn[m]++][1], s);
}

static void glob_pass(int pass, Glob &g, const PassArgs &a, const Tuning &tun, cudaStream_t s, Prof *prof) {
    const unsigned grid = (unsigned)tun.sm_count * 8;
    if (prof && prof->on) cudaEventRecord(prof->ev[pass][B_GLOBAL][0], s);
    if (g.nd) {
        const GlobArgs ga{g.list, g.item_off,  g.xbase, g.xoff, g.ys,  g.prod,         g.ymx,        g.ew_max,
                          g.ech,  g.items_ub, 0,       g.nd,   g.dbmr, g.nwd,          tun.short_walk, tun.seg_walk,
                          g.dval, g.dcols};
        const int64_t words = g.nd * g.nwd;
        if (pass == 0) {
            cudaMemsetAsync(g.dval, 0, (size_t)g.nd * g.dcols * 8, s);
            glob_walk<G_DENSE>(tun, s, a, ga, g.kinds, prof);
            kl(k_glob_dscan, (unsigned)std::max<int64_t>(1, std::min<int64_t>(grid_for(words * 32, 256), grid * 4)),
               256, 0, s, ga);
            glob_rank(g, a, ga, 0, grid, s);
        } else {
            kl(k_glob_dfill, (unsigned)std::max<int64_t>(1, std::min<int64_t>(grid_for(words, 256), grid * 4)), 256,
               0, s, a, ga);
        }
    }
    for (int64_t r0 = g.nd; r0 < g.R; r0 += g.per_round) {
        const GlobArgs ga{g.list, g.item_off, g.xbase, g.xoff, g.ys, g.prod, g.ymx, g.ew_max, g.ech, g.items_ub,
                          r0,     std::min(g.R, r0 + g.per_round), g.bmr, g.nw, tun.short_walk, tun.seg_walk, nullptr, 0};
        const int64_t rows = ga.r1 - ga.r0;
        if (pass == 0 || !g.kept) {
            cudaMemsetAsync(g.bmr, 0, (size_t)rows * g.nw * 8, s);
            glob_walk<G_SYM>(tun, s, a, ga, g.kinds, prof);
            glob_rank(g, a, ga, pass, grid, s);
        }
        if (pass == 1) {
            const int64_t words = rows * g.nw;
            kl(k_glob_fill, (unsigned)std::max<int64_t>(1, std::min<int64_t>(grid_for(words, 256), grid * 4)), 256, 0,
               s, a, ga);
            glob_walk<G_NUM>(tun, s, a, ga, g.kinds, prof);
        }
    }
    if (prof && prof->on) cudaEventRecord(prof->ev[pass][B_GLOBAL][1], s);
}

// ------------------------------------------------------------------ host orchestration

int spgemm_wave(const std::vector<WaveIn> &in, Alloc &al, const Tuning &tun, cudaStream_t s,
                uint64_t max_result_bytes, std::vector<WaveOut> &out, Prof *prof, bool symbolic_only,
                WaveCache *wc, Budget *bud) {
    const int w = (int)in.size();
    out.assign(w, WaveOut{});
    if (w == 0) return MP_OK;
    if (prof) {  // events left by a wave that failed part-way are not this wave's
        for (int m = 0; m < 3; m++) prof->wn[m] = 0, prof->wmiss[m] = false;
        for (int st = 0; st < Prof::NSTAGE; st++) prof->srec[st] = false;
    }
    struct Small {
        BinTally tally;
        uint32_t offsets[NBINS + 1];
        uint32_t cursors[NBINS];
        uint32_t n_long, n_mid, n_huge;
        unsigned pool_head;  // the pooled pass's work queue
    };
    std::vector<Prod> hp(w);
    std::vector<int64_t> row0s(w + 1, 0);
    int64_t dense_cols = 0, max_cols = 0, ml_total = 0;
    std::vector<int64_t> ml_off(w, -1);  // offset of each product's masked-length array, or -1
    for (int p = 0; p < w; p++) {
        const WaveIn &x = in[p];
        Prod &P = hp[p];
        // (a row mask on X usually leaves few rows: then the lengths would cost more to make
        // than they save)
        if (tun.row_lens && !x.rm && x.X.nnz >= x.Y.nrows && x.Y.nrows > 0) {
            ml_off[p] = ml_total;
            ml_total += (x.Y.nrows + 63) / 64 * 64;  // 256-byte aligned slices
        }
        P.X = x.X;
        P.Y = x.Y;
        P.rm = x.rm;
        P.km = x.km;
        P.cm = x.cm;
        P.ymax = x.ymax;
        P.row0 = row0s[p];
        // a row list much shorter than X's rows: the product runs over the listed rows only
        const bool listed = tun.row_lists && x.X.arows && x.X.narows * 8 <= x.X.nrows;
        P.arows = listed ? x.X.arows : nullptr;
        P.nwr = listed ? x.X.narows : x.X.nrows;
        row0s[p + 1] = row0s[p] + P.nwr;
        if (x.Y.ncols <= tun.dense_max_cols) dense_cols = std::max<int64_t>(dense_cols, x.Y.ncols);
        max_cols = std::max<int64_t>(max_cols, x.Y.ncols);
    }
    const int64_t M = row0s[w];
    // with graphs, the workspace persists (laid out for the cache's capacities, grown by
    // half again when a wave needs more; growing drops the graphs captured on it)
    const bool graphs = wc && tun.graphs && !wc->broken;
    int64_t Mc = M;
    int wcp = w;
    if (graphs) {
        if (!wc->ws || M > wc->mcap || w > wc->wcap) {
            wc->drop_graphs();
            if (wc->ws) al.free(wc->ws, s);
            wc->ws = nullptr;
            wc->mcap = std::max<int64_t>(M, wc->mcap + wc->mcap / 2);
            wc->wcap = std::max(w, 2 * wc->wcap);
        }
        Mc = wc->mcap;
        wcp = wc->wcap;
    }
    // workspace: prod u64[M], symbolic and numeric bins i8[M] each, row list u32[M], long rows (one block each) and
    // longer rows (several blocks each) u32[M] each, rowprod i32[M],
    // wave nnz / row pointers i64[M+1], X row sums f64[M], longest masked Y rows u32[M],
    // product descriptors, row0s, per-product stats, two Smalls (M, w: the capacities when
    // the workspace persists)
    const size_t o_prod = 0;
    const size_t o_bin = align256(o_prod + (size_t)Mc * 8);
    const size_t o_nbin = align256(o_bin + (size_t)Mc);
    const size_t o_list = align256(o_nbin + (size_t)Mc);
    const size_t o_long = align256(o_list + (size_t)Mc * 4);
    const size_t o_huge = align256(o_long + (size_t)Mc * 4);
    const size_t o_mid = align256(o_huge + (size_t)Mc * 4);
    const size_t o_rowprod = align256(o_mid + (size_t)Mc * 4);
    const size_t o_grp = align256(o_rowprod + (size_t)Mc * 4);
    const size_t o_xsum = align256(o_grp + (size_t)(Mc + 1) * 8);
    const size_t o_ymx = align256(o_xsum + (size_t)Mc * 8);
    const size_t o_prods = align256(o_ymx + (size_t)Mc * 4);
    const size_t o_row0s = align256(o_prods + sizeof(Prod) * wcp);
    const size_t o_ps = align256(o_row0s + (size_t)(wcp + 1) * 8);
    const size_t o_small = align256(o_ps + sizeof(PStat) * wcp);
    const size_t ws_bytes = align256(o_small + sizeof(Small) * 2);
    // rows split by X entries need the warp-level walk (the staged walk reads product offsets)
    const BinArgs ba{tun.dense_max_cols, tun.dense_min_u, tun.force_class, tun.heavy, tun.warp_prod,
                     tun.glob_dense,     tun.lane_rows,   tun.lbs ? tun.ew_max : -1};
    int rc = MP_OK;
    Glob gl;
    PassArgs pa{};
    Small h_sym, h_num;
    std::vector<PStat> hps(w);
    std::vector<int64_t> reserved(w, 0);  // budget bytes charged for each product's result
    auto unreserve = [&](int p) {
        if (bud && reserved[p]) bud->unreserve(reserved[p]);
        reserved[p] = 0;
    };
    char *ws = graphs ? wc->ws : (char *)al.alloc(ws_bytes, s);
    if (graphs && !ws) ws = wc->ws = (char *)al.alloc(ws_bytes, s);
    if (!ws) return MP_ERR_NOMEM;
    auto ws_free = [&] {
        if (!graphs) al.free(ws, s);
    };
    uint64_t *prod = (uint64_t *)(ws + o_prod);
    int8_t *bin = (int8_t *)(ws + o_bin);
    int8_t *nbin = (int8_t *)(ws + o_nbin);
    uint32_t *list = (uint32_t *)(ws + o_list);
    uint32_t *long_rows = (uint32_t *)(ws + o_long);
    uint32_t *huge_rows = (uint32_t *)(ws + o_huge);
    uint32_t *mid_rows = (uint32_t *)(ws + o_mid);
    int32_t *rowprod = (int32_t *)(ws + o_rowprod);
    int64_t *grp = (int64_t *)(ws + o_grp);
    double *xsum = (double *)(ws + o_xsum);
    uint32_t *ymx = (uint32_t *)(ws + o_ymx);
    Prod *dprods = (Prod *)(ws + o_prods);
    int64_t *drow0s = (int64_t *)(ws + o_row0s);
    PStat *ps = (PStat *)(ws + o_ps);
    Small *sm_sym = (Small *)(ws + o_small);
    Small *sm_num = sm_sym + 1;
    uint32_t *mlbuf = nullptr;  // masked Y-row lengths of the products that use them (row work only)
    auto fail = [&](int code) {
        if (mlbuf) al.free(mlbuf, s);
        for (int p = 0; p < w; p++) {
            unreserve(p);
            if (hp[p].rp) al.free(hp[p].rp, s);
            if (hp[p].ci) al.free(hp[p].ci, s);
            if (hp[p].val) al.free(hp[p].val, s);
        }
        glob_release(gl, al, s);
        ws_free();
        out.assign(w, WaveOut{});
        return code;
    };
    auto cuda_ok = [&](cudaError_t e, const char *what) {
        if (e == cudaSuccess) return true;
        fprintf(stderr, "mp: %s: %s\n", what, cudaGetErrorString(e));
        return false;
    };
    Readback rbk(wc, s);  // the bin tallies, sizes and flags the host reads
    if (ml_total) {
        mlbuf = (uint32_t *)al.alloc((size_t)ml_total * 4, s);
        if (!mlbuf) return fail(MP_ERR_NOMEM);
        for (int p = 0; p < w; p++) {
            if (ml_off[p] < 0) continue;
            uint32_t *ml = mlbuf + ml_off[p];
            hp[p].ml = ml;
            const int64_t n = hp[p].Y.nrows;
            kl(k_masked_len, (unsigned)std::min<int64_t>(grid_for(n, 256), (int64_t)tun.sm_count * 16), 256, 0, s,
               (const int64_t *)hp[p].Y.rp, hp[p].km, n, ml);
        }
    }
    for (int p = 0; p < w; p++) {
        hp[p].rp = (int64_t *)al.alloc((size_t)(in[p].X.nrows + 1) * 8, s);
        if (!hp[p].rp) return fail(MP_ERR_NOMEM);
        if (in[p].X.nrows == 0 && !cuda_ok(cudaMemsetAsync(hp[p].rp, 0, 8, s), "memset")) return fail(MP_ERR_CUDA);
    }
    // the uploads from pinned staging when there is one (no wait for the stream), else from
    // the host vectors
    const size_t up_prods = align256(sizeof(Prod) * w), up_rows = (size_t)(w + 1) * 8;
    const bool staged = stage_reserve(wc, up_prods + up_rows, s);
    const void *src_prods = staged ? wc->stage(hp.data(), sizeof(Prod) * w, 0) : hp.data();
    const void *src_rows = staged ? wc->stage(row0s.data(), up_rows, up_prods) : row0s.data();
    if (!cuda_ok(cudaMemcpyAsync(dprods, src_prods, sizeof(Prod) * w, cudaMemcpyHostToDevice, s), "upload") ||
        !cuda_ok(cudaMemcpyAsync(drow0s, src_rows, up_rows, cudaMemcpyHostToDevice, s), "upload") ||
        !cuda_ok(cudaMemsetAsync(ps, 0, sizeof(PStat) * w, s), "memset") ||
        !cuda_ok(cudaMemsetAsync(sm_sym, 0, sizeof(Small) * 2, s), "memset"))
        return fail(MP_ERR_CUDA);

    pa.prods = dprods;
    pa.rowprod = rowprod;
    pa.list = list;
    pa.nnz = grp;
    pa.ps = ps;
    // 1. row work, symbolic bins, rows grouped by bin
    if (M > 0) {
        const unsigned gr = (unsigned)std::min<int64_t>(grid_for(M, 256), (int64_t)tun.sm_count * 16);
        stage_mark(prof, 0, 0, s);
        kl(k_rowprod, gr, 256, 0, s, drow0s, w, M, rowprod);
        const unsigned g = (unsigned)std::min<int64_t>(grid_for(M, 256), (int64_t)tun.sm_count * 32);
        kl(k_rowwork, g, 256, 0, s, dprods, rowprod, M, prod, xsum, ymx, long_rows, huge_rows, &sm_sym->n_long,
           &sm_sym->n_huge, mid_rows, &sm_sym->n_mid);
        // the mid queue holds at most M rows: no more warps than that
        kl(k_rowwork_mid, (unsigned)std::min<int64_t>((int64_t)tun.sm_count * 8, (M + 7) / 8), 256, 0, s, dprods, rowprod,
           prod, xsum, ymx,
           (const uint32_t *)mid_rows, (const uint32_t *)&sm_sym->n_mid);
        // (huge rows are shared by the whole grid, so this one stays full size)
        kl(k_rowwork_long, (unsigned)tun.sm_count * 4, 256, 0, s, dprods, rowprod, prod, xsum, ymx,
           (const uint32_t *)long_rows, (const uint32_t *)huge_rows, (const uint32_t *)&sm_sym->n_long,
           (const uint32_t *)&sm_sym->n_huge);
        if (mlbuf) {  // only the row work reads the masked lengths (stream-ordered free)
            al.free(mlbuf, s);
            mlbuf = nullptr;
        }
        stage_mark(prof, 0, 1, s);
        stage_mark(prof, 1, 0, s);
        kl(k_binassign, gr, 256, 0, s, dprods, rowprod, prod, (const double *)xsum, (const uint32_t *)ymx, M, ba, bin,
           grp, &sm_sym->tally, ps);
        kl(k_bin_fill, gr, 256, 0, s, bin, M, (const uint32_t *)sm_sym->tally.counts, sm_sym->offsets, sm_sym->cursors,
           list);
        stage_mark(prof, 1, 1, s);
    }
    if (!rbk.get(&h_sym, sm_sym, sizeof(Small)) || !rbk.sync()) return fail(MP_ERR_CUDA);
    pa.counts = sm_sym->tally.counts;
    pa.offsets = sm_sym->offsets;
    pa.pool_head = &sm_sym->pool_head;
    // GLOBAL bin set-up: its rows, work items, product offsets, bitmap rounds
    gl.R = h_sym.tally.counts[B_GLOBAL];
    if (gl.R) stage_mark(prof, 2, 0, s);
    if (gl.R) {
        // dense rows: as many of the qualifying rows as the dense scratch holds at once, each
        // slot as wide as the widest output among them; bitmap slots as wide as the widest
        // output among the rows that take bitmap rounds
        const int64_t nd_all = std::min<int64_t>(gl.R, (int64_t)h_sym.tally.gdense);
        gl.dcols = nd_all ? (int64_t)h_sym.tally.gd_cols : 0;
        gl.nwd = (gl.dcols + 31) / 32;
        const uint64_t dslot = (uint64_t)gl.dcols * 8 + (uint64_t)gl.nwd * 8;
        gl.nd = nd_all ? std::min<int64_t>(nd_all, (int64_t)(tun.dense_scratch_cap / dslot)) : 0;
        gl.nw = (std::max<int64_t>((int64_t)h_sym.tally.gb_cols, gl.nd < nd_all ? gl.dcols : 0) + 31) / 32;
        const int64_t rb = gl.R - gl.nd;
        const uint64_t cap = tun.scratch_cap ? tun.scratch_cap : (4ull << 30);
        gl.per_round = rb ? std::max<int64_t>(1, std::min<int64_t>(rb, (int64_t)(cap / ((uint64_t)gl.nw * 8)))) : 0;
        gl.rounds = rb ? (rb + gl.per_round - 1) / gl.per_round : 0;
        gl.kept = gl.rounds == 1;
        // product offsets only for the X entries of rows split by products
        const int64_t xtot = (int64_t)h_sym.tally.gx_pw;
        gl.prod = prod;
        gl.ymx = ymx;
        gl.ew_max = ba.ew_max;
        gl.ech = std::max<int64_t>(256, tun.ech / 256 * 256);
        gl.kinds = (xtot > 0 ? 1 : 0) | ((uint64_t)xtot < h_sym.tally.xent[B_GLOBAL] ? 2 : 0);
        gl.items_ub = (int64_t)(h_sym.tally.prods[B_GLOBAL] / PCH + h_sym.tally.xent[B_GLOBAL] / gl.ech) + 2 * gl.R + 1;
        gl.list = (uint32_t *)al.alloc((size_t)gl.R * 4, s);
        gl.item_off = (int64_t *)al.alloc((size_t)(gl.R + 1) * 8, s);
        gl.xbase = (int64_t *)al.alloc((size_t)(gl.R + 1) * 8, s);
        gl.xoff = (int64_t *)al.alloc((size_t)(xtot + 1) * 8, s);
        gl.ys = (int64_t *)al.alloc((size_t)(xtot + 1) * 8, s);
        if (!gl.list || !gl.item_off || !gl.xbase || !gl.xoff || !gl.ys) return fail(MP_ERR_NOMEM);
        if (rb) {
            gl.bmr = (uint2 *)al.alloc((size_t)gl.per_round * gl.nw * 8, s);
            if (!gl.bmr) return fail(MP_ERR_NOMEM);
        }
        if (gl.nd) {
            gl.dbmr = (uint2 *)al.alloc((size_t)gl.nd * gl.nwd * 8, s);
            gl.dval = (unsigned long long *)al.alloc((size_t)gl.nd * gl.dcols * 8, s);
            if (!gl.dbmr || !gl.dval) return fail(MP_ERR_NOMEM);
        }
        {
            const int64_t nch = (gl.nw + RCH - 1) / RCH, nchd = (gl.nwd + RCH - 1) / RCH;
            gl.csum = (int64_t *)al.alloc((size_t)std::max<int64_t>(gl.per_round * nch, gl.nd * nchd) * 8 + 8, s);
            if (!gl.csum) return fail(MP_ERR_NOMEM);
        }
        if (nd_all) {
            // qualifying rows first (the two counters live in the first bitmap/rank pair,
            // which the symbolic pass overwrites, until the partition is done)
            uint32_t *cnt = (uint32_t *)(gl.nd ? gl.dbmr : gl.bmr);
            if (!cuda_ok(cudaMemsetAsync(cnt, 0, 8, s), "memset")) return fail(MP_ERR_CUDA);
            kl(k_glob_split, (unsigned)std::min<int64_t>(grid_for(gl.R, 256), 1024), 256, 0, s,
               (const Prod *)dprods, (const int32_t *)rowprod, (const uint32_t *)(list + h_sym.offsets[B_GLOBAL]),
               gl.R, (const uint64_t *)prod, (const uint32_t *)ymx, ba.ew_max, tun.glob_dense, gl.nd, gl.list, cnt, bin,
               &sm_sym->tally);
        } else if (!cuda_ok(cudaMemcpyAsync(gl.list, list + h_sym.offsets[B_GLOBAL], (size_t)gl.R * 4,
                                            cudaMemcpyDeviceToDevice, s), "copy")) {
            return fail(MP_ERR_CUDA);
        }
        kl(k_glob_prep, (unsigned)std::min<int64_t>(grid_for(gl.R, 256), 1024), 256, 0, s, pa, gl.list, gl.R, prod,
           (const uint32_t *)ymx, ba.ew_max, gl.ech, gl.xbase, gl.item_off);
        if (scan_i64(gl.item_off, gl.item_off, gl.R, al, s) || scan_i64(gl.xbase, gl.xbase, gl.R, al, s))
            return fail(MP_ERR_NOMEM);
        if (xtot > 0) {
            kl(k_glob_xlen,
               (unsigned)std::max<int64_t>(1, std::min<int64_t>((xtot + XCH - 1) / XCH, (int64_t)tun.sm_count * 8)), 256,
               0, s, pa, (const uint32_t *)gl.list, gl.R, (const int64_t *)gl.xbase, gl.xoff, gl.ys);
            if (scan_i64(gl.xoff, gl.xoff, xtot, al, s)) return fail(MP_ERR_NOMEM);
        }
    }
    if (gl.R) stage_mark(prof, 2, 1, s);
    // 2-3. symbolic pass, wave row pointers, per-product row pointers and sizes
    if (M > 0) {
        if (graphs) run_pass_graph(0, pa, h_sym.tally.counts, dense_cols, tun, s, prof, *wc);
        else run_pass(0, pa, h_sym.tally.counts, dense_cols, tun, s, prof);
    }
    if (gl.R) glob_pass(0, gl, pa, tun, s, prof);
    stage_mark(prof, 3, 0, s);
    if (scan_i64(grp, grp, M, al, s)) return fail(MP_ERR_NOMEM);
    if (M > 0) kl(k_rebase, (unsigned)std::min<int64_t>(grid_for(M, 256), (int64_t)tun.sm_count * 16), 256, 0, s,
                  dprods, rowprod, grp, M, ps);
    {
        int64_t rows = -1;  // the widest product over a row list
        for (int p = 0; p < w; p++)
            if (hp[p].arows) rows = std::max<int64_t>(rows, in[p].X.nrows + 1);
        for (int p0 = 0; rows > 0 && p0 < w; p0 += 65535)  // grid y is at most 65,535
            kl(k_rp_expand,
               dim3((unsigned)std::min<int64_t>(grid_for(rows, 256), (int64_t)tun.sm_count * 8),
                    (unsigned)std::min(w - p0, 65535)),
               256, 0, s, (const Prod *)(dprods + p0), (const int64_t *)grp);
    }
    stage_mark(prof, 3, 1, s);
    // 3b. numeric bins ahead of the output allocation, read back with the sizes (a product
    // the host then refuses sends the binning round again)
    const bool ahead = !symbolic_only && M > 0;
    const unsigned gnum = (unsigned)std::min<int64_t>(grid_for(M, 256), (int64_t)tun.sm_count * 16);
    auto numeric_bins = [&](int pre) {
        stage_mark(prof, 4, 0, s);
        kl(k_numbin, gnum, 256, 0, s, dprods, rowprod, grp, prod, (const uint32_t *)ymx, M, ba, (const int8_t *)bin,
           nbin, pre, &sm_num->tally, ps);
        kl(k_bin_fill, gnum, 256, 0, s, nbin, M, (const uint32_t *)sm_num->tally.counts, sm_num->offsets,
           sm_num->cursors, list);
        stage_mark(prof, 4, 1, s);
    };
    if (ahead) numeric_bins(1);
    if (!rbk.get(hps.data(), ps, sizeof(PStat) * w) || !rbk.get(&h_sym.tally, &sm_sym->tally, sizeof(h_sym.tally)) ||
        (ahead && !rbk.get(&h_num, sm_num, sizeof(Small))) || !rbk.sync())
        return fail(MP_ERR_CUDA);
    prof_collect(prof, 0, h_sym.tally);
    if (symbolic_only) {
        stage_collect(prof);
        for (int p = 0; p < w; p++) {
            WaveOut &o = out[p];
            o.products = hps[p].prods;
            for (int b = 0; b < NBINS; b++) o.sym_bins[b] = hps[p].sym_bins[b];
            if (hps[p].err) o.status = (hps[p].err & ERR_OVERFLOW) ? MP_ERR_OVERFLOW : MP_ERR_INTERNAL;
            o.m.nrows = in[p].X.nrows;
            o.m.ncols = in[p].Y.ncols;
            o.m.nnz = in[p].X.nrows ? hps[p].nnz : 0;
            al.free(hp[p].rp, s);
        }
        glob_release(gl, al, s);
        ws_free();
        return MP_OK;
    }
    // per product: status, size guard, output arrays
    bool any_out = false, rebin = false;
    for (int p = 0; p < w; p++) {
        WaveOut &o = out[p];
        o.products = hps[p].prods;
        for (int b = 0; b < NBINS; b++) o.sym_bins[b] = hps[p].sym_bins[b];
        const int64_t nnz = in[p].X.nrows ? hps[p].nnz : 0;
        if (hps[p].err) {
            o.status = (hps[p].err & ERR_OVERFLOW) ? MP_ERR_OVERFLOW : MP_ERR_INTERNAL;
            continue;
        }
        Mat m;
        m.nrows = in[p].X.nrows;
        m.ncols = in[p].Y.ncols;
        m.nnz = nnz;
        if (max_result_bytes && m.bytes() > max_result_bytes) {
            o.status = MP_ERR_TOO_LARGE;
            rebin = true;  // its rows were binned
            continue;
        }
        if (bud) {
            if (bud->reserve((int64_t)m.bytes())) {
                o.status = MP_ERR_BUDGET;
                rebin = true;
                continue;
            }
            reserved[p] = (int64_t)m.bytes();
        }
        hp[p].ci = (int32_t *)al.alloc((size_t)std::max<int64_t>(nnz, 1) * 4, s);
        hp[p].val = (uint64_t *)al.alloc((size_t)std::max<int64_t>(nnz, 1) * 8, s);
        if (!hp[p].ci || !hp[p].val) return fail(MP_ERR_NOMEM);
        if (nnz) any_out = true;
        // split rows add their counts with atomics: the counts start at zero (one streaming
        // memset of the product's counts instead of zeros written entry by entry)
        if (nnz && hps[p].sym_bins[B_GLOBAL] &&
            !cuda_ok(cudaMemsetAsync(hp[p].val, 0, (size_t)nnz * 8, s), "memset"))
            return fail(MP_ERR_CUDA);
    }
    // 4. numeric pass; products that failed keep null outputs and their rows are skipped
    if (any_out) {
        // the stream synchronised since the first upload: the staging buffer is free again
        const void *src = staged ? wc->stage(hp.data(), sizeof(Prod) * w, 0) : hp.data();
        if (!cuda_ok(cudaMemcpyAsync(dprods, src, sizeof(Prod) * w, cudaMemcpyHostToDevice, s), "upload"))
            return fail(MP_ERR_CUDA);
        if (rebin || !ahead) {
            // bins again without the refused products' rows: tallies, queue head and each
            // product's numeric bin counts and flag start from zero
            if (!cuda_ok(cudaMemsetAsync(sm_num, 0, sizeof(Small), s), "memset") ||
                !cuda_ok(cudaMemset2DAsync(&ps[0].nerr, sizeof(PStat), 0, sizeof(uint32_t) * (NBINS + 1), (size_t)w,
                                           s),
                         "memset"))
                return fail(MP_ERR_CUDA);
            numeric_bins(0);
            if (!rbk.get(&h_num, sm_num, sizeof(Small)) || !rbk.sync()) return fail(MP_ERR_CUDA);
        }
        pa.counts = sm_num->tally.counts;
        pa.offsets = sm_num->offsets;
        pa.pool_head = &sm_num->pool_head;
        if (graphs) run_pass_graph(1, pa, h_num.tally.counts, dense_cols, tun, s, prof, *wc);
        else run_pass(1, pa, h_num.tally.counts, dense_cols, tun, s, prof);
        if (gl.R) glob_pass(1, gl, pa, tun, s, prof);
        if (!rbk.get(hps.data(), ps, sizeof(PStat) * w) || !rbk.sync()) return fail(MP_ERR_CUDA);
        prof_collect(prof, 1, h_num.tally);
    }
    stage_collect(prof);
    if (!cuda_ok(cudaGetLastError(), "launch")) return fail(MP_ERR_CUDA);
    for (int p = 0; p < w; p++) {
        WaveOut &o = out[p];
        for (int b = 0; b < NBINS; b++) o.num_bins[b] = hps[p].num_bins[b];
        const uint32_t e = hps[p].err | hps[p].nerr;
        if (!o.status && e) o.status = (e & ERR_OVERFLOW) ? MP_ERR_OVERFLOW : MP_ERR_INTERNAL;
        if (o.status) {
            unreserve(p);
            if (hp[p].rp) al.free(hp[p].rp, s);
            if (hp[p].ci) al.free(hp[p].ci, s);
            if (hp[p].val) al.free(hp[p].val, s);
            continue;
        }
        o.m.nrows = in[p].X.nrows;
        o.m.ncols = in[p].Y.ncols;
        o.m.nnz = in[p].X.nrows ? hps[p].nnz : 0;
        // every count is at most (row sum of X) * (bound on Y's values); the row sums are
        // double sums, so the bound carries a relative margin far above their rounding
        double xsmax;
        memcpy(&xsmax, &hps[p].xsmax, sizeof xsmax);
        const double vb = xsmax * (double)in[p].ymax * (1.0 + 1e-6);
        o.m.vmax = hps[p].unsafe || !(vb < 9.2e18) ? UINT64_MAX : (uint64_t)vb + 1;
        o.m.rp = hp[p].rp;
        o.m.ci = hp[p].ci;
        o.m.val = hp[p].val;
        if (hp[p].arows && in[p].xrows_hold) {  // the result's non-empty rows are on its X's list
            o.m.arows = hp[p].arows;
            o.m.narows = hp[p].nwr;
            o.m.arows_hold = in[p].xrows_hold;
        }
    }
    glob_release(gl, al, s);
    ws_free();
    return rc;
}

}  // namespace mp
