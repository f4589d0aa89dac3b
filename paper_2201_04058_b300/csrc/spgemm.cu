// Sparse x sparse products of the metapath chain on sm_103a.
//
// One product C = diag(rm) X diag(km) Y diag(cm) is the constrained-adjacency product of
// Sec. 2 (Problem 1 and the M_c * A that follows it) for one split of the chain: X and Y
// are either base 0/1 adjacency matrices (Def. 1) or earlier uint64 results, and the
// masks are the 0/1 diagonals M of Def. 3 stored as bitmaps. Counts are exact uint64;
// a count beyond 2^64 - 1 raises ERR_OVERFLOW instead of wrapping.
//
// Pipeline (Gustavson row by row, two passes):
//   1. rowwork:  prod_i = sum_{k in X_i, km[k]} nnz(Y_k), the scalar products of row i
//                (an upper bound of nnz(C_i)), and the row's symbolic bin;
//   2. bin fill: row ids grouped by bin (warp-aggregated atomics);
//   3. symbolic: exact nnz(C_i) per bin: warp-per-row or block-per-row hash sets in
//                shared memory, a dense shared-memory bitmap when C is narrow, or a
//                bitmap in global scratch for very long rows;
//   4. scan:     row pointers of C (warp-shuffle block scans, three phases);
//   5. numeric:  rows re-binned by their exact nnz; accumulate (col -> count) with
//                shared-memory 64-bit atomics (hash or dense) or in global scratch,
//                then emit the row in ascending column order (bitonic sort for hash
//                bins, an in-order sweep for dense ones).
// Every row's products are enumerated by a group of threads that scans the lengths of
// the Y rows it needs and then walks the flattened product list with a stride of the
// group size, so consecutive threads read consecutive entries of a Y row.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <utility>

#include "../../include/mp.h"
#include "internal.h"

namespace mp {

std::atomic<uint64_t> g_launches{0};

bool Prof::init() {
    for (int p = 0; p < 2; p++)
        for (int b = 0; b < NBINS; b++)
            for (int e = 0; e < 2; e++)
                if (cudaEventCreate(&ev[p][b][e]) != cudaSuccess) return false;
    return true;
}

void Prof::destroy() {
    for (int p = 0; p < 2; p++)
        for (int b = 0; b < NBINS; b++)
            for (int e = 0; e < 2; e++)
                if (ev[p][b][e]) cudaEventDestroy(ev[p][b][e]);
}

// Every kernel launch of the library goes through kl(), which counts it.
template <class... KArgs, class... Args>
static inline void kl(void (*k)(KArgs...), dim3 g, dim3 b, size_t smem, cudaStream_t s, Args &&...args) {
    k<<<g, b, smem, s>>>(std::forward<Args>(args)...);
    g_launches.fetch_add(1, std::memory_order_relaxed);
}

static constexpr uint32_t EMPTY = 0xffffffffu;
static constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ bool bit_of(const uint32_t *m, uint32_t j) {
    return m == nullptr || ((__ldg(m + (j >> 5)) >> (j & 31)) & 1u);
}

__device__ __forceinline__ uint32_t hash_of(uint32_t j) { return j * 0x9E3779B1u; }

__host__ __device__ __forceinline__ int next_pow2_log(uint64_t x) {
    // smallest e with 2^e >= x (x >= 1)
    int e = 0;
    while ((1ull << e) < x) e++;
    return e;
}

// Bin of a row with prod Gustavson products and at most u output entries (u >= 1), for
// an output of ncols columns. Hash tables are sized T >= 2u (load factor <= 1/2). Rows
// with more than `heavy` products, or whose output is too wide for a shared-memory
// table, go to GLOBAL, where the row is split over many blocks.
__host__ __device__ __forceinline__ int bin_for(uint64_t prod, uint64_t u, int64_t ncols, int dense_max_cols,
                                                int dense_min_u, uint64_t heavy, int force) {
    if ((uint64_t)ncols < u) u = (uint64_t)ncols;
    const bool dense_ok = ncols <= dense_max_cols;
    int e = next_pow2_log(2 * u);
    if (e < 5) e = 5;
    switch (force) {
        case MP_BIN_WARP_HASH:
            if (e <= 10) return B_W32 + (e - 5);
            if (e <= 13) return B_K2048 + (e - 11);
            return dense_ok ? B_DENSE : B_GLOBAL;
        case MP_BIN_BLOCK_HASH:
            if (e <= 13) return B_K2048 + (e < 11 ? 0 : e - 11);
            return dense_ok ? B_DENSE : B_GLOBAL;
        case MP_BIN_DENSE:
            return dense_ok ? B_DENSE : B_GLOBAL;
        case MP_BIN_GLOBAL:
            return B_GLOBAL;
        default:
            break;
    }
    if (prod > heavy) return B_GLOBAL;
    if (dense_ok && u >= (uint64_t)dense_min_u) return B_DENSE;
    if (e <= 10) return B_W32 + (e - 5);
    if (e <= 13) return B_K2048 + (e - 11);
    return dense_ok ? B_DENSE : B_GLOBAL;
}

// ------------------------------------------------------------------ masks

__global__ void k_mask_fill(uint32_t *m, int64_t nw, uint32_t v, int64_t n) {
    int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (w >= nw) return;
    uint32_t x = v;
    if (v && w == nw - 1 && (n & 31)) x = (1u << (n & 31)) - 1u;  // no bits past n
    m[w] = x;
}

// One thread per node; a warp ballot forms one 32-node word.
__global__ void k_mask_and_range(uint32_t *m, const int32_t *prop, int64_t n, int64_t lo,
                                 int64_t hi) {
    int64_t base = (blockIdx.x * (int64_t)blockDim.x) & ~31ll;
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    bool ok = false;
    if (i < n) {
        int64_t v = prop ? (int64_t)__ldg(prop + i) : i;
        ok = v >= lo && v <= hi;
    }
    uint32_t word = __ballot_sync(FULL, ok);
    if ((threadIdx.x & 31) == 0 && i < n) m[(base + (threadIdx.x & ~31)) >> 5] &= word;
}

__global__ void k_set_bits(uint32_t *m, const uint32_t *set, int64_t len, int64_t n) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= len) return;
    uint32_t j = set[t];
    if ((int64_t)j < n) atomicOr(m + (j >> 5), 1u << (j & 31));
}

__global__ void k_and_words(uint32_t *m, const uint32_t *t, int64_t nw) {
    int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (w < nw) m[w] &= t[w];
}

static inline unsigned grid_for(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

void mask_fill(uint32_t *m, int64_t n, bool ones, cudaStream_t s) {
    int64_t nw = (n + 31) / 32;
    if (nw) kl(k_mask_fill, grid_for(nw, 256), 256, 0, s, m, nw, ones ? FULL : 0u, n);
}

void mask_and_range(uint32_t *m, const int32_t *prop, int64_t n, int64_t lo, int64_t hi,
                    cudaStream_t s) {
    if (n) kl(k_mask_and_range, grid_for(n, 256), 256, 0, s, m, prop, n, lo, hi);
}

void mask_and_set(uint32_t *m, uint32_t *tmp, const uint32_t *set, int64_t len, int64_t n,
                  cudaStream_t s) {
    int64_t nw = (n + 31) / 32;
    if (!nw) return;
    kl(k_mask_fill, grid_for(nw, 256), 256, 0, s, tmp, nw, 0u, n);
    if (len) kl(k_set_bits, grid_for(len, 256), 256, 0, s, tmp, set, len, n);
    kl(k_and_words, grid_for(nw, 256), 256, 0, s, m, tmp, nw);
}

// nnz of diag(rm) A diag(cm). Each lane takes one of 32 consecutive rows; rows longer
// than 16 entries are counted by the whole warp, and rows longer than 8192 entries are
// queued and counted by every block (k_masked_nnz_long).
__global__ void k_masked_nnz(DCsr A, const uint32_t *rm, const uint32_t *cm, unsigned long long *out,
                             uint32_t *long_rows, uint32_t *n_long) {
    const int lane = threadIdx.x & 31;
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long c = 0;
    for (int64_t i0 = w * 32; i0 < A.nrows; i0 += nwarps * 32) {
        const int64_t i = i0 + lane;
        int64_t b = 0, e = 0;
        if (i < A.nrows && bit_of(rm, (uint32_t)i)) {
            b = A.rp[i];
            e = A.rp[i + 1];
        }
        if (!cm) {
            c += (unsigned long long)(e - b);
            continue;
        }
        const bool mine = e - b <= 16;
        if (mine)
            for (int64_t p = b; p < e; p++) c += bit_of(cm, (uint32_t)__ldg(A.ci + p));
        if (e - b > 8192) long_rows[atomicAdd(n_long, 1u)] = (uint32_t)i;
        unsigned coop = __ballot_sync(FULL, !mine && e - b <= 8192);
        while (coop) {
            const int src = __ffs(coop) - 1;
            coop &= coop - 1;
            const int64_t bb = __shfl_sync(FULL, b, src), ee = __shfl_sync(FULL, e, src);
            for (int64_t p = bb + lane; p < ee; p += 32) c += bit_of(cm, (uint32_t)__ldg(A.ci + p));
        }
    }
    for (int d = 16; d; d >>= 1) c += __shfl_down_sync(FULL, c, d);
    if (lane == 0 && c) atomicAdd(out, c);
}

__global__ void k_masked_nnz_long(DCsr A, const uint32_t *cm, unsigned long long *out, const uint32_t *long_rows,
                                  const uint32_t *n_long) {
    const uint32_t n = *n_long;
    unsigned long long c = 0;
    for (uint32_t r = 0; r < n; r++) {
        const uint32_t i = long_rows[r];
        for (int64_t p = A.rp[i] + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < A.rp[i + 1];
             p += (int64_t)gridDim.x * blockDim.x)
            c += bit_of(cm, (uint32_t)__ldg(A.ci + p));
    }
    for (int d = 16; d; d >>= 1) c += __shfl_down_sync(FULL, c, d);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

void masked_nnz(const DCsr &A, const uint32_t *rm, const uint32_t *cm, unsigned long long *out, uint32_t *long_rows,
                uint32_t *n_long, cudaStream_t s) {
    if (!A.nrows) return;
    unsigned g = (unsigned)std::min<int64_t>(grid_for(A.nrows * 32, 256), 148 * 16);
    kl(k_masked_nnz, g, 256, 0, s, A, rm, cm, out, long_rows, n_long);
    if (cm) kl(k_masked_nnz_long, 148 * 4, 256, 0, s, A, cm, out, long_rows, n_long);
}

// ------------------------------------------------------------------ scan

static constexpr int SCAN_T = 512, SCAN_I = 8, SCAN_TILE = SCAN_T * SCAN_I;

template <int T>
__device__ __forceinline__ int64_t block_excl_scan(int64_t v, int64_t *warp_sums, int64_t *total) {
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t x = v;
    for (int d = 1; d < 32; d <<= 1) {
        int64_t y = __shfl_up_sync(FULL, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int64_t s = lane < T / 32 ? warp_sums[lane] : 0;
        int64_t t = s;
        for (int d = 1; d < 32; d <<= 1) {
            int64_t y = __shfl_up_sync(FULL, t, d);
            if (lane >= d) t += y;
        }
        if (lane < T / 32) warp_sums[lane] = t - s;
        if (lane == 31) *total = t;
    }
    __syncthreads();
    int64_t r = warp_sums[wid] + x - v;
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(SCAN_T) k_scan_tiles(const int64_t *in, int64_t n, int64_t *part) {
    __shared__ int64_t ws[32];
    __shared__ int64_t tot;
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_I;
    int64_t s = 0;
#pragma unroll
    for (int t = 0; t < SCAN_I; t++)
        if (base + t < n) s += in[base + t];
    block_excl_scan<SCAN_T>(s, ws, &tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_scan_parts(int64_t *part, int64_t nb) {
    __shared__ int64_t ws[32];
    __shared__ int64_t tot;
    int64_t carry = 0;
    for (int64_t b0 = 0; b0 < nb; b0 += 1024) {
        int64_t i = b0 + threadIdx.x;
        int64_t v = i < nb ? part[i] : 0;
        int64_t e = block_excl_scan<1024>(v, ws, &tot);
        if (i < nb) part[i] = carry + e;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) part[nb] = carry;
}

__global__ void __launch_bounds__(SCAN_T) k_scan_apply(const int64_t *in, int64_t *out, int64_t n,
                                                       const int64_t *part, int64_t nb) {
    __shared__ int64_t ws[32];
    __shared__ int64_t tot;
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_I;
    int64_t v[SCAN_I];
    int64_t s = 0;
#pragma unroll
    for (int t = 0; t < SCAN_I; t++) {
        v[t] = base + t < n ? in[base + t] : 0;
        s += v[t];
    }
    int64_t e = block_excl_scan<SCAN_T>(s, ws, &tot) + part[blockIdx.x];
    // all reads of this tile are done (the scan synchronised), so out may alias in
#pragma unroll
    for (int t = 0; t < SCAN_I; t++) {
        if (base + t < n) out[base + t] = e;
        e += v[t];
    }
    if (blockIdx.x == nb - 1 && threadIdx.x == 0) out[n] = part[nb];
}

void scan_i64(const int64_t *in, int64_t *out, int64_t n, Alloc &al, cudaStream_t s) {
    if (n == 0) {
        cudaMemsetAsync(out, 0, sizeof(int64_t), s);
        return;
    }
    int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    int64_t *part = (int64_t *)al.alloc((size_t)(nb + 1) * sizeof(int64_t), s);
    kl(k_scan_tiles, (unsigned)nb, SCAN_T, 0, s, in, n, part);
    kl(k_scan_parts, 1, 1024, 0, s, part, nb);
    kl(k_scan_apply, (unsigned)nb, SCAN_T, 0, s, in, out, n, part, nb);
    al.free(part, s);
}

// ------------------------------------------------------------------ row work + bins

struct BinArgs {
    int64_t ncols;
    int dense_max_cols, dense_min_u, force;
    uint64_t heavy;
};

// Per-bin tallies of one pass: rows, X entries, Gustavson products, output entries and the
// algorithmic bytes of the bin's kernel.
struct BinTally {
    uint32_t counts[NBINS];
    unsigned long long xent[NBINS], prods[NBINS], outn[NBINS], bytes[NBINS];
};

static constexpr int64_t LONGX = 8192;  // X rows longer than this are summed by all blocks

// prod_i = sum over the masked X_i entries of the Y row lengths. Each lane takes one of 32
// consecutive rows; rows longer than 16 entries are summed by the whole warp, one after
// the other, and rows longer than LONGX are queued for k_rowwork_long.
__global__ void k_rowwork(DCsr X, DCsr Y, const uint32_t *rm, const uint32_t *km, uint64_t *prod,
                          uint32_t *long_rows, uint32_t *n_long) {
    const int lane = threadIdx.x & 31;
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i0 = w * 32; i0 < X.nrows; i0 += nwarps * 32) {
        const int64_t i = i0 + lane;
        int64_t b = 0, e = 0;
        if (i < X.nrows && bit_of(rm, (uint32_t)i)) {
            b = X.rp[i];
            e = X.rp[i + 1];
        }
        uint64_t s = 0;
        const bool mine = e - b <= 16;
        if (mine)
            for (int64_t p = b; p < e; p++) {
                const int32_t k = __ldg(X.ci + p);
                if (bit_of(km, (uint32_t)k)) s += (uint64_t)(__ldg(Y.rp + k + 1) - __ldg(Y.rp + k));
            }
        if (e - b > LONGX) long_rows[atomicAdd(n_long, 1u)] = (uint32_t)i;
        unsigned coop = __ballot_sync(FULL, !mine && e - b <= LONGX);
        while (coop) {
            const int src = __ffs(coop) - 1;
            coop &= coop - 1;
            const int64_t bb = __shfl_sync(FULL, b, src), ee = __shfl_sync(FULL, e, src);
            uint64_t c = 0;
            for (int64_t p = bb + lane; p < ee; p += 32) {
                const int32_t k = __ldg(X.ci + p);
                if (bit_of(km, (uint32_t)k)) c += (uint64_t)(__ldg(Y.rp + k + 1) - __ldg(Y.rp + k));
            }
            for (int d = 16; d; d >>= 1) c += __shfl_xor_sync(FULL, c, d);
            if (lane == src) s = c;
        }
        if (i < X.nrows) prod[i] = (e - b > LONGX) ? 0 : s;
    }
}

// The queued long rows: every block takes a strided share of every long row's entries.
__global__ void k_rowwork_long(DCsr X, DCsr Y, const uint32_t *km, uint64_t *prod, const uint32_t *long_rows,
                               const uint32_t *n_long) {
    __shared__ unsigned long long red[32];
    const uint32_t n = *n_long;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (uint32_t r = 0; r < n; r++) {
        const uint32_t i = long_rows[r];
        const int64_t b = X.rp[i], e = X.rp[i + 1];
        unsigned long long s = 0;
        for (int64_t p = b + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < e;
             p += (int64_t)gridDim.x * blockDim.x) {
            const int32_t k = __ldg(X.ci + p);
            if (bit_of(km, (uint32_t)k)) s += (unsigned long long)(__ldg(Y.rp + k + 1) - __ldg(Y.rp + k));
        }
        for (int d = 16; d; d >>= 1) s += __shfl_xor_sync(FULL, s, d);
        if (lane == 0) red[wid] = s;
        __syncthreads();
        if (wid == 0) {
            s = lane < (int)(blockDim.x >> 5) ? red[lane] : 0;
            for (int d = 16; d; d >>= 1) s += __shfl_xor_sync(FULL, s, d);
            if (lane == 0 && s) atomicAdd((unsigned long long *)(prod + i), s);
        }
        __syncthreads();
    }
}

// Symbolic bin of every row from prod_i; rows without products get nnz_i = 0, no bin.
__global__ void k_binassign(const int64_t *xrp, const uint64_t *prod, int64_t m, BinArgs ba, int8_t *bin,
                            int64_t *nnz, BinTally *tally, unsigned long long *total_prod) {
    __shared__ uint32_t hc[NBINS];
    __shared__ unsigned long long hx[NBINS], hp[NBINS], hb[NBINS];
    __shared__ unsigned long long bsum;
    if (threadIdx.x < NBINS) {
        hc[threadIdx.x] = 0;
        hx[threadIdx.x] = 0;
        hp[threadIdx.x] = 0;
        hb[threadIdx.x] = 0;
    }
    if (threadIdx.x == 0) bsum = 0;
    __syncthreads();
    unsigned long long mysum = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t s = prod[i];
        int b = -1;
        if (s) {
            b = bin_for(s, s, ba.ncols, ba.dense_max_cols, ba.dense_min_u, ba.heavy, ba.force);
            const unsigned long long xe = (unsigned long long)(xrp[i + 1] - xrp[i]);
            atomicAdd(&hc[b], 1u);
            atomicAdd(&hx[b], xe);
            atomicAdd(&hp[b], (unsigned long long)s);
            // symbolic bytes: X row pointers + nnz write, per X entry its column id and the
            // two Y row pointers, per product one Y column id
            atomicAdd(&hb[b], 24ull + xe * 20ull + (unsigned long long)s * 4ull);
            mysum += s;
        } else {
            nnz[i] = 0;
        }
        bin[i] = (int8_t)b;
    }
    if (mysum) atomicAdd(&bsum, mysum);
    __syncthreads();
    const int t = threadIdx.x;
    if (t < NBINS && hc[t]) {
        atomicAdd(tally->counts + t, hc[t]);
        atomicAdd(tally->xent + t, hx[t]);
        atomicAdd(tally->prods + t, hp[t]);
        atomicAdd(tally->bytes + t, hb[t]);
    }
    if (t == 0 && bsum) atomicAdd(total_prod, bsum);
}

// Numeric bins from the exact row sizes (nnz = rp[i+1] - rp[i]); rows the symbolic pass
// put in GLOBAL stay there (their bitmaps give the output positions).
__global__ void k_numbin(const int64_t *rp, const int64_t *xrp, const uint64_t *prod, int64_t n, BinArgs ba,
                         bool x_val, bool y_val, int8_t *bin, BinTally *tally, uint32_t *err) {
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
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t z = rp[i + 1] - rp[i];
        int b = -1;
        if (z) {
            if (bin[i] == B_GLOBAL) {
                b = B_GLOBAL;
            } else {
                b = bin_for(prod[i], (uint64_t)z, ba.ncols, ba.dense_max_cols, ba.dense_min_u, ~0ull, ba.force);
                if (b == B_GLOBAL) atomicOr(err, ERR_PROBE);  // cannot happen: nnz <= the symbolic bound
            }
            const unsigned long long xe = (unsigned long long)(xrp[i + 1] - xrp[i]);
            const unsigned long long pr = prod[i];
            atomicAdd(&hc[b], 1u);
            atomicAdd(&hx[b], xe);
            atomicAdd(&hp[b], pr);
            atomicAdd(&ho[b], (unsigned long long)z);
            // numeric bytes: X and C row pointers, per X entry its column id (+ value) and
            // two Y row pointers, per product a Y column id (+ value), per output 12 bytes
            atomicAdd(&hb[b], 32ull + xe * (20ull + (x_val ? 8ull : 0ull)) + pr * (4ull + (y_val ? 8ull : 0ull)) +
                                  (unsigned long long)z * 12ull);
        }
        bin[i] = (int8_t)b;
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

// counts[0..NBINS) -> offsets[0..NBINS]; cursors reset.
__global__ void k_bin_offsets(const uint32_t *counts, uint32_t *offsets, uint32_t *cursors) {
    if (threadIdx.x == 0) {
        uint32_t s = 0;
        for (int b = 0; b < NBINS; b++) {
            offsets[b] = s;
            s += counts[b];
            cursors[b] = 0;
        }
        offsets[NBINS] = s;
    }
}

__global__ void k_bin_fill(const int8_t *bin, int64_t n, const uint32_t *offsets, uint32_t *cursors,
                           uint32_t *list) {
    int lane = threadIdx.x & 31;
    for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x; i0 < n; i0 += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = i0 + threadIdx.x;
        int b = i < n ? bin[i] : -1;
        unsigned peers = __match_any_sync(FULL, b);
        if (b >= 0) {
            int leader = __ffs(peers) - 1;
            uint32_t base = 0;
            if (lane == leader) base = atomicAdd(cursors + b, (uint32_t)__popc(peers));
            base = __shfl_sync(peers, base, leader);
            uint32_t rank = __popc(peers & ((1u << lane) - 1u));
            list[offsets[b] + base + rank] = (uint32_t)i;
        }
    }
}

// ------------------------------------------------------------------ product enumeration

// Per-group staging of one chunk of X_i: exclusive offsets of the masked Y row lengths,
// Y row starts and X values.
struct Stage {
    int64_t off;
    int64_t st;
    uint64_t a;
};

// Enumerate the scalar products of X entries [b, e) (all of row i, or a chunk of it) with a
// group of G threads (G = 32: one warp;
// G = blockDim: one block). f(j, v) is called once per product that passes cm, where v
// = X_ik * Y_kj (1 when both are pattern-only; values only read when VAL).
template <int G, bool VAL, class F>
__device__ __forceinline__ void for_each_product(const DCsr &X, const DCsr &Y, const uint32_t *km,
                                                 const uint32_t *cm, int64_t b, int64_t e, Stage *sg,
                                                 int64_t *gtot, int64_t *warp_sums, int t,
                                                 uint32_t *err, F &&f) {
    const int lane = t & 31;
    for (int64_t c0 = b; c0 < e; c0 += G) {
        const int64_t p = c0 + t;
        int64_t len = 0, st = 0;
        uint64_t a = 1;
        if (p < e) {
            const int32_t k = __ldg(X.ci + p);
            if (bit_of(km, (uint32_t)k)) {
                st = __ldg(Y.rp + k);
                len = __ldg(Y.rp + k + 1) - st;
                if (VAL && X.val) a = __ldg(X.val + p);
            }
        }
        int64_t excl, total;
        if (G == 32) {
            int64_t x = len;
            for (int d = 1; d < 32; d <<= 1) {
                int64_t y = __shfl_up_sync(FULL, x, d);
                if (lane >= d) x += y;
            }
            total = __shfl_sync(FULL, x, 31);
            excl = x - len;
        } else {
            excl = block_excl_scan<G>(len, warp_sums, gtot);
            total = *gtot;
        }
        sg[t].off = excl;
        sg[t].st = st;
        sg[t].a = a;
        if (G == 32) __syncwarp(); else __syncthreads();
        const int nent = (int)min((int64_t)G, e - c0);
        for (int64_t idx = t; idx < total; idx += G) {
            int lo = 0, hi = nent - 1;
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if (sg[mid].off <= idx) lo = mid; else hi = mid - 1;
            }
            const int64_t q = sg[lo].st + (idx - sg[lo].off);
            const uint32_t j = (uint32_t)__ldg(Y.ci + q);
            if (!bit_of(cm, j)) continue;
            uint64_t v = 1;
            if (VAL) {
                const uint64_t av = sg[lo].a;
                const uint64_t bv = Y.val ? __ldg(Y.val + q) : 1ull;
                v = av * bv;
                if (__umul64hi(av, bv)) atomicOr(err, ERR_OVERFLOW);
            }
            f(j, v);
        }
        if (G == 32) __syncwarp(); else __syncthreads();
    }
}

// ------------------------------------------------------------------ hash helpers

// Insert key j; returns 1 if it was not present. Linear probing, at most T probes.
__device__ __forceinline__ int hset_insert(uint32_t *keys, uint32_t mask, uint32_t j, uint32_t *err) {
    uint32_t h = hash_of(j) & mask;
    for (uint32_t n = 0; n <= mask; n++) {
        uint32_t cur = ((volatile uint32_t *)keys)[h];
        if (cur == j) return 0;
        if (cur == EMPTY) {
            uint32_t old = atomicCAS(keys + h, EMPTY, j);
            if (old == EMPTY) return 1;
            if (old == j) return 0;
        }
        h = (h + 1) & mask;
    }
    atomicOr(err, ERR_PROBE);
    return 0;
}

__device__ __forceinline__ void hmap_add(uint32_t *keys, unsigned long long *vals, uint32_t mask,
                                         uint32_t j, uint64_t v, uint32_t *err) {
    uint32_t h = hash_of(j) & mask;
    for (uint32_t n = 0; n <= mask; n++) {
        uint32_t cur = ((volatile uint32_t *)keys)[h];
        if (cur != j && cur == EMPTY) {
            uint32_t old = atomicCAS(keys + h, EMPTY, j);
            cur = (old == EMPTY) ? j : old;
        }
        if (cur == j) {
            unsigned long long old = atomicAdd(vals + h, (unsigned long long)v);
            if (old + v < old) atomicOr(err, ERR_OVERFLOW);
            return;
        }
        h = (h + 1) & mask;
    }
    atomicOr(err, ERR_PROBE);
}

// Bitonic sort (ascending keys, values follow) of n = 2^e entries by a group of G threads.
template <int G>
__device__ __forceinline__ void bitonic(uint32_t *keys, unsigned long long *vals, int n, int t) {
    for (int k = 2; k <= n; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int x = t; x < (n >> 1); x += G) {
                int i = (x / j) * 2 * j + (x % j);
                int l = i + j;
                bool up = (i & k) == 0;
                uint32_t ki = keys[i], kl = keys[l];
                if ((ki > kl) == up) {
                    keys[i] = kl;
                    keys[l] = ki;
                    unsigned long long t0 = vals[i];
                    vals[i] = vals[l];
                    vals[l] = t0;
                }
            }
            if (G == 32) __syncwarp(); else __syncthreads();
        }
    }
}

struct PassArgs {
    DCsr X, Y;
    const uint32_t *km, *cm;
    const uint32_t *list;
    const uint32_t *counts, *offsets;
    int64_t *nnz;          // symbolic output (per row)
    const int64_t *rp;     // numeric: row pointers of C
    int32_t *out_ci;
    uint64_t *out_val;
    uint32_t *err;
};

// ------------------------------------------------------------------ warp-hash bins

template <int T, int W>
__global__ void __launch_bounds__(W * 32) k_sym_warp(PassArgs a, int bin) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    Stage *sg = (Stage *)smem + wid * 32;
    uint32_t *keys = (uint32_t *)((Stage *)smem + W * 32) + wid * T;
    const uint32_t cnt = a.counts[bin], base = a.offsets[bin];
    for (uint32_t r = blockIdx.x * W + wid; r < cnt; r += gridDim.x * W) {
        const int64_t i = a.list[base + r];
        for (int s = lane; s < T; s += 32) keys[s] = EMPTY;
        __syncwarp();
        int c = 0;
        for_each_product<32, false>(a.X, a.Y, a.km, a.cm, a.X.rp[i], a.X.rp[i + 1], sg, nullptr, nullptr, lane, a.err,
                                    [&](uint32_t j, uint64_t) { c += hset_insert(keys, T - 1, j, a.err); });
        for (int d = 16; d; d >>= 1) c += __shfl_xor_sync(FULL, c, d);
        if (lane == 0) a.nnz[i] = c;
        __syncwarp();
    }
}

template <int T, int W>
__global__ void __launch_bounds__(W * 32) k_num_warp(PassArgs a, int bin) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    Stage *sg = (Stage *)smem + wid * 32;
    unsigned long long *vals = (unsigned long long *)((Stage *)smem + W * 32) + wid * T;
    uint32_t *keys = (uint32_t *)((unsigned long long *)((Stage *)smem + W * 32) + W * T) + wid * T;
    const uint32_t cnt = a.counts[bin], base = a.offsets[bin];
    for (uint32_t r = blockIdx.x * W + wid; r < cnt; r += gridDim.x * W) {
        const int64_t i = a.list[base + r];
        for (int s = lane; s < T; s += 32) {
            keys[s] = EMPTY;
            vals[s] = 0;
        }
        __syncwarp();
        for_each_product<32, true>(a.X, a.Y, a.km, a.cm, a.X.rp[i], a.X.rp[i + 1], sg, nullptr, nullptr, lane, a.err,
                                   [&](uint32_t j, uint64_t v) { hmap_add(keys, vals, T - 1, j, v, a.err); });
        __syncwarp();
        // compact occupied slots to the front (in place: writes never pass the read point)
        int n = 0;
        for (int s0 = 0; s0 < T; s0 += 32) {
            uint32_t k = keys[s0 + lane];
            unsigned long long v = vals[s0 + lane];
            unsigned bal = __ballot_sync(FULL, k != EMPTY);
            int pos = n + __popc(bal & ((1u << lane) - 1u));
            __syncwarp();
            if (k != EMPTY) {
                keys[pos] = k;
                vals[pos] = v;
            }
            n += __popc(bal);
            __syncwarp();
        }
        int P = 1;
        while (P < n) P <<= 1;
        for (int s = n + lane; s < P; s += 32) keys[s] = EMPTY;
        __syncwarp();
        bitonic<32>(keys, vals, P, lane);
        const int64_t o = a.rp[i];
        if (lane == 0 && a.rp[i + 1] - o != n) atomicOr(a.err, ERR_COUNT);
        const int m = (int)min((int64_t)n, a.rp[i + 1] - o);
        for (int s = lane; s < m; s += 32) {
            a.out_ci[o + s] = (int32_t)keys[s];
            a.out_val[o + s] = vals[s];
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------------ block-hash bins

template <int T, int NT>
__global__ void __launch_bounds__(NT) k_sym_block(PassArgs a, int bin) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int64_t warp_sums[32];
    __shared__ int64_t gtot;
    __shared__ int cnt_s;
    Stage *sg = (Stage *)smem;
    uint32_t *keys = (uint32_t *)(sg + NT);
    const uint32_t cnt = a.counts[bin], base = a.offsets[bin];
    for (uint32_t r = blockIdx.x; r < cnt; r += gridDim.x) {
        const int64_t i = a.list[base + r];
        for (int s = threadIdx.x; s < T; s += NT) keys[s] = EMPTY;
        if (threadIdx.x == 0) cnt_s = 0;
        __syncthreads();
        int c = 0;
        for_each_product<NT, false>(a.X, a.Y, a.km, a.cm, a.X.rp[i], a.X.rp[i + 1], sg, &gtot, warp_sums, threadIdx.x, a.err,
                                    [&](uint32_t j, uint64_t) { c += hset_insert(keys, T - 1, j, a.err); });
        for (int d = 16; d; d >>= 1) c += __shfl_xor_sync(FULL, c, d);
        if ((threadIdx.x & 31) == 0 && c) atomicAdd(&cnt_s, c);
        __syncthreads();
        if (threadIdx.x == 0) a.nnz[i] = cnt_s;
        __syncthreads();
    }
}

template <int T, int NT>
__global__ void __launch_bounds__(NT) k_num_block(PassArgs a, int bin) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int64_t warp_sums[32];
    __shared__ int64_t gtot;
    constexpr int PER = T / NT;  // slots per thread in the compaction
    Stage *sg = (Stage *)smem;
    unsigned long long *vals = (unsigned long long *)(sg + NT);
    uint32_t *keys = (uint32_t *)(vals + T);
    const uint32_t cnt = a.counts[bin], base = a.offsets[bin];
    for (uint32_t r = blockIdx.x; r < cnt; r += gridDim.x) {
        const int64_t i = a.list[base + r];
        for (int s = threadIdx.x; s < T; s += NT) {
            keys[s] = EMPTY;
            vals[s] = 0;
        }
        __syncthreads();
        for_each_product<NT, true>(a.X, a.Y, a.km, a.cm, a.X.rp[i], a.X.rp[i + 1], sg, &gtot, warp_sums, threadIdx.x, a.err,
                                   [&](uint32_t j, uint64_t v) { hmap_add(keys, vals, T - 1, j, v, a.err); });
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
        int64_t pos = block_excl_scan<NT>(c, warp_sums, &gtot);
        const int n = (int)gtot;
#pragma unroll
        for (int u = 0; u < PER; u++)
            if (k[u] != EMPTY) {
                keys[pos] = k[u];
                vals[pos] = v[u];
                pos++;
            }
        int P = 1;
        while (P < n) P <<= 1;
        __syncthreads();
        for (int s = n + threadIdx.x; s < P; s += NT) keys[s] = EMPTY;
        __syncthreads();
        bitonic<NT>(keys, vals, P, threadIdx.x);
        const int64_t o = a.rp[i];
        if (threadIdx.x == 0 && a.rp[i + 1] - o != n) atomicOr(a.err, ERR_COUNT);
        const int m = (int)min((int64_t)n, a.rp[i + 1] - o);
        for (int s = threadIdx.x; s < m; s += NT) {
            a.out_ci[o + s] = (int32_t)keys[s];
            a.out_val[o + s] = vals[s];
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ dense shared-memory bin

template <int NT>
__global__ void __launch_bounds__(NT) k_sym_dense(PassArgs a, int bin) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int64_t warp_sums[32];
    __shared__ int64_t gtot;
    __shared__ int cnt_s;
    Stage *sg = (Stage *)smem;
    uint32_t *bm = (uint32_t *)(sg + NT);
    const int nw = (int)((a.Y.ncols + 31) >> 5);
    const uint32_t cnt = a.counts[bin], base = a.offsets[bin];
    for (uint32_t r = blockIdx.x; r < cnt; r += gridDim.x) {
        const int64_t i = a.list[base + r];
        for (int s = threadIdx.x; s < nw; s += NT) bm[s] = 0;
        if (threadIdx.x == 0) cnt_s = 0;
        __syncthreads();
        int c = 0;
        for_each_product<NT, false>(a.X, a.Y, a.km, a.cm, a.X.rp[i], a.X.rp[i + 1], sg, &gtot, warp_sums, threadIdx.x, a.err,
                                    [&](uint32_t j, uint64_t) {
                                        uint32_t m = 1u << (j & 31);
                                        c += (atomicOr(bm + (j >> 5), m) & m) == 0;
                                    });
        for (int d = 16; d; d >>= 1) c += __shfl_xor_sync(FULL, c, d);
        if ((threadIdx.x & 31) == 0 && c) atomicAdd(&cnt_s, c);
        __syncthreads();
        if (threadIdx.x == 0) a.nnz[i] = cnt_s;
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
    const int ncols = (int)a.Y.ncols;
    const int per = (ncols + NT - 1) / NT;
    const uint32_t cnt = a.counts[bin], base = a.offsets[bin];
    for (uint32_t r = blockIdx.x; r < cnt; r += gridDim.x) {
        const int64_t i = a.list[base + r];
        for (int s = threadIdx.x; s < ncols; s += NT) acc[s] = 0;
        __syncthreads();
        for_each_product<NT, true>(a.X, a.Y, a.km, a.cm, a.X.rp[i], a.X.rp[i + 1], sg, &gtot, warp_sums, threadIdx.x, a.err,
                                   [&](uint32_t j, uint64_t v) {
                                       unsigned long long old = atomicAdd(acc + j, (unsigned long long)v);
                                       if (old + v < old) atomicOr(a.err, ERR_OVERFLOW);
                                   });
        __syncthreads();
        // in-order sweep: thread t owns columns [t*per, t*per + per)
        const int c0 = threadIdx.x * per;
        const int c1 = min(ncols, c0 + per);
        int c = 0;
        for (int s = c0; s < c1; s++) c += acc[s] != 0;
        int64_t pos = block_excl_scan<NT>(c, warp_sums, &gtot);
        const int64_t o = a.rp[i];
        const int64_t rowlen = a.rp[i + 1] - o;
        if (threadIdx.x == 0 && rowlen != gtot) atomicOr(a.err, ERR_COUNT);
        for (int s = c0; s < c1; s++) {
            unsigned long long v = acc[s];
            if (v) {
                if (pos < rowlen) {
                    a.out_ci[o + pos] = s;
                    a.out_val[o + pos] = v;
                }
                pos++;
            }
        }
        __syncthreads();
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
// Bitmaps and ranks are 8 bytes per 32 output columns per row; rows are processed in
// rounds that fit the scratch cap (one round keeps the symbolic bitmaps for the numeric
// pass, several rounds rebuild them).
static constexpr int64_t PCH = 16384;  // Gustavson products per work item
static constexpr int GNT = 256;        // threads per GLOBAL block
static constexpr int RW = 8;           // bitmap words per thread in the rank pass

struct GlobArgs {
    const uint32_t *list;     // rows of the GLOBAL bin, in symbolic order
    const int64_t *item_off;  // R+1 work-item offsets
    const int64_t *xbase;     // R+1 offsets of each row's X entries in xoff
    const int64_t *xoff;      // per X entry of a GLOBAL row: masked products before it
    const uint64_t *prod;     // prod_i per row
    int64_t r0, r1;           // rows of this round
    uint32_t *bm, *rank;      // (r1 - r0) slots of nw words each
    int64_t nw;
};

// Per GLOBAL row: its X entry count and its number of work items.
__global__ void k_glob_prep(const uint32_t *list, int64_t R, const int64_t *xrp, const uint64_t *prod, int64_t *xlen,
                            int64_t *items) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < R; r += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t i = list[r];
        xlen[r] = xrp[i + 1] - xrp[i];
        items[r] = ((int64_t)prod[i] + PCH - 1) / PCH;
    }
}

// xoff, step 1: the masked Y-row length of every X entry of every GLOBAL row, as one flat
// array (row r's entries start at xbase[r]); a device-wide exclusive scan (scan_i64) then
// turns it into each entry's global product offset.
__global__ void k_glob_xlen(DCsr X, DCsr Y, const uint32_t *km, const uint32_t *list, int64_t R,
                            const int64_t *xbase, int64_t *xoff) {
    const int64_t xtot = xbase[R];
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < xtot; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = R - 1;
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (__ldg(xbase + mid) <= e) lo = mid; else hi = mid - 1;
        }
        const uint32_t i = list[lo];
        const int64_t p = X.rp[i] + (e - xbase[lo]);
        const int32_t k = __ldg(X.ci + p);
        xoff[e] = bit_of(km, (uint32_t)k) ? __ldg(Y.rp + k + 1) - __ldg(Y.rp + k) : 0;
    }
}

// One work item per block iteration: products [s0, s1) of one row. The X entries that
// hold them are staged GNT at a time with their product offsets (from xoff); consecutive
// threads take consecutive products, so a long Y row is read coalesced.
template <bool NUM>
__global__ void __launch_bounds__(GNT) k_glob_set(PassArgs a, GlobArgs g) {
    __shared__ int64_t s_off[GNT + 1];
    __shared__ int64_t s_st[GNT];
    __shared__ uint64_t s_a[GNT];
    const int64_t t0 = g.item_off[g.r0], t1 = g.item_off[g.r1];
    for (int64_t t = t0 + blockIdx.x; t < t1; t += gridDim.x) {
        int64_t lo = g.r0, hi = g.r1 - 1;
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (g.item_off[mid] <= t) lo = mid; else hi = mid - 1;
        }
        const int64_t r = lo;
        const uint32_t i = g.list[r];
        const int64_t xb = a.X.rp[i], xe = a.X.rp[i + 1];
        const int64_t *xo = g.xoff + g.xbase[r];
        // product offsets are global across the GLOBAL rows: this row's start at xo[0]
        const int64_t total = __ldg(xo) + (int64_t)g.prod[i];
        const int64_t s0 = __ldg(xo) + (t - g.item_off[r]) * PCH;
        const int64_t s1 = min(total, s0 + PCH);
        // first X entry whose products reach s0: the last p with xo[p] <= s0
        int64_t plo = 0, phi = xe - xb - 1;
        while (plo < phi) {
            const int64_t mid = (plo + phi + 1) >> 1;
            if (__ldg(xo + mid) <= s0) plo = mid; else phi = mid - 1;
        }
        uint32_t *bm = g.bm + (r - g.r0) * g.nw;
        const uint32_t *rk = g.rank + (r - g.r0) * g.nw;
        unsigned long long *val = NUM ? (unsigned long long *)a.out_val + a.rp[i] : nullptr;
        for (int64_t c0 = xb + plo; c0 < xe; c0 += GNT) {
            const int64_t base = __ldg(xo + (c0 - xb));
            if (base >= s1) break;  // uniform: every thread reads the same base
            const int64_t p = c0 + threadIdx.x;
            const int nent = (int)min((int64_t)GNT, xe - c0);
            if (threadIdx.x < nent) {
                const int32_t k = __ldg(a.X.ci + p);
                s_off[threadIdx.x] = __ldg(xo + (p - xb)) - base;
                s_st[threadIdx.x] = __ldg(a.Y.rp + k);
                s_a[threadIdx.x] = (NUM && a.X.val) ? __ldg(a.X.val + p) : 1ull;
            }
            if (threadIdx.x == 0) s_off[nent] = (c0 + nent < xe ? __ldg(xo + (c0 + nent - xb)) : total) - base;
            __syncthreads();
            const int64_t f0 = max(s0 - base, (int64_t)0), f1 = min(s1 - base, s_off[nent]);
            for (int64_t f = f0 + threadIdx.x; f < f1; f += GNT) {
                int l = 0, h = nent - 1;
                while (l < h) {
                    const int mid = (l + h + 1) >> 1;
                    if (s_off[mid] <= f) l = mid; else h = mid - 1;
                }
                const int64_t q = s_st[l] + (f - s_off[l]);
                const uint32_t j = (uint32_t)__ldg(a.Y.ci + q);
                if (!bit_of(a.cm, j)) continue;
                if (!NUM) {
                    atomicOr(bm + (j >> 5), 1u << (j & 31));
                } else {
                    const uint64_t av = s_a[l];
                    const uint64_t bv = a.Y.val ? __ldg(a.Y.val + q) : 1ull;
                    const uint64_t v = av * bv;
                    if (__umul64hi(av, bv)) atomicOr(a.err, ERR_OVERFLOW);
                    const uint32_t w = j >> 5;
                    const uint32_t pos = __ldg(rk + w) + __popc(__ldg(bm + w) & ((1u << (j & 31)) - 1u));
                    const unsigned long long old = atomicAdd(val + pos, (unsigned long long)v);
                    if (old + v < old) atomicOr(a.err, ERR_OVERFLOW);
                }
            }
            __syncthreads();
        }
    }
}

__global__ void __launch_bounds__(GNT) k_glob_rank(PassArgs a, GlobArgs g, int numeric) {
    __shared__ int64_t warp_sums[32];
    __shared__ int64_t gtot;
    for (int64_t r = g.r0 + blockIdx.x; r < g.r1; r += gridDim.x) {
        const uint32_t i = g.list[r];
        const uint32_t *bm = g.bm + (r - g.r0) * g.nw;
        uint32_t *rk = g.rank + (r - g.r0) * g.nw;
        int64_t carry = 0;
        for (int64_t w0 = 0; w0 < g.nw; w0 += (int64_t)GNT * RW) {
            const int64_t wb = w0 + (int64_t)threadIdx.x * RW;
            int cnt[RW];
            int c = 0;
#pragma unroll
            for (int u = 0; u < RW; u++) {
                cnt[u] = wb + u < g.nw ? __popc(bm[wb + u]) : 0;
                c += cnt[u];
            }
            int64_t ex = carry + block_excl_scan<GNT>(c, warp_sums, &gtot);
#pragma unroll
            for (int u = 0; u < RW; u++) {
                if (wb + u < g.nw) rk[wb + u] = (uint32_t)ex;
                ex += cnt[u];
            }
            carry += gtot;
        }
        if (threadIdx.x == 0) {
            if (!numeric) a.nnz[i] = carry;
            else if (a.rp[i + 1] - a.rp[i] != carry) atomicOr(a.err, ERR_COUNT);
        }
    }
}

// One thread per bitmap word: the word's set bits become consecutive output entries.
__global__ void k_glob_fill(PassArgs a, GlobArgs g) {
    const int64_t total = (g.r1 - g.r0) * g.nw;
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < total; x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t slot = x / g.nw, w = x - slot * g.nw;
        uint32_t word = g.bm[x];
        if (!word) continue;
        const uint32_t i = g.list[g.r0 + slot];
        int64_t pos = a.rp[i] + g.rank[x];
        while (word) {
            const int b = __ffs(word) - 1;
            word &= word - 1;
            a.out_ci[pos] = (int32_t)(w * 32 + b);
            a.out_val[pos] = 0;
            pos++;
        }
    }
}

// ------------------------------------------------------------------ launch helpers

template <class K>
static void launch(K kern, unsigned grid, int nt, size_t smem, cudaStream_t s, const PassArgs &a, int bin) {
    if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kl(kern, grid, nt, smem, s, a, bin);
}

static unsigned blocks_for(uint32_t rows_upper, int rows_per_block, int max_blocks) {
    unsigned g = (unsigned)((rows_upper + rows_per_block - 1) / rows_per_block);
    return std::max(1u, std::min(g, (unsigned)max_blocks));
}

// Launch every non-empty shared-memory bin's kernel of one pass, each grid sized to its
// bin's rows (capped at a few blocks per SM; the kernels loop over their bin). With
// prof, CUDA events bracket each launch. GLOBAL is run separately (glob_pass).
static void run_pass(int pass, const PassArgs &a, const uint32_t *host_counts, int64_t ncols, const Tuning &tun,
                     cudaStream_t s, Prof *prof) {
    const bool numeric = pass == 1;
    const int sms = tun.sm_count;
    const size_t stage = sizeof(Stage);
    for (int b = 0; b < B_GLOBAL; b++) {
        const uint32_t rows = host_counts[b];
        if (!rows) continue;
        if (b == B_DENSE && ncols > tun.dense_max_cols) continue;
        if (prof && prof->on) cudaEventRecord(prof->ev[pass][b][0], s);
        switch (b) {
#define WARP_BIN(BIN, T, W)                                                                              \
    case BIN: {                                                                                          \
        unsigned g = blocks_for(rows, W, sms * 8);                                                       \
        if (numeric)                                                                                     \
            launch(k_num_warp<T, W>, g, W * 32, W * 32 * stage + (size_t)W * T * 12, s, a, BIN);        \
        else                                                                                             \
            launch(k_sym_warp<T, W>, g, W * 32, W * 32 * stage + (size_t)W * T * 4, s, a, BIN);         \
        break;                                                                                           \
    }
            WARP_BIN(B_W32, 32, 8)
            WARP_BIN(B_W64, 64, 8)
            WARP_BIN(B_W128, 128, 8)
            WARP_BIN(B_W256, 256, 8)
            WARP_BIN(B_W512, 512, 4)
            WARP_BIN(B_W1024, 1024, 4)
#undef WARP_BIN
#define BLOCK_BIN(BIN, T, NT)                                                              \
    case BIN: {                                                                            \
        unsigned g = blocks_for(rows, 1, sms * 4);                                         \
        if (numeric)                                                                       \
            launch(k_num_block<T, NT>, g, NT, NT * stage + (size_t)T * 12, s, a, BIN);     \
        else                                                                               \
            launch(k_sym_block<T, NT>, g, NT, NT * stage + (size_t)T * 4, s, a, BIN);      \
        break;                                                                             \
    }
            BLOCK_BIN(B_K2048, 2048, 256)
            BLOCK_BIN(B_K4096, 4096, 512)
            BLOCK_BIN(B_K8192, 8192, 1024)
#undef BLOCK_BIN
            case B_DENSE: {
                unsigned g = blocks_for(rows, 1, sms * 4);
                if (numeric)
                    launch(k_num_dense<256>, g, 256, 256 * stage + (size_t)ncols * 8, s, a, B_DENSE);
                else
                    launch(k_sym_dense<256>, g, 256, 256 * stage + (size_t)((ncols + 31) / 32) * 4, s, a, B_DENSE);
                break;
            }
        }
        if (prof && prof->on) cudaEventRecord(prof->ev[pass][b][1], s);
    }
}

static void prof_collect(Prof *prof, int pass, const BinTally &t, int64_t ncols, const Tuning &tun) {
    if (!prof || !prof->on) return;
    for (int b = 0; b < NBINS; b++) {
        if (!t.counts[b] || (b == B_DENSE && ncols > tun.dense_max_cols)) continue;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, prof->ev[pass][b][0], prof->ev[pass][b][1]) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        KStat &k = prof->k[pass][b];
        k.launches++;
        k.ms += ms;
        k.bytes += (double)t.bytes[b];
    }
}

static inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

#define CK(x)                                                                     \
    do {                                                                          \
        cudaError_t e_ = (x);                                                     \
        if (e_ != cudaSuccess) {                                                  \
            fprintf(stderr, "mp: %s failed: %s\n", #x, cudaGetErrorString(e_));   \
            rc = MP_ERR_CUDA;                                                     \
            goto fail;                                                            \
        }                                                                         \
    } while (0)

// State of the GLOBAL bin of one product across its two passes.
struct Glob {
    int64_t R = 0, nw = 0, per_round = 0, rounds = 0;
    uint32_t *list = nullptr;   // copy of the bin's rows in symbolic order
    int64_t *item_off = nullptr, *xbase = nullptr, *xoff = nullptr;
    const uint64_t *prod = nullptr;
    uint32_t *bm = nullptr, *rank = nullptr;
    bool kept = false;          // bitmaps of a single round survive into the numeric pass
};

static void glob_release(Glob &g, Alloc &al, cudaStream_t s) {
    if (g.list) al.free(g.list, s);
    if (g.item_off) al.free(g.item_off, s);
    if (g.xbase) al.free(g.xbase, s);
    if (g.xoff) al.free(g.xoff, s);
    if (g.bm) al.free(g.bm, s);
    if (g.rank) al.free(g.rank, s);
    g = Glob{};
}

// One pass of the GLOBAL bin (all rounds). pass 0 counts, pass 1 writes the rows.
static void glob_pass(int pass, Glob &g, const PassArgs &a, const Tuning &tun, cudaStream_t s, Prof *prof) {
    const unsigned grid = (unsigned)tun.sm_count * 8;
    if (prof && prof->on) cudaEventRecord(prof->ev[pass][B_GLOBAL][0], s);
    for (int64_t r0 = 0; r0 < g.R; r0 += g.per_round) {
        GlobArgs ga{g.list, g.item_off, g.xbase, g.xoff, g.prod, r0, std::min(g.R, r0 + g.per_round), g.bm, g.rank, g.nw};
        const int64_t rows = ga.r1 - ga.r0;
        if (pass == 0 || !g.kept) {
            cudaMemsetAsync(g.bm, 0, (size_t)rows * g.nw * 4, s);
            kl(k_glob_set<false>, grid, GNT, 0, s, a, ga);
            kl(k_glob_rank, (unsigned)std::min<int64_t>(rows, grid), GNT, 0, s, a, ga, pass);
        }
        if (pass == 1) {
            const int64_t words = rows * g.nw;
            kl(k_glob_fill, (unsigned)std::max<int64_t>(1, std::min<int64_t>(grid_for(words, 256), grid * 4)), 256, 0, s,
               a, ga);
            kl(k_glob_set<true>, grid, GNT, 0, s, a, ga);
        }
    }
    if (prof && prof->on) cudaEventRecord(prof->ev[pass][B_GLOBAL][1], s);
}

int spgemm(const DCsr &X, const DCsr &Y, const uint32_t *rm, const uint32_t *km, const uint32_t *cm,
           Alloc &al, Scratch &scr, const Tuning &tun, cudaStream_t s, uint64_t max_result_bytes,
           Mat *out, Stats *st, Prof *prof) {
    (void)scr;
    const int64_t m = X.nrows;
    out->nrows = m;
    out->ncols = Y.ncols;
    out->nnz = 0;
    struct Small {
        BinTally tally;
        uint32_t offsets[NBINS + 1];
        uint32_t cursors[NBINS];
        uint32_t err;
        uint32_t n_long;
        unsigned long long total_prod;
    };
    // workspace: prod u64[m], bins i8[m], row list u32[m], long-row list, two Small blocks
    const int64_t max_long = m;
    const size_t off_prod = 0;
    const size_t off_bin = align256(off_prod + (size_t)m * 8);
    const size_t off_list = align256(off_bin + (size_t)m);
    const size_t off_long = align256(off_list + (size_t)m * 4);
    const size_t off_small = align256(off_long + (size_t)max_long * 4);
    const size_t ws_bytes = align256(off_small + sizeof(Small) * 2);
    const BinArgs ba{Y.ncols, tun.dense_max_cols, tun.dense_min_u, tun.force_class, tun.heavy};
    int rc = MP_OK;
    int64_t nnz = 0;
    uint32_t err = 0;
    Small h_sym, h_num;
    PassArgs pa{};
    Glob gl;
    uint64_t *prod;
    int8_t *bin;
    uint32_t *list, *long_rows;
    Small *sm_sym, *sm_num;
    char *ws = (char *)al.alloc(ws_bytes, s);
    out->rp = (int64_t *)al.alloc((size_t)(m + 1) * 8, s);
    if (!ws || !out->rp) {
        rc = MP_ERR_NOMEM;
        goto fail;
    }
    prod = (uint64_t *)(ws + off_prod);
    bin = (int8_t *)(ws + off_bin);
    list = (uint32_t *)(ws + off_list);
    long_rows = (uint32_t *)(ws + off_long);
    sm_sym = (Small *)(ws + off_small);
    sm_num = sm_sym + 1;
    CK(cudaMemsetAsync(sm_sym, 0, sizeof(Small) * 2, s));

    // 1-2. per-row work, symbolic bins, rows grouped by bin
    if (m > 0) {
        unsigned g = (unsigned)std::min<int64_t>(grid_for(m * 32, 256), (int64_t)tun.sm_count * 32);
        kl(k_rowwork, g, 256, 0, s, X, Y, rm, km, prod, long_rows, &sm_sym->n_long);
        kl(k_rowwork_long, (unsigned)tun.sm_count * 4, 256, 0, s, X, Y, km, prod, long_rows, &sm_sym->n_long);
        unsigned gf = (unsigned)std::min<int64_t>(grid_for(m, 256), (int64_t)tun.sm_count * 16);
        kl(k_binassign, gf, 256, 0, s, X.rp, prod, m, ba, bin, out->rp, &sm_sym->tally, &sm_sym->total_prod);
        kl(k_bin_offsets, 1, 32, 0, s, sm_sym->tally.counts, sm_sym->offsets, sm_sym->cursors);
        kl(k_bin_fill, gf, 256, 0, s, bin, m, sm_sym->offsets, sm_sym->cursors, list);
    }
    CK(cudaMemcpyAsync(&h_sym, sm_sym, sizeof(Small), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));

    pa.X = X;
    pa.Y = Y;
    pa.km = km;
    pa.cm = cm;
    pa.list = list;
    pa.counts = sm_sym->tally.counts;
    pa.offsets = sm_sym->offsets;
    pa.nnz = out->rp;
    pa.err = &sm_sym->err;
    // GLOBAL bin set-up: its rows, work items, bitmap rounds
    gl.R = h_sym.tally.counts[B_GLOBAL];
    if (gl.R) {
        gl.nw = (Y.ncols + 31) / 32;
        const uint64_t cap = tun.scratch_cap ? tun.scratch_cap : (4ull << 30);
        gl.per_round = std::max<int64_t>(1, std::min<int64_t>(gl.R, (int64_t)(cap / ((uint64_t)gl.nw * 8))));
        gl.rounds = (gl.R + gl.per_round - 1) / gl.per_round;
        gl.kept = gl.rounds == 1;
        const int64_t xtot = (int64_t)h_sym.tally.xent[B_GLOBAL];
        gl.prod = prod;
        gl.list = (uint32_t *)al.alloc((size_t)gl.R * 4, s);
        gl.item_off = (int64_t *)al.alloc((size_t)(gl.R + 1) * 8, s);
        gl.xbase = (int64_t *)al.alloc((size_t)(gl.R + 1) * 8, s);
        gl.xoff = (int64_t *)al.alloc((size_t)(xtot + 1) * 8, s);
        gl.bm = (uint32_t *)al.alloc((size_t)gl.per_round * gl.nw * 4, s);
        gl.rank = (uint32_t *)al.alloc((size_t)gl.per_round * gl.nw * 4, s);
        if (!gl.list || !gl.item_off || !gl.xbase || !gl.xoff || !gl.bm || !gl.rank) {
            rc = MP_ERR_NOMEM;
            goto fail;
        }
        CK(cudaMemcpyAsync(gl.list, list + h_sym.offsets[B_GLOBAL], (size_t)gl.R * 4, cudaMemcpyDeviceToDevice, s));
        kl(k_glob_prep, (unsigned)std::min<int64_t>(grid_for(gl.R, 256), 1024), 256, 0, s, gl.list, gl.R, X.rp, prod,
           gl.xbase, gl.item_off);
        scan_i64(gl.item_off, gl.item_off, gl.R, al, s);
        scan_i64(gl.xbase, gl.xbase, gl.R, al, s);
        kl(k_glob_xlen, (unsigned)std::max<int64_t>(1, std::min<int64_t>(grid_for(xtot, 256), (int64_t)tun.sm_count * 16)),
           256, 0, s, X, Y, km, gl.list, gl.R, gl.xbase, gl.xoff);
        scan_i64(gl.xoff, gl.xoff, xtot, al, s);
    }
    // 3-4. symbolic pass, row pointers
    if (m > 0) run_pass(0, pa, h_sym.tally.counts, Y.ncols, tun, s, prof);
    if (gl.R) glob_pass(0, gl, pa, tun, s, prof);
    scan_i64(out->rp, out->rp, m, al, s);
    CK(cudaMemcpyAsync(&nnz, out->rp + m, 8, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&err, &sm_sym->err, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    prof_collect(prof, 0, h_sym.tally, Y.ncols, tun);
    if (st) {
        st->products += h_sym.total_prod;
        for (int b = 0; b < NBINS; b++) st->sym_bins[b] += h_sym.tally.counts[b];
    }
    if (err) {
        rc = (err & ERR_OVERFLOW) ? MP_ERR_OVERFLOW : MP_ERR_INTERNAL;
        goto fail;
    }
    out->nnz = nnz;
    if (max_result_bytes && out->bytes() > max_result_bytes) {
        rc = MP_ERR_TOO_LARGE;
        goto fail;
    }
    out->ci = (int32_t *)al.alloc((size_t)std::max<int64_t>(nnz, 1) * 4, s);
    out->val = (uint64_t *)al.alloc((size_t)std::max<int64_t>(nnz, 1) * 8, s);
    if (!out->ci || !out->val) {
        rc = MP_ERR_NOMEM;
        goto fail;
    }
    // 5. numeric pass on bins of the exact row sizes (GLOBAL rows keep their bin)
    if (nnz > 0) {
        unsigned g = (unsigned)std::min<int64_t>(grid_for(m, 256), (int64_t)tun.sm_count * 16);
        kl(k_numbin, g, 256, 0, s, out->rp, X.rp, prod, m, ba, X.val != nullptr, Y.val != nullptr, bin,
           &sm_num->tally, &sm_num->err);
        kl(k_bin_offsets, 1, 32, 0, s, sm_num->tally.counts, sm_num->offsets, sm_num->cursors);
        kl(k_bin_fill, g, 256, 0, s, bin, m, sm_num->offsets, sm_num->cursors, list);
        CK(cudaMemcpyAsync(&h_num, sm_num, sizeof(Small), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        pa.counts = sm_num->tally.counts;
        pa.offsets = sm_num->offsets;
        pa.rp = out->rp;
        pa.out_ci = out->ci;
        pa.out_val = out->val;
        pa.err = &sm_num->err;
        run_pass(1, pa, h_num.tally.counts, Y.ncols, tun, s, prof);
        if (gl.R) glob_pass(1, gl, pa, tun, s, prof);
        CK(cudaMemcpyAsync(&err, &sm_num->err, 4, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        prof_collect(prof, 1, h_num.tally, Y.ncols, tun);
        if (st)
            for (int b = 0; b < NBINS; b++) st->num_bins[b] += h_num.tally.counts[b];
        if (err) {
            rc = (err & ERR_OVERFLOW) ? MP_ERR_OVERFLOW : MP_ERR_INTERNAL;
            goto fail;
        }
    }
    CK(cudaGetLastError());
    glob_release(gl, al, s);
    al.free(ws, s);
    if (st) st->nnz += (uint64_t)nnz;
    return MP_OK;
fail:
    glob_release(gl, al, s);
    if (ws) al.free(ws, s);
    if (out->rp) al.free(out->rp, s);
    if (out->ci) al.free(out->ci, s);
    if (out->val) al.free(out->val, s);
    out->rp = nullptr;
    out->ci = nullptr;
    out->val = nullptr;
    return rc;
}
#undef CK

// ------------------------------------------------------------------ length-2 metapaths

__global__ void k_filter_count(DCsr A, const uint32_t *rm, const uint32_t *cm, int64_t *cnt) {
    int lane = threadIdx.x & 31;
    int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = w; i < A.nrows; i += nwarps) {
        int64_t c = 0;
        if (bit_of(rm, (uint32_t)i))
            for (int64_t p = A.rp[i] + lane; p < A.rp[i + 1]; p += 32) c += bit_of(cm, (uint32_t)__ldg(A.ci + p));
        for (int d = 16; d; d >>= 1) c += __shfl_xor_sync(FULL, c, d);
        if (lane == 0) cnt[i] = c;
    }
}

__global__ void k_filter_fill(DCsr A, const uint32_t *rm, const uint32_t *cm, const int64_t *rp,
                              int32_t *ci, uint64_t *val) {
    int lane = threadIdx.x & 31;
    int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = w; i < A.nrows; i += nwarps) {
        if (!bit_of(rm, (uint32_t)i)) continue;
        int64_t o = rp[i];
        for (int64_t p0 = A.rp[i]; p0 < A.rp[i + 1]; p0 += 32) {
            int64_t p = p0 + lane;
            int32_t j = p < A.rp[i + 1] ? __ldg(A.ci + p) : 0;
            bool keep = p < A.rp[i + 1] && bit_of(cm, (uint32_t)j);
            unsigned bal = __ballot_sync(FULL, keep);
            if (keep) {
                int64_t q = o + __popc(bal & ((1u << lane) - 1u));
                ci[q] = j;
                val[q] = A.val ? A.val[p] : 1ull;
            }
            o += __popc(bal);
        }
    }
}

#define CK(x)                                                                     \
    do {                                                                          \
        cudaError_t e_ = (x);                                                     \
        if (e_ != cudaSuccess) {                                                  \
            fprintf(stderr, "mp: %s failed: %s\n", #x, cudaGetErrorString(e_));   \
            return MP_ERR_CUDA;                                                   \
        }                                                                         \
    } while (0)

int filter(const DCsr &A, const uint32_t *rm, const uint32_t *cm, Alloc &al, const Tuning &tun,
           cudaStream_t s, Mat *out) {
    const int64_t m = A.nrows;
    out->nrows = m;
    out->ncols = A.ncols;
    out->rp = (int64_t *)al.alloc((size_t)(m + 1) * 8, s);
    if (!out->rp) return MP_ERR_NOMEM;
    unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(grid_for(m * 32, 256), (int64_t)tun.sm_count * 32));
    if (m) kl(k_filter_count, g, 256, 0, s, A, rm, cm, out->rp);
    scan_i64(out->rp, out->rp, m, al, s);
    int64_t nnz = 0;
    CK(cudaMemcpyAsync(&nnz, out->rp + m, 8, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    out->nnz = nnz;
    out->ci = (int32_t *)al.alloc((size_t)std::max<int64_t>(nnz, 1) * 4, s);
    out->val = (uint64_t *)al.alloc((size_t)std::max<int64_t>(nnz, 1) * 8, s);
    if (!out->ci || !out->val) return MP_ERR_NOMEM;
    if (nnz) kl(k_filter_fill, g, 256, 0, s, A, rm, cm, out->rp, out->ci, out->val);
    CK(cudaGetLastError());
    return MP_OK;
}

}  // namespace mp

namespace mp {

__global__ void k_mask_and_in_values(uint32_t *m, const int32_t *prop, int64_t n, const int64_t *set,
                                     int64_t len) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    bool ok = false;
    if (i < n) {
        const int64_t v = prop[i];
        int64_t lo = 0, hi = len;
        while (lo < hi) {
            int64_t mid = (lo + hi) >> 1;
            if (set[mid] < v) lo = mid + 1; else hi = mid;
        }
        ok = lo < len && set[lo] == v;
    }
    uint32_t word = __ballot_sync(FULL, ok);
    if ((threadIdx.x & 31) == 0 && i < n) m[i >> 5] &= word;
}

void mask_and_in_values(uint32_t *m, const int32_t *prop, int64_t n, const int64_t *set, int64_t len,
                        cudaStream_t s) {
    if (n) kl(k_mask_and_in_values, grid_for(n, 256), 256, 0, s, m, prop, n, set, len);
}

}  // namespace mp
