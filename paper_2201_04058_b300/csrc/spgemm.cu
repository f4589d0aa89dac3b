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

// Bin of a row whose output has at most u entries (u >= 1), for an output of ncols
// columns. Hash tables are sized T >= 2u (load factor <= 1/2).
__host__ __device__ __forceinline__ int bin_for(uint64_t u, int64_t ncols, int dense_max_cols,
                                                int dense_min_u, int force) {
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

// nnz of diag(rm) A diag(cm): one warp per row.
__global__ void k_masked_nnz(DCsr A, const uint32_t *rm, const uint32_t *cm,
                             unsigned long long *out) {
    int lane = threadIdx.x & 31;
    int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long c = 0;
    for (int64_t i = w; i < A.nrows; i += nwarps) {
        if (!bit_of(rm, (uint32_t)i)) continue;
        int64_t b = A.rp[i], e = A.rp[i + 1];
        if (!cm) {
            if (lane == 0) c += (unsigned long long)(e - b);
            continue;
        }
        for (int64_t p = b + lane; p < e; p += 32) c += bit_of(cm, (uint32_t)__ldg(A.ci + p));
    }
    for (int d = 16; d; d >>= 1) c += __shfl_down_sync(FULL, c, d);
    if (lane == 0 && c) atomicAdd(out, c);
}

void masked_nnz(const DCsr &A, const uint32_t *rm, const uint32_t *cm, unsigned long long *out,
                cudaStream_t s) {
    if (!A.nrows) return;
    unsigned g = (unsigned)std::min<int64_t>(grid_for(A.nrows * 32, 256), 148 * 16);
    kl(k_masked_nnz, g, 256, 0, s, A, rm, cm, out);
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
};

// Per-bin tallies of one pass: rows, X entries, Gustavson products and output entries
// (the inputs of the algorithmic byte count of each bin's kernel).
struct BinTally {
    uint32_t counts[NBINS];
    unsigned long long xent[NBINS], prods[NBINS], outn[NBINS];
};

__device__ __forceinline__ void tally_flush(BinTally *g, uint32_t *hc, unsigned long long *hx,
                                            unsigned long long *hp, unsigned long long *ho) {
    const int t = threadIdx.x;
    if (t < NBINS && hc[t]) {
        atomicAdd(g->counts + t, hc[t]);
        atomicAdd(g->xent + t, hx[t]);
        atomicAdd(g->prods + t, hp[t]);
        if (ho) atomicAdd(g->outn + t, ho[t]);
    }
}

// prod_i and the symbolic bin of every row; rows with prod_i = 0 get nnz_i = 0 and no bin.
__global__ void k_rowwork(DCsr X, DCsr Y, const uint32_t *rm, const uint32_t *km, BinArgs ba,
                          uint64_t *prod, int8_t *bin, int64_t *nnz, BinTally *tally,
                          unsigned long long *total_prod) {
    __shared__ uint32_t hc[NBINS];
    __shared__ unsigned long long hx[NBINS], hp[NBINS];
    __shared__ unsigned long long bsum;
    if (threadIdx.x < NBINS) {
        hc[threadIdx.x] = 0;
        hx[threadIdx.x] = 0;
        hp[threadIdx.x] = 0;
    }
    if (threadIdx.x == 0) bsum = 0;
    __syncthreads();
    int lane = threadIdx.x & 31;
    int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long mysum = 0;
    for (int64_t i = w; i < X.nrows; i += nwarps) {
        uint64_t s = 0;
        int64_t b = 0, e = 0;
        if (bit_of(rm, (uint32_t)i)) {
            b = X.rp[i];
            e = X.rp[i + 1];
            for (int64_t p = b + lane; p < e; p += 32) {
                int32_t k = __ldg(X.ci + p);
                if (bit_of(km, (uint32_t)k)) s += (uint64_t)(__ldg(Y.rp + k + 1) - __ldg(Y.rp + k));
            }
            for (int d = 16; d; d >>= 1) s += __shfl_xor_sync(FULL, s, d);
        }
        if (lane == 0) {
            prod[i] = s;
            int bb = -1;
            if (s) {
                bb = bin_for(s, ba.ncols, ba.dense_max_cols, ba.dense_min_u, ba.force);
                atomicAdd(&hc[bb], 1u);
                atomicAdd(&hx[bb], (unsigned long long)(e - b));
                atomicAdd(&hp[bb], (unsigned long long)s);
            } else {
                nnz[i] = 0;
            }
            bin[i] = (int8_t)bb;
            mysum += s;
        }
    }
    if (lane == 0 && mysum) atomicAdd(&bsum, mysum);
    __syncthreads();
    tally_flush(tally, hc, hx, hp, nullptr);
    if (threadIdx.x == 0 && bsum) atomicAdd(total_prod, bsum);
}

// Numeric bins from exact row sizes (nnz = rp[i+1] - rp[i]).
__global__ void k_numbin(const int64_t *rp, const int64_t *xrp, const uint64_t *prod, int64_t n, BinArgs ba,
                         int8_t *bin, BinTally *tally) {
    __shared__ uint32_t hc[NBINS];
    __shared__ unsigned long long hx[NBINS], hp[NBINS], ho[NBINS];
    if (threadIdx.x < NBINS) {
        hc[threadIdx.x] = 0;
        hx[threadIdx.x] = 0;
        hp[threadIdx.x] = 0;
        ho[threadIdx.x] = 0;
    }
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t z = rp[i + 1] - rp[i];
        int b = -1;
        if (z) {
            b = bin_for((uint64_t)z, ba.ncols, ba.dense_max_cols, ba.dense_min_u, ba.force);
            atomicAdd(&hc[b], 1u);
            atomicAdd(&hx[b], (unsigned long long)(xrp[i + 1] - xrp[i]));
            atomicAdd(&hp[b], (unsigned long long)prod[i]);
            atomicAdd(&ho[b], (unsigned long long)z);
        }
        bin[i] = (int8_t)b;
    }
    __syncthreads();
    tally_flush(tally, hc, hx, hp, ho);
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

// Enumerate every scalar product of row i with a group of G threads (G = 32: one warp;
// G = blockDim: one block). f(j, v) is called once per product that passes cm, where v
// = X_ik * Y_kj (1 when both are pattern-only; values only read when VAL).
template <int G, bool VAL, class F>
__device__ __forceinline__ void for_each_product(const DCsr &X, const DCsr &Y, const uint32_t *km,
                                                 const uint32_t *cm, int64_t i, Stage *sg,
                                                 int64_t *gtot, int64_t *warp_sums, int t,
                                                 uint32_t *err, F &&f) {
    const int64_t b = X.rp[i], e = X.rp[i + 1];
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
    char *scratch;         // GLOBAL bin
    size_t scratch_stride;
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
        for_each_product<32, false>(a.X, a.Y, a.km, a.cm, i, sg, nullptr, nullptr, lane, a.err,
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
        for_each_product<32, true>(a.X, a.Y, a.km, a.cm, i, sg, nullptr, nullptr, lane, a.err,
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
        for_each_product<NT, false>(a.X, a.Y, a.km, a.cm, i, sg, &gtot, warp_sums, threadIdx.x, a.err,
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
        for_each_product<NT, true>(a.X, a.Y, a.km, a.cm, i, sg, &gtot, warp_sums, threadIdx.x, a.err,
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
        for_each_product<NT, false>(a.X, a.Y, a.km, a.cm, i, sg, &gtot, warp_sums, threadIdx.x, a.err,
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
        for_each_product<NT, true>(a.X, a.Y, a.km, a.cm, i, sg, &gtot, warp_sums, threadIdx.x, a.err,
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

// ------------------------------------------------------------------ global-scratch bin

// Each block owns one scratch slice: ncols uint64 accumulators, then ceil(ncols/32) bitmap
// words. Both are all-zero on entry and are restored to zero before the block moves on.
template <int NT>
__global__ void __launch_bounds__(NT) k_sym_global(PassArgs a, int bin) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int64_t warp_sums[32];
    __shared__ int64_t gtot;
    __shared__ int cnt_s;
    __shared__ uint32_t wlo, whi;
    Stage *sg = (Stage *)smem;
    char *slice = a.scratch + (size_t)blockIdx.x * a.scratch_stride;
    uint32_t *bm = (uint32_t *)(slice + (size_t)a.Y.ncols * 8);
    const uint32_t cnt = a.counts[bin], base = a.offsets[bin];
    for (uint32_t r = blockIdx.x; r < cnt; r += gridDim.x) {
        const int64_t i = a.list[base + r];
        if (threadIdx.x == 0) {
            cnt_s = 0;
            wlo = 0xffffffffu;
            whi = 0;
        }
        __syncthreads();
        int c = 0;
        uint32_t lo = 0xffffffffu, hi = 0;
        for_each_product<NT, false>(a.X, a.Y, a.km, a.cm, i, sg, &gtot, warp_sums, threadIdx.x, a.err,
                                    [&](uint32_t j, uint64_t) {
                                        uint32_t m = 1u << (j & 31);
                                        c += (atomicOr(bm + (j >> 5), m) & m) == 0;
                                        lo = min(lo, j >> 5);
                                        hi = max(hi, j >> 5);
                                    });
        for (int d = 16; d; d >>= 1) {
            c += __shfl_xor_sync(FULL, c, d);
            lo = min(lo, __shfl_xor_sync(FULL, lo, d));
            hi = max(hi, __shfl_xor_sync(FULL, hi, d));
        }
        if ((threadIdx.x & 31) == 0) {
            if (c) atomicAdd(&cnt_s, c);
            atomicMin(&wlo, lo);
            atomicMax(&whi, hi);
        }
        __syncthreads();
        if (threadIdx.x == 0) a.nnz[i] = cnt_s;
        if (wlo <= whi)
            for (uint32_t s = wlo + threadIdx.x; s <= whi; s += NT) bm[s] = 0;
        __syncthreads();
    }
}

template <int NT>
__global__ void __launch_bounds__(NT) k_num_global(PassArgs a, int bin) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int64_t warp_sums[32];
    __shared__ int64_t gtot;
    __shared__ uint32_t wlo, whi;
    Stage *sg = (Stage *)smem;
    char *slice = a.scratch + (size_t)blockIdx.x * a.scratch_stride;
    unsigned long long *acc = (unsigned long long *)slice;
    uint32_t *bm = (uint32_t *)(slice + (size_t)a.Y.ncols * 8);
    const uint32_t cnt = a.counts[bin], base = a.offsets[bin];
    for (uint32_t r = blockIdx.x; r < cnt; r += gridDim.x) {
        const int64_t i = a.list[base + r];
        if (threadIdx.x == 0) {
            wlo = 0xffffffffu;
            whi = 0;
        }
        __syncthreads();
        uint32_t lo = 0xffffffffu, hi = 0;
        for_each_product<NT, true>(a.X, a.Y, a.km, a.cm, i, sg, &gtot, warp_sums, threadIdx.x, a.err,
                                   [&](uint32_t j, uint64_t v) {
                                       unsigned long long old = atomicAdd(acc + j, (unsigned long long)v);
                                       if (old + v < old) atomicOr(a.err, ERR_OVERFLOW);
                                       if (old == 0) atomicOr(bm + (j >> 5), 1u << (j & 31));
                                       lo = min(lo, j >> 5);
                                       hi = max(hi, j >> 5);
                                   });
        for (int d = 16; d; d >>= 1) {
            lo = min(lo, __shfl_xor_sync(FULL, lo, d));
            hi = max(hi, __shfl_xor_sync(FULL, hi, d));
        }
        if ((threadIdx.x & 31) == 0) {
            atomicMin(&wlo, lo);
            atomicMax(&whi, hi);
        }
        __syncthreads();
        const int64_t o = a.rp[i];
        const int64_t rowlen = a.rp[i + 1] - o;
        int64_t done = 0;
        const uint32_t w0 = wlo, w1 = whi;
        if (w0 <= w1) {
            for (uint32_t t0 = w0; t0 <= w1; t0 += NT) {
                const uint32_t w = t0 + threadIdx.x;
                uint32_t word = (w <= w1) ? bm[w] : 0u;
                int64_t pos = done + block_excl_scan<NT>(__popc(word), warp_sums, &gtot);
                while (word) {
                    const int b = __ffs(word) - 1;
                    word &= word - 1;
                    const uint32_t j = w * 32 + b;
                    if (pos < rowlen) {
                        a.out_ci[o + pos] = (int32_t)j;
                        a.out_val[o + pos] = acc[j];
                    }
                    acc[j] = 0;
                    pos++;
                }
                if (w <= w1) bm[w] = 0;
                done += gtot;
            }
        }
        if (threadIdx.x == 0 && done != rowlen) atomicOr(a.err, ERR_COUNT);
        __syncthreads();
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

// Launch every non-empty bin's kernel of one pass, each grid sized to its bin's rows
// (capped at a few blocks per SM; the kernels loop over their bin). With prof, CUDA
// events bracket each launch.
static void run_pass(int pass, const PassArgs &a, const uint32_t *host_counts, int64_t ncols, int nscr_ctas,
                     const Tuning &tun, cudaStream_t s, Prof *prof) {
    const bool numeric = pass == 1;
    const int sms = tun.sm_count;
    const size_t stage = sizeof(Stage);
    for (int b = 0; b < NBINS; b++) {
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
            case B_GLOBAL: {
                unsigned g = blocks_for(rows, 1, nscr_ctas);
                if (numeric)
                    launch(k_num_global<512>, g, 512, 512 * stage, s, a, B_GLOBAL);
                else
                    launch(k_sym_global<512>, g, 512, 512 * stage, s, a, B_GLOBAL);
                break;
            }
        }
        if (prof && prof->on) cudaEventRecord(prof->ev[pass][b][1], s);
    }
}

// Algorithmic bytes of one bin's kernel in one pass (every X entry: column id, value if
// any, and the two Y row pointers it looks up; every Gustavson product: the Y column id
// and, in the numeric pass, the Y value; every output entry: column id + uint64 value;
// every row: its X row pointers, and its nnz (symbolic) or C row pointers (numeric)).
static double bin_bytes(int pass, const BinTally &t, int b, bool x_val, bool y_val) {
    const double rows = t.counts[b], xe = (double)t.xent[b], pr = (double)t.prods[b], on = (double)t.outn[b];
    if (pass == 0) return rows * 16 + xe * (4 + 16) + pr * 4 + rows * 8;
    return rows * 32 + xe * (4 + (x_val ? 8 : 0) + 16) + pr * (4 + (y_val ? 8 : 0)) + on * 12;
}

static void prof_collect(Prof *prof, int pass, const BinTally &t, bool x_val, bool y_val, int64_t ncols,
                         const Tuning &tun) {
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
        k.bytes += bin_bytes(pass, t, b, x_val, y_val);
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

// Make the scratch hold up to one slice of `stride` bytes per SM, zeroed, within the
// scratch cap. Returns the number of slices available (0 on allocation failure).
static int ensure_scratch(Scratch &scr, size_t stride, const Tuning &tun, Alloc &al, cudaStream_t s) {
    size_t cap = tun.scratch_cap ? tun.scratch_cap : (4ull << 30);
    int fit = (int)std::max<size_t>(1, cap / stride);
    int n = std::min(tun.sm_count, fit);
    size_t need = stride * (size_t)n;
    if (scr.bytes < need) {
        if (scr.base) al.free(scr.base, s);
        scr.base = al.alloc(need, s);
        if (!scr.base) {
            scr.bytes = 0;
            return 0;
        }
        scr.bytes = need;
        cudaMemsetAsync(scr.base, 0, need, s);
    }
    return (int)std::min<size_t>(n, scr.bytes / stride);
}

int spgemm(const DCsr &X, const DCsr &Y, const uint32_t *rm, const uint32_t *km, const uint32_t *cm,
           Alloc &al, Scratch &scr, const Tuning &tun, cudaStream_t s, uint64_t max_result_bytes,
           Mat *out, Stats *st, Prof *prof) {
    const int64_t m = X.nrows;
    out->nrows = m;
    out->ncols = Y.ncols;
    out->nnz = 0;
    struct Small {
        BinTally tally;
        uint32_t offsets[NBINS + 1];
        uint32_t cursors[NBINS];
        uint32_t err;
        unsigned long long total_prod;
    };
    // workspace: prod u64[m], bins i8[m], row list u32[m], two Small blocks
    const size_t off_prod = 0;
    const size_t off_bin = align256(off_prod + (size_t)m * 8);
    const size_t off_list = align256(off_bin + (size_t)m);
    const size_t off_small = align256(off_list + (size_t)m * 4);
    const size_t ws_bytes = align256(off_small + sizeof(Small) * 2);
    const size_t stride = align256((size_t)Y.ncols * 8 + (size_t)((Y.ncols + 31) / 32) * 4);
    const BinArgs ba{Y.ncols, tun.dense_max_cols, tun.dense_min_u, tun.force_class};
    int rc = MP_OK;
    int nscr = 0;
    int64_t nnz = 0;
    uint32_t err = 0;
    Small h_sym, h_num;
    PassArgs pa{};
    uint64_t *prod;
    int8_t *bin;
    uint32_t *list;
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
    sm_sym = (Small *)(ws + off_small);
    sm_num = sm_sym + 1;
    CK(cudaMemsetAsync(sm_sym, 0, sizeof(Small) * 2, s));

    // 1-2. per-row work, symbolic bins, rows grouped by bin
    if (m > 0) {
        unsigned g = (unsigned)std::min<int64_t>(grid_for(m * 32, 256), (int64_t)tun.sm_count * 32);
        kl(k_rowwork, g, 256, 0, s, X, Y, rm, km, ba, prod, bin, out->rp, &sm_sym->tally, &sm_sym->total_prod);
        kl(k_bin_offsets, 1, 32, 0, s, sm_sym->tally.counts, sm_sym->offsets, sm_sym->cursors);
        unsigned gf = (unsigned)std::min<int64_t>(grid_for(m, 256), (int64_t)tun.sm_count * 16);
        kl(k_bin_fill, gf, 256, 0, s, bin, m, sm_sym->offsets, sm_sym->cursors, list);
    }
    CK(cudaMemcpyAsync(&h_sym, sm_sym, sizeof(Small), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (h_sym.tally.counts[B_GLOBAL]) {
        nscr = ensure_scratch(scr, stride, tun, al, s);
        if (!nscr) {
            rc = MP_ERR_NOMEM;
            goto fail;
        }
    }
    // 3-4. symbolic pass, row pointers
    pa.X = X;
    pa.Y = Y;
    pa.km = km;
    pa.cm = cm;
    pa.list = list;
    pa.counts = sm_sym->tally.counts;
    pa.offsets = sm_sym->offsets;
    pa.nnz = out->rp;
    pa.err = &sm_sym->err;
    pa.scratch = (char *)scr.base;
    pa.scratch_stride = stride;
    if (m > 0) run_pass(0, pa, h_sym.tally.counts, Y.ncols, nscr, tun, s, prof);
    scan_i64(out->rp, out->rp, m, al, s);
    CK(cudaMemcpyAsync(&nnz, out->rp + m, 8, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&err, &sm_sym->err, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    prof_collect(prof, 0, h_sym.tally, X.val != nullptr, Y.val != nullptr, Y.ncols, tun);
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
    // 5. numeric pass on bins of the exact row sizes
    if (nnz > 0) {
        unsigned g = (unsigned)std::min<int64_t>(grid_for(m, 256), (int64_t)tun.sm_count * 16);
        kl(k_numbin, g, 256, 0, s, out->rp, X.rp, prod, m, ba, bin, &sm_num->tally);
        kl(k_bin_offsets, 1, 32, 0, s, sm_num->tally.counts, sm_num->offsets, sm_num->cursors);
        kl(k_bin_fill, g, 256, 0, s, bin, m, sm_num->offsets, sm_num->cursors, list);
        CK(cudaMemcpyAsync(&h_num, sm_num, sizeof(Small), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (h_num.tally.counts[B_GLOBAL]) {
            nscr = ensure_scratch(scr, stride, tun, al, s);
            if (!nscr) {
                rc = MP_ERR_NOMEM;
                goto fail;
            }
        }
        pa.counts = sm_num->tally.counts;
        pa.offsets = sm_num->offsets;
        pa.rp = out->rp;
        pa.out_ci = out->ci;
        pa.out_val = out->val;
        pa.err = &sm_num->err;
        pa.scratch = (char *)scr.base;
        run_pass(1, pa, h_num.tally.counts, Y.ncols, nscr, tun, s, prof);
        CK(cudaMemcpyAsync(&err, &sm_num->err, 4, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        prof_collect(prof, 1, h_num.tally, X.val != nullptr, Y.val != nullptr, Y.ncols, tun);
        if (st)
            for (int b = 0; b < NBINS; b++) st->num_bins[b] += h_num.tally.counts[b];
        if (err) {
            rc = (err & ERR_OVERFLOW) ? MP_ERR_OVERFLOW : MP_ERR_INTERNAL;
            goto fail;
        }
    }
    CK(cudaGetLastError());
    al.free(ws, s);
    if (st) st->nnz += (uint64_t)nnz;
    return MP_OK;
fail:
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
