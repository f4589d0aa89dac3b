// Device helpers shared by the engine's kernels (bitmaps, bins, block scans, product
// enumeration, shared-memory hash tables, bitonic sort) and the counting launch helper.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <utility>

#include "../../include/mp.h"
#include "internal.h"

namespace mp {

// Every kernel launch of the library goes through kl(), which counts it.
template <class... KArgs, class... Args>
static inline void kl(void (*k)(KArgs...), dim3 g, dim3 b, size_t smem, cudaStream_t s, Args &&...args) {
    k<<<g, b, smem, s>>>(std::forward<Args>(args)...);
    g_launches.fetch_add(1, std::memory_order_relaxed);
}

static inline unsigned grid_for(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

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
// an output of ncols columns. Hash tables are sized T >= 2u (load factor <= 1/2). A row
// goes to a one-warp bin only if it has at most warp_prod products (else 32 threads would
// grind through it alone); rows with more than `heavy` products, or whose output is too
// wide for a shared-memory table, go to GLOBAL, where the row is split over many blocks.
__host__ __device__ __forceinline__ int bin_for(uint64_t prod, uint64_t u, int64_t ncols, int dense_max_cols,
                                                int dense_min_u, uint64_t heavy, uint64_t warp_prod, int force) {
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
    if (e <= 10 && prod <= warp_prod) return B_W32 + (e - 5);
    if (e <= 13) return B_K2048 + (e < 11 ? 0 : e - 11);
    return dense_ok ? B_DENSE : B_GLOBAL;
}

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

}  // namespace mp
