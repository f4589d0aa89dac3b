// Constraint masks (Def. 3), masked nnz of base relations, the row-pointer scan and the
// length-2 metapath filter.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>

#include "common.cuh"

namespace mp {

// ------------------------------------------------------------------ masks

__global__ void k_mask_fill(uint32_t *m, int64_t nw, uint32_t v, int64_t n) {
    int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (w >= nw) return;
    uint32_t x = v;
    if (v && w == nw - 1 && (n & 31)) x = (1u << (n & 31)) - 1u;  // no bits past n
    m[w] = x;
}

// One thread per node; a warp ballot forms one 32-node word, AND-ed into the mask (or
// stored, for the first constraint of a position).
__global__ void k_mask_and_range(uint32_t *m, const int32_t *prop, int64_t n, int64_t lo,
                                 int64_t hi, int assign) {
    int64_t base = (blockIdx.x * (int64_t)blockDim.x) & ~31ll;
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    bool ok = false;
    if (i < n) {
        int64_t v = prop ? (int64_t)__ldg(prop + i) : i;
        ok = v >= lo && v <= hi;
    }
    uint32_t word = __ballot_sync(FULL, ok);
    if ((threadIdx.x & 31) == 0 && i < n) {
        uint32_t *w = m + ((base + (threadIdx.x & ~31)) >> 5);
        *w = assign ? word : (*w & word);
    }
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


__global__ void k_iota(int32_t *d, int64_t lo, int64_t n) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < n) d[t] = (int32_t)(lo + t);
}

void fill_iota(int32_t *d, int64_t lo, int64_t n, cudaStream_t s) {
    if (n > 0) kl(k_iota, grid_for(n, 256), 256, 0, s, d, lo, n);
}

void mask_fill(uint32_t *m, int64_t n, bool ones, cudaStream_t s) {
    int64_t nw = (n + 31) / 32;
    if (nw) kl(k_mask_fill, grid_for(nw, 256), 256, 0, s, m, nw, ones ? FULL : 0u, n);
}

void mask_and_range(uint32_t *m, const int32_t *prop, int64_t n, int64_t lo, int64_t hi,
                    cudaStream_t s, bool assign) {
    if (n) kl(k_mask_and_range, grid_for(n, 256), 256, 0, s, m, prop, n, lo, hi, (int)assign);
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

// nnz of diag(rm) A diag(cm) when rm selects the listed rows only (ascending ids): one warp
// per listed row, the lanes over its entries.
__global__ void k_masked_nnz_list(DCsr A, const int32_t *rows, int64_t n, const uint32_t *cm, unsigned long long *out) {
    const int lane = threadIdx.x & 31;
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long c = 0;
    for (int64_t r = w; r < n; r += nwarps) {
        const int64_t i = rows[r];
        const int64_t b = A.rp[i], e = A.rp[i + 1];
        if (!cm) {
            if (lane == 0) c += (unsigned long long)(e - b);
            continue;
        }
        for (int64_t p = b + lane; p < e; p += 32) c += bit_of(cm, (uint32_t)__ldg(A.ci + p));
    }
    for (int d = 16; d; d >>= 1) c += __shfl_down_sync(FULL, c, d);
    if (lane == 0 && c) atomicAdd(out, c);
}

void masked_nnz_list(const DCsr &A, const int32_t *rows, int64_t n, const uint32_t *cm, unsigned long long *out,
                     cudaStream_t s) {
    if (n <= 0) return;
    kl(k_masked_nnz_list, (unsigned)std::min<int64_t>(grid_for(n * 32, 256), 148 * 16), 256, 0, s, A, rows, n, cm,
       out);
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

// Short arrays (up to 1024 x SMALL_PER elements) in one block and one launch.
static constexpr int SMALL_PER = 16;

__global__ void __launch_bounds__(1024) k_scan_small(const int64_t *in, int64_t *out, int64_t n) {
    __shared__ int64_t ws[32];
    __shared__ int64_t tot;
    const int64_t base = (int64_t)threadIdx.x * SMALL_PER;
    int64_t v[SMALL_PER];
    int64_t s = 0;
#pragma unroll
    for (int t = 0; t < SMALL_PER; t++) {
        v[t] = base + t < n ? in[base + t] : 0;
        s += v[t];
    }
    int64_t e = block_excl_scan<1024>(s, ws, &tot);
    // every read of the block is done (the scan synchronised), so out may alias in
#pragma unroll
    for (int t = 0; t < SMALL_PER; t++) {
        if (base + t < n) out[base + t] = e;
        e += v[t];
    }
    if (threadIdx.x == 0) out[n] = tot;
}

int scan_i64(const int64_t *in, int64_t *out, int64_t n, Alloc &al, cudaStream_t s) {
    if (n == 0) {
        cudaMemsetAsync(out, 0, sizeof(int64_t), s);
        return MP_OK;
    }
    if (n <= 1024 * SMALL_PER) {
        kl(k_scan_small, 1, 1024, 0, s, in, out, n);
        return MP_OK;
    }
    int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    int64_t *part = (int64_t *)al.alloc((size_t)(nb + 1) * sizeof(int64_t), s);
    if (!part) return MP_ERR_NOMEM;
    kl(k_scan_tiles, (unsigned)nb, SCAN_T, 0, s, in, n, part);
    kl(k_scan_parts, 1, 1024, 0, s, part, nb);
    kl(k_scan_apply, (unsigned)nb, SCAN_T, 0, s, in, out, n, part, nb);
    al.free(part, s);
    return MP_OK;
}

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
    if (scan_i64(out->rp, out->rp, m, al, s)) return MP_ERR_NOMEM;
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

// ------------------------------------------------------------------ column-masked copies

// B = A diag(m) for a pattern CSR A: rows unchanged, each row's entries whose column passes
// m kept in order. Balanced over entries, so a hub row spreads over many blocks: K(e), the
// number of kept entries before flat position e, gives every kept entry its position and
// every row its start (B.rp[r] = K(A.rp[r])). Chunks of CC_CH entries tile positions
// [0, nnz] (the last chunk holds position nnz, where the rows that end the matrix start).
static constexpr int CC_NT = 256, CC_PER = 8, CC_CH = CC_NT * CC_PER;

// A thread's CC_PER consecutive column ids from eb (zeros past nnz): two 16-byte loads when
// they are all in range and aligned, else one at a time.
__device__ __forceinline__ void cc_load(const int32_t *__restrict__ ci, int64_t eb, int64_t nnz, int32_t (&j)[CC_PER]) {
    if (eb + CC_PER <= nnz && (((uintptr_t)(ci + eb)) & 15u) == 0) {
        const int4 a = __ldg((const int4 *)(ci + eb)), b = __ldg((const int4 *)(ci + eb) + 1);
        j[0] = a.x, j[1] = a.y, j[2] = a.z, j[3] = a.w, j[4] = b.x, j[5] = b.y, j[6] = b.z, j[7] = b.w;
        return;
    }
#pragma unroll
    for (int t = 0; t < CC_PER; t++) j[t] = eb + t < nnz ? __ldg(ci + eb + t) : 0;
}

// Also records, per chunk, the first row that starts inside it (first[c], -1 when none:
// the caller fills first with -1 bytes), so the fill pass needs no search for its rows.
__global__ void __launch_bounds__(CC_NT) k_cc_count(const int64_t *__restrict__ rp, int64_t nrows,
                                                    const int32_t *__restrict__ ci, int64_t nnz,
                                                    const uint32_t *__restrict__ m, int64_t nch, int64_t *cnt,
                                                    int64_t *first) {
    __shared__ int64_t ws[32];
    __shared__ int64_t tot;
    for (int64_t r = blockIdx.x * (int64_t)CC_NT + threadIdx.x; r <= nrows; r += (int64_t)gridDim.x * CC_NT) {
        const int64_t c = __ldg(rp + r) / CC_CH;
        if (r == 0 || __ldg(rp + r - 1) / CC_CH < c) first[c] = r;
    }
    for (int64_t c = blockIdx.x; c < nch; c += gridDim.x) {
        const int64_t eb = c * CC_CH + (int64_t)threadIdx.x * CC_PER;
        int32_t j[CC_PER];
        cc_load(ci, eb, nnz, j);
        int64_t n = 0;
#pragma unroll
        for (int t = 0; t < CC_PER; t++)
            if (eb + t < nnz && bit_of(m, (uint32_t)j[t])) n++;
        block_excl_scan<CC_NT>(n, ws, &tot);
        if (threadIdx.x == 0) cnt[c] = tot;
    }
}

__global__ void __launch_bounds__(CC_NT) k_cc_fill(const int64_t *__restrict__ rp, int64_t nrows,
                                                   const int32_t *__restrict__ ci, int64_t nnz,
                                                   const uint32_t *__restrict__ m, int64_t nch,
                                                   const int64_t *__restrict__ base, const int64_t *__restrict__ first,
                                                   int64_t *rp2, int32_t *ci2) {
    __shared__ int64_t ws[32];
    __shared__ int64_t tot;
    __shared__ int32_t pre[CC_CH];  // kept entries of the chunk before each offset
    for (int64_t c = blockIdx.x; c < nch; c += gridDim.x) {
        const int64_t e0 = c * CC_CH;
        const int64_t eb = e0 + (int64_t)threadIdx.x * CC_PER;
        int32_t j[CC_PER];
        bool f[CC_PER];
        cc_load(ci, eb, nnz, j);
        int64_t n = 0;
#pragma unroll
        for (int t = 0; t < CC_PER; t++) {
            f[t] = eb + t < nnz && bit_of(m, (uint32_t)j[t]);
            n += f[t];
        }
        int64_t local = block_excl_scan<CC_NT>(n, ws, &tot);
        int64_t k = base[c] + local;
#pragma unroll
        for (int t = 0; t < CC_PER; t++) {
            pre[threadIdx.x * CC_PER + t] = (int32_t)local;
            if (f[t]) {
                ci2[k++] = j[t];
                local++;
            }
        }
        __syncthreads();
        const int64_t r0 = first[c];  // rows starting in this chunk: r0, r0 + 1, ... (none: -1)
        for (int64_t r = r0 + threadIdx.x; r0 >= 0 && r <= nrows; r += CC_NT) {
            const int64_t a = __ldg(rp + r);
            if (a >= e0 + CC_CH) break;
            rp2[r] = base[c] + pre[a - e0];
        }
        __syncthreads();
    }
}

// The Gustavson products of diag(rm) X diag(km) Y before Y's column mask: the sum over the
// entries (i, k) of X that pass rm and km of |Y row k|, added into *out. Flat over X's
// entries (a row with many entries spreads over the grid); an entry's row is found by
// binary search only when there is a row mask to read.
__global__ void k_raw_products(DCsr X, const uint32_t *__restrict__ rm, const uint32_t *__restrict__ km,
                               const int64_t *__restrict__ yrp, unsigned long long *out) {
    unsigned long long s = 0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < X.nnz; e += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t k = (uint32_t)__ldg(X.ci + e);
        if (!bit_of(km, k)) continue;
        if (rm) {
            int64_t lo = 0, hi = X.nrows - 1;  // the last row starting at or before e
            while (lo < hi) {
                const int64_t mid = (lo + hi + 1) >> 1;
                if (__ldg(X.rp + mid) <= e) lo = mid; else hi = mid - 1;
            }
            if (!bit_of(rm, (uint32_t)lo)) continue;
        }
        s += (unsigned long long)(__ldg(yrp + k + 1) - __ldg(yrp + k));
    }
    for (int d = 16; d; d >>= 1) s += __shfl_xor_sync(FULL, s, d);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(out, s);
}

void raw_products(const DCsr &X, const uint32_t *rm, const uint32_t *km, const int64_t *yrp, const Tuning &tun,
                  cudaStream_t s, unsigned long long *out) {
    if (X.nnz <= 0) return;
    kl(k_raw_products, (unsigned)std::min<int64_t>(grid_for(X.nnz, 256), (int64_t)tun.sm_count * 8), 256, 0, s, X,
       rm, km, yrp, out);
}

int compact_cols(const DCsr &A, const uint32_t *m, Alloc &al, const Tuning &tun, cudaStream_t s, DCsr *out,
                 int64_t **rp_out, int32_t **ci_out) {
    const int64_t nch = A.nnz / CC_CH + 1;
    int64_t *cnt = (int64_t *)al.alloc((size_t)(2 * nch + 1) * 8, s);  // counts, then first rows
    int64_t *first = cnt + nch + 1;
    int64_t *rp2 = (int64_t *)al.alloc((size_t)(A.nrows + 1) * 8, s);
    int32_t *ci2 = (int32_t *)al.alloc((size_t)std::max<int64_t>(A.nnz, 1) * 4, s);  // at most A's entries
    if (!cnt || !rp2 || !ci2) {
        if (cnt) al.free(cnt, s);
        if (rp2) al.free(rp2, s);
        if (ci2) al.free(ci2, s);
        return MP_ERR_NOMEM;
    }
    const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(nch, (int64_t)tun.sm_count * 8));
    cudaMemsetAsync(first, 0xff, (size_t)nch * 8, s);
    kl(k_cc_count, g, CC_NT, 0, s, A.rp, A.nrows, A.ci, A.nnz, m, nch, cnt, first);
    if (scan_i64(cnt, cnt, nch, al, s)) {
        al.free(cnt, s);
        al.free(rp2, s);
        al.free(ci2, s);
        return MP_ERR_NOMEM;
    }
    kl(k_cc_fill, g, CC_NT, 0, s, A.rp, A.nrows, A.ci, A.nnz, m, nch, (const int64_t *)cnt, (const int64_t *)first,
       rp2, ci2);
    al.free(cnt, s);
    *out = DCsr{rp2, ci2, nullptr, A.nrows, A.ncols, A.nnz};  // nnz: an upper bound (not read back)
    *rp_out = rp2;
    *ci_out = ci2;
    return MP_OK;
}

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

// ------------------------------------------------------------------ row sampling

// SplitMix64 output function (Steele, Lea and Flood, 2014) of the counter seed + (i+1)*phi:
// the counter-based generator that picks sampled rows.
__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Rows of A that pass rm and have at least one entry.
__global__ void k_active_rows(DCsr A, const uint32_t *rm, unsigned long long *out) {
    unsigned long long c = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < A.nrows; i += (int64_t)gridDim.x * blockDim.x)
        c += (bit_of(rm, (uint32_t)i) && A.rp[i + 1] > A.rp[i]) ? 1ull : 0ull;
    for (int d = 16; d; d >>= 1) c += __shfl_down_sync(FULL, c, d);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

// Bitmap of the sampled rows: an active row is sampled when its SplitMix64 draw is below
// thr (so each active row is kept with probability thr / 2^64); counts the sampled rows.
__global__ void k_sample_rows(DCsr A, const uint32_t *rm, uint64_t seed, uint64_t thr, uint32_t *bm,
                              unsigned long long *count) {
    const int64_t nw = (A.nrows + 31) / 32;
    for (int64_t i0 = (blockIdx.x * (int64_t)blockDim.x) & ~31ll; i0 < nw * 32; i0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = i0 + (threadIdx.x & 31) + (threadIdx.x & ~31);
        bool take = false;
        if (i < A.nrows && bit_of(rm, (uint32_t)i) && A.rp[i + 1] > A.rp[i]) take = splitmix64(seed, (uint64_t)i) < thr;
        const unsigned word = __ballot_sync(FULL, take);
        if ((threadIdx.x & 31) == 0 && i < nw * 32) {
            bm[i >> 5] = word;
            if (word) atomicAdd(count, (unsigned long long)__popc(word));
        }
    }
}

void active_rows(const DCsr &A, const uint32_t *rm, unsigned long long *out, cudaStream_t s) {
    if (A.nrows) kl(k_active_rows, std::min(grid_for(A.nrows, 256), 1184u), 256, 0, s, A, rm, out);
}

void sample_rows(const DCsr &A, const uint32_t *rm, uint64_t seed, uint64_t thr, uint32_t *bm,
                 unsigned long long *count, cudaStream_t s) {
    const int64_t nw = (A.nrows + 31) / 32;
    if (nw) kl(k_sample_rows, std::min(grid_for(nw * 32, 256), 1184u), 256, 0, s, A, rm, seed, thr, bm, count);
}

}  // namespace mp
