// One output row of a sparse product without any device allocation.
//
// Who needs this: some callers cannot allocate device memory at the moment they need a
// product row. A serving process may have handed all free device memory to its own
// pool, so a cudaMalloc would fail; a latency-critical loop cannot accept the implicit
// device synchronisation that cudaMalloc/cudaFree may cause; an embedding runtime may
// forbid allocation outside its set-up phase. Such a caller passes its own input and
// output buffers, and this entry point works in a fixed scratch area that lives in the
// library itself: a file-scope __device__ array, present on every GPU that loads the
// library until the process exits.
//
// The computation is the split-row method of the engine's GLOBAL bin, for one row:
//   c = (x restricted to km) * Y * diag(cm), exact uint64 counts in ascending column order.
//   1. clear the row bitmap (the array keeps the previous call's contents);
//   2. every product x_k * Y[k, j] sets bit j;
//   3. rank[w] = set bits before word w (one block), total = nnz of the row;
//   4. if nnz fits the caller's capacity: write column ids at their ranks, zero the values,
//      then add every product's count into its slot.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <mutex>
#include <tuple>

#include "common.cuh"

namespace mp {

// Scratch: a bitmap and a rank word per 32 output columns, then two status words.
// ERR_RANGE (status bit): an input id outside its stated range; the call returns MP_ERR_ARG.
static constexpr unsigned long long ERR_RANGE = 8ull;
static constexpr uint32_t NOALLOC_MAX_COLS = 1u << 24;
static constexpr uint32_t NOALLOC_WORDS = NOALLOC_MAX_COLS / 32;
static __device__ __align__(256) uint32_t g_noalloc_scratch[2 * NOALLOC_WORDS + 64];

namespace {

struct NoallocRow {
    uint64_t x_len;
    const int32_t *x_ci;
    const uint64_t *x_val;
    const int64_t *y_rp;
    const int32_t *y_ci;
    const uint64_t *y_val;
    const uint32_t *km, *cm;
    uint32_t nw;
    uint32_t ncols;  // y_cols: column ids at or above it are rejected
};

__global__ void k_na_clear(uint32_t *bm, uint32_t nw, unsigned long long *status) {
    for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < nw; w += gridDim.x * blockDim.x) bm[w] = 0;
    if (blockIdx.x == 0 && threadIdx.x < 2) status[threadIdx.x] = 0;
}

// Blocks take X entries in turn; a block's threads walk that entry's Y row. A column id
// outside [0, y_cols) or a negative row id is never used as an index: it sets ERR_RANGE and
// is skipped.
template <bool NUM>
__global__ void k_na_products(NoallocRow r, uint32_t *bm, const uint32_t *rank, unsigned long long *out_val,
                              unsigned long long *status) {
    for (uint64_t p = blockIdx.x; p < r.x_len; p += gridDim.x) {
        const int32_t k = r.x_ci[p];
        if (k < 0) {
            if (threadIdx.x == 0) atomicOr(status + 1, (unsigned long long)ERR_RANGE);
            continue;
        }
        if (!bit_of(r.km, (uint32_t)k)) continue;
        const uint64_t a = (NUM && r.x_val) ? r.x_val[p] : 1ull;
        for (int64_t q = r.y_rp[k] + threadIdx.x; q < r.y_rp[k + 1]; q += blockDim.x) {
            const int32_t jc = r.y_ci[q];
            if (jc < 0 || (uint32_t)jc >= r.ncols) {
                atomicOr(status + 1, (unsigned long long)ERR_RANGE);
                continue;
            }
            const uint32_t j = (uint32_t)jc;
            if (!bit_of(r.cm, j)) continue;
            if (!NUM) {
                atomicOr(bm + (j >> 5), 1u << (j & 31));
            } else {
                const uint64_t b = r.y_val ? r.y_val[q] : 1ull;
                const uint64_t v = a * b;
                if (__umul64hi(a, b)) atomicOr(status + 1, (unsigned long long)ERR_OVERFLOW);
                const uint32_t w = j >> 5;
                const uint32_t pos = rank[w] + __popc(bm[w] & ((1u << (j & 31)) - 1u));
                const unsigned long long old = atomicAdd(out_val + pos, (unsigned long long)v);
                if (old + v < old) atomicOr(status + 1, (unsigned long long)ERR_OVERFLOW);
            }
        }
    }
}

__global__ void __launch_bounds__(1024) k_na_rank(const uint32_t *bm, uint32_t *rank, uint32_t nw,
                                                  unsigned long long *status) {
    __shared__ int64_t warp_sums[32];
    __shared__ int64_t gtot;
    int64_t carry = 0;
    for (uint32_t w0 = 0; w0 < nw; w0 += 1024) {
        const uint32_t w = w0 + threadIdx.x;
        const int c = w < nw ? __popc(bm[w]) : 0;
        const int64_t ex = block_excl_scan<1024>(c, warp_sums, &gtot);
        if (w < nw) rank[w] = (uint32_t)(carry + ex);
        carry += gtot;
    }
    if (threadIdx.x == 0) status[0] = (unsigned long long)carry;
}

__global__ void k_na_fill(const uint32_t *bm, const uint32_t *rank, uint32_t nw, int32_t *out_ci,
                          uint64_t *out_val) {
    for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < nw; w += gridDim.x * blockDim.x) {
        uint32_t word = bm[w];
        uint32_t pos = rank[w];
        while (word) {
            const int b = __ffs(word) - 1;
            word &= word - 1;
            out_ci[pos] = (int32_t)(w * 32 + b);
            out_val[pos] = 0;
            pos++;
        }
    }
}

std::mutex g_na_mu;
void *g_na_ptr[256] = {};

}  // namespace

}  // namespace mp

using namespace mp;

// The device address of the scratch array on `device`, looked up once per device with
// that device current (host code cannot use the array's name as a device address).
static int noalloc_scratch(int device, uint32_t **out) {
    std::lock_guard<std::mutex> g(g_na_mu);
    if (device < 0 || device >= 256) return MP_ERR_ARG;
    if (!g_na_ptr[device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            fprintf(stderr, "mp: cudaGetSymbolAddress: %s\n", cudaGetErrorString(e));
            cudaGetLastError();
            return MP_ERR_CUDA;
        }
        g_na_ptr[device] = p;
    }
    *out = (uint32_t *)g_na_ptr[device];
    return MP_OK;
}

// Launches one kernel and returns that launch's own error, so an error left behind by the
// caller's earlier, unrelated work is neither reported as ours nor cleared.
template <class... P, class... A>
static cudaError_t na_launch(void (*k)(P...), unsigned grid, unsigned block, cudaStream_t s, A... args) {
    const std::tuple<P...> typed(args...);
    void *argv[sizeof...(P)];
    std::apply([&](const auto &...x) {
        size_t i = 0;
        ((argv[i++] = (void *)&x), ...);
    }, typed);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaLaunchKernel((const void *)k, dim3(grid), dim3(block), argv, 0, s);
}

extern "C" int mp_row_product_noalloc(int32_t device, void *cuda_stream, uint64_t x_len, const int32_t *x_ci,
                                      const uint64_t *x_val, const int64_t *y_rp, const int32_t *y_ci,
                                      const uint64_t *y_val, uint32_t y_cols, const uint32_t *km,
                                      const uint32_t *cm, uint64_t out_cap, int32_t *out_ci, uint64_t *out_val,
                                      uint64_t *out_nnz) {
    if (!out_nnz || (x_len && (!x_ci || !y_rp || !y_ci))) return MP_ERR_ARG;
    if (y_cols > NOALLOC_MAX_COLS) {
        fprintf(stderr, "mp: mp_row_product_noalloc: %u output columns exceed the limit of %u\n", y_cols,
                NOALLOC_MAX_COLS);
        return MP_ERR_TOO_LARGE;
    }
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) return MP_ERR_CUDA;
    if (cur != device && cudaSetDevice(device) != cudaSuccess) return MP_ERR_ARG;
    auto done = [&](int code) {
        if (cur != device) cudaSetDevice(cur);
        return code;
    };
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // the call waits for its stream, which a stream under capture cannot do
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return done(MP_ERR_CUDA);
    if (cap != cudaStreamCaptureStatusNone) return done(MP_ERR_STATE);
    uint32_t *scr = nullptr;
    int rc = noalloc_scratch(device, &scr);
    if (rc) return done(rc);
    const uint32_t nw = (y_cols + 31) / 32;
    uint32_t *bm = scr, *rank = scr + NOALLOC_WORDS;
    unsigned long long *status = (unsigned long long *)(scr + 2 * NOALLOC_WORDS);  // [nnz, error bits]
    const NoallocRow r{x_len, x_ci, x_val, y_rp, y_ci, y_val, km, cm, nw, y_cols};
    const unsigned gw = std::max(1u, std::min(grid_for(nw, 256), 1184u));
    const unsigned gx = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(x_len, 1184));
    unsigned long long *no_val = nullptr;
    unsigned long long h[2] = {0, 0};
    if (na_launch(k_na_clear, gw, 256, s, bm, nw, status) != cudaSuccess) return done(MP_ERR_CUDA);
    if (x_len && na_launch(k_na_products<false>, gx, 256, s, r, bm, (const uint32_t *)rank, no_val, status) !=
                     cudaSuccess)
        return done(MP_ERR_CUDA);
    if (na_launch(k_na_rank, 1, 1024, s, (const uint32_t *)bm, rank, nw, status) != cudaSuccess)
        return done(MP_ERR_CUDA);
    if (cudaMemcpyAsync(h, status, 16, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return done(MP_ERR_CUDA);
    if (h[1] & ERR_RANGE) return done(MP_ERR_ARG);
    if (h[0] > out_cap) {
        *out_nnz = h[0];
        return done(MP_ERR_TOO_LARGE);
    }
    if (h[0] && (!out_ci || !out_val)) return done(MP_ERR_ARG);
    if (h[0]) {
        if (na_launch(k_na_fill, gw, 256, s, (const uint32_t *)bm, (const uint32_t *)rank, nw, out_ci, out_val) !=
                cudaSuccess ||
            na_launch(k_na_products<true>, gx, 256, s, r, bm, (const uint32_t *)rank, (unsigned long long *)out_val,
                      status) != cudaSuccess)
            return done(MP_ERR_CUDA);
        if (cudaMemcpyAsync(h + 1, status + 1, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return done(MP_ERR_CUDA);
        if (h[1] & ERR_OVERFLOW) return done(MP_ERR_OVERFLOW);
    }
    *out_nnz = h[0];
    return done(MP_OK);
}
