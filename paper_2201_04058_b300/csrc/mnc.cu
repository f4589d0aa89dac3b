// Device side of the MNC sketch planner (Sec. 3.2 compares the average-case estimator
// E_ac with MNC, which estimates a product's size from count sketches of its operands).
//
// A leaf factor is a base relation between the masks of its two end positions. Its exact
// sketch is four count vectors, built with one warp per row of the relation or of its
// transpose (the reverse relation, stored beside it):
//   hr[i]  = entries of row i            hc[j]  = entries of column j
//   her[i] = entries of row i in single-entry columns
//   hec[j] = entries of column j in single-entry rows
// plus per vector its sum, non-zero count, maximum and count of entries >= 2.
// Where leaf k meets leaf k+1 (over the node type at position k+1) three sums are fixed
// by the leaves alone: the product count sum hc_k hr_k+1, the exactly counted part
// sum hec_k hr_k+1 + sum (hc_k - hec_k) her_k+1, and the density-map log-sum of the
// remaining products over their p2 = r2_k * c2_k+1 cells. A DP level then asks for
// log-sums sum_t log(1 - x w[t]) with w = hc_k hr_k+1, hc_k or hr_k+1 and x set by the
// scales of the sub-chains it combines; one launch answers all of a level's requests.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <vector>

#include "common.cuh"

namespace mp {

namespace {

static constexpr int64_t MNC_LONG = 4096;  // rows longer than this are shared by all blocks

// out[i] = 0 for rows outside rm; else the entries of row i whose column passes cm and,
// with ref, whose column has ref == 1. One warp per row; rows longer than MNC_LONG get 0
// here and are queued (long_rows, *n_long) for k_mnc_rows_long.
__global__ void k_mnc_rows(DCsr A, const uint32_t *rm, const uint32_t *cm, const uint32_t *ref, uint32_t *out,
                           uint32_t *long_rows, uint32_t *n_long) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < A.nrows; i += nwarps) {
        uint32_t c = 0;
        const int64_t b = A.rp[i], e = A.rp[i + 1];
        if (bit_of(rm, (uint32_t)i)) {
            if (e - b > MNC_LONG) {
                if (lane == 0) long_rows[atomicAdd(n_long, 1u)] = (uint32_t)i;
            } else {
                for (int64_t p = b + lane; p < e; p += 32) {
                    const uint32_t j = (uint32_t)__ldg(A.ci + p);
                    c += bit_of(cm, j) && (!ref || __ldg(ref + j) == 1u);
                }
            }
        }
        for (int d = 16; d; d >>= 1) c += __shfl_xor_sync(FULL, c, d);
        if (lane == 0) out[i] = c;
    }
}

// The queued long rows: every block takes a strided share of every long row's entries and
// adds its count into out[i] (which k_mnc_rows set to 0).
__global__ void k_mnc_rows_long(DCsr A, const uint32_t *cm, const uint32_t *ref, uint32_t *out,
                                const uint32_t *long_rows, const uint32_t *n_long) {
    __shared__ uint32_t red[32];
    const uint32_t n = *n_long;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (uint32_t r = 0; r < n; r++) {
        const int64_t i = long_rows[r];
        uint32_t c = 0;
        for (int64_t p = A.rp[i] + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < A.rp[i + 1];
             p += (int64_t)gridDim.x * blockDim.x) {
            const uint32_t j = (uint32_t)__ldg(A.ci + p);
            c += bit_of(cm, j) && (!ref || __ldg(ref + j) == 1u);
        }
        for (int d = 16; d; d >>= 1) c += __shfl_xor_sync(FULL, c, d);
        if (lane == 0) red[wid] = c;
        __syncthreads();
        if (wid == 0) {
            c = lane < (int)(blockDim.x >> 5) ? red[lane] : 0u;
            for (int d = 16; d; d >>= 1) c += __shfl_xor_sync(FULL, c, d);
            if (lane == 0 && c) atomicAdd(out + i, c);
        }
        __syncthreads();
    }
}

// s[0] += sum v, s[1] += #(v > 0), s[2] = max v, s[3] += #(v >= 2).
__global__ void k_mnc_summary(const uint32_t *v, int64_t n, unsigned long long *s) {
    __shared__ unsigned long long r[4];
    if (threadIdx.x < 4) r[threadIdx.x] = 0;
    __syncthreads();
    unsigned long long sum = 0, nz = 0, mx = 0, ge2 = 0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long x = v[t];
        sum += x;
        nz += x > 0;
        mx = x > mx ? x : mx;
        ge2 += x >= 2;
    }
    for (int d = 16; d; d >>= 1) {
        sum += __shfl_xor_sync(FULL, sum, d);
        nz += __shfl_xor_sync(FULL, nz, d);
        const unsigned long long o = __shfl_xor_sync(FULL, mx, d);
        mx = o > mx ? o : mx;
        ge2 += __shfl_xor_sync(FULL, ge2, d);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&r[0], sum);
        atomicAdd(&r[1], nz);
        atomicMax(&r[2], mx);
        atomicAdd(&r[3], ge2);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicAdd(s, r[0]);
        atomicAdd(s + 1, r[1]);
        atomicMax(s + 2, r[2]);
        atomicAdd(s + 3, r[3]);
    }
}

// One request: w[t] = (a ? a[t] - a2[t] : 1) * (b ? b[t] - b2[t] : 1) over t < n (a2, b2
// may be null = 0). Results: sum_t w[t] and sum_t log(1 - x w[t]) over w > 0, with x taken
// from the request, or, when pa is set, x = 1 / (pa[0] * pb[0]) (no log-sum when that
// product is 0). A term with x w >= 1 sets the request's flag (the log-sum is -inf).
struct DevReq {
    const uint32_t *a, *a2, *b, *b2;
    int64_t n;
    double x;
    const unsigned long long *pa, *pb;
};

__global__ void k_mnc_sums(const DevReq *req, double *sum_w, double *sum_ls, unsigned *flag) {
    __shared__ double rw[32], rl[32];
    __shared__ unsigned rf;
    const DevReq R = req[blockIdx.y];
    double x = R.x;
    if (R.pa) {
        const double pp = (double)R.pa[0] * (double)R.pb[0];
        x = pp > 0 ? 1.0 / pp : 0.0;
    }
    if (threadIdx.x == 0) rf = 0;
    double sw = 0.0, sl = 0.0;
    unsigned f = 0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < R.n; t += (int64_t)gridDim.x * blockDim.x) {
        const double wa = R.a ? (double)__ldg(R.a + t) - (R.a2 ? (double)__ldg(R.a2 + t) : 0.0) : 1.0;
        const double wb = R.b ? (double)__ldg(R.b + t) - (R.b2 ? (double)__ldg(R.b2 + t) : 0.0) : 1.0;
        const double w = wa * wb;
        sw += w;
        if (x > 0.0 && w > 0.0) {
            const double xw = x * w;
            if (xw >= 1.0) f = 1;
            else sl += log1p(-xw);
        }
    }
    for (int d = 16; d; d >>= 1) {
        sw += __shfl_xor_sync(FULL, sw, d);
        sl += __shfl_xor_sync(FULL, sl, d);
    }
    f = __any_sync(FULL, f);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) {
        rw[wid] = sw;
        rl[wid] = sl;
        if (f) rf = 1;
    }
    __syncthreads();
    if (wid == 0) {
        const int nw = (int)(blockDim.x >> 5);
        sw = lane < nw ? rw[lane] : 0.0;
        sl = lane < nw ? rl[lane] : 0.0;
        for (int d = 16; d; d >>= 1) {
            sw += __shfl_xor_sync(FULL, sw, d);
            sl += __shfl_xor_sync(FULL, sl, d);
        }
        if (lane == 0) {
            atomicAdd(sum_w + blockIdx.y, sw);
            atomicAdd(sum_ls + blockIdx.y, sl);
            if (rf) atomicOr(flag + blockIdx.y, 1u);
        }
    }
}

}  // namespace

MncDevice::~MncDevice() {
    if (sum_) al_.free(sum_, s_);
    if (req_) al_.free(req_, s_);
}

int MncDevice::leaf(const MncLeafIn &in, MncSketchPtr known) {
    Leaf L;
    L.in = in;
    L.build = !known;
    L.sk = known ? known : std::make_shared<MncSketch>();
    leaves_.push_back(L);
    return (int)leaves_.size() - 1;
}

int MncDevice::pair(int a, int b) {
    pairs_.emplace_back(a, b);
    return (int)pairs_.size() - 1;
}

int MncDevice::prepare() {
    const size_t nl = leaves_.size(), np = pairs_.size();
    lstat_.assign(nl, MncLeaf{0, 0, 0, 0, 0, 0, 0});
    pstat_.assign(np, MncPair{0, 0, 0});
    if (!nl) return MP_OK;
    sum_ = (unsigned long long *)al_.alloc(nl * 8 * sizeof(unsigned long long), s_);
    if (!sum_) return MP_ERR_NOMEM;
    cudaMemsetAsync(sum_, 0, nl * 8 * sizeof(unsigned long long), s_);
    for (size_t l = 0; l < nl; l++)  // sketches from an earlier batch: their summaries as they were
        if (!leaves_[l].build)
            cudaMemcpyAsync(sum_ + 8 * l, leaves_[l].sk->raw, sizeof(leaves_[l].sk->raw), cudaMemcpyHostToDevice,
                            s_);
    const unsigned gmax = (unsigned)sms_ * 8;
    // one long-row queue (+ its counter) for every row-count pass, reused in stream order
    int64_t qmax = 1;
    for (const Leaf &L : leaves_) qmax = std::max(qmax, std::max(L.in.A.nrows, L.in.A.ncols));
    uint32_t *lq = (uint32_t *)al_.alloc((size_t)(qmax + 1) * 4, s_);
    if (!lq) return MP_ERR_NOMEM;
    auto rows = [&](const DCsr &A, const uint32_t *rm, const uint32_t *cm, const uint32_t *ref, uint32_t *out) {
        if (!A.nrows) return;
        cudaMemsetAsync(lq + qmax, 0, 4, s_);
        kl(k_mnc_rows, std::max(1u, std::min(gmax, grid_for(A.nrows * 32, 256))), 256, 0, s_, A, rm, cm, ref, out,
           lq, lq + qmax);
        kl(k_mnc_rows_long, (unsigned)sms_ * 4, 256, 0, s_, A, cm, ref, out, (const uint32_t *)lq,
           (const uint32_t *)(lq + qmax));
    };
    for (size_t l = 0; l < nl; l++) {
        Leaf &L = leaves_[l];
        if (!L.build) continue;
        MncSketch &K = *L.sk;
        const int64_t m = L.in.A.nrows, n = L.in.A.ncols;
        K.al = &al_;
        K.s = s_;
        K.hr = (uint32_t *)al_.alloc((size_t)std::max<int64_t>(m, 1) * 4, s_);
        K.her = (uint32_t *)al_.alloc((size_t)std::max<int64_t>(m, 1) * 4, s_);
        K.hc = (uint32_t *)al_.alloc((size_t)std::max<int64_t>(n, 1) * 4, s_);
        K.hec = (uint32_t *)al_.alloc((size_t)std::max<int64_t>(n, 1) * 4, s_);
        K.bytes = (size_t)(std::max<int64_t>(m, 1) + std::max<int64_t>(n, 1)) * 8;
        if (!K.hr || !K.her || !K.hc || !K.hec) {
            al_.free(lq, s_);
            return MP_ERR_NOMEM;
        }
        rows(L.in.A, L.in.rm, L.in.cm, nullptr, K.hr);
        rows(L.in.AT, L.in.cm, L.in.rm, nullptr, K.hc);
        rows(L.in.A, L.in.rm, L.in.cm, K.hc, K.her);
        rows(L.in.AT, L.in.cm, L.in.rm, K.hr, K.hec);
        if (m) kl(k_mnc_summary, std::max(1u, std::min(gmax, grid_for(m, 256))), 256, 0, s_, (const uint32_t *)K.hr, m,
                  sum_ + 8 * l);
        if (n) kl(k_mnc_summary, std::max(1u, std::min(gmax, grid_for(n, 256))), 256, 0, s_, (const uint32_t *)K.hc, n,
                  sum_ + 8 * l + 4);
    }
    al_.free(lq, s_);  // stream-ordered: after the passes above
    // per pair: product count, the two exactly counted parts, the remaining log-sum
    std::vector<DevReq> rq;
    for (size_t p = 0; p < np; p++) {
        const MncSketch &A = *leaves_[pairs_[p].first].sk, &B = *leaves_[pairs_[p].second].sk;
        const int64_t n = leaves_[pairs_[p].first].in.A.ncols;
        rq.push_back(DevReq{A.hc, nullptr, B.hr, nullptr, n, 0.0, nullptr, nullptr});
        rq.push_back(DevReq{A.hec, nullptr, B.hr, nullptr, n, 0.0, nullptr, nullptr});
        rq.push_back(DevReq{A.hc, A.hec, B.her, nullptr, n, 0.0, nullptr, nullptr});
        rq.push_back(DevReq{A.hc, A.hec, B.hr, B.her, n, 0.0, sum_ + 8 * pairs_[p].first + 3,
                            sum_ + 8 * pairs_[p].second + 7});
    }
    std::vector<double> w(rq.size()), ls(rq.size());
    std::vector<unsigned> fl(rq.size());
    if (!rq.empty()) {
        const size_t nr = rq.size();
        if (nr > req_cap_) {
            if (req_) al_.free(req_, s_);
            req_cap_ = nr;
            req_ = al_.alloc(nr * (sizeof(DevReq) + 2 * sizeof(double) + sizeof(unsigned)) + 64, s_);
            if (!req_) return MP_ERR_NOMEM;
        }
        DevReq *dq = (DevReq *)req_;
        double *dw = (double *)(dq + req_cap_), *dl = dw + req_cap_;
        unsigned *df = (unsigned *)(dl + req_cap_);
        cudaMemcpyAsync(dq, rq.data(), nr * sizeof(DevReq), cudaMemcpyHostToDevice, s_);
        cudaMemsetAsync(dw, 0, 2 * req_cap_ * sizeof(double) + req_cap_ * sizeof(unsigned), s_);
        int64_t nmax = 1;
        for (auto &r : rq) nmax = std::max(nmax, r.n);
        const unsigned gx = std::max(1u, std::min((unsigned)sms_ * 2, grid_for(nmax, 256)));
        kl(k_mnc_sums, dim3(gx, (unsigned)nr), dim3(256), 0, s_, (const DevReq *)dq, dw, dl, df);
        cudaMemcpyAsync(w.data(), dw, nr * sizeof(double), cudaMemcpyDeviceToHost, s_);
        cudaMemcpyAsync(ls.data(), dl, nr * sizeof(double), cudaMemcpyDeviceToHost, s_);
        cudaMemcpyAsync(fl.data(), df, nr * sizeof(unsigned), cudaMemcpyDeviceToHost, s_);
    }
    std::vector<unsigned long long> hs(nl * 8);
    cudaMemcpyAsync(hs.data(), sum_, nl * 8 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s_);
    if (cudaStreamSynchronize(s_) != cudaSuccess) return MP_ERR_CUDA;
    for (size_t l = 0; l < nl; l++) {
        const unsigned long long *h = hs.data() + 8 * l;
        lstat_[l] = MncLeaf{(double)h[0], (double)h[1], (double)h[2], (double)h[3],
                            (double)h[5], (double)h[6], (double)h[7]};
        if (leaves_[l].build) {
            memcpy(leaves_[l].sk->raw, h, sizeof(leaves_[l].sk->raw));
            leaves_[l].sk->stat = lstat_[l];
        }
    }
    for (size_t p = 0; p < np; p++) {
        MncPair &P = pstat_[p];
        P.dot = w[4 * p];
        P.known = w[4 * p + 1] + w[4 * p + 2];
        P.ls_ext = fl[4 * p + 3] ? -std::numeric_limits<double>::infinity() : ls[4 * p + 3];
    }
    return MP_OK;
}

int MncDevice::eval(const std::vector<MncReq> &req, std::vector<double> &ls) {
    const size_t nr = req.size();
    ls.assign(nr, 0.0);
    if (!nr) return MP_OK;
    if (nr > req_cap_) {
        if (req_) al_.free(req_, s_);
        req_cap_ = std::max<size_t>(nr, 64);
        req_ = al_.alloc(req_cap_ * (sizeof(DevReq) + 2 * sizeof(double) + sizeof(unsigned)) + 64, s_);
        if (!req_) {
            req_cap_ = 0;
            return MP_ERR_NOMEM;
        }
    }
    std::vector<DevReq> rq(nr);
    int64_t nmax = 1;
    for (size_t r = 0; r < nr; r++) {
        const MncSketch &A = *leaves_[pairs_[req[r].pair].first].sk, &B = *leaves_[pairs_[req[r].pair].second].sk;
        rq[r] = DevReq{req[r].kind != MNC_W_ROW ? A.hc : nullptr, nullptr,
                       req[r].kind != MNC_W_COL ? B.hr : nullptr, nullptr,
                       leaves_[pairs_[req[r].pair].first].in.A.ncols, req[r].x, nullptr, nullptr};
        nmax = std::max(nmax, rq[r].n);
    }
    DevReq *dq = (DevReq *)req_;
    double *dw = (double *)(dq + req_cap_), *dl = dw + req_cap_;
    unsigned *df = (unsigned *)(dl + req_cap_);
    std::vector<unsigned> fl(nr);
    cudaMemcpyAsync(dq, rq.data(), nr * sizeof(DevReq), cudaMemcpyHostToDevice, s_);
    cudaMemsetAsync(dw, 0, 2 * req_cap_ * sizeof(double) + req_cap_ * sizeof(unsigned), s_);
    const unsigned gx = std::max(1u, std::min((unsigned)sms_ * 2, grid_for(nmax, 256)));
    kl(k_mnc_sums, dim3(gx, (unsigned)nr), dim3(256), 0, s_, (const DevReq *)dq, dw, dl, df);
    cudaMemcpyAsync(ls.data(), dl, nr * sizeof(double), cudaMemcpyDeviceToHost, s_);
    cudaMemcpyAsync(fl.data(), df, nr * sizeof(unsigned), cudaMemcpyDeviceToHost, s_);
    if (cudaStreamSynchronize(s_) != cudaSuccess) return MP_ERR_CUDA;
    for (size_t r = 0; r < nr; r++)
        if (fl[r]) ls[r] = -std::numeric_limits<double>::infinity();
    return MP_OK;
}

}  // namespace mp
