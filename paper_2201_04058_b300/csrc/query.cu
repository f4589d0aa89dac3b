// Query evaluation: constraint masks (Def. 3), the chain plan (Eq. 1, Eq. 2) and the
// post-order run of the plan's sparse products.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <vector>

#include "engine.h"

using namespace mp;

namespace mp {
void mask_and_in_values(uint32_t *m, const int32_t *prop, int64_t n, const int64_t *sorted_set,
                        int64_t len, cudaStream_t s);
}

int mp_ctx::build_masks(const Query &q, std::vector<uint32_t *> &masks) {
    const int n = (int)q.types.size();
    masks.assign(n, nullptr);
    for (int i = 0; i < n; i++) {
        if (q.cons[i].empty()) continue;
        const int64_t cnt = types[q.types[i]].count;
        const size_t nw = (size_t)(cnt + 31) / 32;
        uint32_t *m = (uint32_t *)alloc->alloc(std::max<size_t>(nw, 1) * 4, stream);
        if (!m) return MP_ERR_NOMEM;
        masks[i] = m;
        mask_fill(m, cnt, true, stream);
        for (const Constraint &c : q.cons[i]) {
            const int32_t *prop = c.prop >= 0 ? props[c.prop].dev : nullptr;
            if (c.op == MP_OP_RANGE || c.op == MP_OP_EQ) {
                mask_and_range(m, prop, cnt, c.lo, c.hi, stream);
                continue;
            }
            // MP_OP_IN
            const int64_t len = (int64_t)c.set.size();
            if (!prop) {
                uint32_t *tmp = (uint32_t *)alloc->alloc(std::max<size_t>(nw, 1) * 4, stream);
                uint32_t *dset = (uint32_t *)alloc->alloc(std::max<int64_t>(len, 1) * 4, stream);
                if (!tmp || !dset) return MP_ERR_NOMEM;
                if (len) cudaMemcpyAsync(dset, c.set.data(), len * 4, cudaMemcpyHostToDevice, stream);
                mask_and_set(m, tmp, dset, len, cnt, stream);
                alloc->free(tmp, stream);
                alloc->free(dset, stream);
            } else {
                std::vector<int64_t> vs(c.set.begin(), c.set.end());
                int64_t *dset = (int64_t *)alloc->alloc(std::max<int64_t>(len, 1) * 8, stream);
                if (!dset) return MP_ERR_NOMEM;
                if (len) cudaMemcpyAsync(dset, vs.data(), len * 8, cudaMemcpyHostToDevice, stream);
                mask_and_in_values(m, prop, cnt, dset, len, stream);
                cudaStreamSynchronize(stream);  // vs is a local host buffer
                alloc->free(dset, stream);
            }
        }
    }
    return MP_OK;
}

void mp_ctx::free_masks(std::vector<uint32_t *> &masks) {
    for (auto *m : masks)
        if (m) alloc->free(m, stream);
    masks.clear();
}

// nnz of every masked factor diag(M_t) A_t diag(M_{t+1}), for the planner.
int mp_ctx::leaf_nnz(const Query &q, const std::vector<uint32_t *> &masks, std::vector<double> &nnz) {
    const int p = (int)q.rels.size();
    nnz.assign(p, 0.0);
    unsigned long long *d = (unsigned long long *)alloc->alloc((size_t)p * 8, stream);
    if (!d) return MP_ERR_NOMEM;
    cudaMemsetAsync(d, 0, (size_t)p * 8, stream);
    bool any = false;
    for (int t = 0; t < p; t++) {
        const Mat &A = rels[q.rels[t]].dev;
        if (masks[t] || masks[t + 1]) {
            uint32_t *lr = (uint32_t *)alloc->alloc((size_t)(A.nrows + 1) * 4, stream);
            if (!lr) {
                alloc->free(d, stream);
                return MP_ERR_NOMEM;
            }
            cudaMemsetAsync(lr + A.nrows, 0, 4, stream);
            masked_nnz(A.view(), masks[t], masks[t + 1], d + t, lr, lr + A.nrows, stream);
            alloc->free(lr, stream);
            any = true;
        } else {
            nnz[t] = (double)A.nnz;
        }
    }
    if (any) {
        std::vector<unsigned long long> h(p);
        cudaMemcpyAsync(h.data(), d, (size_t)p * 8, cudaMemcpyDeviceToHost, stream);
        if (cudaStreamSynchronize(stream) != cudaSuccess) {
            alloc->free(d, stream);
            return MP_ERR_CUDA;
        }
        for (int t = 0; t < p; t++)
            if (masks[t] || masks[t + 1]) nnz[t] = (double)h[t];
    }
    alloc->free(d, stream);
    return MP_OK;
}

int mp_ctx::exec(const Query &q, const std::vector<uint32_t *> &masks, const std::vector<int> &split, int p,
                 int i, int j, Operand &out, Result &r) {
    if (i == j) {
        out.m = rels[q.rels[i]].dev;
        out.owned = false;
        return MP_OK;
    }
    const int k = split[(size_t)i * p + j];
    Operand L, R;
    int rc = exec(q, masks, split, p, i, k, L, r);
    if (rc) return rc;
    rc = exec(q, masks, split, p, k + 1, j, R, r);
    if (rc) {
        if (L.owned) free_mat(L.m);
        return rc;
    }
    // A base relation enters with the masks of its two end positions; an intermediate
    // already carries them (0/1 diagonals are idempotent, so re-applying is harmless).
    const uint32_t *rm = (i == k) ? masks[i] : nullptr;
    const uint32_t *km = (i == k || k + 1 == j) ? masks[k + 1] : nullptr;
    const uint32_t *cm = (k + 1 == j) ? masks[j + 1] : nullptr;
    Mat C;
    rc = spgemm(L.m.view(), R.m.view(), rm, km, cm, *alloc, scratch, tun, stream, cfg.max_result_bytes, &C,
                &r.st, &prof);
    r.n_products++;
    if (L.owned) free_mat(L.m);
    if (R.owned) free_mat(R.m);
    if (rc) {
        free_mat(C);
        return rc;
    }
    out.m = C;
    out.owned = true;
    return MP_OK;
}

int mp_ctx::run_query(const Query &q, Result &r) {
    const int n = (int)q.types.size(), p = n - 1;
    cudaEventRecord(ev0, stream);
    std::vector<uint32_t *> masks;
    int rc = build_masks(q, masks);
    if (!rc && p == 1) {
        rc = filter(rels[q.rels[0]].dev.view(), masks[0], masks[1], *alloc, tun, stream, &r.m);
        if (rc) free_mat(r.m);
    } else if (!rc) {
        std::vector<int> split((size_t)p * p, -1);
        if (cfg.planner == MP_PLAN_LEFT_TO_RIGHT) {
            for (int i = 0; i < p; i++)
                for (int j = i + 1; j < p; j++) split[(size_t)i * p + j] = j - 1;
        } else {
            std::vector<double> dims(n), nnz;
            for (int t = 0; t < n; t++) dims[t] = (double)types[q.types[t]].count;
            rc = leaf_nnz(q, masks, nnz);
            if (!rc) plan_chain(p, dims.data(), nnz.data(), cfg.alpha, cfg.beta, cfg.gamma, nullptr, nullptr,
                                split.data(), nullptr, nullptr);
        }
        if (!rc) {
            Operand out;
            rc = exec(q, masks, split, p, 0, p - 1, out, r);
            if (!rc) r.m = out.m;
        }
    }
    free_masks(masks);
    cudaEventRecord(ev1, stream);
    cudaError_t e = cudaEventSynchronize(ev1);
    if (e != cudaSuccess && !rc) rc = MP_ERR_CUDA;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev0, ev1);
    r.ms = ms;
    r.status = rc;
    return rc;
}

int mp_ctx::run_batch(std::vector<Query> &qs, std::vector<Result> &rs) {
    int first = MP_OK;
    for (size_t i = 0; i < qs.size(); i++) {
        int rc = run_query(qs[i], rs[i]);
        if (rc && first == MP_OK) first = rc;
    }
    return first;
}

void mp_ctx::release_result(Result &r) { free_mat(r.m); }

void mp_ctx::cache_clear() {}
