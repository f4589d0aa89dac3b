// Query and workload evaluation: constraint masks (Def. 3), chain plans (Eq. 1, Eq. 2),
// the product DAG of a batch of queries, and the Overlap-Tree cache (Sec. 3.3, 3.4).
//
// A batch of queries becomes one DAG of sparse products. Every internal node of a
// query's plan is a sub-chain, identified by its node types, relations and the
// constraints on its positions; identical sub-chains of different queries become one
// node, and a sub-chain whose result is cached becomes a finished node. Planning sees
// both as known sub-chains with retrieval cost 0 (end of Sec. 3.2). Nodes run level by
// level (a node's level is one more than its deepest child). After the batch, each
// query's whole result and the longest sub-metapath it computed that has occurred at
// least twice are offered to the cache (Sec. 3.4.1), whose replacement policy decides
// (Alg. 1).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <functional>
#include <map>
#include <memory>
#include <string>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "engine.h"

using namespace mp;
using Query = mp_ctx::Query;
using Result = mp_ctx::Result;

namespace mp {
void mask_and_in_values(uint32_t *m, const int32_t *prop, int64_t n, const int64_t *sorted_set,
                        int64_t len, cudaStream_t s);
}

MatPtr mp_ctx::wrap(const Mat &m, bool charged) {
    auto p = std::make_shared<DevMat>();
    p->m = m;
    p->al = alloc.get();
    p->s = stream;
    p->held = &held;
    p->charged = (int64_t)m.bytes();
    if (!charged) {
        held.fetch_add(p->charged);
        note_held();
    }
    return p;
}

void mp_ctx::free_mat(Mat &m) {
    if (m.rp) alloc->free(m.rp, stream);
    if (m.ci) alloc->free(m.ci, stream);
    if (m.val) alloc->free(m.val, stream);
    m = Mat{};
}

void mp_ctx::release_result(Result &r) { r.m.reset(); }

void mp_ctx::cache_clear() {
    if (cache) cache->clear();
    htier_clear();
}

void mp_ctx::htier_clear() {
    if (htier.arena) cudaStreamSynchronize(stream);  // no copy may still use the arena
    htier.free_blocks.clear();
    if (htier.cap) htier.free_blocks.emplace(0, htier.cap);
    htier.items.clear();
    htier.bytes = 0;
}

bool mp_ctx::htier_init() {
    const size_t cap = (size_t)cfg.host_tier_bytes;
    if (cudaMallocHost((void **)&htier.arena, cap) != cudaSuccess) {
        cudaGetLastError();
        htier.arena = nullptr;
        return false;
    }
    htier.cap = cap;
    htier.free_blocks.clear();
    htier.free_blocks.emplace(0, cap);
    // the copy-back rate the planner prices a load with: one timed copy of up to 64 MB
    const size_t probe = std::min<size_t>(cap, 64u << 20);
    void *d = alloc->alloc(probe, stream);
    if (d) {
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaMemcpyAsync(d, htier.arena, probe, cudaMemcpyHostToDevice, stream);  // warm the path
        cudaEventRecord(e0, stream);
        cudaMemcpyAsync(d, htier.arena, probe, cudaMemcpyHostToDevice, stream);
        cudaEventRecord(e1, stream);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms > 0.f) htier.h2d_gbs = (double)probe / (ms * 1e6);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        alloc->free(d, stream);
    }
    if (htier.h2d_gbs <= 0.0) htier.h2d_gbs = 20.0;
    return true;
}

void mp_ctx::htier_release(size_t off, size_t bytes) {
    auto it = htier.free_blocks.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != htier.free_blocks.end() && it->first + it->second == nx->first) {
        it->second += nx->second;
        htier.free_blocks.erase(nx);
    }
    if (it != htier.free_blocks.begin()) {
        auto pv = std::prev(it);
        if (pv->first + pv->second == it->first) {
            pv->second += it->second;
            htier.free_blocks.erase(it);
        }
    }
}

bool mp_ctx::htier_reserve(size_t bytes, size_t *off) {
    for (;;) {
        for (auto &fb : htier.free_blocks)
            if (fb.second >= bytes) {
                *off = fb.first;
                const size_t rest = fb.second - bytes, at = fb.first + bytes;
                htier.free_blocks.erase(fb.first);
                if (rest) htier.free_blocks.emplace(at, rest);
                return true;
            }
        if (htier.items.empty()) return false;
        auto lru = htier.items.begin();
        for (auto x = htier.items.begin(); x != htier.items.end(); ++x)
            if (x->second.seq < lru->second.seq) lru = x;
        htier_release(lru->second.off, lru->second.bytes);
        htier.bytes -= lru->second.bytes;
        htier.items.erase(lru);
        htier.drops++;
    }
}

void mp_ctx::htier_store(const std::string &id, const MatPtr &m, const std::vector<int32_t> &types,
                         const std::string &key, double c_ms, double c_ops) {
    const size_t cap = (size_t)cfg.host_tier_bytes;
    if (!cap || !m) return;
    auto it = htier.items.find(id);
    if (it != htier.items.end()) {  // already held (loaded back earlier): refresh it
        it->second.seq = ++htier.seq;
        return;
    }
    if (!htier.arena) return;
    const Mat &A = m->m;
    const size_t brp = (size_t)(A.nrows + 1) * 8, bci = (size_t)A.nnz * 4, bval = (size_t)A.nnz * 8;
    const size_t bytes = (brp + bci + bval + 15) & ~(size_t)15;
    if ((double)bytes > 0.8 * (double)cap) return;  // the 80 % rule of the device cache
    size_t off = 0;
    if (!htier_reserve(bytes, &off)) return;
    char *b = htier.arena + off;
    cudaMemcpyAsync(b, A.rp, brp, cudaMemcpyDeviceToHost, stream);
    if (A.nnz) {
        cudaMemcpyAsync(b + brp, A.ci, bci, cudaMemcpyDeviceToHost, stream);
        cudaMemcpyAsync(b + brp + bci, A.val, bval, cudaMemcpyDeviceToHost, stream);
    }
    HostEntry e;
    e.types = types;
    e.key = key;
    e.shape = A;
    e.shape.rp = nullptr;
    e.shape.ci = nullptr;
    e.shape.val = nullptr;
    e.shape.arows = nullptr;  // copied back without its row list (any row may be non-empty)
    e.shape.narows = 0;
    e.shape.arows_hold.reset();
    e.off = off;
    e.bytes = bytes;
    e.c_ms = c_ms;
    e.c_ops = c_ops;
    e.seq = ++htier.seq;
    htier.bytes += bytes;
    htier.items.emplace(id, std::move(e));
    htier.stores++;
}

double mp_ctx::htier_cost(const std::string &id) const {
    auto it = htier.items.find(id);
    if (it == htier.items.end()) return NAN;
    // the recorded cost scaled by (copy-back time / computation time), at most the cost
    const HostEntry &e = it->second;
    const double copy_ms = (double)e.bytes / (htier.h2d_gbs * 1e6);
    return e.c_ms > 0 ? e.c_ops * std::min(1.0, copy_ms / e.c_ms) : e.c_ops;
}

MatPtr mp_ctx::htier_load(const std::string &id) {
    auto it = htier.items.find(id);
    if (it == htier.items.end()) return nullptr;
    it->second.seq = ++htier.seq;  // most recently used: the last the host tier would drop
    const Mat shape = it->second.shape;
    // the budget first (the cache may yield, and its evictions may store into the host tier)
    if (reserve_bytes((int64_t)shape.bytes())) return nullptr;  // the budget cannot hold it: recompute
    it = htier.items.find(id);
    if (it == htier.items.end()) {
        unreserve_bytes((int64_t)shape.bytes());
        return nullptr;
    }
    const HostEntry &e = it->second;
    Mat m = shape;
    const size_t brp = (size_t)(m.nrows + 1) * 8, bci = (size_t)m.nnz * 4, bval = (size_t)m.nnz * 8;
    m.rp = (int64_t *)alloc->alloc(brp, stream);
    m.ci = (int32_t *)alloc->alloc(std::max<size_t>(bci, 4), stream);
    m.val = (uint64_t *)alloc->alloc(std::max<size_t>(bval, 8), stream);
    if (!m.rp || !m.ci || !m.val) {
        unreserve_bytes((int64_t)shape.bytes());
        free_mat(m);
        return nullptr;
    }
    // ordered on the stream before every kernel that reads the result; a later store that
    // reuses this arena block copies into it on the same stream, after this copy
    const char *b = htier.arena + e.off;
    cudaMemcpyAsync(m.rp, b, brp, cudaMemcpyHostToDevice, stream);
    if (m.nnz) {
        cudaMemcpyAsync(m.ci, b + brp, bci, cudaMemcpyHostToDevice, stream);
        cudaMemcpyAsync(m.val, b + brp + bci, bval, cudaMemcpyHostToDevice, stream);
    }
    htier.loads++;
    return wrap(m, true);
}

int mp_ctx::build_masks(const Query &q, std::vector<uint32_t *> &masks, std::vector<int32_t *> *rows,
                        std::vector<int64_t> *nrows, std::vector<std::shared_ptr<const int32_t>> *holds) {
    const int n = (int)q.types.size();
    masks.assign(n, nullptr);
    if (rows) rows->assign(n, nullptr);
    if (nrows) nrows->assign(n, 0);
    if (holds) holds->assign(n, nullptr);
    // a row list's owner: freed (stream ordered) when the query and every result that
    // inherited the list have let go of it
    Alloc *al = alloc.get();
    cudaStream_t s = stream;
    auto hold = [al, s](int32_t *p) { return std::shared_ptr<const int32_t>(p, [al, s](const int32_t *x) { al->free((void *)x, s); }); };
    for (int i = 0; i < n; i++) {
        if (q.cons[i].empty()) continue;
        // a position of the same type with the same constraints (the canonical key) shares
        // its mask (every P of a year-windowed metapath, say)
        for (int j = 0; j < i && !masks[i]; j++)
            if (masks[j] && q.types[j] == q.types[i] && q.pos_keys[j] == q.pos_keys[i]) {
                masks[i] = masks[j];
                if (rows) (*rows)[i] = (*rows)[j];
                if (nrows) (*nrows)[i] = (*nrows)[j];
                if (holds) (*holds)[i] = (*holds)[j];
            }
        if (masks[i]) continue;
        const int64_t cnt = types[q.types[i]].count;
        const size_t nw = (size_t)(cnt + 31) / 32;
        uint32_t *m = (uint32_t *)alloc->alloc(std::max<size_t>(nw, 1) * 4, stream);
        if (!m) return MP_ERR_NOMEM;
        masks[i] = m;
        // the first constraint stores its words when it is a range; otherwise all ones first
        const bool first_range = q.cons[i][0].op == MP_OP_RANGE || q.cons[i][0].op == MP_OP_EQ;
        if (rows && holds && first_range && q.cons[i].size() == 1 && q.cons[i][0].prop < 0) {
            // the position's only constraint is a window of node ids: those ids are its row
            // list when they are few (an anchor entity, say)
            const int64_t lo = std::max<int64_t>(q.cons[i][0].lo, 0);
            const int64_t hi = std::min<int64_t>(q.cons[i][0].hi, cnt - 1);
            const int64_t len = std::max<int64_t>(hi - lo + 1, 0);
            if (len * 8 <= cnt) {
                int32_t *d = (int32_t *)alloc->alloc((size_t)std::max<int64_t>(len, 1) * 4, stream);
                if (!d) return MP_ERR_NOMEM;
                fill_iota(d, lo, len, stream);
                (*rows)[i] = d;
                (*nrows)[i] = len;
                (*holds)[i] = hold(d);
            }
        }
        if (!first_range) mask_fill(m, cnt, true, stream);
        bool first = true;
        for (const Constraint &c : q.cons[i]) {
            const int32_t *prop = c.prop >= 0 ? props[c.prop].dev : nullptr;
            if (c.op == MP_OP_RANGE || c.op == MP_OP_EQ) {
                mask_and_range(m, prop, cnt, c.lo, c.hi, stream, first && first_range);
                first = false;
                continue;
            }
            first = false;
            const int64_t len = (int64_t)c.set.size();
            if (!prop) {
                uint32_t *tmp = (uint32_t *)alloc->alloc(std::max<size_t>(nw, 1) * 4, stream);
                uint32_t *dset = (uint32_t *)alloc->alloc(std::max<int64_t>(len, 1) * 4, stream);
                if (!tmp || !dset) {
                    if (tmp) alloc->free(tmp, stream);
                    if (dset) alloc->free(dset, stream);
                    return MP_ERR_NOMEM;
                }
                if (len) cudaMemcpyAsync(dset, c.set.data(), len * 4, cudaMemcpyHostToDevice, stream);
                mask_and_set(m, tmp, dset, len, cnt, stream);
                alloc->free(tmp, stream);
                if (rows && holds && q.cons[i].size() == 1) {
                    // the position's only constraint: the set (sorted, without repeats since
                    // parsing) is also its row list, without the ids past the type's count
                    (*rows)[i] = (int32_t *)dset;
                    (*nrows)[i] = std::lower_bound(c.set.begin(), c.set.end(), (uint32_t)std::min<int64_t>(cnt, UINT32_MAX)) -
                                  c.set.begin();
                    (*holds)[i] = hold((int32_t *)dset);
                } else {
                    alloc->free(dset, stream);
                }
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
    for (size_t i = 0; i < masks.size(); i++) {
        if (!masks[i]) continue;
        bool shared = false;  // positions with equal constraints hold one mask
        for (size_t j = 0; j < i && !shared; j++) shared = masks[j] == masks[i];
        if (!shared) alloc->free(masks[i], stream);
    }
    masks.clear();
}

namespace {

std::string subchain_key(const Query &q, int i, int j) {
    return window_key(q.pos_keys, (size_t)i, (size_t)(j - i + 2));
}

std::vector<int32_t> subchain_types(const Query &q, int i, int j) {
    return std::vector<int32_t>(q.types.begin() + i, q.types.begin() + j + 2);
}

}  // namespace

mp_ctx::QState::~QState() {
    if (ctx) {
        ctx->free_masks(masks);
        ctx->free_row_lists(rows, nrows);
    }
}

void mp_ctx::free_row_lists(std::vector<int32_t *> &rows, std::vector<int64_t> &nrows) {
    rows.clear();  // the lists themselves go with their owners (shared with results)
    nrows.clear();
}

// ------------------------------------------------------------------ HBM byte budget

bool mp_ctx::evict_one() {
    if (!cache) return false;
    CacheItem it;
    if (!cache->evict_victim(&it)) return false;
    cstats.evictions++;
    OTEntry *ee = otree.entry(it.types.data(), it.types.size(), it.key);
    if (ee) ee->cached = false;
    htier_store(it.id, std::static_pointer_cast<DevMat>(it.payload), it.types, it.key, it.c, ee ? ee->c_ops : 0.0);
    return true;
}

// Charge `bytes` of a result about to be made to the budget; cache entries are evicted
// (the policy's victims first) while the budget cannot hold it. A budget of 0 is no limit.
int mp_ctx::reserve_bytes(int64_t bytes) {
    const int64_t budget = (int64_t)cfg.hbm_budget_bytes;
    if (budget > 0) {
        while (held.load() + bytes > budget && evict_one()) {
        }
        if (held.load() + bytes > budget) return MP_ERR_BUDGET;
    }
    held.fetch_add(bytes);
    note_held();
    return MP_OK;
}

void mp_ctx::unreserve_bytes(int64_t bytes) { held.fetch_sub(bytes); }

namespace {
// The budget as the wave executor sees it.
struct CtxBudget final : mp::Budget {
    mp_ctx *c;
    explicit CtxBudget(mp_ctx *x) : c(x) {}
    int reserve(int64_t bytes) override { return c->reserve_bytes(bytes); }
    void unreserve(int64_t bytes) override { c->unreserve_bytes(bytes); }
};
}  // namespace

// ------------------------------------------------------------------ the executor

int mp_ctx::admit(std::vector<Query> &qs_in, const std::vector<uint64_t> &tickets,
                  const std::vector<std::chrono::steady_clock::time_point> &t0s, std::vector<int64_t> &ids) {
    const size_t nq = qs_in.size();
    ids.assign(nq, -1);
    std::vector<std::shared_ptr<QState>> st(nq);
    std::vector<int> qstatus(nq, MP_OK);
    for (size_t q = 0; q < nq; q++) {
        st[q] = std::make_shared<QState>();
        st[q]->ctx = this;
        st[q]->q = std::move(qs_in[q]);
        qstatus[q] = build_masks(st[q]->q, st[q]->masks, &st[q]->rows, &st[q]->nrows, &st[q]->rows_hold);
    }
    std::vector<Flight *> fl(nq);
    for (size_t q = 0; q < nq; q++) {
        const int64_t id = ex.next_flight++;
        Flight &f = ex.flights[id];
        f.id = id;
        f.qs = st[q];
        f.status = qstatus[q];
        f.ticket = tickets[q];
        f.t0 = t0s[q];
        ids[q] = id;
        fl[q] = &f;  // std::map: stable while other flights come and go
    }
    // a failure before the products join the DAG: every query of this admission reports it
    auto fail_all = [&](int rc) {
        for (size_t q = 0; q < nq; q++)
            if (!fl[q]->status) fl[q]->status = rc;
        return rc;
    };

    // exact nnz of every masked base factor, for the planner: one device array, one sync;
    // counts already seen (same relation, same constraints at both ends) come from a memo
    std::vector<std::vector<double>> leaf(nq);
    {
        size_t total = 0;
        for (auto &x : st) total += x->q.rels.size();
        unsigned long long *d = (unsigned long long *)alloc->alloc(std::max<size_t>(total, 1) * 8, stream);
        if (!d) return fail_all(MP_ERR_NOMEM);
        cudaMemsetAsync(d, 0, std::max<size_t>(total, 1) * 8, stream);
        std::vector<void *> tmp;
        auto free_tmp = [&] {
            for (void *x : tmp) alloc->free(x, stream);
            alloc->free(d, stream);
        };
        std::vector<std::string> keys(total);
        std::unordered_map<std::string, size_t> first;  // key -> slot counted in this batch
        size_t off = 0;
        bool any = false;
        for (size_t q = 0; q < nq; q++) {
            const int p = (int)st[q]->q.rels.size();
            leaf[q].assign(p, -1.0);
            for (int t = 0; t < p; t++) {
                const Mat &A = rels[st[q]->q.rels[t]].dev;
                if (qstatus[q] || !(st[q]->masks[t] || st[q]->masks[t + 1])) continue;
                std::string &key = keys[off + t];
                key = std::to_string(st[q]->q.rels[t]) + "|" + st[q]->q.pos_keys[t] + "|" + st[q]->q.pos_keys[t + 1];
                auto m = leaf_memo.find(key);
                if (m != leaf_memo.end()) {
                    leaf[q][t] = m->second;
                    continue;
                }
                if (first.count(key)) continue;
                first.emplace(key, off + t);
                any = true;
                if ((size_t)t < st[q]->rows.size() && st[q]->rows[t] && st[q]->nrows[t] * 8 <= A.nrows) {
                    // rows selected by node ids: count over the listed rows only
                    masked_nnz_list(A.view(), st[q]->rows[t], st[q]->nrows[t], st[q]->masks[t + 1], d + off + t, stream);
                    continue;
                }
                uint32_t *lr = (uint32_t *)alloc->alloc((size_t)(A.nrows + 1) * 4, stream);
                if (!lr) {
                    free_tmp();
                    return fail_all(MP_ERR_NOMEM);
                }
                cudaMemsetAsync(lr + A.nrows, 0, 4, stream);
                masked_nnz(A.view(), st[q]->masks[t], st[q]->masks[t + 1], d + off + t, lr, lr + A.nrows, stream);
                tmp.push_back(lr);
                any = true;
            }
            off += p;
        }
        std::vector<unsigned long long> h(std::max<size_t>(total, 1), 0);
        if (any) {
            Readback rb(&wcache, stream);
            if (!rb.get(h.data(), d, std::max<size_t>(total, 1) * 8) || !rb.sync()) {
                free_tmp();
                return fail_all(MP_ERR_CUDA);
            }
        }
        free_tmp();
        if (leaf_memo.size() > 65536) leaf_memo.clear();
        for (auto &kv : first) leaf_memo[kv.first] = (double)h[kv.second];
        off = 0;
        for (size_t q = 0; q < nq; q++) {
            for (size_t t = 0; t < st[q]->q.rels.size(); t++) {
                if (leaf[q][t] >= 0) continue;
                const std::string &key = keys[off + t];
                leaf[q][t] = key.empty() ? (double)rels[st[q]->q.rels[t]].dev.nnz : leaf_memo[key];
            }
            off += st[q]->q.rels.size();
        }
    }

    // sampled densities of every adjacent factor pair (MP_PLAN_DP_SAMPLED): the exact
    // output size of up to sample_rows seeded rows of the pair's first factor
    std::vector<std::vector<double>> sampled;
    if (cfg.planner == MP_PLAN_DP_SAMPLED) {
        struct Pair { size_t q; int t; };
        std::vector<Pair> pairs;
        for (size_t q = 0; q < nq; q++)
            if (!qstatus[q])
                for (int t = 0; t + 1 < (int)st[q]->q.rels.size(); t++) pairs.push_back({q, t});
        sampled.assign(nq, std::vector<double>());
        for (size_t q = 0; q < nq; q++) {
            const size_t p = st[q]->q.rels.size();
            sampled[q].assign(p * p, NAN);
        }
        if (!pairs.empty()) {
            const size_t np = pairs.size();
            unsigned long long *d = (unsigned long long *)alloc->alloc(np * 16, stream);
            if (!d) return fail_all(MP_ERR_NOMEM);
            cudaMemsetAsync(d, 0, np * 16, stream);  // [active rows, sampled rows] per pair
            for (size_t k = 0; k < np; k++) {
                const Query &Q = st[pairs[k].q]->q;
                active_rows(rels[Q.rels[pairs[k].t]].dev.view(), st[pairs[k].q]->masks[pairs[k].t], d + 2 * k, stream);
            }
            std::vector<unsigned long long> h(2 * np);
            cudaMemcpyAsync(h.data(), d, np * 16, cudaMemcpyDeviceToHost, stream);
            if (cudaStreamSynchronize(stream) != cudaSuccess) {
                alloc->free(d, stream);
                return fail_all(MP_ERR_CUDA);
            }
            std::vector<uint32_t *> bms(np, nullptr);
            std::vector<WaveIn> win(np);
            const double s_rows = (double)std::max<uint32_t>(cfg.sample_rows, 1);
            for (size_t k = 0; k < np; k++) {
                const Query &Q = st[pairs[k].q]->q;
                const int t = pairs[k].t;
                const Mat &A = rels[Q.rels[t]].dev;
                const double act = (double)h[2 * k];
                const uint64_t thr = act <= s_rows ? UINT64_MAX : (uint64_t)(s_rows / act * 18446744073709551615.0);
                bms[k] = (uint32_t *)alloc->alloc((size_t)std::max<int64_t>((A.nrows + 31) / 32, 1) * 4, stream);
                if (!bms[k]) {
                    for (auto *b : bms)
                        if (b) alloc->free(b, stream);
                    alloc->free(d, stream);
                    return fail_all(MP_ERR_NOMEM);
                }
                const uint64_t seed = cfg.seed ^ (0x9E3779B97F4A7C15ull * (uint64_t)(k + 1));
                sample_rows(A.view(), st[pairs[k].q]->masks[t], seed, thr, bms[k], d + 2 * k + 1, stream);
                win[k].X = A.view();
                win[k].Y = rels[Q.rels[t + 1]].dev.view();
                win[k].rm = bms[k];
                win[k].km = st[pairs[k].q]->masks[t + 1];
                win[k].cm = st[pairs[k].q]->masks[t + 2];
            }
            std::vector<WaveOut> wout;
            int rc = spgemm_wave(win, *alloc, tun, stream, 0, wout, nullptr, true, &wcache);
            cudaMemcpyAsync(h.data(), d, np * 16, cudaMemcpyDeviceToHost, stream);
            if (cudaStreamSynchronize(stream) != cudaSuccess) rc = MP_ERR_CUDA;
            for (auto *b : bms) alloc->free(b, stream);
            alloc->free(d, stream);
            if (rc) return fail_all(rc);
            for (size_t k = 0; k < np; k++) {
                const Query &Q = st[pairs[k].q]->q;
                const int t = pairs[k].t;
                const size_t p = Q.rels.size();
                const double act = (double)h[2 * k], smp = (double)h[2 * k + 1];
                const double rows = (double)rels[Q.rels[t]].dev.nrows, cols = (double)rels[Q.rels[t + 1]].dev.ncols;
                const double dens = smp > 0 ? ((double)wout[k].m.nnz / smp) * act / (rows * cols) : 0.0;
                if (!wout[k].status) sampled[pairs[k].q][(size_t)t * p + t + 1] = dens;
            }
        }
    }

    // MNC sketches (MP_PLAN_DP_MNC): one exact sketch per distinct masked leaf, the fixed
    // sums of every adjacent leaf pair, all in one pass and one sync
    MncDevice mnc(*alloc, stream, tun.sm_count);
    std::vector<std::vector<int>> mleaf(nq), mpair(nq);
    if (cfg.planner == MP_PLAN_DP_MNC) {
        std::unordered_map<std::string, int> lidx;
        std::vector<std::string> lkey;  // per leaf of `mnc`
        std::map<std::pair<int, int>, int> pidx;
        for (size_t q = 0; q < nq; q++) {
            if (qstatus[q]) continue;
            const Query &Q = st[q]->q;
            const int p = (int)Q.rels.size();
            mleaf[q].assign(p, -1);
            mpair[q].assign(p, -1);
            for (int t = 0; t < p; t++) {
                const std::string key =
                    std::to_string(Q.rels[t]) + "|" + Q.pos_keys[t] + "|" + Q.pos_keys[t + 1];
                auto it = lidx.find(key);
                if (it == lidx.end()) {
                    MncLeafIn in{rels[Q.rels[t]].dev.view(), rels[Q.rels[t] ^ 1].dev.view(), st[q]->masks[t],
                                 st[q]->masks[t + 1]};
                    auto mm = mnc_memo.find(key);
                    MncSketchPtr known;
                    if (mm != mnc_memo.end()) {
                        known = mm->second.sk;
                        mm->second.seq = ++mnc_memo_seq;
                    }
                    it = lidx.emplace(key, mnc.leaf(in, known)).first;
                    lkey.push_back(key);
                }
                mleaf[q][t] = it->second;
            }
            for (int k = 0; k + 1 < p; k++) {
                const std::pair<int, int> key(mleaf[q][k], mleaf[q][k + 1]);
                auto it = pidx.find(key);
                if (it == pidx.end()) it = pidx.emplace(key, mnc.pair(key.first, key.second)).first;
                mpair[q][k] = it->second;
            }
        }
        const int rc = mnc.prepare();
        if (rc) return fail_all(rc);
        // keep the new sketches for later batches
        for (size_t l = 0; l < lkey.size(); l++) {
            if (!mnc.built((int)l)) continue;
            MncSketchPtr sk = mnc.sketch((int)l);
            if (sk->bytes > MNC_MEMO_CAP / 2) continue;
            while (mnc_memo_bytes + sk->bytes > MNC_MEMO_CAP && !mnc_memo.empty()) {
                auto lru = mnc_memo.begin();
                for (auto x = mnc_memo.begin(); x != mnc_memo.end(); ++x)
                    if (x->second.seq < lru->second.seq) lru = x;
                mnc_memo_bytes -= lru->second.sk->bytes;
                mnc_memo.erase(lru);
            }
            mnc_memo[lkey[l]] = MncMemo{sk, ++mnc_memo_seq};
            mnc_memo_bytes += sk->bytes;
        }
    }

    // Overlap Tree: every query's metapath and suffixes (Sec. 3.3.2)
    if (cache && !explain.on)
        for (size_t q = 0; q < nq; q++)
            if (!qstatus[q]) otree.insert(st[q]->q.types, st[q]->q.pos_keys);

    // plans, and the queries' products joined to the DAG: a sub-chain whose result is on
    // its way or held (in flight for an earlier query) becomes a shared node
    std::unique_ptr<TraceRange> plan_range(new TraceRange("mp.plan"));
    std::unordered_set<std::string> host_known;  // sub-chains planned as copies from the host tier
    for (size_t q = 0; q < nq; q++) {
        if (qstatus[q]) continue;
        const Query &Q = st[q]->q;
        Flight &F = *fl[q];
        const int64_t fid = ids[q];
        const int n = (int)Q.types.size(), p = n - 1;
        std::vector<double> dims(n);
        for (int t = 0; t < n; t++) dims[t] = (double)types[Q.types[t]].count;
        if (p == 1 && explain.on) {
            explain.p = 1;
            explain.split.assign(1, -1);
            explain.nnz.assign(1, leaf[q][0] >= 0 ? leaf[q][0] : (double)rels[Q.rels[0]].dev.nnz);
            return fail_all(MP_OK);
        }
        if (p == 1) {
            PNode nd;
            nd.id = "filter#" + std::to_string(fid);
            nd.flight = fid;
            nd.qs = st[q];
            nd.filter = true;
            nd.keepers = 1;
            F.keeps.push_back(ex.next_node);
            F.est_bytes = (dims[0] + 1) * 8.0 + 12.0 * (leaf[q][0] >= 0 ? leaf[q][0] : (double)rels[Q.rels[0]].dev.nnz);
            const int64_t nid = ex.next_node++;
            ex.nodes.emplace(nid, std::move(nd));
            F.root = nid;
            ex.est_bytes += F.est_bytes;
            continue;
        }
        // sub-chains already known: in the cache, in flight, or evicted with a recorded cost
        std::vector<double> kc((size_t)p * p, NAN), kr((size_t)p * p, NAN);
        for (int i = 0; i < p; i++)
            for (int j = i + 1; j < p; j++) {
                const std::vector<int32_t> ty = subchain_types(Q, i, j);
                const std::string key = subchain_key(Q, i, j);
                const std::string id = CachePolicy::make_id(ty, key);
                const double cells = dims[i] * dims[j + 1];
                auto it = ex.by_id.find(id);
                if (it != ex.by_id.end() && node(it->second).status) {  // failed: compute anew
                    ex.by_id.erase(it);
                    it = ex.by_id.end();
                }
                if (it != ex.by_id.end()) {
                    kc[(size_t)i * p + j] = 0.0;
                    kr[(size_t)i * p + j] = node(it->second).rho_est;
                    continue;
                }
                if (cache) {
                    CacheItem *ci = cache->find(id);
                    if (ci) {
                        kc[(size_t)i * p + j] = 0.0;
                        kr[(size_t)i * p + j] = (double)std::static_pointer_cast<DevMat>(ci->payload)->m.nnz / cells;
                        continue;
                    }
                    const double hcost = htier_cost(id);
                    if (!std::isnan(hcost)) {  // in the host tier: the cost of copying it back
                        kc[(size_t)i * p + j] = hcost;
                        kr[(size_t)i * p + j] = (double)htier.items[id].shape.nnz / cells;
                        host_known.insert(id);
                        continue;
                    }
                    OTEntry *e = otree.entry(ty.data(), ty.size(), key);
                    if (e && e->c_ops >= 0.0) {
                        kc[(size_t)i * p + j] = e->c_ops;
                        kr[(size_t)i * p + j] = e->nnz / cells;
                    }
                }
            }
        std::vector<int> split((size_t)p * p, -1), split_pure((size_t)p * p, -1);
        std::vector<double> D((size_t)p * p, 0.0);
        if (cfg.planner == MP_PLAN_LEFT_TO_RIGHT) {
            for (int i = 0; i < p; i++)
                for (int j = i + 1; j < p; j++) split[(size_t)i * p + j] = split_pure[(size_t)i * p + j] = j - 1;
            // sizes for the byte estimate: E_ac densities
            std::vector<int> tmp((size_t)p * p);
            plan_chain(p, dims.data(), leaf[q].data(), cfg.alpha, cfg.beta, cfg.gamma, nullptr, nullptr, nullptr,
                       tmp.data(), nullptr, D.data());
        } else if (cfg.planner == MP_PLAN_DP_MNC) {
            // the plan with the known sub-chains and the plan of every sub-chain on its
            // own, level by level; each level's log-sums in one launch
            std::vector<MncLeaf> lv(p);
            std::vector<MncPair> pv(p, MncPair{0, 0, 0});
            for (int t = 0; t < p; t++) lv[t] = mnc.leaf_stat(mleaf[q][t]);
            for (int t = 0; t + 1 < p; t++) pv[t] = mnc.pair_stat(mpair[q][t]);
            std::vector<double> kz((size_t)p * p, NAN);
            for (int i = 0; i < p; i++)
                for (int j = i + 1; j < p; j++)
                    if (!std::isnan(kc[(size_t)i * p + j]))
                        kz[(size_t)i * p + j] = kr[(size_t)i * p + j] * dims[i] * dims[j + 1];
            MncPlan known(p, dims.data(), lv.data(), pv.data(), cfg.alpha, cfg.beta, cfg.gamma, kc.data(),
                          kz.data());
            MncPlan pure(p, dims.data(), lv.data(), pv.data(), cfg.alpha, cfg.beta, cfg.gamma, nullptr, nullptr);
            for (int len = 2; len <= p; len++) {
                std::vector<MncReq> req;
                known.requests(len, req);
                pure.requests(len, req);
                for (MncReq &r : req) r.pair = mpair[q][r.pair];
                std::vector<double> ls;
                const int rc = mnc.eval(req, ls);
                if (rc) return fail_all(rc);
                known.resolve(len, ls.data());
                pure.resolve(len, ls.data());
            }
            for (size_t t = 0; t < (size_t)p * p; t++) {
                split[t] = known.split[t];
                split_pure[t] = pure.split[t];
                const int i = (int)(t / p), j = (int)(t % p);
                D[t] = j >= i ? known.nnz[t] / (dims[i] * dims[j + 1]) : 0.0;
            }
        } else {
            const double *rf = sampled.empty() ? nullptr : sampled[q].data();
            plan_chain(p, dims.data(), leaf[q].data(), cfg.alpha, cfg.beta, cfg.gamma, kc.data(), kr.data(), rf,
                       split.data(), nullptr, D.data());
            // plan of every sub-chain on its own, for known sub-chains that still need computing
            plan_chain(p, dims.data(), leaf[q].data(), cfg.alpha, cfg.beta, cfg.gamma, nullptr, nullptr, rf,
                       split_pure.data(), nullptr, nullptr);
        }
        if (explain.on) {
            explain.p = p;
            explain.split = split;
            explain.nnz.assign((size_t)p * p, 0.0);
            for (int i = 0; i < p; i++)
                for (int j = i; j < p; j++)
                    explain.nnz[(size_t)i * p + j] = D[(size_t)i * p + j] * dims[i] * dims[j + 1];
            return fail_all(MP_OK);
        }
        // register nodes bottom-up
        std::function<int64_t(int, int)> reg = [&](int i, int j) -> int64_t {
            if (i == j) return -1;
            const std::vector<int32_t> ty = subchain_types(Q, i, j);
            const std::string key = subchain_key(Q, i, j);
            const std::string id = CachePolicy::make_id(ty, key);
            auto it = ex.by_id.find(id);
            if (it != ex.by_id.end() && node(it->second).status) {
                ex.by_id.erase(it);
                it = ex.by_id.end();
            }
            if (it != ex.by_id.end()) {
                PNode &x = node(it->second);
                x.consumers++;
                if (x.from_cache) F.r.cache_hits++;
                return it->second;
            }
            PNode nd;
            nd.id = id;
            nd.types = ty;
            nd.key = key;
            nd.flight = fid;
            nd.qs = st[q];
            nd.i = i;
            nd.j = j;
            nd.consumers = 1;
            nd.rho_est = D[(size_t)i * p + j];
            if (cache) {
                CacheItem *ci = cache->find(id);
                if (ci) {
                    nd.res = std::static_pointer_cast<DevMat>(ci->payload);
                    nd.from_cache = true;
                    nd.done = true;
                    cstats.requests++;
                    cstats.hits++;
                    F.r.cache_hits++;
                    cache->request(ty, key, (double)otree.frequency(ty.data(), ty.size(), &key), ci->c, ci->s,
                                   nullptr, nullptr);
                    const int64_t nid = ex.next_node++;
                    ex.nodes.emplace(nid, std::move(nd));
                    ex.by_id.emplace(id, nid);
                    return nid;
                }
            }
            int k = split[(size_t)i * p + j];
            if (k < 0 && host_known.count(id)) {
                const HostEntry &he = htier.items[id];
                const double c_ms = he.c_ms, c_ops = he.c_ops;
                MatPtr hm = htier_load(id);
                if (hm) {
                    nd.res = hm;
                    nd.from_cache = nd.from_host = true;
                    nd.done = true;
                    nd.subtree_ms = c_ms;
                    nd.c_ops = c_ops;
                    F.r.cache_hits++;
                    const int64_t nid = ex.next_node++;
                    ex.nodes.emplace(nid, std::move(nd));
                    ex.by_id.emplace(id, nid);
                    return nid;
                }
            }
            if (k < 0) k = split_pure[(size_t)i * p + j];  // known (evicted) but not at hand: compute it
            nd.k = k;
            nd.left = reg(i, k);
            nd.right = reg(k + 1, j);
            // planned bytes of the result: row pointers and the estimated entries
            F.est_bytes += (dims[i] + 1) * 8.0 + 12.0 * D[(size_t)i * p + j] * dims[i] * dims[j + 1];
            const int64_t nid = ex.next_node++;
            ex.nodes.emplace(nid, std::move(nd));
            ex.by_id.emplace(id, nid);
            return nid;
        };
        F.root = reg(0, p - 1);
        {
            PNode &rt = node(F.root);
            rt.consumers--;  // no parent reads a query's result: its flight keeps it
            rt.keepers++;
            F.keeps.push_back(F.root);
        }
        ex.est_bytes += F.est_bytes;
    }
    plan_range.reset();
    // cache candidates: the longest computed sub-metapath of each query seen at least twice
    // (MP_INSERT_OTREE), none (MP_INSERT_FINAL), or every node the query computes
    // (MP_INSERT_ALL); each is kept until its query finishes and offers it
    for (size_t q = 0; q < nq; q++) {
        Flight &F = *fl[q];
        if (!cache || F.root < 0 || node(F.root).filter) continue;
        if (cfg.insertion == MP_INSERT_OTREE) {
            int64_t best = -1;
            // the query's own products: a node already done (computed for a query admitted
            // earlier) ends the walk, as its operands may be gone
            std::function<void(int64_t)> walk = [&](int64_t x) {
                if (x < 0) return;
                const PNode &nd = node(x);
                if (x != F.root && !nd.from_cache && !nd.filter) {
                    const uint64_t f = otree.frequency(nd.types.data(), nd.types.size(), &nd.key);
                    if (f >= 2 && (best < 0 || nd.types.size() > node(best).types.size())) best = x;
                }
                if (nd.done) return;
                walk(nd.left);
                walk(nd.right);
            };
            walk(F.root);
            F.candidate = best;
            if (best >= 0) {
                node(best).keepers++;
                F.keeps.push_back(best);
            }
        } else if (cfg.insertion == MP_INSERT_ALL) {
            for (auto &kv : ex.nodes)
                if (kv.second.flight == ids[q] && !kv.second.from_cache && kv.first != F.root) {
                    kv.second.keepers++;
                    F.keeps.push_back(kv.first);
                }
            std::sort(F.keeps.begin() + 1, F.keeps.end());
        }
    }
    return MP_OK;
}

// A wave failed as a whole (a CUDA error, device memory exhausted): every product not run
// yet carries its error, and nothing is left waiting for them.
void mp_ctx::abort_nodes(int rc) {
    for (auto &kv : ex.nodes)
        if (!kv.second.done) {
            kv.second.status = rc;
            kv.second.done = true;
        }
    std::vector<int64_t> ids;
    for (auto &kv : ex.nodes) {
        kv.second.consumers = 0;  // every parent is done now
        ids.push_back(kv.first);
    }
    for (int64_t id : ids) release_node(id);
}

void mp_ctx::release_node(int64_t id) {
    auto it = ex.nodes.find(id);
    if (it == ex.nodes.end()) return;
    PNode &nd = it->second;
    if (!nd.done || nd.consumers > 0 || nd.keepers > 0) return;
    auto b = ex.by_id.find(nd.id);
    if (b != ex.by_id.end() && b->second == id) ex.by_id.erase(b);
    ex.nodes.erase(it);
}

int mp_ctx::run_wave() {
    std::vector<int64_t> ready;
    for (auto &kv : ex.nodes) {
        const PNode &nd = kv.second;
        if (nd.done) continue;
        if (nd.left >= 0 && !node(nd.left).done) continue;
        if (nd.right >= 0 && !node(nd.right).done) continue;
        ready.push_back(kv.first);
    }
    if (ready.empty()) return MP_OK;
    std::sort(ready.begin(), ready.end());  // registration order: waves are reproducible
    TraceRange wave_range("mp.wave");
    auto finish_node = [&](int64_t id) {
        PNode &nd = node(id);
        nd.done = true;
        auto fit = ex.flights.find(nd.flight);
        if (fit != ex.flights.end() && !nd.from_cache) {
            Result &r = fit->second.r;
            r.st.products += nd.st.products;
            r.st.nnz += nd.st.nnz;
            for (int b = 0; b < NBINS; b++) {
                r.st.sym_bins[b] += nd.st.sym_bins[b];
                r.st.num_bins[b] += nd.st.num_bins[b];
            }
            r.n_products += nd.filter ? 0 : 1;
            r.ms += nd.ms;
        }
        for (int64_t c : {nd.left, nd.right}) {
            if (c < 0) continue;
            node(c).consumers--;
            release_node(c);
        }
        release_node(id);  // a node whose query gave up on it meanwhile
    };
    CtxBudget bud(this);
    std::vector<int64_t> members;
    std::vector<WaveIn> win;
    std::vector<void *> scratch;  // column-masked copies of leaves, freed after the wave
    std::vector<size_t> ycand;    // wave inputs whose Y copy depends on the products they read
    auto release_scratch = [&] {
        for (void *p : scratch) alloc->free(p, stream);
        scratch.clear();
    };
    // A large pattern leaf enters its product with the mask on its columns applied, so the
    // row work and the walks never read an entry the mask drops: X (no row mask, so all its
    // rows are read) by the middle mask; Y by the column mask when X holds at least an eighth
    // as many entries as Y has rows, or otherwise when the products of X with Y, counted
    // exactly on the device (one count per such product and one synchronisation per wave),
    // read at least half of Y's entries. The middle or column mask then has nothing left to
    // drop.
    auto compact = [&](DCsr &A, const uint32_t *m) {
        DCsr B;
        int64_t *rp = nullptr;
        int32_t *ci = nullptr;
        if (compact_cols(A, m, *alloc, tun, stream, &B, &rp, &ci)) return false;
        scratch.push_back(rp);
        scratch.push_back(ci);
        A = B;
        return true;
    };
    for (int64_t id : ready) {
        PNode &nd = node(id);
        const Query &Q = nd.qs->q;
        const auto &M = nd.qs->masks;
        if (nd.filter) {
            auto t0 = std::chrono::steady_clock::now();
            Mat C;
            nd.status = filter(rels[Q.rels[0]].dev.view(), M[0], M[1], *alloc, tun, stream, &C);
            nd.ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
            nd.subtree_ms = nd.ms;
            if (!nd.status && reserve_bytes((int64_t)C.bytes())) nd.status = MP_ERR_BUDGET;
            if (!nd.status) nd.res = wrap(C, true);
            else free_mat(C);
            finish_node(id);
            continue;
        }
        const int ls = nd.left >= 0 ? node(nd.left).status : MP_OK;
        const int rs = nd.right >= 0 ? node(nd.right).status : MP_OK;
        if (ls || rs) {
            nd.status = ls ? ls : rs;
            finish_node(id);
            continue;
        }
        const int i = nd.i, j = nd.j, k = nd.k;
        WaveIn in;
        in.X = nd.left >= 0 ? node(nd.left).res->m.view() : rels[Q.rels[i]].dev.view();
        if (nd.left >= 0) in.xrows_hold = node(nd.left).res->m.arows_hold;
        in.Y = nd.right >= 0 ? node(nd.right).res->m.view() : rels[Q.rels[j]].dev.view();
        in.ymax = nd.right >= 0 ? node(nd.right).res->m.vmax : 1;
        // a base factor enters with the masks of its end positions; a node's result
        // already carries them (0/1 diagonals are idempotent)
        in.rm = nd.left < 0 ? M[i] : nullptr;
        in.km = (nd.left < 0 || nd.right < 0) ? M[k + 1] : nullptr;
        in.cm = nd.right < 0 ? M[j + 1] : nullptr;
        if (nd.left < 0 && (size_t)i < nd.qs->rows.size() && nd.qs->rows[i]) {
            // a base factor starting at a position constrained by a node-id set: its rows
            // outside the set are masked out, so the set is its row list
            in.X.arows = nd.qs->rows[i];
            in.X.narows = nd.qs->nrows[i];
            in.xrows_hold = nd.qs->rows_hold[i];
        }
        if (tun.compact) {
            if (nd.left < 0 && !in.rm && in.km && !in.X.val && in.X.nnz >= tun.compact_min && compact(in.X, in.km))
                in.km = nullptr;
            if (nd.right < 0 && in.cm && !in.Y.val && in.Y.nnz >= tun.compact_min) {
                if (in.X.nnz * 8 >= in.Y.nrows) {
                    if (compact(in.Y, in.cm)) in.cm = nullptr;
                } else {
                    ycand.push_back(win.size());
                }
            }
        }
        members.push_back(id);
        win.push_back(in);
    }
    if (!ycand.empty()) {
        // the products each candidate reads, in one device array and one copy back
        auto *cnt = (unsigned long long *)alloc->alloc(ycand.size() * 8, stream);
        std::vector<unsigned long long> h(ycand.size(), 0);
        bool ok = cnt && cudaMemsetAsync(cnt, 0, ycand.size() * 8, stream) == cudaSuccess;
        for (size_t c = 0; ok && c < ycand.size(); c++) {
            const WaveIn &in = win[ycand[c]];
            raw_products(in.X, in.rm, in.km, in.Y.rp, tun, stream, cnt + c);
        }
        Readback rb(&wcache, stream);
        ok = ok && rb.get(h.data(), cnt, ycand.size() * 8) && rb.sync();
        if (cnt) alloc->free(cnt, stream);
        if (!ok) cudaGetLastError();  // no copies: the masks apply entry by entry
        for (size_t c = 0; ok && c < ycand.size(); c++) {
            WaveIn &in = win[ycand[c]];
            if ((int64_t)h[c] * 2 >= in.Y.nnz && compact(in.Y, in.cm)) in.cm = nullptr;
        }
    }
    if (members.empty()) return MP_OK;
    std::vector<WaveOut> wout;
    auto t0 = std::chrono::steady_clock::now();
    const int wave_rc =
        spgemm_wave(win, *alloc, tun, stream, cfg.max_result_bytes, wout, &prof, false, &wcache, &bud);
    release_scratch();
    const double wave_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    double wave_prod = 0.0;
    for (auto &o : wout) wave_prod += (double)o.products;
    for (size_t t = 0; t < members.size(); t++) {
        PNode &nd = node(members[t]);
        if (wave_rc) {
            nd.status = wave_rc;
            finish_node(members[t]);
            continue;
        }
        WaveOut &o = wout[t];
        nd.status = o.status;
        nd.st.products = o.products;
        nd.st.nnz = (uint64_t)o.m.nnz;
        for (int b = 0; b < NBINS; b++) {
            nd.st.sym_bins[b] = o.sym_bins[b];
            nd.st.num_bins[b] = o.num_bins[b];
        }
        // the wave's time, shared in proportion to the products each member ran
        nd.ms = wave_prod > 0 ? wave_ms * (double)o.products / wave_prod : wave_ms / (double)members.size();
        const PNode *L = nd.left >= 0 ? &node(nd.left) : nullptr;
        const PNode *R = nd.right >= 0 ? &node(nd.right) : nullptr;
        nd.subtree_ms = nd.ms + (L && !L->from_cache ? L->subtree_ms : 0.0) + (R && !R->from_cache ? R->subtree_ms : 0.0);
        if (!o.status) {
            // Eq. 2 with the actual counts: alpha nnz(X) + beta N_op + gamma nnz(Z)
            const double nnz_x = (double)(L ? L->res->m.nnz : rels[nd.qs->q.rels[nd.i]].dev.nnz);
            nd.c_ops = cfg.alpha * nnz_x + cfg.beta * (double)o.products + cfg.gamma * (double)o.m.nnz;
            if (collect_fit) fit_samples.push_back({nnz_x, (double)o.products, (double)o.m.nnz, nd.ms});
            nd.res = wrap(o.m, true);  // its bytes were charged before its arrays were made
        }
        finish_node(members[t]);
    }
    return wave_rc;
}

void mp_ctx::finish_flights(std::vector<Flight> &done) {
    std::vector<int64_t> fin;
    for (auto &kv : ex.flights) {
        const Flight &F = kv.second;
        if (F.status || F.root < 0 || node(F.root).done) fin.push_back(kv.first);
    }
    if (fin.empty()) return;
    std::unique_ptr<TraceRange> offer_range(cache ? new TraceRange("mp.cache_offers") : nullptr);
    // Sec. 3.4.1: the query's result and its cache candidate are offered to the replacement
    // policy (Alg. 1)
    auto offer = [&](PNode &nd) {
        if ((nd.from_cache && !nd.from_host) || nd.filter || nd.status || !nd.res) return;
        const double f = (double)otree.frequency(nd.types.data(), nd.types.size(), &nd.key);
        std::vector<CacheItem> ev;
        cstats.requests++;
        auto out = cache->request(nd.types, nd.key, f, nd.subtree_ms, (double)nd.res->m.bytes(),
                                  std::static_pointer_cast<void>(nd.res), &ev);
        if (out == CachePolicy::INSERTED) cstats.inserts++;
        if (out == CachePolicy::REJECTED) cstats.rejected++;
        if (out == CachePolicy::HIT) cstats.hits++;
        cstats.evictions += ev.size();
        OTEntry *e = otree.entry(nd.types.data(), nd.types.size(), nd.key);
        if (e) {
            e->cached = out != CachePolicy::REJECTED;
            e->c_ms = nd.subtree_ms;
            e->c_ops = nd.c_ops;
            e->nnz = (double)nd.res->m.nnz;
        }
        for (auto &it : ev) {
            OTEntry *ee = otree.entry(it.types.data(), it.types.size(), it.key);
            if (ee) ee->cached = false;
            htier_store(it.id, std::static_pointer_cast<DevMat>(it.payload), it.types, it.key, it.c,
                        ee ? ee->c_ops : 0.0);
        }
    };
    for (int64_t fid : fin) {
        Flight &F = ex.flights[fid];
        Result &r = F.r;
        if (F.status) {
            r.status = F.status;
        } else {
            PNode &rt = node(F.root);
            r.status = rt.status;
            if (!rt.status) r.m = rt.res;
            // the result first, then the candidate (or, with MP_INSERT_ALL, every node
            // the query computed, in registration order)
            if (cache)
                for (int64_t x : F.keeps) offer(node(x));
        }
        for (int64_t x : F.keeps) {
            node(x).keepers--;
            release_node(x);
        }
        ex.est_bytes -= F.est_bytes;
        F.finished = true;
        done.push_back(std::move(F));
        ex.flights.erase(fid);
    }
    if (ex.flights.empty()) ex.est_bytes = 0.0;
}

void mp_ctx::publish(std::vector<Flight> &done) {
    const auto t1 = std::chrono::steady_clock::now();
    {
        std::lock_guard<std::mutex> g(mu);
        for (Flight &f : done) {
            auto it = results.find(f.ticket);
            if (it == results.end()) continue;  // released before it finished
            f.r.latency_ms = std::chrono::duration<double, std::milli>(t1 - f.t0).count();
            f.r.done = true;
            it->second = std::move(f.r);
        }
    }
    done_cv.notify_all();
}

int mp_ctx::run_batch(std::vector<Query> &qs, std::vector<Result> &rs) {
    TraceRange batch_range("mp.batch");
    const size_t nq = qs.size();
    cudaEventRecord(ev0, stream);
    std::vector<int64_t> ids;
    std::vector<uint64_t> tk(nq, 0);
    std::vector<std::chrono::steady_clock::time_point> t0s(nq, std::chrono::steady_clock::now());
    const int arc = admit(qs, tk, t0s, ids);
    std::unordered_map<int64_t, size_t> mine;
    for (size_t q = 0; q < nq; q++) mine.emplace(ids[q], q);
    if (explain.on) {
        for (size_t q = 0; q < nq; q++) {
            rs[q].status = ex.flights[ids[q]].status;
            ex.flights.erase(ids[q]);
        }
        cudaEventRecord(ev1, stream);
        cudaEventSynchronize(ev1);
        return arc;
    }
    // waves until every query of this batch has finished (flights of the serving loop that
    // finish meanwhile are published as usual)
    size_t left = nq;
    int first = MP_OK;
    for (int guard = 0; left > 0; guard++) {
        std::vector<Flight> done;
        finish_flights(done);
        std::vector<Flight> others;
        for (Flight &f : done) {
            auto m = mine.find(f.id);
            if (m == mine.end()) {
                others.push_back(std::move(f));
                continue;
            }
            rs[m->second] = std::move(f.r);
            left--;
        }
        if (!others.empty()) publish(others);
        if (left == 0) break;
        const int wrc = run_wave();
        if (wrc || guard > 100000) abort_nodes(wrc ? wrc : MP_ERR_INTERNAL);
    }
    for (size_t q = 0; q < nq; q++)
        if (rs[q].status && first == MP_OK) first = rs[q].status;
    cudaEventRecord(ev1, stream);
    cudaError_t e = cudaEventSynchronize(ev1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev0, ev1);
    for (size_t q = 0; q < nq; q++) rs[q].ms = ms;
    if (e != cudaSuccess && first == MP_OK) first = MP_ERR_CUDA;
    return first;
}
