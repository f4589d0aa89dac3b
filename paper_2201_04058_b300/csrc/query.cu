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

MatPtr mp_ctx::wrap(const Mat &m) {
    auto p = std::make_shared<DevMat>();
    p->m = m;
    p->al = alloc.get();
    p->s = stream;
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
    HostEntry &e = it->second;
    Mat m = e.shape;
    const size_t brp = (size_t)(m.nrows + 1) * 8, bci = (size_t)m.nnz * 4, bval = (size_t)m.nnz * 8;
    m.rp = (int64_t *)alloc->alloc(brp, stream);
    m.ci = (int32_t *)alloc->alloc(std::max<size_t>(bci, 4), stream);
    m.val = (uint64_t *)alloc->alloc(std::max<size_t>(bval, 8), stream);
    if (!m.rp || !m.ci || !m.val) {
        free_mat(m);
        return nullptr;
    }
    // ordered on the stream before every kernel that reads the result; the arena block
    // stays put until the batch ends (stores and drops happen after the batch's waves)
    const char *b = htier.arena + e.off;
    cudaMemcpyAsync(m.rp, b, brp, cudaMemcpyHostToDevice, stream);
    if (m.nnz) {
        cudaMemcpyAsync(m.ci, b + brp, bci, cudaMemcpyHostToDevice, stream);
        cudaMemcpyAsync(m.val, b + brp + bci, bval, cudaMemcpyHostToDevice, stream);
    }
    e.seq = ++htier.seq;
    htier.loads++;
    return wrap(m);
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

namespace {

// One sub-chain of some query's plan: factors i..j of query q (positions i..j+1).
struct PNode {
    std::string id;
    std::vector<int32_t> types;
    std::string key;
    int q = -1, i = 0, j = 0, k = 0;  // registering query, its factor range and split
    int left = -1, right = -1;  // child node indices; -1 = the base factor itself
    int level = 0;
    MatPtr res;
    bool from_cache = false;
    bool from_host = false;     // copied back from the host tier (offered to the cache again)
    bool filter = false;        // length-2 query: diag(M_1) A diag(M_2)
    int consumers = 0;
    bool keep = false;          // a query's result or a cache candidate
    int status = MP_OK;
    double ms = 0.0;            // device time of this node's own product
    double subtree_ms = 0.0;    // of every product this node's computation needed
    double c_ops = 0.0;         // Eq. 2 with the product's actual counts
    double rho_est = 0.0;       // planner density estimate (for batch-mates)
    mp::Stats st;
};

std::string subchain_key(const Query &q, int i, int j) {
    return window_key(q.pos_keys, (size_t)i, (size_t)(j - i + 2));
}

std::vector<int32_t> subchain_types(const Query &q, int i, int j) {
    return std::vector<int32_t>(q.types.begin() + i, q.types.begin() + j + 2);
}

}  // namespace

int mp_ctx::run_batch(std::vector<Query> &qs, std::vector<Result> &rs) {
    TraceRange batch_range("mp.batch");
    const size_t nq = qs.size();
    cudaEventRecord(ev0, stream);
    std::vector<std::vector<uint32_t *>> masks(nq);
    std::vector<int> qstatus(nq, MP_OK);
    for (size_t q = 0; q < nq; q++) qstatus[q] = build_masks(qs[q], masks[q]);
    // a batch-wide failure before the products run: every query reports it, nothing leaks
    auto fail_all = [&](int rc) {
        for (size_t q = 0; q < nq; q++) rs[q].status = qstatus[q] ? qstatus[q] : rc;
        for (auto &m : masks) free_masks(m);
        cudaEventRecord(ev1, stream);
        cudaEventSynchronize(ev1);
        return rc;
    };

    // exact nnz of every masked base factor, for the planner: one device array, one sync;
    // counts already seen (same relation, same constraints at both ends) come from a memo
    std::vector<std::vector<double>> leaf(nq);
    {
        size_t total = 0;
        for (auto &q : qs) total += q.rels.size();
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
            const int p = (int)qs[q].rels.size();
            leaf[q].assign(p, -1.0);
            for (int t = 0; t < p; t++) {
                const Mat &A = rels[qs[q].rels[t]].dev;
                if (qstatus[q] || !(masks[q][t] || masks[q][t + 1])) continue;
                std::string &key = keys[off + t];
                key = std::to_string(qs[q].rels[t]) + "|" + qs[q].pos_keys[t] + "|" + qs[q].pos_keys[t + 1];
                auto m = leaf_memo.find(key);
                if (m != leaf_memo.end()) {
                    leaf[q][t] = m->second;
                    continue;
                }
                if (first.count(key)) continue;
                first.emplace(key, off + t);
                uint32_t *lr = (uint32_t *)alloc->alloc((size_t)(A.nrows + 1) * 4, stream);
                if (!lr) {
                    free_tmp();
                    return fail_all(MP_ERR_NOMEM);
                }
                cudaMemsetAsync(lr + A.nrows, 0, 4, stream);
                masked_nnz(A.view(), masks[q][t], masks[q][t + 1], d + off + t, lr, lr + A.nrows, stream);
                tmp.push_back(lr);
                any = true;
            }
            off += p;
        }
        std::vector<unsigned long long> h(std::max<size_t>(total, 1), 0);
        if (any) {
            cudaMemcpyAsync(h.data(), d, std::max<size_t>(total, 1) * 8, cudaMemcpyDeviceToHost, stream);
            if (cudaStreamSynchronize(stream) != cudaSuccess) {
                free_tmp();
                return fail_all(MP_ERR_CUDA);
            }
        }
        free_tmp();
        if (leaf_memo.size() > 65536) leaf_memo.clear();
        for (auto &kv : first) leaf_memo[kv.first] = (double)h[kv.second];
        off = 0;
        for (size_t q = 0; q < nq; q++) {
            for (size_t t = 0; t < qs[q].rels.size(); t++) {
                if (leaf[q][t] >= 0) continue;
                const std::string &key = keys[off + t];
                leaf[q][t] = key.empty() ? (double)rels[qs[q].rels[t]].dev.nnz : leaf_memo[key];
            }
            off += qs[q].rels.size();
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
                for (int t = 0; t + 1 < (int)qs[q].rels.size(); t++) pairs.push_back({q, t});
        sampled.assign(nq, std::vector<double>());
        for (size_t q = 0; q < nq; q++) {
            const size_t p = qs[q].rels.size();
            sampled[q].assign(p * p, NAN);
        }
        if (!pairs.empty()) {
            const size_t np = pairs.size();
            unsigned long long *d = (unsigned long long *)alloc->alloc(np * 16, stream);
            if (!d) return fail_all(MP_ERR_NOMEM);
            cudaMemsetAsync(d, 0, np * 16, stream);  // [active rows, sampled rows] per pair
            for (size_t k = 0; k < np; k++) {
                const Query &Q = qs[pairs[k].q];
                active_rows(rels[Q.rels[pairs[k].t]].dev.view(), masks[pairs[k].q][pairs[k].t], d + 2 * k, stream);
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
                const Query &Q = qs[pairs[k].q];
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
                sample_rows(A.view(), masks[pairs[k].q][t], seed, thr, bms[k], d + 2 * k + 1, stream);
                win[k].X = A.view();
                win[k].Y = rels[Q.rels[t + 1]].dev.view();
                win[k].rm = bms[k];
                win[k].km = masks[pairs[k].q][t + 1];
                win[k].cm = masks[pairs[k].q][t + 2];
            }
            std::vector<WaveOut> wout;
            int rc = spgemm_wave(win, *alloc, tun, stream, 0, wout, nullptr, true, &wcache);
            cudaMemcpyAsync(h.data(), d, np * 16, cudaMemcpyDeviceToHost, stream);
            if (cudaStreamSynchronize(stream) != cudaSuccess) rc = MP_ERR_CUDA;
            for (auto *b : bms) alloc->free(b, stream);
            alloc->free(d, stream);
            if (rc) return fail_all(rc);
            for (size_t k = 0; k < np; k++) {
                const Query &Q = qs[pairs[k].q];
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
            const Query &Q = qs[q];
            const int p = (int)Q.rels.size();
            mleaf[q].assign(p, -1);
            mpair[q].assign(p, -1);
            for (int t = 0; t < p; t++) {
                const std::string key =
                    std::to_string(Q.rels[t]) + "|" + Q.pos_keys[t] + "|" + Q.pos_keys[t + 1];
                auto it = lidx.find(key);
                if (it == lidx.end()) {
                    MncLeafIn in{rels[Q.rels[t]].dev.view(), rels[Q.rels[t] ^ 1].dev.view(), masks[q][t],
                                 masks[q][t + 1]};
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
            if (!qstatus[q]) otree.insert(qs[q].types, qs[q].pos_keys);

    // plans and the product DAG
    std::unique_ptr<TraceRange> plan_range(new TraceRange("mp.plan"));
    std::vector<PNode> nodes;
    std::unordered_map<std::string, int> by_id;
    std::unordered_set<std::string> host_known;  // sub-chains planned as copies from the host tier
    std::vector<int> root(nq, -1);
    for (size_t q = 0; q < nq; q++) {
        if (qstatus[q]) continue;
        const Query &Q = qs[q];
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
            nd.id = "filter#" + std::to_string(q);
            nd.q = (int)q;
            nd.filter = true;
            nd.level = 1;
            nd.keep = true;
            root[q] = (int)nodes.size();
            nodes.push_back(std::move(nd));
            continue;
        }
        // sub-chains already known: in the cache, computed earlier in this batch, or
        // evicted with a recorded cost
        std::vector<double> kc((size_t)p * p, NAN), kr((size_t)p * p, NAN);
        for (int i = 0; i < p; i++)
            for (int j = i + 1; j < p; j++) {
                const std::vector<int32_t> ty = subchain_types(Q, i, j);
                const std::string key = subchain_key(Q, i, j);
                const std::string id = CachePolicy::make_id(ty, key);
                const double cells = dims[i] * dims[j + 1];
                auto it = by_id.find(id);
                if (it != by_id.end()) {
                    kc[(size_t)i * p + j] = 0.0;
                    kr[(size_t)i * p + j] = nodes[it->second].rho_est;
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
        std::function<int(int, int)> reg = [&](int i, int j) -> int {
            if (i == j) return -1;
            const std::vector<int32_t> ty = subchain_types(Q, i, j);
            const std::string key = subchain_key(Q, i, j);
            const std::string id = CachePolicy::make_id(ty, key);
            auto it = by_id.find(id);
            if (it != by_id.end()) {
                nodes[it->second].consumers++;
                return it->second;
            }
            PNode nd;
            nd.id = id;
            nd.types = ty;
            nd.key = key;
            nd.q = (int)q;
            nd.i = i;
            nd.j = j;
            nd.consumers = 1;
            nd.rho_est = D[(size_t)i * p + j];
            if (cache) {
                CacheItem *ci = cache->find(id);
                if (ci) {
                    nd.res = std::static_pointer_cast<DevMat>(ci->payload);
                    nd.from_cache = true;
                    nd.level = 0;
                    cstats.requests++;
                    cstats.hits++;
                    cache->request(ty, key, (double)otree.frequency(ty.data(), ty.size(), &key), ci->c, ci->s,
                                   nullptr, nullptr);
                    const int idx = (int)nodes.size();
                    nodes.push_back(std::move(nd));
                    by_id.emplace(id, idx);
                    return idx;
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
                    nd.level = 0;
                    nd.subtree_ms = c_ms;
                    nd.c_ops = c_ops;
                    const int idx = (int)nodes.size();
                    nodes.push_back(std::move(nd));
                    by_id.emplace(id, idx);
                    return idx;
                }
            }
            if (k < 0) k = split_pure[(size_t)i * p + j];  // known (evicted) but not at hand: compute it
            nd.k = k;
            const int l = reg(i, k);
            const int r = reg(k + 1, j);
            nd.left = l;
            nd.right = r;
            nd.level = 1 + std::max(l >= 0 ? nodes[l].level : 0, r >= 0 ? nodes[r].level : 0);
            const int idx = (int)nodes.size();
            nodes.push_back(std::move(nd));
            by_id.emplace(id, idx);
            return idx;
        };
        root[q] = reg(0, p - 1);
        nodes[root[q]].keep = true;
    }

    plan_range.reset();
    // cache candidates: the longest computed sub-metapath of each query seen at least twice
    // (MP_INSERT_OTREE), none (MP_INSERT_FINAL), or every computed node (MP_INSERT_ALL)
    std::vector<int> candidate(nq, -1);
    if (cache && cfg.insertion == MP_INSERT_ALL)
        for (auto &nd : nodes)
            if (!nd.from_cache && !nd.filter) nd.keep = true;
    if (cache && cfg.insertion == MP_INSERT_OTREE) {
        for (size_t q = 0; q < nq; q++) {
            if (root[q] < 0) continue;
            int best = -1;
            std::function<void(int)> walk = [&](int x) {
                if (x < 0) return;
                const PNode &nd = nodes[x];
                if (x != root[q] && !nd.from_cache && !nd.filter) {
                    const uint64_t f = otree.frequency(nd.types.data(), nd.types.size(), &nd.key);
                    if (f >= 2 && (best < 0 || nd.types.size() > nodes[best].types.size())) best = x;
                }
                walk(nd.left);
                walk(nd.right);
            };
            walk(root[q]);
            candidate[q] = best;
            if (best >= 0) nodes[best].keep = true;
        }
    }

    // run the DAG level by level; every product of a level runs in one wave
    int max_level = 0;
    for (auto &nd : nodes) max_level = std::max(max_level, nd.level);
    auto release_operands = [&](PNode &nd) {
        for (int c : {nd.left, nd.right}) {
            if (c < 0) continue;
            if (--nodes[c].consumers <= 0 && !nodes[c].keep) nodes[c].res.reset();
        }
    };
    int wave_rc = MP_OK;
    for (int lvl = 1; lvl <= max_level && wave_rc == MP_OK; lvl++) {
        char wave_name[32];
        snprintf(wave_name, sizeof(wave_name), "mp.wave level %d", lvl);
        TraceRange wave_range(wave_name);
        std::vector<int> members;
        std::vector<WaveIn> win;
        for (size_t x = 0; x < nodes.size(); x++) {
            PNode &nd = nodes[x];
            if (nd.level != lvl || nd.res) continue;
            const Query &Q = qs[nd.q];
            const auto &M = masks[nd.q];
            if (nd.filter) {
                auto t0 = std::chrono::steady_clock::now();
                Mat C;
                nd.status = filter(rels[Q.rels[0]].dev.view(), M[0], M[1], *alloc, tun, stream, &C);
                nd.ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
                nd.subtree_ms = nd.ms;
                if (!nd.status) nd.res = wrap(C);
                else free_mat(C);
                continue;
            }
            if (nd.left >= 0 && nodes[nd.left].status) {
                nd.status = nodes[nd.left].status;
                release_operands(nd);
                continue;
            }
            if (nd.right >= 0 && nodes[nd.right].status) {
                nd.status = nodes[nd.right].status;
                release_operands(nd);
                continue;
            }
            const int i = nd.i, j = nd.j, k = nd.k;
            WaveIn in;
            in.X = nd.left >= 0 ? nodes[nd.left].res->m.view() : rels[Q.rels[i]].dev.view();
            in.Y = nd.right >= 0 ? nodes[nd.right].res->m.view() : rels[Q.rels[j]].dev.view();
            in.ymax = nd.right >= 0 ? nodes[nd.right].res->m.vmax : 1;
            // a base factor enters with the masks of its end positions; a node's result
            // already carries them (0/1 diagonals are idempotent)
            in.rm = nd.left < 0 ? M[i] : nullptr;
            in.km = (nd.left < 0 || nd.right < 0) ? M[k + 1] : nullptr;
            in.cm = nd.right < 0 ? M[j + 1] : nullptr;
            members.push_back((int)x);
            win.push_back(in);
        }
        if (members.empty()) continue;
        std::vector<WaveOut> wout;
        auto t0 = std::chrono::steady_clock::now();
        wave_rc = spgemm_wave(win, *alloc, tun, stream, cfg.max_result_bytes, wout, &prof, false, &wcache);
        const double wave_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        double wave_prod = 0.0;
        for (auto &o : wout) wave_prod += (double)o.products;
        for (size_t t = 0; t < members.size(); t++) {
            PNode &nd = nodes[members[t]];
            if (wave_rc) {
                nd.status = wave_rc;
                release_operands(nd);
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
            nd.subtree_ms = nd.ms + (nd.left >= 0 && !nodes[nd.left].from_cache ? nodes[nd.left].subtree_ms : 0.0) +
                            (nd.right >= 0 && !nodes[nd.right].from_cache ? nodes[nd.right].subtree_ms : 0.0);
            if (!o.status) {
                // Eq. 2 with the actual counts: alpha nnz(X) + beta N_op + gamma nnz(Z)
                const double nnz_x = (double)(nd.left >= 0 ? nodes[nd.left].res->m.nnz : rels[qs[nd.q].rels[nd.i]].dev.nnz);
                nd.c_ops = cfg.alpha * nnz_x + cfg.beta * (double)o.products + cfg.gamma * (double)o.m.nnz;
                if (collect_fit) fit_samples.push_back({nnz_x, (double)o.products, (double)o.m.nnz, nd.ms});
                nd.res = wrap(o.m);
            }
            release_operands(nd);
        }
    }

    // nodes a failed wave never reached carry its error
    for (auto &nd : nodes)
        if (!nd.res && !nd.status) nd.status = wave_rc ? wave_rc : MP_ERR_INTERNAL;

    // results, statistics, cache insertion (Sec. 3.4.1) under the replacement policy
    int first = MP_OK;
    for (size_t q = 0; q < nq; q++) {
        Result &r = rs[q];
        if (qstatus[q]) {
            r.status = qstatus[q];
        } else {
            PNode &rt = nodes[root[q]];
            r.status = rt.status;
            if (!rt.status) r.m = rt.res;
            std::function<void(int)> acc = [&](int x) {
                if (x < 0) return;
                const PNode &nd = nodes[x];
                if (nd.q == (int)q && !nd.from_cache) {
                    r.st.products += nd.st.products;
                    r.st.nnz += nd.st.nnz;
                    for (int b = 0; b < NBINS; b++) {
                        r.st.sym_bins[b] += nd.st.sym_bins[b];
                        r.st.num_bins[b] += nd.st.num_bins[b];
                    }
                    r.n_products += nd.filter ? 0 : 1;
                }
                if (nd.from_cache) r.cache_hits++;
                acc(nd.left);
                acc(nd.right);
            };
            acc(root[q]);
        }
        if (r.status && first == MP_OK) first = r.status;
    }
    if (cache) {
        TraceRange offer_range("mp.cache_offers");
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
        for (size_t q = 0; q < nq; q++) {
            if (root[q] < 0) continue;
            offer(nodes[root[q]]);
            if (candidate[q] >= 0) offer(nodes[candidate[q]]);
        }
        if (cfg.insertion == MP_INSERT_ALL)
            for (auto &nd : nodes)
                if (nd.keep) offer(nd);
    }
    for (auto &m : masks) free_masks(m);
    nodes.clear();
    cudaEventRecord(ev1, stream);
    cudaError_t e = cudaEventSynchronize(ev1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev0, ev1);
    for (size_t q = 0; q < nq; q++) rs[q].ms = ms;
    if (e != cudaSuccess && first == MP_OK) first = MP_ERR_CUDA;
    return first;
}
