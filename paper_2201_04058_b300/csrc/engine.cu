// Host runtime of the metapath engine and the C ABI of include/mp.h.
//
// A context owns one CUDA stream, a stream-ordered device pool, the device HIN store
// (CSR of every relation in both directions, Sec. 2 Def. 1; int32 properties) and the
// results of submitted queries. A query (Def. 2-3, Problem 1) is evaluated as
//   1. masks: one bitmap per constrained position, the diagonal M_i of Def. 3;
//   2. plan:  Eq. 1 DP over the masked factors' sizes and nnz (planner.cpp);
//   3. run:   the plan tree in post-order, one sparse product per internal node
//             (spgemm.cu), masks applied where a base relation enters a product.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <numeric>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/mp.h"
#include "engine.h"
#include "internal.h"

using namespace mp;
using Query = mp_ctx::Query;
using Result = mp_ctx::Result;

// ------------------------------------------------------------------ allocator

namespace mp {

struct PoolAlloc final : Alloc {
    void *alloc(size_t bytes, cudaStream_t s) override {
        void *p = nullptr;
        if (fail_after == 0) return nullptr;
        if (fail_after != UINT64_MAX) fail_after--;
        if (bytes == 0) bytes = 16;
        if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return p;
    }
    void free(void *p, cudaStream_t s) override {
        if (p) cudaFreeAsync(p, s);
    }
};

// The caller's allocator (mp_config.alloc / .free), e.g. PyTorch's caching allocator.
struct HookAlloc final : Alloc {
    void *(*fa)(size_t, void *, void *);
    void (*ff)(void *, void *, void *);
    void *user;
    HookAlloc(void *(*a)(size_t, void *, void *), void (*f)(void *, void *, void *), void *u)
        : fa(a), ff(f), user(u) {}
    void *alloc(size_t bytes, cudaStream_t s) override {
        if (fail_after == 0) return nullptr;
        if (fail_after != UINT64_MAX) fail_after--;
        if (bytes == 0) bytes = 16;
        return fa(bytes, (void *)s, user);
    }
    void free(void *p, cudaStream_t s) override {
        if (p) ff(p, (void *)s, user);
    }
};

}  // namespace mp

// ------------------------------------------------------------------ context

static int check_cuda(cudaError_t e, const char *what) {
    if (e != cudaSuccess) {
        fprintf(stderr, "mp: %s: %s\n", what, cudaGetErrorString(e));
        return MP_ERR_CUDA;
    }
    return MP_OK;
}

extern "C" void mp_config_default(mp_config *c) {
    if (!c) return;
    memset(c, 0, sizeof(*c));
    c->device = 0;
    c->hbm_budget_bytes = 8ull << 30;
    c->max_slots = 64;
    c->policy = MP_POLICY_ATRAPOS;
    c->planner = MP_PLAN_DP;
    c->cuda_stream = nullptr;
    c->alpha = 1.0;
    c->beta = 1.0;
    c->gamma = 1.0;
    c->force_bin_class = MP_BIN_AUTO;
    c->max_result_bytes = 0;
    c->scratch_bytes = 0;
    c->sample_rows = 1024;
    c->seed = 1;
    c->insertion = MP_INSERT_OTREE;
    c->tune_file = nullptr;
    c->cache_bytes = 0;
    c->otree_construction = MP_OTREE_ONLINE;
    c->alloc = nullptr;
    c->free = nullptr;
    c->alloc_user = nullptr;
}

extern "C" int mp_create(const mp_config *cfg, mp_ctx **out) {
    if (!out) return MP_ERR_ARG;
    *out = nullptr;
    mp_config c;
    if (cfg) c = *cfg; else mp_config_default(&c);
    if (c.policy < 0 || c.policy > MP_POLICY_NONE || c.planner < 0 || c.planner > MP_PLAN_DP_MNC ||
        c.force_bin_class < MP_BIN_AUTO || c.force_bin_class > MP_BIN_GLOBAL || c.insertion < MP_INSERT_OTREE ||
        c.insertion > MP_INSERT_ALL || (c.otree_construction != MP_OTREE_NAIVE && c.otree_construction != MP_OTREE_ONLINE) ||
        (!c.alloc) != (!c.free))
        return MP_ERR_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || c.device < 0 || c.device >= ndev) {
        cudaGetLastError();
        return ndev == 0 ? MP_ERR_CUDA : MP_ERR_ARG;
    }
    if (check_cuda(cudaSetDevice(c.device), "cudaSetDevice")) return MP_ERR_CUDA;
    std::unique_ptr<mp_ctx> ctx(new mp_ctx());
    ctx->cfg = c;
    if (c.cuda_stream) {
        ctx->stream = (cudaStream_t)c.cuda_stream;
        ctx->own_stream = false;
    } else {
        if (check_cuda(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking), "stream")) return MP_ERR_CUDA;
        ctx->own_stream = true;
    }
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, c.device) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c.device);
    ctx->tun.sm_count = sms;
    ctx->tun.force_class = c.force_bin_class;
    if (c.scratch_bytes) ctx->tun.scratch_cap = c.scratch_bytes;
    // optional overrides of the kernel tuning, "key=value,..." (for measuring variants)
    if (const char *e = getenv("MP_TUNING")) {
        std::string t(e);
        size_t a = 0;
        while (a < t.size()) {
            size_t b = t.find(',', a);
            if (b == std::string::npos) b = t.size();
            const std::string kv = t.substr(a, b - a);
            const size_t eq = kv.find('=');
            if (eq != std::string::npos) {
                const std::string k = kv.substr(0, eq);
                const long long v = atoll(kv.c_str() + eq + 1);
                if (k == "combine") ctx->tun.combine = (int)v;
                else if (k == "short_walk") ctx->tun.short_walk = (int)v;
                else if (k == "warp_prod") ctx->tun.warp_prod = (uint64_t)v;
                else if (k == "heavy") ctx->tun.heavy = (uint64_t)v;
                else if (k == "dense_min_u") ctx->tun.dense_min_u = (int)v;
                else if (k == "fail_alloc_after_finalize") ctx->fail_alloc_after = (uint64_t)v;
                else if (k == "glob_dense") ctx->tun.glob_dense = strtod(kv.c_str() + eq + 1, nullptr);
                else if (k == "dense_scratch") ctx->tun.dense_scratch_cap = (uint64_t)v;
                else if (k == "glob_occ") ctx->tun.glob_occ = (int)v;
                else if (k == "seg_walk") ctx->tun.seg_walk = (int)v;
                else if (k == "graphs") ctx->tun.graphs = (int)v;
                else if (k == "lbs") ctx->tun.lbs = (int)v;
                else if (k == "lbs_occ") ctx->tun.lbs_occ = (int)v;
                else if (k == "dsm_cols") ctx->tun.dsm_cols = (int)v;
                else if (k == "lane_rows") ctx->tun.lane_rows = (int)v;
                else if (k == "ew_max") ctx->tun.ew_max = (int)v;
                else if (k == "row_lens") ctx->tun.row_lens = (int)v;
                else if (k == "compact") ctx->tun.compact = (int)v;
                else if (k == "row_lists") ctx->tun.row_lists = (int)v;
                else if (k == "ech") ctx->tun.ech = (int64_t)v;
                else if (k == "prof") {
                    ctx->prof.on = v > 0;
                    ctx->prof.level = (int)v;
                }
                else if (k == "compact_min") ctx->tun.compact_min = (int64_t)v;
                else if (k == "pool") ctx->tun.pool = (int)v;

            }
            a = b + 1;
        }
    }
    if (check_cuda(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking), "stream")) return MP_ERR_CUDA;
    if (c.alloc) ctx->alloc.reset(new HookAlloc(c.alloc, c.free, c.alloc_user));
    else ctx->alloc.reset(new PoolAlloc());
    ctx->otree = OverlapTree(c.otree_construction == MP_OTREE_ONLINE ? OverlapTree::ONLINE : OverlapTree::NAIVE);
    if (c.policy != MP_POLICY_NONE) {
        // the cache's capacity (Sec. 3.4 cache size) within the HBM budget
        uint64_t cap = c.cache_bytes ? c.cache_bytes : c.hbm_budget_bytes;
        if (c.hbm_budget_bytes && cap > c.hbm_budget_bytes) cap = c.hbm_budget_bytes;
        if (!cap) cap = UINT64_MAX / 2;
        ctx->cache.reset(new CachePolicy((double)cap, c.policy));
    }
    if (c.tune_file) {
        if (FILE *f = fopen(c.tune_file, "r")) {
            char buf[4096];
            const size_t n = fread(buf, 1, sizeof(buf) - 1, f);
            fclose(f);
            buf[n] = 0;
            auto num = [&](const char *key, double *v) {
                const char *p = strstr(buf, key);
                if (p && (p = strchr(p, ':'))) *v = strtod(p + 1, nullptr);
            };
            double dmu = ctx->tun.dense_min_u, hv = (double)ctx->tun.heavy;
            double cb = ctx->tun.combine, sw = ctx->tun.short_walk, gw = ctx->tun.seg_walk, oc = ctx->tun.glob_occ;
            double lb = ctx->tun.lbs, lo = ctx->tun.lbs_occ;
            num("\"lbs\"", &lb);
            num("\"lbs_occ\"", &lo);
            ctx->tun.lbs = (int)lb;
            ctx->tun.lbs_occ = (int)lo;
            num("\"dense_min_u\"", &dmu);
            num("\"heavy\"", &hv);
            num("\"combine\"", &cb);
            num("\"short_walk\"", &sw);
            num("\"seg_walk\"", &gw);
            num("\"glob_occ\"", &oc);
            ctx->tun.combine = (int)cb;
            ctx->tun.short_walk = (int)sw;
            ctx->tun.seg_walk = (int)gw;
            ctx->tun.glob_occ = (int)oc;
            num("\"alpha\"", &ctx->cfg.alpha);
            num("\"beta\"", &ctx->cfg.beta);
            num("\"gamma\"", &ctx->cfg.gamma);
            ctx->tun.dense_min_u = (int)dmu;
            ctx->tun.heavy = (uint64_t)hv;
        } else {
            return MP_ERR_NOTFOUND;
        }
        ctx->cfg.tune_file = nullptr;  // the caller's string is not kept
    }
    cudaEventCreate(&ctx->ev0);
    cudaEventCreate(&ctx->ev1);
    if (!ctx->prof.init()) return MP_ERR_CUDA;
    // the host tier's pinned arena is made here, not inside a query
    if (ctx->cache && c.host_tier_bytes && !ctx->htier_init()) return MP_ERR_NOMEM;
    *out = ctx.release();
    return MP_OK;
}

extern "C" void mp_destroy(mp_ctx *ctx) {
    if (!ctx) return;
    mp_serve_stop(ctx);
    cudaSetDevice(ctx->cfg.device);
    {
        std::lock_guard<std::mutex> ge(ctx->exec_mu);
        std::lock_guard<std::mutex> g(ctx->mu);
        ctx->cache_clear();
        ctx->mnc_memo.clear();
        ctx->wcache.clear(*ctx->alloc, ctx->stream);
        for (auto &kv : ctx->results)
            if (kv.second.copy_ev) {
                cudaEventSynchronize(kv.second.copy_ev);
                cudaEventDestroy(kv.second.copy_ev);
            }
        ctx->results.clear();
        for (auto &r : ctx->rels) ctx->free_mat(r.dev);
        for (auto &p : ctx->props)
            if (p.dev) ctx->alloc->free(p.dev, ctx->stream);
        cudaStreamSynchronize(ctx->stream);
        if (ctx->htier.arena) cudaFreeHost(ctx->htier.arena);
        ctx->htier.arena = nullptr;
        cudaEventDestroy(ctx->ev0);
        cudaEventDestroy(ctx->ev1);
        ctx->prof.destroy();
        if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
        if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
    }
    delete ctx;
}

// ------------------------------------------------------------------ HIN ingestion

extern "C" int mp_add_node_type(mp_ctx *ctx, const char *name, uint32_t count, int32_t *type_id) {
    if (!ctx || !name || !*name) return MP_ERR_ARG;
    std::lock_guard<std::mutex> g(ctx->mu);
    if (ctx->finalized) return MP_ERR_STATE;
    for (auto &t : ctx->types)
        if (t.name == name) return MP_ERR_ARG;
    ctx->types.push_back({name, count});
    if (type_id) *type_id = (int32_t)ctx->types.size() - 1;
    return MP_OK;
}

extern "C" int mp_add_property_i32(mp_ctx *ctx, int32_t type_id, const char *prop, const int32_t *values) {
    if (!ctx || !prop || !*prop) return MP_ERR_ARG;
    std::lock_guard<std::mutex> g(ctx->mu);
    if (ctx->finalized) return MP_ERR_STATE;
    if (type_id < 0 || type_id >= (int)ctx->types.size()) return MP_ERR_NOTFOUND;
    const uint32_t n = ctx->types[type_id].count;
    if (n && !values) return MP_ERR_ARG;
    for (auto &p : ctx->props)
        if (p.type == type_id && p.name == prop) return MP_ERR_ARG;
    mp_ctx::Prop p;
    p.type = type_id;
    p.name = prop;
    p.host.assign(values, values + n);
    ctx->props.push_back(std::move(p));
    return MP_OK;
}

extern "C" int mp_add_relation(mp_ctx *ctx, int32_t src_type, int32_t dst_type, uint64_t n_edges,
                               const uint32_t *src, const uint32_t *dst, int32_t *rel_id) {
    if (!ctx) return MP_ERR_ARG;
    std::lock_guard<std::mutex> g(ctx->mu);
    if (ctx->finalized) return MP_ERR_STATE;
    const int nt = (int)ctx->types.size();
    if (src_type < 0 || src_type >= nt || dst_type < 0 || dst_type >= nt) return MP_ERR_NOTFOUND;
    if (n_edges && (!src || !dst)) return MP_ERR_ARG;
    const uint32_t ns = ctx->types[src_type].count, nd = ctx->types[dst_type].count;
    for (uint64_t e = 0; e < n_edges; e++)
        if (src[e] >= ns || dst[e] >= nd) return MP_ERR_ARG;
    mp_ctx::Rel fwd, rev;
    fwd.src = src_type;
    fwd.dst = dst_type;
    fwd.s.assign(src, src + n_edges);
    fwd.d.assign(dst, dst + n_edges);
    rev.src = dst_type;
    rev.dst = src_type;
    ctx->rels.push_back(std::move(fwd));
    ctx->rels.push_back(std::move(rev));
    if (rel_id) *rel_id = (int32_t)ctx->rels.size() - 2;
    return MP_OK;
}

// Host CSR of the 0/1 adjacency of (s, d) pairs: counting sort by row, then sort and
// de-duplicate each row.
static void build_csr(const std::vector<uint32_t> &s, const std::vector<uint32_t> &d, uint32_t nrows,
                      std::vector<int64_t> &rp, std::vector<int32_t> &ci) {
    std::vector<int64_t> cnt((size_t)nrows + 1, 0);
    for (uint32_t x : s) cnt[x + 1]++;
    for (size_t i = 0; i < nrows; i++) cnt[i + 1] += cnt[i];
    std::vector<int32_t> tmp(s.size());
    std::vector<int64_t> cur(cnt.begin(), cnt.end() - 1);
    for (size_t e = 0; e < s.size(); e++) tmp[cur[s[e]]++] = (int32_t)d[e];
    rp.assign((size_t)nrows + 1, 0);
    ci.clear();
    ci.reserve(s.size());
    for (uint32_t i = 0; i < nrows; i++) {
        auto b = tmp.begin() + cnt[i], e = tmp.begin() + cnt[i + 1];
        std::sort(b, e);
        auto last = std::unique(b, e);
        ci.insert(ci.end(), b, last);
        rp[i + 1] = (int64_t)ci.size();
    }
}

extern "C" int mp_finalize_hin(mp_ctx *ctx) {
    if (!ctx) return MP_ERR_ARG;
    std::lock_guard<std::mutex> g(ctx->mu);
    if (ctx->finalized) return MP_ERR_STATE;
    cudaSetDevice(ctx->cfg.device);
    cudaStream_t s = ctx->stream;
    // host CSRs of every relation in both directions, built on host threads (ingestion;
    // Sec. 4.1.4 leaves it out of query time), then uploaded one by one
    const size_t nrel = ctx->rels.size();
    std::vector<std::vector<int64_t>> hrp(nrel);
    std::vector<std::vector<int32_t>> hci(nrel);
    {
        std::vector<std::thread> th;
        for (size_t x = 0; x < nrel; x++) {
            auto &R = ctx->rels[x];
            if (!R.hrp.empty()) {  // loaded from a saved HIN
                hrp[x].swap(R.hrp);
                hci[x].swap(R.hci);
                continue;
            }
            auto &f = ctx->rels[x & ~(size_t)1];
            const uint32_t nr = ctx->types[R.src].count;
            const bool fwd = (x & 1) == 0;
            th.emplace_back([&, x, nr, fwd] {
                if (fwd) build_csr(f.s, f.d, nr, hrp[x], hci[x]);
                else build_csr(f.d, f.s, nr, hrp[x], hci[x]);
            });
        }
        for (auto &t : th) t.join();
    }
    for (size_t r = 0; r < nrel; r += 2) {
        auto &f = ctx->rels[r];
        for (int dir = 0; dir < 2; dir++) {
            auto &R = ctx->rels[r + dir];
            const uint32_t nr = ctx->types[R.src].count, nc = ctx->types[R.dst].count;
            std::vector<int64_t> rp;
            std::vector<int32_t> ci;
            rp.swap(hrp[r + dir]);
            ci.swap(hci[r + dir]);
            Mat &m = R.dev;
            m.nrows = nr;
            m.ncols = nc;
            m.nnz = (int64_t)ci.size();
            m.rp = (int64_t *)ctx->alloc->alloc(rp.size() * 8, s);
            m.ci = (int32_t *)ctx->alloc->alloc(std::max<size_t>(ci.size(), 1) * 4, s);
            if (!m.rp || !m.ci) return MP_ERR_NOMEM;
            if (check_cuda(cudaMemcpyAsync(m.rp, rp.data(), rp.size() * 8, cudaMemcpyHostToDevice, s), "upload"))
                return MP_ERR_CUDA;
            if (!ci.empty() &&
                check_cuda(cudaMemcpyAsync(m.ci, ci.data(), ci.size() * 4, cudaMemcpyHostToDevice, s), "upload"))
                return MP_ERR_CUDA;
            if (check_cuda(cudaStreamSynchronize(s), "upload")) return MP_ERR_CUDA;
        }
        f.s.clear();
        f.s.shrink_to_fit();
        f.d.clear();
        f.d.shrink_to_fit();
    }
    for (auto &p : ctx->props) {
        size_t n = p.host.size();
        p.dev = (int32_t *)ctx->alloc->alloc(std::max<size_t>(n, 1) * 4, s);
        if (!p.dev) return MP_ERR_NOMEM;
        if (n && check_cuda(cudaMemcpyAsync(p.dev, p.host.data(), n * 4, cudaMemcpyHostToDevice, s), "upload"))
            return MP_ERR_CUDA;
    }
    if (check_cuda(cudaStreamSynchronize(s), "upload")) return MP_ERR_CUDA;
    ctx->finalized = true;
    if (ctx->fail_alloc_after != UINT64_MAX) ctx->alloc->fail_after = ctx->fail_alloc_after;
    return MP_OK;
}

// ---- saved HINs: "MPHIN1", then node types, properties and every relation's CSR (both
// directions), all little-endian
static bool wr(FILE *f, const void *p, size_t n) { return fwrite(p, 1, n, f) == n; }
static bool rd(FILE *f, void *p, size_t n) { return fread(p, 1, n, f) == n; }

extern "C" int mp_hin_save(mp_ctx *ctx, const char *path) {
    if (!ctx || !path) return MP_ERR_ARG;
    std::lock_guard<std::mutex> ge(ctx->exec_mu);
    if (!ctx->finalized) return MP_ERR_STATE;
    cudaSetDevice(ctx->cfg.device);
    FILE *f = fopen(path, "wb");
    if (!f) return MP_ERR_ARG;
    bool ok = wr(f, "MPHIN1", 6);
    uint64_t n = ctx->types.size();
    ok = ok && wr(f, &n, 8);
    for (auto &t : ctx->types) {
        uint64_t l = t.name.size();
        ok = ok && wr(f, &l, 8) && wr(f, t.name.data(), l) && wr(f, &t.count, 4);
    }
    n = ctx->props.size();
    ok = ok && wr(f, &n, 8);
    for (auto &p : ctx->props) {
        uint64_t l = p.name.size();
        ok = ok && wr(f, &p.type, 4) && wr(f, &l, 8) && wr(f, p.name.data(), l) &&
             wr(f, p.host.data(), p.host.size() * 4);
    }
    n = ctx->rels.size();
    ok = ok && wr(f, &n, 8);
    for (auto &r : ctx->rels) {
        const Mat &m = r.dev;
        std::vector<int64_t> rp((size_t)m.nrows + 1);
        std::vector<int32_t> ci((size_t)m.nnz);
        if (cudaMemcpy(rp.data(), m.rp, rp.size() * 8, cudaMemcpyDeviceToHost) != cudaSuccess ||
            (m.nnz && cudaMemcpy(ci.data(), m.ci, ci.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess)) {
            fclose(f);
            return MP_ERR_CUDA;
        }
        const int64_t nnz = m.nnz;
        ok = ok && wr(f, &r.src, 4) && wr(f, &r.dst, 4) && wr(f, &nnz, 8) && wr(f, rp.data(), rp.size() * 8) &&
             wr(f, ci.data(), ci.size() * 4);
    }
    ok = (fclose(f) == 0) && ok;
    return ok ? MP_OK : MP_ERR_ARG;
}

extern "C" int mp_hin_load(mp_ctx *ctx, const char *path) {
    if (!ctx || !path) return MP_ERR_ARG;
    std::lock_guard<std::mutex> g(ctx->mu);
    if (ctx->finalized || !ctx->types.empty() || !ctx->rels.empty()) return MP_ERR_STATE;
    FILE *f = fopen(path, "rb");
    if (!f) return MP_ERR_NOTFOUND;
    char magic[6];
    bool ok = rd(f, magic, 6) && memcmp(magic, "MPHIN1", 6) == 0;
    uint64_t n = 0;
    ok = ok && rd(f, &n, 8) && n < (1u << 20);
    for (uint64_t i = 0; ok && i < n; i++) {
        uint64_t l = 0;
        ok = rd(f, &l, 8) && l < 4096;
        std::string name(ok ? l : 0, ' ');
        uint32_t cnt = 0;
        ok = ok && rd(f, &name[0], l) && rd(f, &cnt, 4);
        if (ok) ctx->types.push_back({name, cnt});
    }
    ok = ok && rd(f, &n, 8) && n < (1u << 20);
    for (uint64_t i = 0; ok && i < n; i++) {
        mp_ctx::Prop p;
        uint64_t l = 0;
        ok = rd(f, &p.type, 4) && p.type >= 0 && p.type < (int)ctx->types.size() && rd(f, &l, 8) && l < 4096;
        if (!ok) break;
        p.name.assign(l, ' ');
        p.host.resize(ctx->types[p.type].count);
        ok = rd(f, &p.name[0], l) && rd(f, p.host.data(), p.host.size() * 4);
        if (ok) ctx->props.push_back(std::move(p));
    }
    ok = ok && rd(f, &n, 8) && n % 2 == 0 && n < (1u << 20);
    for (uint64_t i = 0; ok && i < n; i++) {
        mp_ctx::Rel r;
        int64_t nnz = 0;
        ok = rd(f, &r.src, 4) && rd(f, &r.dst, 4) && r.src >= 0 && r.dst >= 0 && r.src < (int)ctx->types.size() &&
             r.dst < (int)ctx->types.size() && rd(f, &nnz, 8) && nnz >= 0;
        if (!ok) break;
        r.hrp.resize((size_t)ctx->types[r.src].count + 1);
        r.hci.resize((size_t)nnz);
        ok = rd(f, r.hrp.data(), r.hrp.size() * 8) && rd(f, r.hci.data(), r.hci.size() * 4) && r.hrp.back() == nnz;
        if (ok) ctx->rels.push_back(std::move(r));
    }
    fclose(f);
    if (!ok) {
        ctx->types.clear();
        ctx->props.clear();
        ctx->rels.clear();
        return MP_ERR_ARG;
    }
    return MP_OK;
}

extern "C" int mp_type_id(mp_ctx *ctx, const char *name, int32_t *type_id) {
    if (!ctx || !name || !type_id) return MP_ERR_ARG;
    std::lock_guard<std::mutex> g(ctx->mu);
    for (size_t t = 0; t < ctx->types.size(); t++)
        if (ctx->types[t].name == name) {
            *type_id = (int32_t)t;
            return MP_OK;
        }
    return MP_ERR_NOTFOUND;
}

extern "C" int mp_property_id(mp_ctx *ctx, int32_t type_id, const char *prop, int32_t *prop_id) {
    if (!ctx || !prop || !prop_id) return MP_ERR_ARG;
    std::lock_guard<std::mutex> g(ctx->mu);
    for (size_t p = 0; p < ctx->props.size(); p++)
        if (ctx->props[p].type == type_id && ctx->props[p].name == prop) {
            *prop_id = (int32_t)p;
            return MP_OK;
        }
    return MP_ERR_NOTFOUND;
}

extern "C" int mp_relation_id(mp_ctx *ctx, int32_t src_type, int32_t dst_type, int32_t *rel_id) {
    if (!ctx || !rel_id) return MP_ERR_ARG;
    std::lock_guard<std::mutex> g(ctx->mu);
    for (size_t r = 0; r < ctx->rels.size(); r++)
        if (ctx->rels[r].src == src_type && ctx->rels[r].dst == dst_type) {
            *rel_id = (int32_t)r;
            return MP_OK;
        }
    return MP_ERR_NOTFOUND;
}

// ------------------------------------------------------------------ queries

int mp_ctx::parse(const mp_query *q, Query &out) {
    if (!q || q->n_types < 2 || !q->types) return MP_ERR_ARG;
    if (q->n_constraints && !q->c) return MP_ERR_ARG;
    const int n = (int)q->n_types;
    out.types.assign(q->types, q->types + n);
    for (int t : out.types)
        if (t < 0 || t >= (int)types.size()) return MP_ERR_NOTFOUND;
    out.rels.resize(n - 1);
    for (int t = 0; t + 1 < n; t++) {
        int r = -1;
        if (q->rels) {
            r = q->rels[t];
            if (r < 0 || r >= (int)rels.size()) return MP_ERR_NOTFOUND;
            if (rels[r].src != out.types[t] || rels[r].dst != out.types[t + 1]) return MP_ERR_ARG;
        } else {
            for (size_t x = 0; x < rels.size(); x++)
                if (rels[x].src == out.types[t] && rels[x].dst == out.types[t + 1]) {
                    r = (int)x;
                    break;
                }
            if (r < 0) return MP_ERR_NOTFOUND;
        }
        out.rels[t] = r;
    }
    out.cons.assign(n, {});
    for (uint32_t c = 0; c < q->n_constraints; c++) {
        const mp_constraint &k = q->c[c];
        if (k.pos < 0 || k.pos >= n) return MP_ERR_ARG;
        if (k.op < MP_OP_RANGE || k.op > MP_OP_IN) return MP_ERR_ARG;
        if (k.prop >= 0) {
            if (k.prop >= (int)props.size() || props[k.prop].type != out.types[k.pos]) return MP_ERR_ARG;
        } else if (k.prop != -1) {
            return MP_ERR_ARG;
        }
        if (k.op == MP_OP_IN && k.set_len && !k.set) return MP_ERR_ARG;
        Constraint cc;
        cc.prop = k.prop;
        cc.op = k.op;
        cc.lo = k.lo;
        cc.hi = k.op == MP_OP_EQ ? k.lo : k.hi;
        if (k.op == MP_OP_IN) {
            cc.set.assign(k.set, k.set + k.set_len);
            std::sort(cc.set.begin(), cc.set.end());
            cc.set.erase(std::unique(cc.set.begin(), cc.set.end()), cc.set.end());
        }
        out.cons[k.pos].push_back(std::move(cc));
    }
    // canonical per-position constraint text (sorted), used by the Overlap Tree and the
    // cache keys; a query with any non-default relation also tags each position > 0 with
    // the relation that enters it, so sub-chains over different relations never share keys
    bool custom_rel = false;
    for (int t = 0; t + 1 < n; t++) {
        for (size_t x = 0; x < rels.size(); x++)
            if (rels[x].src == out.types[t] && rels[x].dst == out.types[t + 1]) {
                if ((int)x != out.rels[t]) custom_rel = true;
                break;
            }
    }
    out.pos_keys.assign(n, std::string());
    for (int i = 0; i < n; i++) {
        std::vector<std::string> parts;
        for (const Constraint &c : out.cons[i]) {
            std::string d = "p" + std::to_string(c.prop) + "o" + std::to_string(c.op);
            if (c.op == MP_OP_IN) {
                d += "{";
                for (size_t e = 0; e < c.set.size(); e++) {
                    if (e) d += ",";
                    d += std::to_string(c.set[e]);
                }
                d += "}";
            } else {
                d += "[" + std::to_string(c.lo) + "," + std::to_string(c.hi) + "]";
            }
            parts.push_back(d);
        }
        std::sort(parts.begin(), parts.end());
        std::string key;
        for (auto &x : parts) {
            if (!key.empty()) key += "&";
            key += x;
        }
        if (custom_rel && i > 0) key += "@r" + std::to_string(out.rels[i - 1]);
        out.pos_keys[i] = key;
    }
    return MP_OK;
}

// Queue parsed queries for the serving loop; tickets come back at once.
static int enqueue(mp_ctx *ctx, std::vector<Query> &qs, mp_ticket *tickets) {
    const auto now = std::chrono::steady_clock::now();
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        for (size_t i = 0; i < qs.size(); i++) {
            tickets[i] = ctx->next_ticket++;
            Result r;
            r.done = false;
            ctx->results.emplace(tickets[i], std::move(r));
        }
    }
    {
        std::lock_guard<std::mutex> g(ctx->qmu);
        for (size_t i = 0; i < qs.size(); i++) ctx->queue.push_back({tickets[i], std::move(qs[i]), now});
    }
    ctx->qcv.notify_one();
    return MP_OK;
}

// Run parsed queries now, on the caller's thread.
static int run_now(mp_ctx *ctx, std::vector<Query> &qs, mp_ticket *tickets) {
    const auto t0 = std::chrono::steady_clock::now();
    std::vector<Result> res(qs.size());
    int first;
    {
        std::lock_guard<std::mutex> ge(ctx->exec_mu);
        cudaSetDevice(ctx->cfg.device);
        first = ctx->run_batch(qs, res);
    }
    const double lat = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    std::lock_guard<std::mutex> g(ctx->mu);
    for (size_t i = 0; i < qs.size(); i++) {
        tickets[i] = ctx->next_ticket++;
        res[i].latency_ms = lat;
        ctx->results.emplace(tickets[i], std::move(res[i]));
    }
    return first;
}

extern "C" int mp_plan_query(mp_ctx *ctx, const mp_query *q, uint32_t cap, int32_t *split, double *nnz,
                             uint32_t *p_out) {
    if (!ctx || !q || !p_out) return MP_ERR_ARG;
    if (!ctx->finalized) return MP_ERR_STATE;
    std::vector<Query> qs(1);
    int rc = ctx->parse(q, qs[0]);
    if (rc) return rc;
    std::vector<Result> res(1);
    std::lock_guard<std::mutex> ge(ctx->exec_mu);
    cudaSetDevice(ctx->cfg.device);
    ctx->explain = mp_ctx::Explain{};
    ctx->explain.on = true;
    rc = ctx->run_batch(qs, res);
    ctx->explain.on = false;
    if (rc) return rc;
    if (res[0].status) return res[0].status;
    const uint32_t p = (uint32_t)ctx->explain.p;
    *p_out = p;
    if ((uint64_t)p * p > cap) return MP_ERR_ARG;
    for (size_t t = 0; t < (size_t)p * p; t++) {
        if (split) split[t] = ctx->explain.split[t];
        if (nnz) nnz[t] = ctx->explain.nnz[t];
    }
    return MP_OK;
}

extern "C" int mp_submit(mp_ctx *ctx, const mp_query *q, mp_ticket *ticket) {
    return mp_submit_batch(ctx, 1, q, ticket);
}

extern "C" int mp_submit_batch(mp_ctx *ctx, uint32_t n, const mp_query *q, mp_ticket *tickets) {
    if (!ctx || (n && (!q || !tickets))) return MP_ERR_ARG;
    if (!ctx->finalized) return MP_ERR_STATE;
    std::vector<Query> qs(n);
    for (uint32_t i = 0; i < n; i++) {
        int rc = ctx->parse(&q[i], qs[i]);
        if (rc) return rc;
    }
    bool serving;
    {
        std::lock_guard<std::mutex> g(ctx->qmu);
        serving = ctx->serving;
    }
    return serving ? enqueue(ctx, qs, tickets) : run_now(ctx, qs, tickets);
}

// The serving loop (continuous batching). Every turn it admits the queries that have
// arrived, as far as free slots (mp_config.max_slots) and the HBM budget allow: their
// plans join the product DAG of the queries already in flight, sharing any sub-chain
// that is on its way or held. It then runs one wave -- every product whose operands are
// ready, whichever query it belongs to, in one set of launches -- and publishes each
// query whose result is complete. A query that arrives while others are on the GPU thus
// starts with the next wave, beside their later products, instead of waiting for them
// to finish. Admission by bytes: new queries wait while the planned result bytes of the
// queries in flight exceed the budget (one query is always admitted when none is in
// flight); the exact size of every product is charged before its arrays are made, where
// the cache yields first (MP_ERR_BUDGET only when the query's work cannot fit at all).
void mp_ctx::serve_loop() {
    cudaSetDevice(cfg.device);
    const size_t slots = cfg.max_slots ? cfg.max_slots : 1;
    const double budget = cfg.hbm_budget_bytes ? (double)cfg.hbm_budget_bytes : INFINITY;
    for (;;) {
        std::vector<Pending> batch;
        {
            std::unique_lock<std::mutex> lk(qmu);
            qcv.wait(lk, [&] { return stop_req || !queue.empty() || inflight > 0; });
            if (queue.empty() && stop_req && inflight == 0) break;
            while (!queue.empty() && inflight + batch.size() < slots &&
                   (inflight + batch.size() == 0 || inflight_bytes < budget)) {
                batch.push_back(std::move(queue.front()));
                queue.pop_front();
            }
        }
        std::vector<Flight> done;
        {
            std::lock_guard<std::mutex> ge(exec_mu);
            TraceRange serve_range("mp.serve_turn");
            if (!batch.empty()) {
                std::vector<Query> qs(batch.size());
                std::vector<uint64_t> tk(batch.size());
                std::vector<std::chrono::steady_clock::time_point> t0s(batch.size());
                for (size_t i = 0; i < batch.size(); i++) {
                    qs[i] = std::move(batch[i].q);
                    tk[i] = batch[i].ticket;
                    t0s[i] = batch[i].t0;
                }
                std::vector<int64_t> ids;
                const size_t before = ex.flights.size();
                if (before) serve_joined += qs.size();  // joining work already on the GPU
                admit(qs, tk, t0s, ids);
                batches++;
                serve_max_inflight = std::max<uint64_t>(serve_max_inflight, ex.flights.size());
            }
            finish_flights(done);  // queries served from the cache or failed at admission
            if (!ex.flights.empty()) {
                serve_waves++;
                const int rc = run_wave();
                if (rc) abort_nodes(rc);
                finish_flights(done);
            }
            batched_queries += done.size();
            std::lock_guard<std::mutex> g(qmu);
            inflight = ex.flights.size();
            inflight_bytes = ex.est_bytes;
        }
        if (!done.empty()) publish(done);
    }
}

extern "C" int mp_serve_start(mp_ctx *ctx) {
    if (!ctx) return MP_ERR_ARG;
    if (!ctx->finalized) return MP_ERR_STATE;
    std::lock_guard<std::mutex> g(ctx->qmu);
    if (ctx->serving) return MP_ERR_STATE;
    ctx->stop_req = false;
    ctx->serving = true;
    ctx->server = std::thread([ctx] { ctx->serve_loop(); });
    return MP_OK;
}

extern "C" int mp_serve_stop(mp_ctx *ctx) {
    if (!ctx) return MP_ERR_ARG;
    {
        std::lock_guard<std::mutex> g(ctx->qmu);
        if (!ctx->serving) return MP_OK;
        ctx->stop_req = true;
    }
    ctx->qcv.notify_all();
    if (ctx->server.joinable()) ctx->server.join();
    std::lock_guard<std::mutex> g(ctx->qmu);
    ctx->serving = false;
    return MP_OK;
}

extern "C" int mp_serve_stats(mp_ctx *ctx, uint64_t *batches, uint64_t *queries, uint64_t *queued) {
    if (!ctx) return MP_ERR_ARG;
    {
        std::lock_guard<std::mutex> ge(ctx->exec_mu);
        if (batches) *batches = ctx->batches;
        if (queries) *queries = ctx->batched_queries;
    }
    std::lock_guard<std::mutex> g(ctx->qmu);
    if (queued) *queued = ctx->queue.size();
    return MP_OK;
}

extern "C" int mp_serve_counters(mp_ctx *ctx, uint64_t *waves, uint64_t *joined, uint64_t *max_inflight) {
    if (!ctx) return MP_ERR_ARG;
    std::lock_guard<std::mutex> ge(ctx->exec_mu);
    if (waves) *waves = ctx->serve_waves;
    if (joined) *joined = ctx->serve_joined;
    if (max_inflight) *max_inflight = ctx->serve_max_inflight;
    return MP_OK;
}

extern "C" int mp_budget_stats(mp_ctx *ctx, uint64_t *held, uint64_t *peak) {
    if (!ctx) return MP_ERR_ARG;
    if (held) *held = (uint64_t)std::max<int64_t>(0, ctx->held.load());
    if (peak) *peak = (uint64_t)std::max<int64_t>(0, ctx->held_peak.load());
    return MP_OK;
}

// Least squares for y ~ a*x0 + b*x1 + c*x2 (normal equations, Cramer's rule).
static bool fit3(const std::vector<std::array<double, 4>> &s, double out[3]) {
    double A[3][3] = {}, B[3] = {};
    for (auto &r : s)
        for (int i = 0; i < 3; i++) {
            B[i] += r[i] * r[3];
            for (int j = 0; j < 3; j++) A[i][j] += r[i] * r[j];
        }
    auto det = [](double M[3][3]) {
        return M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) - M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
               M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
    };
    const double d = det(A);
    if (!(std::fabs(d) > 0)) return false;
    for (int k = 0; k < 3; k++) {
        double M[3][3];
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) M[i][j] = j == k ? B[i] : A[i][j];
        out[k] = det(M) / d;
    }
    return true;
}

extern "C" int mp_autotune(mp_ctx *ctx, uint32_t n, const mp_query *q, uint32_t reps, const char *out_path,
                           double *best_ms) {
    TraceRange tune_range("mp.autotune");
    if (!ctx || !n || !q) return MP_ERR_ARG;
    if (!ctx->finalized) return MP_ERR_STATE;
    std::vector<Query> parsed(n);
    for (uint32_t i = 0; i < n; i++) {
        int rc = ctx->parse(&q[i], parsed[i]);
        if (rc) return rc;
    }
    if (reps == 0) reps = 1;
    std::lock_guard<std::mutex> ge(ctx->exec_mu);
    cudaSetDevice(ctx->cfg.device);
    std::unique_ptr<CachePolicy> saved_cache(ctx->cache.release());  // timings without cache hits
    const Tuning base = ctx->tun;
    const int dmu[] = {64, 256, 1024};
    const uint64_t heavy[] = {16384, 65536, 262144};
    double best = INFINITY;
    Tuning best_t = base;
    std::string log;
    int rc = MP_OK;
    for (int a : dmu)
        for (uint64_t h : heavy) {
            ctx->tun = base;
            ctx->tun.dense_min_u = a;
            ctx->tun.heavy = h;
            std::vector<double> ts;
            for (uint32_t r = 0; r < reps + 1 && !rc; r++) {
                std::vector<Query> qs = parsed;
                std::vector<Result> res(n);
                const auto t0 = std::chrono::steady_clock::now();
                rc = ctx->run_batch(qs, res);
                const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
                if (r) ts.push_back(ms);  // the first run warms up
            }
            if (rc) break;
            std::sort(ts.begin(), ts.end());
            const double med = ts[ts.size() / 2];
            char line[160];
            snprintf(line, sizeof(line), "%s{\"dense_min_u\": %d, \"heavy\": %llu, \"ms\": %.4f}", log.empty() ? "" : ", ", a,
                     (unsigned long long)h, med);
            log += line;
            if (med < best) {
                best = med;
                best_t = ctx->tun;
            }
        }
    // the split-row kernel variants at the best thresholds, one knob flipped at a time from
    // the best so far: combining table, warp-level or block-staged product walk, blocks per
    // SM of the warp walk's adding passes, and (staged walk) its segment walk and occupancy
    for (int v = 0; v < 5 && !rc; v++) {
        ctx->tun = best_t;
        if (v == 0) ctx->tun.combine ^= 1;
        if (v == 1) ctx->tun.lbs ^= 1;
        if (v == 2 && !ctx->tun.lbs) continue;
        if (v == 2) ctx->tun.lbs_occ = ctx->tun.lbs_occ >= 6 ? 4 : 6;
        if (v >= 3 && ctx->tun.lbs) continue;
        if (v == 3) ctx->tun.seg_walk ^= 1;
        if (v == 4) ctx->tun.glob_occ = ctx->tun.glob_occ >= 6 ? 4 : 6;
        std::vector<double> ts;
        for (uint32_t r = 0; r < reps + 1 && !rc; r++) {
            std::vector<Query> qs = parsed;
            std::vector<Result> res(n);
            const auto t0 = std::chrono::steady_clock::now();
            rc = ctx->run_batch(qs, res);
            const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
            if (r) ts.push_back(ms);
        }
        if (rc) break;
        std::sort(ts.begin(), ts.end());
        const double med = ts[ts.size() / 2];
        char line[200];
        snprintf(line, sizeof(line),
                 ", {\"combine\": %d, \"lbs\": %d, \"lbs_occ\": %d, \"seg_walk\": %d, \"glob_occ\": %d, "
                 "\"ms\": %.4f}",
                 ctx->tun.combine, ctx->tun.lbs, ctx->tun.lbs_occ, ctx->tun.seg_walk, ctx->tun.glob_occ, med);
        log += line;
        if (med < best) {
            best = med;
            best_t = ctx->tun;
        }
    }
    ctx->tun = rc ? base : best_t;
    // Eq. 2 coefficients from per-product times, each query run on its own
    double coef[3] = {ctx->cfg.alpha, ctx->cfg.beta, ctx->cfg.gamma};
    bool fitted = false;
    if (!rc) {
        ctx->fit_samples.clear();
        ctx->collect_fit = true;
        for (uint32_t i = 0; i < n && !rc; i++) {
            std::vector<Query> qs(1, parsed[i]);
            std::vector<Result> res(1);
            rc = ctx->run_batch(qs, res);
        }
        ctx->collect_fit = false;
        double c[3];
        if (!rc && ctx->fit_samples.size() >= 3 && fit3(ctx->fit_samples, c)) {
            // a cost model with a negative weight would reward work: keep those terms at a floor
            double fitc[3];
            for (int k = 0; k < 3; k++) fitc[k] = c[k] > 1e-12 ? c[k] : 1e-12;
            // keep the fit only if the plans it chooses do not make the workload slower
            const double old_c[3] = {ctx->cfg.alpha, ctx->cfg.beta, ctx->cfg.gamma};
            ctx->cfg.alpha = fitc[0];
            ctx->cfg.beta = fitc[1];
            ctx->cfg.gamma = fitc[2];
            std::vector<double> ts;
            for (uint32_t r = 0; r < reps + 1 && !rc; r++) {
                std::vector<Query> qs = parsed;
                std::vector<Result> res(n);
                const auto t0 = std::chrono::steady_clock::now();
                rc = ctx->run_batch(qs, res);
                const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
                if (r) ts.push_back(ms);
            }
            if (!rc) {
                std::sort(ts.begin(), ts.end());
                const double med = ts[ts.size() / 2];
                char line[200];
                snprintf(line, sizeof(line), ", {\"fitted_eq2\": true, \"ms\": %.4f}", med);
                log += line;
                if (med <= best) {
                    best = med;
                    for (int k = 0; k < 3; k++) coef[k] = fitc[k];
                    fitted = true;
                } else {
                    ctx->cfg.alpha = old_c[0];
                    ctx->cfg.beta = old_c[1];
                    ctx->cfg.gamma = old_c[2];
                }
            }
        }
        ctx->fit_samples.clear();
    }
    ctx->cache.reset(saved_cache.release());
    if (rc) return rc;
    if (best_ms) *best_ms = best;
    if (out_path) {
        FILE *f = fopen(out_path, "w");
        if (!f) return MP_ERR_ARG;
        fprintf(f, "{\"dense_min_u\": %d, \"heavy\": %llu, \"combine\": %d, \"short_walk\": %d, "
                   "\"seg_walk\": %d, \"glob_occ\": %d, \"lbs\": %d, \"lbs_occ\": %d, "
                   "\"alpha\": %.9g, \"beta\": %.9g, \"gamma\": %.9g, \"fitted\": %s, \"best_ms\": %.4f, "
                   "\"candidates\": [%s]}\n",
                ctx->tun.dense_min_u, (unsigned long long)ctx->tun.heavy, ctx->tun.combine, ctx->tun.short_walk,
                ctx->tun.seg_walk, ctx->tun.glob_occ, ctx->tun.lbs, ctx->tun.lbs_occ, coef[0], coef[1], coef[2],
                fitted ? "true" : "false", best, log.c_str());
        fclose(f);
    }
    return MP_OK;
}

extern "C" int mp_result_latency(mp_ctx *ctx, mp_ticket t, double *ms) {
    if (!ctx || !ms) return MP_ERR_ARG;
    std::lock_guard<std::mutex> g(ctx->mu);
    auto it = ctx->results.find(t);
    if (it == ctx->results.end()) return MP_ERR_NOTFOUND;
    if (!it->second.done) return MP_ERR_STATE;
    *ms = it->second.latency_ms;
    return MP_OK;
}

extern "C" int mp_wait(mp_ctx *ctx, mp_ticket t, uint32_t timeout_ms) {
    if (!ctx) return MP_ERR_ARG;
    std::unique_lock<std::mutex> lk(ctx->mu);
    auto ready = [&] {
        auto it = ctx->results.find(t);
        return it == ctx->results.end() || it->second.done;
    };
    if (timeout_ms == UINT32_MAX) ctx->done_cv.wait(lk, ready);
    else if (!ctx->done_cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) return MP_ERR_TIMEOUT;
    auto it = ctx->results.find(t);
    if (it == ctx->results.end()) return MP_ERR_NOTFOUND;
    return it->second.status;
}

extern "C" int mp_result_info(mp_ctx *ctx, mp_ticket t, uint32_t *rows, uint32_t *cols, uint64_t *nnz) {
    if (!ctx) return MP_ERR_ARG;
    std::lock_guard<std::mutex> g(ctx->mu);
    auto it = ctx->results.find(t);
    if (it == ctx->results.end()) return MP_ERR_NOTFOUND;
    if (!it->second.done) return MP_ERR_STATE;
    if (it->second.status) return it->second.status;
    const Mat &m = it->second.m->m;
    if (rows) *rows = (uint32_t)m.nrows;
    if (cols) *cols = (uint32_t)m.ncols;
    if (nnz) *nnz = (uint64_t)m.nnz;
    return MP_OK;
}

extern "C" int mp_result_copy(mp_ctx *ctx, mp_ticket t, int64_t *row_ptr, int32_t *col, uint64_t *val,
                              int on_device) {
    if (!ctx) return MP_ERR_ARG;
    std::lock_guard<std::mutex> g(ctx->mu);
    auto it = ctx->results.find(t);
    if (it == ctx->results.end()) return MP_ERR_NOTFOUND;
    if (!it->second.done) return MP_ERR_STATE;
    if (it->second.status) return it->second.status;
    cudaSetDevice(ctx->cfg.device);
    const Mat &m = it->second.m->m;
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    cudaStream_t s = ctx->copy_stream;
    if (row_ptr && check_cuda(cudaMemcpyAsync(row_ptr, m.rp, (size_t)(m.nrows + 1) * 8, k, s), "copy"))
        return MP_ERR_CUDA;
    if (m.nnz && col && check_cuda(cudaMemcpyAsync(col, m.ci, (size_t)m.nnz * 4, k, s), "copy"))
        return MP_ERR_CUDA;
    if (m.nnz && val && check_cuda(cudaMemcpyAsync(val, m.val, (size_t)m.nnz * 8, k, s), "copy"))
        return MP_ERR_CUDA;
    return check_cuda(cudaStreamSynchronize(s), "copy");
}

extern "C" int mp_result_copy_async(mp_ctx *ctx, mp_ticket t, int64_t *row_ptr, int32_t *col, uint64_t *val,
                                    int on_device) {
    if (!ctx) return MP_ERR_ARG;
    std::lock_guard<std::mutex> g(ctx->mu);
    auto it = ctx->results.find(t);
    if (it == ctx->results.end()) return MP_ERR_NOTFOUND;
    if (!it->second.done) return MP_ERR_STATE;
    if (it->second.status) return it->second.status;
    cudaSetDevice(ctx->cfg.device);
    const Mat &m = it->second.m->m;
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    cudaStream_t s = ctx->copy_stream;
    if (!it->second.copy_ev &&
        check_cuda(cudaEventCreateWithFlags(&it->second.copy_ev, cudaEventDisableTiming), "event"))
        return MP_ERR_CUDA;
    if (row_ptr && check_cuda(cudaMemcpyAsync(row_ptr, m.rp, (size_t)(m.nrows + 1) * 8, k, s), "copy"))
        return MP_ERR_CUDA;
    if (m.nnz && col && check_cuda(cudaMemcpyAsync(col, m.ci, (size_t)m.nnz * 4, k, s), "copy"))
        return MP_ERR_CUDA;
    if (m.nnz && val && check_cuda(cudaMemcpyAsync(val, m.val, (size_t)m.nnz * 8, k, s), "copy"))
        return MP_ERR_CUDA;
    return check_cuda(cudaEventRecord(it->second.copy_ev, s), "event");
}

extern "C" int mp_result_copy_wait(mp_ctx *ctx, mp_ticket t) {
    if (!ctx) return MP_ERR_ARG;
    cudaEvent_t ev = nullptr;
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        auto it = ctx->results.find(t);
        if (it == ctx->results.end()) return MP_ERR_NOTFOUND;
        ev = it->second.copy_ev;
    }
    if (!ev) return MP_OK;
    return check_cuda(cudaEventSynchronize(ev), "copy");
}

extern "C" int mp_release(mp_ctx *ctx, mp_ticket t) {
    if (!ctx) return MP_ERR_ARG;
    std::lock_guard<std::mutex> g(ctx->mu);
    auto it = ctx->results.find(t);
    if (it == ctx->results.end()) return MP_ERR_NOTFOUND;
    if (it->second.copy_ev) {
        // the result's device memory is freed in the order of the context's stream: let
        // that stream first wait for an asynchronous copy still reading it
        cudaSetDevice(ctx->cfg.device);
        cudaStreamWaitEvent(ctx->stream, it->second.copy_ev, 0);
        cudaEventDestroy(it->second.copy_ev);
    }
    ctx->results.erase(it);
    return MP_OK;
}

extern "C" int mp_result_time(mp_ctx *ctx, mp_ticket t, double *ms) {
    if (!ctx || !ms) return MP_ERR_ARG;
    std::lock_guard<std::mutex> g(ctx->mu);
    auto it = ctx->results.find(t);
    if (it == ctx->results.end()) return MP_ERR_NOTFOUND;
    *ms = it->second.ms;
    return MP_OK;
}

extern "C" int mp_result_stats(mp_ctx *ctx, mp_ticket t, uint64_t *products, uint32_t *sym_bins,
                               uint32_t *num_bins, uint32_t *n_products) {
    if (!ctx) return MP_ERR_ARG;
    std::lock_guard<std::mutex> g(ctx->mu);
    auto it = ctx->results.find(t);
    if (it == ctx->results.end()) return MP_ERR_NOTFOUND;
    const Result &r = it->second;
    if (products) *products = r.st.products;
    for (int b = 0; b < NBINS; b++) {
        if (sym_bins) sym_bins[b] = r.st.sym_bins[b];
        if (num_bins) num_bins[b] = r.st.num_bins[b];
    }
    if (n_products) *n_products = r.n_products;
    return MP_OK;
}

extern "C" int mp_plan_chain(uint32_t p, const double *dims, const double *nnz, double alpha, double beta,
                             double gamma, const double *known_cost, const double *known_rho,
                             const double *rho_fixed, int32_t *split, double *cost) {
    if (p < 1 || !dims || !nnz || !split) return MP_ERR_ARG;
    if ((known_cost == nullptr) != (known_rho == nullptr)) return MP_ERR_ARG;
    for (uint32_t t = 0; t <= p; t++)
        if (!(dims[t] > 0)) return MP_ERR_ARG;
    std::vector<int> sp((size_t)p * p);
    std::vector<double> c((size_t)p * p), r((size_t)p * p);
    plan_chain((int)p, dims, nnz, alpha, beta, gamma, known_cost, known_rho, rho_fixed, sp.data(), c.data(), r.data());
    for (size_t t = 0; t < sp.size(); t++) split[t] = sp[t];
    if (cost)
        for (size_t t = 0; t < c.size(); t++) cost[t] = c[t];
    return MP_OK;
}

extern "C" int mp_kernel_stats(mp_ctx *ctx, mp_kernel_stat *out, uint32_t cap, uint32_t *n, uint64_t *launches) {
    if (!ctx) return MP_ERR_ARG;
    static const char *bins[NBINS] = {"w32",   "w64",   "w128",  "w256",  "w512",   "w1024",
                                      "k2048", "k4096", "k8192", "dense", "global", "lane"};
    std::lock_guard<std::mutex> g(ctx->exec_mu);
    uint32_t w = 0;
    auto put = [&](const char *name, const KStat &k) {
        if (!k.launches || !out || w >= cap) return;
        snprintf(out[w].name, sizeof(out[w].name), "%s", name);
        out[w].launches = k.launches;
        out[w].ms = k.ms;
        out[w].bytes = k.bytes;
        out[w].products = k.prods;
        w++;
    };
    char name[32];
    for (int p = 0; p < 2; p++)
        for (int b = 0; b <= NBINS; b++) {
            snprintf(name, sizeof(name), "%s_%s", p ? "num" : "sym", b < NBINS ? bins[b] : "pool");
            put(name, b < NBINS ? ctx->prof.k[p][b] : ctx->prof.pool[p]);
        }
    put("walk_sym", ctx->prof.walk[0]);
    put("walk_num", ctx->prof.walk[1]);
    put("walk_dense", ctx->prof.walk[2]);
    static const char *stages[Prof::NSTAGE] = {"stage_rowwork", "stage_symbin", "stage_globsetup", "stage_rowptr",
                                                "stage_numbin"};
    for (int st = 0; st < Prof::NSTAGE; st++) put(stages[st], ctx->prof.stage[st]);
    if (n) *n = w;
    if (launches) *launches = g_launches.load();
    return MP_OK;
}

extern "C" int mp_cache_stats(mp_ctx *ctx, uint64_t *requests, uint64_t *hits, uint64_t *inserts,
                              uint64_t *rejected, uint64_t *evictions, uint64_t *bytes, uint64_t *entries) {
    if (!ctx) return MP_ERR_ARG;
    std::lock_guard<std::mutex> g(ctx->exec_mu);
    if (!ctx->cache) return MP_ERR_STATE;
    const auto &c = ctx->cstats;
    if (requests) *requests = c.requests;
    if (hits) *hits = c.hits;
    if (inserts) *inserts = c.inserts;
    if (rejected) *rejected = c.rejected;
    if (evictions) *evictions = c.evictions;
    if (bytes) *bytes = (uint64_t)ctx->cache->used();
    if (entries) *entries = (uint64_t)ctx->cache->size();
    return MP_OK;
}

extern "C" int mp_host_tier_stats(mp_ctx *ctx, uint64_t *stores, uint64_t *loads, uint64_t *drops,
                                  uint64_t *bytes, uint64_t *entries) {
    if (!ctx) return MP_ERR_ARG;
    std::lock_guard<std::mutex> g(ctx->exec_mu);
    if (!ctx->cache || !ctx->cfg.host_tier_bytes) return MP_ERR_STATE;
    const auto &h = ctx->htier;
    if (stores) *stores = h.stores;
    if (loads) *loads = h.loads;
    if (drops) *drops = h.drops;
    if (bytes) *bytes = (uint64_t)h.bytes;
    if (entries) *entries = (uint64_t)h.items.size();
    return MP_OK;
}

extern "C" int mp_graph_stats(mp_ctx *ctx, uint64_t *captures, uint64_t *replays) {
    if (!ctx) return MP_ERR_ARG;
    std::lock_guard<std::mutex> g(ctx->exec_mu);
    if (captures) *captures = ctx->wcache.captures;
    if (replays) *replays = ctx->wcache.replays;
    return MP_OK;
}

extern "C" int mp_kernel_stats_reset(mp_ctx *ctx) {
    if (!ctx) return MP_ERR_ARG;
    std::lock_guard<std::mutex> g(ctx->exec_mu);
    for (int p = 0; p < 2; p++) {
        for (int b = 0; b < NBINS; b++) ctx->prof.k[p][b] = KStat{};
        ctx->prof.pool[p] = KStat{};
    }
    for (int m = 0; m < 3; m++) ctx->prof.walk[m] = KStat{};
    for (int st = 0; st < Prof::NSTAGE; st++) ctx->prof.stage[st] = KStat{};
    return MP_OK;
}

extern "C" const char *mp_strerror(int code) {
    switch (code) {
        case MP_OK: return "ok";
        case MP_ERR_ARG: return "invalid argument";
        case MP_ERR_STATE: return "call not valid in this state";
        case MP_ERR_BUDGET: return "HBM budget exceeded";
        case MP_ERR_TOO_LARGE: return "result exceeds the size guard";
        case MP_ERR_OVERFLOW: return "path count exceeds 2^64-1";
        case MP_ERR_TIMEOUT: return "timed out";
        case MP_ERR_CUDA: return "CUDA error";
        case MP_ERR_NOMEM: return "out of memory";
        case MP_ERR_NOTFOUND: return "not found";
        case MP_ERR_INTERNAL: return "internal consistency check failed";
        default: return "unknown error";
    }
}
