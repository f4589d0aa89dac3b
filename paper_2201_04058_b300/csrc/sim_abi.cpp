// Host-only C entry points over the Overlap Tree and the cache policies, for replaying
// workload traces without a GPU (and for testing them against the CPU oracle).
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mp.h"
#include "otree.h"

struct mp_otree {
    mp::OverlapTree t;
    explicit mp_otree(int construction) : t(construction) {}
};

struct mp_cachesim {
    mp::CachePolicy c;
    std::vector<std::string> evicted;
    mp_cachesim(double cap, int pol) : c(cap, pol) {}
};

extern "C" int mp_otree_create(mp_otree **out) { return mp_otree_create_ex(MP_OTREE_NAIVE, out); }

extern "C" int mp_otree_create_ex(int32_t construction, mp_otree **out) {
    if (!out || (construction != MP_OTREE_NAIVE && construction != MP_OTREE_ONLINE)) return MP_ERR_ARG;
    *out = new mp_otree(construction == MP_OTREE_ONLINE ? mp::OverlapTree::ONLINE : mp::OverlapTree::NAIVE);
    return MP_OK;
}

extern "C" void mp_otree_destroy(mp_otree *t) { delete t; }

extern "C" int mp_otree_insert(mp_otree *t, uint32_t n, const int32_t *types, const char *const *pos_keys) {
    if (!t || !n || !types) return MP_ERR_ARG;
    std::vector<int32_t> ty(types, types + n);
    for (int32_t x : ty)
        if (x < 0) return MP_ERR_ARG;
    std::vector<std::string> keys(n);
    if (pos_keys)
        for (uint32_t i = 0; i < n; i++) keys[i] = pos_keys[i] ? pos_keys[i] : "";
    t->t.insert(ty, keys);
    return MP_OK;
}

extern "C" int mp_otree_frequency(mp_otree *t, uint32_t n, const int32_t *s, const char *key, uint64_t *f) {
    if (!t || !s || !f) return MP_ERR_ARG;
    std::string k = key ? key : "";
    *f = t->t.frequency(s, n, key ? &k : nullptr);
    return MP_OK;
}

extern "C" int mp_otree_info(mp_otree *t, uint64_t *nodes, uint64_t *leaves, int32_t *invariants_ok) {
    if (!t) return MP_ERR_ARG;
    if (nodes) *nodes = t->t.n_nodes();
    if (leaves) *leaves = t->t.n_leaves();
    if (invariants_ok) *invariants_ok = t->t.check(nullptr) ? 1 : 0;
    return MP_OK;
}

extern "C" int mp_cachesim_create(double capacity, int32_t policy, mp_cachesim **out) {
    if (!out || !(capacity > 0) || policy < MP_POLICY_ATRAPOS || policy > MP_POLICY_LRU) return MP_ERR_ARG;
    *out = new mp_cachesim(capacity, policy);
    return MP_OK;
}

extern "C" void mp_cachesim_destroy(mp_cachesim *c) { delete c; }

extern "C" int mp_cachesim_request(mp_cachesim *c, uint32_t n, const int32_t *types, const char *key, double f,
                                   double cost, double size, int32_t *outcome) {
    if (!c || !n || !types || !(size > 0)) return MP_ERR_ARG;
    std::vector<int32_t> ty(types, types + n);
    std::vector<mp::CacheItem> ev;
    auto r = c->c.request(ty, key ? key : "", f, cost, size, nullptr, &ev);
    for (auto &e : ev) c->evicted.push_back(e.id);
    if (outcome) *outcome = (int32_t)r;
    return MP_OK;
}

extern "C" int mp_cachesim_entry(mp_cachesim *c, uint32_t n, const int32_t *types, const char *key, double *cost,
                                 double *utility, int32_t *present) {
    if (!c || !types) return MP_ERR_ARG;
    std::vector<int32_t> ty(types, types + n);
    mp::CacheItem *e = c->c.find(mp::CachePolicy::make_id(ty, key ? key : ""));
    if (present) *present = e ? 1 : 0;
    if (e && cost) *cost = e->c;
    if (e && utility) *utility = e->h;
    return MP_OK;
}

extern "C" int mp_cachesim_evicted(mp_cachesim *c, uint32_t i, char *buf, uint32_t cap, uint32_t *n_total) {
    if (!c) return MP_ERR_ARG;
    if (n_total) *n_total = (uint32_t)c->evicted.size();
    if (buf && cap) {
        if (i >= c->evicted.size()) return MP_ERR_NOTFOUND;
        strncpy(buf, c->evicted[i].c_str(), cap - 1);
        buf[cap - 1] = 0;
    }
    return MP_OK;
}

extern "C" int mp_cachesim_state(mp_cachesim *c, double *L, double *used, uint32_t *items) {
    if (!c) return MP_ERR_ARG;
    if (L) *L = c->c.L();
    if (used) *used = c->c.used();
    if (items) *items = (uint32_t)c->c.size();
    return MP_OK;
}
