// Overlap Tree (Sec. 3.3) and the cache replacement policies of Sec. 3.4 (Alg. 1).
//
// The tree is a generalised suffix tree over the workload's metapaths, built either by the
// naive insertion of Sec. 3.3.2 (for each query, the whole metapath and every proper
// suffix, each ended by the query's own terminator, is walked from the root; a walk that
// stops inside an edge splits it with a new internal node and the rest of the suffix
// becomes a new leaf) or on-line with Ukkonen's algorithm (the footnote of Sec. 3.3.2);
// both give the same tree. Each node on the path to a suffix's leaf counts one more
// occurrence (f), so f is the number of leaves below a node. Each node also keeps a constraints index (Sec. 3.3.4): per
// canonical constraint key of its positions, the entry (f, p, c, rho).
#include "otree.h"

#include <algorithm>
#include <cstdio>
#include <sstream>

namespace mp {

std::string window_key(const std::vector<std::string> &pos_keys, size_t start, size_t len) {
    std::string out;
    for (size_t i = start; i < start + len && i < pos_keys.size(); i++) {
        if (pos_keys[i].empty()) continue;
        if (!out.empty()) out += '|';
        out += std::to_string(i - start);
        out += ':';
        out += pos_keys[i];
    }
    return out;
}

std::string restrict_key(const std::string &key, size_t len) {
    if (key.empty()) return key;
    std::string out;
    size_t a = 0;
    while (a <= key.size()) {
        size_t b = key.find('|', a);
        if (b == std::string::npos) b = key.size();
        const std::string part = key.substr(a, b - a);
        const size_t colon = part.find(':');
        const size_t pos = (size_t)std::stoul(part.substr(0, colon));
        if (pos < len) {
            if (!out.empty()) out += '|';
            out += part;
        }
        a = b + 1;
    }
    return out;
}

// restrict_key(ekey, len) == pkey, without building the restricted key: the parts of ekey
// whose position is below len, joined by '|', must spell pkey exactly.
static bool restricted_equals(const std::string &ekey, size_t len, const std::string &pkey) {
    size_t a = 0, c = 0;  // cursors in ekey and pkey
    bool any = false;
    while (a < ekey.size()) {
        size_t b = ekey.find('|', a);
        if (b == std::string::npos) b = ekey.size();
        size_t pos = 0, d = a;
        while (d < b && ekey[d] >= '0' && ekey[d] <= '9') pos = pos * 10 + (size_t)(ekey[d++] - '0');
        if (pos < len) {
            if (any) {
                if (c >= pkey.size() || pkey[c] != '|') return false;
                c++;
            }
            if (pkey.compare(c, b - a, ekey, a, b - a) != 0) return false;
            c += b - a;
            any = true;
        }
        a = b + 1;
    }
    return c == pkey.size();
}

OverlapTree::OverlapTree(int construction) : construction_(construction == ONLINE ? ONLINE : NAIVE) {
    nodes_.emplace_back();
}

uint64_t OverlapTree::insert(const std::vector<int32_t> &types, const std::vector<std::string> &pos_keys) {
    const uint64_t q = queries_++;
    std::vector<int32_t> s(types);
    s.push_back(-(int32_t)(q + 1));
    const int32_t sid = (int32_t)strs_.size();
    strs_.push_back(std::move(s));
    if (construction_ == ONLINE) insert_online(sid, types.size(), pos_keys);
    else insert_naive(sid, types.size(), pos_keys);
    return q;
}

int32_t OverlapTree::new_leaf(int32_t parent, int32_t sid, int32_t lo) {
    Node leaf;
    leaf.parent = parent;
    leaf.sid = sid;
    leaf.lo = lo;
    leaf.hi = (int32_t)strs_[sid].size();
    leaf.depth = nodes_[parent].depth + (leaf.hi - lo);
    const int32_t id = (int32_t)nodes_.size();
    const int32_t first = strs_[sid][lo];
    nodes_.push_back(std::move(leaf));
    nodes_[parent].children[first] = id;
    leaves_++;
    return id;
}

int32_t OverlapTree::split(int32_t parent, int32_t child, size_t j) {
    Node mid;
    mid.parent = parent;
    mid.sid = nodes_[child].sid;
    mid.lo = nodes_[child].lo;
    mid.hi = nodes_[child].lo + (int32_t)j;
    mid.depth = nodes_[parent].depth + (int32_t)j;
    mid.f = nodes_[child].f;
    for (const auto &kv : nodes_[child].cidx) mid.cidx[restrict_key(kv.first, (size_t)mid.depth)].f += kv.second.f;
    const int32_t mid_id = (int32_t)nodes_.size();
    const int32_t first = sym(child, 0);
    nodes_.push_back(std::move(mid));
    Node &c = nodes_[child];
    c.lo += (int32_t)j;
    // a leaf that now hangs by its terminator alone: its string minus the terminator is
    // the new node's string, so its cache bookkeeping moves up
    if (c.hi - c.lo == 1 && strs_[c.sid][c.lo] < 0) {
        for (auto &kv : c.cidx) {
            OTEntry &m = nodes_[mid_id].cidx[kv.first];
            m.cached = kv.second.cached;
            m.c_ms = kv.second.c_ms;
            m.c_ops = kv.second.c_ops;
            m.nnz = kv.second.nnz;
            kv.second.cached = false;
        }
    }
    c.parent = mid_id;
    nodes_[mid_id].children[strs_[c.sid][c.lo]] = child;
    nodes_[parent].children[first] = mid_id;
    return mid_id;
}

void OverlapTree::count_up(int32_t leaf, size_t start, size_t n, const std::vector<std::string> &pos_keys) {
    for (int32_t x = leaf; x > 0; x = nodes_[x].parent) {
        Node &nd = nodes_[x];
        nd.f++;
        const size_t len = std::min((size_t)nd.depth, n - start);
        nd.cidx[window_key(pos_keys, start, len)].f++;
    }
}

// Sec. 3.3.2: each suffix (terminator included) walks from the root along the longest
// matching path; a walk that stops inside an edge splits it; the rest becomes a new leaf.
void OverlapTree::insert_naive(int32_t sid, size_t n, const std::vector<std::string> &pos_keys) {
    const std::vector<int32_t> &s = strs_[sid];
    const size_t m = s.size();
    for (size_t k = 0; k < n; k++) {
        int32_t node = 0;
        size_t i = k;
        int32_t leaf = -1;
        for (;;) {
            auto it = nodes_[node].children.find(s[i]);
            if (it == nodes_[node].children.end()) {
                leaf = new_leaf(node, sid, (int32_t)i);
                break;
            }
            const int32_t child = it->second;
            const size_t len = edge_len(child);
            size_t j = 0;
            while (j < len && i + j < m && sym(child, j) == s[i + j]) j++;
            if (j == len) {
                node = child;
                i += j;
                continue;
            }
            const int32_t mid = split(node, child, j);
            leaf = new_leaf(mid, sid, (int32_t)(i + j));
            break;
        }
        count_up(leaf, k, n, pos_keys);
    }
}

// Ukkonen's on-line construction, continued over the tree of the earlier metapaths (a
// generalised suffix tree: every earlier string ends with its own terminator, so all its
// suffixes are leaves already). One phase per symbol i extends every pending suffix by
// s[i]: the active point (node, edge, length) marks the longest pending suffix still
// implicit; an extension either finds s[i] already there (the phase ends), or adds a leaf
// at the active point, splitting an edge when the point is inside one; suffix links take
// the active point from one pending suffix to the next without walking from the root.
// Leaves of this metapath get their full label at once (they only ever grow to its end).
// The terminator phase makes every suffix a leaf; the suffix made of the terminator alone
// is not kept (the tree holds the metapath and its proper suffixes, Sec. 3.3.2).
void OverlapTree::insert_online(int32_t sid, size_t n, const std::vector<std::string> &pos_keys) {
    const std::vector<int32_t> &s = strs_[sid];
    const size_t m = s.size();
    std::vector<std::pair<int32_t, size_t>> made;  // (leaf, start of its suffix)
    int32_t an = 0;   // active node
    size_t ae = 0;    // active edge: index into s of its first symbol
    size_t al = 0;    // active length
    size_t rem = 0;   // suffixes still to be made explicit
    for (size_t i = 0; i < m; i++) {
        const int32_t c = s[i];
        rem++;
        int32_t need_link = -1;  // the internal node made last in this phase
        while (rem > 0) {
            if (al == 0) ae = i;
            auto it = nodes_[an].children.find(s[ae]);
            const size_t start = i + 1 - rem;
            if (it == nodes_[an].children.end()) {
                if (!(start == n && an == 0)) made.emplace_back(new_leaf(an, sid, (int32_t)i), start);
                if (need_link >= 0) nodes_[need_link].link = an;
                need_link = -1;
            } else {
                const int32_t nxt = it->second;
                const size_t el = edge_len(nxt);
                if (al >= el) {  // walk down to the next node
                    ae += el;
                    al -= el;
                    an = nxt;
                    continue;
                }
                if (sym(nxt, al) == c) {  // already there: this phase is done
                    if (need_link >= 0) nodes_[need_link].link = an;
                    al++;
                    break;
                }
                const int32_t mid = split(an, nxt, al);
                made.emplace_back(new_leaf(mid, sid, (int32_t)i), start);
                if (need_link >= 0) nodes_[need_link].link = mid;
                need_link = mid;
            }
            rem--;
            if (an == 0 && al > 0) {
                al--;
                ae = i + 1 - rem;
            } else if (an != 0) {
                an = nodes_[an].link;
            }
        }
    }
    for (const auto &lk : made) count_up(lk.first, lk.second, n, pos_keys);
}

int32_t OverlapTree::locate(const int32_t *s, size_t n, bool *exact) const {
    int32_t node = 0;
    size_t i = 0;
    *exact = true;
    while (i < n) {
        auto it = nodes_[node].children.find(s[i]);
        if (it == nodes_[node].children.end()) return -1;
        const int32_t child = it->second;
        const size_t len = edge_len(child);
        size_t j = 0;
        while (j < len && i + j < n) {
            if (sym(child, j) != s[i + j]) return -1;
            j++;
        }
        i += j;
        if (i == n) {
            *exact = j == len;
            return child;
        }
        node = child;
    }
    return node;
}

uint64_t OverlapTree::frequency(const int32_t *s, size_t n, const std::string *key) const {
    bool exact;
    const int32_t x = locate(s, n, &exact);
    if (x < 0) return 0;
    if (!key) return nodes_[x].f;
    // x's keys cover depth(x) positions: where the sub-metapath ends at x they are the
    // lookup keys themselves (one map lookup); inside the edge into x, restrict and count
    if (exact && (size_t)nodes_[x].depth == n) {
        auto it = nodes_[x].cidx.find(*key);
        return it == nodes_[x].cidx.end() ? 0 : it->second.f;
    }
    uint64_t f = 0;
    for (const auto &kv : nodes_[x].cidx)
        if (restricted_equals(kv.first, n, *key)) f += kv.second.f;
    return f;
}

OTEntry *OverlapTree::entry(const int32_t *s, size_t n, const std::string &key) {
    bool exact;
    const int32_t x = locate(s, n, &exact);
    if (x < 0) return nullptr;
    Node &nd = nodes_[x];
    const bool leaf_match = nd.children.empty() && nd.hi > nd.lo && strs_[nd.sid][nd.hi - 1] < 0 &&
                            (size_t)nd.depth == n + 1;
    if (!(exact && (size_t)nd.depth == n) && !leaf_match) return nullptr;
    auto it = nd.cidx.find(key);
    return it == nd.cidx.end() ? nullptr : &it->second;
}

bool OverlapTree::check(std::string *why) const {
    std::vector<uint64_t> below(nodes_.size(), 0);
    // children always have larger ids than their parent at creation, but splits insert a
    // parent after its child; accumulate leaf counts by walking each leaf up instead
    for (size_t x = 1; x < nodes_.size(); x++) {
        if (!nodes_[x].children.empty()) continue;
        for (int32_t y = (int32_t)x; y > 0; y = nodes_[y].parent) below[y]++;
    }
    for (size_t x = 1; x < nodes_.size(); x++) {
        const Node &nd = nodes_[x];
        if (nd.children.empty() && nd.f != 1) {
            if (why) *why = "leaf with f != 1";
            return false;
        }
        if (!nd.children.empty() && nd.children.size() < 2) {
            if (why) *why = "internal node with one child";
            return false;
        }
        if (nd.f != below[x]) {
            if (why) *why = "f differs from the leaves below";
            return false;
        }
    }
    return true;
}

// ------------------------------------------------------------------ cache policies

std::string CachePolicy::make_id(const std::vector<int32_t> &types, const std::string &key) {
    std::string id;
    for (int32_t t : types) {
        id += std::to_string(t);
        id += ',';
    }
    id += '#';
    id += key;
    return id;
}

bool CachePolicy::in_subtree(const CacheItem &p, const CacheItem &e) {
    if (p.types.size() >= e.types.size()) return false;
    if (!std::equal(p.types.begin(), p.types.end(), e.types.begin())) return false;
    return restricted_equals(e.key, p.types.size(), p.key);
}

// f(e) for every item e in p's subtree: only the ids that start with p's types (the range
// of the ordered map from p's type prefix) are candidates.
template <class F>
void CachePolicy::for_subtree(const CacheItem &p, F &&f) {
    std::string prefix;
    for (int32_t t : p.types) {
        prefix += std::to_string(t);
        prefix += ',';
    }
    for (auto it = items_.lower_bound(prefix); it != items_.end() && it->first.compare(0, prefix.size(), prefix) == 0;
         ++it)
        if (in_subtree(p, it->second)) f(it->second);
}

bool CachePolicy::evict_victim(CacheItem *out) {
    if (items_.empty()) return false;
    auto victim = items_.begin();
    for (auto it = items_.begin(); it != items_.end(); ++it) {
        const CacheItem &a = it->second, &b = victim->second;
        const bool better = policy_ == LRU ? a.seq < b.seq : (a.h < b.h || (a.h == b.h && a.seq < b.seq));
        if (better) victim = it;
    }
    CacheItem q = std::move(victim->second);
    items_.erase(victim);
    used_ -= q.s;
    if (policy_ != LRU) L_ = q.h;
    if (policy_ == ATRAPOS)
        for_subtree(q, [&](CacheItem &e) {
            e.c += q.c;
            util(e);
        });
    *out = std::move(q);
    return true;
}

CacheItem *CachePolicy::find(const std::string &id) {
    auto it = items_.find(id);
    return it == items_.end() ? nullptr : &it->second;
}

std::vector<CacheItem *> CachePolicy::items() {
    std::vector<CacheItem *> v;
    for (auto &kv : items_) v.push_back(&kv.second);
    return v;
}

void CachePolicy::clear() {
    items_.clear();
    used_ = 0.0;
}

CachePolicy::Outcome CachePolicy::request(const std::vector<int32_t> &types, const std::string &key, double f,
                                          double c, double s, std::shared_ptr<void> payload,
                                          std::vector<CacheItem> *evicted) {
    const std::string id = make_id(types, key);
    auto hit = items_.find(id);
    if (hit != items_.end()) {
        CacheItem &e = hit->second;
        e.f = f;
        e.l = L_;
        e.seq = ++seq_;
        util(e);
        return HIT;
    }
    if (s > max_fraction_ * capacity_) return REJECTED;
    while (used_ + s > capacity_ && !items_.empty()) {
        CacheItem q;
        evict_victim(&q);
        if (evicted) evicted->push_back(std::move(q));
    }
    CacheItem p;
    p.id = id;
    p.types = types;
    p.key = key;
    p.f = f;
    p.c = c;
    p.s = s;
    p.l = L_;
    p.seq = ++seq_;
    p.payload = std::move(payload);
    util(p);
    used_ += s;
    if (policy_ == ATRAPOS)
        for_subtree(p, [&](CacheItem &e) {
            e.c = std::max(0.0, e.c - p.c);
            util(e);
        });
    items_.emplace(id, std::move(p));
    return INSERTED;
}

}  // namespace mp
