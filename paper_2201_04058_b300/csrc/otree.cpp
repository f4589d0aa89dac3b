// Overlap Tree (Sec. 3.3) and the cache replacement policies of Sec. 3.4 (Alg. 1).
//
// The tree is a generalised suffix tree over the workload's metapaths built by the naive
// insertion of Sec. 3.3.2: for each query, the whole metapath and every proper suffix,
// each ended by the query's own terminator, is walked from the root; a walk that stops
// inside an edge splits it with a new internal node and the rest of the suffix becomes a
// new leaf. Each node on the walk counts one more occurrence (f), so f is the number of
// leaves below a node. Each node also keeps a constraints index (Sec. 3.3.4): per
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

OverlapTree::OverlapTree() { nodes_.emplace_back(); }

uint64_t OverlapTree::insert(const std::vector<int32_t> &types, const std::vector<std::string> &pos_keys) {
    const uint64_t q = queries_++;
    std::vector<int32_t> s(types);
    s.push_back(-(int32_t)(q + 1));
    const size_t n = types.size();
    for (size_t k = 0; k < n; k++) {
        std::vector<int32_t> suf(s.begin() + k, s.end());
        insert_suffix(suf, k, n, pos_keys);
    }
    return q;
}

void OverlapTree::insert_suffix(const std::vector<int32_t> &suf, size_t start, size_t n,
                                const std::vector<std::string> &pos_keys) {
    int32_t node = 0;
    size_t i = 0;
    std::vector<int32_t> path;
    for (;;) {
        auto it = nodes_[node].children.find(suf[i]);
        if (it == nodes_[node].children.end()) {
            Node leaf;
            leaf.parent = node;
            leaf.label.assign(suf.begin() + i, suf.end());
            leaf.depth = nodes_[node].depth + (int32_t)(suf.size() - i);
            const int32_t id = (int32_t)nodes_.size();
            nodes_.push_back(std::move(leaf));
            nodes_[node].children[suf[i]] = id;
            leaves_++;
            path.push_back(id);
            break;
        }
        const int32_t child = it->second;
        const std::vector<int32_t> &lab = nodes_[child].label;
        size_t j = 0;
        while (j < lab.size() && i + j < suf.size() && lab[j] == suf[i + j]) j++;
        if (j == lab.size()) {
            node = child;
            i += j;
            path.push_back(child);
            continue;
        }
        // split the edge into `child` after j symbols
        Node mid;
        mid.parent = node;
        mid.label.assign(lab.begin(), lab.begin() + j);
        mid.depth = nodes_[node].depth + (int32_t)j;
        mid.f = nodes_[child].f;
        for (const auto &kv : nodes_[child].cidx) mid.cidx[restrict_key(kv.first, (size_t)mid.depth)].f += kv.second.f;
        const int32_t mid_id = (int32_t)nodes_.size();
        nodes_.push_back(std::move(mid));
        Node &c = nodes_[child];
        std::vector<int32_t> rest(c.label.begin() + j, c.label.end());
        // a leaf that now hangs by its terminator alone: its string minus the terminator
        // is the new node's string, so its cache bookkeeping moves up
        if (rest.size() == 1 && rest[0] < 0) {
            for (auto &kv : c.cidx) {
                OTEntry &m = nodes_[mid_id].cidx[kv.first];
                m.cached = kv.second.cached;
                m.c_ms = kv.second.c_ms;
                m.c_ops = kv.second.c_ops;
                m.nnz = kv.second.nnz;
                kv.second.cached = false;
            }
        }
        c.label = rest;
        c.parent = mid_id;
        nodes_[mid_id].children[rest[0]] = child;
        nodes_[node].children[suf[i]] = mid_id;
        Node leaf;
        leaf.parent = mid_id;
        leaf.label.assign(suf.begin() + i + j, suf.end());
        leaf.depth = nodes_[mid_id].depth + (int32_t)(suf.size() - i - j);
        const int32_t leaf_id = (int32_t)nodes_.size();
        const int32_t first = leaf.label[0];
        nodes_.push_back(std::move(leaf));
        nodes_[mid_id].children[first] = leaf_id;
        leaves_++;
        path.push_back(mid_id);
        path.push_back(leaf_id);
        break;
    }
    for (int32_t x : path) {
        Node &nd = nodes_[x];
        nd.f++;
        const size_t len = std::min((size_t)nd.depth, n - start);
        nd.cidx[window_key(pos_keys, start, len)].f++;
    }
}

int32_t OverlapTree::locate(const int32_t *s, size_t n, bool *exact) const {
    int32_t node = 0;
    size_t i = 0;
    *exact = true;
    while (i < n) {
        auto it = nodes_[node].children.find(s[i]);
        if (it == nodes_[node].children.end()) return -1;
        const int32_t child = it->second;
        const std::vector<int32_t> &lab = nodes_[child].label;
        size_t j = 0;
        while (j < lab.size() && i + j < n) {
            if (lab[j] != s[i + j]) return -1;
            j++;
        }
        i += j;
        if (i == n) {
            *exact = j == lab.size();
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
    // every occurrence through x carries a key of at least n positions: restrict and count
    uint64_t f = 0;
    for (const auto &kv : nodes_[x].cidx)
        if (restrict_key(kv.first, n) == *key) f += kv.second.f;
    return f;
}

OTEntry *OverlapTree::entry(const int32_t *s, size_t n, const std::string &key) {
    bool exact;
    const int32_t x = locate(s, n, &exact);
    if (x < 0) return nullptr;
    Node &nd = nodes_[x];
    const bool leaf_match = nd.children.empty() && !nd.label.empty() && nd.label.back() < 0 &&
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
    return restrict_key(e.key, p.types.size()) == p.key;
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
            for (auto &kv : items_)
                if (in_subtree(q, kv.second)) {
                    kv.second.c += q.c;
                    util(kv.second);
                }
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
        for (auto &kv : items_)
            if (in_subtree(p, kv.second)) {
                kv.second.c = std::max(0.0, kv.second.c - p.c);
                util(kv.second);
            }
    items_.emplace(id, std::move(p));
    return INSERTED;
}

}  // namespace mp
