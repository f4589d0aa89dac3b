// Overlap Tree (Sec. 3.3) and cache replacement policies (Sec. 3.4, Alg. 1): host side.
#pragma once
#include <cstdint>
#include <map>
#include <memory>
#include <string>
#include <unordered_map>
#include <vector>

namespace mp {

// Canonical constraint key of the window [start, start+len) of a metapath, renumbered
// from 0: "i:<desc>" for every position i with a non-empty description, '|'-joined.
std::string window_key(const std::vector<std::string> &pos_keys, size_t start, size_t len);
// A key restricted to its first `len` positions.
std::string restrict_key(const std::string &key, size_t len);

// (f, p, c, rho) of one sub-metapath under one constraint key (Sec. 3.3.1, 3.3.4).
struct OTEntry {
    uint64_t f = 0;
    bool cached = false;      // p != null
    double c_ms = -1.0;       // recorded cost (device ms) of computing it
    double c_ops = -1.0;      // Eq. 2 with the actual counts of that computation
    double nnz = -1.0;        // recorded nnz of its result (the rho of the paper)
};

// Generalised suffix tree over metapaths; symbols are node type ids (>= 0), the
// terminator of query q is -(q+1). Every node on the path from the root to a suffix's
// leaf counts one occurrence of that suffix. Two constructions give the same tree:
//   NAIVE   the suffix-by-suffix walk of Sec. 3.3.2 (each suffix from the root);
//   ONLINE  Ukkonen's on-line construction (the faster approach the footnote of Sec.
//           3.3.2 points to): one left-to-right pass over the metapath with an active
//           point and suffix links, so the walks that reach known prefixes are skipped.
// A tree keeps one construction for its life (the on-line one needs the suffix links of
// every internal node, which the naive walk does not set).
class OverlapTree {
  public:
    enum Construction { NAIVE = 0, ONLINE = 1 };
    explicit OverlapTree(int construction = NAIVE);
    int construction() const { return construction_; }
    // Insert a metapath with one constraint description per position ("" = none).
    uint64_t insert(const std::vector<int32_t> &types, const std::vector<std::string> &pos_keys);
    // Occurrences of s among inserted metapaths; with key, only those whose
    // constraints on s's positions equal key.
    uint64_t frequency(const int32_t *s, size_t n, const std::string *key) const;
    // Entry of sub-metapath s under key, kept on the node whose string is s (or on the
    // leaf whose string is s plus a terminator). nullptr when s has no node.
    OTEntry *entry(const int32_t *s, size_t n, const std::string &key);
    size_t n_nodes() const { return nodes_.size() - 1; }  // without the root
    size_t n_leaves() const { return leaves_; }
    size_t n_queries() const { return queries_; }
    // Sec. 3.3.3 invariants: every internal non-root node has >= 2 children; leaves have
    // f = 1; every node's f is the number of leaves below it.
    bool check(std::string *why) const;

  private:
    struct Node {
        int32_t parent = -1;
        int32_t sid = -1, lo = 0, hi = 0;  // edge label: strs_[sid][lo, hi)
        int32_t link = 0;                  // suffix link (ONLINE; internal nodes)
        std::unordered_map<int32_t, int32_t> children;
        uint64_t f = 0;
        int32_t depth = 0;
        std::unordered_map<std::string, OTEntry> cidx;
    };
    int construction_;
    std::vector<Node> nodes_;
    std::vector<std::vector<int32_t>> strs_;  // every inserted metapath with its terminator
    size_t leaves_ = 0;
    uint64_t queries_ = 0;
    int32_t sym(int32_t x, size_t j) const { return strs_[nodes_[x].sid][nodes_[x].lo + j]; }
    size_t edge_len(int32_t x) const { return (size_t)(nodes_[x].hi - nodes_[x].lo); }
    int32_t new_leaf(int32_t parent, int32_t sid, int32_t lo);
    // cut the edge into `child` after j symbols with a new node; returns it
    int32_t split(int32_t parent, int32_t child, size_t j);
    // one occurrence of the suffix starting at `start` on the leaf and every ancestor
    void count_up(int32_t leaf, size_t start, size_t n, const std::vector<std::string> &pos_keys);
    void insert_naive(int32_t sid, size_t n, const std::vector<std::string> &pos_keys);
    void insert_online(int32_t sid, size_t n, const std::vector<std::string> &pos_keys);
    // node at or just below the end of s, and whether s ends exactly there; -1 if absent
    int32_t locate(const int32_t *s, size_t n, bool *exact) const;
};

// One cached item of the replacement policy.
struct CacheItem {
    std::string id;                 // types + key
    std::vector<int32_t> types;
    std::string key;
    double f = 0, c = 0, s = 0, h = 0, l = 0;
    uint64_t seq = 0;
    std::shared_ptr<void> payload;  // device result (engine) or nothing (host simulation)
};

// ATRAPOS-OTree (Alg. 1), PGDS or LRU over a byte capacity; items above max_fraction of
// the capacity are never admitted (Sec. 4.1.4).
class CachePolicy {
  public:
    enum { ATRAPOS = 0, PGDS = 1, LRU = 2 };
    enum Outcome { HIT = 0, INSERTED = 1, REJECTED = 2 };
    CachePolicy(double capacity, int policy, double max_fraction = 0.8)
        : capacity_(capacity), policy_(policy), max_fraction_(max_fraction) {}
    // A request of item (types, key) with tree frequency f, cost c and size s. evicted
    // receives the ids evicted to make room, in order.
    Outcome request(const std::vector<int32_t> &types, const std::string &key, double f, double c, double s,
                    std::shared_ptr<void> payload, std::vector<CacheItem> *evicted);
    CacheItem *find(const std::string &id);
    // Evict the policy's victim (as a request that needs room would), into *out; false
    // when the cache is empty. Used when queries need the bytes the cache holds.
    bool evict_victim(CacheItem *out);
    static std::string make_id(const std::vector<int32_t> &types, const std::string &key);
    double used() const { return used_; }
    double capacity() const { return capacity_; }
    double L() const { return L_; }
    size_t size() const { return items_.size(); }
    std::vector<CacheItem *> items();
    void clear();

  private:
    double capacity_;
    int policy_;
    double max_fraction_;
    double L_ = 0.0, used_ = 0.0;
    uint64_t seq_ = 0;
    // ordered by id, which starts with the item's types: the items whose metapath extends a
    // given one are one contiguous range (the Overlap-Tree subtree walks visit only it)
    std::map<std::string, CacheItem> items_;
    static bool in_subtree(const CacheItem &parent, const CacheItem &child);
    template <class F>
    void for_subtree(const CacheItem &parent, F &&f);
    void util(CacheItem &e) const { e.h = e.f * e.c / e.s + e.l; }
};

}  // namespace mp
