// The context object behind the opaque mp_ctx handle of include/mp.h.
#pragma once
#include <cuda_runtime.h>

#include <memory>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/mp.h"
#include "internal.h"

struct mp_ctx {
    struct NodeType {
        std::string name;
        uint32_t count;
    };
    struct Prop {
        int32_t type = -1;
        std::string name;
        std::vector<int32_t> host;
        int32_t *dev = nullptr;
    };
    struct Rel {
        int32_t src = -1, dst = -1;
        std::vector<uint32_t> s, d;  // staged edges (forward relations only), dropped at finalize
        mp::Mat dev;                 // 0/1 CSR, val == nullptr
    };
    struct Constraint {
        int32_t prop = -1, op = 0;
        int64_t lo = 0, hi = 0;
        std::vector<uint32_t> set;
    };
    struct Query {
        std::vector<int32_t> types, rels;
        std::vector<std::vector<Constraint>> cons;  // per position
    };
    struct Result {
        int status = 0;
        mp::Mat m;
        double ms = 0.0;
        mp::Stats st;
        uint32_t n_products = 0;
    };
    struct Operand {
        mp::Mat m;
        bool owned = false;
    };

    mp_config cfg{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::mutex mu;
    std::vector<NodeType> types;
    std::vector<Prop> props;
    std::vector<Rel> rels;
    bool finalized = false;
    std::unordered_map<uint64_t, Result> results;
    uint64_t next_ticket = 1;
    std::unique_ptr<mp::Alloc> alloc;
    mp::Scratch scratch;
    mp::Tuning tun;
    mp::Prof prof;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;

    int parse(const mp_query *q, Query &out);
    int build_masks(const Query &q, std::vector<uint32_t *> &masks);
    void free_masks(std::vector<uint32_t *> &masks);
    int leaf_nnz(const Query &q, const std::vector<uint32_t *> &masks, std::vector<double> &nnz);
    int exec(const Query &q, const std::vector<uint32_t *> &masks, const std::vector<int> &split, int p,
             int i, int j, Operand &out, Result &r);
    int run_query(const Query &q, Result &r);
    int run_batch(std::vector<Query> &qs, std::vector<Result> &rs);
    void free_mat(mp::Mat &m);
    void release_result(Result &r);
    void cache_clear();
};
