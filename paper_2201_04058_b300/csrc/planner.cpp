// Chain-order planner: the matrix-chain dynamic program of Sec. 3.1 (Eq. 1) with the
// sparse product cost of Sec. 3.2 (Eq. 2) and the average-case density estimator E_ac.
//
//   C[i][j] = min_{i <= k < j} C[i][k] + C[k+1][j] + c(A_{i..k} * A_{k+1..j})
//   c(X*Y)  = alpha*nnz(X) + beta*N_op + gamma*nnz(Z)          (Eq. 2)
//   nnz(X) = m*n*rho_X, N_op = m*n*rho_X*l*rho_Y, nnz(Z) = m*l*rho_Z,
//   rho_Z  = 1 - (1 - rho_X*rho_Y)^n                            (E_ac)
//
// D[i][j] keeps the density estimate of each sub-chain (from the split chosen for it).
// Sub-chains whose result is already known (in the cache, or evicted with a recorded
// cost) use that cost and exact density instead of the estimate (end of Sec. 3.2).
// Ties keep the smallest split k. p is at most a few dozen, so O(p^3) is negligible.
// A measured density of a sub-chain's result (rho_fixed, from sampled rows) replaces E_ac
// for that sub-chain; its cost still follows Eq. 2.
#include <algorithm>
#include <cmath>
#include <limits>
#include <vector>

#include "mp.h"

#include "internal.h"

namespace mp {

void plan_chain(int p, const double *dims, const double *nnz, double alpha, double beta,
                double gamma, const double *known_cost, const double *known_rho, const double *rho_fixed,
                int *split, double *cost_out, double *rho_out) {
    std::vector<double> C((size_t)p * p, 0.0), D((size_t)p * p, 0.0);
    auto at = [p](int i, int j) { return (size_t)i * p + j; };
    for (int i = 0; i < p; i++) {
        D[at(i, i)] = nnz[i] / (dims[i] * dims[i + 1]);
        split[at(i, i)] = -1;
    }
    for (int len = 2; len <= p; len++) {
        for (int i = 0; i + len - 1 < p; i++) {
            const int j = i + len - 1;
            if (known_cost && !std::isnan(known_cost[at(i, j)])) {
                C[at(i, j)] = known_cost[at(i, j)];
                D[at(i, j)] = known_rho[at(i, j)];
                split[at(i, j)] = -1;
                continue;
            }
            double best = std::numeric_limits<double>::infinity(), best_rho = 0.0;
            int best_k = -1;
            const double m = dims[i], l = dims[j + 1];
            for (int k = i; k < j; k++) {
                const double n = dims[k + 1];
                const double rx = D[at(i, k)], ry = D[at(k + 1, j)];
                const double fixed = rho_fixed ? rho_fixed[at(i, j)] : NAN;
                const double rz = std::isnan(fixed) ? 1.0 - std::pow(1.0 - rx * ry, n) : fixed;
                const double nnz_x = m * n * rx;
                const double n_op = m * n * rx * l * ry;
                const double nnz_z = m * l * rz;
                const double cost = alpha * nnz_x + beta * n_op + gamma * nnz_z;
                const double total = C[at(i, k)] + C[at(k + 1, j)] + cost;
                if (total < best) {
                    best = total;
                    best_k = k;
                    best_rho = rz;
                }
            }
            C[at(i, j)] = best;
            D[at(i, j)] = best_rho;
            split[at(i, j)] = best_k;
        }
    }
    if (cost_out)
        for (size_t t = 0; t < C.size(); t++) cost_out[t] = C[t];
    if (rho_out)
        for (size_t t = 0; t < D.size(); t++) rho_out[t] = D[t];
}

}  // namespace mp

namespace mp {

MncPlan::MncPlan(int p_, const double *dims, const MncLeaf *leaves, const MncPair *pairs, double alpha, double beta,
                 double gamma, const double *known_cost, const double *known_nnz)
    : p(p_), leaves_(leaves), pairs_(pairs), alpha_(alpha), beta_(beta), gamma_(gamma), known_cost_(known_cost),
      known_nnz_(known_nnz) {
    dims_.assign(dims, dims + p + 1);
    split.assign((size_t)p * p, -1);
    cost.assign((size_t)p * p, 0.0);
    nnz.assign((size_t)p * p, 0.0);
    sk_.assign((size_t)p * p, Sk{0.0, -1, -1, 0.0, 0.0, false});
    for (int i = 0; i < p; i++) {
        sk_[at(i, i)] = Sk{leaves[i].nnz, i, i, 1.0, 1.0, true};
        nnz[at(i, i)] = leaves[i].nnz;
    }
}

// The MNC cases, in order: (1) rows of X or columns of Y hold at most one entry: the
// product count is the size; (2) both operands are leaves: exact parts from the extension
// counts plus the density map over the remaining cells; (3) the density map over the
// non-empty rows of X times the non-empty columns of Y.
void MncPlan::requests(int len, std::vector<MncReq> &out) {
    cand_.assign((size_t)(p - len + 1), std::vector<Cand>());
    for (int i = 0; i + len - 1 < p; i++) {
        const int j = i + len - 1;
        if (known_cost_ && !std::isnan(known_cost_[at(i, j)])) continue;
        const double m = dims_[i], l = dims_[j + 1];
        for (int k = i; k < j; k++) {
            const Sk &X = sk_[at(i, k)], &Y = sk_[at(k + 1, j)];
            const double n = dims_[k + 1];
            Cand c{k, -1, 0.0, 0.0, 0.0};
            const double maxr = X.ra >= 0 ? X.fr * leaves_[X.ra].maxr : X.fr;
            const double maxc = Y.ca >= 0 ? Y.fc * leaves_[Y.ca].maxc : Y.fc;
            const double f = X.fc * Y.fr;
            if (m <= 0 || l <= 0) {
                c.est_fixed = 0.0;
            } else if (maxr <= 1.0 || maxc <= 1.0) {
                const double d = (X.ca >= 0 && Y.ra >= 0) ? pairs_[k].dot
                                 : X.ca >= 0             ? leaves_[k].nnz
                                 : Y.ra >= 0             ? leaves_[k + 1].nnz
                                                         : n;
                c.est_fixed = f * d;
            } else if (X.exact && Y.exact) {
                const double p2 = leaves_[k].r2 * leaves_[k + 1].c2;
                c.est_fixed = pairs_[k].known + (p2 > 0 ? p2 * (1.0 - std::exp(pairs_[k].ls_ext)) : 0.0);
            } else {
                const double nzr = X.fr > 0 ? (X.ra >= 0 ? leaves_[X.ra].nzr : m) : 0.0;
                const double nzc = Y.fc > 0 ? (Y.ca >= 0 ? leaves_[Y.ca].nzc : l) : 0.0;
                const double p3 = nzr * nzc;
                if (p3 > 0) {
                    const double x = f / p3;
                    c.p3 = p3;
                    if (X.ca >= 0 || Y.ra >= 0) {
                        const int kind = (X.ca >= 0 && Y.ra >= 0) ? MNC_W_PAIR : X.ca >= 0 ? MNC_W_COL : MNC_W_ROW;
                        c.need = (int)out.size();
                        out.push_back(MncReq{k, kind, x});
                    } else {
                        c.need = -2;
                        c.ls_const = x >= 1.0 ? -std::numeric_limits<double>::infinity() : n * std::log1p(-x);
                    }
                }
            }
            cand_[i].push_back(c);
        }
    }
}

void MncPlan::resolve(int len, const double *ls) {
    for (int i = 0; i + len - 1 < p; i++) {
        const int j = i + len - 1;
        const double m = dims_[i], l = dims_[j + 1];
        if (known_cost_ && !std::isnan(known_cost_[at(i, j)])) {
            const double z = known_nnz_[at(i, j)];
            cost[at(i, j)] = known_cost_[at(i, j)];
            nnz[at(i, j)] = z;
            split[at(i, j)] = -1;
            sk_[at(i, j)] = Sk{z, -1, -1, m > 0 ? z / m : 0.0, l > 0 ? z / l : 0.0, false};
            continue;
        }
        double best = std::numeric_limits<double>::infinity(), best_z = 0.0;
        int best_k = -1;
        for (const Cand &c : cand_[i]) {
            const int k = c.k;
            const double n = dims_[k + 1];
            const Sk &X = sk_[at(i, k)], &Y = sk_[at(k + 1, j)];
            double z = c.est_fixed;
            if (c.need >= 0) z = c.p3 * (1.0 - std::exp(ls[c.need]));
            else if (c.need == -2) z = c.p3 * (1.0 - std::exp(c.ls_const));
            const double rx = X.nnz / (m * n), ry = Y.nnz / (n * l), rz = z / (m * l);
            const double step = alpha_ * m * n * rx + beta_ * m * n * rx * l * ry + gamma_ * m * l * rz;
            const double total = cost[at(i, k)] + cost[at(k + 1, j)] + step;
            if (total < best) {
                best = total;
                best_k = k;
                best_z = z;
            }
        }
        cost[at(i, j)] = best;
        nnz[at(i, j)] = best_z;
        split[at(i, j)] = best_k;
        const Sk &X = sk_[at(i, best_k)], &Y = sk_[at(best_k + 1, j)];
        sk_[at(i, j)] = Sk{best_z, X.ra, Y.ca, X.nnz > 0 ? X.fr * best_z / X.nnz : 0.0,
                           Y.nnz > 0 ? Y.fc * best_z / Y.nnz : 0.0, false};
    }
}

}  // namespace mp

// ------------------------------------------------------------------ host-only MNC planner

namespace {

double ls_host(const uint32_t *a, const uint32_t *a2, const uint32_t *b, const uint32_t *b2, int64_t n, double x) {
    double s = 0.0;
    for (int64_t t = 0; t < n; t++) {
        const double w = (a ? (double)a[t] - (a2 ? (double)a2[t] : 0.0) : 1.0) *
                         (b ? (double)b[t] - (b2 ? (double)b2[t] : 0.0) : 1.0);
        if (w <= 0) continue;
        if (x * w >= 1.0) return -std::numeric_limits<double>::infinity();
        s += std::log1p(-x * w);
    }
    return s;
}

}  // namespace

extern "C" int mp_plan_chain_mnc(uint32_t p, const double *dims, const uint32_t *const *hr,
                                 const uint32_t *const *hc, const uint32_t *const *her,
                                 const uint32_t *const *hec, double alpha, double beta, double gamma,
                                 const double *known_cost, const double *known_nnz, int32_t *split, double *cost,
                                 double *nnz) {
    if (!p || !dims || !hr || !hc || !her || !hec || !split) return MP_ERR_ARG;
    if ((known_cost == nullptr) != (known_nnz == nullptr)) return MP_ERR_ARG;
    std::vector<mp::MncLeaf> leaves(p);
    for (uint32_t t = 0; t < p; t++) {
        if (!hr[t] || !hc[t] || !her[t] || !hec[t]) return MP_ERR_ARG;
        mp::MncLeaf &L = leaves[t];
        L = mp::MncLeaf{0, 0, 0, 0, 0, 0, 0};
        for (int64_t i = 0; i < (int64_t)dims[t]; i++) {
            L.nnz += hr[t][i];
            L.nzr += hr[t][i] > 0;
            L.maxr = std::max(L.maxr, (double)hr[t][i]);
            L.r2 += hr[t][i] >= 2;
        }
        for (int64_t j = 0; j < (int64_t)dims[t + 1]; j++) {
            L.nzc += hc[t][j] > 0;
            L.maxc = std::max(L.maxc, (double)hc[t][j]);
            L.c2 += hc[t][j] >= 2;
        }
    }
    std::vector<mp::MncPair> pairs(p);
    for (uint32_t k = 0; k + 1 < p; k++) {
        const int64_t n = (int64_t)dims[k + 1];
        mp::MncPair &P = pairs[k];
        P = mp::MncPair{0, 0, 0};
        for (int64_t t = 0; t < n; t++) {
            P.dot += (double)hc[k][t] * hr[k + 1][t];
            P.known += (double)hec[k][t] * hr[k + 1][t] + ((double)hc[k][t] - hec[k][t]) * her[k + 1][t];
        }
        const double p2 = leaves[k].r2 * leaves[k + 1].c2;
        P.ls_ext = p2 > 0 ? ls_host(hc[k], hec[k], hr[k + 1], her[k + 1], n, 1.0 / p2) : 0.0;
    }
    mp::MncPlan plan((int)p, dims, leaves.data(), pairs.data(), alpha, beta, gamma, known_cost, known_nnz);
    for (uint32_t len = 2; len <= p; len++) {
        std::vector<mp::MncReq> req;
        plan.requests((int)len, req);
        std::vector<double> ls(req.size());
        for (size_t r = 0; r < req.size(); r++) {
            const int k = req[r].pair;
            const int64_t n = (int64_t)dims[k + 1];
            const uint32_t *a = req[r].kind != mp::MNC_W_ROW ? hc[k] : nullptr;
            const uint32_t *b = req[r].kind != mp::MNC_W_COL ? hr[k + 1] : nullptr;
            ls[r] = ls_host(a, nullptr, b, nullptr, n, req[r].x);
        }
        plan.resolve((int)len, ls.data());
    }
    for (size_t t = 0; t < (size_t)p * p; t++) {
        split[t] = plan.split[t];
        if (cost) cost[t] = plan.cost[t];
        if (nnz) nnz[t] = plan.nnz[t];
    }
    return MP_OK;
}
