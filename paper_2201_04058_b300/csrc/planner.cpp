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
#include <cmath>
#include <limits>
#include <vector>

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
