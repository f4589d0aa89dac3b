"""Chain-order planning for the oracle (test infrastructure).

Sec. 3.1, Eq. 1: for a chain A_i ... A_j the optimal cost is
    C[i][j] = min_{i <= k < j} C[i][k] + C[k+1][j] + c(A_{i..k} * A_{k+1..j}),
with C[i][i] = 0, a p x p matrix filled by increasing chain length. With the dense cost of
Sec. 3.1 a product of an (m x n) and an (n x l) matrix costs m*n*l operations.

Sec. 3.2, Eq. 2: for sparse X (m x n, density rho_X) and Y (n x l, density rho_Y),
    c(X*Y) ~ alpha*nnz(X) + beta*N_op + gamma*nnz(Z),
    nnz(X) = m*n*rho_X,  N_op = m*n*rho_X*l*rho_Y,  nnz(Z) = m*l*rho_Z,
and rho_Z comes from the average-case estimator E_ac, rho_Z = 1 - (1 - rho_X*rho_Y)^n.
A second p x p matrix D holds the estimated density of every sub-chain, taken from the
split the recursion selects. Sub-chains whose result is known (cached, or evicted with a
recorded cost) replace the estimate: a cached result costs its retrieval (0 here) and has
its exact density; an evicted one costs its recorded recomputation time (end of Sec. 3.2).

Ties go to the smallest split k (the first minimum met when k increases).

Sampled densities (the engine's MP_PLAN_DP_SAMPLED): the exact output size of seeded
sampled rows of a sub-chain, scaled to all its rows, replaces E_ac for that sub-chain's
result density; the DP is otherwise unchanged.
"""
from __future__ import annotations

import itertools


def eac_density(rho_x: float, rho_y: float, n: int) -> float:
    """E_ac: the chance that an entry of Z = X*Y is non-zero when the non-zeros of X
    and Y are uniform: each of the n inner terms is non-zero with prob rho_x*rho_y."""
    return 1.0 - (1.0 - rho_x * rho_y) ** n


def sparse_cost(m, n, l, rho_x, rho_y, rho_z, alpha, beta, gamma):
    """Eq. 2."""
    nnz_x = m * n * rho_x
    n_op = m * n * rho_x * l * rho_y
    nnz_z = m * l * rho_z
    return alpha * nnz_x + beta * n_op + gamma * nnz_z


def chain_dp(dims, leaf_density, product, known=None, rho_fixed=None):
    """Eq. 1. dims[t], dims[t+1] are the sizes of factor t (p = len(dims)-1 factors);
    leaf_density[t] its density; product(m, n, l, rho_x, rho_y) -> (cost, rho_z).
    known maps (i, j) -> (cost, density) for sub-chains whose result is already known.
    rho_fixed maps (i, j) -> a measured density of that sub-chain's result (for example
    from sampled rows): the product cost still follows the cost model, but with this
    density for the result in place of the estimate.
    Returns (C, D, S): cost, density and split matrices (S[i][j] = k, or -1 for leaves and
    known sub-chains)."""
    p = len(dims) - 1
    known = known or {}
    rho_fixed = rho_fixed or {}
    INF = float("inf")
    C = [[0.0] * p for _ in range(p)]
    D = [[0.0] * p for _ in range(p)]
    S = [[-1] * p for _ in range(p)]
    for i in range(p):
        D[i][i] = float(leaf_density[i])
    for length in range(2, p + 1):
        for i in range(0, p - length + 1):
            j = i + length - 1
            if (i, j) in known:
                C[i][j], D[i][j] = (float(x) for x in known[(i, j)])
                continue
            best, best_k, best_rho = INF, -1, 0.0
            for k in range(i, j):
                cost, rho = product(dims[i], dims[k + 1], dims[j + 1], D[i][k], D[k + 1][j],
                                    rho_fixed.get((i, j)))
                total = C[i][k] + C[k + 1][j] + cost
                if total < best:
                    best, best_k, best_rho = total, k, rho
            C[i][j], D[i][j], S[i][j] = best, best_rho, best_k
    return C, D, S


def dense_product(m, n, l, rho_x, rho_y, rho_z=None):
    """Sec. 3.1: m*n*l operations; the dense result has density 1."""
    return float(m) * n * l, 1.0


def sparse_product(alpha=1.0, beta=1.0, gamma=1.0):
    def product(m, n, l, rho_x, rho_y, rho_z=None):
        if rho_z is None:
            rho_z = eac_density(rho_x, rho_y, n)
        return sparse_cost(m, n, l, rho_x, rho_y, rho_z, alpha, beta, gamma), rho_z

    return product


def plan_tree(S, i, j):
    """Nested-tuple parenthesisation of factors i..j from the split matrix."""
    if i == j or S[i][j] < 0:
        return i if i == j else (i, j, "known")
    k = S[i][j]
    return (plan_tree(S, i, k), plan_tree(S, k + 1, j))


def dense_plan(dims):
    C, D, S = chain_dp(dims, [1.0] * (len(dims) - 1), dense_product)
    return C[0][-1], plan_tree(S, 0, len(dims) - 2)


def sparse_plan(dims, nnz, alpha=1.0, beta=1.0, gamma=1.0, known=None, rho_fixed=None):
    """Plan for factors with sizes dims and nnz counts; returns (cost, tree, C, D, S)."""
    p = len(dims) - 1
    rho = [nnz[t] / (float(dims[t]) * dims[t + 1]) for t in range(p)]
    C, D, S = chain_dp(dims, rho, sparse_product(alpha, beta, gamma), known, rho_fixed)
    return C[0][p - 1], plan_tree(S, 0, p - 1), C, D, S


def sampled_density(sample_nnz, n_sampled, n_active, n_rows, n_cols):
    """Density of a product estimated from the exact nnz of n_sampled rows drawn among its
    n_active non-empty rows (the other rows of its n_rows are empty)."""
    if n_sampled == 0 or n_rows == 0 or n_cols == 0:
        return 0.0
    return (sample_nnz / float(n_sampled)) * n_active / (float(n_rows) * n_cols)


def all_trees(i, j):
    """Every parenthesisation of factors i..j (Catalan many)."""
    if i == j:
        yield i
        return
    for k in range(i, j):
        for left, right in itertools.product(list(all_trees(i, k)), list(all_trees(k + 1, j))):
            yield (left, right)
