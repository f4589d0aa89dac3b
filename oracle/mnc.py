"""MNC sketch estimator for the chain planner (test infrastructure).

Sec. 3.2 compares the average-case estimator E_ac with MNC (Sommer et al., "MNC:
Structure-Exploiting Sparsity Estimation for Matrix Expressions", SIGMOD 2019), which
estimates the size of a product from count sketches of its inputs instead of their
densities alone. The paper keeps E_ac because MNC costs more planning time for plans of
the same quality; this module is the plain definition the engine's MNC planner
(MP_PLAN_DP_MNC) is checked against.

Sketch of an m x n pattern matrix A (all counts over the non-zero pattern):
    hr[i]  = non-zeros in row i                 hc[k]  = non-zeros in column k
    her[i] = non-zeros of row i whose column    hec[k] = non-zeros of column k whose row
             holds a single non-zero                     holds a single non-zero
her / hec exist only for sketches built from an actual matrix ("exact" sketches).

Estimate of nnz(A B), A m x n with sketch a, B n x l with sketch b:
  1. max(a.hr) <= 1 or max(b.hc) <= 1: every output row (column) copies one row of B (one
     column of A), so no two products meet: nnz = sum_k a.hc[k] b.hr[k], exactly.
  2. both sketches exact: output entries in single-entry rows of A, and in single-entry
     columns of B, are counted exactly:
         E = sum_k a.hec[k] b.hr[k] + sum_k (a.hc[k] - a.hec[k]) b.her[k];
     the other products, (a.hc - a.hec)[k] x (b.hr - b.her)[k] per k, fall into the
     p = |{i: a.hr[i] >= 2}| * |{j: b.hc[j] >= 2}| remaining cells and are estimated by
     the density map below.
  3. otherwise p = |{i: a.hr[i] > 0}| * |{j: b.hc[j] > 0}| and all products go to the
     density map.
  Density map with p cells: inner index k contributes an outer-product block of
  c[k] r[k] cells, taken as uniform over the p cells, so a cell stays empty with
  probability prod_k (1 - c[k] r[k] / p) and the estimate is p (1 - that product).
  A factor below 0 (c[k] r[k] > p) counts as 0: the block covers every cell.

Propagation (the sketch of an estimated result C = A B with estimate s): rows keep A's
row shape, columns keep B's column shape, both scaled to sum to s:
  hr_C = a.hr * s / sum(a.hr),  hc_C = b.hc * s / sum(b.hc); no her / hec (not exact).
Counts stay real-valued (no rounding).

A sub-chain whose result is already known (cached, or evicted with a recorded cost)
enters the DP with its recorded cost and a uniform sketch of its exact size: every row
holds nnz/m and every column nnz/l.

The DP is Eq. 1 with the cost of Eq. 2, where nnz(X), nnz(Y) are the sizes the sketches
carry (exact for leaves, estimated otherwise) and nnz(Z) is the MNC estimate; the sketch
of each sub-chain comes from the split chosen for it, and ties go to the smallest split.
"""
from __future__ import annotations

import numpy as np

from . import planner as PL


class Sketch:
    __slots__ = ("hr", "hc", "her", "hec")

    def __init__(self, hr, hc, her=None, hec=None):
        self.hr = np.asarray(hr, np.float64)
        self.hc = np.asarray(hc, np.float64)
        self.her = None if her is None else np.asarray(her, np.float64)
        self.hec = None if hec is None else np.asarray(hec, np.float64)

    @property
    def exact(self):
        return self.her is not None and self.hec is not None

    @property
    def nnz(self):
        return float(self.hr.sum())


def sketch_of_dense(A) -> Sketch:
    """Exact sketch of a dense 0/1 (or non-negative) matrix, straight from the definition."""
    P = np.asarray(A) != 0
    hr = P.sum(1)
    hc = P.sum(0)
    her = (P & (hc == 1)[None, :]).sum(1)
    hec = (P & (hr == 1)[:, None]).sum(0)
    return Sketch(hr, hc, her, hec)


def sketch_of_csr(rp, ci, ncols) -> Sketch:
    """Exact sketch of a CSR pattern (rp row pointers, ci column ids)."""
    rp = np.asarray(rp, np.int64)
    ci = np.asarray(ci, np.int64)
    m = len(rp) - 1
    hr = np.diff(rp)
    hc = np.bincount(ci, minlength=int(ncols))
    rows = np.repeat(np.arange(m), hr)
    her = np.bincount(rows, weights=(hc[ci] == 1).astype(np.float64), minlength=m)
    hec = np.bincount(ci, weights=(hr[rows] == 1).astype(np.float64), minlength=int(ncols))
    return Sketch(hr, hc, her, hec)


def uniform_sketch(m, l, nnz) -> Sketch:
    """Sketch of a known result of which only the size is used."""
    return Sketch(np.full(int(m), nnz / m if m else 0.0), np.full(int(l), nnz / l if l else 0.0))


def density_map(c, r, p) -> float:
    """p cells, inner index k covering a uniform block of c[k] r[k] cells."""
    if p <= 0:
        return 0.0
    f = 1.0 - np.asarray(c, np.float64) * np.asarray(r, np.float64) / p
    return float(p * (1.0 - np.prod(np.clip(f, 0.0, None))))


def estimate(a: Sketch, b: Sketch) -> float:
    """MNC estimate of nnz(A B)."""
    if a.hr.size == 0 or b.hc.size == 0:
        return 0.0
    if a.hr.max() <= 1.0 or b.hc.max() <= 1.0:
        return float((a.hc * b.hr).sum())
    if a.exact and b.exact:
        known = float((a.hec * b.hr).sum() + ((a.hc - a.hec) * b.her).sum())
        p = float((a.hr >= 2).sum()) * float((b.hc >= 2).sum())
        return known + density_map(a.hc - a.hec, b.hr - b.her, p)
    p = float((a.hr > 0).sum()) * float((b.hc > 0).sum())
    return density_map(a.hc, b.hr, p)


def propagate(a: Sketch, b: Sketch, s: float) -> Sketch:
    na, nb = a.nnz, b.nnz
    hr = a.hr * (s / na) if na > 0 else np.zeros_like(a.hr)
    hc = b.hc * (s / nb) if nb > 0 else np.zeros_like(b.hc)
    return Sketch(hr, hc)


def mnc_plan(dims, leaves, alpha=1.0, beta=1.0, gamma=1.0, known=None, totals=None):
    """Eq. 1 over sketches. dims[t], dims[t+1]: sizes of factor t; leaves[t]: its exact
    Sketch; known maps (i, j) -> (cost, nnz) for sub-chains whose result is known.
    Returns (cost, tree, C, N, S): cost, estimated nnz and split matrices. A dict passed
    as totals receives the total cost of every candidate split, keyed (i, j, k)."""
    p = len(dims) - 1
    known = known or {}
    INF = float("inf")
    C = [[0.0] * p for _ in range(p)]
    N = [[0.0] * p for _ in range(p)]
    S = [[-1] * p for _ in range(p)]
    K = [[None] * p for _ in range(p)]
    for i in range(p):
        K[i][i] = leaves[i]
        N[i][i] = leaves[i].nnz
    for length in range(2, p + 1):
        for i in range(0, p - length + 1):
            j = i + length - 1
            m, l = dims[i], dims[j + 1]
            if (i, j) in known:
                c, z = known[(i, j)]
                C[i][j], N[i][j] = float(c), float(z)
                K[i][j] = uniform_sketch(m, l, float(z))
                continue
            best, best_k, best_z = INF, -1, 0.0
            for k in range(i, j):
                n = dims[k + 1]
                x, y = K[i][k], K[k + 1][j]
                z = estimate(x, y)
                rx = x.nnz / (float(m) * n)
                ry = y.nnz / (float(n) * l)
                rz = z / (float(m) * l)
                total = C[i][k] + C[k + 1][j] + PL.sparse_cost(m, n, l, rx, ry, rz, alpha, beta, gamma)
                if totals is not None:
                    totals[(i, j, k)] = total
                if total < best:
                    best, best_k, best_z = total, k, z
            C[i][j], N[i][j], S[i][j] = best, best_z, best_k
            K[i][j] = propagate(K[i][best_k], K[best_k + 1][j], best_z)
    return C[0][p - 1], PL.plan_tree(S, 0, p - 1), C, N, S
