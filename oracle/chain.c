/*
 * CPU oracle for the metapath chain product (test infrastructure only).
 *
 * This file is part of the test oracle: only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it. The product path never calls it.
 *
 * What it computes is the plain definition of the metapath query result (Sec. 2,
 * Problem 1 and the constrained adjacency M_c * A that follows it):
 *
 *     A_m = M_1 * A_1 * M_2 * A_2 * ... * A_{n-1} * M_n
 *
 * over the non-negative integers, where A_t is the 0/1 adjacency of the relation between
 * positions t and t+1 (Def. 1) and M_t is the 0/1 diagonal of the nodes that satisfy the
 * constraints at position t (Def. 3). A_m[u][v] counts the instances of the metapath
 * from u to v (Def. 2). Every entry is kept as an exact uint64; an addition or
 * multiplication that would not fit is reported as ORC_OVERFLOW, never wrapped.
 *
 * The method is Gustavson's row-by-row product with a dense accumulator as wide as the
 * output's column count. The order is fixed left to right. Output is canonical CSR:
 * int64 row pointers (empty rows kept), int32 column ids strictly ascending per row,
 * uint64 values >= 1, no stored zeros.
 *
 * Single-threaded and deliberately unoptimised.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_NOMEM (-2)
#define ORC_OVERFLOW (-5)

typedef struct {
    int64_t nrows, ncols;
    const int64_t *rp;   /* nrows+1 */
    const int32_t *ci;   /* rp[nrows] */
    const uint64_t *val; /* NULL: every stored entry is 1 (a 0/1 adjacency) */
} orc_csr;

typedef struct {
    int64_t *rp;
    int32_t *ci;
    uint64_t *val;
    int64_t nnz, cap;
} orc_out;

static int out_push(orc_out *o, int32_t j, uint64_t v) {
    if (o->nnz == o->cap) {
        int64_t cap = o->cap ? o->cap * 2 : 1024;
        int32_t *ci = (int32_t *)realloc(o->ci, (size_t)cap * sizeof(int32_t));
        if (!ci) return ORC_NOMEM;
        o->ci = ci;
        uint64_t *val = (uint64_t *)realloc(o->val, (size_t)cap * sizeof(uint64_t));
        if (!val) return ORC_NOMEM;
        o->val = val;
        o->cap = cap;
    }
    o->ci[o->nnz] = j;
    o->val[o->nnz] = v;
    o->nnz++;
    return ORC_OK;
}

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

void orc_free(void *p) { free(p); }

/*
 * C = diag(rmask) * X * diag(kmask) * Y * diag(cmask); any mask may be NULL (identity).
 * Results are returned in malloc'd arrays the caller releases with orc_free.
 */
int orc_spgemm(const orc_csr *X, const orc_csr *Y, const uint8_t *rmask, const uint8_t *kmask,
               const uint8_t *cmask, int64_t **rp_out, int32_t **ci_out, uint64_t **val_out,
               int64_t *nnz_out) {
    int64_t m = X->nrows, l = Y->ncols;
    uint64_t *acc = (uint64_t *)calloc((size_t)(l > 0 ? l : 1), sizeof(uint64_t));
    uint8_t *seen = (uint8_t *)calloc((size_t)(l > 0 ? l : 1), 1);
    int32_t *touched = (int32_t *)malloc((size_t)(l > 0 ? l : 1) * sizeof(int32_t));
    orc_out o = {0};
    o.rp = (int64_t *)malloc((size_t)(m + 1) * sizeof(int64_t));
    int rc = ORC_OK;
    if (!acc || !seen || !touched || !o.rp) { rc = ORC_NOMEM; goto done; }
    o.rp[0] = 0;
    for (int64_t i = 0; i < m; i++) {
        int64_t nt = 0;
        if (!rmask || rmask[i]) {
            for (int64_t p = X->rp[i]; p < X->rp[i + 1]; p++) {
                int32_t k = X->ci[p];
                if (kmask && !kmask[k]) continue;
                uint64_t a = X->val ? X->val[p] : 1u;
                for (int64_t q = Y->rp[k]; q < Y->rp[k + 1]; q++) {
                    int32_t j = Y->ci[q];
                    if (cmask && !cmask[j]) continue;
                    uint64_t b = Y->val ? Y->val[q] : 1u;
                    uint64_t ab, s;
                    if (__builtin_mul_overflow(a, b, &ab)) { rc = ORC_OVERFLOW; goto done; }
                    if (__builtin_add_overflow(acc[j], ab, &s)) { rc = ORC_OVERFLOW; goto done; }
                    acc[j] = s;
                    if (!seen[j]) { seen[j] = 1; touched[nt++] = j; }
                }
            }
        }
        qsort(touched, (size_t)nt, sizeof(int32_t), cmp_i32);
        for (int64_t t = 0; t < nt; t++) {
            int32_t j = touched[t];
            if (acc[j] > 0 && (rc = out_push(&o, j, acc[j])) != ORC_OK) goto done;
            acc[j] = 0;
            seen[j] = 0;
        }
        o.rp[i + 1] = o.nnz;
    }
done:
    free(acc);
    free(seen);
    free(touched);
    if (rc != ORC_OK) {
        free(o.rp);
        free(o.ci);
        free(o.val);
        return rc;
    }
    *rp_out = o.rp;
    *ci_out = o.ci;
    *val_out = o.val;
    *nnz_out = o.nnz;
    return ORC_OK;
}

/*
 * The whole chain M_1 A_1 M_2 ... A_{nf} M_{nf+1}, left to right. factors[t] maps
 * position t to position t+1; masks has nf+1 entries (NULL = no constraint).
 */
int orc_chain(int nf, const orc_csr *factors, const uint8_t *const *masks, int64_t **rp_out,
              int32_t **ci_out, uint64_t **val_out, int64_t *nnz_out) {
    if (nf < 1) return -1;
    /* R = M_1 * A_1 * M_2, the first constrained factor */
    const orc_csr *A = &factors[0];
    orc_out o = {0};
    o.rp = (int64_t *)malloc((size_t)(A->nrows + 1) * sizeof(int64_t));
    if (!o.rp) return ORC_NOMEM;
    o.rp[0] = 0;
    for (int64_t i = 0; i < A->nrows; i++) {
        if (!masks[0] || masks[0][i]) {
            for (int64_t p = A->rp[i]; p < A->rp[i + 1]; p++) {
                int32_t j = A->ci[p];
                if (masks[1] && !masks[1][j]) continue;
                uint64_t v = A->val ? A->val[p] : 1u;
                if (v > 0 && out_push(&o, j, v) != ORC_OK) {
                    free(o.rp); free(o.ci); free(o.val);
                    return ORC_NOMEM;
                }
            }
        }
        o.rp[i + 1] = o.nnz;
    }
    orc_csr R = {A->nrows, A->ncols, o.rp, o.ci, o.val};
    for (int t = 1; t < nf; t++) {
        int64_t *rp; int32_t *ci; uint64_t *val; int64_t nnz;
        /* R <- R * diag(M_{t+1}) * A_{t+1} * diag(M_{t+2}) (1-based positions) */
        int rc = orc_spgemm(&R, &factors[t], NULL, masks[t], masks[t + 1], &rp, &ci, &val, &nnz);
        free((void *)R.rp); free((void *)R.ci); free((void *)R.val);
        if (rc != ORC_OK) return rc;
        R.nrows = factors[0].nrows; R.ncols = factors[t].ncols;
        R.rp = rp; R.ci = ci; R.val = val;
    }
    *rp_out = (int64_t *)R.rp;
    *ci_out = (int32_t *)R.ci;
    *val_out = (uint64_t *)R.val;
    *nnz_out = R.rp[R.nrows];
    return ORC_OK;
}

/*
 * Row sums of A_m without forming it: r = M_1 A_1 M_2 ... A_{nf} M_{nf+1} * 1, evaluated
 * right to left as a chain of sparse matrix-vector products in O(sum nnz). Each partial sum is
 * checked in 128-bit arithmetic; a sum beyond 2^64-1 returns ORC_OVERFLOW.
 * out has factors[0].nrows entries.
 */
int orc_rowsum(int nf, const orc_csr *factors, const uint8_t *const *masks, uint64_t *out) {
    int64_t n_last = factors[nf - 1].ncols;
    uint64_t *v = (uint64_t *)malloc((size_t)(n_last > 0 ? n_last : 1) * sizeof(uint64_t));
    if (!v) return ORC_NOMEM;
    for (int64_t j = 0; j < n_last; j++) v[j] = (!masks[nf] || masks[nf][j]) ? 1u : 0u;
    for (int t = nf - 1; t >= 0; t--) {
        const orc_csr *A = &factors[t];
        uint64_t *w = (uint64_t *)malloc((size_t)(A->nrows > 0 ? A->nrows : 1) * sizeof(uint64_t));
        if (!w) { free(v); return ORC_NOMEM; }
        for (int64_t i = 0; i < A->nrows; i++) {
            unsigned __int128 s = 0;
            if (!masks[t] || masks[t][i]) {
                for (int64_t p = A->rp[i]; p < A->rp[i + 1]; p++) {
                    unsigned __int128 a = A->val ? A->val[p] : 1u;
                    s += a * v[A->ci[p]];
                    if (s >> 64) { free(w); free(v); return ORC_OVERFLOW; }
                }
            }
            w[i] = (uint64_t)s;
        }
        free(v);
        v = w;
    }
    memcpy(out, v, (size_t)factors[0].nrows * sizeof(uint64_t));
    free(v);
    return ORC_OK;
}

/*
 * Column sums of A_m: c = 1^T M_1 A_1 M_2 ... A_{nf} M_{nf+1}, left to right.
 * out has factors[nf-1].ncols entries.
 */
int orc_colsum(int nf, const orc_csr *factors, const uint8_t *const *masks, uint64_t *out) {
    int64_t n0 = factors[0].nrows;
    uint64_t *v = (uint64_t *)malloc((size_t)(n0 > 0 ? n0 : 1) * sizeof(uint64_t));
    if (!v) return ORC_NOMEM;
    for (int64_t i = 0; i < n0; i++) v[i] = (!masks[0] || masks[0][i]) ? 1u : 0u;
    for (int t = 0; t < nf; t++) {
        const orc_csr *A = &factors[t];
        unsigned __int128 *w = (unsigned __int128 *)calloc((size_t)(A->ncols > 0 ? A->ncols : 1),
                                                           sizeof(unsigned __int128));
        if (!w) { free(v); return ORC_NOMEM; }
        for (int64_t i = 0; i < A->nrows; i++) {
            if (!v[i]) continue;
            for (int64_t p = A->rp[i]; p < A->rp[i + 1]; p++) {
                unsigned __int128 a = A->val ? A->val[p] : 1u;
                w[A->ci[p]] += a * v[i];
            }
        }
        free(v);
        v = (uint64_t *)malloc((size_t)(A->ncols > 0 ? A->ncols : 1) * sizeof(uint64_t));
        if (!v) { free(w); return ORC_NOMEM; }
        for (int64_t j = 0; j < A->ncols; j++) {
            v[j] = 0u;
            if (masks[t + 1] && !masks[t + 1][j]) continue;
            if (w[j] >> 64) { free(w); free(v); return ORC_OVERFLOW; }
            v[j] = (uint64_t)w[j];
        }
        free(w);
    }
    memcpy(out, v, (size_t)factors[nf - 1].ncols * sizeof(uint64_t));
    free(v);
    return ORC_OK;
}
