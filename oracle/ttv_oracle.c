/*
 * ttv_oracle.c -- plain, slow, single-threaded CPU statement of the sparse
 * tensor-times-vector product (TTV).  TEST INFRASTRUCTURE ONLY: the tests,
 * the smoke check and the benchmark's CPU-baseline leg call it; the CUDA
 * library never does, and the two share no code.
 *
 * What it computes (paper Sec. 3.3, Eq. 3, with the multi-vector form of the
 * paragraph before Eq. 3): a d-way sparse tensor A with nonzeros
 * (subs[k, 0..d-1], vals[k]) is multiplied by n_v vectors x_m, one per mode m
 * in the set S of contracted modes, |x_m| = shape[m].  The result has order
 * d - n_v and the surviving modes R = [0, d) \ S in increasing order:
 *
 *     B(i_R) = sum over k with subs[k, R] == i_R of  vals[k] * prod_{m in S} x_m[subs[k, m]]
 *
 * The steps follow the paper's description of pyttb's sptensor.ttv (Sec. 3.3):
 * the surviving dimensions are the set difference of all modes and the
 * contracted ones, rows of subs[:, R] are grouped by distinct value ("unique",
 * which returns them in ascending lexicographic order) and the scaled values
 * are summed per group ("accumarray").  Indices here are 0-based (the paper
 * counts from 1).
 *
 * Readings where the paper says nothing:
 *   - every distinct surviving tuple that occurs in the input is an output
 *     entry, even when its sum is zero (presence is structural);
 *   - duplicate input subscripts are summed like any other group member;
 *   - the product is formed in increasing mode order, in IEEE binary64;
 *   - each group is summed in input order with Neumaier's compensated
 *     summation (A. Neumaier, ZAMM 54, 1974), so the oracle's own error is a
 *     few units in the last place of the exact group sum of the rounded terms;
 *     when the running sum is not finite the plain IEEE sum is the result
 *     (the correction term would turn a lone infinity into a NaN);
 *   - n_v == d gives an order-0 result: one scalar, the multilinear form.
 *
 * Build with -ffp-contract=off: a fused multiply-add would change the rounding
 * of the products and defeat the compensation.
 *
 * Parity pins (tests, -m "not gpu"): brute-force dense contraction in exact
 * rational arithmetic, d = 1 (dot product, Eq. 1) and d = 2 (matrix-vector
 * product, Eq. 2) special cases, all-ones vector = mode sum, linearity, the
 * all-modes multilinear form, mode-order independence, distinct-tuple counts.
 * The dense dot and matrix-vector statements at the end are pinned to exact
 * rational sums, closed forms, the d = 1 and d = 2 TTV bit for bit, and
 * storage-order independence.
 */
#define _GNU_SOURCE
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define ORACLE_MAX_D 16

enum {
    ORACLE_OK = 0,
    ORACLE_ERR_ARG = -1,
    ORACLE_ERR_MODE = -2,
    ORACLE_ERR_VEC_LEN = -3,
    ORACLE_ERR_SUBSCRIPT = -4,
    ORACLE_ERR_NOMEM = -5,
};

typedef struct {
    int32_t order;                   /* d - n_v                                   */
    int64_t shape[ORACLE_MAX_D];     /* shape[R]                                  */
    int64_t nnz;                     /* output entries (prod(shape) when dense)   */
    int64_t *subs;                   /* nnz x order, row-major; NULL when dense   */
    double *vals;                    /* nnz values                                */
} oracle_out;

/* Context for the comparator: the surviving modes and the row-major subs. */
typedef struct {
    const int64_t *subs;
    int32_t d;
    int32_t nr;
    int32_t r[ORACLE_MAX_D];
} group_ctx;

/* Lexicographic order of subs[k, R]; ties keep input order (k ascending). */
static int cmp_rows(const void *pa, const void *pb, void *pctx)
{
    const group_ctx *c = (const group_ctx *)pctx;
    int64_t ka = *(const int64_t *)pa, kb = *(const int64_t *)pb;
    for (int32_t j = 0; j < c->nr; ++j) {
        int64_t a = c->subs[ka * c->d + c->r[j]];
        int64_t b = c->subs[kb * c->d + c->r[j]];
        if (a < b) return -1;
        if (a > b) return 1;
    }
    return (ka > kb) - (ka < kb);
}

static int same_row(const group_ctx *c, int64_t ka, int64_t kb)
{
    for (int32_t j = 0; j < c->nr; ++j)
        if (c->subs[ka * c->d + c->r[j]] != c->subs[kb * c->d + c->r[j]]) return 0;
    return 1;
}

void oracle_free(oracle_out *out)
{
    if (!out) return;
    free(out->subs);
    free(out->vals);
    out->subs = NULL;
    out->vals = NULL;
    out->nnz = 0;
}

/*
 * subs      nnz x d int64, row-major (C order), 0-based
 * vals      nnz doubles
 * modes     n_v distinct contracted modes, any order
 * vec_lens  n_v lengths; vec_lens[i] must equal shape[modes[i]]
 * vecs      n_v pointers to the vectors
 * dense     0: sparse COO result; 1: dense row-major array of prod(shape[R])
 * Returns ORACLE_OK or a negative ORACLE_ERR_*; out is filled only on success.
 */
int oracle_ttv(int32_t d, const int64_t *shape, int64_t nnz,
               const int64_t *subs, const double *vals,
               int32_t n_v, const int32_t *modes, const int64_t *vec_lens,
               const double *const *vecs, int32_t dense, oracle_out *out)
{
    if (!out || !shape || d < 1 || d > ORACLE_MAX_D || nnz < 0) return ORACLE_ERR_ARG;
    if (n_v < 1 || n_v > d || !modes || !vec_lens || !vecs) return ORACLE_ERR_ARG;
    if (nnz > 0 && (!subs || !vals)) return ORACLE_ERR_ARG;
    memset(out, 0, sizeof(*out));
    for (int32_t m = 0; m < d; ++m)
        if (shape[m] < 1) return ORACLE_ERR_ARG;

    /* S: which modes carry a vector, and that vector; R = the rest, ascending. */
    const double *vec_of_mode[ORACLE_MAX_D];
    int32_t in_s[ORACLE_MAX_D];
    for (int32_t m = 0; m < d; ++m) { in_s[m] = 0; vec_of_mode[m] = NULL; }
    for (int32_t i = 0; i < n_v; ++i) {
        int32_t m = modes[i];
        if (m < 0 || m >= d || in_s[m]) return ORACLE_ERR_MODE;
        if (vec_lens[i] != shape[m]) return ORACLE_ERR_VEC_LEN;
        if (!vecs[i]) return ORACLE_ERR_ARG;
        in_s[m] = 1;
        vec_of_mode[m] = vecs[i];
    }
    group_ctx ctx;
    ctx.subs = subs;
    ctx.d = d;
    ctx.nr = 0;
    for (int32_t m = 0; m < d; ++m)
        if (!in_s[m]) ctx.r[ctx.nr++] = m;

    for (int64_t k = 0; k < nnz; ++k)
        for (int32_t m = 0; m < d; ++m)
            if (subs[k * d + m] < 0 || subs[k * d + m] >= shape[m]) return ORACLE_ERR_SUBSCRIPT;

    out->order = ctx.nr;
    for (int32_t j = 0; j < ctx.nr; ++j) out->shape[j] = shape[ctx.r[j]];

    /* Step 1: the scaled value of every nonzero, product in increasing mode order. */
    double *t = (double *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(double));
    int64_t *idx = (int64_t *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int64_t));
    if (!t || !idx) { free(t); free(idx); return ORACLE_ERR_NOMEM; }
    for (int64_t k = 0; k < nnz; ++k) {
        double p = vals[k];
        for (int32_t m = 0; m < d; ++m)
            if (in_s[m]) p = p * vec_of_mode[m][subs[k * d + m]];
        t[k] = p;
        idx[k] = k;
    }

    /* Step 2: order the nonzeros by their surviving tuple ("unique" rows). */
    if (nnz > 1) qsort_r(idx, (size_t)nnz, sizeof(int64_t), cmp_rows, &ctx);

    /* Step 3: one output entry per distinct tuple; Neumaier sum in input order. */
    int64_t groups = 0;
    for (int64_t i = 0; i < nnz; ++i)
        if (i == 0 || !same_row(&ctx, idx[i - 1], idx[i])) ++groups;

    int64_t *gsubs = (int64_t *)malloc((size_t)(groups > 0 ? groups : 1) * (size_t)(ctx.nr > 0 ? ctx.nr : 1) * sizeof(int64_t));
    double *gvals = (double *)malloc((size_t)(groups > 0 ? groups : 1) * sizeof(double));
    if (!gsubs || !gvals) { free(t); free(idx); free(gsubs); free(gvals); return ORACLE_ERR_NOMEM; }

    int64_t g = -1;
    double sum = 0.0, comp = 0.0;
    for (int64_t i = 0; i < nnz; ++i) {
        int64_t k = idx[i];
        if (i == 0 || !same_row(&ctx, idx[i - 1], k)) {
            if (g >= 0) gvals[g] = isfinite(sum) ? sum + comp : sum;
            ++g;
            for (int32_t j = 0; j < ctx.nr; ++j) gsubs[g * ctx.nr + j] = subs[k * d + ctx.r[j]];
            sum = 0.0;
            comp = 0.0;
        }
        double s = sum + t[k];
        if (fabs(sum) >= fabs(t[k])) comp += (sum - s) + t[k];
        else                         comp += (t[k] - s) + sum;
        sum = s;
    }
    if (g >= 0) gvals[g] = isfinite(sum) ? sum + comp : sum;
    free(t);
    free(idx);

    if (!dense) {
        if (ctx.nr == 0 && groups == 0) {
            /* order-0 result of an empty tensor: the scalar 0 */
            out->nnz = 1;
            out->subs = gsubs;
            gvals[0] = 0.0;
            out->vals = gvals;
            return ORACLE_OK;
        }
        out->nnz = groups;
        out->subs = gsubs;
        out->vals = gvals;
        return ORACLE_OK;
    }

    /* Dense result: zero array of prod(shape[R]), row-major over R. */
    int64_t cells = 1;
    for (int32_t j = 0; j < ctx.nr; ++j) cells *= out->shape[j];
    double *dv = (double *)calloc((size_t)cells, sizeof(double));
    if (!dv) { free(gsubs); free(gvals); return ORACLE_ERR_NOMEM; }
    for (int64_t q = 0; q < groups; ++q) {
        int64_t lin = 0;
        for (int32_t j = 0; j < ctx.nr; ++j) lin = lin * out->shape[j] + gsubs[q * ctx.nr + j];
        dv[lin] = gvals[q];
    }
    free(gsubs);
    free(gvals);
    out->nnz = cells;
    out->subs = NULL;
    out->vals = dv;
    return ORACLE_OK;
}

/*
 * Matricized tensor times Khatri-Rao product (MTTKRP) along mode `mode`.
 * The paper names it as the kernel built on the sparse TTV (Sec. 3.3) and as
 * future work (Sec. 5) without writing it out; this is the standard
 * definition.  With factor matrices A_m (shape[m] x rank, row-major) for
 * every m != mode:
 *
 *     M(i, r) = sum over k with subs[k, mode] == i of
 *               vals[k] * prod_{m != mode, increasing} A_m(subs[k, m], r)
 *
 * so column r of M is the all-but-one TTV (Eq. 3 with n_v = d - 1) of the
 * tensor with the vectors A_m(:, r), m != mode.  Each (i, r) is summed in
 * input order with Neumaier's compensated summation, like the TTV groups
 * above, and rows i that no nonzero touches are 0.
 *
 * factors   d pointers; factors[mode] is not read
 * out       shape[mode] x rank doubles, row-major (written in full)
 * Returns ORACLE_OK or a negative ORACLE_ERR_*.
 */
int oracle_mttkrp(int32_t d, const int64_t *shape, int64_t nnz, const int64_t *subs, const double *vals,
                  int32_t mode, int32_t rank, const double *const *factors, double *out)
{
    if (!shape || d < 1 || d > ORACLE_MAX_D || nnz < 0 || rank < 1 || !factors || !out) return ORACLE_ERR_ARG;
    if (mode < 0 || mode >= d) return ORACLE_ERR_MODE;
    if (nnz > 0 && (!subs || !vals)) return ORACLE_ERR_ARG;
    for (int32_t m = 0; m < d; ++m) {
        if (shape[m] < 1) return ORACLE_ERR_ARG;
        if (m != mode && !factors[m]) return ORACLE_ERR_ARG;
    }
    for (int64_t k = 0; k < nnz; ++k)
        for (int32_t m = 0; m < d; ++m)
            if (subs[k * d + m] < 0 || subs[k * d + m] >= shape[m]) return ORACLE_ERR_SUBSCRIPT;

    const int64_t rows = shape[mode];
    double *comp = (double *)calloc((size_t)rows * (size_t)rank, sizeof(double));
    if (!comp) return ORACLE_ERR_NOMEM;
    for (int64_t q = 0; q < rows * rank; ++q) out[q] = 0.0;

    /* input order: every (i, r) sum receives its terms in increasing k */
    for (int64_t k = 0; k < nnz; ++k) {
        const int64_t i = subs[k * d + mode];
        for (int32_t r = 0; r < rank; ++r) {
            double t = vals[k];
            for (int32_t m = 0; m < d; ++m)
                if (m != mode) t = t * factors[m][subs[k * d + m] * rank + r];
            double *sum = &out[i * rank + r];
            double *c = &comp[i * rank + r];
            const double s = *sum + t;
            if (fabs(*sum) >= fabs(t)) *c += (*sum - s) + t;
            else                       *c += (t - s) + *sum;
            *sum = s;
        }
    }
    for (int64_t q = 0; q < rows * rank; ++q)
        if (isfinite(out[q])) out[q] += comp[q];
    free(comp);
    return ORACLE_OK;
}

/*
 * Dense vector dot product (paper Sec. 3.1, Eq. 1) and dense matrix-vector
 * product (paper Sec. 3.2, Eq. 2), the paper's two simple kernels, by their
 * plain definitions:
 *
 *     x . y = sum_{i=0}^{n-1} x[i] * y[i]
 *     y[i]  = sum_{j=0}^{n2-1} A(i, j) * x[j],   i = 0 .. n1-1
 *
 * Each product is rounded to binary64, and each sum runs over increasing i
 * (dot) or j (matrix row) with Neumaier's compensated summation, as the TTV
 * groups above; a non-finite running sum is returned as the plain IEEE sum.
 * A(i, j) is A[i * stride_row + j * stride_col], so row-major ("C") storage
 * has strides (n2, 1) and pyttb's column-major ("F") storage (1, n1).
 */
static double neumaier_sum_products(const double *a, int64_t sa, const double *b, int64_t n)
{
    double sum = 0.0, comp = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        const double t = a[i * sa] * b[i];
        const double s = sum + t;
        if (fabs(sum) >= fabs(t)) comp += (sum - s) + t;
        else                      comp += (t - s) + sum;
        sum = s;
    }
    return isfinite(sum) ? sum + comp : sum;
}

int oracle_dot(int64_t n, const double *x, const double *y, double *out)
{
    if (n < 0 || !out || (n > 0 && (!x || !y))) return ORACLE_ERR_ARG;
    *out = neumaier_sum_products(x, 1, y, n);
    return ORACLE_OK;
}

int oracle_matvec(int64_t n1, int64_t n2, const double *A, int64_t stride_row, int64_t stride_col,
                  const double *x, double *y)
{
    if (n1 < 0 || n2 < 0 || (n1 > 0 && !y) || (n1 > 0 && n2 > 0 && (!A || !x))) return ORACLE_ERR_ARG;
    for (int64_t i = 0; i < n1; ++i)
        y[i] = neumaier_sum_products(A + i * stride_row, stride_col, x, n2);
    return ORACLE_OK;
}
