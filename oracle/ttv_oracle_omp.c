/*
 * ttv_oracle_omp.c -- the oracle's TTV definition (ttv_oracle.c) spread over
 * the host's cores with OpenMP.  TEST AND BENCHMARK INFRASTRUCTURE ONLY: it
 * is the multi-core CPU baseline the benchmark reports beside the one-core
 * oracle; the CUDA library never calls it, and the two share no code.
 *
 * Same definition, same arithmetic, same order (paper Sec. 3.3, Eq. 3, with
 * pyttb's unique/accumarray grouping):
 *   1. every term vals[k] * prod_{m in S} x_m[subs[k, m]], in increasing mode
 *      order, in binary64 (the terms are independent: split over threads);
 *   2. the nonzeros ordered by (surviving tuple, input index): each thread
 *      sorts one contiguous range of the input; splitter tuples drawn from
 *      the sorted ranges cut every range into T key intervals, and thread i
 *      merges interval i of all ranges; the key (tuple, k) is a total order,
 *      so the merged order is exactly the one-core oracle's, and no tuple
 *      spans two intervals;
 *   3. one Neumaier sum per group in that order, as in the one-core oracle;
 *      each thread sums the groups of its interval.
 * The result is therefore bit-identical to oracle_ttv, which the tests check.
 * Build with -ffp-contract=off -fopenmp.
 */
#define _GNU_SOURCE
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_MAX_D 16
#define ORACLE_OMP_MAX_T 256

enum {
    ORACLE_OK = 0,
    ORACLE_ERR_ARG = -1,
    ORACLE_ERR_MODE = -2,
    ORACLE_ERR_VEC_LEN = -3,
    ORACLE_ERR_SUBSCRIPT = -4,
    ORACLE_ERR_NOMEM = -5,
};

typedef struct {
    int32_t order;
    int64_t shape[ORACLE_MAX_D];
    int64_t nnz;
    int64_t *subs;
    double *vals;
} oracle_out;

typedef struct {
    const int64_t *subs;
    int32_t d;
    int32_t nr;
    int32_t r[ORACLE_MAX_D];
} row_ctx;

/* (surviving tuple, input index), lexicographic */
static int row_cmp(const void *pa, const void *pb, void *pctx)
{
    const row_ctx *c = (const row_ctx *)pctx;
    const int64_t ka = *(const int64_t *)pa, kb = *(const int64_t *)pb;
    for (int32_t j = 0; j < c->nr; ++j) {
        const int64_t a = c->subs[ka * c->d + c->r[j]], b = c->subs[kb * c->d + c->r[j]];
        if (a < b) return -1;
        if (a > b) return 1;
    }
    return (ka > kb) - (ka < kb);
}

/* the surviving tuple alone */
static int tuple_cmp(const row_ctx *c, int64_t ka, int64_t kb)
{
    for (int32_t j = 0; j < c->nr; ++j) {
        const int64_t a = c->subs[ka * c->d + c->r[j]], b = c->subs[kb * c->d + c->r[j]];
        if (a < b) return -1;
        if (a > b) return 1;
    }
    return 0;
}

static int tuple_qcmp(const void *pa, const void *pb, void *pctx)
{
    return tuple_cmp((const row_ctx *)pctx, *(const int64_t *)pa, *(const int64_t *)pb);
}

/* first position in sorted idx[lo, hi) whose tuple is not below key's */
static int64_t lower_bound(const row_ctx *c, const int64_t *idx, int64_t lo, int64_t hi, int64_t key)
{
    while (lo < hi) {
        const int64_t mid = lo + (hi - lo) / 2;
        if (tuple_cmp(c, idx[mid], key) < 0) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

static int row_eq(const row_ctx *c, int64_t ka, int64_t kb)
{
    for (int32_t j = 0; j < c->nr; ++j)
        if (c->subs[ka * c->d + c->r[j]] != c->subs[kb * c->d + c->r[j]]) return 0;
    return 1;
}

void oracle_omp_free(oracle_out *out)
{
    if (!out) return;
    free(out->subs);
    free(out->vals);
    out->subs = NULL;
    out->vals = NULL;
    out->nnz = 0;
}

int oracle_omp_max_threads(void) { return omp_get_max_threads(); }

/* Arguments and result as oracle_ttv, plus the thread count (<= 0: all). */
int oracle_ttv_omp(int32_t d, const int64_t *shape, int64_t nnz, const int64_t *subs, const double *vals,
                   int32_t n_v, const int32_t *modes, const int64_t *vec_lens, const double *const *vecs,
                   int32_t dense, int32_t threads, oracle_out *out)
{
    if (!out || !shape || d < 1 || d > ORACLE_MAX_D || nnz < 0) return ORACLE_ERR_ARG;
    if (n_v < 1 || n_v > d || !modes || !vec_lens || !vecs) return ORACLE_ERR_ARG;
    if (nnz > 0 && (!subs || !vals)) return ORACLE_ERR_ARG;
    memset(out, 0, sizeof(*out));
    for (int32_t m = 0; m < d; ++m)
        if (shape[m] < 1) return ORACLE_ERR_ARG;
    const double *vec_of_mode[ORACLE_MAX_D];
    int32_t in_s[ORACLE_MAX_D];
    for (int32_t m = 0; m < d; ++m) { in_s[m] = 0; vec_of_mode[m] = NULL; }
    for (int32_t i = 0; i < n_v; ++i) {
        const int32_t m = modes[i];
        if (m < 0 || m >= d || in_s[m]) return ORACLE_ERR_MODE;
        if (vec_lens[i] != shape[m]) return ORACLE_ERR_VEC_LEN;
        if (!vecs[i]) return ORACLE_ERR_ARG;
        in_s[m] = 1;
        vec_of_mode[m] = vecs[i];
    }
    row_ctx ctx;
    ctx.subs = subs;
    ctx.d = d;
    ctx.nr = 0;
    for (int32_t m = 0; m < d; ++m)
        if (!in_s[m]) ctx.r[ctx.nr++] = m;
    int bad = 0;
    for (int64_t k = 0; k < nnz && !bad; ++k)
        for (int32_t m = 0; m < d; ++m)
            if (subs[k * d + m] < 0 || subs[k * d + m] >= shape[m]) bad = 1;
    if (bad) return ORACLE_ERR_SUBSCRIPT;
    out->order = ctx.nr;
    for (int32_t j = 0; j < ctx.nr; ++j) out->shape[j] = shape[ctx.r[j]];

    int T = threads > 0 ? threads : omp_get_max_threads();
    if (T < 1) T = 1;
    if (T > ORACLE_OMP_MAX_T) T = ORACLE_OMP_MAX_T;
    if ((int64_t)T > nnz) T = nnz > 0 ? (int)nnz : 1;

    const size_t n1 = (size_t)(nnz > 0 ? nnz : 1);
    double *t = (double *)malloc(n1 * sizeof(double));
    int64_t *idx = (int64_t *)malloc(n1 * sizeof(int64_t));
    int64_t *merged = (int64_t *)malloc(n1 * sizeof(int64_t));
    int64_t *lo = (int64_t *)malloc((size_t)(T + 1) * sizeof(int64_t));
    if (!t || !idx || !merged || !lo) {
        free(t); free(idx); free(merged); free(lo);
        return ORACLE_ERR_NOMEM;
    }
    for (int i = 0; i <= T; ++i) lo[i] = nnz * i / T;

    /* Steps 1 and 2a: terms, and each thread's range sorted */
#pragma omp parallel num_threads(T)
    {
        const int me = omp_get_thread_num();
        for (int64_t k = lo[me]; k < lo[me + 1]; ++k) {
            double p = vals[k];
            for (int32_t m = 0; m < d; ++m)
                if (in_s[m]) p = p * vec_of_mode[m][subs[k * d + m]];
            t[k] = p;
            idx[k] = k;
        }
        const int64_t len = lo[me + 1] - lo[me];
        if (len > 1) qsort_r(idx + lo[me], (size_t)len, sizeof(int64_t), row_cmp, &ctx);
    }
    /* Step 2b: splitters -- T samples from every sorted range, sorted by
     * tuple, every T-th kept; interval i holds the tuples in [split[i-1],
     * split[i]) */
    int64_t *samp = (int64_t *)malloc((size_t)T * T * sizeof(int64_t));
    int64_t *cut = (int64_t *)malloc((size_t)T * (T + 1) * sizeof(int64_t));   /* cut[r*(T+1)+i] */
    int64_t *ioff = (int64_t *)malloc((size_t)(T + 1) * sizeof(int64_t));
    int64_t *gcnt = (int64_t *)calloc((size_t)(T + 1), sizeof(int64_t));
    if (!samp || !cut || !ioff || !gcnt) {
        free(t); free(idx); free(merged); free(lo); free(samp); free(cut); free(ioff); free(gcnt);
        return ORACLE_ERR_NOMEM;
    }
    int ns = 0;
    for (int r = 0; r < T; ++r) {
        const int64_t len = lo[r + 1] - lo[r];
        if (len == 0) continue;
        for (int j = 0; j < T; ++j) samp[ns++] = idx[lo[r] + len * j / T];
    }
    if (ns > 1) qsort_r(samp, (size_t)ns, sizeof(int64_t), tuple_qcmp, &ctx);
#pragma omp parallel for num_threads(T)
    for (int r = 0; r < T; ++r) {
        cut[r * (T + 1)] = lo[r];
        cut[r * (T + 1) + T] = lo[r + 1];
        for (int i = 1; i < T; ++i)
            cut[r * (T + 1) + i] = ns > 0 ? lower_bound(&ctx, idx, lo[r], lo[r + 1], samp[(int64_t)ns * i / T])
                                          : lo[r];
    }
    ioff[0] = 0;
    for (int i = 0; i < T; ++i) {
        int64_t c = 0;
        for (int r = 0; r < T; ++r) c += cut[r * (T + 1) + i + 1] - cut[r * (T + 1) + i];
        ioff[i + 1] = ioff[i] + c;
    }
    /* Step 2c: thread i merges interval i of every range (a binary heap of
     * the ranges' current heads, ordered by (tuple, k)) */
#pragma omp parallel num_threads(T)
    {
        const int me = omp_get_thread_num();
        int64_t pos[ORACLE_OMP_MAX_T], end[ORACLE_OMP_MAX_T];
        int heap[ORACLE_OMP_MAX_T];
        int hn = 0;
        for (int r = 0; r < T; ++r) {
            pos[r] = cut[r * (T + 1) + me];
            end[r] = cut[r * (T + 1) + me + 1];
            if (pos[r] < end[r]) {
                /* sift up */
                int c = hn++;
                heap[c] = r;
                while (c > 0) {
                    const int par = (c - 1) / 2;
                    if (row_cmp(&idx[pos[heap[c]]], &idx[pos[heap[par]]], &ctx) >= 0) break;
                    const int tmp = heap[c]; heap[c] = heap[par]; heap[par] = tmp;
                    c = par;
                }
            }
        }
        int64_t q = ioff[me];
        while (hn > 0) {
            const int r = heap[0];
            merged[q++] = idx[pos[r]++];
            if (pos[r] >= end[r]) heap[0] = heap[--hn];
            /* sift down */
            int c = 0;
            for (;;) {
                const int l = 2 * c + 1, rr = l + 1;
                int m = c;
                if (l < hn && row_cmp(&idx[pos[heap[l]]], &idx[pos[heap[m]]], &ctx) < 0) m = l;
                if (rr < hn && row_cmp(&idx[pos[heap[rr]]], &idx[pos[heap[m]]], &ctx) < 0) m = rr;
                if (m == c) break;
                const int tmp = heap[c]; heap[c] = heap[m]; heap[m] = tmp;
                c = m;
            }
        }
        /* groups of this interval (no tuple spans two intervals) */
        int64_t cnt = 0;
        for (int64_t i = ioff[me]; i < ioff[me + 1]; ++i)
            if (i == ioff[me] || !row_eq(&ctx, merged[i - 1], merged[i])) ++cnt;
        gcnt[me + 1] = cnt;
    }
    free(idx);
    free(lo);
    free(samp);
    free(cut);
    for (int i = 0; i < T; ++i) gcnt[i + 1] += gcnt[i];
    const int64_t groups = gcnt[T];

    /* Step 3: one entry per distinct tuple, Neumaier sum in input order;
     * interval i writes groups gcnt[i] .. gcnt[i+1]-1 */
    const size_t g1 = (size_t)(groups > 0 ? groups : 1);
    int64_t *gsubs = (int64_t *)malloc(g1 * (size_t)(ctx.nr > 0 ? ctx.nr : 1) * sizeof(int64_t));
    double *gvals = (double *)malloc(g1 * sizeof(double));
    if (!gsubs || !gvals) { free(t); free(merged); free(ioff); free(gcnt); free(gsubs); free(gvals); return ORACLE_ERR_NOMEM; }
#pragma omp parallel num_threads(T)
    {
        const int me = omp_get_thread_num();
        int64_t g = gcnt[me] - 1;
        double sum = 0.0, comp = 0.0;
        for (int64_t i = ioff[me]; i < ioff[me + 1]; ++i) {
            const int64_t k = merged[i];
            if (i == ioff[me] || !row_eq(&ctx, merged[i - 1], k)) {
                if (g >= gcnt[me]) gvals[g] = isfinite(sum) ? sum + comp : sum;
                ++g;
                for (int32_t j = 0; j < ctx.nr; ++j) gsubs[g * ctx.nr + j] = subs[k * d + ctx.r[j]];
                sum = 0.0;
                comp = 0.0;
            }
            const double s = sum + t[k];
            if (fabs(sum) >= fabs(t[k])) comp += (sum - s) + t[k];
            else                         comp += (t[k] - s) + sum;
            sum = s;
        }
        if (g >= gcnt[me]) gvals[g] = isfinite(sum) ? sum + comp : sum;
    }
    free(t);
    free(merged);
    free(ioff);
    free(gcnt);

    if (!dense) {
        if (ctx.nr == 0 && groups == 0) {
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
