/*
 * ttv.h -- C ABI of the GB300 (sm_103a) sparse tensor-times-vector library.
 *
 * The operation (paper Sec. 3.3, Eq. 3 and the multi-vector paragraph before
 * it): a d-way sparse COO tensor A (int64 subscripts, one value per nonzero)
 * is multiplied by n_v dense vectors x_m, one for each contracted mode m in S.
 * The result has order d - n_v over the surviving modes R = [0,d) \ S, taken
 * in increasing order:
 *
 *     B(i_R) = sum_{k : subs[k,R] == i_R}  vals[k] * prod_{m in S} x_m[subs[k,m]]
 *
 * Conventions shared by every entry point:
 *   - Indices are 0-based (the paper counts from 1; its "mode k = 2" is mode 1).
 *   - Device pointers are plain CUDA device addresses (for example from torch);
 *     the library never takes ownership of inputs.  Host arrays (shape, modes,
 *     the array of vector pointers) are read during the call only.
 *   - A sparse result is canonical COO: one entry per distinct surviving
 *     subscript tuple that occurs in the input (even when its sum is zero),
 *     in ascending lexicographic order of the tuple -- the row order of the
 *     "unique" step the paper describes for pyttb's sptensor.ttv (Sec. 3.3).
 *     Duplicate input subscripts are summed.
 *   - A dense result is a row-major array over shape[R] (last mode fastest).
 *     n_v == d gives an order-0 result: one scalar (nnz 1).
 *   - Calls are asynchronous on `stream` except where stated: unless
 *     opts->async is set, the call synchronises `stream` once at the end to
 *     read the output count and the error word, so out->nnz and the return
 *     code are final on return.
 *   - Return value: TTV_OK (0) or a negative TTV_ERR_*; ttv_last_error()
 *     gives a message for the calling thread's last failure.
 *   - Subscript bounds are checked inside the streaming kernel at no extra
 *     traffic: an out-of-range subscript is skipped and reported as
 *     TTV_ERR_SUBSCRIPT; the output contents are then unspecified.
 */
#ifndef TTV_GB300_H
#define TTV_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TTV_MAX_D 8              /* largest tensor order the kernels accept */

typedef struct CUstream_st *ttv_stream_t;   /* same handle as cudaStream_t; NULL = default stream */

enum {
    TTV_OK = 0,
    TTV_ERR_ARG = -1,            /* null pointer, bad size, bad enum value          */
    TTV_ERR_MODE = -2,           /* contracted mode out of range or repeated        */
    TTV_ERR_VEC_LEN = -3,        /* vector length differs from shape[mode]          */
    TTV_ERR_SUBSCRIPT = -4,      /* a subscript outside [0, shape[m]) (device check)*/
    TTV_ERR_KEY_OVERFLOW = -5,   /* prod(shape[R]) does not fit in 64 bits          */
    TTV_ERR_BUDGET = -6,         /* workspace or server memory budget too small     */
    TTV_ERR_TIMEOUT = -7,        /* a bounded device wait or a server wait ran out  */
    TTV_ERR_CUDA = -8,           /* a CUDA runtime call failed                      */
    TTV_ERR_CAPACITY = -9,       /* caller-provided output buffer too small         */
    TTV_ERR_NOMEM = -10,         /* allocation failed                               */
    TTV_ERR_UNSUPPORTED = -11,   /* combination not implemented                     */
};

typedef enum { TTV_F64 = 0, TTV_F32 = 1 } ttv_dtype;

typedef enum {
    TTV_OUT_SPARSE = 0,          /* canonical COO (default)                          */
    TTV_OUT_DENSE = 1,           /* dense row-major array over shape[R]              */
    TTV_OUT_AUTO = 2             /* dense when nnz_out > 0.5 * prod(shape[R]): the
                                    pyttb conversion rule the paper mentions (Sec. 3.3).
                                    Computed sparse, converted when the result is
                                    finalised (end of a synchronous call, or
                                    ttv_out_sync): a library-allocated result moves
                                    to a new dense buffer; caller buffers are
                                    converted in place when vals_capacity holds every
                                    cell, else the result stays sparse.  is_dense and
                                    nnz report the outcome. */
} ttv_out_format;

typedef enum {
    TTV_PATH_AUTO = 0,           /* autotuner record, else the planner's rule         */
    TTV_PATH_DENSE = 1,          /* block-private dense accumulator (small prod R)    */
    TTV_PATH_SORT = 2,           /* LSD onesweep radix sort + segmented reduction     */
    TTV_PATH_HASH = 3,           /* warp-combined table in HBM (direct-indexed or open
                                    addressing) + compaction; not deterministic, so
                                    deterministic/compensated calls use SORT         */
    TTV_PATH_BUCKET = 4          /* splitter partition + in-shared-memory sort        */
} ttv_path;

typedef enum {
    TTV_ACCUM_FP64 = 0,          /* IEEE binary64 additions                           */
    TTV_ACCUM_COMPENSATED = 1,   /* binary64 with two-sum error compensation          */
    TTV_ACCUM_EXACT = 2          /* 128-bit fixed point, order independent; the dense
                                    path's deterministic mode                         */
} ttv_accum;

/* Input tensor.  subs[k * stride_nz + m * stride_mode] is subscript m of
 * nonzero k: (stride_nz, stride_mode) = (d, 1) for row-major nnz x d (AoS) or
 * (1, nnz) for one contiguous column per mode (SoA, pyttb's column-major
 * layout, paper Sec. 3.2).  Strides are in elements. */
typedef struct {
    const int64_t *subs;         /* device */
    int64_t stride_nz;
    int64_t stride_mode;
    const void *vals;            /* device, nnz values of val_dtype               */
    ttv_dtype val_dtype;
    int64_t nnz;                 /* >= 0                                          */
    const int64_t *shape;        /* host, d sizes >= 1                            */
    int32_t d;                   /* 1 .. TTV_MAX_D                                */
} ttv_tensor;

/* Result.  Before the call the caller either sets subs/vals to NULL (the
 * library allocates them; release with ttv_out_free) or points them at device
 * buffers of subs_capacity x order int64 (row-major) and vals_capacity values
 * (the library writes into them and ttv_out_free leaves them alone).  A safe
 * capacity is ttv_out_capacity(); a smaller one that the result does not fit
 * gives TTV_ERR_CAPACITY.  After the call: order, shape, nnz (valid on return
 * unless opts->async), is_dense, dtype (always TTV_F64 values). */
typedef struct {
    int32_t order;
    int64_t shape[TTV_MAX_D];
    int64_t nnz;                 /* output entries; prod(shape) when dense          */
    int64_t *subs;               /* nnz x order row-major; unused when dense        */
    void *vals;                  /* nnz values                                      */
    int64_t subs_capacity;       /* rows available at subs (caller buffers)         */
    int64_t vals_capacity;       /* values available at vals (caller buffers)       */
    ttv_dtype dtype;
    int32_t is_dense;
    void *internal;              /* library bookkeeping; zero-initialise            */
} ttv_out;

typedef struct {
    int32_t fmt;                 /* ttv_out_format                                  */
    int32_t path;                /* ttv_path                                        */
    int32_t accum;               /* ttv_accum                                       */
    int32_t deterministic;       /* nonzero: bit-identical results run to run       */
    int32_t async;               /* nonzero: do not synchronise; call ttv_out_sync  */
    void *workspace;             /* device scratch, or NULL to let the library
                                    allocate from its stream-ordered pool          */
    size_t workspace_bytes;
} ttv_opts;

/* Defaults: SPARSE, AUTO path, FP64, not forced deterministic, synchronous,
 * library-allocated workspace. */
void ttv_opts_init(ttv_opts *opts);

/* Single-vector TTV, A x_mode v (paper Eq. 3).  v is a device vector of
 * shape[mode] entries of v_dtype.  Result order d - 1. */
int ttv_single(const ttv_tensor *t, int32_t mode, const void *v, ttv_dtype v_dtype,
               ttv_out *out, const ttv_opts *opts, ttv_stream_t stream);

/* Multi-vector TTV (paper Sec. 3.3, n_v in {1..d}): vecs[i] multiplies mode
 * modes[i]; modes are distinct, in any order (the result does not depend on
 * it).  n_v == d - 1 is the all-but-one form; n_v == d gives a scalar. */
int ttv_multi(const ttv_tensor *t, const int32_t *modes, int32_t n_v,
              const void *const *vecs, ttv_dtype v_dtype,
              ttv_out *out, const ttv_opts *opts, ttv_stream_t stream);

/* ttv_multi with the vector lengths (host array, n_v entries) checked
 * against shape[modes[i]] first (paper Sec. 3.3: each vector's size must be
 * that of its mode); a mismatch returns TTV_ERR_VEC_LEN. */
int ttv_multi_checked(const ttv_tensor *t, const int32_t *modes, int32_t n_v,
                      const void *const *vecs, const int64_t *vec_lens, ttv_dtype v_dtype,
                      ttv_out *out, const ttv_opts *opts, ttv_stream_t stream);

/* Upper bounds for caller-allocated results: rows of subs and number of
 * values.  Sparse: min(nnz, prod shape[R]) (at least 1 for order 0).
 * Dense: prod shape[R]. */
int ttv_out_capacity(const ttv_tensor *t, const int32_t *modes, int32_t n_v,
                     const ttv_opts *opts, int64_t *rows, int64_t *values);

/* Device scratch a ttv_multi call with these arguments needs when the caller
 * supplies opts->workspace. */
int ttv_workspace_size(const ttv_tensor *t, const int32_t *modes, int32_t n_v,
                       ttv_dtype v_dtype, const ttv_opts *opts, size_t *bytes);

/* Completes an opts->async call: synchronises its stream, fills out->nnz and
 * returns the call's device-side status. */
int ttv_out_sync(ttv_out *out);

/* Releases what the library allocated for `out` (not caller buffers). */
void ttv_out_free(ttv_out *out);
/* ttv_out_free on outs[0..n) (a batch's results): one call instead of n. */
void ttv_outs_free(ttv_out *outs, int32_t n);

/* Message for the calling thread's last error ("" if none). */
const char *ttv_last_error(void);

/* ---- batched TTV ------------------------------------------------------------
 * Many independent TTVs (paper Eq. 3 each) in one CUDA-graph launch.  The
 * first call with a given set of problems captures them into one graph and
 * instantiates it; a later call with identical problems (same pointers,
 * sizes, modes, output buffers, workspace and options) launches the cached
 * graph without host work per problem.  Every problem whose plan is the sort
 * path with a sparse result runs stage-wise: each stage (keys and terms per
 * order and layout class, the digit-count scan, each 8-bit digit pass, the
 * four reduce-by-key stages) is one launch over all such problems, so they
 * cost about 20 launches together whatever their number.  The other problems
 * (dense, hash and partition paths, dense results) keep their own launch
 * sequences, spread over up to 7 concurrent streams beside it (largest
 * problems first).  Up to 16 graphs are cached; ttv_batch_release() drops
 * them. */
typedef struct {
    ttv_tensor tensor;
    const int32_t *modes;        /* host, n_v contracted modes                    */
    int32_t n_v;
    const void *const *vecs;     /* host array of n_v device vectors              */
    ttv_dtype v_dtype;
} ttv_problem;

/* outs[i] must point at caller buffers (subs/vals with capacities, see
 * ttv_out_capacity); opts->workspace may hold ttv_batch_workspace_size()
 * bytes (else the library allocates one block and keeps it with the cached
 * graph).  Synchronous unless opts->async (then ttv_out_sync each result).
 * Results of a cached graph are rewritten by its next launch.  A problem that
 * fails leaves its error in ttv_out_sync(&outs[i]); the call returns the
 * first failure. */
int ttv_batch(const ttv_problem *probs, int32_t n, ttv_out *outs, const ttv_opts *opts,
              ttv_stream_t stream);
int ttv_batch_workspace_size(const ttv_problem *probs, int32_t n, const ttv_opts *opts, size_t *bytes);
/* Kernel launches one replay of the graph for these problems performs (0 if
 * it is not cached). */
long long ttv_batch_graph_launches(const ttv_problem *probs, int32_t n, const ttv_out *outs, const ttv_opts *opts);
void ttv_batch_release(void);

/* ---- autotuner ----------------------------------------------------------------
 * The paper has no counterpart: it times one fixed CPU kernel per language.
 * Problems fall into classes by (order d, surviving modes, result format,
 * value and vector dtypes, subscript layout, ceil(log2 nnz), ceil(log2 of
 * the key space prod shape[R])).  ttv_autotune runs every applicable
 * candidate on the given problem -- accumulation path (DENSE, SORT, HASH,
 * BUCKET) x CTAs per SM of the streaming pass (2/3/4 for DENSE, 4/8/16 for
 * SORT, 8/16 for HASH) x nonzeros per thread per iteration (DENSE: 1 or 2
 * pairs, 3 = one pair into warp-private accumulators where they fit, or
 * 4 = the bulk-staged persistent kernel with one CTA per SM;
 * HASH: 2 or 4) -- `trials` times
 * after one warm-up run each, takes
 * the median of CUDA-event times on `stream`, and records the fastest for
 * the class.
 * Every later call with path AUTO, fp64 accumulation and no determinism
 * request (ttv_multi, ttv_batch, the server) whose problem falls in a
 * recorded class uses the recorded plan; other calls are unaffected.  The
 * record lives in host memory, shared by all threads; ttv_tune_save /
 * ttv_tune_load keep it in a text file ("ttv-tune 2" header, then one
 * "<class hex> <path> <ctas_per_sm> <items_per_thread> <ms>" line per class;
 * loading merges).
 * ttv_autotune synchronises `stream` once per trial and allocates its own
 * workspace and results; it returns TTV_ERR_ARG for deterministic or
 * non-fp64 options and TTV_ERR_UNSUPPORTED when no candidate can run (an
 * empty tensor). */
#define TTV_TUNE_MAX_CANDIDATES 16
typedef struct {
    int32_t path;                /* chosen ttv_path                                */
    int32_t ctas_per_sm;         /* chosen CTAs per SM of the streaming pass        */
    int32_t items_per_thread;    /* chosen nonzeros per thread (0: path default)    */
    double ms;                   /* its median time                                */
    int32_t n_candidates;        /* candidates that ran                             */
    int32_t cand_path[TTV_TUNE_MAX_CANDIDATES];
    int32_t cand_ctas[TTV_TUNE_MAX_CANDIDATES];
    int32_t cand_items[TTV_TUNE_MAX_CANDIDATES];
    double cand_ms[TTV_TUNE_MAX_CANDIDATES];
} ttv_tune_result;

int ttv_autotune(const ttv_tensor *t, const int32_t *modes, int32_t n_v, const void *const *vecs,
                 ttv_dtype v_dtype, const ttv_opts *opts, int32_t trials, ttv_tune_result *result,
                 ttv_stream_t stream);
int ttv_tune_save(const char *path);     /* TTV_ERR_ARG if the file can not be written */
int ttv_tune_load(const char *path);     /* TTV_ERR_ARG on a missing or malformed file;
                                            nothing is merged then                     */
void ttv_tune_clear(void);
int ttv_tune_count(void);                /* recorded classes */
/* Records a plan for the problem's class by hand, as ttv_autotune would:
 * a concrete path (DENSE, SORT, HASH, BUCKET), CTAs per SM (0: default) and
 * items per thread (0: default), with the meanings listed above.  A path
 * that does not apply to a later problem of the class falls back as for an
 * autotuned record.  TTV_ERR_ARG for an invalid problem or plan. */
int ttv_tune_set(const ttv_tensor *t, const int32_t *modes, int32_t n_v, const ttv_opts *opts, int32_t path,
                 int32_t ctas_per_sm, int32_t items_per_thread);
/* 1 and the recorded plan if the problem's class (vectors taken as FP64 for
 * the class key) has a record, 0 if not, a negative error code for an
 * invalid problem.  path / ctas_per_sm / items_per_thread may be NULL. */
int ttv_tune_lookup(const ttv_tensor *t, const int32_t *modes, int32_t n_v, const ttv_opts *opts, int32_t *path,
                    int32_t *ctas_per_sm, int32_t *items_per_thread);

/* ---- prepared tensors ----------------------------------------------------------
 * For repeated TTVs of one resident tensor along one fixed set of modes S
 * with fresh vectors.  The grouping of Sec. 3.3 (one result row per distinct
 * surviving tuple, ascending) depends on the tensor only, so ttv_prepare
 * sorts the nonzeros once by their surviving key (stable: equal keys keep
 * input order) and keeps, in that order, the values (val_dtype) and the
 * subscripts of the modes in S (int32; every mode in S must be smaller than
 * 2^31), plus a bitmap of where each result row starts (1 bit per nonzero)
 * and the key of every result row; with one surviving mode it also indexes
 * the rows per 128-nonzero chunk for MTTKRP.  ttv_prepared_run is then one streaming
 * reduce-by-key over those arrays with the terms vals * prod x_m[sub_m]
 * formed on the fly in increasing mode order: its result equals, bit for bit,
 * that of ttv_multi with path SORT and fp64 accumulation on the same inputs.
 *
 * ttv_prepare copies what it needs (the caller's arrays may be freed
 * afterwards) into device memory owned by the handle (ttv_prepared_info
 * reports the bytes), synchronises `stream` once and returns
 * TTV_ERR_SUBSCRIPT / TTV_ERR_MODE / TTV_ERR_KEY_OVERFLOW / TTV_ERR_ARG like
 * ttv_multi, TTV_ERR_UNSUPPORTED for nnz >= 2^30 or a contracted mode of
 * 2^31 or more entries.  ttv_prepared_run takes the vectors in the order of
 * the modes given to ttv_prepare (vec_lens may be NULL; else each must equal
 * its mode size), opts as ttv_multi (fmt, workspace, async; accum
 * TTV_ACCUM_FP64, or TTV_ACCUM_COMPENSATED: every run sum then carries a
 * Neumaier error term through all stages and is rounded once; path is
 * ignored), and fills `out` like ttv_multi: for a
 * sparse result nnz_out rows (ttv_prepared_info), for a dense one
 * prod(shape[R]) values.  Runs on one handle may overlap on different
 * streams; ttv_prepared_free synchronises the device and releases it. */
typedef struct ttv_prepared ttv_prepared;
int ttv_prepare(const ttv_tensor *t, const int32_t *modes, int32_t n_v, ttv_prepared **out, ttv_stream_t stream);
int ttv_prepared_run(const ttv_prepared *p, const void *const *vecs, const int64_t *vec_lens, ttv_dtype v_dtype,
                     ttv_out *out, const ttv_opts *opts, ttv_stream_t stream);
int ttv_prepared_info(const ttv_prepared *p, int64_t *nnz_out, int32_t *order, size_t *device_bytes);
int ttv_prepared_workspace_size(const ttv_prepared *p, size_t *bytes);
void ttv_prepared_free(ttv_prepared *p);

/* ---- MTTKRP -------------------------------------------------------------------
 * The matricized tensor times Khatri-Rao product, which the paper names as the
 * kernel built on the sparse TTV (Sec. 3.3) and as future work (Sec. 5).
 * Along mode n with factor matrices A_m (shape[m] x rank, row-major, binary64,
 * device), m != n:
 *     M(i, r) = sum over nonzeros k with subs[k, n] == i of
 *               vals[k] * prod_{m != n, increasing} A_m(subs[k, m], r),
 * so column r is the all-but-one TTV with the vectors A_m(:, r).  `out` is
 * shape[n] x rank row-major binary64 on the device, written in full (rows no
 * nonzero touches are 0).  Sums are formed in a fixed order: results are
 * bit-identical run to run.  rank must be 1..TTV_MTTKRP_MAX_RANK.
 *
 * ttv_mttkrp_prepared runs on a tensor prepared (ttv_prepare) for every mode
 * but n -- the layout sorts the nonzeros by subs[k, n] -- with one factor per
 * prepared mode, in the order the modes were given to ttv_prepare; it is
 * asynchronous on `stream` and takes `workspace` when it holds
 * ttv_mttkrp_workspace_size bytes (else it allocates from the stream-ordered
 * pool).  TTV_ERR_ARG for a tensor not prepared that way, a null factor or a
 * bad rank.  ttv_mttkrp prepares, runs and releases in one call (factors:
 * d pointers, factors[mode] is not read) and synchronises `stream`; errors
 * as ttv_prepare. */
#define TTV_MTTKRP_MAX_RANK 128
int ttv_mttkrp_prepared(const ttv_prepared *p, const double *const *factors, int32_t rank, double *out,
                        void *workspace, size_t workspace_bytes, ttv_stream_t stream);
int ttv_mttkrp_workspace_size(const ttv_prepared *p, int32_t rank, size_t *bytes);
int ttv_mttkrp(const ttv_tensor *t, int32_t mode, const double *const *factors, int32_t rank, double *out,
               ttv_stream_t stream);

/* ---- the paper's two simple kernels on dense operands ---------------------------
 * ttv_dot: x . y = sum_{i<n} x[i] * y[i] (paper Sec. 3.1, Eq. 1).  x and y are
 * device arrays of n elements of `dtype` (float64 or float32, both the same;
 * float32 is upcast exactly); *out (device) receives the binary64 result.
 * ttv_matvec: y[i] = sum_{j<n2} A(i, j) * x[j], i < n1 (paper Sec. 3.2, Eq. 2),
 * with A(i, j) = A[i * stride_row + j * stride_col] (elements): row-major
 * storage has strides (n2, 1), pyttb's column-major storage (1, n1).  One of
 * the strides must be 1 (or the matrix a single row or column), else
 * TTV_ERR_UNSUPPORTED.  A and x are `dtype`, y (device, n1 doubles) binary64.
 * n1 or n2 == 0 gives y = 0 (n1 == 0: nothing written).
 *
 * Both are asynchronous on `stream`.  Each element costs one binary64 fused
 * multiply-add; the combination across lanes, CTAs and column chunks is in
 * a fixed order, so results are bit-identical from run to run (they differ
 * from a sequential sum by rounding only).  `workspace` is used when it holds
 * the *_workspace_size bytes, else scratch comes from the stream-ordered
 * pool.  Errors: TTV_ERR_ARG for a null pointer or a negative size. */
int ttv_dot(const void *x, const void *y, int64_t n, ttv_dtype dtype, double *out, void *workspace,
            size_t workspace_bytes, ttv_stream_t stream);
int ttv_dot_workspace_size(int64_t n, size_t *bytes);
int ttv_matvec(const void *A, int64_t n1, int64_t n2, int64_t stride_row, int64_t stride_col, ttv_dtype dtype,
               const void *x, double *y, void *workspace, size_t workspace_bytes, ttv_stream_t stream);
int ttv_matvec_workspace_size(int64_t n1, int64_t n2, int64_t stride_row, int64_t stride_col, size_t *bytes);

/* ---- serving ------------------------------------------------------------------
 * A continuous-batching TTV server.  Registered tensors stay resident in
 * server-owned device memory.  Requests (contracted modes + host vectors)
 * queue up; a scheduler thread admits any queued request for which a stream
 * slot is free and the memory budget covers its workspace, result and
 * vectors (a request that does not fit yet does not block smaller ones behind
 * it), so the work of several requests overlaps on the GPU.  While more
 * requests wait than slots are free, a free slot takes a group of queued
 * requests with the same options (up to 32, about the queue over the free
 * slots) and runs them as one stage-wise batch (see ttv_batch): the sort-path
 * requests of a group share one launch per stage.  Requests on a prepared
 * layout always run alone.  Latency is measured from submit to completion on
 * the GPU (a group's requests complete together).  Results are
 * library-allocated device buffers handed over by ttv_server_wait (release
 * with ttv_out_free); from completion until claimed only the result counts
 * against the budget.  While unclaimed results keep the budget full, the
 * oldest queued request is still admitted whenever nothing runs, so a client
 * waiting by id always progresses. */
typedef struct ttv_server ttv_server;

typedef struct {
    double p50_us, p99_us, mean_us, max_us;   /* submit -> completion latency    */
    long long completed, admitted, refused, pending;
    double seconds;                           /* since creation or reset          */
    double throughput_rps, throughput_gnnz_s; /* completed requests / nonzeros    */
    size_t bytes_in_use, budget_bytes;
    long long prepared_runs;                  /* requests served from a prepared layout */
    long long grouped_runs;                   /* requests served inside a group of two or more */
} ttv_stats;

/* budget_bytes bounds resident tensors + in-flight requests + unclaimed
 * results (bytes_in_use in ttv_stats); n_slots (1..64)
 * concurrent requests, one CUDA stream each. */
int ttv_server_create(size_t budget_bytes, int32_t n_slots, ttv_server **server);
/* Copies a device tensor (any subscript strides) into the server; it counts
 * against the budget until the server is destroyed.  TTV_ERR_BUDGET if it
 * does not fit. */
int ttv_server_register(ttv_server *server, const ttv_tensor *t, int32_t *tensor_id);
/* Prepares registered tensor `tensor_id` for TTVs along exactly the modes
 * given (see ttv_prepare; the layout counts against the budget until the
 * server is destroyed).  Later requests on that tensor with the same set of
 * modes (any order), path AUTO, no determinism request and fp64 or
 * compensated accumulation run on the prepared layout with no sort passes
 * (fp64: results identical to the sort path; compensated: the prepared
 * run's compensated sums, within the same tolerance).  Synchronous;
 * TTV_ERR_BUDGET if the layout does not fit, errors of ttv_prepare
 * otherwise.  May be called while requests run. */
int ttv_server_prepare(ttv_server *server, int32_t tensor_id, const int32_t *modes, int32_t n_v);
/* Queues a TTV of registered tensor `tensor_id` with n_v host vectors (each
 * shape[modes[i]] entries of v_dtype, copied at submit).  opts may be NULL
 * (its workspace and async fields are ignored).  TTV_ERR_BUDGET if the request
 * could never fit next to the resident tensors. */
int ttv_server_submit(ttv_server *server, int32_t tensor_id, const int32_t *modes, int32_t n_v,
                      const void *const *host_vecs, ttv_dtype v_dtype, const ttv_opts *opts,
                      uint64_t *req_id);
/* Waits up to timeout_us (< 0: forever) for a request and moves its result
 * into *out.  TTV_ERR_TIMEOUT if it is not done in time. */
int ttv_server_wait(ttv_server *server, uint64_t req_id, int64_t timeout_us, ttv_out *out);
/* Waits up to timeout_us (< 0: forever) for any finished request not yet
 * claimed (the oldest first) and moves its id into *req_id and its result
 * into *out; for a client that takes results as they finish, whatever order
 * they finish in (an unclaimed result holds budget, so claiming in
 * submission order behind a slow request holds back admission).  A server's
 * clients should use one of the two waits, not both: this one may take a
 * request another thread waits on by id. */
int ttv_server_wait_any(ttv_server *server, int64_t timeout_us, uint64_t *req_id, ttv_out *out);
int ttv_server_stats(ttv_server *server, ttv_stats *stats);
/* Clears latencies and counters (e.g. after a warm-up). */
int ttv_server_reset_stats(ttv_server *server);
/* Drains running requests, then frees everything the server owns. */
void ttv_server_destroy(ttv_server *server);

/* ---- allocation-free dense TTV ----------------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers
 * that must not allocate device memory (code running under a host
 * application that owns every allocation, a real-time loop that cannot take
 * the allocator's locks or synchronisation, a process whose memory budget
 * belongs to another runtime).  It computes the dense result (prod shape[R]
 * binary64 values, row-major) into the caller's buffer `out` (out_len values)
 * and allocates nothing: its scratch -- a status word and one partial array
 * per CTA -- lives in a fixed device array of TTV_NOALLOC_SCRATCH_BYTES that
 * is part of the library and stays resident on every GPU that loads it until
 * the process exits.
 *   - Limit: prod shape[R] <= 16384 cells (the dense path's shared-memory
 *     accumulator); larger result spaces return TTV_ERR_UNSUPPORTED.  The
 *     fixed scratch holds at least 31 partial arrays of that largest size, so
 *     TTV_ERR_BUDGET (kept as a guard) cannot occur at these limits; for
 *     large results the call runs fewer CTAs, as many as the scratch holds.
 *   - vec_lens may be NULL; otherwise a mismatch returns TTV_ERR_VEC_LEN.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before capturing any stream.
 *   - Synchronous: returns after `stream` has finished the call.
 *   - Every call shares the one array (the status word is cleared at the start
 *     of each call), so calls that overlap on the GPU -- on different streams
 *     or from different host threads -- race and must be serialised. */
#define TTV_NOALLOC_SCRATCH_BYTES (4u << 20)
int ttv_dense_noalloc(const ttv_tensor *t, const int32_t *modes, int32_t n_v,
                      const void *const *vecs, const int64_t *vec_lens, ttv_dtype v_dtype,
                      double *out, int64_t out_len, ttv_stream_t stream);

/* ---- measurement --------------------------------------------------------
 * Every kernel launch of the library is counted; with profiling enabled a
 * CUDA event pair brackets each launch on the launching stream.  The paper
 * times whole calls with monotonic clocks over 30 trials after a warm-up call
 * (Sec. 3 and Sec. 4); these hooks add the per-kernel device view. */

/* Kernel launches the library has issued since load. */
long long ttv_launch_count(void);
/* on != 0: record an event pair around every subsequent launch. */
void ttv_profile_enable(int on);
/* Waits for the recorded events and adds their times to per-kernel totals. */
int ttv_profile_collect(void);
/* Total milliseconds and launches of one kernel (by its name, e.g.
 * "dense_accum"); TTV_ERR_ARG if it has not run. */
int ttv_profile_get(const char *kernel, double *total_ms, long long *launches);
/* Newline-separated kernel names into buf (len bytes); with buf == NULL
 * returns the length needed. */
int ttv_profile_names(char *buf, size_t len);
/* Clears the per-kernel totals. */
void ttv_profile_reset(void);

/* ---- test hooks for the bounded device waits ----------------------------
 * Every wait of a kernel on another CTA's progress (the sort's decoupled
 * look-back across tiles, the staged dense kernel's bulk-copy pipeline) gives
 * up after a poll limit, raises a timeout bit that the call turns into
 * TTV_ERR_TIMEOUT, and lets the kernel finish without hanging.  These hooks
 * let a test make such a wait run out on purpose (the paper has no
 * counterpart; they exist only to test that error path). */
/* polls >= 0: those waits give up after `polls` polls (0: at once); polls < 0
 * restores their own limits.  Affects every later call in the process; a call
 * that runs out returns TTV_ERR_TIMEOUT and its result is not valid. */
int ttv_test_set_wait_polls(long long polls);
/* One thread waits `polls` polls on an mbarrier that nothing arrives on
 * (kind 0) or on a device word that nothing sets (kind 1).  Returns
 * TTV_ERR_TIMEOUT when the wait ran out (the expected outcome), TTV_OK if it
 * did not, TTV_ERR_ARG for another kind. */
int ttv_test_wait_probe(int kind, unsigned int polls);

#ifdef __cplusplus
}
#endif

#endif /* TTV_GB300_H */
