// ttv_api.cu -- the C ABI (include/ttv.h): argument checks, planning of the
// accumulation path, workspace layout, launches and the status read-back.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "ttv_internal.cuh"

namespace ttv {
// kernels in ttv_stream.cu / ttv_sort.cu
void launch_keys_terms(const StreamDesc& p, uint64_t* keys, double* terms, cudaStream_t stream);
size_t dense_smem_bytes(const StreamDesc& p, int want_presence);
int dense_grid(const StreamDesc& p, int want_presence);
void launch_dense(const StreamDesc& p, int want_presence, int compensated, int G, double* partials,
                  uint32_t* pres_partials, double* cell_vals, uint32_t* cell_flags, cudaStream_t stream);
void launch_compact_cells(const StreamDesc& p, const double* cell_vals, const uint32_t* cell_flags, int64_t cap_rows,
                          int64_t* out_subs, double* out_vals, cudaStream_t stream);
struct SegOut {
    int64_t* subs;
    double* vals;
    int64_t cap_rows;
    int dense;
    int compensated;
};
void launch_seg_reduce(const uint64_t* keys, const double* vals, int64_t n, uint32_t* seg_start,
                       unsigned long long* lookback, uint32_t* ticket, uint32_t* long_list, const StreamDesc& p,
                       const SegOut& o, Status* st, cudaStream_t stream);

bool bucket_applicable(const StreamDesc& p);
size_t bucket_workspace_bytes(int64_t nnz, int key_bits);
void launch_bucket(const StreamDesc& p, int key_bits, void* ws, int64_t* out_subs, double* out_vals,
                   int64_t cap_rows, cudaStream_t stream);

constexpr int64_t kDenseMaxCells = 16384;       // key spaces accumulated in shared memory
constexpr size_t kVecSmemMax = 64 * 1024;       // staged vector bytes per CTA
constexpr int64_t kMaxSortN = (1ll << 30) - 1;  // 30-bit counts in the look-back words

// ---------------------------------------------------------------------------
static thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    return fail(TTV_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Pinned host copies of per-call status blocks (a call's status is copied
// here at the end of its stream work, so no device memory outlives a call).
class StatusPool {
   public:
    Status* acquire() {
        std::lock_guard<std::mutex> g(mu_);
        if (free_.empty()) {
            Status* chunk = nullptr;
            if (cudaHostAlloc((void**)&chunk, 256 * sizeof(Status), cudaHostAllocDefault) != cudaSuccess) return nullptr;
            for (int i = 0; i < 256; ++i) free_.push_back(chunk + i);
        }
        Status* s = free_.back();
        free_.pop_back();
        return s;
    }
    void release(Status* s) {
        if (!s) return;
        std::lock_guard<std::mutex> g(mu_);
        free_.push_back(s);
    }

   private:
    std::mutex mu_;
    std::vector<Status*> free_;
};
static StatusPool g_status_pool;

// Library bookkeeping behind ttv_out::internal.
struct OutState {
    Status* hstatus = nullptr;
    cudaStream_t stream = nullptr;
    void* owned_subs = nullptr;
    void* owned_vals = nullptr;
    int dense_out = 0;
    int finalized = 0;
    int nonfinite = 0;          // fixed-point path met inf/nan: rerun in binary64
    int retry_sort = 0;         // bucket path gave up: rerun on the sort path
    int rc = TTV_OK;
};

// Bump allocator over one workspace block (sizes first with base == nullptr).
struct Arena {
    char* base = nullptr;
    size_t off = 0;
    template <typename T>
    T* take(size_t count) {
        off = (off + 255) & ~size_t(255);
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

int num_sms() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
    }
    return n;
}

struct Plan {
    StreamDesc desc;
    FxPlan fx{};
    int use_fx = 0;             // dense path on the fixed-point kernel
    int path = TTV_PATH_DENSE;
    int dense_out = 0;          // result written as a dense array
    int order0 = 0;
    int want_presence = 0;
    int compensated = 0;
    int key_bits = 0;
    int grid = 0;               // dense path CTAs
    int64_t cap_rows = 0, cap_vals = 0;
};

static int bits_for(uint64_t nkeys) {
    if (nkeys <= 1) return 0;
    int b = 0;
    uint64_t x = nkeys - 1;
    while (x) { ++b; x >>= 1; }
    return b;
}

static int make_plan(const ttv_tensor* t, const int32_t* modes, int32_t n_v, const void* const* vecs,
                     ttv_dtype vd, const int64_t* vec_lens, const ttv_opts* o, Plan& pl, bool force_fp64 = false,
                     bool force_sort = false) {
    if (!t || !o) return fail(TTV_ERR_ARG, "null tensor or options");
    if (t->d < 1 || t->d > TTV_MAX_D) return fail(TTV_ERR_ARG, "order d=%d outside 1..%d", t->d, TTV_MAX_D);
    if (t->nnz < 0) return fail(TTV_ERR_ARG, "negative nnz");
    if (!t->shape) return fail(TTV_ERR_ARG, "null shape");
    if (t->nnz > 0 && (!t->subs || !t->vals)) return fail(TTV_ERR_ARG, "null subs or vals");
    if (t->val_dtype != TTV_F64 && t->val_dtype != TTV_F32) return fail(TTV_ERR_ARG, "bad value dtype");
    if (vd != TTV_F64 && vd != TTV_F32) return fail(TTV_ERR_ARG, "bad vector dtype");
    if (n_v < 1 || n_v > t->d) return fail(TTV_ERR_ARG, "n_v=%d outside 1..d", n_v);
    if (!modes || !vecs) return fail(TTV_ERR_ARG, "null modes or vectors");
    if (o->fmt < TTV_OUT_SPARSE || o->fmt > TTV_OUT_AUTO) return fail(TTV_ERR_ARG, "bad output format");
    if (o->path < TTV_PATH_AUTO || o->path > TTV_PATH_BUCKET) return fail(TTV_ERR_ARG, "bad path");
    if (o->accum < TTV_ACCUM_FP64 || o->accum > TTV_ACCUM_EXACT) return fail(TTV_ERR_ARG, "bad accumulation mode");
    for (int m = 0; m < t->d; ++m)
        if (t->shape[m] < 1) return fail(TTV_ERR_ARG, "shape[%d]=%lld < 1", m, (long long)t->shape[m]);

    StreamDesc& p = pl.desc;
    memset(&p, 0, sizeof p);
    p.subs = t->subs;
    p.snz = t->stride_nz;
    p.smode = t->stride_mode;
    p.vals = t->vals;
    p.nnz = t->nnz;
    p.d = t->d;
    p.val_f32 = t->val_dtype == TTV_F32;
    p.vec_f32 = vd == TTV_F32;
    for (int m = 0; m < t->d; ++m) p.shape[m] = t->shape[m];
    for (int i = 0; i < n_v; ++i) {
        const int m = modes[i];
        if (m < 0 || m >= t->d) return fail(TTV_ERR_MODE, "mode %d outside 0..%d", m, t->d - 1);
        if ((p.smask >> m) & 1u) return fail(TTV_ERR_MODE, "mode %d repeated", m);
        if (!vecs[i]) return fail(TTV_ERR_ARG, "null vector for mode %d", m);
        if (vec_lens && vec_lens[i] != t->shape[m])
            return fail(TTV_ERR_VEC_LEN, "vector for mode %d has %lld entries, mode size is %lld", m,
                        (long long)vec_lens[i], (long long)t->shape[m]);
        p.smask |= 1u << m;
        p.vec[m] = vecs[i];
    }
    // surviving modes, row-major strides over them, key space size
    p.nr = 0;
    for (int m = 0; m < t->d; ++m)
        if (!((p.smask >> m) & 1u)) {
            p.rmode[p.nr] = m;
            p.rshape[p.nr] = t->shape[m];
            ++p.nr;
        }
    unsigned __int128 nk = 1;
    for (int j = p.nr - 1; j >= 0; --j) {
        p.kstride[p.rmode[j]] = (uint64_t)nk;
        nk *= (unsigned __int128)p.rshape[j];
        if (nk > (unsigned __int128)UINT64_MAX) return fail(TTV_ERR_KEY_OVERFLOW, "prod of surviving mode sizes exceeds 2^64-1");
    }
    p.nkeys = (uint64_t)nk;
    for (int j = 0; j < p.nr; ++j) udiv_magic((uint64_t)p.rshape[j], p.rmagic[j], p.rsh[j]);
    // vectors staged in shared memory when they fit
    int64_t vt = 0;
    for (int m = 0; m < t->d; ++m)
        if ((p.smask >> m) & 1u) { p.voff[m] = (int32_t)std::min<int64_t>(vt, INT32_MAX); vt += t->shape[m]; }
    p.vtotal = (int32_t)std::min<int64_t>(vt, INT32_MAX);
    p.vec_smem = (size_t)vt * sizeof(double) <= kVecSmemMax;

    pl.order0 = p.nr == 0;
    pl.compensated = o->accum == TTV_ACCUM_COMPENSATED;
    pl.dense_out = o->fmt == TTV_OUT_DENSE || pl.order0;
    pl.key_bits = bits_for(p.nkeys);

    int path = o->path;
    const bool dense_ok = (int64_t)p.nkeys <= kDenseMaxCells;
    const bool want_exact = o->accum == TTV_ACCUM_EXACT || o->deterministic;
    if (path == TTV_PATH_AUTO) {
        if (dense_ok || pl.order0) path = TTV_PATH_DENSE;
        else path = TTV_PATH_SORT;   // the bucket path is selectable; it does not beat the sort path yet
    }
    if (path == TTV_PATH_HASH) path = TTV_PATH_SORT;   // not built yet: sort
    if (path == TTV_PATH_BUCKET && (pl.dense_out || !bucket_applicable(p))) path = TTV_PATH_SORT;
    if (force_sort && path == TTV_PATH_BUCKET) path = TTV_PATH_SORT;
    if (path == TTV_PATH_DENSE && !dense_ok) return fail(TTV_ERR_UNSUPPORTED, "dense path needs prod shape[R] <= %lld", (long long)kDenseMaxCells);
    if (path == TTV_PATH_DENSE) {
        // exact fixed point when asked for determinism (binary64 shared-memory
        // atomics are order dependent); binary64 atomics otherwise
        const int presence = !pl.dense_out;
        pl.fx = plan_dense_fx(p, presence, num_sms());
        pl.use_fx = want_exact && pl.fx.ok && !force_fp64 && p.nnz > 0;
        if (want_exact && !pl.fx.ok && !pl.order0 && p.nnz > 0) path = TTV_PATH_SORT;
    }
    if ((path == TTV_PATH_SORT || path == TTV_PATH_BUCKET) && p.nnz > kMaxSortN)
        return fail(TTV_ERR_UNSUPPORTED, "sparse accumulation supports nnz < 2^30");
    pl.path = path;
    pl.want_presence = (path == TTV_PATH_DENSE) && !pl.dense_out;

    if (pl.dense_out) {
        pl.cap_rows = 0;
        pl.cap_vals = (int64_t)p.nkeys;
    } else {
        const int64_t r = (int64_t)std::min<uint64_t>((uint64_t)std::max<int64_t>(p.nnz, 0), p.nkeys);
        pl.cap_rows = r;
        pl.cap_vals = r;
    }
    if (path == TTV_PATH_DENSE && !pl.use_fx) pl.grid = dense_grid(p, pl.want_presence);
    return TTV_OK;
}

// Validated stream descriptor of a dense-result call (the allocation-free
// entry point in ttv_noalloc.cu builds its launch from this).
int plan_dense_desc(const ttv_tensor* t, const int32_t* modes, int32_t n_v, const void* const* vecs, ttv_dtype vd,
                    const int64_t* vec_lens, StreamDesc* out) {
    g_err.clear();
    ttv_opts o;
    memset(&o, 0, sizeof o);
    o.fmt = TTV_OUT_DENSE;
    o.path = TTV_PATH_DENSE;
    Plan pl;
    int rc = make_plan(t, modes, n_v, vecs, vd, vec_lens, &o, pl);
    if (rc != TTV_OK) return rc;
    *out = pl.desc;
    return TTV_OK;
}

// Workspace layout; with a.base == nullptr it only measures.
struct WsPtrs {
    Status* status;
    // bucket
    void* bucket_ws;
    // dense
    void* fx_ws;
    double* partials;
    uint32_t* pres_partials;
    double* cell_vals;
    uint32_t* cell_flags;
    // sort
    SortBuffers sb;
    uint32_t* seg_start;
    unsigned long long* seg_lookback;
    uint32_t* seg_ticket;
    uint32_t* long_list;
};

static void layout(const Plan& pl, Arena& a, WsPtrs& w) {
    memset(&w, 0, sizeof w);
    const StreamDesc& p = pl.desc;
    w.status = a.take<Status>(1);
    if (pl.path == TTV_PATH_DENSE) {
        const int64_t P = (int64_t)p.nkeys;
        if (pl.use_fx) {
            w.fx_ws = a.take<char>(dense_fx_workspace(p, pl.fx, pl.want_presence));
        } else {
            w.partials = a.take<double>((size_t)pl.grid * P);
            if (pl.want_presence) w.pres_partials = a.take<uint32_t>((size_t)pl.grid * ((P + 31) / 32));
        }
        if (pl.want_presence) {
            w.cell_vals = a.take<double>(P);
            w.cell_flags = a.take<uint32_t>(P);
        }
    } else if (pl.path == TTV_PATH_BUCKET) {
        w.bucket_ws = a.take<char>(bucket_workspace_bytes(p.nnz, pl.key_bits));
    } else {
        const int64_t n = std::max<int64_t>(p.nnz, 1);
        const int npass = (pl.key_bits + 7) / 8;
        const int64_t ntiles = (n + 4095) / 4096;
        w.sb.keys[0] = a.take<uint64_t>(n);
        w.sb.keys[1] = a.take<uint64_t>(n);
        w.sb.vals[0] = a.take<double>(n);
        w.sb.vals[1] = a.take<double>(n);
        w.sb.hist = a.take<uint32_t>((size_t)std::max(npass, 1) * 256);
        w.sb.lookback = a.take<uint32_t>((size_t)std::max(npass, 1) * ntiles * 256);
        w.sb.tickets = a.take<uint32_t>(64);
        w.sb.npass = npass;
        w.sb.ntiles = ntiles;
        w.seg_start = a.take<uint32_t>(n + 1);
        w.seg_lookback = a.take<unsigned long long>(ntiles);
        w.seg_ticket = a.take<uint32_t>(64);
        w.long_list = a.take<uint32_t>(n);
    }
    a.off = (a.off + 255) & ~size_t(255);
}

static size_t workspace_bytes(const Plan& pl) {
    Arena a;
    WsPtrs w;
    layout(pl, a, w);
    return a.off;
}

static int finalize(ttv_out* out) {
    OutState* s = static_cast<OutState*>(out->internal);
    if (!s) return fail(TTV_ERR_ARG, "result has no pending call");
    if (s->finalized) return s->rc;
    cudaError_t e = cudaStreamSynchronize(s->stream);
    s->finalized = 1;
    if (e != cudaSuccess) return s->rc = cuda_fail(e, "stream synchronize");
    const Status& h = *s->hstatus;
    if (!s->dense_out) out->nnz = (int64_t)h.nnz_out;
    if (h.err & kErrSubscript) return s->rc = fail(TTV_ERR_SUBSCRIPT, "a subscript is outside its mode");
    if (h.err & kErrTimeout) return s->rc = fail(TTV_ERR_TIMEOUT, "a bounded device wait ran out");
    if (h.err & kErrCapacity) return s->rc = fail(TTV_ERR_CAPACITY, "result (%llu rows) exceeds the output buffer", (unsigned long long)h.nnz_out);
    if (h.err & kErrInternal) return s->rc = fail(TTV_ERR_CUDA, "internal device check failed");
    if (h.err & kErrRetry) {
        s->retry_sort = 1;
        return s->rc = fail(TTV_ERR_UNSUPPORTED, "bucket path could not place every pair");
    }
    if (h.err & kErrNonFinite) {
        s->nonfinite = 1;
        return s->rc = fail(TTV_ERR_UNSUPPORTED, "non-finite input on the fixed-point dense path");
    }
    return s->rc = TTV_OK;
}

static int execute(const Plan& pl, ttv_out* out, const ttv_opts* o, cudaStream_t stream) {
    const StreamDesc& p0 = pl.desc;
    // result bookkeeping
    if (out->internal) return fail(TTV_ERR_ARG, "ttv_out reused without ttv_out_free");
    OutState* st = new OutState();
    st->stream = stream;
    st->dense_out = pl.dense_out;
    out->internal = st;
    out->order = p0.nr;
    for (int j = 0; j < TTV_MAX_D; ++j) out->shape[j] = j < p0.nr ? p0.rshape[j] : 0;
    out->dtype = TTV_F64;
    out->is_dense = pl.dense_out && !pl.order0;
    out->nnz = pl.dense_out ? (int64_t)p0.nkeys : 0;
    st->hstatus = g_status_pool.acquire();
    if (!st->hstatus) return fail(TTV_ERR_NOMEM, "pinned status allocation failed");
    memset(st->hstatus, 0, sizeof(Status));

    cudaError_t e;
    if (!out->vals) {
        e = cudaMallocAsync(&out->vals, (size_t)std::max<int64_t>(pl.cap_vals, 1) * sizeof(double), stream);
        if (e != cudaSuccess) { out->vals = nullptr; return cuda_fail(e, "output allocation"); }
        st->owned_vals = out->vals;
        out->vals_capacity = pl.cap_vals;
        if (!pl.dense_out && p0.nr > 0) {
            e = cudaMallocAsync((void**)&out->subs, (size_t)std::max<int64_t>(pl.cap_rows, 1) * p0.nr * sizeof(int64_t), stream);
            if (e != cudaSuccess) { out->subs = nullptr; return cuda_fail(e, "output allocation"); }
            st->owned_subs = out->subs;
            out->subs_capacity = pl.cap_rows;
        }
    } else {
        if (pl.dense_out && out->vals_capacity < pl.cap_vals)
            return fail(TTV_ERR_CAPACITY, "dense result needs %lld values", (long long)pl.cap_vals);
        if (!pl.dense_out && p0.nr > 0 && !out->subs) return fail(TTV_ERR_ARG, "caller buffers need subs too");
    }
    const int64_t cap_rows = pl.dense_out ? 0 : std::min(out->subs_capacity, out->vals_capacity);
    const int64_t cap_rows_eff = (!pl.dense_out && p0.nr == 0) ? out->vals_capacity : cap_rows;

    // workspace
    const size_t need = workspace_bytes(pl);
    void* ws = nullptr;
    bool own_ws = false;
    if (o->workspace && o->workspace_bytes >= need) {
        ws = o->workspace;
    } else {
        e = cudaMallocAsync(&ws, need, stream);
        if (e != cudaSuccess) return cuda_fail(e, "workspace allocation");
        own_ws = true;
    }
    Arena a;
    a.base = static_cast<char*>(ws);
    WsPtrs w;
    layout(pl, a, w);
    StreamDesc p = p0;
    p.status = w.status;
    cudaMemsetAsync(w.status, 0, sizeof(Status), stream);

    double* ovals = static_cast<double*>(out->vals);
    if (p.nnz == 0) {
        // empty tensor: zeros when dense, a zero scalar for order 0, else no rows
        if (pl.dense_out) cudaMemsetAsync(ovals, 0, (size_t)std::max<int64_t>(pl.cap_vals, 1) * sizeof(double), stream);
    } else if (pl.path == TTV_PATH_DENSE) {
        double* cell_vals = pl.want_presence ? w.cell_vals : ovals;
        if (pl.use_fx)
            launch_dense_fx(p, pl.fx, pl.want_presence, w.fx_ws, cell_vals, w.cell_flags, stream);
        else
            launch_dense(p, pl.want_presence, pl.compensated, pl.grid, w.partials, w.pres_partials, cell_vals,
                         w.cell_flags, stream);
        if (pl.want_presence) launch_compact_cells(p, w.cell_vals, w.cell_flags, cap_rows_eff, out->subs, ovals, stream);
    } else if (pl.path == TTV_PATH_BUCKET) {
        launch_bucket(p, pl.key_bits, w.bucket_ws, out->subs, ovals, cap_rows_eff, stream);
    } else {
        launch_keys_terms(p, w.sb.keys[0], w.sb.vals[0], stream);
        SortBuffers sb = w.sb;
        const int cur = radix_sort_pairs(sb, p.nnz, pl.key_bits, w.status, stream);
        if (pl.dense_out) cudaMemsetAsync(ovals, 0, (size_t)pl.cap_vals * sizeof(double), stream);
        SegOut so{out->subs, ovals, cap_rows_eff, pl.dense_out, pl.compensated};
        launch_seg_reduce(sb.keys[cur], sb.vals[cur], p.nnz, w.seg_start, w.seg_lookback, w.seg_ticket,
                          w.long_list, p, so, w.status, stream);
    }
    if (pl.order0) {
        // scalar result: nnz 1 whatever the input
        st->dense_out = 1;
        out->nnz = 1;
    }
    e = cudaMemcpyAsync(st->hstatus, w.status, sizeof(Status), cudaMemcpyDeviceToHost, stream);
    if (own_ws) cudaFreeAsync(ws, stream);
    if (e != cudaSuccess) return cuda_fail(e, "status copy");
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    if (o->async) return TTV_OK;
    return finalize(out);
}

static void init_once() {
    static std::once_flag f;
    std::call_once(f, [] {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t thr = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
    });
}

}  // namespace ttv

using namespace ttv;

extern "C" {

void ttv_opts_init(ttv_opts* o) {
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->fmt = TTV_OUT_SPARSE;
    o->path = TTV_PATH_AUTO;
    o->accum = TTV_ACCUM_FP64;
    o->deterministic = 0;
    o->async = 0;
}

const char* ttv_last_error(void) { return g_err.c_str(); }

int ttv_multi_checked(const ttv_tensor* t, const int32_t* modes, int32_t n_v, const void* const* vecs,
                      const int64_t* vec_lens, ttv_dtype v_dtype, ttv_out* out, const ttv_opts* opts,
                      ttv_stream_t stream) {
    g_err.clear();
    if (!out) return fail(TTV_ERR_ARG, "null result");
    ttv_opts def;
    ttv_opts_init(&def);
    const ttv_opts* o = opts ? opts : &def;
    init_once();
    Plan pl;
    int rc = make_plan(t, modes, n_v, vecs, v_dtype, vec_lens, o, pl);
    if (rc != TTV_OK) return rc;
    rc = execute(pl, out, o, reinterpret_cast<cudaStream_t>(stream));
    OutState* s = static_cast<OutState*>(out->internal);
    if (rc == TTV_ERR_UNSUPPORTED && s && (s->nonfinite || s->retry_sort)) {
        // inf or nan in the input: the binary64 kernel propagates them like the
        // definition; a bucket overflow: the sort path has no capacity limits
        Plan p2;
        rc = make_plan(t, modes, n_v, vecs, v_dtype, vec_lens, o, p2, /*force_fp64=*/s->nonfinite != 0,
                       /*force_sort=*/s->retry_sort != 0);
        if (rc != TTV_OK) return rc;
        void* keep_subs = s->owned_subs;
        void* keep_vals = s->owned_vals;
        s->owned_subs = s->owned_vals = nullptr;
        g_status_pool.release(s->hstatus);
        delete s;
        out->internal = nullptr;
        rc = execute(p2, out, o, reinterpret_cast<cudaStream_t>(stream));
        OutState* s2 = static_cast<OutState*>(out->internal);
        if (s2) {
            s2->owned_subs = keep_subs;
            s2->owned_vals = keep_vals;
        }
    }
    return rc;
}

int ttv_multi(const ttv_tensor* t, const int32_t* modes, int32_t n_v, const void* const* vecs, ttv_dtype v_dtype,
              ttv_out* out, const ttv_opts* opts, ttv_stream_t stream) {
    return ttv_multi_checked(t, modes, n_v, vecs, nullptr, v_dtype, out, opts, stream);
}

int ttv_single(const ttv_tensor* t, int32_t mode, const void* v, ttv_dtype v_dtype, ttv_out* out,
               const ttv_opts* opts, ttv_stream_t stream) {
    const void* vecs[1] = {v};
    return ttv_multi_checked(t, &mode, 1, vecs, nullptr, v_dtype, out, opts, stream);
}

int ttv_out_capacity(const ttv_tensor* t, const int32_t* modes, int32_t n_v, const ttv_opts* opts, int64_t* rows,
                     int64_t* values) {
    g_err.clear();
    if (!rows || !values) return fail(TTV_ERR_ARG, "null result pointers");
    ttv_opts def;
    ttv_opts_init(&def);
    const ttv_opts* o = opts ? opts : &def;
    std::vector<const void*> dummy((size_t)std::max(n_v, 0), reinterpret_cast<const void*>(0x10));
    Plan pl;
    int rc = make_plan(t, modes, n_v, dummy.data(), TTV_F64, nullptr, o, pl);
    if (rc != TTV_OK) return rc;
    *rows = pl.cap_rows;
    *values = std::max<int64_t>(pl.cap_vals, 1);
    return TTV_OK;
}

int ttv_workspace_size(const ttv_tensor* t, const int32_t* modes, int32_t n_v, ttv_dtype v_dtype,
                       const ttv_opts* opts, size_t* bytes) {
    g_err.clear();
    if (!bytes) return fail(TTV_ERR_ARG, "null bytes");
    ttv_opts def;
    ttv_opts_init(&def);
    const ttv_opts* o = opts ? opts : &def;
    std::vector<const void*> dummy((size_t)std::max(n_v, 0), reinterpret_cast<const void*>(0x10));
    Plan pl;
    int rc = make_plan(t, modes, n_v, dummy.data(), v_dtype, nullptr, o, pl);
    if (rc != TTV_OK) return rc;
    *bytes = workspace_bytes(pl);
    return TTV_OK;
}

int ttv_out_sync(ttv_out* out) {
    if (!out) return fail(TTV_ERR_ARG, "null result");
    return finalize(out);
}

void ttv_out_free(ttv_out* out) {
    if (!out || !out->internal) return;
    OutState* s = static_cast<OutState*>(out->internal);
    if (s->owned_subs) { cudaFreeAsync(s->owned_subs, s->stream); out->subs = nullptr; }
    if (s->owned_vals) { cudaFreeAsync(s->owned_vals, s->stream); out->vals = nullptr; }
    if (!s->finalized) cudaStreamSynchronize(s->stream);
    g_status_pool.release(s->hstatus);
    delete s;
    out->internal = nullptr;
}

}  // extern "C"
