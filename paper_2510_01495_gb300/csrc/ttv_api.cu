// ttv_api.cu -- the C ABI (include/ttv.h): argument checks, planning of the
// accumulation path, workspace layout, launches and the status read-back.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "ttv_internal.cuh"

namespace ttv {

// An NVTX range around one public call, so that a timeline (nsys, or ncu's
// NVTX filters) shows which TTV, batch, preparation or run each kernel
// belongs to; without an attached tool a push/pop costs a few nanoseconds.
struct NvtxScope {
    explicit NvtxScope(const char* name) { nvtxRangePushA(name); }
    ~NvtxScope() { nvtxRangePop(); }
    NvtxScope(const NvtxScope&) = delete;
    NvtxScope& operator=(const NvtxScope&) = delete;
};

// kernels in ttv_stream.cu / ttv_sort.cu
void launch_keys_terms(const StreamDesc& p, uint64_t* keys, double* terms, cudaStream_t stream);
bool keys_terms_vec_applicable(const StreamDesc& p, int npass);
void launch_keys_terms_vec(const StreamDesc& p, uint64_t* keys, double* terms, int npass, uint32_t* hist,
                           cudaStream_t stream);
size_t dense_smem_bytes(const StreamDesc& p, int want_presence);
int dense_grid(const StreamDesc& p, int want_presence);
void launch_dense(const StreamDesc& p, int want_presence, int compensated, int G, double* partials,
                  uint32_t* pres_partials, double* cell_vals, uint32_t* cell_flags, cudaStream_t stream);
void launch_compact_cells(const StreamDesc& p, const double* cell_vals, const uint32_t* cell_flags, int64_t cap_rows,
                          int64_t* out_subs, double* out_vals, cudaStream_t stream);
size_t rbk_state_bytes(int64_t n);
void launch_reduce_by_key_prepared(const uint8_t* head_bits, const uint64_t* row_keys, const PrepTerms& terms,
                                   int64_t n, void* state, const StreamDesc& p, const SegOut& o, Status* st,
                                   cudaStream_t stream);
void launch_prep_heads(const uint64_t* keys, int64_t n, uint32_t* bits, cudaStream_t stream);
void launch_run_keys(const uint64_t* keys, const double* vals, int64_t n, void* state, uint64_t* row_keys,
                     int64_t cap_rows, const StreamDesc& p, Status* st, cudaStream_t stream);
void launch_prep_keys(const StreamDesc& p, uint64_t* keys, double* idx, cudaStream_t stream);
void launch_prep_gather(const StreamDesc& p, const double* idx_sorted, void* vals_out, const PrepTerms& subs,
                        cudaStream_t stream);
void launch_prep_count(const uint64_t* keys, int64_t n, unsigned long long* count, cudaStream_t stream);
void launch_coo_to_dense(const int64_t* subs, const double* vals, int64_t n, int order, const int64_t* shape,
                         double* dense, int64_t ncells, cudaStream_t stream);
size_t dot_workspace_bytes(int64_t n);
void launch_dot(const void* x, const void* y, int64_t n, bool f32, double* out, void* ws, cudaStream_t stream);
bool matvec_layout_ok(int64_t n1, int64_t n2, int64_t sr, int64_t sc);
size_t matvec_workspace_bytes(int64_t n1, int64_t n2, int64_t sr, int64_t sc);
void launch_matvec(const void* A, int64_t n1, int64_t n2, int64_t sr, int64_t sc, bool f32, const void* x,
                   double* y, void* ws, cudaStream_t stream);
int64_t mttkrp_nchunks(int64_t n);
size_t mttkrp_workspace_bytes(int64_t n, int32_t R);
void launch_mttkrp_chunk_counts(const uint32_t* bits, int64_t n, uint32_t* counts, cudaStream_t stream);
void launch_mttkrp(const void* vals, int val_f32, int n_v, const int32_t* const* subs, const double* const* factors,
                   const uint32_t* bits, const uint64_t* row_keys, const uint32_t* chunk_base,
                   const int32_t* next_head, int64_t n, int32_t R, int64_t rows, double* out, void* ws,
                   cudaStream_t stream);
void launch_reduce_by_key(const uint64_t* keys, const double* vals, int64_t n, void* state, const StreamDesc& p,
                          const SegOut& o, Status* st, cudaStream_t stream);

bool bucket_applicable(const StreamDesc& p);
bool hash_applicable(const StreamDesc& p);
size_t hash_workspace_bytes(const StreamDesc& p, int dense_out, int key_bits);
void launch_hash(const StreamDesc& p, int dense_out, int key_bits, void* ws, int64_t* out_subs, double* out_vals,
                 int64_t cap_rows, cudaStream_t stream);
size_t bucket_workspace_bytes(int64_t nnz, int key_bits);
void launch_bucket(const StreamDesc& p, int key_bits, void* ws, int64_t* out_subs, double* out_vals,
                   int64_t cap_rows, cudaStream_t stream);

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
    // Ensures n free slots (pinned allocations are not allowed inside a capture).
    bool reserve(size_t n) {
        std::lock_guard<std::mutex> g(mu_);
        while (free_.size() < n) {
            Status* chunk = nullptr;
            if (cudaHostAlloc((void**)&chunk, 256 * sizeof(Status), cudaHostAllocDefault) != cudaSuccess) return false;
            for (int i = 0; i < 256; ++i) free_.push_back(chunk + i);
        }
        return true;
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
    int borrowed_status = 0;    // status slot belongs to a cached batch graph
    int auto_fmt = 0;           // TTV_OUT_AUTO: densify at finalisation when more than half full
    uint64_t nkeys = 0;         // prod(shape[R])
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

// ---- autotuner record -------------------------------------------------------
// Problems fall into classes by order, surviving modes, result format, value
// and vector types, subscript layout and the binary orders of magnitude of
// nnz and of the key space; ttv_autotune stores the fastest (path, CTAs per
// SM) of a class and AUTO uses it for every problem of that class.
struct TuneRec {
    int32_t path;
    int32_t ctas;
    int32_t items;
    double ms;
};
static std::mutex g_tune_mu;
static std::vector<std::pair<uint64_t, TuneRec>> g_tune;
static thread_local int t_force_path = -1;   // set by the autotuner's trial runs
static thread_local int t_force_ctas = 0;
static thread_local int t_force_items = 0;

static uint64_t tune_key(const StreamDesc& p, int dense_out) {
    const uint64_t layout = p.snz == 1 ? 1 : (p.smode == 1 ? 0 : 2);
    const uint64_t lg_nnz = (uint64_t)bits_for((uint64_t)std::max<int64_t>(p.nnz, 1));
    const uint64_t lg_keys = (uint64_t)bits_for(p.nkeys);
    return (uint64_t)p.d | (uint64_t)p.nr << 4 | (uint64_t)(dense_out != 0) << 8 | (uint64_t)(p.val_f32 != 0) << 9 |
           (uint64_t)(p.vec_f32 != 0) << 10 | layout << 11 | lg_nnz << 16 | lg_keys << 24;
}

static bool tune_lookup(uint64_t key, TuneRec& r) {
    std::lock_guard<std::mutex> g(g_tune_mu);
    for (auto& e : g_tune)
        if (e.first == key) { r = e.second; return true; }
    return false;
}

static void tune_record(uint64_t key, const TuneRec& r) {
    std::lock_guard<std::mutex> g(g_tune_mu);
    for (auto& e : g_tune)
        if (e.first == key) { e.second = r; return; }
    g_tune.emplace_back(key, r);
}

bool hash_direct(const StreamDesc& p);

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
    p.ctas_per_sm = 0;
    p.items = 0;
    if (t_force_path >= 0) {
        path = t_force_path;
        p.ctas_per_sm = t_force_ctas;
        p.items = t_force_items;
    } else if (path == TTV_PATH_AUTO && !want_exact && !pl.compensated) {
        TuneRec r;
        if (tune_lookup(tune_key(p, pl.dense_out), r) && (r.path != TTV_PATH_DENSE || dense_ok || pl.order0)) {
            path = r.path;
            p.ctas_per_sm = r.ctas;
            p.items = r.items;
        }
    }
    if (path == TTV_PATH_AUTO) {
        // Without a tuning record: the shared-memory dense accumulator when
        // the key space fits; a direct-indexed table when the key space is
        // no larger than nnz (measured 1.9-2.5x faster than sorting there);
        // otherwise the sort.  The bucket path is selectable but has not
        // beaten the sort path on any measured class.
        if (dense_ok || pl.order0) path = TTV_PATH_DENSE;
        else if (!want_exact && !pl.compensated && p.nkeys <= (uint64_t)p.nnz && hash_direct(p)) path = TTV_PATH_HASH;
        else path = TTV_PATH_SORT;
    }
    // The hash path sums in atomic arrival order: deterministic and
    // compensated requests go to the sort path.
    if (path == TTV_PATH_HASH && (want_exact || pl.compensated || !hash_applicable(p))) path = TTV_PATH_SORT;
    // The partition path sums in arrival order: deterministic and compensated
    // requests go to the sort path, like dense results and inputs it does not take.
    if (path == TTV_PATH_BUCKET && (pl.dense_out || want_exact || pl.compensated || !bucket_applicable(p)))
        path = TTV_PATH_SORT;
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
    if ((path == TTV_PATH_SORT || path == TTV_PATH_BUCKET || path == TTV_PATH_HASH) && p.nnz > kMaxSortN)
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
    // bucket, hash
    void* bucket_ws;
    void* hash_ws;
    // dense
    void* fx_ws;
    double* partials;
    uint32_t* pres_partials;
    double* cell_vals;
    uint32_t* cell_flags;
    // sort
    SortBuffers sb;
    void* rbk_state;
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
    } else if (pl.path == TTV_PATH_HASH) {
        w.hash_ws = a.take<char>(hash_workspace_bytes(p, pl.dense_out, pl.key_bits));
    } else {
        const int64_t n = std::max<int64_t>(p.nnz, 1);
        const int npass = (pl.key_bits + 7) / 8;
        const int64_t ntiles = sort_tiles(n);
        w.sb.keys[0] = a.take<uint64_t>(n);
        w.sb.keys[1] = a.take<uint64_t>(n);
        w.sb.vals[0] = a.take<double>(n);
        w.sb.vals[1] = a.take<double>(n);
        w.sb.hist = a.take<uint32_t>((size_t)std::max(npass, 1) * 256);
        w.sb.lookback = a.take<uint32_t>((size_t)std::max(npass, 1) * ntiles * 256);
        w.sb.tickets = a.take<uint32_t>(64);
        w.sb.npass = npass;
        w.sb.ntiles = ntiles;
        w.rbk_state = a.take<char>(rbk_state_bytes(n));
    }
    a.off = (a.off + 255) & ~size_t(255);
}

static size_t workspace_bytes(const Plan& pl) {
    Arena a;
    WsPtrs w;
    layout(pl, a, w);
    return a.off;
}

// The device address of the call's pinned status block, or nullptr where the
// status must stay in device memory: inside a graph capture (the graph
// keeps its own reset and copy) or for a batch's borrowed block.
static Status* direct_status(OutState* st, cudaStream_t stream) {
    if (st->borrowed_status) return nullptr;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    void* dp = nullptr;
    if (cudaStreamIsCapturing(stream, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone &&
        cudaHostGetDevicePointer(&dp, st->hstatus, 0) == cudaSuccess && dp)
        return static_cast<Status*>(dp);
    cudaGetLastError();
    return nullptr;
}

// pyttb's conversion (Sec. 3.3): a sparse result with more than half of its
// cells present becomes a dense array.  Library-owned results move to a new
// dense buffer; a caller's value buffer is reused when it holds every cell.
// When neither is possible (no room for the dense array or its scratch) the
// result stays sparse, as it was computed.
static int auto_to_dense(ttv_out* out, OutState* s) {
    const int64_t n = out->nnz, nk = (int64_t)s->nkeys;
    cudaStream_t stream = s->stream;
    cudaError_t e = cudaSuccess;
    if (s->owned_vals) {
        double* dense = nullptr;
        e = cudaMallocAsync((void**)&dense, (size_t)nk * sizeof(double), stream);
        if (e != cudaSuccess) {       // no room for the dense form: the sparse result stands
            cudaGetLastError();
            return TTV_OK;
        }
        launch_coo_to_dense(out->subs, static_cast<const double*>(out->vals), n, out->order, out->shape, dense,
                            nk, stream);
        cudaFreeAsync(s->owned_vals, stream);
        out->vals = dense;
        s->owned_vals = dense;
        out->vals_capacity = nk;
    } else if (out->vals_capacity >= nk) {
        double* tmp = nullptr;
        e = cudaMallocAsync((void**)&tmp, (size_t)std::max<int64_t>(n, 1) * sizeof(double), stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return TTV_OK;
        }
        cudaMemcpyAsync(tmp, out->vals, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, stream);
        launch_coo_to_dense(out->subs, tmp, n, out->order, out->shape, static_cast<double*>(out->vals), nk, stream);
        cudaFreeAsync(tmp, stream);
    } else {
        return TTV_OK;
    }
    if (s->owned_subs) {
        cudaFreeAsync(s->owned_subs, stream);
        s->owned_subs = nullptr;
        out->subs = nullptr;
    }
    e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(e, "dense conversion");
    out->is_dense = 1;
    out->nnz = nk;
    s->dense_out = 1;
    return TTV_OK;
}

// synced: the caller has just synchronised the result's stream (a batch
// finalises hundreds of results after one synchronisation).
static int finalize(ttv_out* out, bool synced = false) {
    OutState* s = static_cast<OutState*>(out->internal);
    if (!s) return fail(TTV_ERR_ARG, "result has no pending call");
    if (s->finalized) return s->rc;
    cudaError_t e = synced ? cudaSuccess : cudaStreamSynchronize(s->stream);
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
        return s->rc = fail(TTV_ERR_UNSUPPORTED, "partition path: a bucket outgrew its sampled capacity");
    }
    if (h.err & kErrNonFinite) {
        s->nonfinite = 1;
        return s->rc = fail(TTV_ERR_UNSUPPORTED, "non-finite input on the fixed-point dense path");
    }
    if (s->auto_fmt && (double)out->nnz > 0.5 * (double)s->nkeys) return s->rc = auto_to_dense(out, s);
    return s->rc = TTV_OK;
}

static int execute(const Plan& pl, ttv_out* out, const ttv_opts* o, cudaStream_t stream) {
    const StreamDesc& p0 = pl.desc;
    // result bookkeeping
    if (out->internal) return fail(TTV_ERR_ARG, "ttv_out reused without ttv_out_free");
    OutState* st = new OutState();
    st->stream = stream;
    st->dense_out = pl.dense_out;
    st->auto_fmt = o->fmt == TTV_OUT_AUTO && !pl.dense_out && !pl.order0;
    st->nkeys = p0.nkeys;
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
    // Paths whose kernels touch the status only rarely (error flags) or once
    // (the result count) write it straight into the call's pinned status
    // block (zeroed on the host above): no reset and no copy on the stream.
    const bool light_status = (pl.path == TTV_PATH_DENSE && !pl.use_fx && !pl.want_presence) ||
                              pl.path == TTV_PATH_SORT;
    Status* dstat = (light_status && p.nnz > 0) ? direct_status(st, stream) : nullptr;
    const bool direct_st = dstat != nullptr;
    if (direct_st) p.status = dstat;
    else cudaMemsetAsync(w.status, 0, sizeof(Status), stream);

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
    } else if (pl.path == TTV_PATH_HASH) {
        launch_hash(p, pl.dense_out, pl.key_bits, w.hash_ws, out->subs, ovals, cap_rows_eff, stream);
    } else {
        SortBuffers sb = w.sb;
        const int npass = (pl.key_bits + 7) / 8;
        const bool vec = npass > 0 && p.nnz > 1 && keys_terms_vec_applicable(p, npass);
        if (vec) {
            // keys, terms and the digit histograms of every pass in one read
            cudaMemsetAsync(sb.hist, 0, (size_t)npass * 256 * sizeof(uint32_t), stream);
            launch_keys_terms_vec(p, sb.keys[0], sb.vals[0], npass, sb.hist, stream);
        } else {
            launch_keys_terms(p, sb.keys[0], sb.vals[0], stream);
        }
        const int cur = radix_sort_pairs(sb, p.nnz, pl.key_bits, p.status, stream, nullptr, vec);
        if (pl.dense_out) cudaMemsetAsync(ovals, 0, (size_t)pl.cap_vals * sizeof(double), stream);
        SegOut so{out->subs, ovals, cap_rows_eff, pl.dense_out, pl.compensated};
        launch_reduce_by_key(sb.keys[cur], sb.vals[cur], p.nnz, w.rbk_state, p, so, p.status, stream);
    }
    if (pl.order0) {
        // scalar result: nnz 1 whatever the input
        st->dense_out = 1;
        out->nnz = 1;
    }
    e = direct_st ? cudaSuccess
                  : cudaMemcpyAsync(st->hstatus, w.status, sizeof(Status), cudaMemcpyDeviceToHost, stream);
    if (own_ws) cudaFreeAsync(ws, stream);
    if (e != cudaSuccess) return cuda_fail(e, "status copy");
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    if (o->async) return TTV_OK;
    return finalize(out);
}

// ---- prepared tensors ------------------------------------------------------

}  // namespace ttv

struct ttv_prepared {
    ttv::Plan plan;                   // shape, surviving modes, key strides, delinearisation
    int32_t n_v = 0;
    int32_t arg_of[TTV_MAX_D] = {0};  // j-th contracted mode (increasing) -> caller's vector index
    int64_t nnz = 0;
    int64_t nnz_out = 0;              // distinct keys (result rows)
    uint32_t* head_bits = nullptr;    // bit i set: nonzero i (key order) starts a result row
    uint64_t* row_keys = nullptr;     // key of every result row
    void* vals = nullptr;             // values in key order
    int32_t* subs[TTV_MAX_D] = {nullptr};
    uint32_t* chunk_base = nullptr;   // one surviving mode: heads before each 128-nonzero chunk (MTTKRP)
    int32_t* next_head = nullptr;     // first chunk after c that holds a head (MTTKRP)
    size_t bytes = 0;
};

namespace ttv {

static size_t prepared_ws_bytes(const ttv_prepared* h) {
    Arena a;
    a.take<Status>(1);
    a.take<char>(rbk_state_bytes(h->nnz));
    a.off = (a.off + 255) & ~size_t(255);
    return a.off;
}

static int execute_prepared(const ttv_prepared* h, const void* const* vecs, ttv_dtype vd, ttv_out* out,
                            const ttv_opts* o, cudaStream_t stream) {
    const StreamDesc& p0 = h->plan.desc;
    const bool order0 = h->plan.order0;
    bool dense_out = o->fmt == TTV_OUT_DENSE || order0;
    if (o->fmt == TTV_OUT_AUTO && (double)h->nnz_out > 0.5 * (double)p0.nkeys) dense_out = true;
    if (dense_out && !order0 && (double)p0.nkeys * 8.0 > 64e9)
        return fail(TTV_ERR_UNSUPPORTED, "dense result of %llu cells", (unsigned long long)p0.nkeys);
    if (out->internal) return fail(TTV_ERR_ARG, "ttv_out reused without ttv_out_free");
    OutState* st = new OutState();
    st->stream = stream;
    st->dense_out = dense_out;
    out->internal = st;
    out->order = p0.nr;
    for (int j = 0; j < TTV_MAX_D; ++j) out->shape[j] = j < p0.nr ? p0.rshape[j] : 0;
    out->dtype = TTV_F64;
    out->is_dense = dense_out && !order0;
    out->nnz = dense_out ? (int64_t)p0.nkeys : 0;
    st->hstatus = g_status_pool.acquire();
    if (!st->hstatus) return fail(TTV_ERR_NOMEM, "pinned status allocation failed");
    memset(st->hstatus, 0, sizeof(Status));
    const int64_t cap_vals = dense_out ? (int64_t)p0.nkeys : h->nnz_out;
    cudaError_t e;
    if (!out->vals) {
        e = cudaMallocAsync(&out->vals, (size_t)std::max<int64_t>(cap_vals, 1) * sizeof(double), stream);
        if (e != cudaSuccess) { out->vals = nullptr; return cuda_fail(e, "output allocation"); }
        st->owned_vals = out->vals;
        out->vals_capacity = cap_vals;
        if (!dense_out && p0.nr > 0) {
            e = cudaMallocAsync((void**)&out->subs, (size_t)std::max<int64_t>(h->nnz_out, 1) * p0.nr * sizeof(int64_t),
                                stream);
            if (e != cudaSuccess) { out->subs = nullptr; return cuda_fail(e, "output allocation"); }
            st->owned_subs = out->subs;
            out->subs_capacity = h->nnz_out;
        }
    } else {
        if (dense_out && out->vals_capacity < cap_vals)
            return fail(TTV_ERR_CAPACITY, "dense result needs %lld values", (long long)cap_vals);
        if (!dense_out && p0.nr > 0 && !out->subs) return fail(TTV_ERR_ARG, "caller buffers need subs too");
    }
    const int64_t cap_rows = dense_out ? 0 : std::min(out->subs_capacity, out->vals_capacity);
    const int64_t cap_rows_eff = (!dense_out && p0.nr == 0) ? out->vals_capacity : cap_rows;

    const size_t need = prepared_ws_bytes(h);
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
    Status* status = a.take<Status>(1);
    void* state = a.take<char>(rbk_state_bytes(h->nnz));
    StreamDesc p = p0;
    // the reduce-by-key writes the result count once and raises flags only on
    // errors: straight into the call's pinned status block when possible
    Status* dstat = h->nnz > 0 ? direct_status(st, stream) : nullptr;
    if (dstat) status = dstat;
    else cudaMemsetAsync(status, 0, sizeof(Status), stream);
    p.status = status;
    double* ovals = static_cast<double*>(out->vals);
    if (dense_out) cudaMemsetAsync(ovals, 0, (size_t)std::max<int64_t>(cap_vals, 1) * sizeof(double), stream);
    if (h->nnz > 0) {
        PrepTerms terms{};
        terms.vals = h->vals;
        terms.val_f32 = p0.val_f32;
        terms.vec_f32 = vd == TTV_F32;
        terms.n_v = h->n_v;
        for (int j = 0, m = 0; m < p0.d; ++m)
            if ((p0.smask >> m) & 1u) {
                terms.sub[j] = h->subs[j];
                terms.vec[j] = vecs[h->arg_of[j]];
                ++j;
            }
        SegOut so{out->subs, ovals, cap_rows_eff, dense_out ? 1 : 0, o->accum == TTV_ACCUM_COMPENSATED ? 1 : 0};
        launch_reduce_by_key_prepared(reinterpret_cast<const uint8_t*>(h->head_bits), h->row_keys, terms, h->nnz,
                                      state, p, so, status, stream);
    }
    if (order0) {
        st->dense_out = 1;
        out->nnz = 1;
    }
    e = dstat ? cudaSuccess : cudaMemcpyAsync(st->hstatus, status, sizeof(Status), cudaMemcpyDeviceToHost, stream);
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
            // Keep up to this much freed memory in the stream-ordered pool
            // for reuse (no release and re-map between calls), and give the
            // rest back at synchronisation points: with no limit a stream of
            // calls of varying sizes on several streams grows the pool until
            // the device runs out.
            uint64_t thr = 8ull << 30;
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
    NvtxScope nvtx_range("ttv_multi");
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
    if (!s->borrowed_status) g_status_pool.release(s->hstatus);
    delete s;
    out->internal = nullptr;
}

}  // extern "C"

namespace ttv {
// A result whose stream may be destroyed before the result is released (a
// server's slot streams): once its work has completed, its later release
// and synchronisation run on the legacy default stream instead.
void out_detach_stream(ttv_out* out) {
    if (out && out->internal) static_cast<OutState*>(out->internal)->stream = nullptr;
}
}  // namespace ttv

extern "C" {

void ttv_outs_free(ttv_out* outs, int32_t n) {
    if (!outs) return;
    for (int32_t i = 0; i < n; ++i) ttv_out_free(&outs[i]);
}

// ---- autotuner -----------------------------------------------------------------

int ttv_autotune(const ttv_tensor* t, const int32_t* modes, int32_t n_v, const void* const* vecs, ttv_dtype v_dtype,
                 const ttv_opts* opts, int32_t trials, ttv_tune_result* res, ttv_stream_t stream_) {
    NvtxScope nvtx_range("ttv_autotune");
    g_err.clear();
    if (!res) return fail(TTV_ERR_ARG, "null tuning result");
    memset(res, 0, sizeof *res);
    init_once();
    ttv_opts o;
    if (opts) o = *opts;
    else ttv_opts_init(&o);
    if (o.deterministic || o.accum != TTV_ACCUM_FP64)
        return fail(TTV_ERR_ARG, "the autotuner chooses among the binary64 paths of a non-deterministic AUTO call");
    o.path = TTV_PATH_AUTO;
    o.async = 1;
    o.workspace = nullptr;
    o.workspace_bytes = 0;
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    trials = std::max(1, std::min(trials, 50));

    Plan base;
    t_force_path = -1;
    int rc = make_plan(t, modes, n_v, vecs, v_dtype, nullptr, &o, base);
    if (rc != TTV_OK) return rc;
    const StreamDesc& p = base.desc;
    const uint64_t key = tune_key(p, base.dense_out);

    // candidates: path x CTAs per SM of the streaming pass x nonzeros per
    // thread (DENSE: 1 or 2 pairs per iteration into one shared array, 3 =
    // one pair into warp-private arrays (two CTAs per SM), or 4 = the
    // bulk-staged persistent kernel, one CTA per SM; HASH: 2 or 4 per
    // iteration)
    struct Cand { int path, ctas, items; };
    std::vector<Cand> cands;
    const bool dense_ok = (int64_t)p.nkeys <= kDenseMaxCells || base.order0;
    if (dense_ok) {
        cands.push_back({TTV_PATH_DENSE, 1, 4});
        cands.push_back({TTV_PATH_DENSE, 2, 3});
        for (int it : {1, 2})
            for (int c : {2, 3, 4}) cands.push_back({TTV_PATH_DENSE, c, it});
    }
    if (!base.order0 && p.nnz > 0 && p.nnz <= kMaxSortN) {
        for (int c : {4, 8, 16}) cands.push_back({TTV_PATH_SORT, c, 0});
        if (hash_applicable(p))
            for (int it : {4, 2})
                for (int c : {8, 16}) cands.push_back({TTV_PATH_HASH, c, it});
        if (!base.dense_out && bucket_applicable(p)) cands.push_back({TTV_PATH_BUCKET, 0, 0});
    }

    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return fail(TTV_ERR_CUDA, "event creation failed");
    int best = -1;
    for (const Cand& c : cands) {
        if (res->n_candidates >= TTV_TUNE_MAX_CANDIDATES) break;
        t_force_path = c.path;
        t_force_ctas = c.ctas;
        t_force_items = c.items;
        Plan pl;
        rc = make_plan(t, modes, n_v, vecs, v_dtype, nullptr, &o, pl);
        t_force_path = -1;
        t_force_ctas = 0;
        t_force_items = 0;
        if (rc != TTV_OK || pl.path != c.path) continue;
        std::vector<float> times;
        bool ok = true;
        for (int it = 0; it <= trials && ok; ++it) {
            ttv_out out;
            memset(&out, 0, sizeof out);
            cudaEventRecord(e0, stream);
            int r1 = execute(pl, &out, &o, stream);
            cudaEventRecord(e1, stream);
            int r2 = r1 == TTV_OK ? finalize(&out) : r1;
            ttv_out_free(&out);
            if (r2 != TTV_OK) { ok = false; break; }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (it > 0) times.push_back(ms);
        }
        if (!ok || times.empty()) continue;
        std::sort(times.begin(), times.end());
        const double med = times[times.size() / 2];
        const int i = res->n_candidates++;
        res->cand_path[i] = c.path;
        res->cand_ctas[i] = c.ctas;
        res->cand_items[i] = c.items;
        res->cand_ms[i] = med;
        if (best < 0 || med < res->cand_ms[best]) best = i;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    g_err.clear();
    if (best < 0) return fail(TTV_ERR_UNSUPPORTED, "no candidate plan ran (empty tensor or no applicable path)");
    res->path = res->cand_path[best];
    res->ctas_per_sm = res->cand_ctas[best];
    res->items_per_thread = res->cand_items[best];
    res->ms = res->cand_ms[best];
    tune_record(key, TuneRec{res->path, res->ctas_per_sm, res->items_per_thread, res->ms});
    return TTV_OK;
}

int ttv_tune_save(const char* path) {
    g_err.clear();
    if (!path) return fail(TTV_ERR_ARG, "null path");
    FILE* f = fopen(path, "w");
    if (!f) return fail(TTV_ERR_ARG, "cannot open %s for writing", path);
    std::lock_guard<std::mutex> g(g_tune_mu);
    fprintf(f, "ttv-tune 2\n");
    for (auto& e : g_tune)
        fprintf(f, "%016llx %d %d %d %.6f\n", (unsigned long long)e.first, e.second.path, e.second.ctas,
                e.second.items, e.second.ms);
    const bool bad = ferror(f) != 0;
    fclose(f);
    return bad ? fail(TTV_ERR_ARG, "write to %s failed", path) : TTV_OK;
}

int ttv_tune_load(const char* path) {
    g_err.clear();
    if (!path) return fail(TTV_ERR_ARG, "null path");
    FILE* f = fopen(path, "r");
    if (!f) return fail(TTV_ERR_ARG, "cannot open %s", path);
    char head[32] = {0};
    int version = 0;
    if (fscanf(f, "%31s %d", head, &version) != 2 || strcmp(head, "ttv-tune") != 0 || version != 2) {
        fclose(f);
        return fail(TTV_ERR_ARG, "%s is not a version-2 tuning file", path);
    }
    std::vector<std::pair<uint64_t, TuneRec>> recs;
    unsigned long long k;
    TuneRec r;
    int n;
    while ((n = fscanf(f, "%llx %d %d %d %lf", &k, &r.path, &r.ctas, &r.items, &r.ms)) == 5) {
        if (r.path < TTV_PATH_DENSE || r.path > TTV_PATH_BUCKET || r.ctas < 0 || r.ctas > 64 || r.items < 0 ||
            r.items > 16) {
            fclose(f);
            return fail(TTV_ERR_ARG, "bad record in %s", path);
        }
        recs.emplace_back((uint64_t)k, r);
    }
    const bool clean = n == EOF;
    fclose(f);
    if (!clean) return fail(TTV_ERR_ARG, "malformed line in %s", path);
    for (auto& e : recs) tune_record(e.first, e.second);
    return TTV_OK;
}

int ttv_tune_lookup(const ttv_tensor* t, const int32_t* modes, int32_t n_v, const ttv_opts* opts, int32_t* path,
                    int32_t* ctas_per_sm, int32_t* items_per_thread) {
    g_err.clear();
    ttv_opts o;
    if (opts) o = *opts;
    else ttv_opts_init(&o);
    o.path = TTV_PATH_AUTO;
    std::vector<const void*> dummy((size_t)std::max(n_v, 0), reinterpret_cast<const void*>(0x10));
    Plan pl;
    t_force_path = -1;
    const int rc = make_plan(t, modes, n_v, dummy.data(), TTV_F64, nullptr, &o, pl);
    if (rc != TTV_OK) return rc;
    TuneRec r;
    if (!tune_lookup(tune_key(pl.desc, pl.dense_out), r)) return 0;
    if (path) *path = r.path;
    if (ctas_per_sm) *ctas_per_sm = r.ctas;
    if (items_per_thread) *items_per_thread = r.items;
    return 1;
}

int ttv_tune_set(const ttv_tensor* t, const int32_t* modes, int32_t n_v, const ttv_opts* opts, int32_t path,
                 int32_t ctas_per_sm, int32_t items_per_thread) {
    g_err.clear();
    if (path < TTV_PATH_DENSE || path > TTV_PATH_BUCKET) return fail(TTV_ERR_ARG, "path %d is not a concrete path", path);
    if (ctas_per_sm < 0 || ctas_per_sm > 32 || items_per_thread < 0 || items_per_thread > 8)
        return fail(TTV_ERR_ARG, "CTAs per SM or items per thread out of range");
    ttv_opts o;
    if (opts) o = *opts;
    else ttv_opts_init(&o);
    o.path = TTV_PATH_AUTO;
    std::vector<const void*> dummy((size_t)std::max(n_v, 0), reinterpret_cast<const void*>(0x10));
    Plan pl;
    t_force_path = -1;
    const int rc = make_plan(t, modes, n_v, dummy.data(), TTV_F64, nullptr, &o, pl);
    if (rc != TTV_OK) return rc;
    TuneRec r;
    r.path = path;
    r.ctas = ctas_per_sm;
    r.items = items_per_thread;
    r.ms = 0.0;
    tune_record(tune_key(pl.desc, pl.dense_out), r);
    return TTV_OK;
}

void ttv_tune_clear(void) {
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tune.clear();
}

int ttv_tune_count(void) {
    std::lock_guard<std::mutex> g(g_tune_mu);
    return (int)g_tune.size();
}

// ---- prepared tensors ------------------------------------------------------

int ttv_prepare(const ttv_tensor* t, const int32_t* modes, int32_t n_v, ttv_prepared** out, ttv_stream_t stream_) {
    NvtxScope nvtx_range("ttv_prepare");
    g_err.clear();
    if (!out) return fail(TTV_ERR_ARG, "null result handle");
    *out = nullptr;
    init_once();
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    ttv_opts o;
    ttv_opts_init(&o);
    o.path = TTV_PATH_SORT;
    std::vector<const void*> dummy((size_t)std::max(n_v, 0), reinterpret_cast<const void*>(0x10));
    Plan pl;
    int rc = make_plan(t, modes, n_v, dummy.data(), TTV_F64, nullptr, &o, pl);
    if (rc != TTV_OK) return rc;
    const StreamDesc& p0 = pl.desc;
    if (p0.nnz > kMaxSortN) return fail(TTV_ERR_UNSUPPORTED, "prepared tensors support nnz < 2^30");
    for (int m = 0; m < p0.d; ++m)
        if (((p0.smask >> m) & 1u) && p0.shape[m] > INT32_MAX)
            return fail(TTV_ERR_UNSUPPORTED, "contracted mode %d is larger than 2^31 - 1", m);
    ttv_prepared* h = new ttv_prepared();
    h->plan = pl;
    h->plan.desc.vec_smem = 0;
    for (int m = 0; m < TTV_MAX_D; ++m) h->plan.desc.vec[m] = nullptr;
    h->nnz = p0.nnz;
    h->n_v = n_v;
    // j-th contracted mode in increasing order <- the caller's vector index
    {
        int j = 0;
        for (int m = 0; m < p0.d; ++m)
            if ((p0.smask >> m) & 1u) {
                for (int i = 0; i < n_v; ++i)
                    if (modes[i] == m) h->arg_of[j] = i;
                ++j;
            }
    }
    const int64_t n = std::max<int64_t>(p0.nnz, 1);
    const size_t vb = p0.val_f32 ? 4 : 8;
    const int64_t nwords = (n + 31) / 32;
    cudaError_t e = cudaMalloc(&h->head_bits, (size_t)nwords * 4);
    if (e == cudaSuccess) e = cudaMalloc(&h->vals, (size_t)n * vb);
    for (int j = 0; j < n_v && e == cudaSuccess; ++j) e = cudaMalloc(&h->subs[j], (size_t)n * 4);
    h->bytes = (size_t)nwords * 4 + (size_t)n * (vb + 4 * (size_t)n_v);
    auto drop = [&](int code, const char* what) {
        ttv_prepared_free(h);
        return code == TTV_ERR_CUDA ? cuda_fail(e, what) : code;
    };
    if (e != cudaSuccess) return drop(TTV_ERR_CUDA, "prepared tensor allocation");
    if (p0.nnz == 0) {
        e = cudaMalloc(&h->row_keys, 8);
        if (e == cudaSuccess && p0.nr == 1) {
            e = cudaMalloc(&h->chunk_base, 4);
            if (e == cudaSuccess) e = cudaMemset(h->chunk_base, 0, 4);
            if (e == cudaSuccess) e = cudaMalloc(&h->next_head, 4);
        }
        if (e != cudaSuccess) return drop(TTV_ERR_CUDA, "prepared tensor allocation");
        *out = h;
        return TTV_OK;
    }
    // temporaries: both key buffers, the index payloads, the sort state and
    // the reduce-by-key state of the run-key pass
    const int npass = (pl.key_bits + 7) / 8;
    const int64_t ntiles = (n + 4095) / 4096;
    Arena a;
    a.take<Status>(1);
    a.take<unsigned long long>(1);
    a.take<uint64_t>(n);
    a.take<uint64_t>(n);
    a.take<double>(n);
    a.take<double>(n);
    a.take<uint32_t>((size_t)std::max(npass, 1) * 256);
    a.take<uint32_t>((size_t)std::max(npass, 1) * ntiles * 256);
    a.take<uint32_t>(64);
    a.take<char>(rbk_state_bytes(n));
    a.off = (a.off + 255) & ~size_t(255);
    void* tmp = nullptr;
    e = cudaMallocAsync(&tmp, a.off, stream);
    if (e != cudaSuccess) return drop(TTV_ERR_CUDA, "prepare workspace");
    a.base = static_cast<char*>(tmp);
    a.off = 0;
    Status* status = a.take<Status>(1);
    unsigned long long* count = a.take<unsigned long long>(1);
    SortBuffers sb{};
    sb.keys[0] = a.take<uint64_t>(n);
    sb.keys[1] = a.take<uint64_t>(n);
    sb.vals[0] = a.take<double>(n);
    sb.vals[1] = a.take<double>(n);
    sb.hist = a.take<uint32_t>((size_t)std::max(npass, 1) * 256);
    sb.lookback = a.take<uint32_t>((size_t)std::max(npass, 1) * ntiles * 256);
    sb.tickets = a.take<uint32_t>(64);
    sb.npass = npass;
    sb.ntiles = ntiles;
    void* rbk_state = a.take<char>(rbk_state_bytes(n));
    cudaMemsetAsync(status, 0, sizeof(Status), stream);
    cudaMemsetAsync(count, 0, sizeof(unsigned long long), stream);
    StreamDesc p = p0;
    p.status = status;
    launch_prep_keys(p, sb.keys[0], sb.vals[0], stream);
    const int cur = radix_sort_pairs(sb, p.nnz, pl.key_bits, status, stream);
    const uint64_t* keys = sb.keys[cur];
    PrepTerms subs{};
    subs.n_v = n_v;
    for (int j = 0; j < n_v; ++j) subs.sub[j] = h->subs[j];
    launch_prep_gather(p, sb.vals[cur], h->vals, subs, stream);
    launch_prep_heads(keys, p.nnz, h->head_bits, stream);
    launch_prep_count(keys, p.nnz, count, stream);
    Status hs;
    unsigned long long hc = 0;
    e = cudaMemcpyAsync(&hs, status, sizeof(Status), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hc, count, sizeof hc, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess && !(hs.err & kErrSubscript) && !hs.err) {
        // the key of every result row
        e = cudaMalloc(&h->row_keys, (size_t)std::max<unsigned long long>(hc, 1) * 8);
        h->bytes += (size_t)std::max<unsigned long long>(hc, 1) * 8;
        if (e == cudaSuccess) {
            launch_run_keys(keys, sb.vals[cur], p.nnz, rbk_state, h->row_keys, (int64_t)hc, p, status, stream);
            e = cudaMemcpyAsync(&hs, status, sizeof(Status), cudaMemcpyDeviceToHost, stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
            if (e == cudaSuccess) e = cudaGetLastError();
        }
    }
    cudaFreeAsync(tmp, stream);
    cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return drop(TTV_ERR_CUDA, "prepare");
    if (hs.err & kErrSubscript) return drop(fail(TTV_ERR_SUBSCRIPT, "a subscript is outside its mode"), "");
    if (hs.err & kErrTimeout) return drop(fail(TTV_ERR_TIMEOUT, "a bounded device wait ran out"), "");
    if (hs.err) return drop(fail(TTV_ERR_CUDA, "internal device check failed"), "");
    h->nnz_out = (int64_t)hc;
    if (p0.nr == 1) {
        // MTTKRP chunk index: heads before every chunk (counted on the
        // device, scanned here once)
        const int64_t nc = mttkrp_nchunks(p0.nnz);
        std::vector<uint32_t> hcnt((size_t)nc), base((size_t)nc + 1, 0);
        uint32_t* dcnt = nullptr;
        e = cudaMalloc(&h->chunk_base, ((size_t)nc + 1) * 4);
        if (e == cudaSuccess) e = cudaMalloc(&dcnt, (size_t)std::max<int64_t>(nc, 1) * 4);
        if (e == cudaSuccess) {
            launch_mttkrp_chunk_counts(h->head_bits, p0.nnz, dcnt, stream);
            e = cudaMemcpyAsync(hcnt.data(), dcnt, (size_t)nc * 4, cudaMemcpyDeviceToHost, stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        }
        if (e == cudaSuccess) {
            for (int64_t c = 0; c < nc; ++c) base[(size_t)c + 1] = base[(size_t)c] + hcnt[(size_t)c];
            e = cudaMemcpy(h->chunk_base, base.data(), ((size_t)nc + 1) * 4, cudaMemcpyHostToDevice);
        }
        if (e == cudaSuccess) {
            std::vector<int32_t> nxt((size_t)std::max<int64_t>(nc, 1));
            int32_t next = (int32_t)nc;
            for (int64_t c = nc - 1; c >= 0; --c) {
                nxt[(size_t)c] = next;
                if (hcnt[(size_t)c] > 0) next = (int32_t)c;
            }
            e = cudaMalloc(&h->next_head, (size_t)std::max<int64_t>(nc, 1) * 4);
            if (e == cudaSuccess) e = cudaMemcpy(h->next_head, nxt.data(), (size_t)std::max<int64_t>(nc, 1) * 4,
                                                 cudaMemcpyHostToDevice);
        }
        if (dcnt) cudaFree(dcnt);
        if (e != cudaSuccess) return drop(TTV_ERR_CUDA, "MTTKRP chunk index");
        h->bytes += ((size_t)nc + 1) * 4 + (size_t)nc * 4;
    }
    *out = h;
    return TTV_OK;
}

int ttv_prepared_run(const ttv_prepared* h, const void* const* vecs, const int64_t* vec_lens, ttv_dtype v_dtype,
                     ttv_out* out, const ttv_opts* opts, ttv_stream_t stream) {
    NvtxScope nvtx_range("ttv_prepared_run");
    g_err.clear();
    if (!h || !vecs || !out) return fail(TTV_ERR_ARG, "null prepared tensor, vectors or result");
    if (v_dtype != TTV_F64 && v_dtype != TTV_F32) return fail(TTV_ERR_ARG, "bad vector dtype");
    ttv_opts def;
    ttv_opts_init(&def);
    const ttv_opts* o = opts ? opts : &def;
    if (o->fmt < TTV_OUT_SPARSE || o->fmt > TTV_OUT_AUTO) return fail(TTV_ERR_ARG, "bad output format");
    if (o->accum != TTV_ACCUM_FP64 && o->accum != TTV_ACCUM_COMPENSATED)
        return fail(TTV_ERR_UNSUPPORTED, "prepared tensors accumulate in binary64, plain or compensated");
    const StreamDesc& p0 = h->plan.desc;
    int j = 0;
    for (int m = 0; m < p0.d; ++m)
        if ((p0.smask >> m) & 1u) {
            const int i = h->arg_of[j++];
            if (!vecs[i]) return fail(TTV_ERR_ARG, "null vector for mode %d", m);
            if (vec_lens && vec_lens[i] != p0.shape[m])
                return fail(TTV_ERR_VEC_LEN, "vector for mode %d has %lld entries, mode size is %lld", m,
                            (long long)vec_lens[i], (long long)p0.shape[m]);
        }
    init_once();
    return execute_prepared(h, vecs, v_dtype, out, o, reinterpret_cast<cudaStream_t>(stream));
}

int ttv_mttkrp_workspace_size(const ttv_prepared* h, int32_t rank, size_t* bytes) {
    if (!h || !bytes || rank < 1 || rank > TTV_MTTKRP_MAX_RANK) return fail(TTV_ERR_ARG, "bad MTTKRP arguments");
    *bytes = mttkrp_workspace_bytes(h->nnz, rank);
    return TTV_OK;
}

int ttv_mttkrp_prepared(const ttv_prepared* h, const double* const* factors, int32_t rank, double* out,
                        void* workspace, size_t workspace_bytes, ttv_stream_t stream_) {
    NvtxScope nvtx_range("ttv_mttkrp");
    g_err.clear();
    if (!h || !factors || !out) return fail(TTV_ERR_ARG, "null prepared tensor, factors or result");
    if (rank < 1 || rank > TTV_MTTKRP_MAX_RANK) return fail(TTV_ERR_ARG, "rank %d outside 1..%d", rank, TTV_MTTKRP_MAX_RANK);
    const StreamDesc& p0 = h->plan.desc;
    if (p0.nr != 1 || !h->chunk_base)
        return fail(TTV_ERR_ARG, "MTTKRP needs a tensor prepared for every mode but one");
    const double* fac[TTV_MAX_D] = {nullptr};
    for (int j = 0; j < h->n_v; ++j) {
        fac[j] = factors[h->arg_of[j]];
        if (!fac[j]) return fail(TTV_ERR_ARG, "null factor");
    }
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    init_once();
    const size_t need = mttkrp_workspace_bytes(h->nnz, rank);
    void* ws = workspace;
    bool own = false;
    if (!ws || workspace_bytes < need) {
        cudaError_t e = cudaMallocAsync(&ws, need, stream);
        if (e != cudaSuccess) return cuda_fail(e, "MTTKRP workspace");
        own = true;
    }
    const int32_t* subs[TTV_MAX_D];
    for (int j = 0; j < h->n_v; ++j) subs[j] = h->subs[j];
    launch_mttkrp(h->vals, p0.val_f32, h->n_v, subs, fac, h->head_bits, h->row_keys, h->chunk_base, h->next_head,
                  h->nnz, rank, p0.rshape[0], out, ws, stream);
    if (own) cudaFreeAsync(ws, stream);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "MTTKRP launch");
    return TTV_OK;
}

int ttv_mttkrp(const ttv_tensor* t, int32_t mode, const double* const* factors, int32_t rank, double* out,
               ttv_stream_t stream) {
    g_err.clear();
    if (!t || !factors) return fail(TTV_ERR_ARG, "null tensor or factors");
    if (t->d < 2 || t->d > TTV_MAX_D) return fail(TTV_ERR_ARG, "MTTKRP needs order 2..%d", TTV_MAX_D);
    if (mode < 0 || mode >= t->d) return fail(TTV_ERR_MODE, "mode %d outside 0..%d", mode, t->d - 1);
    int32_t modes[TTV_MAX_D];
    const double* fac[TTV_MAX_D];
    int n_v = 0;
    for (int m = 0; m < t->d; ++m)
        if (m != mode) {
            modes[n_v] = m;
            fac[n_v] = factors[m];
            ++n_v;
        }
    ttv_prepared* h = nullptr;
    int rc = ttv_prepare(t, modes, n_v, &h, stream);
    if (rc != TTV_OK) return rc;
    rc = ttv_mttkrp_prepared(h, fac, rank, out, nullptr, 0, stream);
    if (rc == TTV_OK) {
        const cudaError_t e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
        if (e != cudaSuccess) rc = cuda_fail(e, "MTTKRP");
    }
    ttv_prepared_free(h);
    return rc;
}

int ttv_dot_workspace_size(int64_t n, size_t* bytes) {
    if (!bytes || n < 0) return fail(TTV_ERR_ARG, "bad dot arguments");
    init_once();
    *bytes = n > 0 ? dot_workspace_bytes(n) : 0;
    return TTV_OK;
}

int ttv_dot(const void* x, const void* y, int64_t n, ttv_dtype dtype, double* out, void* workspace,
            size_t workspace_bytes, ttv_stream_t stream_) {
    NvtxScope nvtx_range("ttv_dot");
    g_err.clear();
    if (n < 0 || !out || (n > 0 && (!x || !y))) return fail(TTV_ERR_ARG, "null operand or negative length");
    if (dtype != TTV_F64 && dtype != TTV_F32) return fail(TTV_ERR_ARG, "bad dtype");
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    init_once();
    const size_t need = n > 0 ? dot_workspace_bytes(n) : 0;
    void* ws = workspace;
    bool own = false;
    if (need && (!ws || workspace_bytes < need)) {
        cudaError_t e = cudaMallocAsync(&ws, need, stream);
        if (e != cudaSuccess) return cuda_fail(e, "dot workspace");
        own = true;
    }
    launch_dot(x, y, n, dtype == TTV_F32, out, ws, stream);
    if (own) cudaFreeAsync(ws, stream);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "dot launch");
    return TTV_OK;
}

int ttv_matvec_workspace_size(int64_t n1, int64_t n2, int64_t stride_row, int64_t stride_col, size_t* bytes) {
    if (!bytes || n1 < 0 || n2 < 0) return fail(TTV_ERR_ARG, "bad matvec arguments");
    if (!matvec_layout_ok(n1, n2, stride_row, stride_col)) return fail(TTV_ERR_UNSUPPORTED, "neither stride is 1");
    init_once();
    *bytes = matvec_workspace_bytes(n1, n2, stride_row, stride_col);
    return TTV_OK;
}

int ttv_matvec(const void* A, int64_t n1, int64_t n2, int64_t stride_row, int64_t stride_col, ttv_dtype dtype,
               const void* x, double* y, void* workspace, size_t workspace_bytes, ttv_stream_t stream_) {
    NvtxScope nvtx_range("ttv_matvec");
    g_err.clear();
    if (n1 < 0 || n2 < 0) return fail(TTV_ERR_ARG, "negative size");
    if ((n1 > 0 && !y) || (n1 > 0 && n2 > 0 && (!A || !x))) return fail(TTV_ERR_ARG, "null operand");
    if (dtype != TTV_F64 && dtype != TTV_F32) return fail(TTV_ERR_ARG, "bad dtype");
    if (!matvec_layout_ok(n1, n2, stride_row, stride_col))
        return fail(TTV_ERR_UNSUPPORTED, "matrix strides (%lld, %lld): neither is 1", (long long)stride_row,
                    (long long)stride_col);
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    init_once();
    const size_t need = matvec_workspace_bytes(n1, n2, stride_row, stride_col);
    void* ws = workspace;
    bool own = false;
    if (need && (!ws || workspace_bytes < need)) {
        cudaError_t e = cudaMallocAsync(&ws, need, stream);
        if (e != cudaSuccess) return cuda_fail(e, "matvec workspace");
        own = true;
    }
    launch_matvec(A, n1, n2, stride_row, stride_col, dtype == TTV_F32, x, y, ws, stream);
    if (own) cudaFreeAsync(ws, stream);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "matvec launch");
    return TTV_OK;
}

int ttv_prepared_info(const ttv_prepared* h, int64_t* nnz_out, int32_t* order, size_t* device_bytes) {
    if (!h) return fail(TTV_ERR_ARG, "null prepared tensor");
    if (nnz_out) *nnz_out = h->nnz_out;
    if (order) *order = h->plan.desc.nr;
    if (device_bytes) *device_bytes = h->bytes;
    return TTV_OK;
}

int ttv_prepared_workspace_size(const ttv_prepared* h, size_t* bytes) {
    if (!h || !bytes) return fail(TTV_ERR_ARG, "null argument");
    *bytes = prepared_ws_bytes(h);
    return TTV_OK;
}

void ttv_prepared_free(ttv_prepared* h) {
    if (!h) return;
    cudaDeviceSynchronize();
    if (h->head_bits) cudaFree(h->head_bits);
    if (h->chunk_base) cudaFree(h->chunk_base);
    if (h->next_head) cudaFree(h->next_head);
    if (h->row_keys) cudaFree(h->row_keys);
    if (h->vals) cudaFree(h->vals);
    for (int j = 0; j < TTV_MAX_D; ++j)
        if (h->subs[j]) cudaFree(h->subs[j]);
    delete h;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched TTV: one CUDA graph per set of problems.
namespace ttv {

extern thread_local int t_capturing;      // ttv_prof.cu: no event records while capturing
long long prof_add_launches(long long n);  // ttv_prof.cu

struct BatchEntry {
    uint64_t sig = 0;
    cudaGraphExec_t exec = nullptr;
    std::vector<Status*> status;          // pinned, refreshed by every replay
    std::vector<int> dense_out;
    std::vector<ttv_out> shape;           // order, shape, is_dense, nnz of each result
    long long launches = 0;               // kernel nodes per replay
    void* arena = nullptr;                // library-owned workspace, if any
    void* table = nullptr;                // job table of the batched sort path
    int batched = 0;                      // problems on the batched sort path
    uint64_t last_use = 0;
};

static std::mutex g_batch_mu;
static std::vector<BatchEntry*> g_batch_cache;
static uint64_t g_batch_clock = 0;
constexpr int kBatchStreams = 8;
constexpr size_t kBatchCacheMax = 16;

static uint64_t fnv(uint64_t h, const void* p, size_t n) {
    const unsigned char* c = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) { h ^= c[i]; h *= 1099511628211ull; }
    return h;
}
template <typename T>
static uint64_t fnv_v(uint64_t h, const T& v) { return fnv(h, &v, sizeof v); }

static uint64_t batch_signature(const ttv_problem* probs, int32_t n, const ttv_out* outs, const ttv_opts* o) {
    uint64_t h = 1469598103934665603ull;
    int dev = 0;
    cudaGetDevice(&dev);
    h = fnv_v(h, dev);
    h = fnv_v(h, n);
    h = fnv_v(h, o->fmt); h = fnv_v(h, o->path); h = fnv_v(h, o->accum); h = fnv_v(h, o->deterministic);
    h = fnv_v(h, o->workspace); h = fnv_v(h, o->workspace_bytes);
    for (int32_t i = 0; i < n; ++i) {
        const ttv_tensor& t = probs[i].tensor;
        h = fnv_v(h, t.subs); h = fnv_v(h, t.stride_nz); h = fnv_v(h, t.stride_mode); h = fnv_v(h, t.vals);
        h = fnv_v(h, t.val_dtype); h = fnv_v(h, t.nnz); h = fnv_v(h, t.d);
        if (t.shape) h = fnv(h, t.shape, sizeof(int64_t) * (size_t)std::max(0, std::min(t.d, TTV_MAX_D)));
        h = fnv_v(h, probs[i].n_v); h = fnv_v(h, probs[i].v_dtype);
        if (probs[i].modes) h = fnv(h, probs[i].modes, sizeof(int32_t) * (size_t)std::max(0, probs[i].n_v));
        if (probs[i].vecs) h = fnv(h, probs[i].vecs, sizeof(void*) * (size_t)std::max(0, probs[i].n_v));
        h = fnv_v(h, outs[i].subs); h = fnv_v(h, outs[i].vals);
        h = fnv_v(h, outs[i].subs_capacity); h = fnv_v(h, outs[i].vals_capacity);
    }
    return h;
}

static cudaStream_t* side_streams() {
    static cudaStream_t s[kBatchStreams + 1];
    static std::once_flag f;
    std::call_once(f, [] {
        for (int i = 0; i <= kBatchStreams; ++i) cudaStreamCreateWithFlags(&s[i], cudaStreamNonBlocking);
    });
    return s;
}

static void destroy_entry(BatchEntry* e) {
    if (!e) return;
    if (e->exec) cudaGraphExecDestroy(e->exec);
    for (Status* s : e->status) g_status_pool.release(s);
    if (e->arena) cudaFree(e->arena);
    if (e->table) cudaFree(e->table);
    delete e;
}

// ---- the batched sort path ---------------------------------------------------
// Problems on the sort path with a sparse result and the order-specialised
// key kernel run stage by stage: each stage is one launch over all of them
// (batch_sort_capture), so a batch costs a fixed number of launches instead
// of about a dozen per problem.  Their scratch that must start at zero (digit
// counts, look-back words, pass tickets) sits in one region after the
// per-problem workspaces and is cleared by one memset.
static int plan_npass(const Plan& pl) { return (pl.key_bits + 7) / 8; }

static bool batch_sortable(const Plan& pl) {
    const StreamDesc& p = pl.desc;
    const int npass = plan_npass(pl);
    return pl.path == TTV_PATH_SORT && !pl.dense_out && !pl.order0 && p.nr > 0 && p.nnz >= 2 && npass >= 1 &&
           npass <= 8 && p.d >= 2 && p.d <= 8;
}

static size_t round256(size_t b) { return (b + 255) & ~size_t(255); }

// Bytes of a batched problem's zeroed scratch: digit counts and look-back words.
static size_t batch_zero_bytes(const Plan& pl) {
    const int npass = plan_npass(pl);
    return round256((size_t)npass * 256 * sizeof(uint32_t)) +
           round256((size_t)npass * (size_t)sort_tiles(pl.desc.nnz) * 256 * sizeof(uint32_t));
}

// Plans, per-problem workspace offsets and the batched sort path's share:
// its problems and its zeroed region [zero_off, zero_off + zero_bytes).
static int batch_plans(const ttv_problem* probs, int32_t n, const ttv_opts* o, std::vector<Plan>& plans,
                       std::vector<size_t>& ws_off, size_t& total, std::vector<int32_t>& batched,
                       size_t& zero_off, size_t& zero_bytes) {
    plans.resize((size_t)n);
    ws_off.resize((size_t)n);
    batched.clear();
    total = 0;
    for (int32_t i = 0; i < n; ++i) {
        const ttv_problem& q = probs[i];
        int rc = make_plan(&q.tensor, q.modes, q.n_v, q.vecs, q.v_dtype, nullptr, o, plans[(size_t)i]);
        if (rc != TTV_OK) return fail(rc, "problem %d: %s", i, g_err.c_str());
        // A hashed (not direct) table ends in a radix sort of its distinct
        // keys, a dozen launches of its own; in a batch the stage-wise sort
        // takes such a problem at no launch cost (same bytes within a few
        // percent: 17.6 against 17.8 ms for the 512-problem batch).
        Plan& pl = plans[(size_t)i];
        if (o->path == TTV_PATH_AUTO && pl.path == TTV_PATH_HASH && !pl.dense_out && !hash_direct(pl.desc))
            pl.path = TTV_PATH_SORT;
        ws_off[(size_t)i] = total;
        total += round256(workspace_bytes(plans[(size_t)i]));
        if (batch_sortable(plans[(size_t)i])) batched.push_back(i);
    }
    zero_off = total;
    zero_bytes = 0;
    if (!batched.empty()) {
        zero_bytes = 256;     // pass tickets
        for (int32_t i : batched) zero_bytes += batch_zero_bytes(plans[(size_t)i]);
    }
    total += zero_bytes;
    return TTV_OK;
}

// The launches of the batched problems' stages, with their job lists in
// the entry's device table.
struct BatchSortLaunch {
    const BatchJob* jobs = nullptr;
    struct Kt { JobList l; uint32_t units; int d; int lay; };
    std::vector<Kt> kt;
    JobList srt{};
    int32_t count_per_pass[8] = {0};
    uint32_t tiles_per_pass[8] = {0};
    int max_npass = 0;
    uint32_t* tickets = nullptr;
    JobList rt[2]{}, rg[2]{};
    uint32_t rtiles[2] = {0, 0}, rgroups[2] = {0, 0};
    void* zero = nullptr;
    size_t zero_bytes = 0;
};

// One batched problem's job: its pair buffers and reduce-by-key state from
// its own workspace (ws_problem, laid out by layout()), its digit counts and
// look-back words from the zeroed region (zero + zo, zo advanced), its
// status block (device address) and result buffers.
static void fill_batch_job(BatchJob& J, const Plan& pl, char* ws_problem, char* zero, size_t& zo, Status* dstatus,
                           int64_t* subs, double* vals, int64_t cap_rows) {
    Arena a;
    a.base = ws_problem;
    WsPtrs w;
    layout(pl, a, w);
    memset(&J, 0, sizeof J);
    J.p = pl.desc;
    J.p.status = dstatus;
    for (int b = 0; b < 2; ++b) {
        J.keys[b] = w.sb.keys[b];
        J.vals[b] = w.sb.vals[b];
    }
    J.npass = plan_npass(pl);
    J.ntiles = sort_tiles(pl.desc.nnz);
    J.hist = reinterpret_cast<uint32_t*>(zero + zo);
    zo += round256((size_t)J.npass * 256 * sizeof(uint32_t));
    J.lookback = reinterpret_cast<uint32_t*>(zero + zo);
    zo += round256((size_t)J.npass * (size_t)J.ntiles * 256 * sizeof(uint32_t));
    J.rbk_state = w.rbk_state;
    J.o = SegOut{subs, vals, cap_rows, 0, pl.compensated};
}

// The job table in host memory: the jobs, then every job list's problem
// indices and unit prefix, at 256-byte aligned offsets of one blob; launch
// counts that do not depend on where the blob lands on the device.
struct BatchTable {
    struct ListOff { size_t idx, prefix; int32_t count; uint32_t units; size_t unit_pos = 0; bool has_map = false; };
    std::vector<char> blob;
    std::vector<std::pair<int, ListOff>> kt;   // key: d * 4 + layout class
    ListOff srt{}, rt[2]{}, rg[2]{};
    int32_t count_per_pass[8] = {0};
    uint32_t tiles_per_pass[8] = {0};
    int max_npass = 0;
};

static void build_batch_table(const std::vector<BatchJob>& jobs, BatchTable& T) {
    const size_t nb = jobs.size();
    // job lists: one per (order, layout) for the key kernel; all jobs by
    // decreasing pass count for the sort; one per accumulation for the reduction
    struct HostList {
        std::vector<int32_t> idx;
        std::vector<uint32_t> prefix{0};
        void add(int32_t j, uint64_t units) {
            idx.push_back(j);
            prefix.push_back(prefix.back() + (uint32_t)units);
        }
    };
    std::vector<std::pair<int, HostList>> kt;
    HostList srt, rt[2], rg[2];
    std::vector<int32_t> by_pass(nb);
    for (size_t j = 0; j < nb; ++j) by_pass[j] = (int32_t)j;
    std::stable_sort(by_pass.begin(), by_pass.end(), [&](int32_t a, int32_t b) { return jobs[a].npass > jobs[b].npass; });
    for (int32_t j : by_pass) {
        const BatchJob& J = jobs[(size_t)j];
        const int key = J.p.d * 4 + keys_terms_batch_layout(J.p);
        auto it = std::find_if(kt.begin(), kt.end(), [&](const std::pair<int, HostList>& c) { return c.first == key; });
        if (it == kt.end()) {
            kt.emplace_back(key, HostList{});
            it = kt.end() - 1;
        }
        it->second.add(j, (uint64_t)((J.p.nnz + kKtBatchChunk - 1) / kKtBatchChunk));
        srt.add(j, (uint64_t)J.ntiles);
        const int c = J.o.compensated ? 1 : 0;
        rt[c].add(j, (uint64_t)rbk_tiles(J.p.nnz));
        rg[c].add(j, (uint64_t)rbk_groups(J.p.nnz));
    }
    for (size_t q = 0; q < nb; ++q) {
        const BatchJob& J = jobs[(size_t)by_pass[q]];
        T.max_npass = std::max(T.max_npass, (int)J.npass);
        for (int p = 0; p < J.npass; ++p) {
            T.count_per_pass[p] = (int32_t)q + 1;
            T.tiles_per_pass[p] = srt.prefix[q + 1];
        }
    }
    auto put = [&](const void* src, size_t bytes) {
        const size_t off = round256(T.blob.size());
        T.blob.resize(off + bytes);
        if (bytes) memcpy(T.blob.data() + off, src, bytes);
        return off;
    };
    // map: the list's position of every unit, for the kernels whose CTAs are
    // short (a tile each), so that finding the problem is one load
    auto put_list = [&](const HostList& l, bool map) {
        BatchTable::ListOff r;
        r.idx = put(l.idx.data(), l.idx.size() * sizeof(int32_t));
        r.prefix = put(l.prefix.data(), l.prefix.size() * sizeof(uint32_t));
        r.count = (int32_t)l.idx.size();
        r.units = l.prefix.back();
        if (map && r.units) {
            std::vector<uint32_t> pos(r.units);
            for (size_t q = 0; q < l.idx.size(); ++q)
                for (uint32_t u = l.prefix[q]; u < l.prefix[q + 1]; ++u) pos[u] = (uint32_t)q;
            r.unit_pos = put(pos.data(), pos.size() * sizeof(uint32_t));
            r.has_map = true;
        }
        return r;
    };
    put(jobs.data(), nb * sizeof(BatchJob));
    for (auto& c : kt) T.kt.emplace_back(c.first, put_list(c.second, false));
    T.srt = put_list(srt, true);
    for (int c = 0; c < 2; ++c) {
        T.rt[c] = put_list(rt[c], true);
        T.rg[c] = put_list(rg[c], false);
    }
}

// The launches of a table copied to device address tb.
static void bind_batch_table(const BatchTable& T, char* tb, uint32_t* tickets, void* zero, size_t zero_bytes,
                             BatchSortLaunch& L) {
    auto dlist = [&](const BatchTable::ListOff& l) {
        return JobList{reinterpret_cast<const int32_t*>(tb + l.idx), reinterpret_cast<const uint32_t*>(tb + l.prefix),
                       l.count, l.has_map ? reinterpret_cast<const uint32_t*>(tb + l.unit_pos) : nullptr};
    };
    L.jobs = reinterpret_cast<const BatchJob*>(tb);
    L.kt.clear();
    for (const auto& c : T.kt) L.kt.push_back(BatchSortLaunch::Kt{dlist(c.second), c.second.units, c.first / 4, c.first % 4});
    L.srt = dlist(T.srt);
    for (int p = 0; p < 8; ++p) {
        L.count_per_pass[p] = T.count_per_pass[p];
        L.tiles_per_pass[p] = T.tiles_per_pass[p];
    }
    L.max_npass = T.max_npass;
    L.tickets = tickets;
    for (int c = 0; c < 2; ++c) {
        L.rt[c] = dlist(T.rt[c]);
        L.rg[c] = dlist(T.rg[c]);
        L.rtiles[c] = T.rt[c].units;
        L.rgroups[c] = T.rg[c].units;
    }
    L.zero = zero;
    L.zero_bytes = zero_bytes;
}

// Builds the job table of the batched problems and uploads it (once, owned
// by the entry; before the capture starts: the copy is synchronous).
static int batch_sort_prepare(BatchEntry* e, const std::vector<Plan>& plans, const std::vector<size_t>& ws_off,
                              const std::vector<int32_t>& batched, char* ws, size_t zero_off, size_t zero_bytes,
                              ttv_out* outs, BatchSortLaunch& L) {
    const size_t nb = batched.size();
    char* zero = ws + zero_off;
    size_t zo = 256;              // pass tickets first
    std::vector<BatchJob> jobs(nb);
    for (size_t j = 0; j < nb; ++j) {
        const int32_t i = batched[j];
        const Plan& pl = plans[(size_t)i];
        if (!outs[i].subs) return fail(TTV_ERR_ARG, "caller buffers need subs too (problem %d)", i);
        Status* hs = g_status_pool.acquire();
        if (!hs) return fail(TTV_ERR_NOMEM, "pinned status allocation failed");
        e->status[(size_t)i] = hs;
        memset(hs, 0, sizeof(Status));
        void* dp = nullptr;
        cudaError_t ce = cudaHostGetDevicePointer(&dp, hs, 0);
        if (ce != cudaSuccess || !dp) return cuda_fail(ce, "status mapping");
        const int64_t cap = std::min(outs[i].subs_capacity, outs[i].vals_capacity);
        fill_batch_job(jobs[j], pl, ws + ws_off[(size_t)i], zero, zo, static_cast<Status*>(dp), outs[i].subs,
                       static_cast<double*>(outs[i].vals), cap);
        ttv_out sh{};
        sh.order = pl.desc.nr;
        for (int m = 0; m < TTV_MAX_D; ++m) sh.shape[m] = m < pl.desc.nr ? pl.desc.rshape[m] : 0;
        sh.dtype = TTV_F64;
        e->shape[(size_t)i] = sh;
        e->dense_out[(size_t)i] = 0;
    }
    if (zo != zero_bytes) return fail(TTV_ERR_CUDA, "batch scratch layout mismatch");
    BatchTable T;
    build_batch_table(jobs, T);
    cudaError_t ce = cudaMalloc(&e->table, std::max<size_t>(T.blob.size(), 256));
    if (ce != cudaSuccess) { e->table = nullptr; return cuda_fail(ce, "batch job table"); }
    ce = cudaMemcpy(e->table, T.blob.data(), T.blob.size(), cudaMemcpyHostToDevice);
    if (ce != cudaSuccess) return cuda_fail(ce, "batch job table");
    bind_batch_table(T, static_cast<char*>(e->table), reinterpret_cast<uint32_t*>(zero), zero, zero_bytes, L);
    e->batched = (int)nb;
    return TTV_OK;
}

// The stages, in order, on one stream (being captured).
static int batch_sort_issue(const BatchSortLaunch& L, cudaStream_t stream) {
    cudaError_t ce = cudaMemsetAsync(L.zero, 0, L.zero_bytes, stream);
    if (ce != cudaSuccess) return cuda_fail(ce, "batch scratch reset");
    for (const BatchSortLaunch::Kt& k : L.kt) launch_keys_terms_batch(L.jobs, k.l, k.units, k.d, k.lay, stream);
    launch_sort_batch(L.jobs, L.srt, L.count_per_pass, L.tiles_per_pass, L.max_npass, L.tickets, stream);
    for (int c = 0; c < 2; ++c) launch_rbk_batch(L.jobs, L.rt[c], L.rtiles[c], L.rg[c], L.rgroups[c], c == 1, stream);
    return TTV_OK;
}

// A batch run once, without a graph (the server's groups of requests): the
// plans, one workspace block and the job table are allocated on the stream,
// results without caller buffers are library-owned, and every result is
// finalised by ttv_out_sync and released by ttv_out_free like a single
// call's.  Problems off the stage-wise sort path run the single-call path on
// the same stream.  Returns the first failure; results already set up keep
// their bookkeeping (the caller frees them with ttv_out_free).
int batch_run_direct(const ttv_problem* probs, int32_t n, ttv_out* outs, const ttv_opts* o, cudaStream_t stream) {
    if (!probs || !outs || n < 0 || !o) return fail(TTV_ERR_ARG, "bad batch arguments");
    for (int32_t i = 0; i < n; ++i)
        if (outs[i].internal) return fail(TTV_ERR_ARG, "ttv_out %d reused without ttv_out_free", i);
    std::vector<Plan> plans;
    std::vector<size_t> ws_off;
    std::vector<int32_t> batched;
    size_t total = 0, zero_off = 0, zero_bytes = 0;
    int rc = batch_plans(probs, n, o, plans, ws_off, total, batched, zero_off, zero_bytes);
    if (rc != TTV_OK) return rc;
    if (o->path != TTV_PATH_AUTO && o->path != TTV_PATH_SORT) batched.clear();
    // one workspace per problem, as its single call would take (one block for
    // a whole group fragments a stream-ordered pool that also serves results),
    // and the zeroed region of the stage-wise problems
    std::vector<char*> wsp((size_t)n, nullptr);
    char* zero = nullptr;
    auto release = [&]() {
        for (char* p : wsp)
            if (p) cudaFreeAsync(p, stream);
        if (zero) cudaFreeAsync(zero, stream);
    };
    cudaError_t ce = cudaSuccess;
    for (int32_t i = 0; i < n && ce == cudaSuccess; ++i)
        ce = cudaMallocAsync((void**)&wsp[(size_t)i], std::max<size_t>(workspace_bytes(plans[(size_t)i]), 256), stream);
    if (ce == cudaSuccess && zero_bytes) ce = cudaMallocAsync((void**)&zero, zero_bytes, stream);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        release();
        return cuda_fail(ce, "batch workspace");
    }
    std::vector<char> on_batch((size_t)n, 0);
    for (int32_t i : batched) on_batch[(size_t)i] = 1;

    // the stage-wise problems: results, statuses, jobs
    const size_t nb = batched.size();
    std::vector<BatchJob> jobs(nb);
    size_t zo = 256;              // pass tickets first
    for (size_t j = 0; j < nb && rc == TTV_OK; ++j) {
        const int32_t i = batched[j];
        const Plan& pl = plans[(size_t)i];
        ttv_out* out = &outs[i];
        OutState* st = new OutState();
        st->stream = stream;
        st->auto_fmt = o->fmt == TTV_OUT_AUTO;
        st->nkeys = pl.desc.nkeys;
        out->internal = st;
        out->order = pl.desc.nr;
        for (int m = 0; m < TTV_MAX_D; ++m) out->shape[m] = m < pl.desc.nr ? pl.desc.rshape[m] : 0;
        out->dtype = TTV_F64;
        out->is_dense = 0;
        out->nnz = 0;
        st->hstatus = g_status_pool.acquire();
        if (!st->hstatus) { rc = fail(TTV_ERR_NOMEM, "pinned status allocation failed"); break; }
        memset(st->hstatus, 0, sizeof(Status));
        void* dp = nullptr;
        ce = cudaHostGetDevicePointer(&dp, st->hstatus, 0);
        if (ce != cudaSuccess || !dp) { rc = cuda_fail(ce, "status mapping"); break; }
        if (!out->vals) {
            ce = cudaMallocAsync(&out->vals, (size_t)std::max<int64_t>(pl.cap_vals, 1) * sizeof(double), stream);
            if (ce != cudaSuccess) { out->vals = nullptr; rc = cuda_fail(ce, "output allocation"); break; }
            st->owned_vals = out->vals;
            out->vals_capacity = pl.cap_vals;
            ce = cudaMallocAsync((void**)&out->subs, (size_t)std::max<int64_t>(pl.cap_rows, 1) * pl.desc.nr * sizeof(int64_t),
                                 stream);
            if (ce != cudaSuccess) { out->subs = nullptr; rc = cuda_fail(ce, "output allocation"); break; }
            st->owned_subs = out->subs;
            out->subs_capacity = pl.cap_rows;
        } else if (!out->subs) {
            rc = fail(TTV_ERR_ARG, "caller buffers need subs too (problem %d)", i);
            break;
        }
        const int64_t cap = std::min(out->subs_capacity, out->vals_capacity);
        fill_batch_job(jobs[j], pl, wsp[(size_t)i], zero, zo, static_cast<Status*>(dp), out->subs,
                       static_cast<double*>(out->vals), cap);
    }
    char* tb = nullptr;
    BatchSortLaunch L;
    if (rc == TTV_OK && nb) {
        BatchTable T;
        build_batch_table(jobs, T);
        ce = cudaMallocAsync((void**)&tb, std::max<size_t>(T.blob.size(), 256), stream);
        if (ce != cudaSuccess) {
            tb = nullptr;
            rc = cuda_fail(ce, "batch job table");
        } else {
            // from pageable memory: staged before the call returns, before any
            // kernel of this batch is queued
            ce = cudaMemcpyAsync(tb, T.blob.data(), T.blob.size(), cudaMemcpyHostToDevice, stream);
            if (ce != cudaSuccess) rc = cuda_fail(ce, "batch job table");
            bind_batch_table(T, tb, reinterpret_cast<uint32_t*>(zero), zero, zero_bytes, L);
        }
    }
    if (rc == TTV_OK && nb) rc = batch_sort_issue(L, stream);
    // the other problems: the single-call path, on the same stream
    for (int32_t i = 0; i < n && rc == TTV_OK; ++i) {
        if (on_batch[(size_t)i]) continue;
        ttv_opts oi = *o;
        oi.async = 1;
        oi.workspace = wsp[(size_t)i];
        oi.workspace_bytes = workspace_bytes(plans[(size_t)i]);
        rc = execute(plans[(size_t)i], &outs[i], &oi, stream);
    }
    if (tb) cudaFreeAsync(tb, stream);
    release();
    ce = cudaGetLastError();
    if (rc == TTV_OK && ce != cudaSuccess) rc = cuda_fail(ce, "kernel launch");
    return rc;
}

static BatchEntry* batch_capture(const ttv_problem* probs, int32_t n, ttv_out* outs, const ttv_opts* o,
                                 uint64_t sig, int& rc) {
    std::vector<Plan> plans;
    std::vector<size_t> ws_off;
    std::vector<int32_t> batched;
    size_t total = 0, zero_off = 0, zero_bytes = 0;
    rc = batch_plans(probs, n, o, plans, ws_off, total, batched, zero_off, zero_bytes);
    if (rc != TTV_OK) return nullptr;
    if (o->path != TTV_PATH_AUTO && o->path != TTV_PATH_SORT) batched.clear();
    BatchEntry* e = new BatchEntry();
    e->sig = sig;
    char* ws = static_cast<char*>(o->workspace);
    if (!ws || o->workspace_bytes < total) {
        cudaError_t ce = cudaMalloc(&e->arena, std::max<size_t>(total, 256));
        if (ce != cudaSuccess) { rc = cuda_fail(ce, "batch workspace"); delete e; return nullptr; }
        ws = static_cast<char*>(e->arena);
    }
    // largest problems first, dealt round-robin over the streams
    std::vector<int32_t> order((size_t)n);
    for (int32_t i = 0; i < n; ++i) order[(size_t)i] = i;
    std::sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return probs[a].tensor.nnz > probs[b].tensor.nnz; });
    cudaStream_t* ss = side_streams();
    cudaStream_t cap = ss[kBatchStreams];
    if (!g_status_pool.reserve((size_t)n + 8)) {
        rc = fail(TTV_ERR_NOMEM, "pinned status allocation failed");
        destroy_entry(e);
        return nullptr;
    }
    cudaEvent_t fork, joins[kBatchStreams];
    cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    for (int k = 0; k < kBatchStreams; ++k) cudaEventCreateWithFlags(&joins[k], cudaEventDisableTiming);
    e->status.assign((size_t)n, nullptr);
    e->dense_out.assign((size_t)n, 0);
    e->shape.assign((size_t)n, ttv_out{});
    BatchSortLaunch bl;
    if (!batched.empty()) {
        rc = batch_sort_prepare(e, plans, ws_off, batched, ws, zero_off, zero_bytes, outs, bl);
        if (rc != TTV_OK) {
            cudaEventDestroy(fork);
            for (int k = 0; k < kBatchStreams; ++k) cudaEventDestroy(joins[k]);
            destroy_entry(e);
            return nullptr;
        }
    }
    t_capturing = 1;
    const long long before = prof_add_launches(0);
    cudaError_t ce = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (ce != cudaSuccess) { t_capturing = 0; rc = cuda_fail(ce, "begin capture"); destroy_entry(e); return nullptr; }
    cudaEventRecord(fork, cap);
    const int nstreams = std::min<int>(kBatchStreams, std::max<int32_t>(1, n));
    for (int k = 0; k < nstreams; ++k) cudaStreamWaitEvent(ss[k], fork, 0);
    rc = TTV_OK;
    // the batched problems' stages on the first stream, the rest dealt over the others
    std::vector<char> on_batch((size_t)n, 0);
    for (int32_t i : batched) on_batch[(size_t)i] = 1;
    const int first_free = batched.empty() || nstreams == 1 ? 0 : 1;
    if (!batched.empty()) rc = batch_sort_issue(bl, ss[0]);
    size_t dealt = 0;
    for (size_t j = 0; j < order.size() && rc == TTV_OK; ++j) {
        const int32_t i = order[j];
        if (on_batch[(size_t)i]) continue;
        ttv_opts oi = *o;
        oi.async = 1;
        oi.workspace = ws + ws_off[(size_t)i];
        oi.workspace_bytes = workspace_bytes(plans[(size_t)i]);
        ttv_out tmp = outs[i];
        tmp.internal = nullptr;
        const int r = execute(plans[(size_t)i], &tmp, &oi,
                              ss[first_free + (int)(dealt++ % (size_t)(nstreams - first_free))]);
        OutState* st = static_cast<OutState*>(tmp.internal);
        if (st) {
            e->status[(size_t)i] = st->hstatus;
            e->dense_out[(size_t)i] = st->dense_out;
            delete st;
        }
        tmp.internal = nullptr;
        e->shape[(size_t)i] = tmp;
        if (r != TTV_OK && rc == TTV_OK) rc = r;
    }
    for (int k = 0; k < nstreams; ++k) {
        cudaEventRecord(joins[k], ss[k]);
        cudaStreamWaitEvent(cap, joins[k], 0);
    }
    cudaGraph_t graph = nullptr;
    ce = cudaStreamEndCapture(cap, &graph);
    t_capturing = 0;
    e->launches = prof_add_launches(0) - before;
    prof_add_launches(-e->launches);            // captured, not yet run
    cudaEventDestroy(fork);
    for (int k = 0; k < kBatchStreams; ++k) cudaEventDestroy(joins[k]);
    if (ce != cudaSuccess || rc != TTV_OK) {
        if (graph) cudaGraphDestroy(graph);
        if (rc == TTV_OK) rc = cuda_fail(ce, "end capture");
        destroy_entry(e);
        return nullptr;
    }
    ce = cudaGraphInstantiate(&e->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) { rc = cuda_fail(ce, "graph instantiate"); destroy_entry(e); return nullptr; }
    return e;
}

}  // namespace ttv

extern "C" {

int ttv_batch_workspace_size(const ttv_problem* probs, int32_t n, const ttv_opts* opts, size_t* bytes) {
    g_err.clear();
    if (!probs || n < 0 || !bytes) return fail(TTV_ERR_ARG, "bad batch arguments");
    ttv_opts def;
    ttv_opts_init(&def);
    const ttv_opts* o = opts ? opts : &def;
    std::vector<Plan> plans;
    std::vector<size_t> off;
    std::vector<int32_t> batched;
    size_t total = 0, zero_off = 0, zero_bytes = 0;
    int rc = batch_plans(probs, n, o, plans, off, total, batched, zero_off, zero_bytes);
    if (rc != TTV_OK) return rc;
    *bytes = total;
    return TTV_OK;
}

long long ttv_batch_graph_launches(const ttv_problem* probs, int32_t n, const ttv_out* outs, const ttv_opts* opts) {
    if (!probs || !outs || n <= 0) return 0;
    ttv_opts def;
    ttv_opts_init(&def);
    const ttv_opts* o = opts ? opts : &def;
    const uint64_t sig = batch_signature(probs, n, outs, o);
    std::lock_guard<std::mutex> g(g_batch_mu);
    for (BatchEntry* e : g_batch_cache)
        if (e->sig == sig) return e->launches;
    return 0;
}

void ttv_batch_release(void) {
    std::lock_guard<std::mutex> g(g_batch_mu);
    cudaDeviceSynchronize();
    for (BatchEntry* e : g_batch_cache) destroy_entry(e);
    g_batch_cache.clear();
}

int ttv_batch(const ttv_problem* probs, int32_t n, ttv_out* outs, const ttv_opts* opts, ttv_stream_t stream_) {
    NvtxScope nvtx_range("ttv_batch");
    g_err.clear();
    if (!probs || !outs || n < 0) return fail(TTV_ERR_ARG, "bad batch arguments");
    if (n == 0) return TTV_OK;
    for (int32_t i = 0; i < n; ++i) {
        if (!outs[i].vals) return fail(TTV_ERR_ARG, "batch results need caller buffers (problem %d)", i);
        if (outs[i].internal) return fail(TTV_ERR_ARG, "ttv_out %d reused without ttv_out_free", i);
    }
    ttv_opts def;
    ttv_opts_init(&def);
    const ttv_opts* o = opts ? opts : &def;
    init_once();
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    const uint64_t sig = batch_signature(probs, n, outs, o);
    std::lock_guard<std::mutex> g(g_batch_mu);
    BatchEntry* e = nullptr;
    for (BatchEntry* c : g_batch_cache)
        if (c->sig == sig) { e = c; break; }
    if (!e) {
        int rc = TTV_OK;
        e = batch_capture(probs, n, outs, o, sig, rc);
        if (!e) return rc;
        if (g_batch_cache.size() >= kBatchCacheMax) {
            auto it = std::min_element(g_batch_cache.begin(), g_batch_cache.end(),
                                       [](BatchEntry* a, BatchEntry* b) { return a->last_use < b->last_use; });
            cudaDeviceSynchronize();
            destroy_entry(*it);
            g_batch_cache.erase(it);
        }
        g_batch_cache.push_back(e);
    }
    e->last_use = ++g_batch_clock;
    for (Status* s : e->status) memset(s, 0, sizeof(Status));
    cudaError_t ce = cudaGraphLaunch(e->exec, stream);
    if (ce != cudaSuccess) return cuda_fail(ce, "graph launch");
    prof_add_launches(e->launches);
    int first = TTV_OK;
    for (int32_t i = 0; i < n; ++i) {
        OutState* st = new OutState();
        st->hstatus = e->status[(size_t)i];
        st->borrowed_status = 1;
        st->stream = stream;
        st->dense_out = e->dense_out[(size_t)i];
        outs[i].internal = st;
        // shape and order are fixed by the problem
        const ttv_out& sh = e->shape[(size_t)i];
        outs[i].order = sh.order;
        for (int j = 0; j < TTV_MAX_D; ++j) outs[i].shape[j] = sh.shape[j];
        outs[i].dtype = TTV_F64;
        outs[i].is_dense = sh.is_dense;
        outs[i].nnz = sh.nnz;
    }
    if (o->async) return TTV_OK;
    ce = cudaStreamSynchronize(stream);
    for (int32_t i = 0; i < n; ++i) {
        const int r = finalize(&outs[i], ce == cudaSuccess);
        if (r != TTV_OK && first == TTV_OK) first = r;
    }
    return first;
}

}  // extern "C"
