// ttv_internal.cuh -- device-side descriptors and helpers shared by the
// kernels of the sparse TTV library (sm_103a).  Nothing here is part of the
// C ABI; include/ttv.h is.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/ttv.h"
#include "ttv_udiv.h"

namespace ttv {

constexpr int64_t kDenseMaxCells = 16384;       // key spaces accumulated in shared memory

constexpr int kMaxD = TTV_MAX_D;

// Error bits accumulated in Status::err by kernels (host maps them to codes).
enum : uint32_t {
    kErrSubscript = 1u << 0,   // a subscript outside [0, shape[m])
    kErrTimeout = 1u << 1,     // a bounded spin wait ran out
    kErrCapacity = 1u << 2,    // result larger than the output buffer
    kErrInternal = 1u << 3,    // an internal invariant failed (bucket overflow ...)
    kErrNonFinite = 1u << 4,   // inf/nan met by a fixed-point accumulator
    kErrRetry = 1u << 5,       // bucket path gave up (skewed sample): rerun on the sort path
};

// Per-call device status block (lives in the call's workspace).
struct Status {
    uint32_t err;
    uint32_t pad;
    unsigned long long nnz_out;      // entries of a sparse result
    unsigned long long long_count;   // long segments queued for the warp pass
    unsigned long long aux[5];
};

// Everything a streaming kernel needs to turn nonzero k into (key, term).
// Modes are visited in increasing order, so the product is formed in
// increasing mode order: vals[k] * x_{m1}[.] * x_{m2}[.] ...
struct StreamDesc {
    const int64_t* subs;
    int64_t snz, smode;               // element strides of subs
    const void* vals;
    int64_t nnz;
    int32_t d;
    int32_t val_f32;                  // 1: vals are float
    int32_t vec_f32;                  // 1: vectors are float
    int32_t vec_smem;                 // 1: vectors staged in shared memory
    uint32_t smask;                   // bit m set: mode m is contracted
    int32_t nr;                       // surviving modes
    int64_t shape[kMaxD];
    uint64_t kstride[kMaxD];          // row-major stride of mode m over R (0 if contracted)
    const void* vec[kMaxD];           // vector of mode m (nullptr if surviving)
    int32_t voff[kMaxD];              // offset of mode m's vector in the staged buffer
    int32_t vtotal;                   // staged entries
    uint64_t nkeys;                   // prod shape[R] (key space size)
    int32_t rmode[kMaxD];             // surviving modes, ascending
    int64_t rshape[kMaxD];            // shape of the result
    uint64_t rmagic[kMaxD];           // division by rshape[j] (see udiv_invariant)
    uint32_t rsh[kMaxD];              // shift pair: sh1 | sh2 << 8
    int32_t ctas_per_sm;              // grid of the streaming pass: CTAs per SM (0: default)
    int32_t items;                    // nonzeros (dense: pairs) per thread per iteration (0: default)
    Status* status;
};



__device__ __forceinline__ void set_error(Status* st, uint32_t bit) {
    atomicOr(&st->err, bit);
}


// ---- exact significand arithmetic (integer units; GB300's FP64 pipe is ~2/clk/SM) ----
// |x| = M * 2^(E - 63) with M in [2^63, 2^64); zero gives M = 0.
struct Sig {
    unsigned long long M;
    int E;
    uint32_t neg;
    uint32_t bad;     // inf or nan
    uint32_t wide;    // some nonzero partial product left [2^-1021, 2^1023)
};

__device__ __forceinline__ Sig decompose(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    Sig s;
    s.wide = 0;
    s.neg = (uint32_t)(b >> 63);
    const int ex = (int)((b >> 52) & 0x7FF);
    const unsigned long long f = b & ((1ull << 52) - 1);
    s.bad = ex == 0x7FF;
    if (ex == 0) {
        if (f == 0) {
            s.M = 0;
            s.E = -(1 << 28);
        } else {
            const int lz = __clzll(f);
            s.M = f << lz;
            s.E = -1011 - lz;
        }
    } else {
        s.M = (f | (1ull << 52)) << 11;
        s.E = ex - 1023;
    }
    return s;
}

// a *= b on significands: high 64 bits of the 128-bit product, renormalised
// (truncation error below 2^-62 relative). A nonzero partial product whose
// exponent falls outside [-1021, 1022] sets `wide`: there the binary64 chain
// of Eq. 3 may overflow, underflow or lose bits to a subnormal step, so the
// caller recomputes that term as the chain itself. The one-exponent margin
// covers the chain's own rounding of the partial products.
__device__ __forceinline__ void sig_mul(Sig& a, const Sig& b) {
    const unsigned long long hi = __umul64hi(a.M, b.M);
    const bool top = (hi >> 63) != 0;
    a.M = top ? hi : (hi << 1);
    a.E = a.E + b.E + (top ? 1 : 0);
    a.neg ^= b.neg;
    a.bad |= b.bad;
    if (b.M == 0) a.M = 0;
    a.wide |= (uint32_t)(a.M != 0) & (uint32_t)((unsigned)(a.E + 1021) > 2043u);
}

// Nearest binary64 of a significand (ties to even); infinities and
// subnormal results take the general scalbn route.
__device__ __forceinline__ double sig_to_double(const Sig& s) {
    if (s.M == 0) return s.neg ? -0.0 : 0.0;
    unsigned long long mant = s.M >> 11;                 // 53 bits, top bit set
    const unsigned long long rest = s.M & 0x7FFull;
    if (rest > 0x400ull || (rest == 0x400ull && (mant & 1ull))) ++mant;
    int E = s.E;
    if (mant >> 53) { mant >>= 1; ++E; }
    if (E >= -1022 && E <= 1023) {
        const unsigned long long bits = ((unsigned long long)s.neg << 63) |
                                        ((unsigned long long)(E + 1023) << 52) | (mant & ((1ull << 52) - 1));
        return __longlong_as_double((long long)bits);
    }
    const double r = scalbn((double)(s.M >> 11), E - 52);
    return s.neg ? -r : r;
}

// A staged vector entry, decomposed once per CTA (16 bytes: one LDS.128).
struct __align__(16) SigEntry {
    unsigned long long M;
    int E;
    uint32_t neg_bad;    // bit 0: sign, bit 1: inf/nan
};

__device__ __forceinline__ Sig sig_of(const SigEntry& e) {
    Sig s;
    s.wide = 0;
    s.M = e.M;
    s.E = e.E;
    s.neg = e.neg_bad & 1u;
    s.bad = (e.neg_bad >> 1) & 1u;
    return s;
}

// Stage the contracted vectors in shared memory as decomposed significands.
__device__ __forceinline__ void stage_vectors_sig(const StreamDesc& p, SigEntry* sv) {
    if (!p.vec_smem) return;
    for (int m = 0; m < p.d; ++m) {
        if (!((p.smask >> m) & 1u)) continue;
        const int64_t n = p.shape[m];
        SigEntry* dst = sv + p.voff[m];
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
            const double x = p.vec_f32 ? (double)__ldg(static_cast<const float*>(p.vec[m]) + i)
                                       : __ldg(static_cast<const double*>(p.vec[m]) + i);
            const Sig s = decompose(x);
            SigEntry e;
            e.M = s.M;
            e.E = s.E;
            e.neg_bad = s.neg | (s.bad << 1);
            dst[i] = e;
        }
    }
}

// Stage the contracted vectors in shared memory as doubles (exact for floats).
__device__ __forceinline__ void stage_vectors(const StreamDesc& p, double* sv) {
    if (!p.vec_smem) return;
    for (int m = 0; m < p.d; ++m) {
        if (!((p.smask >> m) & 1u)) continue;
        const int64_t n = p.shape[m];
        double* dst = sv + p.voff[m];
        if (p.vec_f32) {
            const float* src = static_cast<const float*>(p.vec[m]);
            for (int64_t i = threadIdx.x; i < n; i += blockDim.x) dst[i] = (double)__ldg(src + i);
        } else {
            const double* src = static_cast<const double*>(p.vec[m]);
            for (int64_t i = threadIdx.x; i < n; i += blockDim.x) dst[i] = __ldg(src + i);
        }
    }
}

__device__ __forceinline__ double load_val(const StreamDesc& p, int64_t k) {
    if (p.val_f32) return (double)__ldcs(static_cast<const float*>(p.vals) + k);
    return __ldcs(static_cast<const double*>(p.vals) + k);
}

__device__ __forceinline__ double load_vec(const StreamDesc& p, const double* sv, int m, int64_t s) {
    if (p.vec_smem) return sv[p.voff[m] + s];
    if (p.vec_f32) return (double)__ldg(static_cast<const float*>(p.vec[m]) + s);
    return __ldg(static_cast<const double*>(p.vec[m]) + s);
}

// U consecutive-in-stride nonzeros per thread: loads first, then arithmetic,
// so that U * (d + 1) independent loads are in flight per thread.
// Returns false (and flags the status) for a nonzero with a bad subscript.
template <int U>
struct Batch {
    int64_t s[U][kMaxD];
    double v[U];
};

template <int U>
__device__ __forceinline__ void load_batch(const StreamDesc& p, const int64_t* ks, bool const* ok, Batch<U>& b) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
        if (!ok[u]) continue;
        const int64_t* row = p.subs + ks[u] * p.snz;
#pragma unroll
        for (int m = 0; m < kMaxD; ++m)
            if (m < p.d) b.s[u][m] = __ldcs(row + m * p.smode);
        b.v[u] = load_val(p, ks[u]);
    }
}

// Key (row-major linear index over R) and term of one loaded nonzero.
__device__ __forceinline__ bool key_term(const StreamDesc& p, const double* sv, const int64_t* s, double val,
                                         uint64_t& key, double& t) {
    bool good = true;
    uint64_t kk = 0;
    double tt = val;
#pragma unroll
    for (int m = 0; m < kMaxD; ++m) {
        if (m >= p.d) break;
        const int64_t sm = s[m];
        if (sm < 0 || sm >= p.shape[m]) { good = false; continue; }
        if ((p.smask >> m) & 1u) tt = tt * load_vec(p, sv, m, sm);
        else kk += (uint64_t)sm * p.kstride[m];
    }
    key = kk;
    t = tt;
    return good;
}

// Same as key_term with the product formed on integer units: the value and
// each gathered entry as significands, multiplied exactly to 64 bits and
// rounded once to binary64 (within one unit of the binary64 product chain).
// Inf/nan operands, and terms whose partial products leave the normal
// binary64 range, take the binary64 chain, so overflow, underflow and
// subnormal steps round exactly as Eq. 3's chain does.
__device__ __forceinline__ bool key_term_sig(const StreamDesc& p, const SigEntry* sve, const int64_t* s, double val,
                                             uint64_t& key, double& t) {
    bool good = true;
    uint64_t kk = 0;
    Sig acc = decompose(val);
#pragma unroll
    for (int m = 0; m < kMaxD; ++m) {
        if (m >= p.d) break;
        const int64_t sm = s[m];
        if (sm < 0 || sm >= p.shape[m]) { good = false; continue; }
        if ((p.smask >> m) & 1u) {
            if (p.vec_smem) {
                sig_mul(acc, sig_of(sve[p.voff[m] + sm]));
            } else {
                const double x = p.vec_f32 ? (double)__ldg(static_cast<const float*>(p.vec[m]) + sm)
                                           : __ldg(static_cast<const double*>(p.vec[m]) + sm);
                sig_mul(acc, decompose(x));
            }
        } else {
            kk += (uint64_t)sm * p.kstride[m];
        }
    }
    key = kk;
    if (good && (acc.bad | acc.wide)) {
        double tt = val;
#pragma unroll
        for (int m = 0; m < kMaxD; ++m)
            if (m < p.d && ((p.smask >> m) & 1u))
                tt = tt * (p.vec_f32 ? (double)__ldg(static_cast<const float*>(p.vec[m]) + s[m])
                                     : __ldg(static_cast<const double*>(p.vec[m]) + s[m]));
        t = tt;
    } else {
        t = sig_to_double(acc);
    }
    return good;
}

// Inverse of the linearisation: key -> result subscripts (row-major over R),
// with multiply-high division by the invariant mode sizes.
__device__ __forceinline__ void delinearise(const StreamDesc& p, uint64_t key, int64_t* out_row) {
    for (int j = p.nr - 1; j >= 0; --j) {
        const uint64_t n = (uint64_t)p.rshape[j];
        const uint64_t q = udiv_invariant(key, p.rmagic[j], p.rsh[j]);
        out_row[j] = (int64_t)(key - q * n);
        key = q;
    }
}

// ---- test hook: shortened wait limits ---------------------------------------
// 0 (the default): every bounded wait keeps its own poll limit.  v > 0: the
// waits that read wait_limit() give up after v - 1 polls, so that a test can
// make them run out on purpose and check the error status that follows.
// Each translation unit holds its own copy; ttv_test_set_wait_polls sets all.
static __device__ uint32_t g_wait_override = 0;
__device__ __forceinline__ uint32_t wait_limit(uint32_t dflt) {
    const uint32_t o = *reinterpret_cast<const volatile uint32_t*>(&g_wait_override);
    return o ? o - 1 : dflt;
}
static inline cudaError_t set_wait_override_here(uint32_t v) {
    return cudaMemcpyToSymbol(g_wait_override, &v, sizeof v);
}

// Bounded spin on a 32-bit word until pred(value) holds; false on timeout.
template <typename Pred>
__device__ __forceinline__ bool spin_until(const volatile uint32_t* addr, uint32_t& value, Pred pred,
                                           uint32_t max_iters = 1u << 22) {
    for (uint32_t it = 0; it < max_iters; ++it) {
        value = *addr;
        if (pred(value)) return true;
        if (it > 64) __nanosleep(64);
    }
    return false;
}

// ---- launch bookkeeping (ttv_prof.cu) --------------------------------------
void prof_begin(const char* name, cudaStream_t s);
void prof_end(cudaStream_t s);

// Raises a kernel's dynamic shared memory limit to at least `bytes`, never
// lowering it: a lower limit set for one problem would make launches (and
// captured graph nodes) sized for another fail.  Thread-safe.
void smem_limit_at_least(const void* kernel, size_t bytes);
template <class K>
inline void smem_at_least(K* kernel, size_t bytes) {
    smem_limit_at_least(reinterpret_cast<const void*>(kernel), bytes);
}
// Every kernel launch goes through this: counted, and timed when profiling.
#define TTV_LAUNCH(name, stream, ...)      \
    do {                                   \
        ::ttv::prof_begin(name, stream);   \
        __VA_ARGS__;                       \
        ::ttv::prof_end(stream);           \
    } while (0)

// ---- host-side launch helpers (implemented in the .cu files) -------------

// Plan of the fixed-point dense path (ttv_dense_fx.cu).
struct FxPlan {
    bool ok;
    int tile, stages, grid, headroom, aos;
    size_t stage_bytes, smem_total, cells_off, pres_off, vec_off, stage_off, bar_off;
    int64_t chunk;
};
FxPlan plan_dense_fx(const StreamDesc& p, int want_presence, int num_sms);
size_t dense_fx_workspace(const StreamDesc& p, const FxPlan& fp, int want_presence);
void launch_dense_fx(const StreamDesc& p, const FxPlan& fp, int want_presence, void* ws, double* cell_vals,
                     uint32_t* cell_flags, cudaStream_t stream);
int num_sms();

struct SortBuffers {
    uint64_t* keys[2];
    double* vals[2];
    uint32_t* hist;         // npass x 256
    uint32_t* lookback;     // npass x ntiles x 256
    uint32_t* tickets;      // npass counters
    int npass;
    int64_t ntiles;
};

size_t sort_workspace_bytes(int64_t n, int bits);

// Where a segmented reduction writes: result rows (subs, vals) of a sparse
// result, or vals indexed by key for a dense one; with row_keys set, only the
// key of every run (row) is written there.
struct SegOut {
    int64_t* subs;          // rows of the sparse result (nullptr when dense)
    double* vals;           // values; dense: indexed by key
    int64_t cap_rows;       // capacity in rows (sparse)
    int dense;
    int compensated;
    uint64_t* row_keys = nullptr;
};

// Terms of a prepared tensor (see ttv_prepare): values and the contracted
// modes' subscripts stored in key order, the contracted modes in increasing
// order with their vectors.
struct PrepTerms {
    const void* vals;
    int32_t val_f32;
    int32_t vec_f32;
    int32_t n_v;
    const int32_t* sub[kMaxD];
    const void* vec[kMaxD];
};
// One problem of a batch on the sort path run stage-wise: every stage
// (keys and terms, histogram scan, each digit pass, the reduce-by-key
// stages) is one launch over all problems of the batch, each CTA finding its
// problem and its tile by a binary search over per-problem unit counts.
struct BatchJob {
    StreamDesc p;               // p.status: the problem's status block
    uint64_t* keys[2];          // pair buffers (nnz each, 16-byte aligned)
    double* vals[2];
    uint32_t* hist;             // npass x 256 digit counts, zeroed before the batch
    uint32_t* lookback;         // npass x ntiles x 256 look-back words, zeroed before the batch
    void* rbk_state;            // rbk_state_bytes(nnz)
    SegOut o;                   // sparse result rows
    int64_t ntiles;             // radix-sort tiles
    int32_t npass;              // 8-bit digit passes (1..8)
    int32_t pad;
};

// The problems one batched stage covers: idx[0..count) in the order of
// prefix, prefix[j] = units (CTAs or warps) before problem idx[j],
// prefix[count] = the total.
struct JobList {
    const int32_t* idx;
    const uint32_t* prefix;
    int32_t count;
    const uint32_t* unit_pos = nullptr;   // position in the list of every unit (nullptr: search prefix)
};

constexpr int64_t kKtBatchChunk = 16384;   // nonzeros per CTA of the batched key kernel
int64_t sort_tiles(int64_t n);             // radix-sort tiles of n pairs
int64_t rbk_tiles(int64_t n);              // reduce-by-key tiles of n pairs
int64_t rbk_groups(int64_t n);             // reduce-by-key tile groups of n pairs

// The stages over a batch; every job list is in device memory.
int keys_terms_batch_layout(const StreamDesc& p);
void launch_keys_terms_batch(const BatchJob* jobs, const JobList& l, uint32_t units, int d, int lay,
                             cudaStream_t stream);
void launch_sort_batch(const BatchJob* jobs, const JobList& all, const int32_t* count_per_pass,
                       const uint32_t* tiles_per_pass, int max_npass, uint32_t* tickets, cudaStream_t stream);
void launch_rbk_batch(const BatchJob* jobs, const JobList& tiles, uint32_t ntiles, const JobList& groups,
                      uint32_t ngroup_warps, bool compensated, cudaStream_t stream);

// Sorts (keys, vals) stably by the low `bits` bits of the key; returns which
// buffer (0/1) holds the result.  With n_dev, the pair count is
// min(n, *n_dev), read on the device (n is then the upper bound the buffers
// and grids are sized for).
// hist_ready: sb.hist already holds the digit counts of every pass (the
// specialised key kernel counts them while it writes the keys).
int radix_sort_pairs(SortBuffers& sb, int64_t n, int bits, Status* st, cudaStream_t stream,
                     const unsigned long long* n_dev = nullptr, bool hist_ready = false);

}  // namespace ttv
