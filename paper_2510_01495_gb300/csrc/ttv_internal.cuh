// ttv_internal.cuh -- device-side descriptors and helpers shared by the
// kernels of the sparse TTV library (sm_103a).  Nothing here is part of the
// C ABI; include/ttv.h is.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/ttv.h"

namespace ttv {

constexpr int kMaxD = TTV_MAX_D;

// Error bits accumulated in Status::err by kernels (host maps them to codes).
enum : uint32_t {
    kErrSubscript = 1u << 0,   // a subscript outside [0, shape[m])
    kErrTimeout = 1u << 1,     // a bounded spin wait ran out
    kErrCapacity = 1u << 2,    // result larger than the output buffer
    kErrInternal = 1u << 3,    // an internal invariant failed (bucket overflow ...)
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
    Status* status;
};

__device__ __forceinline__ void set_error(Status* st, uint32_t bit) {
    atomicOr(&st->err, bit);
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

// Inverse of the linearisation: key -> result subscripts (row-major over R).
__device__ __forceinline__ void delinearise(const StreamDesc& p, uint64_t key, int64_t* out_row) {
    for (int j = p.nr - 1; j >= 0; --j) {
        const uint64_t n = (uint64_t)p.rshape[j];
        out_row[j] = (int64_t)(key % n);
        key /= n;
    }
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
// Every kernel launch goes through this: counted, and timed when profiling.
#define TTV_LAUNCH(name, stream, ...)      \
    do {                                   \
        ::ttv::prof_begin(name, stream);   \
        __VA_ARGS__;                       \
        ::ttv::prof_end(stream);           \
    } while (0)

// ---- host-side launch helpers (implemented in the .cu files) -------------

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
// Sorts (keys, vals) stably by the low `bits` bits of the key; returns which
// buffer (0/1) holds the result.
int radix_sort_pairs(SortBuffers& sb, int64_t n, int bits, Status* st, cudaStream_t stream);

}  // namespace ttv
