// ttv_keys.cu -- order-specialised front end of the sort path.
//
// Same (key, term) per nonzero as k_keys_terms (ttv_stream.cu): the term is
// vals[k] times the gathered vector entries in increasing mode order, the key
// the row-major index of the surviving subscripts (paper Sec. 3.3, Eq. 3).
// Compiled per tensor order D and subscript layout, each thread takes two
// consecutive nonzeros with 16-byte loads (one column pair per mode under
// SoA, two rows under AoS) and writes the two keys and terms with 16-byte
// stores.  As a side job it counts the 8-bit digits of every radix pass into
// shared-memory histograms, so the sort needs no separate histogram pass over
// the keys.
#include <algorithm>

#include "ttv_internal.cuh"

namespace ttv {

constexpr int kKtThreads = 256;
constexpr int kKtMaxPass = 8;

template <int D>
__device__ __forceinline__ bool kt_item(const StreamDesc& p, const double* sv, const int64_t* s, double val,
                                        uint64_t& key, double& t) {
    bool good = true;
    uint64_t kk = 0;
    double tt = val;
#pragma unroll
    for (int m = 0; m < D; ++m) {
        const int64_t sm = s[m];
        good &= (uint64_t)sm < (uint64_t)p.shape[m];
        const int64_t si = good ? sm : 0;
        if ((p.smask >> m) & 1u) tt = tt * load_vec(p, sv, m, si);
        else kk += (uint64_t)si * p.kstride[m];
    }
    key = kk;
    t = tt;
    return good;
}

// Pairs q0 + threadIdx.x, + stride, ... below q1 (pair q: nonzeros 2q and
// 2q + 1), the odd last nonzero too when `tail`; digit counts into sh.
// Subscript layouts: AoS rows, SoA columns with an even stride (16-byte
// column-pair loads), or any strides (one 8-byte load per subscript).
enum { kLayAoS = 0, kLaySoA = 1, kLayAny = 2 };

template <int D, int kLay>
__device__ __forceinline__ void kt_range(const StreamDesc& p, const double* sv, uint64_t* __restrict__ keys,
                                         double* __restrict__ terms, int npass, uint32_t* sh, int64_t q0,
                                         int64_t q1, int64_t stride, bool tail) {
    const double* vd = static_cast<const double*>(p.vals);
    const float* vf = static_cast<const float*>(p.vals);
    auto count = [&](uint64_t key) {
        for (int q = 0; q < npass; ++q) atomicAdd(&sh[q * 256 + ((key >> (8 * q)) & 255u)], 1u);
    };
    for (int64_t q = q0 + threadIdx.x; q < q1; q += stride) {
        const int64_t k = 2 * q;
        int64_t s0[D], s1[D];
        if constexpr (kLay == kLayAny) {
#pragma unroll
            for (int m = 0; m < D; ++m) {
                s0[m] = __ldcs(p.subs + k * p.snz + m * p.smode);
                s1[m] = __ldcs(p.subs + (k + 1) * p.snz + m * p.smode);
            }
        } else if constexpr (kLay == kLaySoA) {
#pragma unroll
            for (int m = 0; m < D; ++m) {
                const longlong2 w = __ldcs(reinterpret_cast<const longlong2*>(p.subs + m * p.smode + k));
                s0[m] = w.x;
                s1[m] = w.y;
            }
        } else {
            const longlong2* row = reinterpret_cast<const longlong2*>(p.subs + k * D);
#pragma unroll
            for (int j = 0; j < D; ++j) {
                const longlong2 w = __ldcs(row + j);
                const int e0 = 2 * j, e1 = 2 * j + 1;
                if (e0 < D) s0[e0] = w.x; else s1[e0 - D] = w.x;
                if (e1 < D) s0[e1] = w.y; else s1[e1 - D] = w.y;
            }
        }
        double v0, v1;
        if (kLay == kLayAny) {
            v0 = p.val_f32 ? (double)__ldcs(vf + k) : __ldcs(vd + k);
            v1 = p.val_f32 ? (double)__ldcs(vf + k + 1) : __ldcs(vd + k + 1);
        } else if (p.val_f32) {
            const float2 w = __ldcs(reinterpret_cast<const float2*>(vf + k));
            v0 = (double)w.x;
            v1 = (double)w.y;
        } else {
            const double2 w = __ldcs(reinterpret_cast<const double2*>(vd + k));
            v0 = w.x;
            v1 = w.y;
        }
        uint64_t k0, k1;
        double t0, t1;
        const bool g0 = kt_item<D>(p, sv, s0, v0, k0, t0);
        const bool g1 = kt_item<D>(p, sv, s1, v1, k1, t1);
        if (!(g0 && g1)) {
            set_error(p.status, kErrSubscript);
            if (!g0) { k0 = 0; t0 = 0.0; }
            if (!g1) { k1 = 0; t1 = 0.0; }
        }
        reinterpret_cast<ulonglong2*>(keys)[q] = make_ulonglong2(k0, k1);
        reinterpret_cast<double2*>(terms)[q] = make_double2(t0, t1);
        count(k0);
        count(k1);
    }
    // odd tail
    if ((p.nnz & 1) && tail && threadIdx.x == 0) {
        const int64_t k = p.nnz - 1;
        int64_t s0[D];
#pragma unroll
        for (int m = 0; m < D; ++m) s0[m] = p.subs[k * p.snz + m * p.smode];
        const double v0 = p.val_f32 ? (double)vf[k] : vd[k];
        uint64_t k0;
        double t0;
        if (!kt_item<D>(p, sv, s0, v0, k0, t0)) {
            set_error(p.status, kErrSubscript);
            k0 = 0;
            t0 = 0.0;
        }
        keys[k] = k0;
        terms[k] = t0;
        count(k0);
    }
}

template <int D, bool kSoA>
__global__ void __launch_bounds__(kKtThreads) k_keys_terms_vec(StreamDesc p, uint64_t* __restrict__ keys,
                                                               double* __restrict__ terms, int npass,
                                                               uint32_t* __restrict__ hist) {
    extern __shared__ double sv[];
    __shared__ uint32_t sh[kKtMaxPass * 256];
    for (int i = threadIdx.x; i < npass * 256; i += kKtThreads) sh[i] = 0;
    stage_vectors(p, sv);
    __syncthreads();
    kt_range<D, kSoA ? kLaySoA : kLayAoS>(p, sv, keys, terms, npass, sh, (int64_t)blockIdx.x * kKtThreads, p.nnz / 2,
                      (int64_t)gridDim.x * kKtThreads, blockIdx.x == 0);
    __syncthreads();
    for (int i = threadIdx.x; i < npass * 256; i += kKtThreads)
        if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

// Batched form: CTA c takes chunk c - prefix[j] (kKtBatchChunk nonzeros) of
// problem idx[j]; vectors are gathered from global memory (L2) rather than
// staged, a chunk being too short to repay staging a whole vector.
template <int D, int kLay>
__global__ void __launch_bounds__(kKtThreads) k_keys_terms_batch(const BatchJob* __restrict__ jobs, JobList l) {
    __shared__ uint32_t sh[kKtMaxPass * 256];
    __shared__ __align__(16) StreamDesc sp;
    __shared__ int s_pos;
    if (threadIdx.x == 0) {
        int lo = 0, hi = l.count;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (__ldg(l.prefix + mid) <= blockIdx.x) lo = mid;
            else hi = mid;
        }
        s_pos = lo;
    }
    __syncthreads();
    const int pos = s_pos;
    const BatchJob& J = jobs[__ldg(l.idx + pos)];
    static_assert(sizeof(StreamDesc) % 8 == 0, "descriptor copied in 8-byte words");
    for (int i = threadIdx.x; i < (int)(sizeof(StreamDesc) / 8); i += kKtThreads)
        reinterpret_cast<uint64_t*>(&sp)[i] = reinterpret_cast<const uint64_t*>(&J.p)[i];
    const int npass = J.npass;
    for (int i = threadIdx.x; i < npass * 256; i += kKtThreads) sh[i] = 0;
    __syncthreads();
    if (threadIdx.x == 0) sp.vec_smem = 0;
    __syncthreads();
    const int64_t chunk = (int64_t)blockIdx.x - __ldg(l.prefix + pos);
    const int64_t nchunks = (sp.nnz + kKtBatchChunk - 1) / kKtBatchChunk;
    const int64_t q0 = chunk * (kKtBatchChunk / 2);
    const int64_t q1 = min(sp.nnz / 2, q0 + kKtBatchChunk / 2);
    kt_range<D, kLay>(sp, nullptr, J.keys[0], J.vals[0], npass, sh, q0, q1, kKtThreads, chunk == nchunks - 1);
    __syncthreads();
    for (int i = threadIdx.x; i < npass * 256; i += kKtThreads)
        if (sh[i]) atomicAdd(&J.hist[i], sh[i]);
}

typedef void (*KtKernel)(StreamDesc, uint64_t*, double*, int, uint32_t*);

template <int D>
static KtKernel kt_pick(bool soa) {
    return soa ? k_keys_terms_vec<D, true> : k_keys_terms_vec<D, false>;
}

static KtKernel kt_kernel(int d, bool soa) {
    switch (d) {
        case 2: return kt_pick<2>(soa);
        case 3: return kt_pick<3>(soa);
        case 4: return kt_pick<4>(soa);
        case 5: return kt_pick<5>(soa);
        case 6: return kt_pick<6>(soa);
        case 7: return kt_pick<7>(soa);
        case 8: return kt_pick<8>(soa);
        default: return nullptr;
    }
}

// Whether the specialised kernel applies: order 2..8, 16-byte aligned
// subscripts and values, SoA with an even column stride or AoS.
bool keys_terms_vec_applicable(const StreamDesc& p, int npass) {
    if (p.d < 2 || p.d > 8 || npass > kKtMaxPass) return false;
    const uintptr_t sb = reinterpret_cast<uintptr_t>(p.subs), vb = reinterpret_cast<uintptr_t>(p.vals);
    if ((sb & 15) || (vb & 15)) return false;
    const bool soa = p.snz == 1 && (p.smode % 2 == 0);
    const bool aos = p.snz == p.d && p.smode == 1;
    return soa || aos;
}

// keys/terms: 16-byte aligned buffers of nnz entries; hist: npass x 256
// counters, zeroed by the caller.
void launch_keys_terms_vec(const StreamDesc& p, uint64_t* keys, double* terms, int npass, uint32_t* hist,
                           cudaStream_t stream) {
    if (p.nnz <= 0) return;
    KtKernel k = kt_kernel(p.d, p.snz == 1);
    const size_t smem = p.vec_smem ? (size_t)p.vtotal * sizeof(double) : 0;
    smem_at_least(k, smem);
    const int per_sm = p.ctas_per_sm > 0 ? p.ctas_per_sm : 8;
    const int64_t want = (p.nnz / 2 + kKtThreads - 1) / kKtThreads;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)num_sms() * per_sm));
    TTV_LAUNCH("keys_terms", stream, k<<<grid, kKtThreads, smem, stream>>>(p, keys, terms, npass, hist));
}

typedef void (*KtBatchKernel)(const BatchJob*, JobList);

template <int D>
static KtBatchKernel ktb_pick(int lay) {
    return lay == kLayAoS ? k_keys_terms_batch<D, kLayAoS>
                          : lay == kLaySoA ? k_keys_terms_batch<D, kLaySoA> : k_keys_terms_batch<D, kLayAny>;
}

// The batched key kernel's layout class of a problem: 0 AoS rows, 1 SoA
// columns with an even stride (both with 16-byte aligned subscripts and
// values), 2 anything else.
int keys_terms_batch_layout(const StreamDesc& p) {
    const uintptr_t sb = reinterpret_cast<uintptr_t>(p.subs), vb = reinterpret_cast<uintptr_t>(p.vals);
    const bool aligned = !(sb & 15) && !(vb & 15);
    if (aligned && p.snz == p.d && p.smode == 1) return kLayAoS;
    if (aligned && p.snz == 1 && p.smode % 2 == 0) return kLaySoA;
    return kLayAny;
}

// Keys, terms and digit counts of every problem in l (all of order d and
// layout class lay); units = total chunks.
void launch_keys_terms_batch(const BatchJob* jobs, const JobList& l, uint32_t units, int d, int lay,
                             cudaStream_t stream) {
    if (l.count <= 0 || units == 0) return;
    KtBatchKernel k = nullptr;
    switch (d) {
        case 2: k = ktb_pick<2>(lay); break;
        case 3: k = ktb_pick<3>(lay); break;
        case 4: k = ktb_pick<4>(lay); break;
        case 5: k = ktb_pick<5>(lay); break;
        case 6: k = ktb_pick<6>(lay); break;
        case 7: k = ktb_pick<7>(lay); break;
        case 8: k = ktb_pick<8>(lay); break;
        default: return;
    }
    TTV_LAUNCH("keys_terms_batch", stream, k<<<units, kKtThreads, 0, stream>>>(jobs, l));
}

}  // namespace ttv
