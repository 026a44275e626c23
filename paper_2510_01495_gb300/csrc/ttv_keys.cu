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

template <int D, bool kSoA>
__global__ void __launch_bounds__(kKtThreads) k_keys_terms_vec(StreamDesc p, uint64_t* __restrict__ keys,
                                                               double* __restrict__ terms, int npass,
                                                               uint32_t* __restrict__ hist) {
    extern __shared__ double sv[];
    __shared__ uint32_t sh[kKtMaxPass * 256];
    for (int i = threadIdx.x; i < npass * 256; i += kKtThreads) sh[i] = 0;
    stage_vectors(p, sv);
    __syncthreads();
    const double* vd = static_cast<const double*>(p.vals);
    const float* vf = static_cast<const float*>(p.vals);
    const int64_t npairs = p.nnz / 2;
    const int64_t stride = (int64_t)gridDim.x * kKtThreads;
    auto count = [&](uint64_t key) {
        for (int q = 0; q < npass; ++q) atomicAdd(&sh[q * 256 + ((key >> (8 * q)) & 255u)], 1u);
    };
    for (int64_t q = (int64_t)blockIdx.x * kKtThreads + threadIdx.x; q < npairs; q += stride) {
        const int64_t k = 2 * q;
        int64_t s0[D], s1[D];
        if constexpr (kSoA) {
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
        if (p.val_f32) {
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
    if ((p.nnz & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
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
    __syncthreads();
    for (int i = threadIdx.x; i < npass * 256; i += kKtThreads)
        if (sh[i]) atomicAdd(&hist[i], sh[i]);
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
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)std::max<size_t>(smem, 1));
    const int per_sm = p.ctas_per_sm > 0 ? p.ctas_per_sm : 8;
    const int64_t want = (p.nnz / 2 + kKtThreads - 1) / kKtThreads;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)num_sms() * per_sm));
    TTV_LAUNCH("keys_terms", stream, k<<<grid, kKtThreads, smem, stream>>>(p, keys, terms, npass, hist));
}

}  // namespace ttv
