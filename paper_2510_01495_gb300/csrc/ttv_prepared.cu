// ttv_prepared.cu -- kernels that prepare a resident tensor for repeated TTVs
// along a fixed set of contracted modes.
//
// The result of a TTV along modes S has one row per distinct surviving tuple,
// in ascending key order (paper Sec. 3.3, Eq. 3, with pyttb's unique /
// accumarray grouping), and which nonzeros fall into which row depends only
// on the tensor, not on the vectors.  Preparing sorts the nonzeros once by
// their key (stable: equal keys keep input order) and stores, in that order,
// the values and the contracted modes' subscripts (int32), plus a bitmap of
// where each result row starts and each row's key.  A later TTV with fresh
// vectors is then a single streaming reduce-by-key over these arrays
// (ttv_sort.cu, PrepTerms with BitHeads): no radix passes, and 12 bytes read
// per nonzero (binary64 values, one vector) instead of a key and a term.
#include <algorithm>

#include "ttv_internal.cuh"

namespace ttv {

// key of every nonzero, and its index (stored in the sort's 8-byte payload)
__global__ void __launch_bounds__(256) k_prep_keys(StreamDesc p, uint64_t* __restrict__ keys,
                                                   double* __restrict__ idx) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < p.nnz; k += stride) {
        uint64_t key = 0;
        bool good = true;
        for (int m = 0; m < p.d; ++m) {
            const int64_t s = p.subs[k * p.snz + m * p.smode];
            good &= (uint64_t)s < (uint64_t)p.shape[m];
            if (!((p.smask >> m) & 1u)) key += (uint64_t)(good ? s : 0) * p.kstride[m];
        }
        if (!good) {
            set_error(p.status, kErrSubscript);
            key = 0;
        }
        keys[k] = key;
        idx[k] = __longlong_as_double(k);
    }
}

// values and contracted subscripts (the j-th contracted mode in increasing
// order goes to out_subs.sub[j]) in key order
__global__ void __launch_bounds__(256) k_prep_gather(StreamDesc p, const double* __restrict__ idx_sorted,
                                                     void* __restrict__ vals_out, PrepTerms out_subs) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p.nnz; i += stride) {
        const int64_t k = (int64_t)__double_as_longlong(idx_sorted[i]);
        if (p.val_f32) static_cast<float*>(vals_out)[i] = static_cast<const float*>(p.vals)[k];
        else static_cast<double*>(vals_out)[i] = static_cast<const double*>(p.vals)[k];
        int j = 0;
        for (int m = 0; m < p.d; ++m)
            if ((p.smask >> m) & 1u)
                const_cast<int32_t*>(out_subs.sub[j++])[i] = (int32_t)p.subs[k * p.snz + m * p.smode];
    }
}

// distinct keys of a sorted key array
__global__ void __launch_bounds__(256) k_prep_count(const uint64_t* __restrict__ keys, int64_t n,
                                                    unsigned long long* __restrict__ count) {
    unsigned long long c = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        c += (i == 0 || keys[i] != keys[i - 1]) ? 1ull : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

// head bitmap of a sorted key array: bit i of word i/32 set when i starts a run
__global__ void __launch_bounds__(256) k_prep_heads(const uint64_t* __restrict__ keys, int64_t n,
                                                    uint32_t* __restrict__ bits) {
    const int lane = threadIdx.x & 31;
    const int64_t nwords = (n + 31) / 32;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < nwords; w += warps) {
        const int64_t i = w * 32 + lane;
        const bool head = i < n && (i == 0 || keys[i] != keys[i - 1]);
        const uint32_t b = __ballot_sync(0xffffffffu, head);
        if (lane == 0) bits[w] = b;
    }
}

void launch_prep_heads(const uint64_t* keys, int64_t n, uint32_t* bits, cudaStream_t stream) {
    if (n <= 0) return;
    const int64_t nwords = (n + 31) / 32;
    const int g = (int)std::max<int64_t>(1, std::min<int64_t>((nwords * 32 + 255) / 256, (int64_t)num_sms() * 8));
    TTV_LAUNCH("prep_heads", stream, k_prep_heads<<<g, 256, 0, stream>>>(keys, n, bits));
}

void launch_prep_keys(const StreamDesc& p, uint64_t* keys, double* idx, cudaStream_t stream) {
    if (p.nnz <= 0) return;
    const int g = (int)std::max<int64_t>(1, std::min<int64_t>((p.nnz + 255) / 256, (int64_t)num_sms() * 8));
    TTV_LAUNCH("prep_keys", stream, k_prep_keys<<<g, 256, 0, stream>>>(p, keys, idx));
}

void launch_prep_gather(const StreamDesc& p, const double* idx_sorted, void* vals_out, const PrepTerms& subs,
                        cudaStream_t stream) {
    if (p.nnz <= 0) return;
    const int g = (int)std::max<int64_t>(1, std::min<int64_t>((p.nnz + 255) / 256, (int64_t)num_sms() * 8));
    TTV_LAUNCH("prep_gather", stream, k_prep_gather<<<g, 256, 0, stream>>>(p, idx_sorted, vals_out, subs));
}

void launch_prep_count(const uint64_t* keys, int64_t n, unsigned long long* count, cudaStream_t stream) {
    if (n <= 0) return;
    const int g = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)num_sms() * 8));
    TTV_LAUNCH("prep_count", stream, k_prep_count<<<g, 256, 0, stream>>>(keys, n, count));
}

}  // namespace ttv
