// ttv_stream.cu -- the streaming pass over the nonzeros (gather, scale,
// linearise) and the dense-accumulator path for small result key spaces.
//
// Every kernel here reads subs/vals exactly once with streaming (evict-first)
// loads, forms the term vals[k] * prod_{m in S} x_m[subs[k,m]] in increasing
// mode order, and the row-major key of the surviving subscripts (paper
// Sec. 3.3, Eq. 3).  A subscript outside its mode is skipped and flagged.
#include <algorithm>

#include "ttv_internal.cuh"

namespace ttv {

constexpr int kStreamThreads = 256;
constexpr int kUnroll = 4;

// ---------------------------------------------------------------------------
// (key, term) for every nonzero, for the sort path.
__global__ void __launch_bounds__(kStreamThreads) k_keys_terms(StreamDesc p, uint64_t* __restrict__ keys,
                                                               double* __restrict__ terms) {
    extern __shared__ double sv[];
    stage_vectors(p, sv);
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k0 < p.nnz; k0 += stride * kUnroll) {
        int64_t ks[kUnroll];
        bool ok[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            ks[u] = k0 + u * stride;
            ok[u] = ks[u] < p.nnz;
        }
        Batch<kUnroll> b;
        load_batch<kUnroll>(p, ks, ok, b);
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            if (!ok[u]) continue;
            uint64_t key;
            double t;
            if (!key_term(p, sv, b.s[u], b.v[u], key, t)) {
                set_error(p.status, kErrSubscript);
                key = 0;
                t = 0.0;
            }
            keys[ks[u]] = key;
            terms[ks[u]] = t;
        }
    }
}

void launch_keys_terms(const StreamDesc& p, uint64_t* keys, double* terms, cudaStream_t stream) {
    if (p.nnz <= 0) return;
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = p.vec_smem ? (size_t)p.vtotal * sizeof(double) : 0;
    smem_at_least(k_keys_terms, smem);
    const int64_t want = (p.nnz + kStreamThreads * kUnroll - 1) / (kStreamThreads * kUnroll);
    const int per_sm = p.ctas_per_sm > 0 ? p.ctas_per_sm : 8;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)nsm * per_sm));
    TTV_LAUNCH("keys_terms", stream, k_keys_terms<<<grid, kStreamThreads, smem, stream>>>(p, keys, terms));
}

// ---------------------------------------------------------------------------
// Dense path: each CTA accumulates a contiguous chunk of nonzeros into a
// private shared-memory array over the whole key space (plus a presence
// bitmap when the result is sparse), then writes its partial array.  A second
// kernel combines the partials cell by cell in a fixed order.
struct DenseSmemLayout {
    size_t acc_off, pres_off, vec_off, total;
};

// Products on integer units (exact significand multiplies) instead of the
// binary64 chain.  Off until the order-specialised kernels land: in the
// generic kernel the extra integer instructions cost more than the FP64
// multiplies they replace.
static int use_int_products(const StreamDesc& p) { (void)p; return 0; }

static DenseSmemLayout dense_layout(const StreamDesc& p, int want_presence) {
    DenseSmemLayout L;
    L.acc_off = 0;
    size_t off = (size_t)p.nkeys * sizeof(double);
    L.pres_off = off;
    if (want_presence) off += ((p.nkeys + 31) / 32) * sizeof(uint32_t);
    off = (off + 15) & ~size_t(15);
    L.vec_off = off;
    if (p.vec_smem) off += (size_t)p.vtotal * (use_int_products(p) ? sizeof(SigEntry) : sizeof(double));
    L.total = off;
    return L;
}

template <bool kIntProducts>
__global__ void __launch_bounds__(kStreamThreads) k_dense_accum(StreamDesc p, int64_t chunk, int want_presence,
                                                                size_t pres_off, size_t vec_off,
                                                                double* __restrict__ partials,
                                                                uint32_t* __restrict__ pres_partials) {
    extern __shared__ __align__(16) unsigned char dsm[];
    double* acc = reinterpret_cast<double*>(dsm);
    uint32_t* pres = reinterpret_cast<uint32_t*>(dsm + pres_off);
    double* sv = reinterpret_cast<double*>(dsm + vec_off);
    SigEntry* sve = reinterpret_cast<SigEntry*>(dsm + vec_off);
    const int64_t P = (int64_t)p.nkeys;
    const int64_t npres = (P + 31) / 32;
    for (int64_t i = threadIdx.x; i < P; i += blockDim.x) acc[i] = 0.0;
    if (want_presence)
        for (int64_t i = threadIdx.x; i < npres; i += blockDim.x) pres[i] = 0u;
    if (kIntProducts) stage_vectors_sig(p, sve);
    else stage_vectors(p, sv);
    __syncthreads();

    const int64_t lo = (int64_t)blockIdx.x * chunk;
    const int64_t hi = min(p.nnz, lo + chunk);
    for (int64_t k0 = lo + threadIdx.x; k0 < hi; k0 += (int64_t)blockDim.x * kUnroll) {
        int64_t ks[kUnroll];
        bool ok[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            ks[u] = k0 + (int64_t)u * blockDim.x;
            ok[u] = ks[u] < hi;
        }
        Batch<kUnroll> b;
        load_batch<kUnroll>(p, ks, ok, b);
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            if (!ok[u]) continue;
            uint64_t key;
            double t;
            bool good;
            if constexpr (kIntProducts) good = key_term_sig(p, sve, b.s[u], b.v[u], key, t);
            else good = key_term(p, sv, b.s[u], b.v[u], key, t);
            if (!good) {
                set_error(p.status, kErrSubscript);
                continue;
            }
            atomicAdd(&acc[key], t);
            if (want_presence) atomicOr(&pres[key >> 5], 1u << (key & 31));
        }
    }
    __syncthreads();
    double* my = partials + (size_t)blockIdx.x * P;
    for (int64_t i = threadIdx.x; i < P; i += blockDim.x) my[i] = acc[i];
    if (want_presence) {
        uint32_t* mp = pres_partials + (size_t)blockIdx.x * npres;
        for (int64_t i = threadIdx.x; i < npres; i += blockDim.x) mp[i] = pres[i];
    }
}

// One warp per cell: lane l sums partials l, l+32, ... then a fixed shuffle
// tree; the order never depends on timing.
__global__ void __launch_bounds__(256) k_dense_reduce(int64_t P, int G, const double* __restrict__ partials,
                                                      const uint32_t* __restrict__ pres_partials, int want_presence,
                                                      int compensated, double* __restrict__ cell_vals,
                                                      uint32_t* __restrict__ cell_flags) {
    const int lane = threadIdx.x & 31;
    const int64_t cell = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (cell >= P) return;
    const int64_t npres = (P + 31) / 32;
    double sum = 0.0, comp = 0.0;
    uint32_t any = 0;
    for (int b = lane; b < G; b += 32) {
        const double x = partials[(size_t)b * P + cell];
        if (compensated) {
            const double s = sum + x, bp = s - sum;
            comp += (sum - (s - bp)) + (x - bp);
            sum = s;
        } else {
            sum += x;
        }
        if (want_presence) any |= (pres_partials[(size_t)b * npres + (cell >> 5)] >> (cell & 31)) & 1u;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const double os = __shfl_xor_sync(0xffffffffu, sum, off);
        const double oc = __shfl_xor_sync(0xffffffffu, comp, off);
        const bool lower = (lane & off) == 0;
        if (compensated) {
            const double a = lower ? sum : os, b2 = lower ? os : sum;
            const double s = a + b2, bp = s - a;
            const double e = (a - (s - bp)) + (b2 - bp);
            comp = (lower ? comp + oc : oc + comp) + e;
            sum = s;
        } else {
            sum = lower ? sum + os : os + sum;
        }
    }
    any = __any_sync(0xffffffffu, any) ? 1u : 0u;
    if (lane == 0) {
        cell_vals[cell] = (compensated && isfinite(sum)) ? sum + comp : sum;   // an infinite sum stays infinite
        if (want_presence) cell_flags[cell] = any;
    }
}

// Sparse result from the dense path: present cells in ascending key order.
// One CTA of 1024 threads; each owns a contiguous run of cells.
__global__ void __launch_bounds__(1024) k_compact_cells(StreamDesc p, const double* __restrict__ cell_vals,
                                                        const uint32_t* __restrict__ cell_flags, int64_t cap_rows,
                                                        int64_t* __restrict__ out_subs, double* __restrict__ out_vals) {
    __shared__ uint32_t wt[32];
    const int64_t P = (int64_t)p.nkeys;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t per = (P + 1023) / 1024;
    const int64_t c0 = (int64_t)tid * per, c1 = min(P, c0 + per);
    uint32_t cnt = 0;
    for (int64_t c = c0; c < c1; ++c) cnt += cell_flags[c] ? 1u : 0u;
    uint32_t inc = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) wt[warp] = inc;
    __syncthreads();
    uint32_t before = 0, total = 0;
    for (int w = 0; w < 32; ++w) {
        if (w < warp) before += wt[w];
        total += wt[w];
    }
    if (tid == 0) p.status->nnz_out = total;
    if ((int64_t)total > cap_rows) {
        if (tid == 0) set_error(p.status, kErrCapacity);
        return;
    }
    uint32_t pos = before + inc - cnt;
    for (int64_t c = c0; c < c1; ++c) {
        if (!cell_flags[c]) continue;
        if (p.nr > 0) delinearise(p, (uint64_t)c, out_subs + (int64_t)pos * p.nr);
        out_vals[pos] = cell_vals[c];
        ++pos;
    }
}

size_t dense_smem_bytes(const StreamDesc& p, int want_presence) { return dense_layout(p, want_presence).total; }

// order-specialised kernel (ttv_dense_vec.cu)
bool dense_vec_applicable(const StreamDesc& p);
int dense_vec_grid(const StreamDesc& p, int want_presence);
void launch_dense_vec(const StreamDesc& p, int want_presence, int G, double* partials, uint32_t* pres_partials,
                      cudaStream_t stream);

int dense_grid(const StreamDesc& p, int want_presence) {
    if (dense_vec_applicable(p)) return dense_vec_grid(p, want_presence);
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = dense_layout(p, want_presence).total;
    int per_sm = 1;
    if (use_int_products(p)) {
        smem_at_least(k_dense_accum<true>, smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dense_accum<true>, kStreamThreads, smem);
    } else {
        smem_at_least(k_dense_accum<false>, smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dense_accum<false>, kStreamThreads, smem);
    }
    per_sm = std::max(1, std::min(per_sm, p.ctas_per_sm > 0 ? p.ctas_per_sm : 4));
    // at least ~4 unrolled sweeps of the block per CTA so that zeroing and
    // writing the partial array stay small next to the streaming work
    const int64_t min_chunk = std::max<int64_t>((int64_t)kStreamThreads * kUnroll * 4, (int64_t)p.nkeys * 4);
    const int64_t by_work = std::max<int64_t>(1, (p.nnz + min_chunk - 1) / min_chunk);
    return (int)std::max<int64_t>(1, std::min<int64_t>(by_work, (int64_t)nsm * per_sm));
}

void launch_dense(const StreamDesc& p, int want_presence, int compensated, int G, double* partials,
                  uint32_t* pres_partials, double* cell_vals, uint32_t* cell_flags, cudaStream_t stream) {
    const DenseSmemLayout L = dense_layout(p, want_presence);
    const int64_t chunk = std::max<int64_t>(1, (p.nnz + G - 1) / G);
    if (dense_vec_applicable(p)) {
        launch_dense_vec(p, want_presence, G, partials, pres_partials, stream);
    } else if (use_int_products(p)) {
        smem_at_least(k_dense_accum<true>, L.total);
        TTV_LAUNCH("dense_accum", stream, k_dense_accum<true><<<G, kStreamThreads, L.total, stream>>>(
                                              p, chunk, want_presence, L.pres_off, L.vec_off, partials, pres_partials));
    } else {
        smem_at_least(k_dense_accum<false>, L.total);
        TTV_LAUNCH("dense_accum", stream, k_dense_accum<false><<<G, kStreamThreads, L.total, stream>>>(
                                              p, chunk, want_presence, L.pres_off, L.vec_off, partials, pres_partials));
    }
    const int64_t P = (int64_t)p.nkeys;
    const int64_t blocks = (P * 32 + 255) / 256;
    TTV_LAUNCH("dense_reduce", stream, k_dense_reduce<<<(unsigned)blocks, 256, 0, stream>>>(P, G, partials, pres_partials, want_presence, compensated,
                                                        cell_vals, cell_flags));
}

void launch_compact_cells(const StreamDesc& p, const double* cell_vals, const uint32_t* cell_flags, int64_t cap_rows,
                          int64_t* out_subs, double* out_vals, cudaStream_t stream) {
    TTV_LAUNCH("compact_cells", stream, k_compact_cells<<<1, 1024, 0, stream>>>(p, cell_vals, cell_flags, cap_rows, out_subs, out_vals));
}

}  // namespace ttv
