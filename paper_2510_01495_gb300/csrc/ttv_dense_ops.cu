// ttv_dense_ops.cu -- the paper's two simple kernels on dense operands:
// the vector dot product (Sec. 3.1, Eq. 1) and the dense matrix-vector
// product (Sec. 3.2, Eq. 2).
//
//     x . y = sum_i x[i] * y[i]            y[i] = sum_j A(i, j) * x[j]
//
// Both stream their operands once and are bound by HBM on paper, but GB300's
// binary64 rate (about 5.3e11 fused multiply-adds per second) caps a
// one-multiply-add-per-element loop at 8 bytes per multiply-add: 4.2 TB/s
// for the matrix, 8.5 TB/s for the dot product's two streams.  So every
// element costs exactly one fused multiply-add and nothing else in binary64;
// the cross-lane and cross-CTA combination is a fixed shuffle tree and a
// fixed-order pass over per-CTA partials, so results are bit-identical from
// run to run.
//
// A(i, j) is A[i * stride_row + j * stride_col]: row-major storage has
// strides (n2, 1), pyttb's column-major storage (1, n1).
#include <algorithm>

#include "ttv_internal.cuh"

namespace ttv {

constexpr int kDotThreads = 256;
constexpr int kDotCtasPerSm = 8;

template <bool kF32>
__device__ __forceinline__ void dot_pair(const void* x, const void* y, int64_t q, double& a0, double& a1) {
    if constexpr (kF32) {
        const float2 u = __ldcs(reinterpret_cast<const float2*>(x) + q);
        const float2 v = __ldcs(reinterpret_cast<const float2*>(y) + q);
        a0 = fma((double)u.x, (double)v.x, a0);
        a1 = fma((double)u.y, (double)v.y, a1);
    } else {
        const double2 u = __ldcs(reinterpret_cast<const double2*>(x) + q);
        const double2 v = __ldcs(reinterpret_cast<const double2*>(y) + q);
        a0 = fma(u.x, v.x, a0);
        a1 = fma(u.y, v.y, a1);
    }
}

// Fixed-order block sum of one double per thread; the result is valid in
// thread 0.
__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = v + __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) sh[w] = v;
    __syncthreads();
    if (w == 0) {
        v = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = v + __shfl_xor_sync(0xffffffffu, v, o);
    }
    return v;
}

// Per-CTA partial sums: thread t takes element pairs t, t + T, ... (T = all
// threads), two running multiply-add chains per thread, unrolled by two
// pairs.  Vector loads need both bases 16-byte (f64) / 8-byte (f32)
// aligned; otherwise elements are read one at a time.
template <bool kF32>
__global__ void __launch_bounds__(kDotThreads) k_dot(const void* __restrict__ x, const void* __restrict__ y,
                                                     int64_t n, int vec, double* __restrict__ partial) {
    __shared__ double sh[kDotThreads / 32];
    const int64_t T = (int64_t)gridDim.x * kDotThreads;
    const int64_t t = (int64_t)blockIdx.x * kDotThreads + threadIdx.x;
    double a0 = 0.0, a1 = 0.0, b0 = 0.0, b1 = 0.0;
    int64_t tail = 0;
    if (vec) {
        const int64_t npairs = n / 2;
        int64_t q = t;
        for (; q + T < npairs; q += 2 * T) {
            dot_pair<kF32>(x, y, q, a0, a1);
            dot_pair<kF32>(x, y, q + T, b0, b1);
        }
        if (q < npairs) dot_pair<kF32>(x, y, q, a0, a1);
        tail = 2 * npairs;
    }
    for (int64_t i = tail + t; i < n; i += T) {
        if constexpr (kF32)
            a0 = fma((double)reinterpret_cast<const float*>(x)[i], (double)reinterpret_cast<const float*>(y)[i], a0);
        else
            a0 = fma(reinterpret_cast<const double*>(x)[i], reinterpret_cast<const double*>(y)[i], a0);
    }
    const double v = block_sum((a0 + a1) + (b0 + b1), sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = v;
}

// One CTA: thread t sums partials t, t + 1024, ... in order, then the tree.
__global__ void __launch_bounds__(1024) k_sum_partials(const double* __restrict__ partial, int n,
                                                       double* __restrict__ out) {
    __shared__ double sh[32];
    double v = 0.0;
    for (int i = threadIdx.x; i < n; i += 1024) v = v + partial[i];
    v = block_sum(v, sh);
    if (threadIdx.x == 0) *out = v;
}

int dot_grid(int64_t n) {
    const int64_t want = (n / 2 + kDotThreads - 1) / kDotThreads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)num_sms() * kDotCtasPerSm));
}

size_t dot_workspace_bytes(int64_t n) { return (size_t)dot_grid(n) * sizeof(double); }

void launch_dot(const void* x, const void* y, int64_t n, bool f32, double* out, void* ws, cudaStream_t stream) {
    if (n <= 0) {
        cudaMemsetAsync(out, 0, sizeof(double), stream);
        return;
    }
    const int g = dot_grid(n);
    const uintptr_t al = f32 ? 8 : 16;
    const int vec = (reinterpret_cast<uintptr_t>(x) % al == 0) && (reinterpret_cast<uintptr_t>(y) % al == 0);
    double* partial = static_cast<double*>(ws);
    if (f32) TTV_LAUNCH("dot", stream, k_dot<true><<<g, kDotThreads, 0, stream>>>(x, y, n, vec, partial));
    else TTV_LAUNCH("dot", stream, k_dot<false><<<g, kDotThreads, 0, stream>>>(x, y, n, vec, partial));
    TTV_LAUNCH("dot_final", stream, k_sum_partials<<<1, 1024, 0, stream>>>(partial, g, out));
}

// ---- canonical COO -> dense (the automatic result format) ----------------------------

struct DenseShape {
    int order;
    int64_t shape[kMaxD];
};

__global__ void __launch_bounds__(256) k_coo_to_dense(const int64_t* __restrict__ subs, const double* __restrict__ vals,
                                                      int64_t n, DenseShape sh, double* __restrict__ dense) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
        int64_t key = 0;
        for (int j = 0; j < sh.order; ++j) key = key * sh.shape[j] + subs[r * sh.order + j];
        dense[key] = vals[r];
    }
}

// dense (ncells doubles) = 0, then every row's value at its row-major cell;
// the rows are distinct, so the order of the writes does not matter.
void launch_coo_to_dense(const int64_t* subs, const double* vals, int64_t n, int order, const int64_t* shape,
                         double* dense, int64_t ncells, cudaStream_t stream) {
    cudaMemsetAsync(dense, 0, (size_t)std::max<int64_t>(ncells, 1) * sizeof(double), stream);
    if (n <= 0) return;
    DenseShape sh{};
    sh.order = order;
    for (int j = 0; j < order && j < kMaxD; ++j) sh.shape[j] = shape[j];
    const int g = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)num_sms() * 8));
    TTV_LAUNCH("coo_to_dense", stream, k_coo_to_dense<<<g, 256, 0, stream>>>(subs, vals, n, sh, dense));
}

// ---- matrix-vector product ----------------------------------------------------------

constexpr int kMvThreads = 256;
constexpr int kMvRowsPerLane = 4;      // column-major: rows per lane (128 per warp)

struct MvArgs {
    const void* A;
    const void* x;
    int64_t n1, n2, sr, sc;
    int64_t nchunks, chunk;           // column chunks and their length
    double* y;                        // written directly when nchunks == 1
    double* partial;                  // nchunks x n1 otherwise
    int pair;                         // rows kernel: element pairs with one vector load each
};

template <bool kF32>
__device__ __forceinline__ double2 ld2_stream(const void* p, int64_t i) {
    if constexpr (kF32) {
        const float2 v = __ldcs(reinterpret_cast<const float2*>(reinterpret_cast<const float*>(p) + i));
        return make_double2((double)v.x, (double)v.y);
    } else {
        return __ldcs(reinterpret_cast<const double2*>(reinterpret_cast<const double*>(p) + i));
    }
}
template <bool kF32>
__device__ __forceinline__ double2 ld2(const void* p, int64_t i) {
    if constexpr (kF32) {
        const float2 v = __ldg(reinterpret_cast<const float2*>(reinterpret_cast<const float*>(p) + i));
        return make_double2((double)v.x, (double)v.y);
    } else {
        return __ldg(reinterpret_cast<const double2*>(reinterpret_cast<const double*>(p) + i));
    }
}

template <bool kF32>
__device__ __forceinline__ double ld(const void* p, int64_t i) {
    if constexpr (kF32) return (double)__ldg(reinterpret_cast<const float*>(p) + i);
    else return __ldg(reinterpret_cast<const double*>(p) + i);
}
template <bool kF32>
__device__ __forceinline__ double ld_stream(const void* p, int64_t i) {
    if constexpr (kF32) return (double)__ldcs(reinterpret_cast<const float*>(p) + i);
    else return __ldcs(reinterpret_cast<const double*>(p) + i);
}

// Rows contiguous (stride_col == 1).  A group of kG lanes takes one (row,
// column chunk): its lanes stride the chunk's elements with four running
// multiply-adds each, then a fixed shuffle tree inside the group.
template <int kG, bool kF32>
__global__ void __launch_bounds__(kMvThreads) k_mv_rows(MvArgs a) {
    constexpr int kGroups = 32 / kG;
    const int lane = threadIdx.x & 31, gl = lane % kG, grp = lane / kG;
    const int64_t items = a.n1 * a.nchunks;
    const int64_t nwarps = ((int64_t)gridDim.x * kMvThreads) >> 5;
    for (int64_t w = ((int64_t)blockIdx.x * kMvThreads + threadIdx.x) >> 5; w * kGroups < items; w += nwarps) {
        const int64_t it = w * kGroups + grp;        // item: chunk-major, so neighbours share the chunk of x
        double s = 0.0;
        int64_t row = 0, c = 0;
        if (it < items) {
            c = it / a.n1;
            row = it - c * a.n1;
            const int64_t j0 = c * a.chunk, j1 = min(a.n2, j0 + a.chunk);
            const int64_t base = row * a.sr;
            double acc[4] = {0.0, 0.0, 0.0, 0.0};
            if (a.pair) {
                // lane gl takes elements (j, j + 1), j = j0 + 2 gl + 2 kG t: one
                // vector load of A and of x per pair (base and j0 are even)
                int64_t j = j0 + 2 * gl;
                for (; j + 6 * kG + 1 < j1; j += 8 * kG) {
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const double2 av = ld2_stream<kF32>(a.A, base + j + 2 * kG * u);
                        const double2 xv = ld2<kF32>(a.x, j + 2 * kG * u);
                        acc[u] = fma(av.x, xv.x, acc[u]);
                        acc[u] = fma(av.y, xv.y, acc[u]);
                    }
                }
                for (; j + 1 < j1; j += 2 * kG) {
                    const double2 av = ld2_stream<kF32>(a.A, base + j);
                    const double2 xv = ld2<kF32>(a.x, j);
                    acc[0] = fma(av.x, xv.x, acc[0]);
                    acc[0] = fma(av.y, xv.y, acc[0]);
                }
                if (j < j1) acc[1] = fma(ld_stream<kF32>(a.A, base + j), ld<kF32>(a.x, j), acc[1]);
            } else {
                int64_t j = j0 + gl;
                for (; j + 3 * kG < j1; j += 4 * kG) {
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        acc[u] = fma(ld_stream<kF32>(a.A, base + j + u * kG), ld<kF32>(a.x, j + u * kG), acc[u]);
                }
                for (; j < j1; j += kG) acc[0] = fma(ld_stream<kF32>(a.A, base + j), ld<kF32>(a.x, j), acc[0]);
            }
            s = (acc[0] + acc[1]) + (acc[2] + acc[3]);
        }
#pragma unroll
        for (int o = kG / 2; o > 0; o >>= 1) s = s + __shfl_xor_sync(0xffffffffu, s, o);
        if (it < items && gl == 0) {
            if (a.nchunks == 1) a.y[row] = s;
            else a.partial[c * a.n1 + row] = s;
        }
    }
}

// Columns contiguous (stride_row == 1).  A warp takes 128 consecutive rows
// (lane l: rows l, l + 32, l + 64, l + 96) over one column chunk: per column
// one coalesced 256-byte load per row quarter and a broadcast x[j].
template <bool kF32>
__global__ void __launch_bounds__(kMvThreads) k_mv_cols(MvArgs a) {
    constexpr int kRows = 32 * kMvRowsPerLane;
    const int lane = threadIdx.x & 31;
    const int64_t rblocks = (a.n1 + kRows - 1) / kRows;
    const int64_t items = rblocks * a.nchunks;
    const int64_t nwarps = ((int64_t)gridDim.x * kMvThreads) >> 5;
    for (int64_t it = ((int64_t)blockIdx.x * kMvThreads + threadIdx.x) >> 5; it < items; it += nwarps) {
        const int64_t c = it / rblocks, rb = it - c * rblocks;
        const int64_t r0 = rb * kRows + lane;
        const int64_t j0 = c * a.chunk, j1 = min(a.n2, j0 + a.chunk);
        double acc[kMvRowsPerLane];
        bool ok[kMvRowsPerLane];
#pragma unroll
        for (int q = 0; q < kMvRowsPerLane; ++q) {
            acc[q] = 0.0;
            ok[q] = r0 + 32 * q < a.n1;
        }
        for (int64_t j = j0; j < j1; ++j) {
            const double xj = ld<kF32>(a.x, j);
            const int64_t col = j * a.sc;
#pragma unroll
            for (int q = 0; q < kMvRowsPerLane; ++q)
                if (ok[q]) acc[q] = fma(ld_stream<kF32>(a.A, col + r0 + 32 * q), xj, acc[q]);
        }
#pragma unroll
        for (int q = 0; q < kMvRowsPerLane; ++q)
            if (ok[q]) {
                if (a.nchunks == 1) a.y[r0 + 32 * q] = acc[q];
                else a.partial[c * a.n1 + r0 + 32 * q] = acc[q];
            }
    }
}

// y[i] = sum over chunks, in chunk order.
__global__ void __launch_bounds__(256) k_mv_reduce(const double* __restrict__ partial, int64_t n1, int64_t nchunks,
                                                   double* __restrict__ y) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n1; i += stride) {
        double s = 0.0;
        for (int64_t c = 0; c < nchunks; ++c) s = s + partial[c * n1 + i];
        y[i] = s;
    }
}

struct MvPlan {
    bool rows;          // rows contiguous
    int g;              // lanes per row (rows kernel)
    int64_t nchunks, chunk;
};

// The rows kernel reads A[i * sr + j] (any sr; needs unit column stride or a
// single column), the columns kernel A[j * sc + i] (any sc; needs unit row
// stride or a single row).
static MvPlan mv_plan(int64_t n1, int64_t n2, int64_t sr, int64_t sc) {
    MvPlan p{};
    p.rows = (sc == 1 && n2 > 1) || !(sr == 1 || n1 == 1);
    // enough independent items for every SM: about 32 warps' worth per SM
    const int64_t want = (int64_t)num_sms() * 32;
    if (p.rows) {
        int64_t nc = std::max<int64_t>(1, std::min<int64_t>((want + n1 - 1) / n1, (n2 + 1023) / 1024));
        p.chunk = (n2 + nc - 1) / nc;
        p.chunk = (p.chunk + 63) / 64 * 64;
        p.nchunks = std::max<int64_t>(1, (n2 + p.chunk - 1) / p.chunk);
        const int64_t per = std::min(p.chunk, n2) / 8;      // lanes so that each has at least 8 elements
        p.g = per >= 32 ? 32 : per >= 16 ? 16 : per >= 8 ? 8 : per >= 4 ? 4 : per >= 2 ? 2 : 1;
    } else {
        const int64_t rblocks = (n1 + 32 * kMvRowsPerLane - 1) / (32 * kMvRowsPerLane);
        int64_t nc = std::max<int64_t>(1, std::min<int64_t>((want + rblocks - 1) / rblocks, (n2 + 63) / 64));
        p.chunk = (n2 + nc - 1) / nc;
        p.nchunks = std::max<int64_t>(1, (n2 + p.chunk - 1) / p.chunk);
        p.g = 32;
    }
    return p;
}

// Layouts the kernels take: unit column stride (rows contiguous), unit row
// stride (columns contiguous), or a single row or column with any stride.
bool matvec_layout_ok(int64_t n1, int64_t n2, int64_t sr, int64_t sc) {
    return sc == 1 || sr == 1 || n1 == 1 || n2 == 1;
}

size_t matvec_workspace_bytes(int64_t n1, int64_t n2, int64_t sr, int64_t sc) {
    if (n1 <= 0 || n2 <= 0) return 0;
    const MvPlan p = mv_plan(n1, n2, sr, sc);
    return p.nchunks > 1 ? (size_t)p.nchunks * n1 * sizeof(double) : 0;
}

void launch_matvec(const void* A, int64_t n1, int64_t n2, int64_t sr, int64_t sc, bool f32, const void* x,
                   double* y, void* ws, cudaStream_t stream) {
    if (n1 <= 0) return;
    if (n2 <= 0) {
        cudaMemsetAsync(y, 0, (size_t)n1 * sizeof(double), stream);
        return;
    }
    const MvPlan p = mv_plan(n1, n2, sr, sc);
    MvArgs a{A, x, n1, n2, sr, sc, p.nchunks, p.chunk, y, static_cast<double*>(ws), 0};
    const uintptr_t al = f32 ? 8 : 16;
    a.pair = p.rows && sc == 1 && (sr % 2 == 0 || n1 == 1) && reinterpret_cast<uintptr_t>(A) % al == 0 &&
             reinterpret_cast<uintptr_t>(x) % al == 0 && (p.nchunks == 1 || p.chunk % 2 == 0);
    auto grid = [](int64_t warps) {
        return (int)std::max<int64_t>(1, std::min<int64_t>((warps * 32 + kMvThreads - 1) / kMvThreads,
                                                           (int64_t)num_sms() * 8));
    };
    if (p.rows) {
        const int64_t warps = (n1 * p.nchunks * p.g + 31) / 32;
        const int gr = grid(warps);
#define TTV_MV_ROWS(G)                                                                                  \
    case G:                                                                                             \
        if (f32) TTV_LAUNCH("matvec", stream, k_mv_rows<G, true><<<gr, kMvThreads, 0, stream>>>(a));    \
        else TTV_LAUNCH("matvec", stream, k_mv_rows<G, false><<<gr, kMvThreads, 0, stream>>>(a));       \
        break;
        switch (p.g) {
            TTV_MV_ROWS(1)
            TTV_MV_ROWS(2)
            TTV_MV_ROWS(4)
            TTV_MV_ROWS(8)
            TTV_MV_ROWS(16)
            default: TTV_MV_ROWS(32)
        }
#undef TTV_MV_ROWS
    } else {
        const int64_t warps = ((n1 + 32 * kMvRowsPerLane - 1) / (32 * kMvRowsPerLane)) * p.nchunks;
        const int gr = grid(warps);
        if (f32) TTV_LAUNCH("matvec", stream, k_mv_cols<true><<<gr, kMvThreads, 0, stream>>>(a));
        else TTV_LAUNCH("matvec", stream, k_mv_cols<false><<<gr, kMvThreads, 0, stream>>>(a));
    }
    if (p.nchunks > 1) {
        const int gr = (int)std::max<int64_t>(1, std::min<int64_t>((n1 + 255) / 256, (int64_t)num_sms() * 8));
        TTV_LAUNCH("matvec_reduce", stream,
                   k_mv_reduce<<<gr, 256, 0, stream>>>(static_cast<const double*>(ws), n1, p.nchunks, y));
    }
}

}  // namespace ttv
