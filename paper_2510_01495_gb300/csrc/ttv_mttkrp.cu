// ttv_mttkrp.cu -- MTTKRP on a prepared tensor.
//
// The paper names the matricized tensor times Khatri-Rao product as the
// kernel built on the sparse TTV (Sec. 3.3) and as future work (Sec. 5).
// Along mode n with factor matrices A_m (shape[m] x R, row-major):
//
//     M(i, r) = sum over nonzeros k with subs[k, n] == i of
//               vals[k] * prod_{m != n, increasing} A_m(subs[k, m], r)
//
// i.e. column r is the all-but-one TTV with the vectors A_m(:, r).  A tensor
// prepared for the modes m != n (ttv_prepare) has its nonzeros sorted by
// subs[k, n], a head bitmap marking where each row i starts, and the row's i
// in row_keys.  The nonzeros are cut into chunks of 128.  A group of lanes
// per chunk walks its nonzeros in order (lanes own rank components; a
// nonzero per lane is loaded at a time and broadcast with shuffles), writes
// every row that starts and ends inside the chunk, and leaves the sums of
// the chunk's first (open on the left) and last (open on the right) pieces
// in a side buffer.  A fix-up pass adds, for every row that crosses chunk
// ends, its pieces in chunk order, taking whole aligned runs of 64 and 4096
// chunks from precomputed sums.  Every sum is thus formed in an order fixed
// by the layout: results are bit-identical from run to run.
#include <algorithm>

#include "ttv_internal.cuh"

namespace ttv {

constexpr int kMtChunk = 128;           // nonzeros per chunk (4 bitmap words)
constexpr int kMtThreads = 256;

struct MtArgs {
    const double* vals;                 // binary64 values in key order (or float)
    int32_t val_f32;
    int32_t n_v;
    const int32_t* sub[kMaxD];          // contracted subscripts, increasing mode order
    const double* fac[kMaxD];           // factor of the j-th contracted mode, shape x R row-major
    const uint32_t* bits;               // head bitmap
    const uint64_t* row_keys;           // i of every row
    const uint32_t* chunk_base;         // heads before each chunk
    const int32_t* next_head;           // first chunk after c holding a head (nchunks when none)
    int64_t n;
    int64_t nchunks;
    int32_t R;
    double* out;                        // rows x R
    double* lead;                       // nchunks x R: sum before the chunk's first head (all of it when none)
    double* trail;                      // nchunks x R: sum from the chunk's last head
    int64_t* trail_row;                 // nchunks: row index of that last head, -1 when the chunk has none
    double* block_sum;                  // nblocks x R: sum of the leads of 64 consecutive chunks
    double* super_sum;                  // nsupers x R: sum of 64 consecutive block sums
    int64_t nblocks, nsupers;
};

constexpr int kMtBlock = 64;            // chunks per block, blocks per super-block

// One group of kG lanes per chunk, 32 / kG chunks per warp (so that ranks of
// 8 or 16 still keep every lane busy); lane j of a group owns the rank
// components j, j + kG, ... (kRPL of them).  Compiled per number of
// contracted modes kNV, so that the factor loads of a nonzero all issue
// before its products.  Each term is vals[k] times the factor entries in
// increasing mode order, added to the running row sum.
template <int kG, int kRPL, int kNV>
__global__ void __launch_bounds__(kMtThreads) k_mttkrp_chunks(MtArgs a) {
    constexpr int kGroups = 32 / kG;
    const int lane = threadIdx.x & 31;
    const int gl = lane % kG, grp = lane / kG;
    const int64_t nwarps = ((int64_t)gridDim.x * kMtThreads) >> 5;
    const int64_t nwc = (a.nchunks + kGroups - 1) / kGroups;
    for (int64_t wc = ((int64_t)blockIdx.x * kMtThreads + threadIdx.x) >> 5; wc < nwc; wc += nwarps) {
        const int64_t c = wc * kGroups + grp;
        const bool live = c < a.nchunks;
        const int64_t k0 = c * kMtChunk;
        const int64_t kend = live ? min(a.n, k0 + kMtChunk) : k0;
        uint32_t h = live ? a.chunk_base[c] : 0u;
        double acc[kRPL];
#pragma unroll
        for (int i = 0; i < kRPL; ++i) acc[i] = 0.0;
        bool seen = false;
        for (int g = 0; g < kMtChunk; g += kG) {              // same trip count in every group
            const int64_t kg = k0 + g;
            const int64_t k = kg + gl;
            const bool ok = k < kend;
            const double val = ok ? (a.val_f32 ? (double)reinterpret_cast<const float*>(a.vals)[k] : a.vals[k]) : 0.0;
            int32_t sub[kNV];
#pragma unroll
            for (int j = 0; j < kNV; ++j) sub[j] = ok ? a.sub[j][k] : 0;
            const int cnt = (int)max((int64_t)0, min((int64_t)kG, kend - kg));
            const uint32_t word = cnt > 0 ? (a.bits[kg >> 5] >> (kg & 31)) : 0u;
            for (int q = 0; q < kG; ++q) {
                const double v = __shfl_sync(0xffffffffu, val, q, kG);
                int32_t s[kNV];
#pragma unroll
                for (int j = 0; j < kNV; ++j) s[j] = __shfl_sync(0xffffffffu, sub[j], q, kG);
                if (q >= cnt) continue;
                if ((word >> q) & 1u) {
                    // a row starts: the one before it is complete (or is this chunk's lead)
                    if (seen) {
                        const int64_t row = (int64_t)a.row_keys[h - 1];
#pragma unroll
                        for (int i = 0; i < kRPL; ++i) {
                            const int r = gl + kG * i;
                            if (r < a.R) a.out[row * a.R + r] = acc[i];
                        }
                    } else {
#pragma unroll
                        for (int i = 0; i < kRPL; ++i) {
                            const int r = gl + kG * i;
                            if (r < a.R) a.lead[c * a.R + r] = acc[i];
                        }
                    }
                    seen = true;
                    ++h;
#pragma unroll
                    for (int i = 0; i < kRPL; ++i) acc[i] = 0.0;
                }
#pragma unroll
                for (int i = 0; i < kRPL; ++i) {
                    const int r = gl + kG * i;
                    if (r < a.R) {
                        double f[kNV];
#pragma unroll
                        for (int j = 0; j < kNV; ++j) f[j] = __ldg(a.fac[j] + (int64_t)s[j] * a.R + r);
                        double t = v;
#pragma unroll
                        for (int j = 0; j < kNV; ++j) t = t * f[j];
                        acc[i] = acc[i] + t;
                    }
                }
            }
        }
        if (live) {
            double* dst = seen ? a.trail : a.lead;
#pragma unroll
            for (int i = 0; i < kRPL; ++i) {
                const int r = gl + kG * i;
                if (r < a.R) dst[c * a.R + r] = acc[i];
            }
            if (gl == 0) a.trail_row[c] = seen ? (int64_t)(h - 1) : -1;
        }
    }
}

typedef void (*MtKernel)(MtArgs);

template <int kG, int kRPL>
static MtKernel mt_pick(int n_v) {
    switch (n_v) {
        case 1: return k_mttkrp_chunks<kG, kRPL, 1>;
        case 2: return k_mttkrp_chunks<kG, kRPL, 2>;
        case 3: return k_mttkrp_chunks<kG, kRPL, 3>;
        case 4: return k_mttkrp_chunks<kG, kRPL, 4>;
        case 5: return k_mttkrp_chunks<kG, kRPL, 5>;
        case 6: return k_mttkrp_chunks<kG, kRPL, 6>;
        default: return k_mttkrp_chunks<kG, kRPL, 7>;
    }
}

// Sums of the leads of aligned runs of 64 chunks (src = lead) or of 64
// block sums (src = block_sum), in index order; used only where every chunk
// covered lies inside one row, where a chunk's lead is its whole sum.
template <int kRPL>
__global__ void __launch_bounds__(kMtThreads) k_mttkrp_blocksum(const double* __restrict__ src, int64_t nsrc,
                                                                double* __restrict__ dst, int64_t ndst, int32_t R) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * kMtThreads) >> 5;
    for (int64_t b = ((int64_t)blockIdx.x * kMtThreads + threadIdx.x) >> 5; b < ndst; b += nwarps) {
        double acc[kRPL];
#pragma unroll
        for (int i = 0; i < kRPL; ++i) acc[i] = 0.0;
        const int64_t lo = b * kMtBlock, hi = min(nsrc, lo + kMtBlock);
        for (int64_t c = lo; c < hi; ++c)
#pragma unroll
            for (int i = 0; i < kRPL; ++i) {
                const int r = lane + 32 * i;
                if (r < R) acc[i] = acc[i] + src[c * R + r];
            }
#pragma unroll
        for (int i = 0; i < kRPL; ++i) {
            const int r = lane + 32 * i;
            if (r < R) dst[b * R + r] = acc[i];
        }
    }
}

// Rows that cross chunk ends: the last piece of chunk c, then every chunk
// up to the next one holding a head (whole aligned super-blocks and blocks
// taken from their sums, the rest chunk by chunk), then that chunk's lead --
// left to right, in a decomposition fixed by c and the head positions.
template <int kRPL>
__global__ void __launch_bounds__(kMtThreads) k_mttkrp_fixup(MtArgs a) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * kMtThreads) >> 5;
    constexpr int64_t kSuper = (int64_t)kMtBlock * kMtBlock;
    for (int64_t c = ((int64_t)blockIdx.x * kMtThreads + threadIdx.x) >> 5; c < a.nchunks; c += nwarps) {
        const int64_t row_idx = a.trail_row[c];
        if (row_idx < 0) continue;
        double acc[kRPL];
#pragma unroll
        for (int i = 0; i < kRPL; ++i) {
            const int r = lane + 32 * i;
            acc[i] = r < a.R ? a.trail[c * a.R + r] : 0.0;
        }
        const int64_t c_end = a.next_head[c];
        int64_t c2 = c + 1;
        while (c2 < c_end) {
            const double* src;
            if (c2 % kSuper == 0 && c2 + kSuper <= c_end) {
                src = a.super_sum + (c2 / kSuper) * a.R;
                c2 += kSuper;
            } else if (c2 % kMtBlock == 0 && c2 + kMtBlock <= c_end) {
                src = a.block_sum + (c2 / kMtBlock) * a.R;
                c2 += kMtBlock;
            } else {
                src = a.lead + c2 * a.R;
                c2 += 1;
            }
#pragma unroll
            for (int i = 0; i < kRPL; ++i) {
                const int r = lane + 32 * i;
                if (r < a.R) acc[i] = acc[i] + src[r];
            }
        }
        if (c_end < a.nchunks)   // the part of the next row-starting chunk before its first head
#pragma unroll
            for (int i = 0; i < kRPL; ++i) {
                const int r = lane + 32 * i;
                if (r < a.R) acc[i] = acc[i] + a.lead[c_end * a.R + r];
            }
        const int64_t row = (int64_t)a.row_keys[row_idx];
#pragma unroll
        for (int i = 0; i < kRPL; ++i) {
            const int r = lane + 32 * i;
            if (r < a.R) a.out[row * a.R + r] = acc[i];
        }
    }
}

// heads in every chunk of 256 (8 bitmap words)
__global__ void __launch_bounds__(256) k_mttkrp_chunk_counts(const uint32_t* __restrict__ bits, int64_t n,
                                                             uint32_t* __restrict__ counts, int64_t nchunks) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t nwords = (n + 31) / 32;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nchunks; c += stride) {
        uint32_t s = 0;
        for (int w = 0; w < kMtChunk / 32; ++w) {
            const int64_t wi = c * (kMtChunk / 32) + w;
            if (wi < nwords) s += __popc(bits[wi]);
        }
        counts[c] = s;
    }
}

int64_t mttkrp_nchunks(int64_t n) { return (std::max<int64_t>(n, 0) + kMtChunk - 1) / kMtChunk; }

size_t mttkrp_workspace_bytes(int64_t n, int32_t R) {
    const int64_t nc = std::max<int64_t>(mttkrp_nchunks(n), 1);
    const int64_t nb = (nc + kMtBlock - 1) / kMtBlock, ns = (nb + kMtBlock - 1) / kMtBlock;
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    return al((size_t)nc * R * 8) * 2 + al((size_t)nc * 8) + al((size_t)nb * R * 8) + al((size_t)ns * R * 8);
}

void launch_mttkrp_chunk_counts(const uint32_t* bits, int64_t n, uint32_t* counts, cudaStream_t stream) {
    const int64_t nc = mttkrp_nchunks(n);
    if (nc <= 0) return;
    const int g = (int)std::max<int64_t>(1, std::min<int64_t>((nc + 255) / 256, (int64_t)num_sms() * 8));
    TTV_LAUNCH("mttkrp_counts", stream, k_mttkrp_chunk_counts<<<g, 256, 0, stream>>>(bits, n, counts, nc));
}

// factors: one device pointer per contracted mode in increasing mode order;
// out: rows x R (zeroed here first); ws: mttkrp_workspace_bytes(n, R).
void launch_mttkrp(const void* vals, int val_f32, int n_v, const int32_t* const* subs, const double* const* factors,
                   const uint32_t* bits, const uint64_t* row_keys, const uint32_t* chunk_base,
                   const int32_t* next_head, int64_t n, int32_t R, int64_t rows, double* out, void* ws,
                   cudaStream_t stream) {
    cudaMemsetAsync(out, 0, (size_t)std::max<int64_t>(rows, 1) * R * sizeof(double), stream);
    if (n <= 0) return;
    MtArgs a{};
    a.vals = static_cast<const double*>(vals);
    a.val_f32 = val_f32;
    a.n_v = n_v;
    for (int j = 0; j < n_v; ++j) {
        a.sub[j] = subs[j];
        a.fac[j] = factors[j];
    }
    a.bits = bits;
    a.row_keys = row_keys;
    a.chunk_base = chunk_base;
    a.next_head = next_head;
    a.n = n;
    a.nchunks = mttkrp_nchunks(n);
    a.R = R;
    a.out = out;
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    char* w = static_cast<char*>(ws);
    a.lead = reinterpret_cast<double*>(w);
    a.trail = reinterpret_cast<double*>(w + al((size_t)a.nchunks * R * 8));
    a.trail_row = reinterpret_cast<int64_t*>(w + 2 * al((size_t)a.nchunks * R * 8));
    a.nblocks = (a.nchunks + kMtBlock - 1) / kMtBlock;
    a.nsupers = (a.nblocks + kMtBlock - 1) / kMtBlock;
    a.block_sum = reinterpret_cast<double*>(w + 2 * al((size_t)a.nchunks * R * 8) + al((size_t)a.nchunks * 8));
    a.super_sum = a.block_sum + al((size_t)a.nblocks * R * 8) / 8;
    auto grid = [](int64_t warps) {
        return (int)std::max<int64_t>(1, std::min<int64_t>((warps * 32 + kMtThreads - 1) / kMtThreads,
                                                           (int64_t)num_sms() * 16));
    };
    const int g = grid(a.nchunks);
    auto run = [&](MtKernel chunks, int groups, auto blocks, auto fixup) {
        TTV_LAUNCH("mttkrp_chunks", stream,
                   chunks<<<grid((a.nchunks + groups - 1) / groups), kMtThreads, 0, stream>>>(a));
        TTV_LAUNCH("mttkrp_blocks", stream,
                   blocks<<<grid(a.nblocks), kMtThreads, 0, stream>>>(a.lead, a.nchunks, a.block_sum, a.nblocks, R));
        TTV_LAUNCH("mttkrp_blocks", stream,
                   blocks<<<grid(a.nsupers), kMtThreads, 0, stream>>>(a.block_sum, a.nblocks, a.super_sum, a.nsupers,
                                                                      R));
        TTV_LAUNCH("mttkrp_fixup", stream, fixup<<<g, kMtThreads, 0, stream>>>(a));
    };
    if (R <= 8) run(mt_pick<8, 1>(n_v), 4, k_mttkrp_blocksum<1>, k_mttkrp_fixup<1>);
    else if (R <= 16) run(mt_pick<16, 1>(n_v), 2, k_mttkrp_blocksum<1>, k_mttkrp_fixup<1>);
    else if (R <= 32) run(mt_pick<32, 1>(n_v), 1, k_mttkrp_blocksum<1>, k_mttkrp_fixup<1>);
    else if (R <= 64) run(mt_pick<32, 2>(n_v), 1, k_mttkrp_blocksum<2>, k_mttkrp_fixup<2>);
    else run(mt_pick<32, 4>(n_v), 1, k_mttkrp_blocksum<4>, k_mttkrp_fixup<4>);
}

}  // namespace ttv
