// ttv_bucket.cu -- the bucket path for large sparse results: the (key, term)
// pairs are partitioned into ~64K key-range buckets in two coalesced passes,
// then each bucket is sorted and reduced on chip and emitted in key order.
//
// Traffic per nonzero: the input once (8d + w bytes), the 16-byte pair
// written and read twice, and the result rows -- no multi-pass global sort.
// (A single pass straight into tens of thousands of buckets turns every pair
// into its own scattered 16-byte store; on GB300 that alone costs more than
// the second pass.)
//
//  1. k_bkt_sample   keys of S nonzeros spread evenly over the input
//  2. radix sort of the samples (the onesweep sort of ttv_sort.cu)
//  3. k_bkt_bounds   fine bucket boundaries F from the sample quantiles (a key
//                    that fills more than one quantile gets a bucket of its
//                    own); level-1 buckets are runs of 256 fine buckets; both
//                    levels get Eytzinger-ordered search trees and regions
//                    sized from the sample with a wide margin
//  4. k_bkt_part1    streams subs/vals, forms (key, term), finds the level-1
//                    bucket, sorts a tile of 4096 pairs by bucket in shared
//                    memory and writes each bucket's run with one reservation
//  5. k_bkt_part2    the same over level-1 regions into the fine buckets
//  6. k_bkt_process  one CTA per fine bucket, in key order: a stable LSD
//                    radix sort of the bucket in registers/shared memory, a
//                    fixed-order segmented reduction, and the unique keys
//                    written at the bucket's output offset, found by a
//                    warp-wide decoupled look-back.  A bucket larger than the
//                    on-chip capacity is split into key sub-ranges by
//                    histograms; a single key is summed without sorting.
// A region overflow (the sample badly misjudged a bucket) sets an error bit
// and the host re-runs the call on the sort path.
#include <algorithm>
#include <climits>

#include "ttv_internal.cuh"

namespace ttv {

constexpr int kBktFineQuantiles = 16384;      // fine buckets (before heavy-key extras)
constexpr int kBktMaxFine = 65535;            // fine boundaries
constexpr int kBktFan = 256;                  // fine buckets per level-1 bucket
constexpr int kBktMaxL1 = (kBktMaxFine + 1) / kBktFan;   // 256 level-1 buckets
constexpr int kBktThreads = 512;              // process kernel
constexpr int kBktWarps = kBktThreads / 32;
constexpr int kBktItems = 16;                 // pairs per thread in registers
constexpr int kBktCap = kBktThreads * kBktItems;   // 8192 pairs on chip
constexpr int kBktDigitBits = 11;
constexpr int kBktRadix = 1 << kBktDigitBits;
constexpr int kPartThreads = 512;             // partition kernels
constexpr int kPartPairs = 4;                 // input pairs (2 nonzeros) per thread per tile
constexpr int kPartTile = kPartThreads * kPartPairs * 2;   // 4096 nonzeros per tile
constexpr int kEytLevels = 8;                 // 255-node search trees
constexpr unsigned long long kLbAgg = 1ull << 62;
constexpr unsigned long long kLbInc = 2ull << 62;
constexpr unsigned long long kLbMask = (1ull << 62) - 1;

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint32_t lane_lt_mask() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Rank of key among the 255 entries of an Eytzinger-ordered complete search
// tree (node i has children 2i and 2i+1, padding entries are UINT64_MAX):
// the number of entries < key.
__device__ __forceinline__ uint32_t eyt_rank(const uint64_t* t, uint64_t key) {
    uint32_t i = 1;
#pragma unroll
    for (int l = 0; l < kEytLevels; ++l) i = 2 * i + (t[i] < key ? 1u : 0u);
    return i - (1u << kEytLevels);
}

// ---- 1. samples --------------------------------------------------------------
__global__ void k_bkt_sample(StreamDesc p, int S, uint64_t* __restrict__ out, double* __restrict__ dummy) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= S) return;
    const int64_t k = (int64_t)(((unsigned __int128)i * (unsigned __int128)p.nnz) / (unsigned)S);
    uint64_t key = 0;
    for (int m = 0; m < p.d; ++m) {
        const int64_t s = p.subs[k * p.snz + m * p.smode];
        if ((uint64_t)s >= (uint64_t)p.shape[m]) { key = 0; break; }
        if (!((p.smask >> m) & 1u)) key += (uint64_t)s * p.kstride[m];
    }
    out[i] = key;
    dummy[i] = 0.0;
}

// ---- 3. boundaries, search trees and regions (one CTA of 1024 threads) --------
// Quantile q_i = sample[i * S / B], i = 1..B-1.  Fine boundaries F are the
// distinct quantiles; a value that is the quantile at two or more consecutive
// positions is "heavy" and also gets the boundary value - 1 in front of it,
// so that it owns the fine bucket (value - 1, value].  Fine bucket j holds the
// keys in (F[j-1], F[j]]; level-1 bucket b holds fine buckets 256b..256b+255.
struct BktBoundsOut {
    uint64_t* fine;                  // [kBktMaxFine]
    uint32_t* nfine;
    uint64_t* l1_eyt;                // [256] tree over F[256b + 255]
    uint64_t* fine_eyt;              // [kBktMaxL1][256] tree over F[256b .. 256b + 254]
    unsigned long long* region1;     // [kBktMaxL1]
    unsigned long long* cap1;
    unsigned long long* region;      // [kBktMaxFine + 1]
    unsigned long long* cap;
    int64_t total1, total2;
};

__device__ uint32_t sample_lower(const uint64_t* sorted, int S, uint64_t v) {   // first index with sorted[i] > v
    int lo = 0, hi = S;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (sorted[mid] <= v) lo = mid + 1; else hi = mid;
    }
    return (uint32_t)lo;
}

__global__ void __launch_bounds__(1024) k_bkt_bounds(const uint64_t* __restrict__ sorted, int S, int B, int64_t nnz,
                                                     BktBoundsOut o, Status* st) {
    __shared__ uint32_t wsum[32];
    __shared__ unsigned long long wsum2[32];
    __shared__ uint32_t s_nf;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int per = (B + 1023) / 1024;
    // pass 1: how many boundaries each quantile contributes (0, 1 or 2)
    uint32_t cnt = 0;
    for (int j = 0; j < per; ++j) {
        const int i = 1 + tid * per + j;
        if (i >= B) break;
        const uint64_t q = sorted[(int64_t)i * S / B];
        const uint64_t qp = i > 1 ? sorted[(int64_t)(i - 1) * S / B] : 0ull;
        const uint64_t qn = i + 1 < B ? sorted[(int64_t)(i + 1) * S / B] : ~0ull;
        if (i > 1 && q == qp) continue;
        const bool heavy = (i + 1 < B) && qn == q;
        cnt += 1;
        if (heavy && q > 0 && (i == 1 || qp < q - 1)) cnt += 1;
    }
    uint32_t inc = cnt;
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += y;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    uint32_t before = 0, total = 0;
    for (int w = 0; w < 32; ++w) {
        if (w < warp) before += wsum[w];
        total += wsum[w];
    }
    uint32_t pos = before + inc - cnt;
    const bool fits = total <= (uint32_t)kBktMaxFine;
    for (int j = 0; j < per && fits; ++j) {
        const int i = 1 + tid * per + j;
        if (i >= B) break;
        const uint64_t q = sorted[(int64_t)i * S / B];
        const uint64_t qp = i > 1 ? sorted[(int64_t)(i - 1) * S / B] : 0ull;
        const uint64_t qn = i + 1 < B ? sorted[(int64_t)(i + 1) * S / B] : ~0ull;
        if (i > 1 && q == qp) continue;
        const bool heavy = (i + 1 < B) && qn == q;
        if (heavy && q > 0 && (i == 1 || qp < q - 1)) o.fine[pos++] = q - 1;
        o.fine[pos++] = q;
    }
    if (tid == 0) {
        s_nf = fits ? total : 0u;
        *o.nfine = s_nf;
        if (!fits) set_error(st, kErrRetry);
    }
    __syncthreads();
    const uint32_t nf = s_nf;
    const uint32_t nl1 = (nf >> 8) + 1;                   // level-1 buckets
    // search trees: level 1 over F[256b + 255], b < nl1 - 1; fine slices of 255
    for (uint32_t node = 1 + tid; node < 256; node += 1024) {
        // in-order rank of Eytzinger node `node` in a 255-node complete tree
        const int depth = 31 - __clz(node);
        const uint32_t r = ((2u * (node - (1u << depth)) + 1u) << (kEytLevels - 1 - depth)) - 1u;
        o.l1_eyt[node] = (r < nl1 - 1) ? o.fine[256 * r + 255] : ~0ull;
    }
    for (uint32_t e = tid; e < nl1 * 256; e += 1024) {
        const uint32_t b = e >> 8, node = e & 255;
        if (node == 0) continue;
        const int depth = 31 - __clz(node);
        const uint32_t r = ((2u * (node - (1u << depth)) + 1u) << (kEytLevels - 1 - depth)) - 1u;
        const uint32_t fi = 256 * b + r;
        o.fine_eyt[(size_t)b * 256 + node] = (r < 255 && fi < nf) ? o.fine[fi] : ~0ull;
    }
}

// Estimated pairs of every fine bucket (2 x its sample share plus a margin),
// one thread per bucket.
__global__ void k_bkt_caps(const uint64_t* __restrict__ sorted, int S, int64_t nnz, const uint64_t* __restrict__ fine,
                           const uint32_t* __restrict__ nfine, unsigned long long* __restrict__ cap) {
    const uint32_t nf = *nfine;
    const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b > nf) return;
    const uint32_t a = b == 0 ? 0u : sample_lower(sorted, S, fine[b - 1]);
    const uint32_t e = b == nf ? (uint32_t)S : sample_lower(sorted, S, fine[b]);
    cap[b] = (unsigned long long)(2.0 * (double)(e - a) * (double)nnz / (double)S) + 256ull;
}

// Regions from the capacities: exclusive scan over fine buckets, and the
// level-1 capacities as sums over their 256 fine buckets (one CTA).
__global__ void __launch_bounds__(1024) k_bkt_regions(const uint32_t* __restrict__ nfine, int64_t total1,
                                                      int64_t total2, unsigned long long* __restrict__ cap,
                                                      unsigned long long* __restrict__ region,
                                                      unsigned long long* __restrict__ cap1,
                                                      unsigned long long* __restrict__ region1) {
    __shared__ unsigned long long wsum[32];
    __shared__ unsigned long long l1[kBktMaxL1];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t nbk = *nfine + 1;
    const uint32_t nl1 = (nbk - 1) / 256 + 1;
    const int per = (int)((nbk + 1023) / 1024);
    unsigned long long sum = 0;
    for (int j = 0; j < per; ++j) {
        const uint32_t b = (uint32_t)tid * per + j;
        if (b < nbk) sum += cap[b];
    }
    unsigned long long inc = sum;
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += y;
    }
    if (lane == 31) wsum[warp] = inc;
    for (int i = tid; i < kBktMaxL1; i += 1024) l1[i] = 0;
    __syncthreads();
    unsigned long long off = 0;
    for (int w = 0; w < warp; ++w) off += wsum[w];
    off += inc - sum;
    for (int j = 0; j < per; ++j) {
        const uint32_t b = (uint32_t)tid * per + j;
        if (b >= nbk) break;
        const unsigned long long c = cap[b];
        region[b] = off;
        cap[b] = off >= (unsigned long long)total2 ? 0ull : min(c, (unsigned long long)total2 - off);
        atomicAdd(&l1[b >> 8], c);
        off += c;
    }
    __syncthreads();
    if (tid == 0) {
        unsigned long long acc = 0;
        for (uint32_t b = 0; b < nl1; ++b) {
            const unsigned long long c = l1[b] + 4ull * kPartTile;
            region1[b] = acc;
            cap1[b] = acc >= (unsigned long long)total1 ? 0ull : min(c, (unsigned long long)total1 - acc);
            acc += c;
        }
    }
}

// ---- 4./5. partition passes ---------------------------------------------------------
template <int D, bool kSoA>
__device__ __forceinline__ void bkt_load_pair(const StreamDesc& p, int64_t k, int64_t (&s0)[D], int64_t (&s1)[D],
                                              double& v0, double& v1) {
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
    if (p.val_f32) {
        const float2 w = __ldcs(reinterpret_cast<const float2*>(static_cast<const float*>(p.vals) + k));
        v0 = w.x;
        v1 = w.y;
    } else {
        const double2 w = __ldcs(reinterpret_cast<const double2*>(static_cast<const double*>(p.vals) + k));
        v0 = w.x;
        v1 = w.y;
    }
}

template <int D>
__device__ __forceinline__ bool bkt_key_term(const StreamDesc& p, const int64_t (&s)[D], double val, uint64_t& key,
                                             double& t) {
    bool good = true;
#pragma unroll
    for (int m = 0; m < D; ++m) good &= (uint64_t)s[m] < (uint64_t)p.shape[m];
    uint64_t kk = 0;
    double tt = val;
#pragma unroll
    for (int m = 0; m < D; ++m) {
        const int64_t sm = good ? s[m] : 0;
        if ((p.smask >> m) & 1u)
            tt = tt * (p.vec_f32 ? (double)__ldg(static_cast<const float*>(p.vec[m]) + sm)
                                 : __ldg(static_cast<const double*>(p.vec[m]) + sm));
        else kk += (uint64_t)sm * p.kstride[m];
    }
    key = kk;
    t = tt;
    return good;
}

// Shared state of a partition tile: the pairs sorted by local bucket.
struct PartSmem {
    ulonglong2 stage[kPartTile];
    uint16_t sbid[kPartTile];
    uint32_t hist[kBktFan];
    uint32_t tstart[kBktFan];
    unsigned long long gbase[kBktFan];
    uint64_t tree[256];
    uint32_t scan_tmp[kPartThreads / 32];
    uint32_t s_total;
    uint32_t s_tile;
    uint32_t s_b1;
};

// Rank of an item among equal local buckets of the tile (warp multi-split +
// one shared atomic per group), then the tile's runs written out coalesced.
// Items: (key, term, local bucket, valid) for 2 * kPartPairs per thread.
__device__ void part_tile_flush(PartSmem& sm, const uint64_t (&key)[2 * kPartPairs], const double (&t)[2 * kPartPairs],
                                const uint32_t (&lb)[2 * kPartPairs], const bool (&use)[2 * kPartPairs],
                                uint32_t bucket_base, unsigned long long* __restrict__ count,
                                const unsigned long long* __restrict__ region, const unsigned long long* __restrict__ cap,
                                ulonglong2* __restrict__ out, Status* st) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lt = lane_lt_mask();
    uint32_t rank[2 * kPartPairs];
#pragma unroll
    for (int i = 0; i < 2 * kPartPairs; ++i) {
        const uint32_t g = use[i] ? lb[i] : 0xFFFFu;
        const uint32_t mask = __match_any_sync(0xffffffffu, g);
        const int leader = __ffs(mask) - 1;
        uint32_t base = 0;
        if (lane == leader && g != 0xFFFFu) base = atomicAdd(&sm.hist[g], (uint32_t)__popc(mask));
        base = __shfl_sync(0xffffffffu, base, leader);
        rank[i] = base + __popc(mask & lt);
    }
    __syncthreads();
    if (tid < kBktFan) {
        // exclusive scan of the 256 bucket counts (8 warps of 32)
        const uint32_t c = sm.hist[tid];
        uint32_t inc = c;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, d);
            if (lane >= d) inc += y;
        }
        if (lane == 31) sm.scan_tmp[warp] = inc;
    }
    __syncthreads();
    if (tid < kBktFan) {
        const uint32_t c = sm.hist[tid];
        uint32_t before = 0;
        for (int w = 0; w < warp; ++w) before += sm.scan_tmp[w];
        uint32_t inc = c;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, d);
            if (lane >= d) inc += y;
        }
        sm.tstart[tid] = before + inc - c;
        if (tid == kBktFan - 1) sm.s_total = before + inc;
        unsigned long long gb = 0;
        if (c) {
            const unsigned long long at = atomicAdd(&count[bucket_base + tid], (unsigned long long)c);
            if (at + c > cap[bucket_base + tid]) set_error(st, kErrRetry);
            gb = region[bucket_base + tid] + at;
        }
        sm.gbase[tid] = gb;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 2 * kPartPairs; ++i) {
        if (!use[i]) continue;
        const uint32_t at = sm.tstart[lb[i]] + rank[i];
        sm.stage[at] = make_ulonglong2(key[i], (unsigned long long)__double_as_longlong(t[i]));
        sm.sbid[at] = (uint16_t)lb[i];
    }
    __syncthreads();
    const uint32_t total = sm.s_total;
    for (uint32_t i = tid; i < total; i += kPartThreads) {
        const uint32_t b = sm.sbid[i];
        const unsigned long long dest = sm.gbase[b] + (i - sm.tstart[b]);
        if (dest < region[bucket_base + b] + cap[bucket_base + b]) __stcg(out + dest, sm.stage[i]);
    }
    __syncthreads();
    for (int i = tid; i < kBktFan; i += kPartThreads) sm.hist[i] = 0;
    __syncthreads();
}

template <int D, bool kSoA>
__global__ void __launch_bounds__(kPartThreads, 2) k_bkt_part1(StreamDesc p, const uint64_t* __restrict__ l1_eyt,
                                                            const unsigned long long* __restrict__ region1,
                                                            const unsigned long long* __restrict__ cap1,
                                                            unsigned long long* __restrict__ count1,
                                                            ulonglong2* __restrict__ pairs1) {
    extern __shared__ __align__(16) unsigned char psm_raw[];
    PartSmem& sm = *reinterpret_cast<PartSmem*>(psm_raw);
    const int tid = threadIdx.x;
    for (int i = tid; i < 256; i += kPartThreads) sm.tree[i] = l1_eyt[i];
    for (int i = tid; i < kBktFan; i += kPartThreads) sm.hist[i] = 0;
    __syncthreads();
    const int64_t ntiles = (p.nnz + kPartTile - 1) / kPartTile;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t k0 = tile * kPartTile;
        uint64_t key[2 * kPartPairs];
        double t[2 * kPartPairs];
        uint32_t lb[2 * kPartPairs];
        bool use[2 * kPartPairs];
#pragma unroll
        for (int j = 0; j < kPartPairs; ++j) {
            const int64_t k = k0 + 2 * ((int64_t)j * kPartThreads + tid);
            use[2 * j] = use[2 * j + 1] = false;
            if (k + 1 < p.nnz) {
                int64_t s0[D], s1[D];
                double v0, v1;
                bkt_load_pair<D, kSoA>(p, k, s0, s1, v0, v1);
                use[2 * j] = bkt_key_term<D>(p, s0, v0, key[2 * j], t[2 * j]);
                use[2 * j + 1] = bkt_key_term<D>(p, s1, v1, key[2 * j + 1], t[2 * j + 1]);
                if (!use[2 * j] || !use[2 * j + 1]) set_error(p.status, kErrSubscript);
            } else if (k < p.nnz) {             // odd last nonzero
                int64_t s0[D];
#pragma unroll
                for (int m = 0; m < D; ++m) s0[m] = p.subs[k * p.snz + m * p.smode];
                const double v0 = p.val_f32 ? (double)static_cast<const float*>(p.vals)[k]
                                            : static_cast<const double*>(p.vals)[k];
                use[2 * j] = bkt_key_term<D>(p, s0, v0, key[2 * j], t[2 * j]);
                if (!use[2 * j]) set_error(p.status, kErrSubscript);
            }
        }
#pragma unroll
        for (int i = 0; i < 2 * kPartPairs; ++i) lb[i] = use[i] ? eyt_rank(sm.tree, key[i]) : 0u;
        part_tile_flush(sm, key, t, lb, use, 0u, count1, region1, cap1, pairs1, p.status);
    }
}

// Tiles of the level-1 regions: tile_start[b] = tiles before level-1 bucket b.
__global__ void k_bkt_tiles(const uint32_t* __restrict__ nfine, const unsigned long long* __restrict__ count1,
                            const unsigned long long* __restrict__ cap1, uint32_t* __restrict__ tile_start) {
    if (threadIdx.x != 0) return;
    const uint32_t nl1 = (*nfine >> 8) + 1;
    uint32_t acc = 0;
    for (uint32_t b = 0; b < nl1; ++b) {
        tile_start[b] = acc;
        const unsigned long long n = min(count1[b], cap1[b]);
        acc += (uint32_t)((n + kPartTile - 1) / kPartTile);
    }
    tile_start[nl1] = acc;
}

__global__ void __launch_bounds__(kPartThreads, 2) k_bkt_part2(const uint32_t* __restrict__ nfine,
                                                            const uint64_t* __restrict__ fine_eyt,
                                                            const uint32_t* __restrict__ tile_start,
                                                            const unsigned long long* __restrict__ region1,
                                                            const unsigned long long* __restrict__ cap1,
                                                            const unsigned long long* __restrict__ count1,
                                                            const ulonglong2* __restrict__ pairs1,
                                                            const unsigned long long* __restrict__ region,
                                                            const unsigned long long* __restrict__ cap,
                                                            unsigned long long* __restrict__ count,
                                                            ulonglong2* __restrict__ pairs, uint32_t* ticket,
                                                            Status* st) {
    extern __shared__ __align__(16) unsigned char psm_raw[];
    PartSmem& sm = *reinterpret_cast<PartSmem*>(psm_raw);
    const int tid = threadIdx.x;
    const uint32_t nl1 = (*nfine >> 8) + 1;
    const uint32_t ntiles = tile_start[nl1];
    for (int i = tid; i < kBktFan; i += kPartThreads) sm.hist[i] = 0;
    for (;;) {
        if (tid == 0) {
            const uint32_t g = atomicAdd(ticket, 1u);
            uint32_t lo = 0, hi = nl1;                  // last b with tile_start[b] <= g
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if (tile_start[mid] <= g) lo = mid; else hi = mid;
            }
            sm.s_tile = g;
            sm.s_b1 = lo;
        }
        __syncthreads();
        const uint32_t g = sm.s_tile, b1 = sm.s_b1;
        if (g >= ntiles) break;
        for (int i = tid; i < 256; i += kPartThreads) sm.tree[i] = fine_eyt[(size_t)b1 * 256 + i];
        __syncthreads();
        const unsigned long long n1 = min(count1[b1], cap1[b1]);
        const unsigned long long off = (unsigned long long)(g - tile_start[b1]) * kPartTile;
        uint64_t key[2 * kPartPairs];
        double t[2 * kPartPairs];
        uint32_t lb[2 * kPartPairs];
        bool use[2 * kPartPairs];
#pragma unroll
        for (int i = 0; i < 2 * kPartPairs; ++i) {
            const unsigned long long idx = off + (unsigned long long)i * kPartThreads + tid;
            use[i] = idx < n1;
            if (use[i]) {
                const ulonglong2 w = __ldcs(pairs1 + region1[b1] + idx);
                key[i] = w.x;
                t[i] = __longlong_as_double((long long)w.y);
                lb[i] = eyt_rank(sm.tree, key[i]);
            } else {
                key[i] = 0;
                t[i] = 0.0;
                lb[i] = 0;
            }
        }
        part_tile_flush(sm, key, t, lb, use, b1 * kBktFan, count, region, cap, pairs, st);
    }
}

// ---- 5. per-bucket sort, reduce and emit ---------------------------------------
// Shared arrays of pairs are padded by one slot every 16 so that a thread
// reading 16 consecutive pairs and a warp reading 32 consecutive ones both
// stay free of bank conflicts.
__device__ __forceinline__ uint32_t bpad(uint32_t i) { return i + (i >> 4); }
constexpr int kBktPadded = kBktCap + kBktCap / 16;

struct BktSmem {
    uint64_t skeys[kBktPadded];
    double svals[kBktPadded];
    uint16_t whist[kBktWarps][kBktRadix + 4];   // per-warp digit counts, then prefixes
    union {
        uint32_t dstart[kBktRadix];              // digit starts (sorting)
        uint32_t hist11[2048];                   // key sub-range histogram (splitting)
    };
    uint32_t scan_tmp[kBktThreads / 32];
    double lead[kBktThreads];                    // a thread's sum before its first head
    uint32_t has_head[kBktThreads];
    uint64_t red_min[kBktThreads / 32], red_max[kBktThreads / 32];
    uint64_t stack_lo[64], stack_hi[64];
    unsigned long long stack_n[64];
    int gstart[64], gend[64];
    unsigned long long gcnt[64];
    int stack_top;
    uint32_t s_ticket;
    unsigned long long s_excl;
    uint32_t s_flag;
};

__device__ __forceinline__ uint32_t bscan_excl(uint32_t x, uint32_t* tmp, uint32_t& total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) tmp[warp] = inc;
    __syncthreads();
    uint32_t before = 0, all = 0;
#pragma unroll
    for (int w = 0; w < kBktThreads / 32; ++w) {
        const uint32_t t = tmp[w];
        if (w < warp) before += t;
        all += t;
    }
    total = all;
    __syncthreads();
    return before + inc - x;
}

__device__ __forceinline__ int bits_of_range(uint64_t span) {     // bits to index 0..span
    return span == 0 ? 0 : 64 - __clzll(span);
}

// Smallest and largest key among the valid pairs in registers (all threads).
__device__ __forceinline__ void bkt_minmax(BktSmem& sm, const uint64_t (&k)[kBktItems], const bool (&ok)[kBktItems],
                                           uint64_t& mn, uint64_t& mx) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t a = ~0ull, z = 0;
#pragma unroll
    for (int j = 0; j < kBktItems; ++j)
        if (ok[j]) { a = min(a, k[j]); z = max(z, k[j]); }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a = min(a, (uint64_t)__shfl_xor_sync(0xffffffffu, (unsigned long long)a, o));
        z = max(z, (uint64_t)__shfl_xor_sync(0xffffffffu, (unsigned long long)z, o));
    }
    if (lane == 0) { sm.red_min[warp] = a; sm.red_max[warp] = z; }
    __syncthreads();
    mn = ~0ull;
    mx = 0;
#pragma unroll
    for (int w = 0; w < kBktWarps; ++w) { mn = min(mn, sm.red_min[w]); mx = max(mx, sm.red_max[w]); }
    __syncthreads();
}

// Stable LSD radix sort of one part's pairs by key - lo over `bits` bits.
// On entry the pairs are in registers, blocked per warp (item j of lane l of
// warp w is sequence position w*512 + j*32 + l) with ok[] marking the real
// ones; on exit the shared arrays hold them in key order at bpad(0..nvalid).
__device__ void bkt_sort_part(BktSmem& sm, uint64_t (&k)[kBktItems], double (&v)[kBktItems],
                              bool (&ok)[kBktItems], uint32_t nvalid, uint64_t lo, int bits) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lt = lane_lt_mask();
    const int passes = bits <= 0 ? 1 : (bits + kBktDigitBits - 1) / kBktDigitBits;
    for (int pass = 0; pass < passes; ++pass) {
        const int shift = pass * kBktDigitBits;
        // warps and rows past the valid pairs carry nothing: skip them (uniform per warp)
        const uint32_t wbase = (uint32_t)warp * (kBktItems * 32);
        const int rows = nvalid <= wbase ? 0 : (int)min((uint32_t)kBktItems, (nvalid - wbase + 31) / 32);
        uint32_t* wz = reinterpret_cast<uint32_t*>(sm.whist[warp]);
        for (int i = lane; i < (kBktRadix + 4) / 2; i += 32) wz[i] = 0u;
        __syncwarp();
        uint32_t dig[kBktItems], rank[kBktItems];
#pragma unroll
        for (int j = 0; j < kBktItems; ++j) {
            dig[j] = ok[j] ? (uint32_t)(((k[j] - lo) >> shift) & (kBktRadix - 1)) : (uint32_t)kBktRadix;
            rank[j] = 0;
            if (j >= rows) continue;
            const uint32_t mask = __match_any_sync(0xffffffffu, dig[j]);
            const int leader = __ffs(mask) - 1;
            uint32_t b = 0;
            if (lane == leader) {
                b = sm.whist[warp][dig[j]];
                sm.whist[warp][dig[j]] = (uint16_t)(b + __popc(mask));
            }
            b = __shfl_sync(0xffffffffu, b, leader);
            rank[j] = b + __popc(mask & lt);
            __syncwarp();
        }
        __syncthreads();
        // thread t owns digits 4t..4t+3: prefix over warps, then digit starts
        uint32_t tot[4] = {0, 0, 0, 0};
        for (int w = 0; w < kBktWarps; ++w) {
            uint2* cell = reinterpret_cast<uint2*>(&sm.whist[w][4 * tid]);
            const uint2 c = *cell;
            const uint32_t c0 = c.x & 0xFFFFu, c1 = c.x >> 16, c2 = c.y & 0xFFFFu, c3 = c.y >> 16;
            *cell = make_uint2(tot[0] | (tot[1] << 16), tot[2] | (tot[3] << 16));
            tot[0] += c0; tot[1] += c1; tot[2] += c2; tot[3] += c3;
        }
        uint32_t all;
        const uint32_t ex = bscan_excl(tot[0] + tot[1] + tot[2] + tot[3], sm.scan_tmp, all);
        sm.dstart[4 * tid] = ex;
        sm.dstart[4 * tid + 1] = ex + tot[0];
        sm.dstart[4 * tid + 2] = ex + tot[0] + tot[1];
        sm.dstart[4 * tid + 3] = ex + tot[0] + tot[1] + tot[2];
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kBktItems; ++j) {
            if (dig[j] >= (uint32_t)kBktRadix) continue;
            const uint32_t pos = bpad(sm.dstart[dig[j]] + sm.whist[warp][dig[j]] + rank[j]);
            sm.skeys[pos] = k[j];
            sm.svals[pos] = v[j];
        }
        __syncthreads();
        if (pass + 1 < passes) {
#pragma unroll
            for (int j = 0; j < kBktItems; ++j) {
                const uint32_t pos = (uint32_t)(warp * (kBktItems * 32) + j * 32 + lane);
                ok[j] = pos < nvalid;
                if (j >= rows) { ok[j] = false; continue; }
                k[j] = ok[j] ? sm.skeys[bpad(pos)] : 0ull;
                v[j] = ok[j] ? sm.svals[bpad(pos)] : 0.0;
            }
            __syncthreads();
        }
    }
}

// Segmented reduction of the sorted pairs bpad(0..n): thread t takes the 16
// consecutive pairs 16t..16t+15 into registers; k[j] keeps the key, v[j]
// becomes the sum from pair j to the end of its run inside the thread, bit j
// of `heads` marks a run start.  Returns the number of unique keys; hb is the
// number of run starts before thread t.  Order of additions is fixed.
__device__ uint32_t bkt_reduce_regs(BktSmem& sm, uint32_t n, uint64_t (&k)[kBktItems], double (&v)[kBktItems],
                                    uint32_t& heads, uint32_t& hb) {
    const int tid = threadIdx.x;
    const uint32_t b0 = (uint32_t)tid * kBktItems;
    uint64_t prev = (b0 > 0 && b0 <= n && b0 - 1 < n) ? sm.skeys[bpad(b0 - 1)] : ~0ull;
    heads = 0;
#pragma unroll
    for (int j = 0; j < kBktItems; ++j) {
        const uint32_t q = b0 + j;
        if (q < n) {
            k[j] = sm.skeys[bpad(q)];
            v[j] = sm.svals[bpad(q)];
            if (q == 0 || k[j] != prev) heads |= 1u << j;
            prev = k[j];
        } else {
            k[j] = 0;
            v[j] = 0.0;
        }
    }
    // suffix sums inside the thread, each stopping at the next run start
#pragma unroll
    for (int j = kBktItems - 2; j >= 0; --j)
        if (!((heads >> (j + 1)) & 1u) && b0 + j + 1 < n) v[j] += v[j + 1];
    const uint32_t nh = __popc(heads);
    uint32_t U;
    hb = bscan_excl(nh, sm.scan_tmp, U);
    sm.lead[tid] = (heads & 1u) ? 0.0 : v[0];     // pairs before the first run start
    sm.has_head[tid] = (b0 < n) ? (nh > 0 ? 1u : 0u) : 1u;   // past the end stops the walk
    __syncthreads();
    return U;
}

// Writes the runs that start in this thread at out_base + (their index).
__device__ void bkt_emit_regs(BktSmem& sm, uint32_t n, const uint64_t (&k)[kBktItems], const double (&v)[kBktItems],
                              uint32_t heads, uint32_t hb, const StreamDesc& p, int64_t* out_subs, double* out_vals,
                              unsigned long long out_base, int64_t cap_rows, Status* st) {
    const int tid = threadIdx.x;
    if (heads == 0) return;
    const int last = 31 - __clz(heads);
    uint32_t u = hb;
#pragma unroll
    for (int j = 0; j < kBktItems; ++j) {
        if (!((heads >> j) & 1u)) continue;
        double sum = v[j];
        if (j == last && (uint32_t)tid * kBktItems + kBktItems < n) {
            // the run continues into the following threads: their leading sums
            for (int t2 = tid + 1; t2 < kBktThreads; ++t2) {
                if ((uint32_t)t2 * kBktItems >= n) break;
                sum += sm.lead[t2];
                if (sm.has_head[t2]) break;
            }
        }
        const unsigned long long row = out_base + u;
        if ((int64_t)row < cap_rows) {
            if (p.nr > 0) delinearise(p, k[j], out_subs + row * p.nr);
            out_vals[row] = sum;
        } else {
            set_error(st, kErrCapacity);
        }
        ++u;
    }
}

struct BktProcParams {
    StreamDesc p;
    const uint64_t* bounds;
    const uint32_t* nbounds;
    const unsigned long long* region;
    const unsigned long long* cap;
    const unsigned long long* count;
    unsigned long long* lookback;
    uint32_t* ticket;
    const ulonglong2* pairs;      // fine regions: (key, term bits)
    int64_t* out_subs;
    double* out_vals;
    int64_t cap_rows;
};

// Look-back over the buckets before this one: exclusive prefix of unique
// counts.  Called by all 32 lanes of warp 0: each round reads the 32 nearest
// predecessors at once (one L2 round trip), sums their published counts up
// to the nearest one that already carries its inclusive prefix, and stops
// there -- so a walk over the ~150 buckets in flight costs a few round trips.
__device__ unsigned long long bkt_lookback(BktProcParams& f, uint32_t b, unsigned long long U) {
    const int lane = threadIdx.x & 31;
    unsigned long long* my = f.lookback + b;
    if (b == 0) {
        if (lane == 0) st_relaxed_u64(my, kLbInc | U);
        return 0;
    }
    if (lane == 0) st_relaxed_u64(my, kLbAgg | U);
    const volatile uint32_t* err = &f.p.status->err;
    unsigned long long excl = 0;
    int64_t j0 = (int64_t)b - 1;
    for (int round = 0; round < (1 << 20); ++round) {
        const int64_t j = j0 - lane;
        unsigned long long val = kLbInc;                  // before bucket 0: inclusive zero
        if (j >= 0) {
            // bounded: ~1 s at most; once any wait has given up, later ones do not wait
            for (uint32_t it = 0; it < (1u << 20); ++it) {
                val = ld_relaxed_u64(f.lookback + j);
                if (val & (kLbAgg | kLbInc)) break;
                if ((it & 1023) == 1023 && (*err & kErrTimeout)) break;
                if (it > 32) __nanosleep(256);
            }
            if (!(val & (kLbAgg | kLbInc))) {
                set_error(f.p.status, kErrTimeout);
                val = kLbInc;
            }
        }
        const uint32_t inc_mask = __ballot_sync(0xffffffffu, (val & kLbInc) != 0);
        const int first = inc_mask ? __ffs(inc_mask) - 1 : 32;
        unsigned long long c = (lane <= first) ? (val & kLbMask) : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        excl += c;
        if (inc_mask) break;
        j0 -= 32;
    }
    if (lane == 0) st_relaxed_u64(my, kLbInc | (excl + U));
    return excl;
}

// Pairs of bucket region [base, base+n) whose key lies in [plo, phi], into
// registers blocked per warp (through shared memory when filtering).
__device__ uint32_t bkt_gather(BktSmem& sm, const BktProcParams& f, unsigned long long base, uint32_t n,
                               uint64_t plo, uint64_t phi, bool filter, uint64_t (&k)[kBktItems],
                               double (&v)[kBktItems], bool (&ok)[kBktItems]) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (!filter) {
#pragma unroll
        for (int j = 0; j < kBktItems; ++j) {
            const uint32_t pos = (uint32_t)(warp * (kBktItems * 32) + j * 32 + lane);
            ok[j] = pos < n;
            ulonglong2 w = make_ulonglong2(0ull, 0ull);
            if (ok[j]) w = __ldcs(f.pairs + base + pos);
            k[j] = w.x;
            v[j] = __longlong_as_double((long long)w.y);
        }
        return n;
    }
    if (tid == 0) sm.s_flag = 0;
    __syncthreads();
    const uint32_t lt = lane_lt_mask();
    for (uint32_t i0 = 0; i0 < n; i0 += kBktThreads) {
        const uint32_t i = i0 + tid;
        ulonglong2 w = make_ulonglong2(0ull, 0ull);
        bool in = false;
        if (i < n) {
            w = f.pairs[base + i];
            in = w.x >= plo && w.x <= phi;
        }
        // one shared atomic per warp: the leader reserves the warp's matches
        const uint32_t m = __ballot_sync(0xffffffffu, in);
        uint32_t at = 0;
        if (lane == 0 && m) at = atomicAdd(&sm.s_flag, (uint32_t)__popc(m));
        at = __shfl_sync(0xffffffffu, at, 0) + __popc(m & lt);
        if (in && at < (uint32_t)kBktCap) {
            sm.skeys[bpad(at)] = w.x;
            sm.svals[bpad(at)] = __longlong_as_double((long long)w.y);
        }
    }
    __syncthreads();
    const uint32_t m = min(sm.s_flag, (uint32_t)kBktCap);
#pragma unroll
    for (int j = 0; j < kBktItems; ++j) {
        const uint32_t pos = (uint32_t)(warp * (kBktItems * 32) + j * 32 + lane);
        ok[j] = pos < m;
        k[j] = ok[j] ? sm.skeys[bpad(pos)] : 0ull;
        v[j] = ok[j] ? sm.svals[bpad(pos)] : 0.0;
    }
    __syncthreads();
    return m;
}

// Sum of every pair with key == key0 in the region, fixed order.
__device__ double bkt_single_key_sum(BktSmem& sm, const BktProcParams& f, unsigned long long base, uint32_t n,
                                     uint64_t key0) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double s = 0.0;
    for (uint32_t i = tid; i < n; i += kBktThreads) {
        const ulonglong2 w = f.pairs[base + i];
        if (w.x == key0) s += __longlong_as_double((long long)w.y);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) sm.lead[warp] = s;
    __syncthreads();
    double tot = 0.0;
    for (int w = 0; w < kBktWarps; ++w) tot += sm.lead[w];
    __syncthreads();
    return tot;
}

__global__ void __launch_bounds__(kBktThreads, 1) k_bkt_process(BktProcParams f) {
    extern __shared__ __align__(16) unsigned char bsm_raw[];
    BktSmem& sm = *reinterpret_cast<BktSmem*>(bsm_raw);
    const StreamDesc& p = f.p;
    const int tid = threadIdx.x;
    const uint32_t nb = *f.nbounds;
    const uint32_t nbk = nb + 1;
    uint64_t k[kBktItems];
    double v[kBktItems];
    bool ok[kBktItems];
    for (;;) {
        if (tid == 0) sm.s_ticket = atomicAdd(f.ticket, 1u);
        __syncthreads();
        const uint32_t b = sm.s_ticket;
        __syncthreads();
        if (b >= nbk) break;
        const unsigned long long base = f.region[b];
        const uint32_t n = (uint32_t)min(f.count[b], f.cap[b]);
        const uint64_t lo = b == 0 ? 0ull : f.bounds[b - 1] + 1;
        const uint64_t hi = b == nb ? p.nkeys - 1 : f.bounds[b];
        if (n == 0) {
            if (tid < 32) {
                const unsigned long long e = bkt_lookback(f, b, 0);
                if (tid == 0) {
                    sm.s_excl = e;
                    if (b == nb) p.status->nnz_out = e;
                }
            }
            __syncthreads();
            continue;
        }
        if (n <= (uint32_t)kBktCap) {
            // the common case: the whole bucket on chip, one sort over the keys' span
            bkt_gather(sm, f, base, n, lo, hi, false, k, v, ok);
            uint64_t mn, mx;
            bkt_minmax(sm, k, ok, mn, mx);
            bkt_sort_part(sm, k, v, ok, n, mn, bits_of_range(mx - mn));
            uint32_t heads, hb;
            const uint32_t U = bkt_reduce_regs(sm, n, k, v, heads, hb);
            if (tid < 32) {
                const unsigned long long e = bkt_lookback(f, b, U);
                if (tid == 0) {
                    sm.s_excl = e;
                    if (b == nb) p.status->nnz_out = e + U;
                }
            }
            __syncthreads();
            bkt_emit_regs(sm, n, k, v, heads, hb, p, f.out_subs, f.out_vals, sm.s_excl, f.cap_rows, p.status);
            __syncthreads();
            continue;
        }
        // oversized: split the key range by histograms until every part fits;
        // sweep 0 counts unique keys, sweep 1 emits them.
        if (tid == 0) atomicAdd(&p.status->aux[0], 1ull);
        unsigned long long total_u = 0;
        for (int sweep = 0; sweep < 2; ++sweep) {
            unsigned long long out_at = sweep ? sm.s_excl : 0ull;
            if (tid == 0) {
                sm.stack_top = 1;
                sm.stack_lo[0] = lo;
                sm.stack_hi[0] = hi;
                sm.stack_n[0] = n;
            }
            __syncthreads();
            for (int guard = 0;; ++guard) {
                const int top = sm.stack_top;
                if (top == 0) break;
                if (guard > 100000) {          // never reached: every split narrows the range
                    if (tid == 0) set_error(p.status, kErrRetry);
                    break;
                }
                const uint64_t plo = sm.stack_lo[top - 1], phi = sm.stack_hi[top - 1];
                const unsigned long long pn = sm.stack_n[top - 1];
                __syncthreads();
                if (tid == 0) sm.stack_top = top - 1;
                __syncthreads();
                if (pn == 0) continue;
                if (pn <= (unsigned long long)kBktCap) {
                    const uint32_t m = bkt_gather(sm, f, base, n, plo, phi, true, k, v, ok);
                    uint64_t mn, mx;
                    bkt_minmax(sm, k, ok, mn, mx);
                    bkt_sort_part(sm, k, v, ok, m, mn, bits_of_range(mx - mn));
                    uint32_t heads, hb;
                    const uint32_t U = bkt_reduce_regs(sm, m, k, v, heads, hb);
                    if (sweep == 1)
                        bkt_emit_regs(sm, m, k, v, heads, hb, p, f.out_subs, f.out_vals, out_at, f.cap_rows, p.status);
                    __syncthreads();
                    out_at += U;
                    total_u += U;
                    continue;
                }
                if (plo == phi) {
                    const double sum = bkt_single_key_sum(sm, f, base, n, plo);
                    if (sweep == 1 && tid == 0) {
                        if ((int64_t)out_at < f.cap_rows) {
                            if (p.nr > 0) delinearise(p, plo, f.out_subs + out_at * p.nr);
                            f.out_vals[out_at] = sum;
                        } else {
                            set_error(p.status, kErrCapacity);
                        }
                    }
                    out_at += 1;
                    total_u += 1;
                    __syncthreads();
                    continue;
                }
                // histogram of the top 11 bits of key - plo inside [plo, phi]
                const int bits = bits_of_range(phi - plo);
                const int shift = bits > 11 ? bits - 11 : 0;
                for (int i = tid; i < 2048; i += kBktThreads) sm.hist11[i] = 0;
                __syncthreads();
                for (uint32_t i = tid; i < n; i += kBktThreads) {
                    const uint64_t kk = f.pairs[base + i].x;
                    if (kk >= plo && kk <= phi) atomicAdd(&sm.hist11[(kk - plo) >> shift], 1u);
                }
                __syncthreads();
                if (tid == 0) {
                    const int nbins = (int)((phi - plo) >> shift) + 1;
                    int ng = 0;
                    int start = 0;
                    unsigned long long acc = 0;
                    int t = sm.stack_top;
                    int* gstart = sm.gstart;
                    int* gend = sm.gend;
                    unsigned long long* gcnt = sm.gcnt;
                    bool overflow = false;
                    // an over-full bin is always a group of its own (its key range is
                    // strictly narrower than the part's, since a part spans >= 2 bins);
                    // groups without pairs are dropped
                    auto close = [&](int a, int e, unsigned long long c) {
                        if (c == 0) return;
                        if (ng < 64) { gstart[ng] = a; gend[ng] = e; gcnt[ng] = c; ++ng; }
                        else overflow = true;
                    };
                    for (int i = 0; i < nbins; ++i) {
                        const unsigned long long c = sm.hist11[i];
                        if (c > (unsigned long long)kBktCap) {
                            close(start, i - 1, acc);
                            close(i, i, c);
                            start = i + 1;
                            acc = 0;
                            continue;
                        }
                        if (acc + c > (unsigned long long)kBktCap) {
                            close(start, i - 1, acc);
                            start = i;
                            acc = 0;
                        }
                        acc += c;
                    }
                    if (start < nbins) close(start, nbins - 1, acc);
                    if (overflow || t + ng > 64) {
                        set_error(p.status, kErrRetry);
                        sm.stack_top = 0;
                    } else {
                        for (int g = ng - 1; g >= 0; --g) {
                            const uint64_t glo = plo + ((uint64_t)gstart[g] << shift);
                            uint64_t ghi = plo + (((uint64_t)gend[g] + 1) << shift) - 1;
                            if (ghi > phi || ghi < glo) ghi = phi;
                            sm.stack_lo[t] = glo;
                            sm.stack_hi[t] = ghi;
                            sm.stack_n[t] = gcnt[g];
                            ++t;
                        }
                        sm.stack_top = t;
                    }
                }
                __syncthreads();
            }
            if (sweep == 0) {
                if (tid < 32) {
                    const unsigned long long e = bkt_lookback(f, b, total_u);
                    if (tid == 0) {
                        sm.s_excl = e;
                        if (b == nb) p.status->nnz_out = e + total_u;
                    }
                }
                __syncthreads();
                total_u = 0;
            }
        }
    }
}

// ---- host side ------------------------------------------------------------------
struct BucketPlan {
    int S, B;
    int64_t total1, total2;
};

BucketPlan plan_bucket(int64_t nnz) {
    BucketPlan bp;
    bp.B = (int)std::max<int64_t>(2, std::min<int64_t>(kBktFineQuantiles, (nnz + 4095) / 4096));
    bp.S = (int)std::min<int64_t>(nnz, std::max<int64_t>(64 * (int64_t)bp.B, 1 << 16));
    bp.S = std::min(bp.S, 1 << 20);
    bp.total1 = 2 * nnz + (int64_t)kBktMaxL1 * 4 * kPartTile;
    bp.total2 = 2 * nnz + 256ll * (kBktMaxFine + 1);
    return bp;
}

namespace {
struct BucketLayout {
    uint64_t* samples[2];
    double* sample_vals[2];
    char* sort_ws;
    uint64_t* fine;
    uint32_t* nfine;
    uint64_t* l1_eyt;
    uint64_t* fine_eyt;
    unsigned long long *region1, *cap1, *count1;
    uint32_t* tile_start;
    uint32_t* tickets;
    unsigned long long *region, *cap, *count, *lookback;
    ulonglong2* pairs1;
    ulonglong2* pairs;
    size_t bytes;
};

BucketLayout bucket_layout(const BucketPlan& bp, int key_bits, char* base) {
    BucketLayout L;
    size_t off = 0;
    auto take = [&](size_t x) {
        char* r = base ? base + off : nullptr;
        off += (x + 255) & ~size_t(255);
        return r;
    };
    L.samples[0] = reinterpret_cast<uint64_t*>(take((size_t)bp.S * 8));
    L.samples[1] = reinterpret_cast<uint64_t*>(take((size_t)bp.S * 8));
    L.sample_vals[0] = reinterpret_cast<double*>(take((size_t)bp.S * 8));
    L.sample_vals[1] = reinterpret_cast<double*>(take((size_t)bp.S * 8));
    L.sort_ws = take(sort_workspace_bytes(bp.S, key_bits));
    L.fine = reinterpret_cast<uint64_t*>(take((size_t)kBktMaxFine * 8));
    L.nfine = reinterpret_cast<uint32_t*>(take(64));
    L.l1_eyt = reinterpret_cast<uint64_t*>(take(256 * 8));
    L.fine_eyt = reinterpret_cast<uint64_t*>(take((size_t)kBktMaxL1 * 256 * 8));
    L.region1 = reinterpret_cast<unsigned long long*>(take((size_t)kBktMaxL1 * 8 * 3));
    L.cap1 = L.region1 + kBktMaxL1;
    L.count1 = L.cap1 + kBktMaxL1;
    L.tile_start = reinterpret_cast<uint32_t*>(take((size_t)(kBktMaxL1 + 1) * 4));
    L.tickets = reinterpret_cast<uint32_t*>(take(64));
    const size_t nfb = kBktMaxFine + 1;
    L.region = reinterpret_cast<unsigned long long*>(take(nfb * 8 * 4));
    L.cap = L.region + nfb;
    L.count = L.cap + nfb;
    L.lookback = L.count + nfb;
    L.pairs1 = reinterpret_cast<ulonglong2*>(take((size_t)bp.total1 * 16));
    L.pairs = reinterpret_cast<ulonglong2*>(take((size_t)bp.total2 * 16));
    L.bytes = off;
    return L;
}
}  // namespace

size_t bucket_workspace_bytes(int64_t nnz, int key_bits) {
    return bucket_layout(plan_bucket(nnz), key_bits, nullptr).bytes;
}

typedef void (*BktPart1Kernel)(StreamDesc, const uint64_t*, const unsigned long long*, const unsigned long long*,
                               unsigned long long*, ulonglong2*);

template <int D>
static BktPart1Kernel pick_part1(bool soa) { return soa ? k_bkt_part1<D, true> : k_bkt_part1<D, false>; }

static BktPart1Kernel part1_kernel(int d, bool soa) {
    switch (d) {
        case 2: return pick_part1<2>(soa);
        case 3: return pick_part1<3>(soa);
        case 4: return pick_part1<4>(soa);
        case 5: return pick_part1<5>(soa);
        case 6: return pick_part1<6>(soa);
        default: return nullptr;
    }
}

bool bucket_applicable(const StreamDesc& p) {
    if (p.d < 2 || p.d > 6 || p.nnz < 2) return false;
    const uintptr_t sb = reinterpret_cast<uintptr_t>(p.subs), vb = reinterpret_cast<uintptr_t>(p.vals);
    if ((sb & 15) || (vb & 15)) return false;
    const bool soa = p.snz == 1 && (p.smode % 2 == 0);
    const bool aos = p.snz == p.d && p.smode == 1;
    return soa || aos;
}

void launch_bucket(const StreamDesc& p, int key_bits, void* ws, int64_t* out_subs, double* out_vals,
                   int64_t cap_rows, cudaStream_t stream) {
    const BucketPlan bp = plan_bucket(p.nnz);
    BucketLayout L = bucket_layout(bp, key_bits, static_cast<char*>(ws));
    // sort scratch for the samples (same layout as sort_workspace_bytes)
    SortBuffers ssb;
    {
        const int npass = (key_bits + 7) / 8;
        const int64_t ntiles = (bp.S + 4095) / 4096;
        char* q = L.sort_ws;
        auto t2 = [&](size_t x) { char* r = q; q += (x + 255) & ~size_t(255); return r; };
        t2((size_t)bp.S * 8 * 4);
        ssb.keys[0] = L.samples[0];
        ssb.keys[1] = L.samples[1];
        ssb.vals[0] = L.sample_vals[0];
        ssb.vals[1] = L.sample_vals[1];
        ssb.hist = reinterpret_cast<uint32_t*>(t2((size_t)std::max(npass, 1) * 256 * 4));
        ssb.lookback = reinterpret_cast<uint32_t*>(t2((size_t)std::max(npass, 1) * ntiles * 256 * 4));
        ssb.tickets = reinterpret_cast<uint32_t*>(t2(64 * 4));
        ssb.npass = npass;
        ssb.ntiles = ntiles;
    }
    cudaMemsetAsync(L.count1, 0, (size_t)kBktMaxL1 * 8, stream);
    cudaMemsetAsync(L.count, 0, (size_t)(kBktMaxFine + 1) * 8 * 2, stream);     // count + lookback
    cudaMemsetAsync(L.tickets, 0, 64, stream);
    TTV_LAUNCH("bkt_sample", stream,
               k_bkt_sample<<<(bp.S + 255) / 256, 256, 0, stream>>>(p, bp.S, L.samples[0], L.sample_vals[0]));
    const int cur = radix_sort_pairs(ssb, bp.S, key_bits, p.status, stream);
    BktBoundsOut bo;
    bo.fine = L.fine;
    bo.nfine = L.nfine;
    bo.l1_eyt = L.l1_eyt;
    bo.fine_eyt = L.fine_eyt;
    bo.region1 = L.region1;
    bo.cap1 = L.cap1;
    bo.region = L.region;
    bo.cap = L.cap;
    bo.total1 = bp.total1;
    bo.total2 = bp.total2;
    TTV_LAUNCH("bkt_bounds", stream, k_bkt_bounds<<<1, 1024, 0, stream>>>(L.samples[cur], bp.S, bp.B, p.nnz, bo, p.status));
    TTV_LAUNCH("bkt_caps", stream,
               k_bkt_caps<<<(kBktMaxFine + 1 + 255) / 256, 256, 0, stream>>>(L.samples[cur], bp.S, p.nnz, L.fine,
                                                                               L.nfine, L.cap));
    TTV_LAUNCH("bkt_regions", stream,
               k_bkt_regions<<<1, 1024, 0, stream>>>(L.nfine, bp.total1, bp.total2, L.cap, L.region, L.cap1,
                                                    L.region1));
    const bool soa = p.snz == 1;
    BktPart1Kernel pk = part1_kernel(p.d, soa);
    const size_t psmem = sizeof(PartSmem);
    cudaFuncSetAttribute(pk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psmem);
    cudaFuncSetAttribute(k_bkt_part2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psmem);
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pk, kPartThreads, psmem);
    const int pgrid = num_sms() * std::max(1, per_sm);
    TTV_LAUNCH("bkt_part1", stream,
               pk<<<pgrid, kPartThreads, psmem, stream>>>(p, L.l1_eyt, L.region1, L.cap1, L.count1, L.pairs1));
    TTV_LAUNCH("bkt_tiles", stream, k_bkt_tiles<<<1, 32, 0, stream>>>(L.nfine, L.count1, L.cap1, L.tile_start));
    int per_sm2 = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm2, k_bkt_part2, kPartThreads, psmem);
    TTV_LAUNCH("bkt_part2", stream,
               k_bkt_part2<<<num_sms() * std::max(1, per_sm2), kPartThreads, psmem, stream>>>(
                   L.nfine, L.fine_eyt, L.tile_start, L.region1, L.cap1, L.count1, L.pairs1, L.region, L.cap, L.count,
                   L.pairs, L.tickets, p.status));
    BktProcParams f;
    f.p = p;
    f.bounds = L.fine;
    f.nbounds = L.nfine;
    f.region = L.region;
    f.cap = L.cap;
    f.count = L.count;
    f.lookback = L.lookback;
    f.ticket = L.tickets + 1;
    f.pairs = L.pairs;
    f.out_subs = out_subs;
    f.out_vals = out_vals;
    f.cap_rows = cap_rows;
    const size_t smem = sizeof(BktSmem);
    cudaFuncSetAttribute(k_bkt_process, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    TTV_LAUNCH("bkt_process", stream, k_bkt_process<<<num_sms(), kBktThreads, smem, stream>>>(f));
}

}  // namespace ttv
