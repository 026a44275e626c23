// ttv_sort.cu -- stable LSD radix sort of (uint64 key, double term) pairs and
// the segmented reduction that turns sorted pairs into the canonical COO result.
//
// The sort is a "onesweep" LSD radix sort (A. Adinets and D. Merrill,
// "Onesweep: A Faster Least Significant Digit Radix Sort for GPUs", 2022):
// one upfront pass histograms every digit of every key; then each 8-bit digit
// pass ranks a tile of keys in shared memory (warp-level multi-split with
// __match_any_sync), publishes the tile's per-digit counts with a decoupled
// look-back across tiles, and scatters through a shared-memory staging buffer
// so that global writes of one digit are contiguous.  Tiles take a ticket from
// a global counter, so a tile only waits on tiles that are already running;
// every wait is bounded and reports kErrTimeout instead of hanging.
//
// Stability matters: equal keys keep their input order, so the reduction
// by key that follows (binary64 or compensated) sums every group in an order
// fixed by the input alone, and the result is bit-identical from run to run.
#include <cstdio>

#include "ttv_internal.cuh"

namespace ttv {

constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
// A digit pass takes 4096-pair tiles with 256 threads of 16 pairs, three
// CTAs per SM (measured against 512 threads of 8 pairs at two CTAs per SM:
// 8.60 against 8.91 ms for the 1e8-nonzero Zipf TTV).
constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;      // 4096 keys per tile
constexpr int kScanWarps = 8;                              // warps of the 256-thread scans
constexpr int kHistStride = kRadix + 1;                    // +1: padding bucket for absent items
constexpr uint32_t kFlagAgg = 1u << 30;
constexpr uint32_t kFlagInc = 2u << 30;
constexpr uint32_t kCountMask = (1u << 30) - 1;
constexpr int kLookWindow = 8;          // predecessor tiles read per look-back round trip

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed(uint32_t* p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Exclusive scan of one value per thread over a 256-thread block.
__device__ __forceinline__ uint32_t block_exclusive_scan_256(uint32_t x, uint32_t* warp_tot, uint32_t& total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    uint32_t before = 0, all = 0;
#pragma unroll
    for (int w = 0; w < kScanWarps; ++w) {
        uint32_t t = warp_tot[w];
        if (w < warp) before += t;
        all += t;
    }
    total = all;
    __syncthreads();
    return before + inc - x;
}

// ---------------------------------------------------------------------------
// Histogram of every digit pass in one read of the keys.
__global__ void __launch_bounds__(256) k_radix_hist(const uint64_t* __restrict__ keys, int64_t n, int npass,
                                                    uint32_t* __restrict__ hist,
                                                    const unsigned long long* __restrict__ n_dev) {
    __shared__ uint32_t sh[8 * kRadix];
    if (n_dev) n = min(n, (int64_t)*n_dev);
    for (int i = threadIdx.x; i < npass * kRadix; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint64_t k = __ldcs(keys + i);
        for (int p = 0; p < npass; ++p) atomicAdd(&sh[p * kRadix + ((k >> (p * kRadixBits)) & (kRadix - 1))], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < npass * kRadix; i += blockDim.x)
        if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

// In place: hist[p][d] -> exclusive prefix over digits of pass p.
__global__ void __launch_bounds__(256) k_radix_hist_scan(uint32_t* hist, int npass) {
    __shared__ uint32_t wt[kScanWarps];
    for (int p = 0; p < npass; ++p) {
        uint32_t x = hist[p * kRadix + threadIdx.x];
        uint32_t total;
        uint32_t ex = block_exclusive_scan_256(x, wt, total);
        hist[p * kRadix + threadIdx.x] = ex;
        __syncthreads();
    }
}

// One digit pass.  Dynamic shared memory: warp histograms, digit starts,
// global bases and a 4096-pair staging buffer.
struct OnesweepSmem {
    uint32_t whist[kSortWarps * kHistStride];
    uint32_t gdelta[kRadix];         // output index of tile slot j: gdelta[digit] + j
    uint32_t warp_tot[kSortWarps];
    uint32_t tile;
    uint32_t pad[3];
    uint64_t keys[kSortTile];
    double vals[kSortTile];
};

// Exclusive scan of the digit counts held by threads [0, kRadix) of a
// kSortThreads block; the other threads only pass through the barriers.
__device__ __forceinline__ uint32_t digit_exclusive_scan(uint32_t x, uint32_t* warp_tot) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31 && warp < kRadix / 32) warp_tot[warp] = inc;
    __syncthreads();
    uint32_t before = 0;
#pragma unroll
    for (int w = 0; w < kRadix / 32; ++w)
        if (w < warp) before += warp_tot[w];
    return before + inc - x;
}

// The pass over one tile, once the CTA holds its ticket and its warp
// histograms are zero (called by the single-problem and the batched kernel).
__device__ __forceinline__ void onesweep_tile(OnesweepSmem& sm, const uint64_t* __restrict__ keys_in,
                                              const double* __restrict__ vals_in, uint64_t* __restrict__ keys_out,
                                              double* __restrict__ vals_out, int64_t n, int shift,
                                              const uint32_t* __restrict__ digit_off, uint32_t* lookback,
                                              Status* st, uint32_t tile) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t base = (int64_t)tile * kSortTile;
    if (base >= n) return;
    const bool digit_thread = tid < kRadix;        // thread t < 256 owns digit t
    const uint32_t doff = digit_thread ? __ldg(digit_off + tid) : 0u;   // needed after the look-back

    // Keys first: ranking needs only them, and they go to shared memory
    // before the values are loaded, so that at most 8 keys or 8 values (plus
    // one packed word per item) are live per thread.
    uint64_t k[kSortItems];
    uint32_t rd[kSortItems];     // rank << 9 | digit, then the staging slot
    const int64_t wbase = base + warp * (kSortItems * 32) + lane;
#pragma unroll
    for (int i = 0; i < kSortItems; ++i) {
        const int64_t idx = wbase + i * 32;
        k[i] = idx < n ? __ldcs(keys_in + idx) : 0ull;
    }
    // Warp-level multi-split: rank of each item among equal digits of its
    // warp.  The lanes holding the same digit are found by one ballot per
    // digit bit, measured faster than __match_any_sync here; a ninth ballot
    // (the padding bucket of absent items) only in the last, partial tile
    // (8.35 against 8.66 ms for the 1e8 Zipf TTV with nine everywhere).
    uint32_t* wh = sm.whist + warp * kHistStride;
    const uint32_t lt = lanemask_lt();
    const bool full_tile = base + kSortTile <= n;
#pragma unroll
    for (int i = 0; i < kSortItems; ++i) {
        // padding bucket kRadix for absent items: never published or written
        const uint32_t dig = wbase + i * 32 < n ? (uint32_t)(k[i] >> shift) & (kRadix - 1) : (uint32_t)kRadix;
        uint32_t mask = 0xffffffffu;
#pragma unroll
        for (int b = 0; b < kRadixBits + (full_tile ? 0 : 1); ++b) {
            const uint32_t bit = (dig >> b) & 1u;
            const uint32_t bal = __ballot_sync(0xffffffffu, bit);
            mask &= bit ? bal : ~bal;
        }
        const int leader = __ffs(mask) - 1;
        uint32_t b = 0;
        // a plain read and write of the warp's counter (measured faster
        // than a shared atomic: 8.74 against 9.06 ms for the 1e8 Zipf TTV);
        // the __syncwarp below orders it before the next item's access
        if (lane == leader) {
            b = wh[dig];
            wh[dig] = b + __popc(mask);
        }
        b = __shfl_sync(0xffffffffu, b, leader);
        rd[i] = (b + __popc(mask & lt)) << 9 | dig;
        __syncwarp();
    }
    __syncthreads();

    // Thread t owns digit t: prefix over warps, tile count, tile-local start.
    uint32_t cnt = 0;
    if (digit_thread) {
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) {
            const uint32_t c = sm.whist[w * kHistStride + tid];
            sm.whist[w * kHistStride + tid] = cnt;
            cnt += c;
        }
    }
    const uint32_t start = digit_exclusive_scan(cnt, sm.warp_tot);
    if (digit_thread) {
        // each warp's slot base for digit t: the digit's tile start folded in
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) sm.whist[w * kHistStride + tid] += start;
    }
    __syncthreads();

    // Keys into shared memory in digit order (stable); keep each item's slot.
    constexpr uint32_t kAbsent = 0xffffffffu;
#pragma unroll
    for (int i = 0; i < kSortItems; ++i) {
        const uint32_t dig = rd[i] & 511u;
        if (dig < (uint32_t)kRadix) {
            const uint32_t pos = sm.whist[warp * kHistStride + dig] + (rd[i] >> 9);
            sm.keys[pos] = k[i];
            rd[i] = pos;
        } else {
            rd[i] = kAbsent;
        }
    }
    // Values: loads issued now, consumed after the look-back.
    double v[kSortItems];
#pragma unroll
    for (int i = 0; i < kSortItems; ++i) {
        const int64_t idx = wbase + i * 32;
        v[i] = idx < n ? __ldcs(vals_in + idx) : 0.0;
    }

    // Decoupled look-back across tiles for digit t.  The words of up to
    // kLookWindow predecessors are loaded together (one L2 round trip for
    // the window rather than one per tile), then taken in order; a word not
    // yet published is polled on its own.
    uint32_t* my = lookback + (size_t)tile * kRadix + tid;
    uint32_t exclusive = 0;
    if (!digit_thread) {
    } else if (tile == 0) {
        st_relaxed(my, kFlagInc | cnt);
    } else {
        st_relaxed(my, kFlagAgg | cnt);
        int64_t j = (int64_t)tile - 1;
        const uint32_t polls = wait_limit(1u << 24);
        bool done = false;
        while (!done && j >= 0) {
            uint32_t w[kLookWindow];
#pragma unroll
            for (int u = 0; u < kLookWindow; ++u)
                w[u] = j - u >= 0 ? ld_relaxed(lookback + (size_t)(j - u) * kRadix + tid) : 0u;
#pragma unroll
            for (int u = 0; u < kLookWindow; ++u) {
                if (done || j - u < 0) { done = true; break; }
                uint32_t val = w[u];
                if (!(val & (kFlagAgg | kFlagInc))) {
                    const uint32_t* q = lookback + (size_t)(j - u) * kRadix + tid;
                    bool ok = false;
                    for (uint32_t it = 0; it < polls; ++it) {
                        val = ld_relaxed(q);
                        if (val & (kFlagAgg | kFlagInc)) { ok = true; break; }
                        if (it > 32) __nanosleep(32);
                    }
                    if (!ok) { set_error(st, kErrTimeout); done = true; break; }
                }
                exclusive += val & kCountMask;
                if (val & kFlagInc) done = true;
            }
            j -= kLookWindow;
        }
        st_relaxed(my, kFlagInc | ((exclusive + cnt) & kCountMask));
    }
    if (digit_thread) sm.gdelta[tid] = doff + exclusive - start;
#pragma unroll
    for (int i = 0; i < kSortItems; ++i)
        if (rd[i] != kAbsent) sm.vals[rd[i]] = v[i];
    __syncthreads();

    // Out: consecutive threads write consecutive slots of each digit run.
    const int tile_n = (int)min((int64_t)kSortTile, n - base);
    for (int j = tid; j < tile_n; j += kSortThreads) {
        const uint64_t kk = sm.keys[j];
        const uint32_t d = (uint32_t)(kk >> shift) & (kRadix - 1);
        const uint32_t out = sm.gdelta[d] + (uint32_t)j;
        if ((int64_t)out >= n) continue;     // only after a look-back ran out: offsets are then unreliable
        keys_out[out] = kk;
        vals_out[out] = sm.vals[j];
    }
}

__global__ void __launch_bounds__(kSortThreads, 3) k_onesweep(const uint64_t* __restrict__ keys_in,
                                                           const double* __restrict__ vals_in,
                                                           uint64_t* __restrict__ keys_out,
                                                           double* __restrict__ vals_out, int64_t n, int shift,
                                                           const uint32_t* __restrict__ digit_off,
                                                           uint32_t* lookback, uint32_t* ticket, Status* st,
                                                           const unsigned long long* __restrict__ n_dev) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    OnesweepSmem& sm = *reinterpret_cast<OnesweepSmem*>(smem_raw);
    const int tid = threadIdx.x;
    if (tid == 0) sm.tile = atomicAdd(ticket, 1u);
    for (int i = tid; i < kSortWarps * kHistStride; i += kSortThreads) sm.whist[i] = 0;
    __syncthreads();
    const uint32_t tile = sm.tile;
    // With the count on the device, tiles past it have nothing to do; no
    // tile with work waits on them (look-back only reads earlier tiles).
    if (n_dev) n = min(n, (int64_t)*n_dev);
    onesweep_tile(sm, keys_in, vals_in, keys_out, vals_out, n, shift, digit_off, lookback, st, tile);
}

// The position in a job list of the problem that unit t falls in:
// prefix[j] <= t < prefix[j + 1] (problems with no units are skipped).
__device__ __forceinline__ int job_of(const uint32_t* __restrict__ prefix, int count, uint32_t t) {
    int lo = 0, hi = count;          // prefix[lo] <= t < prefix[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(prefix + mid) <= t) lo = mid;
        else hi = mid;
    }
    return lo;
}

// The position in job list l of the problem unit t belongs to: one load from
// the list's unit map when it has one, else a binary search of its prefix.
__device__ __forceinline__ int job_at(const JobList& l, uint32_t t) {
    return l.unit_pos ? (int)__ldg(l.unit_pos + t) : job_of(l.prefix, l.count, t);
}

// One digit pass over the tiles of every problem of a batch with more than
// `pass` digits (the list's first l.count problems).  CTAs take global
// tickets, problem after problem, so each problem's tiles are claimed in
// increasing order and its look-back only waits on tiles claimed before.
__global__ void __launch_bounds__(kSortThreads, 3) k_onesweep_batch(const BatchJob* __restrict__ jobs, JobList l,
                                                                 int pass, uint32_t* ticket) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    OnesweepSmem& sm = *reinterpret_cast<OnesweepSmem*>(smem_raw);
    __shared__ int s_pos;
    const int tid = threadIdx.x;
    if (tid == 0) {
        const uint32_t t = atomicAdd(ticket, 1u);
        sm.tile = t;
        s_pos = t < __ldg(l.prefix + l.count) ? job_at(l, t) : -1;
    }
    for (int i = tid; i < kSortWarps * kHistStride; i += kSortThreads) sm.whist[i] = 0;
    __syncthreads();
    const int pos = s_pos;
    if (pos < 0) return;
    const BatchJob& J = jobs[__ldg(l.idx + pos)];
    const int cur = pass & 1;
    onesweep_tile(sm, J.keys[cur], J.vals[cur], J.keys[cur ^ 1], J.vals[cur ^ 1], J.p.nnz, pass * kRadixBits,
                  J.hist + pass * kRadix, J.lookback + (size_t)pass * J.ntiles * kRadix, J.p.status,
                  sm.tile - __ldg(l.prefix + pos));
}

// Each problem's digit counts into exclusive prefixes: one CTA per problem.
__global__ void __launch_bounds__(256) k_radix_hist_scan_batch(const BatchJob* __restrict__ jobs, JobList l) {
    __shared__ uint32_t wt[kScanWarps];
    const BatchJob& J = jobs[__ldg(l.idx + blockIdx.x)];
    for (int p = 0; p < J.npass; ++p) {
        uint32_t x = J.hist[p * kRadix + threadIdx.x];
        uint32_t total;
        uint32_t ex = block_exclusive_scan_256(x, wt, total);
        J.hist[p * kRadix + threadIdx.x] = ex;
        __syncthreads();
    }
}

int64_t sort_tiles(int64_t n) { return (std::max<int64_t>(n, 1) + kSortTile - 1) / kSortTile; }

// Digit passes of a batch: the list is ordered by decreasing pass count, so
// pass p covers its first count_per_pass[p] problems (tiles_per_pass[p]
// tiles); tickets: one zeroed counter per pass.
void launch_sort_batch(const BatchJob* jobs, const JobList& all, const int32_t* count_per_pass,
                       const uint32_t* tiles_per_pass, int max_npass, uint32_t* tickets, cudaStream_t stream) {
    if (all.count <= 0 || max_npass <= 0) return;
    TTV_LAUNCH("radix_hist_scan", stream, k_radix_hist_scan_batch<<<(unsigned)all.count, 256, 0, stream>>>(jobs, all));
    const size_t smem = sizeof(OnesweepSmem);
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_onesweep_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(k_onesweep_batch, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
        attr_set = true;
    }
    for (int p = 0; p < max_npass; ++p) {
        if (count_per_pass[p] <= 0 || tiles_per_pass[p] == 0) break;
        JobList lp = all;
        lp.count = count_per_pass[p];
        TTV_LAUNCH("onesweep_batch", stream,
                   k_onesweep_batch<<<tiles_per_pass[p], kSortThreads, smem, stream>>>(jobs, lp, p, tickets + p));
    }
}

cudaError_t sort_set_wait_override(uint32_t v) { return set_wait_override_here(v); }

size_t sort_workspace_bytes(int64_t n, int bits) {
    const int npass = bits <= 0 ? 0 : (bits + kRadixBits - 1) / kRadixBits;
    const int64_t ntiles = (n + kSortTile - 1) / kSortTile;
    size_t b = 0;
    b += 2 * (size_t)n * sizeof(uint64_t) + 2 * (size_t)n * sizeof(double) + 4 * 256;
    b += (size_t)npass * kRadix * sizeof(uint32_t) + 256;
    b += (size_t)npass * ntiles * kRadix * sizeof(uint32_t) + 256;
    b += 64 * sizeof(uint32_t) + 256;
    return b;
}

int radix_sort_pairs(SortBuffers& sb, int64_t n, int bits, Status* st, cudaStream_t stream,
                     const unsigned long long* n_dev, bool hist_ready) {
    const int npass = bits <= 0 ? 0 : (bits + kRadixBits - 1) / kRadixBits;
    if (npass == 0 || n <= 1) return 0;
    const int64_t ntiles = (n + kSortTile - 1) / kSortTile;
    if (!hist_ready) cudaMemsetAsync(sb.hist, 0, (size_t)npass * kRadix * sizeof(uint32_t), stream);
    cudaMemsetAsync(sb.lookback, 0, (size_t)npass * ntiles * kRadix * sizeof(uint32_t), stream);
    cudaMemsetAsync(sb.tickets, 0, 64 * sizeof(uint32_t), stream);
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int hblocks = (int)std::min<int64_t>((int64_t)nsm * 4, (n + 255) / 256);
    if (!hist_ready)
        TTV_LAUNCH("radix_hist", stream, k_radix_hist<<<hblocks, 256, 0, stream>>>(sb.keys[0], n, npass, sb.hist, n_dev));
    TTV_LAUNCH("radix_hist_scan", stream, k_radix_hist_scan<<<1, 256, 0, stream>>>(sb.hist, npass));
    const size_t smem = sizeof(OnesweepSmem);
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_onesweep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        // all of the unified L1 as shared memory: three 75 KB CTAs per SM
        cudaFuncSetAttribute(k_onesweep, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
        attr_set = true;
    }
    int cur = 0;
    for (int p = 0; p < npass; ++p) {
        TTV_LAUNCH("onesweep", stream, k_onesweep<<<(unsigned)ntiles, kSortThreads, smem, stream>>>(
            sb.keys[cur], sb.vals[cur], sb.keys[cur ^ 1], sb.vals[cur ^ 1], n, p * kRadixBits,
            sb.hist + p * kRadix, sb.lookback + (size_t)p * ntiles * kRadix, sb.tickets + p, st, n_dev));
        cur ^= 1;
    }
    return cur;
}

// ---------------------------------------------------------------------------
// Reduce-by-key of sorted pairs (binary64 accumulation), in three passes
// with no waiting between tiles.
//
// A pair is a head when its key differs from its predecessor's.  Every
// thread takes 8 consecutive pairs (16-byte loads) and summarises them as
// (heads, has_head, open value: the sum since its last head, or of all its
// pairs when it has none).  Summaries combine left to right by
//     (ca, fa, va) . (cb, fb, vb) = (ca + cb, fa | fb, fb ? vb : va + vb).
//   k_rbk_tiles  one summary per 2048-pair tile (fixed shuffle tree);
//   k_rbk_groups one warp per 32 tiles: in-group exclusive prefixes and the
//                group summary (fixed shuffle tree);
//   k_rbk_scan   one CTA: exclusive scan of the group summaries (each thread
//                a fixed chunk, then a fixed tree over the chunks): heads
//                before each group and the open value entering it;
//   k_rbk_emit   the tile again: in-tile exclusive scan, then every head
//                closes the segment before it (the last pair closes the
//                last one): key and sum staged in shared memory at the
//                segment's row within the tile, then written out coalesced,
//                the key delinearised into the surviving subscripts.
// Every combination happens in an order fixed by the data layout alone, so
// the result is bit-identical from run to run.
constexpr int kRbkThreads = 256;
constexpr int kRbkItems = 8;
constexpr int kRbkTile = kRbkThreads * kRbkItems;
constexpr int kRbkScanThreads = 1024;

struct RbkSum {                  // a summary: values first for alignment
    double val;
    double comp;                 // compensated sums: the running error term (0 otherwise)
    uint32_t cnt;
    uint32_t flag;
};

// s + c += x with Neumaier's correction
__device__ __forceinline__ void nm_add(double& s, double& c, double x) {
    const double t = s + x;
    c += fabs(s) >= fabs(x) ? (s - t) + x : (x - t) + s;
    s = t;
}

// The value of a compensated sum s + c.  Once s is not finite the plain sum
// is the value: the correction would turn a lone infinity into a NaN, while
// Eq. 3's plain sum keeps it.
__device__ __forceinline__ double nm_value(double s, double c) { return isfinite(s) ? s + c : s; }

// (ca, fa, va, ka) . (cb, fb, vb, kb) -> b; kComp carries the error terms k
template <bool kComp>
__device__ __forceinline__ void seg_combine(uint32_t ca, uint32_t fa, double va, double ka, uint32_t& cb,
                                            uint32_t& fb, double& vb, double& kb) {
    cb = ca + cb;
    if constexpr (kComp) {
        if (!fb) {
            double sv = va, sk = ka;
            nm_add(sv, sk, vb);
            vb = sv;
            kb = sk + kb;
        }
    } else {
        vb = fb ? vb : va + vb;
    }
    fb = fa | fb;
}

// This thread's pairs of tile `tile` and their summary.
struct RbkPairs {
    uint64_t k[kRbkItems];
    double v[kRbkItems];
    double done[kRbkItems];      // at a head: the sum of the run it closes (at the first head: of the items before it)
    uint64_t prev0;
    int nmine;
    int64_t g0;
    uint32_t heads, cnt, flag;
    double open;
    double first_done;           // done[] at this thread's first head (0 when it has none)
    double open_k, first_k;      // compensated sums: error terms of open and first_done
};

// Terms of the sort path: stored next to the sorted keys.
struct PairTerms {
    const double* vals;
    __device__ __forceinline__ double term(int64_t k) const { return __ldcs(vals + k); }
    __device__ __forceinline__ void load(int64_t g0, int nmine, double* v) const {
        if (nmine == kRbkItems) {
            // the pair buffers are 16-byte aligned and g0 is a multiple of 8
#pragma unroll
            for (int q = 0; q < kRbkItems / 2; ++q) {
                const double2 vv = __ldcs(reinterpret_cast<const double2*>(vals + g0) + q);
                v[2 * q] = vv.x;
                v[2 * q + 1] = vv.y;
            }
        } else {
#pragma unroll
            for (int i = 0; i < kRbkItems; ++i) v[i] = i < nmine ? vals[g0 + i] : 0.0;
        }
    }
};

// Terms of a prepared tensor: formed on the fly from the value and the
// contracted modes' subscripts stored in key order, the product taken in
// increasing mode order exactly as the streaming kernels take it.
struct PrepTermsDev {
    PrepTerms t;
    __device__ __forceinline__ double x(int j, int32_t s) const {
        return t.vec_f32 ? (double)__ldg(static_cast<const float*>(t.vec[j]) + s)
                         : __ldg(static_cast<const double*>(t.vec[j]) + s);
    }
    __device__ __forceinline__ double term(int64_t k) const {
        double tt = t.val_f32 ? (double)__ldcs(static_cast<const float*>(t.vals) + k)
                              : __ldcs(static_cast<const double*>(t.vals) + k);
        for (int j = 0; j < t.n_v; ++j) tt = tt * x(j, __ldcs(t.sub[j] + k));
        return tt;
    }
    __device__ __forceinline__ void load(int64_t g0, int nmine, double* v) const {
        if (t.n_v == 1 && nmine == kRbkItems) {
            // one vector, a full run of 8: 16-byte loads of the values and
            // subscripts (the arrays are 256-byte aligned, g0 a multiple of 8),
            // then 8 independent gathers
            int32_t sb[kRbkItems];
#pragma unroll
            for (int q = 0; q < kRbkItems / 4; ++q) {
                const int4 w = __ldcs(reinterpret_cast<const int4*>(t.sub[0] + g0) + q);
                sb[4 * q] = w.x;
                sb[4 * q + 1] = w.y;
                sb[4 * q + 2] = w.z;
                sb[4 * q + 3] = w.w;
            }
            if (t.val_f32) {
#pragma unroll
                for (int q = 0; q < kRbkItems / 4; ++q) {
                    const float4 w = __ldcs(reinterpret_cast<const float4*>(static_cast<const float*>(t.vals) + g0) + q);
                    v[4 * q] = (double)w.x;
                    v[4 * q + 1] = (double)w.y;
                    v[4 * q + 2] = (double)w.z;
                    v[4 * q + 3] = (double)w.w;
                }
            } else {
#pragma unroll
                for (int q = 0; q < kRbkItems / 2; ++q) {
                    const double2 w =
                        __ldcs(reinterpret_cast<const double2*>(static_cast<const double*>(t.vals) + g0) + q);
                    v[2 * q] = w.x;
                    v[2 * q + 1] = w.y;
                }
            }
            double xs[kRbkItems];
#pragma unroll
            for (int i = 0; i < kRbkItems; ++i) xs[i] = x(0, sb[i]);
#pragma unroll
            for (int i = 0; i < kRbkItems; ++i) v[i] = v[i] * xs[i];
            return;
        }
#pragma unroll
        for (int i = 0; i < kRbkItems; ++i) {
            if (i < nmine) {
                const int64_t k = g0 + i;
                double tt = t.val_f32 ? (double)__ldcs(static_cast<const float*>(t.vals) + k)
                                      : __ldcs(static_cast<const double*>(t.vals) + k);
                for (int j = 0; j < t.n_v; ++j) tt = tt * x(j, __ldcs(t.sub[j] + k));
                v[i] = tt;
            } else {
                v[i] = 0.0;
            }
        }
    }
};

// Where the run heads come from: comparing neighbouring sorted keys, or a
// prepared bitmap (bit i of byte i/8 set when pair i starts a run) with the
// key of every run stored by run index.
struct KeyHeads {
    static constexpr bool kBits = false;
    const uint64_t* keys;
};
struct BitHeads {
    static constexpr bool kBits = true;
    const uint8_t* bits;
    const uint64_t* row_keys;
};
__device__ __forceinline__ const uint64_t* key_array(const KeyHeads& h) { return h.keys; }
__device__ __forceinline__ const uint64_t* key_array(const BitHeads&) { return nullptr; }

// This thread's run heads in tile `tile` (bit i: pair g0 + i starts a run)
// and its pair count, without the terms.
template <class H>
__device__ __forceinline__ uint32_t rbk_heads(const H& hd, int64_t n, int64_t g0, int nmine) {
    if (nmine <= 0) return 0u;
    if constexpr (H::kBits) {
        return (uint32_t)hd.bits[g0 >> 3] & ((1u << nmine) - 1u);
    } else {
        const uint64_t* keys = key_array(hd);
        uint64_t k[kRbkItems];
        if (nmine == kRbkItems) {
#pragma unroll
            for (int q = 0; q < kRbkItems / 2; ++q) {
                const ulonglong2 kk = __ldcs(reinterpret_cast<const ulonglong2*>(keys + g0) + q);
                k[2 * q] = kk.x;
                k[2 * q + 1] = kk.y;
            }
        } else {
#pragma unroll
            for (int i = 0; i < kRbkItems; ++i) k[i] = i < nmine ? keys[g0 + i] : ~0ull;
        }
        uint64_t prev = g0 > 0 ? keys[g0 - 1] : ~0ull;
        uint32_t heads = 0;
#pragma unroll
        for (int i = 0; i < kRbkItems; ++i) {
            if (i < nmine && (k[i] != prev || g0 + i == 0)) heads |= 1u << i;
            prev = k[i];
        }
        return heads;
    }
}

template <bool kComp, class H, class Src>
__device__ __forceinline__ void rbk_load(const H& hd, const Src& src, int64_t n, int64_t tile, RbkPairs& r) {
    r.g0 = tile * kRbkTile + (int64_t)threadIdx.x * kRbkItems;
    r.nmine = (int)max((int64_t)0, min((int64_t)kRbkItems, n - r.g0));
    if constexpr (H::kBits) {
        src.load(r.g0, r.nmine, r.v);
        // g0 is a multiple of 8: this thread's heads are one byte
        r.heads = r.nmine > 0 ? (uint32_t)hd.bits[r.g0 >> 3] & ((1u << r.nmine) - 1u) : 0u;
        r.prev0 = 0;
        r.cnt = __popc(r.heads);
        r.flag = r.heads != 0;
        double acc = 0.0, ak = 0.0;
        r.first_done = 0.0;
        r.first_k = 0.0;
        const int fh = r.heads ? __ffs(r.heads) - 1 : kRbkItems;
#pragma unroll
        for (int i = 0; i < kRbkItems; ++i) {
            r.done[i] = 0.0;
            if (i < r.nmine) {
                if ((r.heads >> i) & 1u) {
                    if constexpr (kComp) {
                        r.done[i] = nm_value(acc, ak);   // a run closed inside the range: final value
                        if (i == fh) { r.first_done = acc; r.first_k = ak; }
                        ak = 0.0;
                    } else {
                        r.done[i] = acc;
                        if (i == fh) r.first_done = acc;
                    }
                    acc = r.v[i];
                } else {
                    if constexpr (kComp) nm_add(acc, ak, r.v[i]);
                    else acc = acc + r.v[i];
                }
            }
        }
        r.open = acc;
        r.open_k = ak;
        return;
    }
    const uint64_t* keys = key_array(hd);
    if (r.nmine == kRbkItems) {
        // the key buffer is 16-byte aligned and g0 is a multiple of 8
#pragma unroll
        for (int q = 0; q < kRbkItems / 2; ++q) {
            const ulonglong2 kk = __ldcs(reinterpret_cast<const ulonglong2*>(keys + r.g0) + q);
            r.k[2 * q] = kk.x;
            r.k[2 * q + 1] = kk.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < kRbkItems; ++i) r.k[i] = i < r.nmine ? keys[r.g0 + i] : ~0ull;
    }
    src.load(r.g0, r.nmine, r.v);
    r.prev0 = (r.g0 > 0 && r.nmine > 0) ? keys[r.g0 - 1] : ~0ull;   // keys are < 2^64 - 1
    r.heads = 0;
    r.cnt = 0;
    r.flag = 0;
    double acc = 0.0, ak = 0.0;
    uint64_t prev = r.prev0;
    r.first_done = 0.0;
    r.first_k = 0.0;
#pragma unroll
    for (int i = 0; i < kRbkItems; ++i) {
        r.done[i] = 0.0;
        if (i < r.nmine) {
            if (r.k[i] != prev || r.g0 + i == 0) {
                if constexpr (kComp) {
                    if (!r.flag) { r.first_done = acc; r.first_k = ak; }
                    r.done[i] = nm_value(acc, ak);
                    ak = 0.0;
                } else {
                    if (!r.flag) r.first_done = acc;
                    r.done[i] = acc;
                }
                r.heads |= 1u << i;
                ++r.cnt;
                r.flag = 1;
                acc = r.v[i];
            } else {
                if constexpr (kComp) nm_add(acc, ak, r.v[i]);
                else acc = acc + r.v[i];
            }
            prev = r.k[i];
        }
    }
    r.open = acc;
    r.open_k = ak;
}

// Block scan of the thread summaries: each thread gets its exclusive prefix
// within the tile; returns the tile total (all threads).
struct RbkScanSmem {
    uint32_t cnt[kRbkThreads / 32];
    uint32_t flag[kRbkThreads / 32];
    double val[kRbkThreads / 32];
    double kv[kRbkThreads / 32];
    uint32_t pcnt[kRbkThreads / 32 + 1];   // exclusive prefix of warp w; [8]: the tile total
    uint32_t pflag[kRbkThreads / 32 + 1];
    double pval[kRbkThreads / 32 + 1];
    double pk[kRbkThreads / 32 + 1];
};

template <bool kComp>
__device__ __forceinline__ void rbk_block_scan(const RbkPairs& r, RbkScanSmem& ss, uint32_t& xc, uint32_t& xf,
                                               double& xv, double& xk, uint32_t& tc, uint32_t& tf, double& tv,
                                               double& tk) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t c = r.cnt, f = r.flag;
    double v = r.open, k = kComp ? r.open_k : 0.0;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t c2 = __shfl_up_sync(0xffffffffu, c, off);
        const uint32_t f2 = __shfl_up_sync(0xffffffffu, f, off);
        const double v2 = __shfl_up_sync(0xffffffffu, v, off);
        const double k2 = kComp ? __shfl_up_sync(0xffffffffu, k, off) : 0.0;
        if (lane >= off) seg_combine<kComp>(c2, f2, v2, k2, c, f, v, k);
    }
    if (lane == 31) {
        ss.cnt[warp] = c;
        ss.flag[warp] = f;
        ss.val[warp] = v;
        if (kComp) ss.kv[warp] = k;
    }
    xc = __shfl_up_sync(0xffffffffu, c, 1);
    xf = __shfl_up_sync(0xffffffffu, f, 1);
    xv = __shfl_up_sync(0xffffffffu, v, 1);
    xk = kComp ? __shfl_up_sync(0xffffffffu, k, 1) : 0.0;
    if (lane == 0) { xc = 0; xf = 0; xv = 0.0; xk = 0.0; }
    __syncthreads();
    // warp prefixes, folded left to right over the 8 warps by one thread
    if (threadIdx.x == 0) {
        uint32_t pc = ss.cnt[0], pf = ss.flag[0];
        double pv = ss.val[0], pk = kComp ? ss.kv[0] : 0.0;
#pragma unroll
        for (int w = 1; w < kRbkThreads / 32; ++w) {
            ss.pcnt[w] = pc;
            ss.pflag[w] = pf;
            ss.pval[w] = pv;
            if (kComp) ss.pk[w] = pk;
            uint32_t cw = ss.cnt[w], fw = ss.flag[w];
            double vw = ss.val[w], kw = kComp ? ss.kv[w] : 0.0;
            seg_combine<kComp>(pc, pf, pv, pk, cw, fw, vw, kw);
            pc = cw;
            pf = fw;
            pv = vw;
            pk = kw;
        }
        ss.pcnt[kRbkThreads / 32] = pc;
        ss.pflag[kRbkThreads / 32] = pf;
        ss.pval[kRbkThreads / 32] = pv;
        if (kComp) ss.pk[kRbkThreads / 32] = pk;
    }
    __syncthreads();
    if (warp > 0)
        seg_combine<kComp>(ss.pcnt[warp], ss.pflag[warp], ss.pval[warp], kComp ? ss.pk[warp] : 0.0, xc, xf, xv, xk);
    tc = ss.pcnt[kRbkThreads / 32];
    tf = ss.pflag[kRbkThreads / 32];
    tv = ss.pval[kRbkThreads / 32];
    tk = kComp ? ss.pk[kRbkThreads / 32] : 0.0;
}

// A tile's summary needs its head count and the sum of the terms after its
// last head (all its terms when it has none): only the thread holding the
// last head and the threads after it form and add terms.  The partial sums
// are combined in a fixed order (shuffle tree, then warps left to right).
template <bool kComp, class H, class Src>
__device__ __forceinline__ void rbk_tiles_body(const H& hd, const Src& src, int64_t n, int64_t tile,
                                               RbkSum* __restrict__ out) {
    __shared__ int s_last[kRbkThreads / 32];
    __shared__ uint32_t s_cnt[kRbkThreads / 32];
    __shared__ double s_val[kRbkThreads / 32];
    __shared__ double s_k[kRbkThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t g0 = tile * kRbkTile + (int64_t)tid * kRbkItems;
    const int nmine = (int)max((int64_t)0, min((int64_t)kRbkItems, n - g0));
    const uint32_t heads = rbk_heads(hd, n, g0, nmine);
    // last thread with a head (-1: none) and the head count
    const int wl = __reduce_max_sync(0xffffffffu, heads ? tid : -1);
    const uint32_t wc = __reduce_add_sync(0xffffffffu, (uint32_t)__popc(heads));
    if (lane == 0) {
        s_last[warp] = wl;
        s_cnt[warp] = wc;
    }
    __syncthreads();
    int last = -1;
    uint32_t cnt = 0;
#pragma unroll
    for (int w = 0; w < kRbkThreads / 32; ++w) {
        last = max(last, s_last[w]);
        cnt += s_cnt[w];
    }
    double c = 0.0, ck = 0.0;
    if (tid >= last && nmine > 0) {
        const int start = tid == last ? 31 - __clz(heads) : 0;   // this thread's last head
        c = src.term(g0 + start);
        for (int i = start + 1; i < nmine; ++i) {
            if constexpr (kComp) nm_add(c, ck, src.term(g0 + i));
            else c = c + src.term(g0 + i);
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const double oc = __shfl_down_sync(0xffffffffu, c, off);
        if constexpr (kComp) {
            const double ok = __shfl_down_sync(0xffffffffu, ck, off);
            nm_add(c, ck, oc);
            ck = ck + ok;
        } else {
            c = c + oc;
        }
    }
    __syncthreads();
    if (lane == 0) {
        s_val[warp] = c;
        if (kComp) s_k[warp] = ck;
    }
    __syncthreads();
    if (tid == 0) {
        double v = 0.0, vk = 0.0;
        for (int w = max(last, 0) >> 5; w < kRbkThreads / 32; ++w) {
            if constexpr (kComp) {
                nm_add(v, vk, s_val[w]);
                vk = vk + s_k[w];
            } else {
                v = v + s_val[w];
            }
        }
        RbkSum t;
        t.val = v;
        t.comp = vk;
        t.cnt = cnt;
        t.flag = last >= 0;
        *out = t;
    }
}

template <bool kComp, class H, class Src>
__global__ void __launch_bounds__(kRbkThreads) k_rbk_tiles(H hd, Src src, int64_t n, RbkSum* __restrict__ tiles) {
    rbk_tiles_body<kComp>(hd, src, n, blockIdx.x, tiles + blockIdx.x);
}

// One warp per group of 32 tiles: each tile's exclusive prefix within the
// group (ingroup[t]) and the group's summary (groups[g]).
constexpr int kRbkGroup = 32;

// Group g of a problem's tiles, by one whole warp.
template <bool kComp>
__device__ __forceinline__ void rbk_group_body(const RbkSum* __restrict__ tiles, int64_t ntiles,
                                               RbkSum* __restrict__ ingroup, RbkSum* __restrict__ groups,
                                               int64_t g, int lane) {
    const int64_t t = g * kRbkGroup + lane;
    RbkSum a = t < ntiles ? tiles[t] : RbkSum{0.0, 0.0, 0u, 0u};
    uint32_t c = a.cnt, f = a.flag;
    double v = a.val, k = kComp ? a.comp : 0.0;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t c2 = __shfl_up_sync(0xffffffffu, c, off);
        const uint32_t f2 = __shfl_up_sync(0xffffffffu, f, off);
        const double v2 = __shfl_up_sync(0xffffffffu, v, off);
        const double k2 = kComp ? __shfl_up_sync(0xffffffffu, k, off) : 0.0;
        if (lane >= off) seg_combine<kComp>(c2, f2, v2, k2, c, f, v, k);
    }
    uint32_t xc = __shfl_up_sync(0xffffffffu, c, 1);
    uint32_t xf = __shfl_up_sync(0xffffffffu, f, 1);
    double xv = __shfl_up_sync(0xffffffffu, v, 1);
    double xk = kComp ? __shfl_up_sync(0xffffffffu, k, 1) : 0.0;
    if (lane == 0) { xc = 0; xf = 0; xv = 0.0; xk = 0.0; }
    if (t < ntiles) ingroup[t] = RbkSum{xv, xk, xc, xf};
    if (lane == 31) groups[g] = RbkSum{v, k, c, f};
}

template <bool kComp>
__global__ void __launch_bounds__(256) k_rbk_groups(const RbkSum* __restrict__ tiles, int64_t ntiles,
                                                    RbkSum* __restrict__ ingroup, RbkSum* __restrict__ groups,
                                                    int64_t ngroups) {
    const int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (g >= ngroups) return;
    rbk_group_body<kComp>(tiles, ntiles, ingroup, groups, g, threadIdx.x & 31);
}

// Exclusive scan of the group summaries; gprefix[g] = open value entering
// group g, gheads[g] = heads before it; the total head count is the result
// size.
// (va, ka) then (vb, kb) into b: the compensated left-to-right sum of two
// partial sums; plain addition without kComp.
template <bool kComp>
__device__ __forceinline__ void cat_sum(double va, double ka, double& vb, double& kb) {
    if constexpr (kComp) {
        double sv = va, sk = ka;
        nm_add(sv, sk, vb);
        vb = sv;
        kb = sk + kb;
    } else {
        vb = va + vb;
    }
}

template <bool kComp>
__device__ __forceinline__ void rbk_scan_body(const RbkSum* __restrict__ groups, int64_t ngroups,
                                              RbkSum* __restrict__ gprefix, unsigned long long* __restrict__ gheads,
                                              Status* st) {
    __shared__ uint32_t s_flag[kRbkScanThreads / 32];
    __shared__ double s_val[kRbkScanThreads / 32];
    __shared__ double s_k[kRbkScanThreads / 32];
    __shared__ unsigned long long s_base[kRbkScanThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t per = (ngroups + kRbkScanThreads - 1) / kRbkScanThreads;
    const int64_t lo = min(ngroups, (int64_t)tid * per), hi = min(ngroups, lo + per);
    // chunk summary, left to right (head counts in 64 bits)
    unsigned long long cc = 0;
    uint32_t cf = 0;
    double cv = 0.0, ck = 0.0;
    for (int64_t t = lo; t < hi; ++t) {
        const RbkSum a = groups[t];
        cc += a.cnt;
        if (a.flag) {
            cv = a.val;
            ck = kComp ? a.comp : 0.0;
        } else {
            double av = a.val, ak = kComp ? a.comp : 0.0;
            cat_sum<kComp>(cv, ck, av, ak);
            cv = av;
            ck = ak;
        }
        cf |= a.flag;
    }
    // exclusive scan over chunks: counts by warp sums, values by a fixed tree
    unsigned long long c = cc;
    uint32_t f = cf;
    double v = cv, k = ck;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const unsigned long long c2 = __shfl_up_sync(0xffffffffu, c, off);
        const uint32_t f2 = __shfl_up_sync(0xffffffffu, f, off);
        const double v2 = __shfl_up_sync(0xffffffffu, v, off);
        const double k2 = kComp ? __shfl_up_sync(0xffffffffu, k, off) : 0.0;
        if (lane >= off) {
            c = c2 + c;
            if (!f) cat_sum<kComp>(v2, k2, v, k);
            f = f2 | f;
        }
    }
    if (lane == 31) {
        s_base[warp] = c;
        s_flag[warp] = f;
        s_val[warp] = v;
        s_k[warp] = k;
    }
    unsigned long long xc = __shfl_up_sync(0xffffffffu, c, 1);
    uint32_t xf = __shfl_up_sync(0xffffffffu, f, 1);
    double xv = __shfl_up_sync(0xffffffffu, v, 1);
    double xk = kComp ? __shfl_up_sync(0xffffffffu, k, 1) : 0.0;
    if (lane == 0) { xc = 0; xf = 0; xv = 0.0; xk = 0.0; }
    __syncthreads();
    unsigned long long pc = 0;
    double pv = 0.0, pk = 0.0;
    for (int w = 0; w < warp; ++w) {
        pc = pc + s_base[w];
        if (s_flag[w]) {
            pv = s_val[w];
            pk = kComp ? s_k[w] : 0.0;
        } else {
            double wv = s_val[w], wk = kComp ? s_k[w] : 0.0;
            cat_sum<kComp>(pv, pk, wv, wk);
            pv = wv;
            pk = wk;
        }
    }
    // this chunk's exclusive prefix = warp prefix . lane-exclusive
    unsigned long long rc = pc + xc;
    double rv = xv, rk = xk;
    if (!xf) cat_sum<kComp>(pv, pk, rv, rk);
    for (int64_t t = lo; t < hi; ++t) {
        gprefix[t] = RbkSum{rv, rk, 0u, 0u};
        gheads[t] = rc;
        const RbkSum a = groups[t];
        rc += a.cnt;
        if (a.flag) {
            rv = a.val;
            rk = kComp ? a.comp : 0.0;
        } else {
            double av = a.val, ak = kComp ? a.comp : 0.0;
            cat_sum<kComp>(rv, rk, av, ak);
            rv = av;
            rk = ak;
        }
    }
    if (hi == ngroups && lo < hi) st->nnz_out = rc;
}

template <bool kComp>
__global__ void __launch_bounds__(kRbkScanThreads) k_rbk_scan(const RbkSum* __restrict__ groups, int64_t ngroups,
                                                              RbkSum* __restrict__ gprefix,
                                                              unsigned long long* __restrict__ gheads,
                                                              Status* st) {
    rbk_scan_body<kComp>(groups, ngroups, gprefix, gheads, st);
}

struct RbkEmitSmem {
    uint64_t row_key[kRbkTile + 1];        // closed segments of this tile, by row
    double row_val[kRbkTile + 1];
    RbkScanSmem ss;
};

// Resident CTAs per SM: 5 for prepared runs (48 registers; measured 1.26 ms
// against 1.34 at 4 on the 1e8 Zipf run), 4 for sorted pairs (their key
// comparisons spill too much at 48 registers: 1.05 against 1.04 ms).
template <class H>
constexpr int rbk_emit_ctas() { return H::kBits ? 5 : 4; }

template <bool kComp, class H, class Src>
__device__ __forceinline__ void rbk_emit_body(RbkEmitSmem& sm, const H& hd, const Src& src, int64_t n, int64_t tile,
                                              const RbkSum* __restrict__ ingroup,
                                              const RbkSum* __restrict__ gprefix,
                                              const unsigned long long* __restrict__ gheads, const StreamDesc& p,
                                              const SegOut& o, Status* st) {
    const int64_t ntiles = (n + kRbkTile - 1) / kRbkTile;
    // Sorted pairs (4 CTAs per SM, 64 registers): the tile's carries are
    // loaded first, since they do not depend on its pairs and loaded after
    // the block scan's barriers they add an L2 round trip (0.97 against
    // 1.04 ms per 1e8 pairs).  Prepared runs (5 CTAs per SM, 48 registers)
    // load them after the scan: holding them across it cost more there
    // (1.42 against 1.26 ms).
    constexpr bool kEarly = !H::kBits;
    const int64_t g = tile / kRbkGroup;
    RbkSum ig{0.0, 0.0, 0u, 0u};
    double gp_val = 0.0, gp_comp = 0.0;
    unsigned long long gh = 0;
    if constexpr (kEarly) {
        ig = ingroup[tile];
        gp_val = gprefix[g].val;
        gp_comp = kComp ? gprefix[g].comp : 0.0;
        gh = gheads[g];
    }
    RbkPairs r;
    rbk_load<kComp>(hd, src, n, tile, r);
    uint32_t xc, xf, tc, tf;
    double xv, xk, tv, tk;
    rbk_block_scan<kComp>(r, sm.ss, xc, xf, xv, xk, tc, tf, tv, tk);
    if constexpr (!kEarly) {
        ig = ingroup[tile];
        gp_val = gprefix[g].val;
        gp_comp = kComp ? gprefix[g].comp : 0.0;
        gh = gheads[g];
    }
    // open value entering the tile: group prefix . in-group prefix
    double carry = ig.val, carry_k = kComp ? ig.comp : 0.0;
    if (!ig.flag) cat_sum<kComp>(gp_val, gp_comp, carry, carry_k);
    const unsigned long long hb = gh + ig.cnt;
    // value of the run open when this thread's range starts
    double base = xv, base_k = xk;
    if (!xf) cat_sum<kComp>(carry, carry_k, base, base_k);
    // a head at tile-local head index h closes the segment at row h - first
    // of this tile (first = 1 in tile 0, whose first head closes nothing);
    // the sum of a run that starts inside this thread's range was formed by
    // rbk_load, the run open at the start adds `base` to its part here
    const int first = tile == 0 ? 1 : 0;
    int h = (int)xc;
    uint64_t prev = r.prev0;
    // the first head closes the run open at the range start: its sum is
    // base + the part formed here (one add per thread, not per head)
    const int fh = r.heads ? __ffs(r.heads) - 1 : kRbkItems;
    double closed_first = r.first_done, closed_first_k = kComp ? r.first_k : 0.0;
    cat_sum<kComp>(base, base_k, closed_first, closed_first_k);
    if (kComp) closed_first = nm_value(closed_first, closed_first_k);
#pragma unroll
    for (int i = 0; i < kRbkItems; ++i) {
        if (i < r.nmine) {
            if ((r.heads >> i) & 1u) {
                if (r.g0 + i > 0) {
                    if constexpr (!H::kBits) sm.row_key[h - first] = prev;
                    sm.row_val[h - first] = i == fh ? closed_first : r.done[i];
                }
                ++h;
            }
            prev = r.k[i];
        }
    }
    const bool last_tile = tile == ntiles - 1;
    if (r.nmine > 0 && r.g0 + r.nmine == n) {   // the last pair closes the last segment
        if constexpr (!H::kBits) sm.row_key[h - first] = prev;
        double lv = r.open, lk = kComp ? r.open_k : 0.0;
        if (!r.flag) cat_sum<kComp>(base, base_k, lv, lk);
        sm.row_val[h - first] = kComp ? nm_value(lv, lk) : lv;
    }
    __syncthreads();
    const int nrows = (int)tc - first + (last_tile ? 1 : 0);
    const int64_t row0 = (int64_t)hb - 1 + first;
    const bool even_rows = (p.nr % 2 == 0) && ((reinterpret_cast<uintptr_t>(o.subs) & 15) == 0);
    for (int q = threadIdx.x; q < nrows; q += kRbkThreads) {
        const int64_t row = row0 + q;
        uint64_t key;
        if constexpr (H::kBits) key = hd.row_keys[row];
        else key = sm.row_key[q];
        const double val = sm.row_val[q];
        if (o.row_keys) {
            o.row_keys[row] = key;   // only the run keys are wanted
        } else if (o.dense) {
            o.vals[(int64_t)key] = val;
        } else if (row < o.cap_rows) {
            int64_t* dst = o.subs + row * p.nr;
            if (even_rows) {
                // 16-byte stores: the row starts on a 16-byte boundary
                // delinearise with every index known at compile time, so
                // that the subscripts stay in registers
                int64_t sub[kMaxD];
                uint64_t kk = key;
#pragma unroll
                for (int j = kMaxD - 1; j >= 0; --j) {
                    sub[j] = 0;
                    if (j < p.nr) {
                        const uint64_t nj = (uint64_t)p.rshape[j];
                        const uint64_t q = udiv_invariant(kk, p.rmagic[j], p.rsh[j]);
                        sub[j] = (int64_t)(kk - q * nj);
                        kk = q;
                    }
                }
#pragma unroll
                for (int j = 0; j < kMaxD; j += 2)
                    if (j < p.nr) reinterpret_cast<longlong2*>(dst)[j / 2] = make_longlong2(sub[j], sub[j + 1]);
            } else {
                delinearise(p, key, dst);
            }
            o.vals[row] = val;
        } else {
            set_error(st, kErrCapacity);
        }
    }
}

template <bool kComp, class H, class Src>
__global__ void __launch_bounds__(kRbkThreads, rbk_emit_ctas<H>()) k_rbk_emit(H hd, Src src, int64_t n,
                                                             const RbkSum* __restrict__ ingroup,
                                                             const RbkSum* __restrict__ gprefix,
                                                             const unsigned long long* __restrict__ gheads,
                                                             StreamDesc p, SegOut o, Status* st) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    RbkEmitSmem& sm = *reinterpret_cast<RbkEmitSmem*>(smem_raw);
    rbk_emit_body<kComp>(sm, hd, src, n, (int64_t)blockIdx.x, ingroup, gprefix, gheads, p, o, st);
}

size_t rbk_state_bytes(int64_t n) {
    const int64_t ntiles = (std::max<int64_t>(n, 1) + kRbkTile - 1) / kRbkTile;
    const int64_t ngroups = (ntiles + kRbkGroup - 1) / kRbkGroup;
    return (size_t)ntiles * 2 * sizeof(RbkSum) +
           (size_t)ngroups * (2 * sizeof(RbkSum) + sizeof(unsigned long long)) + 512;
}

template <bool kComp, class H, class Src>
static void rbk_launch(const H& hd, const Src& src, int64_t n, void* state, const StreamDesc& p, const SegOut& o,
                       Status* st, cudaStream_t stream) {
    if (n <= 0) return;
    const int64_t ntiles = (n + kRbkTile - 1) / kRbkTile;
    const int64_t ngroups = (ntiles + kRbkGroup - 1) / kRbkGroup;
    RbkSum* tiles = static_cast<RbkSum*>(state);
    RbkSum* ingroup = tiles + ntiles;
    RbkSum* groups = ingroup + ntiles;
    RbkSum* gprefix = groups + ngroups;
    unsigned long long* gheads = reinterpret_cast<unsigned long long*>(gprefix + ngroups);
    const size_t smem = sizeof(RbkEmitSmem);
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_rbk_emit<kComp, H, Src>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(k_rbk_emit<kComp, H, Src>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
        attr_set = true;
    }
    TTV_LAUNCH("rbk_tiles", stream,
               k_rbk_tiles<kComp, H, Src><<<(unsigned)ntiles, kRbkThreads, 0, stream>>>(hd, src, n, tiles));
    TTV_LAUNCH("rbk_groups", stream,
               k_rbk_groups<kComp><<<(unsigned)((ngroups * 32 + 255) / 256), 256, 0, stream>>>(tiles, ntiles, ingroup,
                                                                                             groups, ngroups));
    TTV_LAUNCH("rbk_scan", stream,
               k_rbk_scan<kComp><<<1, kRbkScanThreads, 0, stream>>>(groups, ngroups, gprefix, gheads, st));
    TTV_LAUNCH("rbk_emit", stream,
               k_rbk_emit<kComp, H, Src><<<(unsigned)ntiles, kRbkThreads, smem, stream>>>(hd, src, n, ingroup,
                                                                                           gprefix, gheads, p, o, st));
}

void launch_reduce_by_key(const uint64_t* keys, const double* vals, int64_t n, void* state, const StreamDesc& p,
                          const SegOut& o, Status* st, cudaStream_t stream) {
    if (o.compensated) rbk_launch<true>(KeyHeads{keys}, PairTerms{vals}, n, state, p, o, st, stream);
    else rbk_launch<false>(KeyHeads{keys}, PairTerms{vals}, n, state, p, o, st, stream);
}

// The key of every run of a sorted key array, by run index (vals: any n
// doubles; their sums are not written).
void launch_run_keys(const uint64_t* keys, const double* vals, int64_t n, void* state, uint64_t* row_keys,
                     int64_t cap_rows, const StreamDesc& p, Status* st, cudaStream_t stream) {
    SegOut o{nullptr, nullptr, cap_rows, 0, 0};
    o.row_keys = row_keys;
    rbk_launch<false>(KeyHeads{keys}, PairTerms{vals}, n, state, p, o, st, stream);
}

void launch_reduce_by_key_prepared(const uint8_t* head_bits, const uint64_t* row_keys, const PrepTerms& terms,
                                   int64_t n, void* state, const StreamDesc& p, const SegOut& o, Status* st,
                                   cudaStream_t stream) {
    // o.compensated: the run sums carry a Neumaier error term through every
    // stage (thread, tile, group, scan) and are rounded once when written
    if (o.compensated) rbk_launch<true>(BitHeads{head_bits, row_keys}, PrepTermsDev{terms}, n, state, p, o, st, stream);
    else rbk_launch<false>(BitHeads{head_bits, row_keys}, PrepTermsDev{terms}, n, state, p, o, st, stream);
}


// ---- the reduce-by-key stages over a batch ---------------------------------
struct RbkState {
    RbkSum* tiles;
    RbkSum* ingroup;
    RbkSum* groups;
    RbkSum* gprefix;
    unsigned long long* gheads;
    int64_t ntiles, ngroups;
};

// The layout rbk_launch uses for state of n pairs.
__host__ __device__ __forceinline__ RbkState rbk_state_of(void* state, int64_t n) {
    RbkState r;
    r.ntiles = (n + kRbkTile - 1) / kRbkTile;
    r.ngroups = (r.ntiles + kRbkGroup - 1) / kRbkGroup;
    r.tiles = static_cast<RbkSum*>(state);
    r.ingroup = r.tiles + r.ntiles;
    r.groups = r.ingroup + r.ntiles;
    r.gprefix = r.groups + r.ngroups;
    r.gheads = reinterpret_cast<unsigned long long*>(r.gprefix + r.ngroups);
    return r;
}

int64_t rbk_tiles(int64_t n) { return (std::max<int64_t>(n, 1) + kRbkTile - 1) / kRbkTile; }
int64_t rbk_groups(int64_t n) { return (rbk_tiles(n) + kRbkGroup - 1) / kRbkGroup; }

// The sorted pairs of a job: the buffer its last digit pass wrote.
__device__ __forceinline__ const uint64_t* job_keys(const BatchJob& J) { return J.keys[J.npass & 1]; }
__device__ __forceinline__ const double* job_vals(const BatchJob& J) { return J.vals[J.npass & 1]; }

template <bool kComp>
__global__ void __launch_bounds__(kRbkThreads) k_rbk_tiles_batch(const BatchJob* __restrict__ jobs, JobList l) {
    __shared__ int s_pos;
    if (threadIdx.x == 0) s_pos = job_at(l, blockIdx.x);
    __syncthreads();
    const int pos = s_pos;
    const BatchJob& J = jobs[__ldg(l.idx + pos)];
    const int64_t tile = blockIdx.x - __ldg(l.prefix + pos);
    const RbkState rs = rbk_state_of(J.rbk_state, J.p.nnz);
    rbk_tiles_body<kComp>(KeyHeads{job_keys(J)}, PairTerms{job_vals(J)}, J.p.nnz, tile, rs.tiles + tile);
}

// One warp per group; l counts groups.
template <bool kComp>
__global__ void __launch_bounds__(256) k_rbk_groups_batch(const BatchJob* __restrict__ jobs, JobList l) {
    const uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= __ldg(l.prefix + l.count)) return;
    const int pos = job_of(l.prefix, l.count, w);
    const BatchJob& J = jobs[__ldg(l.idx + pos)];
    const RbkState rs = rbk_state_of(J.rbk_state, J.p.nnz);
    rbk_group_body<kComp>(rs.tiles, rs.ntiles, rs.ingroup, rs.groups, (int64_t)(w - __ldg(l.prefix + pos)),
                          threadIdx.x & 31);
}

// One CTA per problem.
template <bool kComp>
__global__ void __launch_bounds__(kRbkScanThreads) k_rbk_scan_batch(const BatchJob* __restrict__ jobs, JobList l) {
    const BatchJob& J = jobs[__ldg(l.idx + blockIdx.x)];
    const RbkState rs = rbk_state_of(J.rbk_state, J.p.nnz);
    rbk_scan_body<kComp>(rs.groups, rs.ngroups, rs.gprefix, rs.gheads, J.p.status);
}

template <bool kComp>
__global__ void __launch_bounds__(kRbkThreads, rbk_emit_ctas<KeyHeads>()) k_rbk_emit_batch(
    const BatchJob* __restrict__ jobs, JobList l) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    RbkEmitSmem& sm = *reinterpret_cast<RbkEmitSmem*>(smem_raw);
    __shared__ int s_pos;
    if (threadIdx.x == 0) s_pos = job_at(l, blockIdx.x);
    __syncthreads();
    const int pos = s_pos;
    const BatchJob& J = jobs[__ldg(l.idx + pos)];
    const int64_t tile = blockIdx.x - __ldg(l.prefix + pos);
    const RbkState rs = rbk_state_of(J.rbk_state, J.p.nnz);
    rbk_emit_body<kComp>(sm, KeyHeads{job_keys(J)}, PairTerms{job_vals(J)}, J.p.nnz, tile, rs.ingroup, rs.gprefix,
                         rs.gheads, J.p, J.o, J.p.status);
}

template <bool kComp>
static void rbk_batch(const BatchJob* jobs, const JobList& tiles, uint32_t ntiles, const JobList& groups,
                      uint32_t ngroup_warps, cudaStream_t stream) {
    const size_t smem = sizeof(RbkEmitSmem);
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_rbk_emit_batch<kComp>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(k_rbk_emit_batch<kComp>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
        attr_set = true;
    }
    TTV_LAUNCH("rbk_tiles_batch", stream, k_rbk_tiles_batch<kComp><<<ntiles, kRbkThreads, 0, stream>>>(jobs, tiles));
    TTV_LAUNCH("rbk_groups_batch", stream,
               k_rbk_groups_batch<kComp><<<(ngroup_warps * 32 + 255) / 256, 256, 0, stream>>>(jobs, groups));
    TTV_LAUNCH("rbk_scan_batch", stream,
               k_rbk_scan_batch<kComp><<<(unsigned)tiles.count, kRbkScanThreads, 0, stream>>>(jobs, tiles));
    TTV_LAUNCH("rbk_emit_batch", stream,
               k_rbk_emit_batch<kComp><<<ntiles, kRbkThreads, smem, stream>>>(jobs, tiles));
}

// tiles counts reduce-by-key tiles, groups their groups of 32 (one warp
// each), both over the same problems in the same order.
void launch_rbk_batch(const BatchJob* jobs, const JobList& tiles, uint32_t ntiles, const JobList& groups,
                      uint32_t ngroup_warps, bool compensated, cudaStream_t stream) {
    if (tiles.count <= 0 || ntiles == 0) return;
    if (compensated) rbk_batch<true>(jobs, tiles, ntiles, groups, ngroup_warps, stream);
    else rbk_batch<false>(jobs, tiles, ntiles, groups, ngroup_warps, stream);
}

}  // namespace ttv
