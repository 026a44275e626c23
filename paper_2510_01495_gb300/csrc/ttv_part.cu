// ttv_part.cu -- the partition path for large sparse results (selected as
// TTV_PATH_BUCKET): one streaming pass that writes every (key, term) pair
// once into a key-range bucket, then one on-chip pass per bucket that sorts,
// sums and emits it in key order (paper Sec. 3.3, Eq. 3: the surviving
// subscripts grouped and their scaled values summed, pyttb's unique /
// accumarray, in ascending lexicographic order).
//
// Traffic per nonzero: the input once (8d + w bytes), the 16-byte pair
// written once and read once, the result rows once -- against six read +
// write passes over the pairs for an LSD radix sort of 47-bit keys.
//
//  1. k_part_sample   keys of S nonzeros (blocks of 32 spread evenly over the
//                     input), sorted by the onesweep sort of ttv_sort.cu.
//  2. k_part_bounds   fine key-range boundaries from the sample quantiles (a
//                     key that fills half a quantile or more gets a bucket of
//                     its own), grouped eight to a coarse bucket; the coarse
//                     buckets' region capacities from their sample counts.
//  3. k_part_scatter  persistent CTAs stream subs/vals, form the packed key
//                     and the term, find the coarse bucket (search tree in
//                     shared memory), group a tile of pairs by bucket and
//                     append them through per-bucket write-combining buffers
//                     in shared memory, so that every global write is a whole
//                     64-byte chunk; one global atomic reserves four chunks.
//  4. k_part_process  thread-block clusters of four CTAs, one coarse bucket
//                     at a time: in each of two rounds every CTA reads its
//                     quarter of the bucket (from HBM, then from L2) and sends
//                     each pair's sort word to the CTA that owns its fine
//                     bucket through distributed shared memory; each CTA
//                     radix-sorts its fine bucket on chip, sums equal keys,
//                     finds its output offset by a decoupled look-back over
//                     the fine buckets and writes its rows.
//
// Keys are bit-packed (each surviving mode in ceil(log2 size) bits, last
// mode lowest), which orders them like the row-major index and turns the
// inverse into shifts and masks.  Sums run in binary64 in the order the pairs
// reach the sort, so results are not bit-reproducible from run to run (the
// deterministic and compensated options go to the sort path).  Whenever a
// capacity estimated from the sample proves too small, an error bit is set
// and the host reruns the call on the sort path.
#include <algorithm>
#include <climits>
#include <cmath>

#include <cooperative_groups.h>

#include "ttv_internal.cuh"

namespace cg = cooperative_groups;

namespace ttv {

constexpr int kPartCmax = 2048;                 // coarse buckets (phase A bins)
constexpr int kPartFine = 8;                    // fine buckets per coarse bucket
constexpr int kPartFmax = kPartCmax * kPartFine;
constexpr int kPartTreeLevels = 11;             // 2047-node search tree over the coarse boundaries
constexpr int kPartChunk = 4;                   // pairs per 64-byte chunk
constexpr int kPartResv = 4;                    // chunks reserved per global atomic
constexpr int kPartIdxBits = 17;                // pair index within a coarse region
constexpr int64_t kPartRegionMax = 1ll << kPartIdxBits;
constexpr int kPartMaxLocalBits = 64 - kPartIdxBits;
constexpr int kPartSampleMax = 1 << 20;
constexpr int kPartMinNnz = 1 << 16;
constexpr uint64_t kPartSentinel = ~0ull;       // no packed key reaches it (keys < 2^63)

// ---- phase A geometry
constexpr int kScatThreads = 1024;
constexpr int kScatPer = 2;                     // nonzeros per thread per tile
constexpr int kScatTile = kScatThreads * kScatPer;
constexpr int kScatBinsPer = kPartCmax / kScatThreads;   // bins owned by a thread in the scans
constexpr int kScatMaxJobs = (kScatTile + (kPartChunk - 1) * kPartCmax) / kPartChunk;

// ---- phase B geometry
constexpr int kProcCluster = 8;                 // CTAs per cluster: one per fine bucket
constexpr int kProcThreads = 1024;
constexpr int kProcWarps = kProcThreads / 32;
constexpr int kProcIpt = 12;                    // sort words per thread
constexpr int kProcCap = kProcThreads * kProcIpt;   // fine-bucket capacity (words)

struct PartDesc {
    int32_t nr;
    int32_t keybits;
    int32_t mshift[kMaxD];       // packed-key shift of input mode m (-1: contracted)
    int32_t rshift[kMaxD];       // shift of surviving mode j (result order)
    uint64_t rmask[kMaxD];
    uint64_t keyend;             // largest packed key + 1
    int64_t S;                   // samples
    int32_t Q;                   // samples per quantile block
    int32_t Fq;                  // quantile blocks
    int32_t holes;               // pairs per coarse region set aside for phase A's partial chunks
    int32_t ga;                  // phase A CTAs
    int64_t region_pairs;        // pairs the region array holds
};

struct PartWs {
    SortBuffers sb;              // sample sort
    uint64_t* fine_lo;           // [kPartFmax + 1]
    uint64_t* tree;              // [1 << kPartTreeLevels] (index 0 unused)
    uint64_t* coarse_base;       // [kPartCmax + 1] region start, in chunks
    uint32_t* coarse_cap;        // [kPartCmax] region capacity, in chunks
    uint32_t* cursor;            // [kPartCmax] chunks reserved
    unsigned long long* lb;      // [kPartCmax] look-back words, one per coarse bucket
    int32_t* meta;               // [0] fine buckets (multiple of 8), [1] coarse buckets,
                                 // [2] nonzero: the streaming pass overflowed a region
    double2* region;             // (key bits, term) pairs
};

struct Carve {
    char* base;
    size_t off;
    template <typename T>
    T* take(size_t count) {
        off = (off + 255) & ~size_t(255);
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

static int64_t part_samples(int64_t nnz) {
    // at most a quarter of the nonzeros, in whole blocks of 32
    int64_t s = std::min<int64_t>(kPartSampleMax, (nnz / 4) & ~int64_t(31));
    return std::max<int64_t>(s, 32);
}

static int64_t part_region_pairs(int64_t nnz, int holes) {
    // sum of the per-bucket capacities k_part_bounds can ask for: the sample
    // estimates (nnz in total), seven standard deviations of each (at most
    // 7 nnz sqrt(C/S) by Cauchy-Schwarz), the holes, a floor and rounding
    const int64_t S = part_samples(nnz);
    const double dev = 7.0 * (double)nnz * std::sqrt((double)kPartCmax / (double)S);
    const double floor_pairs = 8.0 * (double)nnz / (double)S + 64.0;
    return (int64_t)((double)nnz + dev) + (int64_t)kPartCmax * (holes + (int64_t)floor_pairs + 2 * kPartChunk);
}

static Carve part_layout(char* base, int64_t nnz, int key_bits, PartWs& w, int holes) {
    Carve a{base, 0};
    const int64_t S = part_samples(nnz);
    // the samples are sorted on packed keys, which can be a few bits wider
    // than the row-major key space: room for the widest (eight passes)
    (void)key_bits;
    const int npass = 8;
    const int64_t ntiles = sort_tiles(S);
    w.sb.keys[0] = a.take<uint64_t>(S);
    w.sb.keys[1] = a.take<uint64_t>(S);
    w.sb.vals[0] = a.take<double>(S);
    w.sb.vals[1] = a.take<double>(S);
    w.sb.hist = a.take<uint32_t>((size_t)npass * 256);
    w.sb.lookback = a.take<uint32_t>((size_t)npass * ntiles * 256);
    w.sb.tickets = a.take<uint32_t>(64);
    w.sb.npass = npass;
    w.sb.ntiles = ntiles;
    w.fine_lo = a.take<uint64_t>(kPartFmax + 1);
    w.tree = a.take<uint64_t>(1 << kPartTreeLevels);
    w.coarse_base = a.take<uint64_t>(kPartCmax + 1);
    w.coarse_cap = a.take<uint32_t>(kPartCmax);
    w.cursor = a.take<uint32_t>(kPartCmax);
    w.lb = a.take<unsigned long long>(kPartFmax);
    w.meta = a.take<int32_t>(64);
    w.region = a.take<double2>((size_t)part_region_pairs(nnz, holes));
    a.off = (a.off + 255) & ~size_t(255);
    return a;
}

// Packed key of a nonzero's surviving subscripts; false for a subscript
// outside its mode.
template <int D>
__device__ __forceinline__ bool part_key(const StreamDesc& p, const PartDesc& q, const int64_t* s, uint64_t& key) {
    bool good = true;
    uint64_t k = 0;
#pragma unroll
    for (int m = 0; m < D; ++m) {
        good &= (uint64_t)s[m] < (uint64_t)p.shape[m];
        if (q.mshift[m] >= 0) k |= (uint64_t)s[m] << q.mshift[m];
    }
    key = k;
    return good;
}

// ---- 1. samples ----------------------------------------------------------------
// One warp per block of 32 consecutive nonzeros; blocks evenly spaced.
template <int D>
__global__ void __launch_bounds__(256) k_part_sample(StreamDesc p, PartDesc q, int64_t stride,
                                                     uint64_t* __restrict__ smp) {
    const int64_t b = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (b * 32 >= q.S) return;
    const int64_t k = b * stride + (threadIdx.x & 31);
    int64_t s[D];
#pragma unroll
    for (int m = 0; m < D; ++m) s[m] = __ldg(p.subs + k * p.snz + m * p.smode);
    uint64_t key;
    if (!part_key<D>(p, q, s, key)) key = 0;     // the streaming pass reports it
    smp[b * 32 + (threadIdx.x & 31)] = key;
}

// ---- 2. bucket boundaries ---------------------------------------------------------
constexpr int kBndThreads = 1024;

__device__ __forceinline__ int64_t lower_bound_u64(const uint64_t* a, int64_t n, uint64_t x) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (__ldg(a + mid) < x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Largest candidate boundary of quantile block j (0 if it has none).
__device__ __forceinline__ uint64_t block_last_candidate(const uint64_t* smp, const PartDesc& q, int j) {
    const int64_t S = q.S;
    const int dsp = max(1, q.Q / 4);
    uint64_t last = j >= 1 ? __ldg(smp + (int64_t)j * q.Q) : 0ull;
    const int64_t i1 = min((int64_t)(S - dsp), (int64_t)(j + 1) * q.Q);
    for (int64_t i = (int64_t)j * q.Q; i < i1; i += dsp) {
        const uint64_t v = __ldg(smp + i);
        if (v == __ldg(smp + i + dsp)) last = max(last, v + 1);
    }
    return last;
}

// Block scan helper: exclusive prefix of v over the CTA; total in *tot.
template <int T>
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* warp_sums, uint32_t* tot) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < T / 32 ? warp_sums[lane] : 0u;
        uint32_t z = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, z, o);
            if (lane >= o) z += y;
        }
        if (lane < T / 32) warp_sums[lane] = z - w;
        if (lane == T / 32 - 1) *tot = z;
    }
    __syncthreads();
    const uint32_t r = warp_sums[warp] + x - v;
    __syncthreads();
    return r;
}

// One CTA.  Fine boundaries: fine_lo[0] = 0, then in increasing order the
// first sample of every quantile block (Q samples) and, for every key that
// fills at least half a block (a run of equal samples found at the detection
// points, Q/4 apart), the pair v, v + 1 so that v gets a bucket of its own.
// Padded with zero-width buckets at keyend to a multiple of eight.
__global__ void __launch_bounds__(kBndThreads) k_part_bounds(const uint64_t* __restrict__ smp, PartDesc q,
                                                             int64_t nnz, PartWs w, Status* st) {
    __shared__ uint32_t s_warp[32];
    __shared__ uint32_t s_tot;
    __shared__ int s_bad;
    const int tid = threadIdx.x;
    const int64_t S = q.S;
    const int dsp = max(1, q.Q / 4);
    if (tid == 0) s_bad = 0;
    const int per = (q.Fq + kBndThreads - 1) / kBndThreads;
    const int j0 = min(q.Fq, tid * per), j1 = min(q.Fq, j0 + per);
    const uint64_t start_last = j0 >= 1 ? block_last_candidate(smp, q, j0 - 1) : 0ull;

    // pass 0 counts the boundaries of this thread's blocks, pass 1 writes them
    uint32_t mine = 0, base = 0;
    for (int pass = 0; pass < 2; ++pass) {
        uint64_t last = start_last;
        uint32_t n = 0;
        auto emit = [&](uint64_t x) {
            if (x > last) {
                if (pass == 1) {
                    const uint32_t at = 1 + base + n;
                    if (at < (uint32_t)kPartFmax) w.fine_lo[at] = x;
                }
                ++n;
                last = x;
            }
        };
        for (int j = j0; j < j1; ++j) {
            if (j >= 1) emit(__ldg(smp + (int64_t)j * q.Q));
            const int64_t i1 = min((int64_t)(S - dsp), (int64_t)(j + 1) * q.Q);
            for (int64_t i = (int64_t)j * q.Q; i < i1; i += dsp) {
                const uint64_t v = __ldg(smp + i);
                if (v == __ldg(smp + i + dsp)) {
                    emit(v);
                    emit(v + 1);
                }
            }
        }
        if (pass == 0) {
            mine = n;
            base = block_excl_scan<kBndThreads>(mine, s_warp, &s_tot);
        }
    }
    __syncthreads();
    const uint32_t nf = 1 + s_tot;                  // fine buckets before padding
    const uint32_t fpad = (nf + kPartFine - 1) / kPartFine * kPartFine;
    if (fpad > (uint32_t)kPartFmax) {
        if (tid == 0) {
            set_error(st, kErrRetry);
            w.meta[0] = 0;
            w.meta[1] = 0;
        }
        return;
    }
    if (tid == 0) w.fine_lo[0] = 0;
    for (uint32_t f = nf + tid; f <= fpad; f += kBndThreads) w.fine_lo[f] = q.keyend;
    __syncthreads();
    const int C = (int)(fpad / kPartFine);
    // local keys and region indices share one 64-bit sort word
    for (uint32_t f = tid; f < nf; f += kBndThreads)
        if (w.fine_lo[f + 1] - w.fine_lo[f] > (1ull << kPartMaxLocalBits)) s_bad = 1;
    // region capacity of each coarse bucket from its sample count
    const double scale = (double)nnz / (double)S;
    uint32_t capc[kScatBinsPer];
    uint32_t sum = 0;
#pragma unroll
    for (int r = 0; r < kScatBinsPer; ++r) {
        const int c = tid * kScatBinsPer + r;
        uint32_t cap = 0;
        if (c < C) {
            const uint64_t lo = w.fine_lo[c * kPartFine], hi = w.fine_lo[c * kPartFine + kPartFine];
            if (hi > lo) {
                const int64_t cnt = lower_bound_u64(smp, S, hi) - lower_bound_u64(smp, S, lo);
                const double est = (double)cnt * scale;
                const double pairs = est + 7.0 * est / sqrt((double)(cnt > 1 ? cnt : 1)) + 8.0 * scale + 64.0 +
                                     (double)q.holes;
                const double chunks = ceil(pairs / kPartChunk);
                if (chunks * kPartChunk >= (double)kPartRegionMax) s_bad = 1;
                cap = (uint32_t)min(chunks, (double)(kPartRegionMax / kPartChunk - 1));
            }
        }
        capc[r] = cap;
        sum += cap;
    }
    const uint32_t off = block_excl_scan<kBndThreads>(sum, s_warp, &s_tot);
    uint32_t run = off;
#pragma unroll
    for (int r = 0; r < kScatBinsPer; ++r) {
        const int c = tid * kScatBinsPer + r;
        if (c < C) {
            w.coarse_base[c] = run;
            w.coarse_cap[c] = capc[r];
        }
        run += capc[r];
    }
    if (tid == 0) {
        w.coarse_base[C] = s_tot;
        if ((int64_t)s_tot * kPartChunk > q.region_pairs) s_bad = 1;
    }
    // search tree over the coarse boundaries fine_lo[8], fine_lo[16], ...
    for (int i = 1 + tid; i < (1 << kPartTreeLevels); i += kBndThreads) {
        const int dep = 31 - __clz(i);
        const int o = i - (1 << dep);
        const int pos = ((2 * o + 1) << (kPartTreeLevels - 1 - dep)) - 1;
        w.tree[i] = pos < C - 1 ? w.fine_lo[(pos + 1) * kPartFine] : kPartSentinel;
    }
    __syncthreads();
    if (tid == 0) {
        w.meta[0] = s_bad ? 0 : (int32_t)fpad;
        w.meta[1] = s_bad ? 0 : C;
        if (s_bad) set_error(st, kErrRetry);
    }
}

// ---- 3. the streaming partition pass ------------------------------------------------
struct ScatSmem {
    uint64_t tree[1 << kPartTreeLevels];
    double2 left[kPartCmax][kPartChunk - 1];     // pairs waiting for a whole chunk
    double2 stage[kScatTile];                    // this tile's pairs grouped by bucket
    uint32_t hist[kPartCmax];                    // counts, then group starts in stage
    uint32_t rpos[kPartCmax];                    // next reserved chunk (absolute)
    uint32_t job_dest[kScatMaxJobs];             // chunk written by a job
    uint32_t job_src[kScatMaxJobs];              // bucket << 10 | chunk of its sequence
    uint8_t lcnt[kPartCmax];                     // pairs in left[b]
    uint8_t rleft[kPartCmax];                    // reserved chunks not yet written
    uint32_t warp[32];
    uint32_t tot;
};

template <int D, bool kSoA>
struct ScatRaw {
    longlong2 s[kSoA ? D : 1];
    longlong2 a[kSoA ? 1 : D];
    double2 v;
};

template <int D, bool kSoA>
__device__ __forceinline__ void scat_load(const StreamDesc& p, int64_t k0, ScatRaw<D, kSoA>& r) {
    if (k0 + 1 < p.nnz) {
        if constexpr (kSoA) {
#pragma unroll
            for (int m = 0; m < D; ++m) r.s[m] = __ldcs(reinterpret_cast<const longlong2*>(p.subs + m * p.smode + k0));
        } else {
            const longlong2* row = reinterpret_cast<const longlong2*>(p.subs + k0 * D);
#pragma unroll
            for (int j = 0; j < D; ++j) r.a[j] = __ldcs(row + j);
        }
        if (p.val_f32) {
            const float2 f = __ldcs(reinterpret_cast<const float2*>(static_cast<const float*>(p.vals) + k0));
            r.v = make_double2((double)f.x, (double)f.y);
        } else {
            r.v = __ldcs(reinterpret_cast<const double2*>(static_cast<const double*>(p.vals) + k0));
        }
    } else if (k0 < p.nnz) {
        // the odd last nonzero
        if constexpr (kSoA) {
#pragma unroll
            for (int m = 0; m < D; ++m) r.s[m] = make_longlong2(p.subs[m * p.smode + k0], 0);
        } else {
#pragma unroll
            for (int j = 0; j < D; ++j) {
                const int e0 = 2 * j, e1 = 2 * j + 1;
                r.a[j] = make_longlong2(e0 < D ? p.subs[k0 * D + e0] : 0, e1 < D ? p.subs[k0 * D + e1] : 0);
            }
        }
        r.v = make_double2(p.val_f32 ? (double)static_cast<const float*>(p.vals)[k0]
                                     : static_cast<const double*>(p.vals)[k0], 0.0);
    }
}

template <int D>
__device__ __forceinline__ double part_term(const StreamDesc& p, const int64_t* s, double val) {
    double t = val;
#pragma unroll
    for (int m = 0; m < D; ++m)
        if ((p.smask >> m) & 1u)
            t = t * (p.vec_f32 ? (double)__ldg(static_cast<const float*>(p.vec[m]) + s[m])
                               : __ldg(static_cast<const double*>(p.vec[m]) + s[m]));
    return t;
}

// Coarse bucket of a key: the number of coarse boundaries <= key, by the
// Eytzinger tree (top five levels from registers via shuffles).
__device__ __forceinline__ uint32_t scat_bin(const uint64_t* tree, uint64_t top, uint64_t key) {
    uint32_t i = 1;
#pragma unroll
    for (int l = 0; l < 5; ++l) {
        const uint64_t t = __shfl_sync(0xffffffffu, top, (int)i - 1);
        i = 2 * i + (t <= key ? 1u : 0u);
    }
#pragma unroll
    for (int l = 5; l < kPartTreeLevels; ++l) i = 2 * i + (tree[i] <= key ? 1u : 0u);
    return i - (1u << kPartTreeLevels);
}

template <int D, bool kSoA>
__global__ void __launch_bounds__(kScatThreads, 1) k_part_scatter(StreamDesc p, PartDesc q, PartWs w) {
    extern __shared__ __align__(16) unsigned char scat_raw[];
    ScatSmem& sm = *reinterpret_cast<ScatSmem*>(scat_raw);
    const int tid = threadIdx.x;
    const int C = w.meta[1];
    if (C == 0) return;                       // the boundaries failed: the call reruns on the sort path
    for (int i = tid; i < (1 << kPartTreeLevels); i += kScatThreads) sm.tree[i] = w.tree[i];
    for (int b = tid; b < kPartCmax; b += kScatThreads) {
        sm.hist[b] = 0;
        sm.lcnt[b] = 0;
        sm.rleft[b] = 0;
        sm.rpos[b] = 0;
    }
    __syncthreads();
    const uint64_t top = sm.tree[(tid & 31) + 1];
    const int64_t ntiles = (p.nnz + kScatTile - 1) / kScatTile;

    int64_t tile = blockIdx.x;
    ScatRaw<D, kSoA> raw;
    if (tile < ntiles) scat_load<D, kSoA>(p, tile * kScatTile + 2 * tid, raw);
    while (tile < ntiles) {
        const int64_t k0 = tile * kScatTile + 2 * tid;
        // ---- keys, terms, buckets of this thread's two nonzeros
        uint64_t key[2];
        double term[2];
        uint32_t bin[2], rank[2];
        bool ok[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            int64_t s[D];
            if constexpr (kSoA) {
#pragma unroll
                for (int m = 0; m < D; ++m) s[m] = u ? raw.s[m].y : raw.s[m].x;
            } else {
#pragma unroll
                for (int m = 0; m < D; ++m) {
                    const int e = u * D + m;
                    s[m] = (e & 1) ? raw.a[e >> 1].y : raw.a[e >> 1].x;
                }
            }
            const bool present = k0 + u < p.nnz;
            uint64_t kk = 0;
            const bool good = part_key<D>(p, q, s, kk);
            if (present && !good) set_error(p.status, kErrSubscript);
            ok[u] = present && good;
            key[u] = ok[u] ? kk : 0ull;
            term[u] = ok[u] ? part_term<D>(p, s, u ? raw.v.y : raw.v.x) : 0.0;
            bin[u] = scat_bin(sm.tree, top, key[u]);
        }
        const int64_t next = tile + gridDim.x;
        if (next < ntiles) scat_load<D, kSoA>(p, next * kScatTile + 2 * tid, raw);   // in flight meanwhile
#pragma unroll
        for (int u = 0; u < 2; ++u) rank[u] = ok[u] ? atomicAdd(&sm.hist[bin[u]], 1u) : 0u;
        __syncthreads();

        // ---- per bucket: group starts, whole chunks, reservations, jobs
        uint32_t cnt[kScatBinsPer], tot[kScatBinsPer], nch[kScatBinsPer], at[kScatBinsPer];
        uint32_t packed = 0;
#pragma unroll
        for (int r = 0; r < kScatBinsPer; ++r) {
            const int b = tid * kScatBinsPer + r;
            cnt[r] = sm.hist[b];
            tot[r] = sm.lcnt[b] + cnt[r];
            nch[r] = tot[r] / kPartChunk;
            packed += (cnt[r] << 16) | nch[r];
            // reserve chunks now; the reply is first needed after the scan
            const uint32_t rl = sm.rleft[b];
            at[r] = nch[r] > rl ? atomicAdd(&w.cursor[b], max(nch[r] - rl, (uint32_t)kPartResv)) : 0u;
        }
        const uint32_t excl = block_excl_scan<kScatThreads>(packed, sm.warp, &sm.tot);
        const uint32_t njobs = sm.tot & 0xFFFFu;
        uint32_t sstart = excl >> 16, jstart = excl & 0xFFFFu;
#pragma unroll
        for (int r = 0; r < kScatBinsPer; ++r) {
            const int b = tid * kScatBinsPer + r;
            sm.hist[b] = sstart;
            uint32_t k = nch[r];
            const uint32_t at_r = at[r];
            if (k) {
                const uint32_t rl = sm.rleft[b], rp = sm.rpos[b];
                uint32_t fresh = 0, got = 0;
                if (k > rl) {
                    got = max(k - rl, (uint32_t)kPartResv);
                    const uint32_t at = at_r;
                    if (at + got > w.coarse_cap[b]) {
                        set_error(p.status, kErrRetry);      // region too small: the call reruns
                        atomicOr(&w.meta[2], 1);
                        k = 0;
                        nch[r] = 0;
                        got = 0;
                    }
                    fresh = (uint32_t)w.coarse_base[b] + at;
                }
                for (uint32_t i = 0; i < k; ++i) {
                    sm.job_dest[jstart + i] = i < rl ? rp + i : fresh + (i - rl);
                    sm.job_src[jstart + i] = ((uint32_t)b << 10) | i;
                }
                if (k > rl) {
                    sm.rpos[b] = fresh + (k - rl);
                    sm.rleft[b] = (uint8_t)(got - (k - rl));
                } else if (k) {
                    sm.rpos[b] = rp + k;
                    sm.rleft[b] = (uint8_t)(rl - k);
                }
                // jobs of a bucket whose region overflowed stay unwritten
                for (uint32_t i = k; i < (tot[r] / kPartChunk); ++i) sm.job_src[jstart + i] = 0xFFFFFFFFu;
            }
            sstart += cnt[r];
            jstart += tot[r] / kPartChunk;
        }
        __syncthreads();
        // ---- group the tile's pairs by bucket
#pragma unroll
        for (int u = 0; u < 2; ++u)
            if (ok[u]) sm.stage[sm.hist[bin[u]] + rank[u]] = make_double2(__longlong_as_double((long long)key[u]), term[u]);
        __syncthreads();
        // ---- whole chunks: four lanes per chunk, one 64-byte store group
        for (uint32_t j = tid >> 2; j < njobs; j += kScatThreads / 4) {
            const uint32_t src = sm.job_src[j];
            if (src == 0xFFFFFFFFu) continue;
            const uint32_t b = src >> 10, e = (src & 1023u) * kPartChunk + (tid & 3);
            const uint32_t l = sm.lcnt[b];
            const double2 x = e < l ? sm.left[b][e] : sm.stage[sm.hist[b] + e - l];
            w.region[(size_t)sm.job_dest[j] * kPartChunk + (tid & 3)] = x;
        }
        __syncthreads();
        // ---- what is left waits for the next tile
#pragma unroll
        for (int r = 0; r < kScatBinsPer; ++r) {
            const int b = tid * kScatBinsPer + r;
            const uint32_t l = sm.lcnt[b], t = tot[r], k = t / kPartChunk;
            if (nch[r] == 0 && k > 0) {
                sm.lcnt[b] = 0;          // overflowed bucket: its pairs are dropped (the call reruns)
            } else {
                for (uint32_t e = k * kPartChunk; e < t; ++e)
                    if (e >= l || k > 0) sm.left[b][e - k * kPartChunk] = e < l ? sm.left[b][e] : sm.stage[sm.hist[b] + e - l];
                sm.lcnt[b] = (uint8_t)(t - k * kPartChunk);
            }
            sm.hist[b] = 0;
        }
        __syncthreads();
        tile = next;
    }

    // ---- close every bucket: the waiting pairs, padded with sentinels, and
    // every reserved chunk not yet written become whole chunks
    const double2 pad = make_double2(__longlong_as_double((long long)kPartSentinel), 0.0);
#pragma unroll
    for (int r = 0; r < kScatBinsPer; ++r) {
        const int b = tid * kScatBinsPer + r;
        if (b >= C) continue;
        uint32_t l = sm.lcnt[b], rl = sm.rleft[b], rp = sm.rpos[b];
        if (l) {
            if (rl == 0) {
                const uint32_t at = atomicAdd(&w.cursor[b], 1u);
                if (at + 1 > w.coarse_cap[b]) {
                    set_error(p.status, kErrRetry);
                    atomicOr(&w.meta[2], 1);
                    continue;
                }
                rp = (uint32_t)w.coarse_base[b] + at;
                rl = 1;
            }
            for (int e = 0; e < kPartChunk; ++e) w.region[(size_t)rp * kPartChunk + e] = e < (int)l ? sm.left[b][e] : pad;
            ++rp;
            --rl;
        }
        for (; rl > 0; --rl, ++rp)
            for (int e = 0; e < kPartChunk; ++e) w.region[(size_t)rp * kPartChunk + e] = pad;
    }
}

// ---- 4. per coarse bucket: exchange, sort, sum, emit ------------------------------
__device__ __forceinline__ unsigned long long part_ld_relaxed(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void part_st_relaxed(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint32_t part_lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

constexpr unsigned long long kLbAggFlag = 1ull << 62;
constexpr unsigned long long kLbIncFlag = 2ull << 62;
constexpr unsigned long long kLbValue = (1ull << 62) - 1;
constexpr int kHistPad = 264;                   // 256 digits, one for absent items, padding

struct ProcSmem {
    uint64_t words[kProcCap];                   // sort words (local key << kPartIdxBits | region index)
    double terms[kProcCap];                     // their terms, in sorted order
    uint16_t whist[kProcWarps][kHistPad];       // per-warp digit counts, then offsets
    uint32_t dstart[256];
    uint32_t cnt[kProcCluster][kProcCluster];   // [source][target] sort words sent
    uint32_t scnt[kProcCluster][kProcCluster];  // [source][target] pairs of single-key targets
    double psum[kProcCluster];                  // [source] partial sum of this CTA's single key
    double ssum[kProcCluster];                  // this source's single-key sums, per target
    uint32_t sfill[kProcCluster];               // this source's single-key pairs, per target
    uint32_t fill[kProcCluster];                // this source's sort-word slots used, per target
    uint32_t off[kProcCluster];                 // this source's first slot in each target
    uint64_t flo[kPartFine + 1];                // fine boundaries of the coarse bucket
    uint32_t red[kProcWarps][kProcCluster];
    uint32_t wend[kProcWarps], whead[kProcWarps], wrow[kProcWarps], warp_u[kProcWarps];
    double wtail[kProcWarps], wcarry[kProcWarps];
    uint64_t wmin[kProcWarps], wmax[kProcWarps];
    uint32_t cU[kProcCluster];                  // rows of each fine bucket of the coarse bucket
    uint32_t n, nsing, ovf, tot_u;
    double sval;
    uint64_t kmin, kspan, bcast;
    int32_t rsh[kMaxD];                         // result field shifts and masks
    uint64_t rmk[kMaxD];
};

// Inclusive sum of a count over the CTA; total in sm.tot_u.
__device__ __forceinline__ uint32_t proc_count_scan(ProcSmem& sm, uint32_t x) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sm.warp_u[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const uint32_t w0 = lane < kProcWarps ? sm.warp_u[lane] : 0u;
        uint32_t z = w0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, z, o);
            if (lane >= o) z += y;
        }
        if (lane < kProcWarps) sm.warp_u[lane] = z - w0;
        if (lane == kProcWarps - 1) sm.tot_u = z;
    }
    __syncthreads();
    const uint32_t r = sm.warp_u[warp] + x;
    __syncthreads();
    return r;
}

// Stable LSD radix sort of words[0, n) by local key, over the bits of
// (key - smallest key) only, eight bits per pass.
__device__ void proc_sort(ProcSmem& sm, uint32_t n) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint64_t mn = ~0ull, mx = 0;
    for (uint32_t pos = tid; pos < n; pos += kProcThreads) {
        const uint64_t k = sm.words[pos] >> kPartIdxBits;
        mn = k < mn ? k : mn;
        mx = k > mx ? k : mx;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const uint64_t a = __shfl_xor_sync(0xffffffffu, mn, o), b = __shfl_xor_sync(0xffffffffu, mx, o);
        mn = a < mn ? a : mn;
        mx = b > mx ? b : mx;
    }
    if (lane == 0) {
        sm.wmin[warp] = mn;
        sm.wmax[warp] = mx;
    }
    __syncthreads();
    if (tid == 0) {
        uint64_t a = ~0ull, b = 0;
        for (int w2 = 0; w2 < kProcWarps; ++w2) {
            a = sm.wmin[w2] < a ? sm.wmin[w2] : a;
            b = sm.wmax[w2] > b ? sm.wmax[w2] : b;
        }
        sm.kmin = a;
        sm.kspan = b - a;
    }
    __syncthreads();
    const uint64_t kmin = sm.kmin, span = sm.kspan;
    const int rb = span ? 64 - __clzll((long long)span) : 0;
    const int passes = (rb + 7) / 8;
    if (passes == 0) return;          // one key: already in order
    const uint32_t lt = part_lanemask_lt();
    const int ipt = (int)((n + kProcThreads - 1) / kProcThreads);
    const uint32_t wbase = (uint32_t)(warp * 32 * ipt) + lane;
    uint64_t x[kProcIpt];
    uint32_t rk[kProcIpt];
#pragma unroll
    for (int i = 0; i < kProcIpt; ++i) {
        const uint32_t pos = wbase + 32u * i;
        x[i] = (i < ipt && pos < n) ? sm.words[pos] : 0ull;
    }
    for (int pass = 0; pass < passes; ++pass) {
        const int shift = 8 * pass;
        for (int j = lane; j < kHistPad; j += 32) sm.whist[warp][j] = 0;
        __syncwarp();
#pragma unroll
        for (int i = 0; i < kProcIpt; ++i) {
            if (i < ipt) {       // uniform over the CTA
                const uint32_t pos = wbase + 32u * i;
                const uint32_t dig =
                    pos < n ? (uint32_t)((((x[i] >> kPartIdxBits) - kmin) >> shift) & 255u) : 256u;
                const uint32_t mask = __match_any_sync(0xffffffffu, dig);
                const int leader = __ffs(mask) - 1;
                uint32_t b = 0;
                if (lane == leader) {
                    b = sm.whist[warp][dig];
                    sm.whist[warp][dig] = (uint16_t)(b + __popc(mask));
                }
                b = __shfl_sync(0xffffffffu, b, leader);
                rk[i] = b + __popc(mask & lt);
                __syncwarp();
            }
        }
        __syncthreads();
        uint32_t dt = 0;
        if (tid < 256) {
            for (int w2 = 0; w2 < kProcWarps; ++w2) {
                const uint32_t c2 = sm.whist[w2][tid];
                sm.whist[w2][tid] = (uint16_t)dt;
                dt += c2;
            }
        }
        const uint32_t incl = proc_count_scan(sm, tid < 256 ? dt : 0u);
        if (tid < 256) sm.dstart[tid] = incl - dt;
        __syncthreads();
#pragma unroll
        for (int i = 0; i < kProcIpt; ++i) {
            const uint32_t pos = wbase + 32u * i;
            if (i < ipt && pos < n) {
                const uint32_t dig = (uint32_t)((((x[i] >> kPartIdxBits) - kmin) >> shift) & 255u);
                sm.words[sm.dstart[dig] + sm.whist[warp][dig] + rk[i]] = x[i];
            }
        }
        __syncthreads();
        if (pass + 1 < passes) {
#pragma unroll
            for (int i = 0; i < kProcIpt; ++i) {
                const uint32_t pos = wbase + 32u * i;
                x[i] = (i < ipt && pos < n) ? sm.words[pos] : 0ull;
            }
        }
    }
}

// Walk positions in the warp-contiguous order w*32*ipt + 32*i + lane.
// Gather pass: each sorted word's term from the coarse region (L2), the
// warp's rows (segment ends) and heads, and the sum of its items after its
// last head (the open segment carried into the next warp).
__device__ void proc_gather(ProcSmem& sm, uint32_t n, int ipt, const double2* __restrict__ region) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t imask = (1ull << kPartIdxBits) - 1;
    const uint32_t base = (uint32_t)(warp * 32 * ipt);
    double run = 0.0;
    uint32_t ne = 0, nh = 0;
    for (int i = 0; i < ipt; ++i) {
        const uint32_t pos = base + 32u * i + lane;
        const bool valid = pos < n;
        double t = 0.0;
        bool head = false, end = false;
        if (valid) {
            const uint64_t w = sm.words[pos];
            const uint64_t key = w >> kPartIdxBits;
            t = __ldg(&region[w & imask].y);
            sm.terms[pos] = t;
            head = pos == 0 || (sm.words[pos - 1] >> kPartIdxBits) != key;
            end = pos + 1 == n || (sm.words[pos + 1] >> kPartIdxBits) != key;
        }
        const uint32_t hb = __ballot_sync(0xffffffffu, head);
        if (hb) {
            const int hl = 31 - __clz(hb);
            run = lane >= hl ? t : 0.0;
        } else {
            run += t;
        }
        ne += __popc(__ballot_sync(0xffffffffu, end));
        nh += __popc(hb);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) run += __shfl_xor_sync(0xffffffffu, run, o);
    if (lane == 0) {
        sm.wend[warp] = ne;
        sm.whead[warp] = nh;
        sm.wtail[warp] = run;
    }
}

// Emit walk over the same positions: warp-wide segmented sums; the rows that
// end in a step are compacted into the warp's staging slots and written as one
// contiguous block of subscripts and one of values.
struct RowStage {
    uint64_t key[32];
    double val[32];
};

__device__ void proc_emit(const ProcSmem& sm, RowStage& stg, uint32_t n, int ipt, double carry, int64_t row0,
                          uint64_t flo_g, int nr, int64_t* __restrict__ out_subs, double* __restrict__ out_vals,
                          int64_t cap_rows) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt = part_lanemask_lt();
    const uint32_t base = (uint32_t)(warp * 32 * ipt);
    const int per = 32 / nr;                 // rows per store instruction
    const int lrow = lane / nr, lfld = lane - lrow * nr;
    double csum = carry;
    int64_t row = row0;
    for (int i = 0; i < ipt; ++i) {
        const uint32_t pos = base + 32u * i + lane;
        const bool valid = pos < n;
        uint64_t key = 0;
        double t = 0.0;
        bool head = false, end = false;
        if (valid) {
            key = sm.words[pos] >> kPartIdxBits;
            t = sm.terms[pos];
            head = pos == 0 || (sm.words[pos - 1] >> kPartIdxBits) != key;
            end = pos + 1 == n || (sm.words[pos + 1] >> kPartIdxBits) != key;
        }
        uint32_t f = head ? 1u : 0u;
        double v = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t f2 = __shfl_up_sync(0xffffffffu, f, o);
            const double v2 = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) {
                if (!f) v = v2 + v;
                f |= f2;
            }
        }
        const double sv = f ? v : csum + v;
        const uint32_t eb = __ballot_sync(0xffffffffu, end);
        const int nrows = __popc(eb);
        if (end) {
            const int k = __popc(eb & lt);
            stg.key[k] = flo_g + key;
            stg.val[k] = sv;
        }
        __syncwarp();
        const int64_t avail = cap_rows - row;
        const int nw = (int)(avail < nrows ? (avail > 0 ? avail : 0) : nrows);
        for (int r0 = 0; r0 < nw; r0 += per) {
            const int r = r0 + lrow;
            if (lrow < per && r < nw) {
                const uint64_t full = stg.key[r];
                out_subs[(row + r) * nr + lfld] = (int64_t)((full >> sm.rsh[lfld]) & sm.rmk[lfld]);
            }
        }
        if (lane < nw) out_vals[row + lane] = stg.val[lane];
        __syncwarp();
        row += nrows;
        csum = __shfl_sync(0xffffffffu, sv, 31);
    }
}

// Fine bucket (within the coarse bucket) of a key: boundaries flo[1..7] <= key.
__device__ __forceinline__ int proc_fine(const uint64_t* flo, uint64_t key) {
    int g = 0;
#pragma unroll
    for (int j = 1; j < kPartFine; ++j) g += key >= flo[j] ? 1 : 0;
    return g;
}

__global__ void __cluster_dims__(kProcCluster, 1, 1) __launch_bounds__(kProcThreads, 1)
    k_part_process(PartDesc q, PartWs w, Status* st, int64_t* __restrict__ out_subs, double* __restrict__ out_vals,
                   int64_t cap_rows) {
    extern __shared__ __align__(16) unsigned char proc_raw[];
    ProcSmem& sm = *reinterpret_cast<ProcSmem*>(proc_raw);
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lt = part_lanemask_lt();
    // written before this kernel, so every CTA of a cluster takes the same branch
    const int C = w.meta[1];
    if (C == 0 || w.meta[2] != 0) return;
    const int ncl = (int)(gridDim.x / kProcCluster), cid = (int)(blockIdx.x / kProcCluster);
    if (tid < kMaxD) {
        sm.rsh[tid] = q.rshift[tid];
        sm.rmk[tid] = q.rmask[tid];
    }

    for (int c = cid; c < C; c += ncl) {
        if (tid <= kPartFine) sm.flo[tid] = w.fine_lo[(int64_t)c * kPartFine + tid];
        if (tid < kProcCluster) {
            sm.ssum[tid] = 0.0;
            sm.sfill[tid] = 0;
            sm.fill[tid] = 0;
        }
        const uint32_t nch = min(w.cursor[c], w.coarse_cap[c]);
        const double2* reg = w.region + (int64_t)w.coarse_base[c] * kPartChunk;
        const uint32_t np = nch * kPartChunk;
        const uint32_t lo = (uint32_t)((uint64_t)np * rank / kProcCluster);
        const uint32_t hi = (uint32_t)((uint64_t)np * (rank + 1) / kProcCluster);
        __syncthreads();
        uint64_t flo[kPartFine + 1];
#pragma unroll
        for (int j = 0; j <= kPartFine; ++j) flo[j] = sm.flo[j];
        uint32_t single = 0;          // bit g: fine bucket g holds one key
#pragma unroll
        for (int j = 0; j < kPartFine; ++j) single |= (flo[j + 1] - flo[j] == 1 ? 1u : 0u) << j;

        // ---- pass 1: what this CTA's share sends to each fine bucket's CTA
        uint64_t pk = 0;              // eight 8-bit counts (at most ~20 pairs per thread)
        for (uint32_t i0 = lo + tid; i0 < hi; i0 += 8 * kProcThreads) {
            double2 pr[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const uint32_t i = i0 + k * kProcThreads;
                pr[k] = i < hi ? reg[i] : make_double2(__longlong_as_double((long long)kPartSentinel), 0.0);
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const uint64_t key = (uint64_t)__double_as_longlong(pr[k].x);
                if (key == kPartSentinel) continue;
                const int g = proc_fine(flo, key);
                if ((single >> g) & 1u) {
                    atomicAdd(&sm.ssum[g], pr[k].y);
                    atomicAdd(&sm.sfill[g], 1u);
                } else {
                    pk += 1ull << (8 * g);
                }
            }
        }
        uint32_t u[kProcCluster];
#pragma unroll
        for (int t = 0; t < kProcCluster; ++t) {
            uint32_t v = (uint32_t)(pk >> (8 * t)) & 255u;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            u[t] = v;
        }
        if (lane == 0)
#pragma unroll
            for (int t = 0; t < kProcCluster; ++t) sm.red[warp][t] = u[t];
        __syncthreads();
        if (tid < kProcCluster) {
            uint32_t s = 0;
            for (int w2 = 0; w2 < kProcWarps; ++w2) s += sm.red[w2][tid];
            // to every CTA of the cluster: this source's count for target tid
            for (int x2 = 0; x2 < kProcCluster; ++x2) {
                ProcSmem* peer = cl.map_shared_rank(&sm, x2);
                peer->cnt[rank][tid] = s;
                peer->scnt[rank][tid] = sm.sfill[tid];
            }
            cl.map_shared_rank(&sm, tid)->psum[rank] = sm.ssum[tid];
        }
        cl.sync();
        if (tid == 0) {
            uint32_t ovf = 0;
            for (int t = 0; t < kProcCluster; ++t) {
                uint32_t s = 0;
                for (int src = 0; src < kProcCluster; ++src) {
                    if (src == rank) sm.off[t] = s;
                    s += sm.cnt[src][t];
                }
                ovf |= s > (uint32_t)kProcCap ? 1u : 0u;
                if (t == rank) sm.n = s;
            }
            uint32_t ns = 0;
            double sv = 0.0;
            for (int src = 0; src < kProcCluster; ++src) {
                ns += sm.scnt[src][rank];
                sv += sm.psum[src];
            }
            sm.ovf = ovf;
            sm.nsing = ns;
            sm.sval = sv;
        }
        __syncthreads();
        const bool overflow = sm.ovf != 0;
        const uint32_t n = sm.n;
        // ---- pass 2: sort words to their fine bucket's CTA
        if (!overflow) {
            for (uint32_t i0 = lo + (tid & ~31u); i0 < hi; i0 += kProcThreads) {
                const uint32_t i = i0 + lane;
                uint64_t key = kPartSentinel;
                if (i < hi) key = (uint64_t)__double_as_longlong(reg[i].x);
                int g = kPartFine;
                if (key != kPartSentinel) {
                    g = proc_fine(flo, key);
                    if ((single >> g) & 1u) g = kPartFine;
                }
                const uint32_t mask = __match_any_sync(0xffffffffu, (uint32_t)g);
                const int leader = __ffs(mask) - 1;
                uint32_t b = 0;
                if (lane == leader && g < kPartFine) b = atomicAdd(&sm.fill[g], (uint32_t)__popc(mask));
                b = __shfl_sync(0xffffffffu, b, leader);
                if (g < kPartFine) {
                    uint64_t* dst = cl.map_shared_rank(sm.words, g);
                    dst[sm.off[g] + b + __popc(mask & lt)] = ((key - sm.flo[g]) << kPartIdxBits) | (uint64_t)i;
                }
            }
        }
        cl.sync();

        // ---- this CTA's fine bucket (fine bucket `rank` of the coarse bucket)
        const uint64_t flo_g = sm.flo[rank], width = sm.flo[rank + 1] - flo_g;
        const int ipt = (int)((n + kProcThreads - 1) / kProcThreads);
        const bool sorted = !overflow && width > 1 && n > 0;
        uint32_t U = 0;
        if (overflow) {
            if (tid == 0) set_error(st, kErrRetry);
        } else if (width == 1) {
            U = sm.nsing > 0 ? 1u : 0u;
        } else if (sorted) {
            proc_sort(sm, n);
            proc_gather(sm, n, ipt, reg);
            __syncthreads();
            if (tid == 0) {
                // rows before each warp, and the open segment's sum entering it
                uint32_t rows = 0;
                double run = 0.0;
                for (int w2 = 0; w2 < kProcWarps; ++w2) {
                    sm.wrow[w2] = rows;
                    sm.wcarry[w2] = run;
                    rows += sm.wend[w2];
                    run = sm.whead[w2] ? sm.wtail[w2] : run + sm.wtail[w2];
                }
                sm.tot_u = rows;
            }
            __syncthreads();
            U = sm.tot_u;
        }
        // ---- output offset: the cluster's eight counts through distributed
        // shared memory, then a warp-wide decoupled look-back over the coarse
        // buckets (32 predecessors per round trip)
        if (tid == 0)
            for (int x2 = 0; x2 < kProcCluster; ++x2) cl.map_shared_rank(&sm, x2)->cU[rank] = U;
        cl.sync();
        if (tid < 32) {
            uint32_t pre = 0, uc = 0;
#pragma unroll
            for (int x2 = 0; x2 < kProcCluster; ++x2) {
                const uint32_t v2 = sm.cU[x2];
                if (x2 < rank) pre += v2;
                uc += v2;
            }
            if (rank == 0 && lane == 0) part_st_relaxed(&w.lb[c], (c == 0 ? kLbIncFlag : kLbAggFlag) | uc);
            unsigned long long excl = 0;
            const uint32_t polls = wait_limit(1u << 24);
            for (int64_t j = (int64_t)c - 1; j >= 0; j -= 32) {
                const int64_t idx = j - lane;
                unsigned long long v = 0;
                uint32_t first = 32, it = 0;
                bool timed_out = false;
                for (;;) {
                    v = idx >= 0 ? part_ld_relaxed(&w.lb[idx]) : kLbIncFlag;
                    const uint32_t fl = (uint32_t)(v >> 62);
                    const uint32_t inc = __ballot_sync(0xffffffffu, fl == 2u);
                    first = inc ? (uint32_t)(__ffs(inc) - 1) : 32u;
                    const uint32_t upto = first >= 31 ? 0xffffffffu : ((2u << first) - 1u);
                    if (!(__ballot_sync(0xffffffffu, fl == 0u) & upto)) break;
                    if (++it >= polls) { timed_out = true; break; }
                    if (it > 16) __nanosleep(32);
                }
                if (timed_out) {
                    if (lane == 0) set_error(st, kErrTimeout);
                    break;
                }
                unsigned long long part = ((uint32_t)lane <= first) ? (v & kLbValue) : 0ull;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
                excl += part;
                if (first < 32) break;
            }
            if (lane == 0) {
                if (rank == 0 && c > 0) part_st_relaxed(&w.lb[c], kLbIncFlag | ((excl + uc) & kLbValue));
                if (rank == 0 && c == C - 1) *reinterpret_cast<volatile unsigned long long*>(&st->nnz_out) = excl + uc;
                excl += pre;
                sm.bcast = excl;
                if (excl + U > (unsigned long long)cap_rows) set_error(st, kErrCapacity);
                if (width == 1 && U && (int64_t)excl < cap_rows) {
                    for (int j = 0; j < q.nr; ++j)
                        out_subs[(int64_t)excl * q.nr + j] = (int64_t)((flo_g >> sm.rsh[j]) & sm.rmk[j]);
                    out_vals[excl] = sm.sval;
                }
            }
        }
        __syncthreads();
        if (sorted) {
            // the digit histograms are free now: 512 bytes of row staging per warp
            RowStage* stg = reinterpret_cast<RowStage*>(&sm.whist[0][0]);
            proc_emit(sm, stg[warp], n, ipt, sm.wcarry[warp], (int64_t)sm.bcast + sm.wrow[warp], flo_g, q.nr,
                      out_subs, out_vals, cap_rows);
        }
        __syncthreads();
    }
}

// ---- host side ------------------------------------------------------------------
typedef void (*SampleKernel)(StreamDesc, PartDesc, int64_t, uint64_t*);
typedef void (*ScatKernel)(StreamDesc, PartDesc, PartWs);

template <int D>
static ScatKernel scat_pick(bool soa) {
    return soa ? k_part_scatter<D, true> : k_part_scatter<D, false>;
}

static SampleKernel sample_kernel(int d) {
    switch (d) {
        case 2: return k_part_sample<2>;
        case 3: return k_part_sample<3>;
        case 4: return k_part_sample<4>;
        case 5: return k_part_sample<5>;
        case 6: return k_part_sample<6>;
        case 7: return k_part_sample<7>;
        case 8: return k_part_sample<8>;
        default: return nullptr;
    }
}

static ScatKernel scat_kernel(int d, bool soa) {
    switch (d) {
        case 2: return scat_pick<2>(soa);
        case 3: return scat_pick<3>(soa);
        case 4: return scat_pick<4>(soa);
        case 5: return scat_pick<5>(soa);
        case 6: return scat_pick<6>(soa);
        case 7: return scat_pick<7>(soa);
        case 8: return scat_pick<8>(soa);
        default: return nullptr;
    }
}

static int part_key_bits(const StreamDesc& p) {
    int bits = 0;
    for (int j = 0; j < p.nr; ++j) {
        const uint64_t n = (uint64_t)p.rshape[j];
        bits += n > 1 ? 64 - __builtin_clzll(n - 1) : 0;
    }
    return bits;
}

static int part_ga(int64_t nnz) {
    const int64_t ntiles = (nnz + kScatTile - 1) / kScatTile;
    return (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, num_sms()));
}

static int part_holes(int64_t nnz) { return part_ga(nnz) * (kPartResv + 1) * kPartChunk; }

bool bucket_applicable(const StreamDesc& p) {
    if (p.d < 2 || p.d > 8 || p.nr < 1) return false;
    if (p.nnz < kPartMinNnz || p.nnz > (1ll << 30)) return false;
    if (part_key_bits(p) > 63) return false;
    const uintptr_t sb = reinterpret_cast<uintptr_t>(p.subs), vb = reinterpret_cast<uintptr_t>(p.vals);
    if ((sb & 15) || (vb & 15)) return false;
    const bool soa = p.snz == 1 && (p.smode % 2 == 0);
    const bool aos = p.snz == p.d && p.smode == 1;
    return soa || aos;
}

size_t bucket_workspace_bytes(int64_t nnz, int key_bits) {
    PartWs w;
    return part_layout(nullptr, std::max<int64_t>(nnz, 1), std::max(key_bits, 1), w, part_holes(nnz)).off;
}

static int part_clusters() {
    static int ncl = 0;
    if (ncl) return ncl;
    cudaFuncSetAttribute(k_part_process, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(ProcSmem));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kProcCluster * 64);
    cfg.blockDim = dim3(kProcThreads);
    cfg.dynamicSmemBytes = sizeof(ProcSmem);
    cudaLaunchAttribute a;
    a.id = cudaLaunchAttributeClusterDimension;
    a.val.clusterDim.x = kProcCluster;
    a.val.clusterDim.y = 1;
    a.val.clusterDim.z = 1;
    cfg.attrs = &a;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_part_process, &cfg) != cudaSuccess || n < 1) {
        cudaGetLastError();
        n = 1;
    }
    ncl = n;
    return ncl;
}

void launch_bucket(const StreamDesc& p, int key_bits, void* ws, int64_t* out_subs, double* out_vals,
                   int64_t cap_rows, cudaStream_t stream) {
    (void)key_bits;
    PartDesc q;
    memset(&q, 0, sizeof q);
    q.nr = p.nr;
    int shift = 0;
    for (int j = p.nr - 1; j >= 0; --j) {
        const uint64_t n = (uint64_t)p.rshape[j];
        const int b = n > 1 ? 64 - __builtin_clzll(n - 1) : 0;
        q.rshift[j] = shift;
        q.rmask[j] = b ? ((1ull << b) - 1) : 0ull;
        q.keyend += (n - 1) << shift;
        shift += b;
    }
    q.keyend += 1;
    q.keybits = shift;
    for (int m = 0; m < kMaxD; ++m) q.mshift[m] = -1;
    for (int j = 0; j < p.nr; ++j) q.mshift[p.rmode[j]] = q.rshift[j];
    const int64_t nnz = p.nnz;
    q.S = part_samples(nnz);
    const int64_t ftarget = std::max<int64_t>(8, std::min<int64_t>(nnz / 6000, kPartFmax * 7 / 8));
    q.Q = (int32_t)std::max<int64_t>(8, q.S / ftarget);
    q.Fq = (int32_t)((q.S + q.Q - 1) / q.Q);
    q.ga = part_ga(nnz);
    q.holes = part_holes(nnz);
    q.region_pairs = part_region_pairs(nnz, q.holes);

    PartWs w;
    part_layout(static_cast<char*>(ws), nnz, std::max(q.keybits, 1), w, q.holes);
    cudaMemsetAsync(w.cursor, 0, kPartCmax * sizeof(uint32_t), stream);
    cudaMemsetAsync(w.lb, 0, kPartFmax * sizeof(unsigned long long), stream);
    cudaMemsetAsync(w.meta, 0, 64 * sizeof(int32_t), stream);

    // 1. samples, sorted
    const int64_t nblk = q.S / 32;
    const int64_t stride = nnz / nblk;
    TTV_LAUNCH("part_sample", stream,
               sample_kernel(p.d)<<<(unsigned)((nblk + 7) / 8), 256, 0, stream>>>(p, q, stride, w.sb.keys[0]));
    const int cur = radix_sort_pairs(w.sb, q.S, q.keybits, p.status, stream, nullptr, false);
    // 2. boundaries and region capacities
    TTV_LAUNCH("part_bounds", stream, k_part_bounds<<<1, kBndThreads, 0, stream>>>(w.sb.keys[cur], q, nnz, w, p.status));
    // 3. the streaming partition
    ScatKernel sk = scat_kernel(p.d, p.snz == 1);
    cudaFuncSetAttribute(sk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(ScatSmem));
    TTV_LAUNCH("part_scatter", stream, sk<<<q.ga, kScatThreads, sizeof(ScatSmem), stream>>>(p, q, w));
    // 4. per coarse bucket: exchange, sort, sum, emit (every cluster resident at once)
    const int ncl = part_clusters();
    TTV_LAUNCH("part_process", stream,
               k_part_process<<<(unsigned)(ncl * kProcCluster), kProcThreads, sizeof(ProcSmem), stream>>>(
                   q, w, p.status, out_subs, out_vals, cap_rows));
}

}  // namespace ttv
