// ttv_hash.cu -- accumulation through a table in HBM (the hash path).
//
// The sort path moves every (key, term) pair through every digit pass.  When
// many nonzeros share a surviving tuple, or the key space is not much larger
// than nnz, it is cheaper to combine the terms first and order only the
// distinct keys.  One streaming pass computes (key, term) exactly like the
// sort path (paper Sec. 3.3, Eq. 3: the term is vals[k] times the gathered
// vector entries in increasing mode order, the key the row-major index of the
// surviving subscripts), combines equal keys inside each warp
// (__match_any_sync, summed by the lowest lane in lane order), and adds the
// warp's sum into a table entry with a binary64 atomic in L2:
//
//   direct  (key space <= 4 x the table bound): entry = key; a presence bitmap
//           marks the keys that occur, so compaction in slot order is already
//           ascending key order and no sort is needed;
//   hashed  (larger key spaces): open addressing with linear probing over
//           2^b 16-byte (key, sum) slots, b chosen for a load factor <= 0.8 at
//           the worst case (every nonzero its own key); compaction writes the
//           distinct (key, sum) pairs, which the onesweep sort then orders.
//
// A direct table is compacted in key order: presence bits counted per
// 4096-entry tile, one scan into row offsets, one gather.  A hashed table is
// compacted in any order (each CTA reserves its range from a counter) and
// sorted.  The distinct-key count stays on the device: the sort and the emit
// read it there, so the call never waits on the host.
//
// Sums are formed in atomic arrival order, so the hash path is not
// deterministic run to run (the sort path is); the planner sends
// deterministic and compensated requests to the sort path.
#include <algorithm>

#include "ttv_internal.cuh"

namespace ttv {

constexpr unsigned long long kHashEmpty = ~0ull;   // keys are < nkeys <= 2^64 - 1
constexpr int kHashThreads = 256;
// nonzeros per thread per iteration of the insert: 2 (default: measured
// faster than 4 on every class tried, the insert being bound by L2 atomics
// rather than by loads in flight) or 4, picked per problem class by the
// autotuner
constexpr int kHashTileShift = 12;                 // entries per count tile: 4096
constexpr int kHashTile = 1 << kHashTileShift;
constexpr int kHashItems = kHashTile / kHashThreads;

struct __align__(16) HashSlot {
    unsigned long long key;
    double val;
};

struct HashPlan {
    int direct;          // 1: entry index = key
    int log2cap;         // hashed table: 2^log2cap slots
    int64_t entries;     // direct: nkeys rounded up to a tile; hashed: 2^log2cap
    int64_t ntiles;
    int64_t bound;       // distinct keys can not exceed this: min(nnz, nkeys)
};

HashPlan plan_hash(const StreamDesc& p) {
    HashPlan h{};
    h.bound = (int64_t)std::min<uint64_t>((uint64_t)std::max<int64_t>(p.nnz, 1), p.nkeys);
    // 1.25 x bound, rounded up to a power of two (load factor <= 0.8)
    int b = kHashTileShift;
    while (b < 40 && ((int64_t)1 << b) < h.bound + h.bound / 4) ++b;
    h.log2cap = b;
    const int64_t cap = (int64_t)1 << b;
    h.direct = p.nkeys <= (uint64_t)cap * 4;
    h.entries = h.direct ? (int64_t)((p.nkeys + kHashTile - 1) / kHashTile) * kHashTile : cap;
    h.ntiles = h.entries / kHashTile;
    return h;
}

bool hash_applicable(const StreamDesc& p) {
    return plan_hash(p).log2cap < 40;
}

bool hash_direct(const StreamDesc& p) {
    return plan_hash(p).direct != 0;
}

// Workspace: table, presence bitmap (direct), tile counts and offsets, and
// for the hashed table the two pair buffers of the sort.
struct HashWs {
    HashSlot* slots;
    double* dvals;
    uint32_t* bits;
    uint32_t* tile_count;
    unsigned long long* tile_off;
    SortBuffers sb;
};

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

size_t hash_workspace_bytes(const StreamDesc& p, int dense_out, int key_bits) {
    const HashPlan h = plan_hash(p);
    size_t b = 0;
    if (h.direct) {
        b += align256((size_t)h.entries * sizeof(double));
        b += align256((size_t)h.entries / 32 * sizeof(uint32_t));
    } else {
        b += align256((size_t)h.entries * sizeof(HashSlot));
    }
    b += align256((size_t)h.ntiles * sizeof(uint32_t));
    b += align256((size_t)(h.ntiles + 1) * sizeof(unsigned long long));
    if (!h.direct && !dense_out) b += sort_workspace_bytes(h.bound, key_bits) + 4 * 256;
    return b;
}

static HashWs carve(const StreamDesc& p, const HashPlan& h, int dense_out, int key_bits, void* ws) {
    HashWs w{};
    char* c = static_cast<char*>(ws);
    auto take = [&](size_t bytes) {
        char* r = c;
        c += align256(bytes);
        return r;
    };
    if (h.direct) {
        w.dvals = reinterpret_cast<double*>(take((size_t)h.entries * sizeof(double)));
        w.bits = reinterpret_cast<uint32_t*>(take((size_t)h.entries / 32 * sizeof(uint32_t)));
    } else {
        w.slots = reinterpret_cast<HashSlot*>(take((size_t)h.entries * sizeof(HashSlot)));
    }
    w.tile_count = reinterpret_cast<uint32_t*>(take((size_t)h.ntiles * sizeof(uint32_t)));
    w.tile_off = reinterpret_cast<unsigned long long*>(take((size_t)(h.ntiles + 1) * sizeof(unsigned long long)));
    if (!h.direct && !dense_out) {
        const int npass = key_bits <= 0 ? 0 : (key_bits + 7) / 8;
        const int64_t n = h.bound;
        const int64_t ntiles = sort_tiles(n);
        w.sb.keys[0] = reinterpret_cast<uint64_t*>(take((size_t)n * 8));
        w.sb.keys[1] = reinterpret_cast<uint64_t*>(take((size_t)n * 8));
        w.sb.vals[0] = reinterpret_cast<double*>(take((size_t)n * 8));
        w.sb.vals[1] = reinterpret_cast<double*>(take((size_t)n * 8));
        w.sb.hist = reinterpret_cast<uint32_t*>(take((size_t)std::max(npass, 1) * 256 * 4));
        w.sb.lookback = reinterpret_cast<uint32_t*>(take((size_t)std::max(npass, 1) * ntiles * 256 * 4));
        w.sb.tickets = reinterpret_cast<uint32_t*>(take(64 * 4));
        w.sb.npass = npass;
        w.sb.ntiles = ntiles;
    }
    return w;
}

__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kHashThreads) k_hash_init(HashSlot* __restrict__ slots, int64_t n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        HashSlot s;
        s.key = kHashEmpty;
        s.val = 0.0;
        slots[i] = s;
    }
}

// Hashed table: continues a linear probe after the first slot h0 held
// another key.  Bounded by the table size; running past it (impossible at a
// load factor <= 0.8) flags an internal error.
__device__ __noinline__ void hash_probe_on(uint64_t key, double t, uint64_t h0, HashSlot* slots, int log2cap,
                                           Status* st) {
    const uint64_t mask = ((uint64_t)1 << log2cap) - 1;
    uint64_t h = (h0 + 1) & mask;
    for (uint64_t it = 1; it <= mask; ++it) {
        HashSlot* s = slots + h;
        const unsigned long long cur = atomicCAS(&s->key, kHashEmpty, (unsigned long long)key);
        if (cur == kHashEmpty || cur == key) {
            atomicAdd(&s->val, t);
            return;
        }
        h = (h + 1) & mask;
    }
    set_error(st, kErrInternal);
}

// Streaming pass: (key, term) per nonzero, warp-combined, added to the table.
// With dense_out and a direct table the table is the caller's result array.
//
// Each thread holds kHashUnroll nonzeros; their first atomics (compare-and-
// swap of the home slot) are issued back to back so that kHashUnroll L2/DRAM
// round trips are in flight per thread, and only the rare second probe runs
// one at a time.  L2 atomics are the limit of this kernel (about 3e10 64-bit
// atomics per second measured on GB300), so an insert costs the fewest
// possible: direct = presence OR (skipped when the bit reads set) + binary64
// add; hashed = compare-and-swap + binary64 add.  Entries are counted
// afterwards, not here.
template <bool kDirect, int kHashUnroll>
__global__ void __launch_bounds__(kHashThreads) k_hash_insert(StreamDesc p, HashSlot* slots, double* dvals,
                                                              uint32_t* bits, int log2cap, uint32_t* tile_count) {
    extern __shared__ double sv[];
    __shared__ double s_t[kHashThreads];   // terms of lanes that share a key
    stage_vectors(p, sv);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    double* wt = s_t + (threadIdx.x & ~31);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // Warp-uniform loop: every lane runs every iteration so the warp
    // intrinsics below see the full warp.
    const int64_t warp_base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31);
    for (int64_t w0 = warp_base; w0 < p.nnz; w0 += stride * kHashUnroll) {
        int64_t ks[kHashUnroll];
        bool ok[kHashUnroll];
#pragma unroll
        for (int u = 0; u < kHashUnroll; ++u) {
            ks[u] = w0 + u * stride + lane;
            ok[u] = ks[u] < p.nnz;
        }
        Batch<kHashUnroll> b;
        load_batch<kHashUnroll>(p, ks, ok, b);
        uint64_t key[kHashUnroll];
        double t[kHashUnroll];
        bool ins[kHashUnroll];
#pragma unroll
        for (int u = 0; u < kHashUnroll; ++u) {
            key[u] = kHashEmpty;
            t[u] = 0.0;
            bool valid = ok[u];
            if (valid && !key_term(p, sv, b.s[u], b.v[u], key[u], t[u])) {
                set_error(p.status, kErrSubscript);
                valid = false;
            }
            if (!valid) key[u] = kHashEmpty;
            const uint32_t peers = __match_any_sync(0xffffffffu, key[u]);
            const int leader = __ffs(peers) - 1;
            if (__any_sync(0xffffffffu, valid && peers != (1u << lane))) {
                // lanes with equal keys: the lowest lane adds the others in lane order
                wt[lane] = t[u];
                __syncwarp();
                if (valid && lane == leader) {
                    for (uint32_t m = peers & (peers - 1); m; m &= m - 1) t[u] += wt[__ffs(m) - 1];
                }
                __syncwarp();
            }
            ins[u] = valid && lane == leader;
        }
        if constexpr (kDirect) {
#pragma unroll
            for (int u = 0; u < kHashUnroll; ++u) {
                if (!ins[u]) continue;
                uint32_t* w = bits + (key[u] >> 5);
                const uint32_t bit = 1u << (key[u] & 31);
                if (!(ld_relaxed_u32(w) & bit)) atomicOr(w, bit);
                atomicAdd(dvals + key[u], t[u]);
            }
        } else {
            uint64_t h[kHashUnroll];
            unsigned long long cur[kHashUnroll];
#pragma unroll
            for (int u = 0; u < kHashUnroll; ++u) {
                h[u] = (key[u] * 0x9E3779B97F4A7C15ull) >> (64 - log2cap);
                cur[u] = ins[u] ? atomicCAS(&slots[h[u]].key, kHashEmpty, (unsigned long long)key[u]) : 0ull;
            }
#pragma unroll
            for (int u = 0; u < kHashUnroll; ++u) {
                if (!ins[u]) continue;
                if (cur[u] == kHashEmpty) atomicAdd(tile_count + (h[u] >> kHashTileShift), 1u);
                if (cur[u] == kHashEmpty || cur[u] == key[u])
                    atomicAdd(&slots[h[u]].val, t[u]);
                else
                    hash_probe_on(key[u], t[u], h[u], slots, log2cap, p.status);
            }
        }
    }
}

// Direct table: entries present per 4096-entry tile, one warp per tile
// (128 presence words, popc).
__global__ void __launch_bounds__(256) k_hash_count_bits(const uint32_t* __restrict__ bits, int64_t ntiles,
                                                         uint32_t* __restrict__ tile_count) {
    const int lane = threadIdx.x & 31;
    const int64_t tile = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (tile >= ntiles) return;
    const uint4 w = reinterpret_cast<const uint4*>(bits + tile * (kHashTile / 32))[lane];
    uint32_t c = __popc(w.x) + __popc(w.y) + __popc(w.z) + __popc(w.w);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) tile_count[tile] = c;
}

// One CTA: exclusive scan of the tile counts into offsets; total = distinct
// keys (status nnz_out).  A sparse result larger than cap_rows flags
// kErrCapacity (the gather then writes only rows below the capacity).
__global__ void __launch_bounds__(1024) k_hash_scan(const uint32_t* __restrict__ tile_count, int64_t ntiles,
                                                    unsigned long long* __restrict__ tile_off, int64_t cap_rows,
                                                    int check_cap, Status* st) {
    __shared__ unsigned long long warp_tot[32];
    __shared__ unsigned long long carry;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < ntiles; base += 1024) {
        const int64_t i = base + tid;
        const unsigned long long x = i < ntiles ? tile_count[i] : 0ull;
        unsigned long long inc = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) warp_tot[warp] = inc;
        __syncthreads();
        unsigned long long before = 0, all = 0;
        for (int w = 0; w < 32; ++w) {
            const unsigned long long tw = warp_tot[w];
            if (w < warp) before += tw;
            all += tw;
        }
        const unsigned long long c = carry;
        if (i < ntiles) tile_off[i] = c + before + inc - x;
        __syncthreads();
        if (tid == 0) carry = c + all;
        __syncthreads();
    }
    if (tid == 0) {
        tile_off[ntiles] = carry;
        st->nnz_out = carry;
        if (check_cap && (long long)carry > cap_rows) set_error(st, kErrCapacity);
    }
}

// Compaction of one 4096-entry tile per CTA: entry tile*4096 + i*256 + tid is
// thread tid's i-th item, so (i, warp, lane) order is entry order.  Direct
// tables (tile_off from the scan) write result rows in key order, or dense
// cells; hashed tables write dense cells, or (key, sum) pairs for the sort at
// a range the CTA reserves from the distinct-key counter (order is restored
// by the sort, so no scan is needed).
struct GatherOut {
    int mode;                // 0: result rows; 1: dense cells; 2: pairs for the sort
    int64_t* subs;
    double* vals;
    uint64_t* pkeys;
    double* pvals;
    int64_t cap_rows;
};

template <bool kDirect>
__global__ void __launch_bounds__(kHashThreads) k_hash_gather(const HashSlot* __restrict__ slots,
                                                              const double* __restrict__ dvals,
                                                              const uint32_t* __restrict__ bits,
                                                              const unsigned long long* __restrict__ tile_off,
                                                              StreamDesc p, GatherOut o, Status* st) {
    __shared__ uint32_t wcnt[kHashItems][kHashThreads / 32];
    __shared__ uint32_t woff[kHashItems][kHashThreads / 32];
    __shared__ unsigned long long s_t0;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t tile = blockIdx.x;
    const int64_t base = tile * kHashTile;
    uint32_t occ[kHashItems];
    uint64_t key[kHashItems];
    double val[kHashItems];
#pragma unroll
    for (int i = 0; i < kHashItems; ++i) {
        const int64_t e = base + i * kHashThreads + tid;
        if constexpr (kDirect) {
            const uint32_t word = bits[e >> 5];   // one word per warp: the warp's 32 entries
            occ[i] = word;
            key[i] = (uint64_t)e;
            val[i] = ((word >> lane) & 1u) ? dvals[e] : 0.0;
        } else {
            const HashSlot s = slots[e];
            occ[i] = __ballot_sync(0xffffffffu, s.key != kHashEmpty);
            key[i] = s.key;
            val[i] = s.val;
        }
        if (lane == 0) wcnt[i][warp] = __popc(occ[i]);
    }
    __syncthreads();
    if (tid < 32) {
        // exclusive scan over the 128 (i, warp) counts in (i, warp) order
        uint32_t run = 0;
        const int per = kHashItems * (kHashThreads / 32) / 32;   // 4 counts per lane
        uint32_t c[per];
        uint32_t mine = 0;
#pragma unroll
        for (int q = 0; q < per; ++q) {
            const int idx = lane * per + q;
            c[q] = wcnt[idx / (kHashThreads / 32)][idx % (kHashThreads / 32)];
            mine += c[q];
        }
        uint32_t inc = mine;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, off);
            if (lane >= off) inc += y;
        }
        run = inc - mine;
#pragma unroll
        for (int q = 0; q < per; ++q) {
            const int idx = lane * per + q;
            woff[idx / (kHashThreads / 32)][idx % (kHashThreads / 32)] = run;
            run += c[q];
        }
        if (lane == 31) {
            // run = tile total
            if (tile_off) s_t0 = tile_off[tile];
            else s_t0 = (o.mode == 2 && run) ? atomicAdd(&st->nnz_out, (unsigned long long)run) : 0ull;
        }
    }
    __syncthreads();
    const unsigned long long t0 = s_t0;
    const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
    for (int i = 0; i < kHashItems; ++i) {
        if (!((occ[i] >> lane) & 1u)) continue;
        const int64_t r = (int64_t)(t0 + woff[i][warp] + __popc(occ[i] & lt));
        if (o.mode == 1) {
            o.vals[key[i]] = val[i];
        } else if (o.mode == 2) {
            o.pkeys[r] = key[i];
            o.pvals[r] = val[i];
        } else if (r < o.cap_rows) {
            if (p.nr > 0) delinearise(p, key[i], o.subs + r * p.nr);
            o.vals[r] = val[i];
        }
    }
}

// Sorted distinct pairs -> result rows.
__global__ void __launch_bounds__(256) k_hash_emit(const uint64_t* __restrict__ keys, const double* __restrict__ vals,
                                                   StreamDesc p, int64_t* __restrict__ out_subs,
                                                   double* __restrict__ out_vals, int64_t cap_rows,
                                                   Status* st) {
    const int64_t n = (int64_t)*(const volatile unsigned long long*)&st->nnz_out;
    const int64_t lim = std::min(n, cap_rows);
    if (n > cap_rows && blockIdx.x == 0 && threadIdx.x == 0) set_error(st, kErrCapacity);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < lim; j += stride) {
        delinearise(p, keys[j], out_subs + j * p.nr);
        out_vals[j] = vals[j];
    }
}

// ---------------------------------------------------------------------------
void launch_hash(const StreamDesc& p, int dense_out, int key_bits, void* ws, int64_t* out_subs, double* out_vals,
                 int64_t cap_rows, cudaStream_t stream) {
    if (p.nnz <= 0) return;
    const HashPlan h = plan_hash(p);
    HashWs w = carve(p, h, dense_out, key_bits, ws);
    const int nsm = num_sms();

    // table initialisation
    cudaMemsetAsync(w.tile_count, 0, (size_t)h.ntiles * sizeof(uint32_t), stream);
    double* acc = w.dvals;
    if (h.direct) {
        // dense result on a direct table: accumulate into the result itself
        if (dense_out) acc = out_vals;
        cudaMemsetAsync(acc, 0, (size_t)(dense_out ? p.nkeys : h.entries) * sizeof(double), stream);
        cudaMemsetAsync(w.bits, 0, (size_t)h.entries / 32 * sizeof(uint32_t), stream);
    } else {
        const int g = (int)std::min<int64_t>((int64_t)nsm * 8, (h.entries + kHashThreads - 1) / kHashThreads);
        TTV_LAUNCH("hash_init", stream, k_hash_init<<<g, kHashThreads, 0, stream>>>(w.slots, h.entries));
        if (dense_out) cudaMemsetAsync(out_vals, 0, (size_t)p.nkeys * sizeof(double), stream);
    }

    // insert
    const size_t smem = p.vec_smem ? (size_t)p.vtotal * sizeof(double) : 0;
    const int unroll = p.items == 4 ? 4 : 2;
    auto kins = h.direct ? (unroll == 2 ? k_hash_insert<true, 2> : k_hash_insert<true, 4>)
                         : (unroll == 2 ? k_hash_insert<false, 2> : k_hash_insert<false, 4>);
    smem_at_least(kins, smem);
    const int64_t want = (p.nnz + kHashThreads * unroll - 1) / (kHashThreads * unroll);
    const int per_sm = p.ctas_per_sm > 0 ? p.ctas_per_sm : 8;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)nsm * per_sm));
    TTV_LAUNCH("hash_insert", stream, kins<<<grid, kHashThreads, smem, stream>>>(p, w.slots, acc, w.bits, h.log2cap, w.tile_count));
    if (h.direct && dense_out) return;   // the dense result is complete

    if (h.direct) {
        // presence counts per tile -> row offsets in key order
        TTV_LAUNCH("hash_count", stream,
                   k_hash_count_bits<<<(unsigned)((h.ntiles * 32 + 255) / 256), 256, 0, stream>>>(w.bits, h.ntiles,
                                                                                                  w.tile_count));
        TTV_LAUNCH("hash_scan", stream,
                   k_hash_scan<<<1, 1024, 0, stream>>>(w.tile_count, h.ntiles, w.tile_off, cap_rows, 1, p.status));
    }
    GatherOut o{};
    o.subs = out_subs;
    o.vals = out_vals;
    o.cap_rows = cap_rows;
    o.mode = dense_out ? 1 : (h.direct ? 0 : 2);
    o.pkeys = w.sb.keys[0];
    o.pvals = w.sb.vals[0];
    auto kg = h.direct ? k_hash_gather<true> : k_hash_gather<false>;
    TTV_LAUNCH("hash_gather", stream,
               kg<<<(unsigned)h.ntiles, kHashThreads, 0, stream>>>(w.slots, w.dvals, w.bits,
                                                                    h.direct ? w.tile_off : nullptr, p, o, p.status));
    if (h.direct || dense_out) return;

    // hashed table, sparse result: order the distinct keys, then emit rows
    unsigned long long* n_dev = &p.status->nnz_out;
    SortBuffers sb = w.sb;
    const int cur = radix_sort_pairs(sb, h.bound, key_bits, p.status, stream, n_dev);
    const int eg = (int)std::min<int64_t>((int64_t)nsm * 8, (h.bound + 255) / 256);
    TTV_LAUNCH("hash_emit", stream,
               k_hash_emit<<<eg, 256, 0, stream>>>(sb.keys[cur], sb.vals[cur], p, out_subs, out_vals, cap_rows,
                                                   p.status));
}

}  // namespace ttv
