// ttv_dense_fx.cu -- dense-accumulator TTV path for small result key spaces,
// built for GB300's balance of units.
//
// * Loads: tiles of the subscript columns and values are staged in shared
//   memory by bulk asynchronous copies (cp.async.bulk, completion on an
//   mbarrier), several tiles in flight per CTA, one persistent CTA per SM.
// * Products: GB300 issues FP64 multiplies at only ~2 per clock per SM, so the
//   term vals[k] * prod x_m[.] is formed from the operands' integer
//   significands: each factor becomes (sign, 64-bit significand, exponent) and
//   the significands are multiplied with 64x64 -> high-64 integer products
//   (truncation error < 2^-62 relative per factor).
// * Accumulation: every term is converted to a 128-bit two's-complement fixed
//   point number whose unit 2^L is set per CTA from the largest term exponent
//   seen so far (the accumulators are shifted right when a later tile raises
//   it).  Integer addition is associative, so the result does not depend on
//   the order of the atomics: the path is deterministic, and each cell is the
//   correctly rounded value of its exact fixed-point sum.  The headroom covers
//   the sum of every term of the tensor, so cross-CTA sums cannot overflow.
//
// Error bound per result cell: (terms in the cell) x 2^(L-1) from rounding
// terms to the grid, plus 2^(Lmax-1) per CTA from aligning the CTA partials,
// plus one final rounding to binary64, where 2^L is about 2^-(127-H) times
// the CTA's largest term and H = ceil(log2(nnz)) + 2.
#include <algorithm>
#include <climits>

#include "ttv_internal.cuh"
#include "ttv_tma.cuh"

namespace ttv {

constexpr int kFxThreads = 512;
constexpr int kFxMaxStages = 4;

typedef __int128 i128;
typedef unsigned __int128 u128;

struct FxParams {
    StreamDesc p;
    int64_t chunk;             // nonzeros per CTA (multiple of tile)
    int tile;                  // nonzeros per stage (multiple of 4)
    int stages;
    int headroom;              // H
    int want_presence;
    int aos;                   // 1: subs rows contiguous (stride_nz == d, stride_mode == 1)
    size_t stage_bytes;
    size_t cells_off, pres_off, vec_off, stage_off, bar_off, smem_total;
    unsigned long long* part_lo;   // [G][P]
    long long* part_hi;            // [G][P]
    int* part_L;                   // [G]
    uint32_t* pres_partials;       // [G][ceil(P/32)]
};

// Term significand in units of 2^L as a signed 128-bit integer (rounded).
__device__ __forceinline__ i128 to_fixed(const Sig& t, int L) {
    if (t.M == 0) return 0;
    const int s = t.E - 63 - L;            // value = M * 2^s units
    u128 mag;
    if (s >= 0) {
        mag = s >= 64 ? (u128)0 : ((u128)t.M << s);    // s < 64 by the headroom
    } else {
        const int r = -s;
        if (r > 64) mag = 0;
        else if (r == 64) mag = (u128)(t.M >> 63);
        else mag = (u128)((t.M >> r) + ((t.M >> (r - 1)) & 1ull));
    }
    return t.neg ? -(i128)mag : (i128)mag;
}

__device__ __forceinline__ i128 shift_right_round(i128 v, int r) {
    if (r <= 0) return v;
    if (r >= 127) return 0;
    return (v + ((i128)1 << (r - 1))) >> r;
}

// ---- the kernel -------------------------------------------------------------
__global__ void __launch_bounds__(kFxThreads, 1) k_dense_fx(FxParams f) {
    extern __shared__ __align__(128) unsigned char fsm[];
    const StreamDesc& p = f.p;
    const int tid = threadIdx.x;
    const int64_t P = (int64_t)p.nkeys;
    unsigned long long* cell_lo = reinterpret_cast<unsigned long long*>(fsm + f.cells_off);
    long long* cell_hi = reinterpret_cast<long long*>(cell_lo + P);
    uint32_t* pres = reinterpret_cast<uint32_t*>(fsm + f.pres_off);
    double* sv = reinterpret_cast<double*>(fsm + f.vec_off);
    unsigned char* stage0 = fsm + f.stage_off;
    uint64_t* full = reinterpret_cast<uint64_t*>(fsm + f.bar_off);
    __shared__ int s_red[2][kFxThreads / 32];      // by tile parity: no reuse race
    __shared__ int s_Ecur;

    const int64_t npres = (P + 31) / 32;
    for (int64_t i = tid; i < P; i += kFxThreads) { cell_lo[i] = 0ull; cell_hi[i] = 0ll; }
    if (f.want_presence)
        for (int64_t i = tid; i < npres; i += kFxThreads) pres[i] = 0u;
    stage_vectors(p, sv);
    if (tid == 0) {
        for (int s = 0; s < f.stages; ++s) mbar_init(&full[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_Ecur = INT_MIN;
    }
    __syncthreads();

    const int64_t lo = (int64_t)blockIdx.x * f.chunk;
    const int64_t hi = min(p.nnz, lo + f.chunk);
    const int64_t ntiles = hi > lo ? (hi - lo + f.tile - 1) / f.tile : 0;
    const int d = p.d;
    const int vb = p.val_f32 ? 4 : 8;

    // thread 0 issues tile i into stage i % stages
    auto issue = [&](int64_t i) {
        const int64_t k0 = lo + i * f.tile;
        const int cnt = (int)min((int64_t)f.tile, hi - k0);
        unsigned char* st = stage0 + (size_t)(i % f.stages) * f.stage_bytes;
        uint64_t* bar = &full[i % f.stages];
        // bulk copies need 16-byte multiples; leftovers are read directly
        const int cs = f.aos ? cnt : (cnt & ~1);            // int64 column elements copied
        const int cv = p.val_f32 ? (cnt & ~3) : (cnt & ~1);  // value elements copied
        uint32_t bytes = 0;
        if (f.aos) {
            const uint32_t b = (uint32_t)((int64_t)cnt * d * 8) & ~15u;
            bytes += b;
        } else {
            bytes += (uint32_t)cs * 8u * (uint32_t)d;
        }
        bytes += (uint32_t)cv * (uint32_t)vb;
        mbar_expect_tx(bar, bytes);
        if (f.aos) {
            const uint32_t b = (uint32_t)((int64_t)cnt * d * 8) & ~15u;
            if (b) bulk_g2s(st, p.subs + k0 * d, b, bar);
        } else if (cs) {
            for (int m = 0; m < d; ++m)
                bulk_g2s(st + (size_t)m * f.tile * 8, p.subs + (int64_t)m * p.smode + k0, (uint32_t)cs * 8u, bar);
        }
        unsigned char* vdst = st + (size_t)d * f.tile * 8;
        if (cv) bulk_g2s(vdst, static_cast<const unsigned char*>(p.vals) + k0 * vb, (uint32_t)cv * vb, bar);
    };
    if (tid == 0)
        for (int64_t i = 0; i < ntiles && i < (int64_t)f.stages; ++i) issue(i);

    constexpr int kItems = 8;     // items per thread per tile (tile <= 8 * threads)
    for (int64_t i = 0; i < ntiles; ++i) {
        const int64_t k0 = lo + i * f.tile;
        const int cnt = (int)min((int64_t)f.tile, hi - k0);
        const unsigned char* st = stage0 + (size_t)(i % f.stages) * f.stage_bytes;
        if (!mbar_wait(&full[i % f.stages], (uint32_t)((i / f.stages) & 1))) {
            set_error(p.status, kErrTimeout);
        }
        const int cs = f.aos ? cnt : (cnt & ~1);
        const int cv = p.val_f32 ? (cnt & ~3) : (cnt & ~1);
        const int aos_copied = f.aos ? (int)((((int64_t)cnt * d * 8) & ~15ll) / 8) : 0;
        const int64_t* scol = reinterpret_cast<const int64_t*>(st);
        const unsigned char* svals = st + (size_t)d * f.tile * 8;

        Sig tv[kItems];
        uint32_t key[kItems];
        int emax = INT_MIN;
#pragma unroll
        for (int u = 0; u < kItems; ++u) {
            const int j = tid + u * kFxThreads;
            tv[u].M = 0;
            tv[u].E = -(1 << 28);
            tv[u].neg = 0;
            tv[u].bad = 0;
            tv[u].wide = 0;
            key[u] = 0xFFFFFFFFu;
            if (j >= cnt) continue;
            const int64_t k = k0 + j;
            double val;
            if (j < cv) val = p.val_f32 ? (double)reinterpret_cast<const float*>(svals)[j]
                                        : reinterpret_cast<const double*>(svals)[j];
            else val = load_val(p, k);
            Sig t = decompose(val);
            uint64_t kk = 0;
            bool good = true;
            int64_t ss[kMaxD];
#pragma unroll
            for (int m = 0; m < kMaxD; ++m) {
                ss[m] = 0;
                if (m >= d) break;
                int64_t sm;
                if (f.aos) sm = (j * d + m < aos_copied) ? scol[j * d + m] : p.subs[k * d + m];
                else sm = j < cs ? scol[(size_t)m * f.tile + j] : p.subs[(int64_t)m * p.smode + k];
                if (sm < 0 || sm >= p.shape[m]) { good = false; continue; }
                ss[m] = sm;
                if ((p.smask >> m) & 1u) sig_mul(t, decompose(load_vec(p, sv, m, sm)));
                else kk += (uint64_t)sm * p.kstride[m];
            }
            if (!good) { set_error(p.status, kErrSubscript); continue; }
            if (t.wide && !t.bad) {
                // a partial product left the normal range: the term is Eq. 3's
                // binary64 chain itself, taken exactly into the fixed point
                double tt = val;
#pragma unroll
                for (int m = 0; m < kMaxD; ++m)
                    if (m < d && ((p.smask >> m) & 1u)) tt = tt * load_vec(p, sv, m, ss[m]);
                t = decompose(tt);
            }
            if (t.bad) set_error(p.status, kErrNonFinite);
            tv[u] = t;
            key[u] = (uint32_t)kk;
            if (t.M) emax = max(emax, t.E);
        }
        // block maximum of the term exponents of this tile
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
        if ((tid & 31) == 0) s_red[i & 1][tid >> 5] = emax;
        __syncthreads();     // also: every thread is done reading this stage
        int tmax = INT_MIN;
#pragma unroll
        for (int w = 0; w < kFxThreads / 32; ++w) tmax = max(tmax, s_red[i & 1][w]);
        const int Ecur = s_Ecur;
        if (tid == 0 && i + f.stages < ntiles) issue(i + f.stages);
        if (tmax > Ecur) {
            // raise the window: shift every cell right by the exponent growth
            if (Ecur != INT_MIN) {
                const int r = tmax - Ecur;
                for (int64_t c = tid; c < P; c += kFxThreads) {
                    i128 v = ((i128)cell_hi[c] << 64) | (i128)cell_lo[c];
                    v = shift_right_round(v, r);
                    cell_lo[c] = (unsigned long long)v;
                    cell_hi[c] = (long long)(v >> 64);
                }
            }
            __syncthreads();
            if (tid == 0) s_Ecur = tmax;
            __syncthreads();
        }
        const int L = s_Ecur + f.headroom - 126;
#pragma unroll
        for (int u = 0; u < kItems; ++u) {
            if (key[u] == 0xFFFFFFFFu) continue;
            if (f.want_presence) atomicOr(&pres[key[u] >> 5], 1u << (key[u] & 31));
            const i128 F = to_fixed(tv[u], L);
            if (F == 0) continue;
            const unsigned long long flo = (unsigned long long)F;
            const unsigned long long fhi = (unsigned long long)(F >> 64);
            const unsigned long long old = atomicAdd(&cell_lo[key[u]], flo);
            const unsigned long long carry = (old + flo < old) ? 1ull : 0ull;
            atomicAdd(reinterpret_cast<unsigned long long*>(&cell_hi[key[u]]), fhi + carry);
        }
    }
    __syncthreads();
    unsigned long long* plo = f.part_lo + (size_t)blockIdx.x * P;
    long long* phi = f.part_hi + (size_t)blockIdx.x * P;
    for (int64_t c = tid; c < P; c += kFxThreads) { plo[c] = cell_lo[c]; phi[c] = cell_hi[c]; }
    if (tid == 0) f.part_L[blockIdx.x] = (s_Ecur == INT_MIN) ? INT_MIN : s_Ecur + f.headroom - 126;
    if (f.want_presence) {
        uint32_t* mp = f.pres_partials + (size_t)blockIdx.x * npres;
        for (int64_t c = tid; c < npres; c += kFxThreads) mp[c] = pres[c];
    }
}

// Exact int128 (units of 2^L) -> nearest binary64.
__device__ __forceinline__ double fixed_to_double(i128 v, int L) {
    if (v == 0) return 0.0;
    const bool neg = v < 0;
    u128 m = neg ? (u128)(-v) : (u128)v;
    const unsigned long long mh = (unsigned long long)(m >> 64), ml = (unsigned long long)m;
    const int top = mh ? 127 - __clzll(mh) : 63 - __clzll(ml);     // index of the leading bit
    unsigned long long sig;      // 53 significant bits, rounded to nearest even
    int exp2;                    // value = sig * 2^exp2 * 2^L
    if (top <= 52) {
        sig = ml;
        exp2 = 0;
    } else {
        const int sh = top - 52;
        const u128 q = m >> sh;
        const u128 rem = m - (q << sh);
        const u128 half = (u128)1 << (sh - 1);
        sig = (unsigned long long)q;
        if (rem > half || (rem == half && (sig & 1ull))) ++sig;
        exp2 = sh;
    }
    const double r = scalbn((double)sig, exp2 + L);
    return neg ? -r : r;
}

// One warp per cell: align every CTA partial to the largest unit, add
// exactly in 128-bit integers, round once.
__global__ void __launch_bounds__(256) k_dense_fx_reduce(int64_t P, int G, const unsigned long long* __restrict__ part_lo,
                                                         const long long* __restrict__ part_hi,
                                                         const int* __restrict__ part_L,
                                                         const uint32_t* __restrict__ pres_partials, int want_presence,
                                                         double* __restrict__ cell_vals, uint32_t* __restrict__ cell_flags) {
    const int lane = threadIdx.x & 31;
    const int64_t cell = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (cell >= P) return;
    int Lmax = INT_MIN;
    for (int b = lane; b < G; b += 32) Lmax = max(Lmax, part_L[b]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) Lmax = max(Lmax, __shfl_xor_sync(0xffffffffu, Lmax, o));
    const int64_t npres = (P + 31) / 32;
    i128 acc = 0;
    uint32_t any = 0;
    for (int b = lane; b < G; b += 32) {
        const int Lb = part_L[b];
        if (want_presence) any |= (pres_partials[(size_t)b * npres + (cell >> 5)] >> (cell & 31)) & 1u;
        if (Lb == INT_MIN) continue;
        const i128 v = ((i128)part_hi[(size_t)b * P + cell] << 64) | (i128)part_lo[(size_t)b * P + cell];
        acc += shift_right_round(v, Lmax - Lb);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long alo = __shfl_xor_sync(0xffffffffu, (unsigned long long)acc, o);
        const unsigned long long ahi = __shfl_xor_sync(0xffffffffu, (unsigned long long)(acc >> 64), o);
        acc += ((i128)(long long)ahi << 64) | (i128)alo;
    }
    any = __any_sync(0xffffffffu, any) ? 1u : 0u;
    if (lane == 0) {
        cell_vals[cell] = Lmax == INT_MIN ? 0.0 : fixed_to_double(acc, Lmax);
        if (want_presence) cell_flags[cell] = any;
    }
}

// ---- host side ---------------------------------------------------------------

static int max_smem_optin() {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return v > 0 ? v : 232448;
}

FxPlan plan_dense_fx(const StreamDesc& p, int want_presence, int num_sms) {
    FxPlan fp{};
    fp.ok = false;
    const bool soa = p.snz == 1;
    const bool aos = p.smode == 1 && p.snz == p.d;
    if (!soa && !aos) return fp;
    // bulk copies need 16-byte aligned sources
    const uintptr_t sb = reinterpret_cast<uintptr_t>(p.subs), vbp = reinterpret_cast<uintptr_t>(p.vals);
    if ((sb & 15) || (vbp & 15)) return fp;
    if (soa && p.d > 1 && ((p.smode * 8) % 16)) return fp;
    fp.aos = aos && !soa ? 1 : 0;
    if (p.d == 1) fp.aos = 0;
    const int vb = p.val_f32 ? 4 : 8;
    const int64_t P = (int64_t)p.nkeys;
    size_t off = 0;
    fp.cells_off = 0;
    off += (size_t)P * 16;
    fp.pres_off = off;
    if (want_presence) off += (size_t)((P + 31) / 32) * 4;
    off = (off + 15) & ~size_t(15);
    fp.vec_off = off;
    if (p.vec_smem) off += (size_t)p.vtotal * 8;
    off = (off + 127) & ~size_t(127);
    fp.stage_off = off;
    const size_t budget = (size_t)max_smem_optin() - 2048;
    if (off + 64 >= budget) return fp;
    const size_t per_nz = (size_t)p.d * 8 + vb;
    // largest tile (multiple of 512, at most 8 items per thread) with >= 2 stages
    int tile = 8 * kFxThreads;
    int stages = 0;
    while (tile >= 512) {
        const size_t sbytes = ((size_t)tile * per_nz + 127) & ~size_t(127);
        stages = (int)std::min<size_t>(kFxMaxStages, (budget - off - 64) / sbytes);
        if (stages >= 2 && (size_t)tile * per_nz * stages >= 96 * 1024) break;
        if (stages >= 3) break;
        tile -= 512;
    }
    if (tile < 512 || stages < 2) return fp;
    fp.tile = tile;
    fp.stages = stages;
    fp.stage_bytes = ((size_t)tile * per_nz + 127) & ~size_t(127);
    fp.bar_off = fp.stage_off + fp.stage_bytes * stages;
    fp.smem_total = fp.bar_off + 8 * kFxMaxStages;
    // one CTA per SM, chunks a whole number of tiles
    const int64_t tiles = (p.nnz + tile - 1) / tile;
    fp.grid = (int)std::max<int64_t>(1, std::min<int64_t>(num_sms, tiles));
    const int64_t tiles_per = (tiles + fp.grid - 1) / fp.grid;
    fp.chunk = tiles_per * tile;
    fp.grid = (int)((tiles + tiles_per - 1) / tiles_per);
    int h = 0;
    while (h < 62 && ((int64_t)1 << h) < p.nnz + 1) ++h;
    fp.headroom = h + 2;
    fp.ok = true;
    return fp;
}

size_t dense_fx_workspace(const StreamDesc& p, const FxPlan& fp, int want_presence) {
    const int64_t P = (int64_t)p.nkeys;
    size_t b = 0;
    b += (size_t)fp.grid * P * 16 + 256;
    b += (size_t)fp.grid * 4 + 256;
    if (want_presence) b += (size_t)fp.grid * ((P + 31) / 32) * 4 + 256;
    return b;
}

void launch_dense_fx(const StreamDesc& p, const FxPlan& fp, int want_presence, void* ws, double* cell_vals,
                     uint32_t* cell_flags, cudaStream_t stream) {
    const int64_t P = (int64_t)p.nkeys;
    char* w = static_cast<char*>(ws);
    auto take = [&](size_t bytes) {
        char* r = w;
        w += (bytes + 255) & ~size_t(255);
        return r;
    };
    FxParams f;
    f.p = p;
    f.chunk = fp.chunk;
    f.tile = fp.tile;
    f.stages = fp.stages;
    f.headroom = fp.headroom;
    f.want_presence = want_presence;
    f.aos = fp.aos;
    f.stage_bytes = fp.stage_bytes;
    f.cells_off = fp.cells_off;
    f.pres_off = fp.pres_off;
    f.vec_off = fp.vec_off;
    f.stage_off = fp.stage_off;
    f.bar_off = fp.bar_off;
    f.smem_total = fp.smem_total;
    f.part_lo = reinterpret_cast<unsigned long long*>(take((size_t)fp.grid * P * 8));
    f.part_hi = reinterpret_cast<long long*>(take((size_t)fp.grid * P * 8));
    f.part_L = reinterpret_cast<int*>(take((size_t)fp.grid * 4));
    f.pres_partials = want_presence ? reinterpret_cast<uint32_t*>(take((size_t)fp.grid * ((P + 31) / 32) * 4)) : nullptr;
    smem_at_least(k_dense_fx, fp.smem_total);
    TTV_LAUNCH("dense_fx", stream, k_dense_fx<<<fp.grid, kFxThreads, fp.smem_total, stream>>>(f));
    const int64_t blocks = (P * 32 + 255) / 256;
    TTV_LAUNCH("dense_fx_reduce", stream,
               k_dense_fx_reduce<<<(unsigned)blocks, 256, 0, stream>>>(P, fp.grid, f.part_lo, f.part_hi, f.part_L,
                                                                      f.pres_partials, want_presence, cell_vals,
                                                                      cell_flags));
}

}  // namespace ttv
