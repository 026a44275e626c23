// ttv_dense_vec.cu -- order-specialised dense accumulation kernel.
//
// Same computation as k_dense_accum (ttv_stream.cu), compiled per tensor
// order D and subscript layout so that the per-mode loop is fully unrolled
// with no runtime order checks, and every thread loads two consecutive
// nonzeros per 16-byte access (one column element pair under the SoA layout,
// two rows under AoS).  With kIntP the term is formed from exact integer
// significand products (GB300's FP64 pipe issues ~1.7 operations per clock
// per SM, so three binary64 multiplies per nonzero would cap the kernel below
// the HBM rate); the accumulation is one binary64 add per nonzero into the
// CTA's shared-memory array, as in the generic kernel.
#include <algorithm>

#include "ttv_internal.cuh"
#include "ttv_tma.cuh"

namespace ttv {

constexpr int kVecThreads = 256;
// Pairs of nonzeros per thread per iteration: 1 (59 registers, 4 CTAs per
// SM; the default) or 2 (more loads in flight per thread, 3 CTAs per SM);
// the autotuner picks per problem class.

template <int D, bool kIntP, bool kPriv = false>
__device__ __forceinline__ void dense_item(const StreamDesc& p, const double* sv, const SigEntry* sve,
                                           const int64_t* s, double val, double* acc, uint32_t* pres,
                                           int want_presence) {
    bool good = true;
#pragma unroll
    for (int m = 0; m < D; ++m) good &= (uint64_t)s[m] < (uint64_t)p.shape[m];
    if (!good) {
        set_error(p.status, kErrSubscript);
        return;
    }
    uint64_t key = 0;
    double t;
    if constexpr (kIntP) {
        Sig a = decompose(val);
#pragma unroll
        for (int m = 0; m < D; ++m) {
            if ((p.smask >> m) & 1u) sig_mul(a, sig_of(sve[p.voff[m] + s[m]]));
            else key += (uint64_t)s[m] * p.kstride[m];
        }
        if (a.bad | a.wide) {
            double tt = val;
#pragma unroll
            for (int m = 0; m < D; ++m)
                if ((p.smask >> m) & 1u)
                    tt = tt * (p.vec_f32 ? (double)__ldg(static_cast<const float*>(p.vec[m]) + s[m])
                                         : __ldg(static_cast<const double*>(p.vec[m]) + s[m]));
            t = tt;
        } else {
            t = sig_to_double(a);
        }
    } else {
        t = val;
#pragma unroll
        for (int m = 0; m < D; ++m) {
            if ((p.smask >> m) & 1u) t = t * sv[p.voff[m] + s[m]];
            else key += (uint64_t)s[m] * p.kstride[m];
        }
    }
    if constexpr (kPriv) {
        // the warp's own accumulator: a plain add unless another active lane
        // of the warp hits the same cell in this step
        const uint32_t same = __match_any_sync(__activemask(), (uint32_t)key);
        if (__popc(same) == 1) acc[key] += t;
        else atomicAdd(&acc[key], t);
    } else {
        atomicAdd(&acc[key], t);
    }
    if (want_presence) atomicOr(&pres[key >> 5], 1u << (key & 31));
}

// kVecPairs == 3: one pair per iteration into warp-private accumulators
// (eight arrays of P cells per CTA, two CTAs per SM): the binary64 add is a
// plain read-modify-write instead of a compare-and-swap loop.
template <int D, bool kSoA, bool kIntP, int kVecPairs>
__global__ void __launch_bounds__(kVecThreads, kVecPairs == 1 ? 4 : (kVecPairs == 2 ? 3 : 2)) k_dense_vec(StreamDesc p, int64_t chunk, int want_presence,
                                                           size_t pres_off, size_t vec_off,
                                                           double* __restrict__ partials,
                                                           uint32_t* __restrict__ pres_partials) {
    extern __shared__ __align__(16) unsigned char dsm[];
    double* acc = reinterpret_cast<double*>(dsm);
    uint32_t* pres = reinterpret_cast<uint32_t*>(dsm + pres_off);
    double* sv = reinterpret_cast<double*>(dsm + vec_off);
    SigEntry* sve = reinterpret_cast<SigEntry*>(dsm + vec_off);
    constexpr bool kPriv = kVecPairs == 3;
    constexpr int kPairs = kPriv ? 1 : kVecPairs;
    constexpr int kCopies = kPriv ? kVecThreads / 32 : 1;
    const int64_t P = (int64_t)p.nkeys;
    const int64_t npres = (P + 31) / 32;
    for (int64_t i = threadIdx.x; i < P * kCopies; i += kVecThreads) acc[i] = 0.0;
    double* wacc = acc + (kPriv ? (int64_t)(threadIdx.x >> 5) * P : 0);
    if (want_presence)
        for (int64_t i = threadIdx.x; i < npres; i += kVecThreads) pres[i] = 0u;
    if (kIntP) stage_vectors_sig(p, sve);
    else stage_vectors(p, sv);
    __syncthreads();

    const int64_t lo = (int64_t)blockIdx.x * chunk;               // even
    const int64_t hi = min(p.nnz, lo + chunk);
    const int64_t npairs = hi > lo ? (hi - lo) / 2 : 0;            // whole pairs
    const double* vd = static_cast<const double*>(p.vals);
    const float* vf = static_cast<const float*>(p.vals);

    for (int64_t q0 = threadIdx.x; q0 < npairs; q0 += (int64_t)kVecThreads * kPairs) {
        int64_t s[kPairs][2][D];
        double v[kPairs][2];
        bool ok[kPairs];
#pragma unroll
        for (int u = 0; u < kPairs; ++u) {
            const int64_t q = q0 + (int64_t)u * kVecThreads;
            ok[u] = q < npairs;
            if (!ok[u]) continue;
            const int64_t k = lo + 2 * q;
            if constexpr (kSoA) {
#pragma unroll
                for (int m = 0; m < D; ++m) {
                    const longlong2 w = __ldcs(reinterpret_cast<const longlong2*>(p.subs + m * p.smode + k));
                    s[u][0][m] = w.x;
                    s[u][1][m] = w.y;
                }
            } else {
                const longlong2* row = reinterpret_cast<const longlong2*>(p.subs + k * D);
#pragma unroll
                for (int j = 0; j < D; ++j) {
                    const longlong2 w = __ldcs(row + j);
                    const int e0 = 2 * j, e1 = 2 * j + 1;
                    if (e0 < D) s[u][0][e0] = w.x; else s[u][1][e0 - D] = w.x;
                    if (e1 < D) s[u][0][e1] = w.y; else s[u][1][e1 - D] = w.y;
                }
            }
            if (p.val_f32) {
                const float2 w = __ldcs(reinterpret_cast<const float2*>(vf + k));
                v[u][0] = (double)w.x;
                v[u][1] = (double)w.y;
            } else {
                const double2 w = __ldcs(reinterpret_cast<const double2*>(vd + k));
                v[u][0] = w.x;
                v[u][1] = w.y;
            }
        }
#pragma unroll
        for (int u = 0; u < kPairs; ++u) {
            if (!ok[u]) continue;
            dense_item<D, kIntP, kPriv>(p, sv, sve, s[u][0], v[u][0], wacc, pres, want_presence);
            dense_item<D, kIntP, kPriv>(p, sv, sve, s[u][1], v[u][1], wacc, pres, want_presence);
        }
    }
    // odd tail of the last chunk
    if (threadIdx.x == 0 && hi > lo && ((hi - lo) & 1)) {
        const int64_t k = hi - 1;
        int64_t s1[D];
#pragma unroll
        for (int m = 0; m < D; ++m) s1[m] = p.subs[k * p.snz + m * p.smode];
        const double v1 = p.val_f32 ? (double)vf[k] : vd[k];
        dense_item<D, kIntP, kPriv>(p, sv, sve, s1, v1, wacc, pres, want_presence);
    }
    __syncthreads();
    double* my = partials + (size_t)blockIdx.x * P;
    for (int64_t i = threadIdx.x; i < P; i += kVecThreads) {
        double x = acc[i];
#pragma unroll
        for (int c = 1; c < kCopies; ++c) x += acc[c * P + i];     // fixed order
        my[i] = x;
    }
    if (want_presence) {
        uint32_t* mp = pres_partials + (size_t)blockIdx.x * npres;
        for (int64_t i = threadIdx.x; i < npres; i += kVecThreads) mp[i] = pres[i];
    }
}

// ---- bulk-staged persistent variant -------------------------------------------
// One CTA per SM.  A producer warp streams the CTA's range of nonzeros into
// shared memory, tile by tile, with cp.async.bulk copies that complete on a
// per-stage mbarrier; 31 consumer warps form the terms from the staged
// subscripts and values and add them into the shared accumulator, then
// release the stage on a second mbarrier.  The loads stay in flight (up to
// four tiles) while the consumers work, instead of every thread waiting on
// its own global loads.
constexpr int kTmaThreads = 1024;
constexpr int kTmaConsumers = kTmaThreads - 32;     // warps 0..30
constexpr int kTmaTile = 2 * kTmaConsumers;          // 1984 nonzeros per stage
constexpr int kTmaMaxStages = 4;
constexpr size_t kTmaSmemMax = 226 * 1024;   // under the 227 KB opt-in, with room for static shared memory

struct TmaLayout {
    size_t pres_off, vec_off, stage_off, bar_off, total, stage_bytes;
    int stages;
};

static TmaLayout tma_layout(const StreamDesc& p, int want_presence, bool intp) {
    TmaLayout L{};
    size_t off = (size_t)p.nkeys * sizeof(double);
    L.pres_off = off;
    if (want_presence) off += ((p.nkeys + 31) / 32) * sizeof(uint32_t);
    off = (off + 15) & ~size_t(15);
    L.vec_off = off;
    off += (size_t)p.vtotal * (intp ? sizeof(SigEntry) : sizeof(double));
    off = (off + 127) & ~size_t(127);
    L.stage_off = off;
    const size_t vb = p.val_f32 ? 4 : 8;
    L.stage_bytes = (size_t)kTmaTile * (8 * (size_t)p.d + vb);
    L.stage_bytes = (L.stage_bytes + 127) & ~size_t(127);
    const size_t bars = 2 * kTmaMaxStages * sizeof(uint64_t);
    const size_t room = kTmaSmemMax > off + bars ? kTmaSmemMax - off - bars : 0;
    L.stages = (int)std::min<size_t>(kTmaMaxStages, room / L.stage_bytes);
    L.bar_off = off + (size_t)std::max(L.stages, 0) * L.stage_bytes;
    L.total = L.bar_off + bars;
    return L;
}

template <int D, bool kSoA, bool kIntP>
__global__ void __launch_bounds__(kTmaThreads, 1) k_dense_tma(StreamDesc p, int64_t chunk, int want_presence,
                                                             TmaLayout L, double* __restrict__ partials,
                                                             uint32_t* __restrict__ pres_partials) {
    extern __shared__ __align__(128) unsigned char tsm[];
    double* acc = reinterpret_cast<double*>(tsm);
    uint32_t* pres = reinterpret_cast<uint32_t*>(tsm + L.pres_off);
    double* sv = reinterpret_cast<double*>(tsm + L.vec_off);
    SigEntry* sve = reinterpret_cast<SigEntry*>(tsm + L.vec_off);
    unsigned char* stage0 = tsm + L.stage_off;
    uint64_t* full = reinterpret_cast<uint64_t*>(tsm + L.bar_off);
    uint64_t* empty = full + kTmaMaxStages;
    __shared__ int s_err;
    __shared__ long long s_issued;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int S = L.stages;
    const int64_t P = (int64_t)p.nkeys;
    const int64_t npres = (P + 31) / 32;
    for (int64_t i = tid; i < P; i += kTmaThreads) acc[i] = 0.0;
    if (want_presence)
        for (int64_t i = tid; i < npres; i += kTmaThreads) pres[i] = 0u;
    if (kIntP) stage_vectors_sig(p, sve);
    else stage_vectors(p, sv);
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kTmaConsumers / 32);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_err = 0;
        s_issued = 0;
    }
    __syncthreads();

    const int64_t lo = (int64_t)blockIdx.x * chunk;     // a multiple of 4
    const int64_t hi = min(p.nnz, lo + chunk);
    const int64_t ntiles = hi > lo ? (hi - lo + kTmaTile - 1) / kTmaTile : 0;
    const int vb = p.val_f32 ? 4 : 8;
    const double* vd = static_cast<const double*>(p.vals);
    const float* vf = static_cast<const float*>(p.vals);

    if (warp == kTmaThreads / 32 - 1) {
        // producer: tile i goes to stage i % S once its previous use is released
        if (lane == 0) {
            int64_t i = 0;
            for (; i < ntiles; ++i) {
                const int s = (int)(i % S);
                if (i >= S && !mbar_wait(&empty[s], (uint32_t)(((i / S) - 1) & 1), wait_limit(1u << 24))) {
                    set_error(p.status, kErrTimeout);
                    s_err = 1;
                    break;
                }
                const int64_t k0 = lo + i * kTmaTile;
                const int cnt = (int)min((int64_t)kTmaTile, hi - k0);
                unsigned char* st = stage0 + (size_t)s * L.stage_bytes;
                // copies of whole 16-byte units; the few elements past them are read directly
                const uint32_t sb = kSoA ? (uint32_t)(cnt & ~1) * 8u : ((uint32_t)cnt * 8u * D) & ~15u;
                const uint32_t vbytes = p.val_f32 ? (uint32_t)(cnt & ~3) * 4u : (uint32_t)(cnt & ~1) * 8u;
                mbar_expect_tx(&full[s], (kSoA ? sb * D : sb) + vbytes);
                if (kSoA) {
                    if (sb)
#pragma unroll
                        for (int m = 0; m < D; ++m)
                            bulk_g2s(st + (size_t)m * kTmaTile * 8, p.subs + (int64_t)m * p.smode + k0, sb, &full[s]);
                } else if (sb) {
                    bulk_g2s(st, p.subs + k0 * D, sb, &full[s]);
                }
                if (vbytes)
                    bulk_g2s(st + (size_t)D * kTmaTile * 8, static_cast<const unsigned char*>(p.vals) + k0 * vb,
                             vbytes, &full[s]);
            }
            s_issued = i;
        }
    } else {
        // consumers: two nonzeros of every tile per thread
        for (int64_t i = 0; i < ntiles; ++i) {
            const int s = (int)(i % S);
            if (!mbar_wait(&full[s], (uint32_t)((i / S) & 1), wait_limit(1u << 24))) {
                set_error(p.status, kErrTimeout);
                s_err = 1;
                break;
            }
            const int64_t k0 = lo + i * kTmaTile;
            const int cnt = (int)min((int64_t)kTmaTile, hi - k0);
            const unsigned char* st = stage0 + (size_t)s * L.stage_bytes;
            const int64_t* scol = reinterpret_cast<const int64_t*>(st);
            const int cs = kSoA ? (cnt & ~1) : (int)((((uint32_t)cnt * 8u * D) & ~15u) / 8u);
            const int cv = p.val_f32 ? (cnt & ~3) : (cnt & ~1);
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int j = tid + u * kTmaConsumers;
                if (j >= cnt) continue;
                const int64_t k = k0 + j;
                int64_t sj[D];
#pragma unroll
                for (int m = 0; m < D; ++m) {
                    if (kSoA) sj[m] = j < cs ? scol[(size_t)m * kTmaTile + j] : p.subs[(int64_t)m * p.smode + k];
                    else sj[m] = j * D + m < cs ? scol[j * D + m] : p.subs[k * D + m];
                }
                double v;
                if (j < cv) v = p.val_f32 ? (double)reinterpret_cast<const float*>(st + (size_t)D * kTmaTile * 8)[j]
                                          : reinterpret_cast<const double*>(st + (size_t)D * kTmaTile * 8)[j];
                else v = p.val_f32 ? (double)vf[k] : vd[k];
                dense_item<D, kIntP>(p, sv, sve, sj, v, acc, pres, want_presence);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
        }
    }
    __syncthreads();
    if (tid == 0 && s_err) {
        // a wait ran out: let every copy already issued land before the CTA exits
        const int64_t issued = s_issued;
        for (int64_t i = max((int64_t)0, issued - S); i < issued; ++i)
            mbar_wait(&full[i % S], (uint32_t)((i / S) & 1), 1u << 20);
    }
    double* my = partials + (size_t)blockIdx.x * P;
    for (int64_t i = tid; i < P; i += kTmaThreads) my[i] = acc[i];
    if (want_presence) {
        uint32_t* mp = pres_partials + (size_t)blockIdx.x * npres;
        for (int64_t i = tid; i < npres; i += kTmaThreads) mp[i] = pres[i];
    }
}

typedef void (*DenseTmaKernel)(StreamDesc, int64_t, int, TmaLayout, double*, uint32_t*);

template <int D>
static DenseTmaKernel pick_tma(bool soa, bool intp) {
    if (soa) return intp ? k_dense_tma<D, true, true> : k_dense_tma<D, true, false>;
    return intp ? k_dense_tma<D, false, true> : k_dense_tma<D, false, false>;
}

static DenseTmaKernel dense_tma_kernel(int d, bool soa, bool intp) {
    switch (d) {
        case 2: return pick_tma<2>(soa, intp);
        case 3: return pick_tma<3>(soa, intp);
        case 4: return pick_tma<4>(soa, intp);
        case 5: return pick_tma<5>(soa, intp);
        case 6: return pick_tma<6>(soa, intp);
        default: return nullptr;
    }
}

// ---- host side ------------------------------------------------------------
typedef void (*DenseVecKernel)(StreamDesc, int64_t, int, size_t, size_t, double*, uint32_t*);

template <int D, int P>
static DenseVecKernel pick_p(bool soa, bool intp) {
    if (soa) return intp ? k_dense_vec<D, true, true, P> : k_dense_vec<D, true, false, P>;
    return intp ? k_dense_vec<D, false, true, P> : k_dense_vec<D, false, false, P>;
}

template <int D>
static DenseVecKernel pick(bool soa, bool intp, int pairs) {
    return pairs == 3 ? pick_p<D, 3>(soa, intp) : pairs == 2 ? pick_p<D, 2>(soa, intp) : pick_p<D, 1>(soa, intp);
}

int dense_vec_products_int(const StreamDesc& p);

// Accumulator layout: 1 = one shared array per CTA (binary64 atomics; the
// default), 2 = the same with two pairs per thread per iteration, 3 = one
// array per warp with plain adds (an autotuner candidate where the eight
// copies, the staged vectors and no presence bits fit in half an SM's shared
// memory).  On the all-but-one 1000^4 problem mode 3 takes 173 us against
// mode 1's 105 us: the binary64 compare-and-swap adds cost less than the
// halved occupancy.
constexpr size_t kPrivSmemMax = 110 * 1024;

static int dense_vec_mode(const StreamDesc& p, int want_presence) {
    if (p.items == 2) return 2;
    if (p.items == 3) {
        const size_t vec = (size_t)p.vtotal * (dense_vec_products_int(p) ? sizeof(SigEntry) : sizeof(double));
        const size_t priv = (size_t)p.nkeys * sizeof(double) * (kVecThreads / 32) + 16 + vec;
        if (!want_presence && priv <= kPrivSmemMax) return 3;
    }
    return 1;
}

static size_t dense_vec_acc_bytes(const StreamDesc& p, int want_presence) {
    return (size_t)p.nkeys * sizeof(double) * (dense_vec_mode(p, want_presence) == 3 ? kVecThreads / 32 : 1);
}

static DenseVecKernel dense_vec_kernel(int d, bool soa, bool intp, int pairs) {
    switch (d) {
        case 2: return pick<2>(soa, intp, pairs);
        case 3: return pick<3>(soa, intp, pairs);
        case 4: return pick<4>(soa, intp, pairs);
        case 5: return pick<5>(soa, intp, pairs);
        case 6: return pick<6>(soa, intp, pairs);
        default: return nullptr;
    }
}

// Whether the specialised kernel applies: order 2..6, staged vectors, and
// 16-byte aligned pairs under an SoA or AoS layout.
bool dense_vec_applicable(const StreamDesc& p) {
    if (p.d < 2 || p.d > 6 || !p.vec_smem) return false;
    const uintptr_t sb = reinterpret_cast<uintptr_t>(p.subs), vb = reinterpret_cast<uintptr_t>(p.vals);
    if ((sb & 15) || (vb & 15)) return false;
    const bool soa = p.snz == 1 && (p.smode % 2 == 0);
    const bool aos = p.snz == p.d && p.smode == 1;
    return soa || aos;
}

int dense_vec_products_int(const StreamDesc& p) { return __builtin_popcount(p.smask) >= 2; }

size_t dense_vec_smem(const StreamDesc& p, int want_presence) {
    size_t off = dense_vec_acc_bytes(p, want_presence);
    if (want_presence) off += ((p.nkeys + 31) / 32) * sizeof(uint32_t);
    off = (off + 15) & ~size_t(15);
    off += (size_t)p.vtotal * (dense_vec_products_int(p) ? sizeof(SigEntry) : sizeof(double));
    return off;
}

// The bulk-staged kernel is the autotuner's items == 4 candidate, used when
// at least two stages fit beside the accumulator and the staged vectors and
// there are enough nonzeros for every SM to stream several tiles.  It is not
// the default: on the all-but-one 1000^4 problem it takes 113 us against the
// register-loading kernel's 105 us, because the limit there is the shared
// memory atomics and significand loads, not the global loads it overlaps.
static bool use_tma(const StreamDesc& p, int want_presence) {
    if (p.items != 4) return false;
    if (p.val_f32 && (reinterpret_cast<uintptr_t>(p.vals) & 15)) return false;
    if (p.nnz < (int64_t)num_sms() * kTmaTile * 2) return false;
    return tma_layout(p, want_presence, dense_vec_products_int(p) != 0).stages >= 2;
}

static int64_t tma_chunk(const StreamDesc& p, int G) {
    int64_t chunk = (p.nnz + G - 1) / G;
    return (chunk + 3) & ~int64_t(3);
}

int dense_vec_grid(const StreamDesc& p, int want_presence) {
    if (use_tma(p, want_presence)) return num_sms();
    const bool soa = p.snz == 1;
    const int mode = dense_vec_mode(p, want_presence);
    DenseVecKernel k = dense_vec_kernel(p.d, soa, dense_vec_products_int(p), mode);
    const size_t smem = dense_vec_smem(p, want_presence);
    smem_at_least(k, smem);
    cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kVecThreads, smem);
    per_sm = std::max(1, std::min(per_sm, p.ctas_per_sm > 0 ? p.ctas_per_sm : 4));
    const int64_t min_chunk = std::max<int64_t>((int64_t)kVecThreads * (mode == 2 ? 2 : 1) * 2 * 4, (int64_t)p.nkeys * 4);
    const int64_t by_work = std::max<int64_t>(1, (p.nnz + min_chunk - 1) / min_chunk);
    return (int)std::max<int64_t>(1, std::min<int64_t>(by_work, (int64_t)num_sms() * per_sm));
}

void launch_dense_vec(const StreamDesc& p, int want_presence, int G, double* partials, uint32_t* pres_partials,
                      cudaStream_t stream) {
    const bool soa = p.snz == 1;
    if (use_tma(p, want_presence) && G == num_sms()) {
        const bool intp = dense_vec_products_int(p) != 0;
        DenseTmaKernel k = dense_tma_kernel(p.d, soa, intp);
        const TmaLayout L = tma_layout(p, want_presence, intp);
        smem_at_least(k, L.total);
        TTV_LAUNCH("dense_accum", stream,
                   k<<<G, kTmaThreads, L.total, stream>>>(p, tma_chunk(p, G), want_presence, L, partials,
                                                          pres_partials));
        return;
    }
    DenseVecKernel k = dense_vec_kernel(p.d, soa, dense_vec_products_int(p), dense_vec_mode(p, want_presence));
    const size_t smem = dense_vec_smem(p, want_presence);
    size_t pres_off = dense_vec_acc_bytes(p, want_presence);
    size_t vec_off = pres_off + (want_presence ? ((p.nkeys + 31) / 32) * sizeof(uint32_t) : 0);
    vec_off = (vec_off + 15) & ~size_t(15);
    int64_t chunk = (p.nnz + G - 1) / G;
    chunk = (chunk + 1) & ~int64_t(1);
    smem_at_least(k, smem);
    TTV_LAUNCH("dense_accum", stream,
               k<<<G, kVecThreads, smem, stream>>>(p, chunk, want_presence, pres_off, vec_off, partials,
                                                   pres_partials));
}

cudaError_t dense_vec_set_wait_override(uint32_t v) { return set_wait_override_here(v); }

// ---- test hook: a wait that must run out -------------------------------------
// One thread waits, with the given poll limit, on an mbarrier that nothing
// arrives on (kind 0) or on a global word that nothing sets (kind 1), and
// raises kErrTimeout when the wait runs out.  No copy is in flight, so the
// CTA may simply return.
__global__ void k_wait_probe(int kind, uint32_t polls, const uint32_t* word, Status* st) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    bool ok;
    if (kind == 0) {
        mbar_init(&bar, 1);
        ok = mbar_wait(&bar, 0, polls);
    } else {
        uint32_t v = 0;
        ok = spin_until(word, v, [](uint32_t x) { return x != 0u; }, polls);
    }
    if (!ok) set_error(st, kErrTimeout);
}

// 1: the wait ran out (status raised), 0: it did not; negative: CUDA error.
int wait_probe(int kind, uint32_t polls, cudaStream_t stream) {
    Status* st = nullptr;
    if (cudaMalloc(&st, sizeof(Status) + 256) != cudaSuccess) return -1;
    uint32_t* word = reinterpret_cast<uint32_t*>(reinterpret_cast<unsigned char*>(st) + sizeof(Status));
    int rc = -1;
    Status h;
    if (cudaMemsetAsync(st, 0, sizeof(Status) + 256, stream) == cudaSuccess) {
        TTV_LAUNCH("wait_probe", stream, k_wait_probe<<<1, 32, 0, stream>>>(kind, polls, word, st));
        if (cudaGetLastError() == cudaSuccess &&
            cudaMemcpyAsync(&h, st, sizeof(Status), cudaMemcpyDeviceToHost, stream) == cudaSuccess &&
            cudaStreamSynchronize(stream) == cudaSuccess)
            rc = (h.err & kErrTimeout) ? 1 : 0;
    }
    cudaFree(st);
    return rc;
}

}  // namespace ttv
