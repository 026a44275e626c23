// ttv_noalloc.cu -- dense-result TTV that allocates no memory at all.
//
// Who needs this: code that runs where a cudaMalloc is not allowed or not
// wanted -- for example inside a host callback or a plugin whose host
// application owns every device allocation, a real-time loop that must not
// take the allocator's locks or trigger its synchronisation, or a process
// that has handed its whole memory budget to another runtime.  Such a caller
// can still hand over its own input and output buffers; what it cannot do is
// let the library obtain scratch space behind its back.
//
// So this entry point keeps its scratch (the status word and the per-CTA
// partial sums of the dense accumulator) in one fixed array of device memory
// that is part of the loaded library image.  Every GPU that loads the library
// holds that array (kNoAllocScratchBytes) until the process exits.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "ttv_internal.cuh"

namespace ttv {

// from ttv_stream.cu / ttv_api.cu (unchanged paths, reused here)
int dense_grid(const StreamDesc& p, int want_presence);
void launch_dense(const StreamDesc& p, int want_presence, int compensated, int G, double* partials,
                  uint32_t* pres_partials, double* cell_vals, uint32_t* cell_flags, cudaStream_t stream);
int plan_dense_desc(const ttv_tensor* t, const int32_t* modes, int32_t n_v, const void* const* vecs, ttv_dtype vd,
                    const int64_t* vec_lens, StreamDesc* out);
int fail(int code, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);

constexpr size_t kNoAllocScratchBytes = TTV_NOALLOC_SCRATCH_BYTES;
constexpr size_t kNoAllocStatusBytes = 256;
// The scratch holds many partial arrays of the largest dense result, so the
// budget check below is a guard that the documented limits never reach.
static_assert(kNoAllocScratchBytes >= kNoAllocStatusBytes + 31 * kDenseMaxCells * sizeof(double),
              "fixed scratch smaller than 31 partial arrays of the largest dense result");

// The scratch array.  In host code this name is only a host-side stand-in:
// its device address must be fetched with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of g_noalloc_scratch, looked up once per device.
static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[64] = {nullptr};

static int noalloc_scratch(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return fail(TTV_ERR_UNSUPPORTED, "device ordinal %d not supported", dev);
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
        g_noalloc_addr[dev] = ptr;
    }
    *out = g_noalloc_addr[dev];
    return TTV_OK;
}

}  // namespace ttv

using namespace ttv;

extern "C" int ttv_dense_noalloc(const ttv_tensor* t, const int32_t* modes, int32_t n_v, const void* const* vecs,
                                 const int64_t* vec_lens, ttv_dtype v_dtype, double* out, int64_t out_len,
                                 ttv_stream_t stream_) {
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    StreamDesc p;
    int rc = plan_dense_desc(t, modes, n_v, vecs, v_dtype, vec_lens, &p);
    if (rc != TTV_OK) return rc;
    const int64_t P = (int64_t)p.nkeys;
    if (!out) return fail(TTV_ERR_ARG, "null output");
    if (out_len < P) return fail(TTV_ERR_CAPACITY, "dense result needs %lld values, buffer has %lld", (long long)P,
                                 (long long)out_len);
    // how many CTA partial arrays fit next to the status block
    const size_t room = (kNoAllocScratchBytes - kNoAllocStatusBytes) / sizeof(double);
    if ((size_t)P > room)
        return fail(TTV_ERR_BUDGET, "result of %lld cells exceeds the fixed scratch (%zu bytes)", (long long)P,
                    kNoAllocScratchBytes);
    void* base = nullptr;
    rc = noalloc_scratch(&base);
    if (rc != TTV_OK) return rc;
    Status* st = static_cast<Status*>(base);
    double* partials = reinterpret_cast<double*>(static_cast<unsigned char*>(base) + kNoAllocStatusBytes);
    p.status = st;

    cudaError_t e = cudaMemsetAsync(st, 0, sizeof(Status), stream);       // error word must start at zero
    if (e != cudaSuccess) return cuda_fail(e, "status reset");
    if (p.nnz == 0) {
        e = cudaMemsetAsync(out, 0, (size_t)P * sizeof(double), stream);
        if (e != cudaSuccess) return cuda_fail(e, "zero result");
    } else {
        int G = dense_grid(p, 0);
        G = (int)std::min<int64_t>((int64_t)G, (int64_t)(room / (size_t)P));
        if (G < 1) G = 1;
        // every CTA overwrites its whole partial array, so no clearing is needed
        launch_dense(p, 0, 0, G, partials, nullptr, out, nullptr, stream);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    Status h;
    memset(&h, 0, sizeof h);
    e = cudaMemcpyAsync(&h, st, sizeof(Status), cudaMemcpyDeviceToHost, stream);
    if (e != cudaSuccess) return cuda_fail(e, "status read");
    e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
    if (h.err & kErrSubscript) return fail(TTV_ERR_SUBSCRIPT, "a subscript is outside its mode");
    if (h.err) return fail(TTV_ERR_CUDA, "device error bits 0x%x", h.err);
    return TTV_OK;
}
