// ttv_prof.cu -- launch counting and optional per-kernel CUDA-event timing.
// Every kernel launch of the library goes through prof_begin/prof_end.  When
// profiling is enabled, an event pair brackets the launch on its own stream
// and ttv_profile_collect() folds the elapsed times into per-kernel totals.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "ttv_internal.cuh"

namespace ttv {

static std::atomic<long long> g_launches{0};
static std::atomic<int> g_prof_on{0};
struct Pending {
    const char* name;
    cudaEvent_t a, b;
};
static std::mutex g_prof_mu;
static std::vector<Pending> g_pending;
static std::vector<cudaEvent_t> g_free_events;
static std::map<std::string, std::pair<double, long long>> g_totals;
static thread_local Pending t_open{nullptr, nullptr, nullptr};
thread_local int t_capturing = 0;     // inside a graph capture: count, never record events

void smem_limit_at_least(const void* kernel, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, size_t> limit;   // (device, kernel) -> bytes set
    if (bytes <= 48 * 1024) return;      // the default limit
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> g(mu);
    size_t& cur = limit[{dev, kernel}];
    if (bytes <= cur) return;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) == cudaSuccess)
        cur = bytes;
    else
        cudaGetLastError();   // the launch reports the error
}

long long prof_add_launches(long long n) { return g_launches.fetch_add(n) + n; }

static cudaEvent_t get_event() {
    if (!g_free_events.empty()) {
        cudaEvent_t e = g_free_events.back();
        g_free_events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void prof_begin(const char* name, cudaStream_t s) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (t_capturing || !g_prof_on.load(std::memory_order_relaxed)) return;
    std::lock_guard<std::mutex> g(g_prof_mu);
    t_open.name = name;
    t_open.a = get_event();
    t_open.b = get_event();
    cudaEventRecord(t_open.a, s);
}

void prof_end(cudaStream_t s) {
    if (!t_open.name) return;
    std::lock_guard<std::mutex> g(g_prof_mu);
    cudaEventRecord(t_open.b, s);
    g_pending.push_back(t_open);
    t_open = Pending{nullptr, nullptr, nullptr};
}

cudaError_t sort_set_wait_override(uint32_t v);
cudaError_t dense_vec_set_wait_override(uint32_t v);
int wait_probe(int kind, uint32_t polls, cudaStream_t stream);

}  // namespace ttv

using namespace ttv;

extern "C" {

int ttv_test_set_wait_polls(long long polls) {
    const uint32_t v = polls < 0 ? 0u : (uint32_t)std::min<long long>(polls, 0xFFFFFFFELL) + 1u;
    if (sort_set_wait_override(v) != cudaSuccess || dense_vec_set_wait_override(v) != cudaSuccess)
        return TTV_ERR_CUDA;
    return TTV_OK;
}

int ttv_test_wait_probe(int kind, unsigned int polls) {
    if (kind != 0 && kind != 1) return TTV_ERR_ARG;
    const int r = wait_probe(kind, polls, nullptr);
    if (r < 0) return TTV_ERR_CUDA;
    return r ? TTV_ERR_TIMEOUT : TTV_OK;
}

long long ttv_launch_count(void) { return g_launches.load(); }

void ttv_profile_enable(int on) { g_prof_on.store(on ? 1 : 0); }

int ttv_profile_collect(void) {
    std::lock_guard<std::mutex> g(g_prof_mu);
    for (auto& p : g_pending) {
        if (cudaEventSynchronize(p.b) != cudaSuccess) return TTV_ERR_CUDA;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, p.a, p.b);
        auto& t = g_totals[p.name];
        t.first += ms;
        t.second += 1;
        g_free_events.push_back(p.a);
        g_free_events.push_back(p.b);
    }
    g_pending.clear();
    return TTV_OK;
}

int ttv_profile_get(const char* kernel, double* total_ms, long long* launches) {
    std::lock_guard<std::mutex> g(g_prof_mu);
    auto it = g_totals.find(kernel ? kernel : "");
    if (it == g_totals.end()) {
        if (total_ms) *total_ms = 0.0;
        if (launches) *launches = 0;
        return TTV_ERR_ARG;
    }
    if (total_ms) *total_ms = it->second.first;
    if (launches) *launches = it->second.second;
    return TTV_OK;
}

int ttv_profile_names(char* buf, size_t len) {
    std::lock_guard<std::mutex> g(g_prof_mu);
    std::string all;
    for (auto& kv : g_totals) { all += kv.first; all += '\n'; }
    if (!buf || len == 0) return (int)all.size() + 1;
    strncpy(buf, all.c_str(), len - 1);
    buf[len - 1] = 0;
    return TTV_OK;
}

void ttv_profile_reset(void) {
    std::lock_guard<std::mutex> g(g_prof_mu);
    g_totals.clear();
}

}  // extern "C"
