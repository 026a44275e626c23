// ttv_serve.cpp -- continuous-batching TTV server (host side of the C ABI).
//
// Tensors are registered once and stay resident in server-owned device
// memory (subscripts as one contiguous column per mode).  Clients submit TTV
// requests (contracted modes + host vectors); a scheduler thread admits
// queued requests whenever a stream slot is free and the memory budget
// allows the request's workspace, result and vectors, scanning past a request
// that does not fit yet so that smaller ones behind it can start.  Admitted
// requests run on their slot's stream, so the work of several requests
// overlaps on the GPU; completion is polled with events, results are handed
// to waiting clients, and latencies (submit to completion) feed the p50/p99
// statistics.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/ttv.h"

namespace ttv {
int fail(int code, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);
int batch_run_direct(const ttv_problem* probs, int32_t n, ttv_out* outs, const ttv_opts* o, cudaStream_t stream);
void out_detach_stream(ttv_out* out);
}  // namespace ttv

namespace {

using Clock = std::chrono::steady_clock;

struct PreparedModes {
    uint32_t mask = 0;               // contracted modes
    std::vector<int32_t> modes;      // in the order given to ttv_prepare
    ttv_prepared* h = nullptr;
    size_t bytes = 0;
};

struct Resident {
    int64_t* subs = nullptr;     // d columns of nnz
    void* vals = nullptr;
    ttv_dtype val_dtype = TTV_F64;
    int64_t nnz = 0;
    int32_t d = 0;
    int64_t shape[TTV_MAX_D] = {0};
    size_t bytes = 0;
    std::vector<std::shared_ptr<PreparedModes>> prepared;
};

struct Request {
    uint64_t id = 0;
    int32_t tensor = 0;
    std::vector<int32_t> modes;
    std::vector<unsigned char> vecs;          // packed host vectors
    std::vector<size_t> vec_off;
    ttv_dtype v_dtype = TTV_F64;
    ttv_opts opts{};
    size_t need = 0;                          // admission estimate (bytes)
    size_t res_bytes = 0;                     // the result's part of it, held from completion until claimed
    int64_t nnz = 0;
    Clock::time_point submitted;
    // in flight
    int slot = -1;
    void* dvecs = nullptr;
    ttv_out out{};
    int rc = TTV_OK;
    std::string msg;                          // the library's message when rc != TTV_OK
    bool done = false;
    double latency_us = 0;
};

// A slot runs one request, or a group of requests as one stage-wise batch
// (ttv::batch_run_direct) when more are queued than slots are free.
struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    void* pinned = nullptr;
    size_t pinned_bytes = 0;
    std::shared_ptr<Request> req;
    std::vector<std::shared_ptr<Request>> group;
    void* gvecs = nullptr;                    // the group's vectors, one device block
    bool busy() const { return (bool)req || !group.empty(); }
};

constexpr size_t kGroupMax = 32;              // requests per group

}  // namespace

struct ttv_server {
    size_t budget = 0;
    std::atomic<size_t> in_use{0};
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Request>> queue;
    std::map<uint64_t, std::shared_ptr<Request>> finished;
    std::map<uint64_t, std::shared_ptr<Request>> running;
    std::vector<Slot> slots;
    std::vector<Resident> tensors;
    std::vector<double> lat_us;
    uint64_t next_id = 1;
    long long admitted = 0, refused = 0, completed = 0, prepared_runs = 0, grouped_runs = 0;
    double nnz_done = 0;
    Clock::time_point t0;
    bool stop = false;
    std::thread sched;
};

namespace {

void free_resident(Resident& r) {
    if (r.subs) cudaFree(r.subs);
    if (r.vals) cudaFree(r.vals);
    r.subs = nullptr;
    r.vals = nullptr;
    for (auto& pm : r.prepared) ttv_prepared_free(pm->h);
    r.prepared.clear();
}

// Finishes one request of a slot whose event has completed.
void complete_one(ttv_server* s, Slot& sl, const std::shared_ptr<Request>& r) {
    if (r->rc == TTV_OK) {
        r->rc = ttv_out_sync(&r->out);
        if (r->rc != TTV_OK) r->msg = ttv_last_error();
    }
    // the slot's work for this result is complete (its event): the client may
    // release the result after the server, and so the slot stream, are gone
    ttv::out_detach_stream(&r->out);
    // the result now belongs to the client: its buffers must not be touched here
    if (r->dvecs) cudaFreeAsync(r->dvecs, sl.stream);
    r->latency_us = std::chrono::duration<double, std::micro>(Clock::now() - r->submitted).count();
    std::lock_guard<std::mutex> g(s->mu);
    // From completion until the client claims it, only the result counts
    // against the budget.  A client waiting by id for a request that the
    // unclaimed results keep out still progresses: with nothing running, the
    // oldest queued request is admitted over the budget (the scheduler).
    s->in_use -= r->need;
    s->in_use += r->res_bytes;
    r->done = true;
    s->running.erase(r->id);
    s->finished[r->id] = r;
    s->lat_us.push_back(r->latency_us);
    s->completed += 1;
    s->nnz_done += (double)r->nnz;
    s->cv_done.notify_all();
    s->cv_work.notify_all();
}

void complete(ttv_server* s, Slot& sl) {
    if (sl.req) {
        std::shared_ptr<Request> r = sl.req;
        sl.req.reset();
        complete_one(s, sl, r);
        return;
    }
    std::vector<std::shared_ptr<Request>> g;
    g.swap(sl.group);
    if (sl.gvecs) cudaFreeAsync(sl.gvecs, sl.stream);
    sl.gvecs = nullptr;
    for (const auto& r : g) complete_one(s, sl, r);
}

// Starts a request on a free slot (scheduler thread, lock not held).
void start(ttv_server* s, Slot& sl, const std::shared_ptr<Request>& r) {
    sl.req = r;
    r->slot = (int)(&sl - s->slots.data());
    Resident t;
    std::shared_ptr<PreparedModes> prep;
    {
        std::lock_guard<std::mutex> g(s->mu);
        t = s->tensors[(size_t)r->tensor];
    }
    if ((r->opts.accum == TTV_ACCUM_FP64 || r->opts.accum == TTV_ACCUM_COMPENSATED) &&
        r->opts.path == TTV_PATH_AUTO && !r->opts.deterministic) {
        uint32_t mask = 0;
        for (int32_t m : r->modes) mask |= 1u << m;
        for (auto& pm : t.prepared)
            if (pm->mask == mask) prep = pm;
    }
    const size_t vbytes = r->vecs.size();
    if (sl.pinned_bytes < vbytes) {
        if (sl.pinned) cudaFreeHost(sl.pinned);
        sl.pinned_bytes = std::max<size_t>(vbytes, 1 << 16);
        if (cudaHostAlloc(&sl.pinned, sl.pinned_bytes, cudaHostAllocDefault) != cudaSuccess) {
            sl.pinned = nullptr;
            sl.pinned_bytes = 0;
        }
    }
    cudaError_t e = cudaSuccess;
    if (vbytes) {
        e = cudaMallocAsync(&r->dvecs, vbytes, sl.stream);
        if (e == cudaSuccess) {
            if (sl.pinned) {
                memcpy(sl.pinned, r->vecs.data(), vbytes);
                e = cudaMemcpyAsync(r->dvecs, sl.pinned, vbytes, cudaMemcpyHostToDevice, sl.stream);
            } else {
                e = cudaMemcpyAsync(r->dvecs, r->vecs.data(), vbytes, cudaMemcpyHostToDevice, sl.stream);
            }
        }
    }
    if (e != cudaSuccess) {
        r->rc = ttv::cuda_fail(e, "request vectors");
        r->msg = ttv_last_error();
    } else {
        std::vector<const void*> vp(r->modes.size());
        std::vector<int64_t> lens(r->modes.size());
        for (size_t i = 0; i < r->modes.size(); ++i) {
            vp[i] = static_cast<char*>(r->dvecs) + r->vec_off[i];
            lens[i] = t.shape[r->modes[i]];
        }
        ttv_tensor tt;
        tt.subs = t.subs;
        tt.stride_nz = 1;
        tt.stride_mode = t.nnz;
        tt.vals = t.vals;
        tt.val_dtype = t.val_dtype;
        tt.nnz = t.nnz;
        tt.shape = t.shape;
        tt.d = t.d;
        memset(&r->out, 0, sizeof r->out);
        ttv_opts o = r->opts;
        o.async = 1;
        o.workspace = nullptr;
        o.workspace_bytes = 0;
        if (prep) {
            // vectors in the order the layout was prepared with
            std::vector<const void*> pv(prep->modes.size());
            std::vector<int64_t> pl(prep->modes.size());
            for (size_t k = 0; k < prep->modes.size(); ++k)
                for (size_t i = 0; i < r->modes.size(); ++i)
                    if (r->modes[i] == prep->modes[k]) {
                        pv[k] = vp[i];
                        pl[k] = lens[i];
                    }
            r->rc = ttv_prepared_run(prep->h, pv.data(), pl.data(), r->v_dtype, &r->out, &o,
                                     reinterpret_cast<ttv_stream_t>(sl.stream));
            if (r->rc != TTV_OK) r->msg = ttv_last_error();
            std::lock_guard<std::mutex> g(s->mu);
            s->prepared_runs += 1;
        } else {
            r->rc = ttv_multi_checked(&tt, r->modes.data(), (int32_t)r->modes.size(), vp.data(), lens.data(),
                                      r->v_dtype, &r->out, &o, reinterpret_cast<ttv_stream_t>(sl.stream));
            if (r->rc != TTV_OK) r->msg = ttv_last_error();
        }
    }
    cudaEventRecord(sl.done, sl.stream);
}

// Whether a request runs on a prepared layout (the single-request path);
// called with the server's lock held.
bool uses_prepared(const ttv_server* s, const Request& r) {
    if (!((r.opts.accum == TTV_ACCUM_FP64 || r.opts.accum == TTV_ACCUM_COMPENSATED) &&
          r.opts.path == TTV_PATH_AUTO && !r.opts.deterministic))
        return false;
    uint32_t mask = 0;
    for (int32_t m : r.modes) mask |= 1u << m;
    for (const auto& pm : s->tensors[(size_t)r.tensor].prepared)
        if (pm->mask == mask) return true;
    return false;
}

// Requests that may share a group: the same options (one batch takes one
// set) and the same vector type.
bool same_kind(const Request& a, const Request& b) {
    return a.opts.fmt == b.opts.fmt && a.opts.path == b.opts.path && a.opts.accum == b.opts.accum &&
           a.opts.deterministic == b.opts.deterministic && a.v_dtype == b.v_dtype;
}

// Starts a group of requests on a free slot as one stage-wise batch
// (scheduler thread, lock not held): their vectors in one upload, then
// ttv::batch_run_direct on the slot's stream.
void start_group(ttv_server* s, Slot& sl) {
    std::vector<std::shared_ptr<Request>>& g = sl.group;
    const size_t n = g.size();
    std::vector<Resident> ts(n);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (size_t k = 0; k < n; ++k) ts[k] = s->tensors[(size_t)g[k]->tensor];
    }
    for (size_t k = 0; k < n; ++k) g[k]->slot = (int)(&sl - s->slots.data());
    std::vector<size_t> base(n);
    size_t vbytes = 0;
    for (size_t k = 0; k < n; ++k) {
        base[k] = vbytes;
        vbytes += (g[k]->vecs.size() + 255) & ~size_t(255);
    }
    if (sl.pinned_bytes < vbytes) {
        if (sl.pinned) cudaFreeHost(sl.pinned);
        sl.pinned_bytes = std::max<size_t>(vbytes, 1 << 16);
        if (cudaHostAlloc(&sl.pinned, sl.pinned_bytes, cudaHostAllocDefault) != cudaSuccess) {
            sl.pinned = nullptr;
            sl.pinned_bytes = 0;
        }
    }
    cudaError_t e = cudaMallocAsync(&sl.gvecs, std::max<size_t>(vbytes, 256), sl.stream);
    if (e == cudaSuccess) {
        if (sl.pinned) {
            for (size_t k = 0; k < n; ++k) memcpy(static_cast<char*>(sl.pinned) + base[k], g[k]->vecs.data(), g[k]->vecs.size());
            e = cudaMemcpyAsync(sl.gvecs, sl.pinned, vbytes, cudaMemcpyHostToDevice, sl.stream);
        } else {
            for (size_t k = 0; k < n && e == cudaSuccess; ++k)
                e = cudaMemcpyAsync(static_cast<char*>(sl.gvecs) + base[k], g[k]->vecs.data(), g[k]->vecs.size(),
                                    cudaMemcpyHostToDevice, sl.stream);
        }
    } else {
        sl.gvecs = nullptr;
    }
    int rc = TTV_OK;
    std::string msg;
    if (e != cudaSuccess) {
        rc = ttv::cuda_fail(e, "request vectors");
        msg = ttv_last_error();
    } else {
        std::vector<ttv_problem> probs(n);
        std::vector<std::vector<const void*>> vps(n);
        std::vector<ttv_out> outs(n);
        for (size_t k = 0; k < n; ++k) {
            const Request& r = *g[k];
            vps[k].resize(r.modes.size());
            for (size_t i = 0; i < r.modes.size(); ++i)
                vps[k][i] = static_cast<char*>(sl.gvecs) + base[k] + r.vec_off[i];
            ttv_tensor& tt = probs[k].tensor;
            tt.subs = ts[k].subs;
            tt.stride_nz = 1;
            tt.stride_mode = ts[k].nnz;
            tt.vals = ts[k].vals;
            tt.val_dtype = ts[k].val_dtype;
            tt.nnz = ts[k].nnz;
            tt.shape = ts[k].shape;
            tt.d = ts[k].d;
            probs[k].modes = r.modes.data();
            probs[k].n_v = (int32_t)r.modes.size();
            probs[k].vecs = vps[k].data();
            probs[k].v_dtype = r.v_dtype;
            memset(&outs[k], 0, sizeof outs[k]);
        }
        ttv_opts o = g[0]->opts;
        o.async = 1;
        o.workspace = nullptr;
        o.workspace_bytes = 0;
        rc = ttv::batch_run_direct(probs.data(), (int32_t)n, outs.data(), &o, sl.stream);
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->grouped_runs += (long long)n;
        }
        if (rc != TTV_OK) msg = ttv_last_error();
        for (size_t k = 0; k < n; ++k) g[k]->out = outs[k];
    }
    for (size_t k = 0; k < n; ++k) {
        g[k]->rc = rc;
        g[k]->msg = msg;
    }
    cudaEventRecord(sl.done, sl.stream);
}

void scheduler(ttv_server* s) {
    cudaSetDevice(s->device);
    // While requests run, completions are polled without sleeping (a short
    // sleep rounds up to the kernel's timer slack, tens of microseconds,
    // which light-load latency would pay on every request); after this long
    // without any completion or admission the loop backs off to short sleeps.
    const auto spin_limit = std::chrono::microseconds(500);
    Clock::time_point last_event = Clock::now();
    for (;;) {
        // completions (an error state also ends the request: it is reported, never waited on)
        for (Slot& sl : s->slots) {
            if (!sl.busy()) continue;
            const cudaError_t q = cudaEventQuery(sl.done);
            if (q == cudaErrorNotReady) continue;
            if (q != cudaSuccess) {
                const int rc = ttv::cuda_fail(q, "request");
                const std::string msg = ttv_last_error();
                if (sl.req && sl.req->rc == TTV_OK) {
                    sl.req->rc = rc;
                    sl.req->msg = msg;
                }
                for (auto& r : sl.group)
                    if (r->rc == TTV_OK) {
                        r->rc = rc;
                        r->msg = msg;
                    }
            }
            complete(s, sl);
            last_event = Clock::now();
        }
        std::unique_lock<std::mutex> lk(s->mu);
        if (s->stop && s->queue.empty()) {
            bool busy = false;
            for (Slot& sl : s->slots) busy |= sl.busy();
            if (!busy) return;
        }
        // admissions: any queued request that fits, in submission order; the
        // picks are made under the lock, the launches after releasing it.
        // While no more requests wait than slots are free, each runs on its
        // own slot; beyond that, a free slot takes a group of requests of the
        // same kind (up to kGroupMax, about the queue over the free slots),
        // which runs as one stage-wise batch.
        size_t nfree = 0;
        for (Slot& sl : s->slots) nfree += sl.busy() ? 0 : 1;
        const size_t per_slot =
            nfree ? std::min<size_t>(kGroupMax, std::max<size_t>(1, (s->queue.size() + nfree - 1) / nfree)) : 1;
        std::vector<std::pair<Slot*, std::shared_ptr<Request>>> picks;
        std::vector<Slot*> group_picks;
        for (auto it = s->queue.begin(); it != s->queue.end();) {
            Slot* free_slot = nullptr;
            for (Slot& sl : s->slots)
                if (!sl.busy()) { free_slot = &sl; break; }
            if (!free_slot) break;
            const std::shared_ptr<Request> r = *it;
            if (s->in_use + r->need > s->budget) {
                bool idle = picks.empty() && group_picks.empty();
                for (Slot& sl : s->slots) idle = idle && !sl.busy();
                if (!(idle && it == s->queue.begin())) { ++it; continue; }
            }
            s->in_use += r->need;
            s->admitted += 1;
            s->running[r->id] = r;
            it = s->queue.erase(it);
            if (per_slot == 1 || uses_prepared(s, *r)) {
                free_slot->req = r;              // reserved
                picks.emplace_back(free_slot, r);
                continue;
            }
            // a group: r and the next admissible requests of its kind (erasing
            // from the middle of a deque invalidates its iterators: the scan
            // goes on from the front, where only requests that did not fit
            // the budget remain before r's successors)
            // A group holds at most a slot's share of the budget (or its
            // first request, if that is larger): one slot's group allocates
            // its workspace as one block, and groups of large requests would
            // otherwise hold many times the memory of the same requests
            // running one per slot.
            free_slot->group.push_back(r);   // reserved
            const size_t gcap = std::max(r->need, s->budget / s->slots.size());
            size_t gneed = r->need;
            for (auto jt = s->queue.begin(); jt != s->queue.end() && free_slot->group.size() < per_slot;) {
                const std::shared_ptr<Request> q = *jt;
                if (!same_kind(*r, *q) || uses_prepared(s, *q) || s->in_use + q->need > s->budget ||
                    gneed + q->need > gcap) {
                    ++jt;
                    continue;
                }
                gneed += q->need;
                s->in_use += q->need;
                s->admitted += 1;
                s->running[q->id] = q;
                free_slot->group.push_back(q);
                jt = s->queue.erase(jt);
            }
            it = s->queue.begin();
            group_picks.push_back(free_slot);
        }
        const bool started = !picks.empty() || !group_picks.empty();
        if (started) {
            lk.unlock();
            for (auto& pr : picks) start(s, *pr.first, pr.second);
            for (Slot* sl : group_picks) {
                if (sl->group.size() == 1) {
                    // a group of one: the single-request path
                    std::shared_ptr<Request> r = sl->group[0];
                    sl->group.clear();
                    start(s, *sl, r);
                } else {
                    start_group(s, *sl);
                }
            }
            lk.lock();
        }
        bool any_running = false;
        for (Slot& sl : s->slots) any_running |= sl.busy();
        if (started) {
            last_event = Clock::now();
        } else if (any_running) {
            lk.unlock();
            if (Clock::now() - last_event < spin_limit) std::this_thread::yield();
            else std::this_thread::sleep_for(std::chrono::microseconds(20));
        } else {
            s->cv_work.wait_for(lk, std::chrono::milliseconds(2));
            last_event = Clock::now();
        }
    }
}

double percentile(std::vector<double> v, double q) {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const double pos = q * (double)(v.size() - 1);
    const size_t i = (size_t)pos;
    const double f = pos - (double)i;
    return i + 1 < v.size() ? v[i] * (1 - f) + v[i + 1] * f : v[i];
}

}  // namespace

extern "C" {

int ttv_server_create(size_t budget_bytes, int32_t n_slots, ttv_server** out) {
    if (!out || n_slots < 1 || n_slots > 64 || budget_bytes == 0) return ttv::fail(TTV_ERR_ARG, "bad server arguments");
    ttv_server* s = new ttv_server();
    s->budget = budget_bytes;
    cudaGetDevice(&s->device);
    s->slots.resize((size_t)n_slots);
    for (Slot& sl : s->slots) {
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess) {
            ttv_server_destroy(s);
            return ttv::fail(TTV_ERR_CUDA, "server streams");
        }
    }
    s->t0 = Clock::now();
    s->sched = std::thread(scheduler, s);
    *out = s;
    return TTV_OK;
}

int ttv_server_register(ttv_server* s, const ttv_tensor* t, int32_t* tensor_id) {
    if (!s || !t || !tensor_id || t->d < 1 || t->d > TTV_MAX_D || t->nnz < 0 || !t->shape)
        return ttv::fail(TTV_ERR_ARG, "bad tensor");
    Resident r;
    r.nnz = t->nnz;
    r.d = t->d;
    r.val_dtype = t->val_dtype;
    for (int m = 0; m < t->d; ++m) r.shape[m] = t->shape[m];
    const size_t vb = t->val_dtype == TTV_F32 ? 4 : 8;
    r.bytes = (size_t)std::max<int64_t>(t->nnz, 1) * ((size_t)t->d * 8 + vb);
    {
        std::lock_guard<std::mutex> g(s->mu);
        if (s->in_use + r.bytes > s->budget) return ttv::fail(TTV_ERR_BUDGET, "tensor does not fit the budget");
        s->in_use += r.bytes;
    }
    cudaError_t e = cudaMalloc(&r.subs, (size_t)std::max<int64_t>(t->nnz, 1) * t->d * 8);
    if (e == cudaSuccess) e = cudaMalloc(&r.vals, (size_t)std::max<int64_t>(t->nnz, 1) * vb);
    if (e == cudaSuccess && t->nnz > 0) {
        for (int m = 0; m < t->d && e == cudaSuccess; ++m)
            e = cudaMemcpy2D(r.subs + (size_t)m * t->nnz, 8, t->subs + (size_t)m * t->stride_mode,
                             (size_t)t->stride_nz * 8, 8, (size_t)t->nnz, cudaMemcpyDeviceToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(r.vals, t->vals, (size_t)t->nnz * vb, cudaMemcpyDeviceToDevice);
    }
    if (e != cudaSuccess) {
        free_resident(r);
        std::lock_guard<std::mutex> g(s->mu);
        s->in_use -= r.bytes;
        return ttv::cuda_fail(e, "register");
    }
    std::lock_guard<std::mutex> g(s->mu);
    s->tensors.push_back(r);
    *tensor_id = (int32_t)s->tensors.size() - 1;
    return TTV_OK;
}

int ttv_server_prepare(ttv_server* s, int32_t tensor_id, const int32_t* modes, int32_t n_v) {
    if (!s || !modes || n_v < 1 || n_v > TTV_MAX_D) return ttv::fail(TTV_ERR_ARG, "bad prepare request");
    Resident t;
    {
        std::lock_guard<std::mutex> g(s->mu);
        if (tensor_id < 0 || (size_t)tensor_id >= s->tensors.size()) return ttv::fail(TTV_ERR_ARG, "unknown tensor");
        t = s->tensors[(size_t)tensor_id];
    }
    ttv_tensor tt;
    tt.subs = t.subs;
    tt.stride_nz = 1;
    tt.stride_mode = t.nnz;
    tt.vals = t.vals;
    tt.val_dtype = t.val_dtype;
    tt.nnz = t.nnz;
    tt.shape = t.shape;
    tt.d = t.d;
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess)
        return ttv::fail(TTV_ERR_CUDA, "prepare stream");
    ttv_prepared* h = nullptr;
    int rc = ttv_prepare(&tt, modes, n_v, &h, reinterpret_cast<ttv_stream_t>(st));
    cudaStreamDestroy(st);
    if (rc != TTV_OK) return rc;
    auto pm = std::make_shared<PreparedModes>();
    pm->h = h;
    pm->modes.assign(modes, modes + n_v);
    for (int32_t i = 0; i < n_v; ++i) pm->mask |= 1u << modes[i];
    ttv_prepared_info(h, nullptr, nullptr, &pm->bytes);
    std::lock_guard<std::mutex> g(s->mu);
    if (s->in_use + pm->bytes > s->budget) {
        ttv_prepared_free(h);
        return ttv::fail(TTV_ERR_BUDGET, "prepared layout (%zu bytes) does not fit the budget", pm->bytes);
    }
    s->in_use += pm->bytes;
    s->tensors[(size_t)tensor_id].bytes += pm->bytes;
    s->tensors[(size_t)tensor_id].prepared.push_back(pm);
    return TTV_OK;
}

int ttv_server_submit(ttv_server* s, int32_t tensor_id, const int32_t* modes, int32_t n_v,
                      const void* const* host_vecs, ttv_dtype v_dtype, const ttv_opts* opts, uint64_t* req_id) {
    if (!s || !modes || !host_vecs || !req_id || n_v < 1) return ttv::fail(TTV_ERR_ARG, "bad request");
    auto r = std::make_shared<Request>();
    Resident t;
    {
        std::lock_guard<std::mutex> g(s->mu);
        if (tensor_id < 0 || (size_t)tensor_id >= s->tensors.size()) return ttv::fail(TTV_ERR_ARG, "unknown tensor");
        t = s->tensors[(size_t)tensor_id];
    }
    if (opts) r->opts = *opts;
    else ttv_opts_init(&r->opts);
    r->tensor = tensor_id;
    r->v_dtype = v_dtype;
    r->nnz = t.nnz;
    const size_t eb = v_dtype == TTV_F32 ? 4 : 8;
    size_t off = 0;
    for (int32_t i = 0; i < n_v; ++i) {
        const int32_t m = modes[i];
        if (m < 0 || m >= t.d) return ttv::fail(TTV_ERR_MODE, "mode %d outside 0..%d", m, t.d - 1);
        r->modes.push_back(m);
        r->vec_off.push_back(off);
        off += ((size_t)t.shape[m] * eb + 255) & ~size_t(255);
    }
    r->vecs.resize(off);
    for (int32_t i = 0; i < n_v; ++i)
        memcpy(r->vecs.data() + r->vec_off[(size_t)i], host_vecs[i], (size_t)t.shape[modes[i]] * eb);
    // admission estimate: workspace + result + vectors
    ttv_tensor tt;
    tt.subs = t.subs;
    tt.stride_nz = 1;
    tt.stride_mode = t.nnz;
    tt.vals = t.vals;
    tt.val_dtype = t.val_dtype;
    tt.nnz = t.nnz;
    tt.shape = t.shape;
    tt.d = t.d;
    size_t ws = 0;
    int64_t rows = 0, nvals = 0;
    int rc = ttv_workspace_size(&tt, modes, n_v, v_dtype, &r->opts, &ws);
    if (rc == TTV_OK) rc = ttv_out_capacity(&tt, modes, n_v, &r->opts, &rows, &nvals);
    if (rc != TTV_OK) return rc;
    r->res_bytes = (size_t)rows * (size_t)(t.d - n_v) * 8 + (size_t)nvals * 8;
    r->need = ws + r->res_bytes + off;
    std::lock_guard<std::mutex> g(s->mu);
    size_t resident = 0;
    for (const Resident& x : s->tensors) resident += x.bytes;
    if (r->need + resident > s->budget) {
        s->refused += 1;
        return ttv::fail(TTV_ERR_BUDGET, "request needs %zu bytes beyond the resident tensors", r->need);
    }
    r->id = s->next_id++;
    r->submitted = Clock::now();
    s->queue.push_back(r);
    *req_id = r->id;
    s->cv_work.notify_all();
    return TTV_OK;
}

int ttv_server_wait(ttv_server* s, uint64_t req_id, int64_t timeout_us, ttv_out* out) {
    if (!s || !out) return ttv::fail(TTV_ERR_ARG, "bad wait");
    std::unique_lock<std::mutex> lk(s->mu);
    auto ready = [&] { return s->finished.count(req_id) > 0; };
    if (timeout_us < 0) {
        s->cv_done.wait(lk, ready);
    } else if (!s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready)) {
        return ttv::fail(TTV_ERR_TIMEOUT, "request %llu not finished", (unsigned long long)req_id);
    }
    std::shared_ptr<Request> r = s->finished[req_id];
    s->finished.erase(req_id);
    s->in_use -= r->res_bytes;
    s->cv_work.notify_all();
    *out = r->out;                       // ownership of the result moves to the caller
    memset(&r->out, 0, sizeof r->out);
    if (r->rc != TTV_OK)
        return ttv::fail(r->rc, "request %llu failed (%d): %s", (unsigned long long)req_id, r->rc, r->msg.c_str());
    return TTV_OK;
}

int ttv_server_wait_any(ttv_server* s, int64_t timeout_us, uint64_t* req_id, ttv_out* out) {
    if (!s || !out || !req_id) return ttv::fail(TTV_ERR_ARG, "bad wait");
    std::unique_lock<std::mutex> lk(s->mu);
    auto ready = [&] { return !s->finished.empty(); };
    if (timeout_us < 0) {
        s->cv_done.wait(lk, ready);
    } else if (!s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready)) {
        return ttv::fail(TTV_ERR_TIMEOUT, "no request finished");
    }
    auto it = s->finished.begin();           // the oldest finished request
    std::shared_ptr<Request> r = it->second;
    s->finished.erase(it);
    s->in_use -= r->res_bytes;
    s->cv_work.notify_all();
    *req_id = r->id;
    *out = r->out;                           // ownership of the result moves to the caller
    memset(&r->out, 0, sizeof r->out);
    if (r->rc != TTV_OK)
        return ttv::fail(r->rc, "request %llu failed (%d): %s", (unsigned long long)r->id, r->rc, r->msg.c_str());
    return TTV_OK;
}

int ttv_server_stats(ttv_server* s, ttv_stats* st) {
    if (!s || !st) return ttv::fail(TTV_ERR_ARG, "bad stats");
    std::lock_guard<std::mutex> g(s->mu);
    memset(st, 0, sizeof *st);
    st->p50_us = percentile(s->lat_us, 0.50);
    st->p99_us = percentile(s->lat_us, 0.99);
    double sum = 0, mx = 0;
    for (double v : s->lat_us) { sum += v; mx = std::max(mx, v); }
    st->mean_us = s->lat_us.empty() ? 0 : sum / (double)s->lat_us.size();
    st->max_us = mx;
    st->completed = s->completed;
    st->admitted = s->admitted;
    st->refused = s->refused;
    st->pending = (long long)s->queue.size() + (long long)s->running.size();
    const double secs = std::chrono::duration<double>(Clock::now() - s->t0).count();
    st->seconds = secs;
    st->throughput_rps = secs > 0 ? (double)s->completed / secs : 0;
    st->throughput_gnnz_s = secs > 0 ? s->nnz_done / secs / 1e9 : 0;
    st->bytes_in_use = s->in_use;
    st->budget_bytes = s->budget;
    st->prepared_runs = s->prepared_runs;
    st->grouped_runs = s->grouped_runs;
    return TTV_OK;
}

int ttv_server_reset_stats(ttv_server* s) {
    if (!s) return ttv::fail(TTV_ERR_ARG, "bad server");
    std::lock_guard<std::mutex> g(s->mu);
    s->lat_us.clear();
    s->completed = 0;
    s->admitted = 0;
    s->refused = 0;
    s->prepared_runs = 0;
    s->grouped_runs = 0;
    s->nnz_done = 0;
    s->t0 = Clock::now();
    return TTV_OK;
}

void ttv_server_destroy(ttv_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stop = true;
        s->queue.clear();
        s->cv_work.notify_all();
    }
    if (s->sched.joinable()) s->sched.join();
    for (auto& kv : s->finished) ttv_out_free(&kv.second->out);
    for (Slot& sl : s->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.pinned) cudaFreeHost(sl.pinned);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    for (Resident& r : s->tensors) free_resident(r);
    delete s;
}

}  // extern "C"
