// kv_serve.cu -- continuous-batching server over one context.
//
// Queries (a system plus a verification problem) are submitted from any host
// thread.  One worker thread owns the context: it admits queued queries in
// arrival order whenever a slot is free and the context pool can hold the
// query's system and problem (the memory model of Sec. 4.2-4.3 via kv_problem's
// reservation; a query that does not fit waits for a running one to finish),
// enqueues each admitted query's whole path on the slot's own stream -- so
// the kernels of different queries overlap on the device -- and, when a
// slot's completion event has fired, copies the results to host storage,
// releases the query's device memory and frees the slot for the next query.
// kv_poll hands a finished query's results to the caller.
//
// CSR systems are shared: queries naming the same host arrays (row_ptr, col,
// val, b) with the same n, symmetry and precision use one device copy, built
// when the first of them is admitted and kept while any query naming it is
// queued or running.  Building a CSR system (validation, upload, value
// conversion, the log-norm pass of Sec. 4.2) is host work of the worker
// thread, up to about a tenth of a second at n = 2e6, so a system that many
// queries verify is built once.  When the pool cannot hold an admission, the
// copies that no running query uses are released first and rebuilt on demand.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <tuple>
#include <thread>
#include <unordered_map>
#include <vector>

#include "kv_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

// Identity of a shared CSR system: the host arrays and the sizes and flags
// kv_system_csr takes.
using CsrKey = std::tuple<int64_t, const void*, const void*, const void*, const void*, int32_t, int32_t>;

struct SharedSys {
    kv_sys* sys = nullptr;  // device copy, nullptr until built (or after release); written by
                            // the worker under the server mutex
    int64_t refs = 0;       // queued + running queries naming it (under the server mutex)
    int64_t running = 0;    // running queries using the copy (worker thread only)
};

struct Request {
    uint64_t ticket = 0;
    kv_query q{};
    std::vector<kv_column> cols;
    Clock::time_point t_submit, t_admit, t_done;
    int status = KV_ENOTREADY;
    std::string error;
    // results (host)
    std::vector<double> lo, hi, zstar, beta0, err_bound;
    std::vector<int32_t> m_used;
    int32_t viol_step = -1, viol_row = -1;
    double ystar = 0.0;
    // while running
    kv_sys* sys = nullptr;  // owned by the request for grid systems, else shared->sys
    SharedSys* shared = nullptr;
    std::map<CsrKey, SharedSys>::iterator shared_it;
    kv_prob* prob = nullptr;
    int slot = -1;
};

}  // namespace

struct kv_server {
    kv_ctx* ctx = nullptr;
    cudaStream_t ctx_stream = nullptr;  // the context's own stream, restored on destroy
    int nslots = 0;
    std::vector<cudaStream_t> streams;
    std::vector<Request*> running;  // per slot
    std::deque<Request*> pending;
    std::unordered_map<uint64_t, Request*> all;
    std::map<CsrKey, SharedSys> systems;  // shared CSR systems, under mu
    std::mutex mu;
    std::condition_variable cv;
    std::thread worker;
    std::atomic<bool> stop{false};
    uint64_t next_ticket = 1;
    int64_t admitted = 0, completed = 0, waits_for_memory = 0;
    int64_t systems_built = 0, systems_reused = 0, systems_released = 0;
    int max_running = 0;
};

namespace {

int set_stream_and(kv_server* s, int slot) {
    s->ctx->stream = s->streams[slot];
    return KV_OK;
}

// Drops r's reference to its shared CSR system; the last reference releases
// the device copy and the entry.
void drop_shared(kv_server* s, Request* r) {
    kv_sys* dead = nullptr;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (--r->shared->refs == 0) {
            dead = r->shared->sys;
            s->systems.erase(r->shared_it);
        }
    }
    r->shared = nullptr;
    kv_sys_destroy(dead);
}

// Releases the device copies of the shared systems that no running query uses,
// except `keep`; a query naming one rebuilds it on admission.  Returns how many
// copies were released.
int release_idle_systems(kv_server* s, const SharedSys* keep) {
    std::vector<kv_sys*> idle;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (auto& kv : s->systems) {
            SharedSys& e = kv.second;
            if (&e != keep && e.sys && e.running == 0) {
                idle.push_back(e.sys);
                e.sys = nullptr;
            }
        }
        s->systems_released += (int64_t)idle.size();
    }
    for (kv_sys* x : idle) kv_sys_destroy(x);
    return (int)idle.size();
}

// Create (or take the shared copy of) the query's system and its problem on
// the slot's stream and enqueue it.  Returns KV_OK, KV_ENOMEM (does not fit
// now) or another error; on an error the request holds no device memory but
// its shared system's copy, which stays for the next attempt.
int admit(kv_server* s, Request* r, int slot) {
    set_stream_and(s, slot);
    const kv_query& q = r->q;
    int rc;
    bool reused = false;
    if (q.kind == 0) {
        rc = q.face ? kv_system_grid(s->ctx, &r->sys, q.ndim, q.dims, q.coef, q.h, q.face, q.b)
                    : kv_system_stencil(s->ctx, &r->sys, q.ndim, q.dims, q.coef, q.h, q.b);
        if (rc) return rc;
    } else {
        SharedSys* e = r->shared;
        reused = e->sys != nullptr;
        if (!reused) {
            kv_sys* built = nullptr;
            rc = kv_system_csr(s->ctx, &built, q.n, q.row_ptr, q.col, q.val, q.b, q.symmetric, q.precision, 0);
            if (rc) return rc;
            std::lock_guard<std::mutex> lk(s->mu);
            e->sys = built;
            s->systems_built++;
        }
        r->sys = e->sys;
    }
    auto release = [&]() {
        if (!r->shared) kv_sys_destroy(r->sys);
        r->sys = nullptr;
    };
    kv_problem_desc d = q.desc;
    d.cols = r->cols.data();
    rc = kv_problem(s->ctx, &r->prob, r->sys, &d, q.precision);
    if (rc) {
        release();
        return rc;
    }
    rc = kv_enqueue(r->prob);
    if (rc) {
        kv_prob_destroy(r->prob);
        r->prob = nullptr;
        release();
        return rc;
    }
    if (r->shared) {
        r->shared->running++;
        if (reused) {
            std::lock_guard<std::mutex> lk(s->mu);
            s->systems_reused++;
        }
    }
    r->slot = slot;
    r->t_admit = Clock::now();
    return KV_OK;
}

// Copies a finished query's results to host storage and releases its device
// memory; returns its status, which the caller publishes under the mutex
// (kv_poll reads the results only after seeing the status there).
int finish(kv_server* s, Request* r) {
    set_stream_and(s, r->slot);
    const kv_problem_desc& d = r->q.desc;
    const size_t S = (size_t)d.steps + 1;
    r->lo.assign((size_t)d.o * S, 0.0);
    r->hi.assign((size_t)d.o * S, 0.0);
    int32_t runs = d.i, transposed = 0;  // per-run arrays: o entries with the transpose dynamics
    kv_problem_runs(r->prob, &runs, &transposed);
    r->zstar.assign((size_t)d.i, 0.0);
    r->beta0.assign((size_t)runs, 0.0);
    r->m_used.assign((size_t)runs, 0);
    r->err_bound.assign((size_t)runs, 0.0);
    kv_result res{};
    res.lo = r->lo.data();
    res.hi = r->hi.data();
    res.z_star = r->zstar.data();
    res.beta0 = r->beta0.data();
    res.m_used = r->m_used.data();
    res.err_bound = r->err_bound.data();
    const int rc = kv_fetch(r->prob, &res);
    if (rc) r->error = kv_last_error();
    r->viol_step = res.first_violation_step;
    r->viol_row = res.violation_row;
    r->ystar = res.y_star;
    kv_prob_destroy(r->prob);
    r->prob = nullptr;
    if (r->shared) {
        r->shared->running--;
        drop_shared(s, r);
    } else {
        kv_sys_destroy(r->sys);
    }
    r->sys = nullptr;
    r->t_done = Clock::now();
    return rc;
}

void worker_loop(kv_server* s) {
    cudaSetDevice(s->ctx->device);
    while (true) {
        bool busy = false;
        // completions
        for (int k = 0; k < s->nslots; ++k) {
            Request* r = s->running[k];
            if (!r) continue;
            busy = true;
            if (cudaEventQuery(r->prob->done_ev) == cudaSuccess) {
                const int rc = finish(s, r);
                std::lock_guard<std::mutex> lk(s->mu);
                r->status = rc;
                s->running[k] = nullptr;
                s->completed++;
            }
        }
        // admissions, in arrival order
        while (true) {
            Request* r = nullptr;
            int slot = -1;
            {
                std::lock_guard<std::mutex> lk(s->mu);
                if (s->pending.empty()) break;
                for (int k = 0; k < s->nslots; ++k)
                    if (!s->running[k]) {
                        slot = k;
                        break;
                    }
                if (slot < 0) break;
                r = s->pending.front();
            }
            int rc = admit(s, r, slot);
            if (rc == KV_ENOMEM && release_idle_systems(s, r->shared) > 0) rc = admit(s, r, slot);
            std::unique_lock<std::mutex> lk(s->mu);
            if (rc == KV_OK) {
                s->pending.pop_front();
                s->running[slot] = r;
                s->admitted++;
                int nr = 0;
                for (auto* x : s->running) nr += x != nullptr;
                if (nr > s->max_running) s->max_running = nr;
                busy = true;
                continue;
            }
            bool any_running = false;
            for (auto* x : s->running) any_running |= x != nullptr;
            if (rc == KV_ENOMEM && any_running) {
                s->waits_for_memory++;  // wait for a running query to release memory
                break;
            }
            // cannot run even on an idle device, or another error: fail it
            s->pending.pop_front();
            r->error = kv_last_error();
            if (r->shared) {
                lk.unlock();
                drop_shared(s, r);
                lk.lock();
            }
            r->status = rc;
            r->t_done = Clock::now();
            s->completed++;
        }
        if (s->stop.load()) {
            bool idle = true;
            {
                std::lock_guard<std::mutex> lk(s->mu);
                for (auto* x : s->running) idle &= x == nullptr;
                idle &= s->pending.empty();
            }
            if (idle) break;
        }
        if (!busy) {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv.wait_for(lk, std::chrono::microseconds(200));
        } else {
            std::this_thread::sleep_for(std::chrono::microseconds(20));
        }
    }
}

}  // namespace

extern "C" {

int kv_server_create(kv_ctx* ctx, kv_server** out, int32_t slots) {
    if (!ctx || !out || slots < 1 || slots > 256) {
        kv::set_error("kv_server_create: bad arguments (slots in [1, 256])");
        return KV_EINVAL;
    }
    *out = nullptr;
    kv_server* s = new kv_server();
    s->ctx = ctx;
    s->ctx_stream = ctx->stream;
    s->nslots = slots;
    ::kv::DeviceGuard kv_device_guard_(ctx->device);
    for (int k = 0; k < slots; ++k) {
        cudaStream_t st;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            for (auto x : s->streams) cudaStreamDestroy(x);
            delete s;
            kv::set_error("kv_server_create: stream creation failed");
            return KV_ECUDA;
        }
        s->streams.push_back(st);
    }
    s->running.assign(slots, nullptr);
    s->worker = std::thread(worker_loop, s);
    *out = s;
    return KV_OK;
}

int kv_server_destroy(kv_server* s) {
    if (!s) return KV_OK;
    s->stop.store(true);
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    ::kv::DeviceGuard kv_device_guard_(s->ctx->device);
    for (auto& kv : s->all) delete kv.second;
    for (auto x : s->streams) cudaStreamSynchronize(x);
    for (auto& kv : s->systems) kv_sys_destroy(kv.second.sys);  // none once every query has finished
    s->systems.clear();
    s->ctx->stream = s->ctx_stream;
    for (auto x : s->streams) cudaStreamDestroy(x);
    delete s;
    return KV_OK;
}

int kv_submit(kv_server* s, const kv_query* q, uint64_t* ticket) {
    if (!s || !q || !ticket || q->desc.i < 1 || !q->desc.cols) {
        kv::set_error("kv_submit: bad arguments");
        return KV_EINVAL;
    }
    if (q->kind != 0 && q->kind != 1) {
        kv::set_error("kv_submit: kind must be 0 (grid) or 1 (CSR)");
        return KV_EINVAL;
    }
    Request* r = new Request();
    r->q = *q;
    r->cols.assign(q->desc.cols, q->desc.cols + q->desc.i);
    r->t_submit = Clock::now();
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop.load()) {
        delete r;
        kv::set_error("kv_submit: server is shutting down");
        return KV_EBUSY;
    }
    if (q->kind == 1) {
        const CsrKey key{q->n, q->row_ptr, q->col, q->val, q->b, q->symmetric, q->precision};
        r->shared_it = s->systems.try_emplace(key).first;
        r->shared = &r->shared_it->second;
        r->shared->refs++;
    }
    r->ticket = s->next_ticket++;
    s->all[r->ticket] = r;
    s->pending.push_back(r);
    *ticket = r->ticket;
    s->cv.notify_all();
    return KV_OK;
}

int kv_poll(kv_server* s, uint64_t ticket, kv_result* out, double* latency_ms) {
    if (!s || !out) {
        kv::set_error("kv_poll: NULL argument");
        return KV_EINVAL;
    }
    Request* r = nullptr;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->all.find(ticket);
        if (it == s->all.end()) {
            kv::set_error("kv_poll: unknown ticket %llu", (unsigned long long)ticket);
            return KV_EINVAL;
        }
        r = it->second;
        if (r->status == KV_ENOTREADY) return KV_ENOTREADY;
        if (r->status == KV_OK && (!out->lo || !out->hi)) {  // the result stays pollable
            kv::set_error("kv_poll: lo and hi are required");
            return KV_EINVAL;
        }
        s->all.erase(it);
    }
    const int rc = r->status;
    if (rc == KV_OK) {
        std::copy(r->lo.begin(), r->lo.end(), out->lo);
        std::copy(r->hi.begin(), r->hi.end(), out->hi);
        if (out->beta0) std::copy(r->beta0.begin(), r->beta0.end(), out->beta0);
        if (out->m_used) std::copy(r->m_used.begin(), r->m_used.end(), out->m_used);
        if (out->err_bound) std::copy(r->err_bound.begin(), r->err_bound.end(), out->err_bound);
        if (out->z_star && r->viol_step >= 0) std::copy(r->zstar.begin(), r->zstar.end(), out->z_star);
        out->first_violation_step = r->viol_step;
        out->violation_row = r->viol_row;
        out->y_star = r->ystar;
    } else {
        kv::set_error("%s", r->error.c_str());
    }
    if (latency_ms) latency_ms[0] = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
    delete r;
    return rc;
}

int kv_server_stats(kv_server* s, int64_t* admitted, int64_t* completed, int64_t* pending, int32_t* max_running,
                    int64_t* memory_waits) {
    if (!s) {
        kv::set_error("kv_server_stats: NULL server");
        return KV_EINVAL;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    if (admitted) *admitted = s->admitted;
    if (completed) *completed = s->completed;
    if (pending) *pending = (int64_t)s->pending.size();
    if (max_running) *max_running = s->max_running;
    if (memory_waits) *memory_waits = s->waits_for_memory;
    return KV_OK;
}

int kv_server_system_stats(kv_server* s, int64_t* built, int64_t* reused, int64_t* released, int64_t* resident) {
    if (!s) {
        kv::set_error("kv_server_system_stats: NULL server");
        return KV_EINVAL;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    if (built) *built = s->systems_built;
    if (reused) *reused = s->systems_reused;
    if (released) *released = s->systems_released;
    if (resident) {
        *resident = 0;
        for (auto& kv : s->systems) *resident += kv.second.sys != nullptr;
    }
    return KV_OK;
}

}  // extern "C"
