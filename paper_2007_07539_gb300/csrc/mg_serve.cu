// Concurrent batch solves and the serving engine of libmgfp
// (mg_solve_batch, mg_submit, mg_poll, mg_serve_configure).
//
// Both drive the per-solve IR state machine of mg_host.cu without blocking:
// each hierarchy has its own stream, every solve keeps one action in flight,
// and a host loop advances whichever solve's state event has completed.  So
// the kernels of different solves overlap on the device, and in the serving
// engine new requests start while others are running ("continuous
// batching"): a queued request is admitted as soon as its hierarchy is idle,
// a slot is free (max_inflight) and its working-set bytes fit the memory
// budget next to the requests already in flight.
#include <cuda_runtime.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "mg_host.h"

using namespace mgi;

// ---------------------------------------------------------------- batch
mg_status mgi_batch_run(std::vector<mgi_hier*>& hs, const double* const* b, double* const* u, mg_result* res) {
    const int n = (int)hs.size();
    std::vector<int> state(n, 0);  // 0 running, 1 done, 2 failed
    mg_status first_bad = MG_OK;
    int active = 0;
    for (int i = 0; i < n; ++i) {
        cudaSetDevice(hs[i]->device);
        mg_status st = mgi_solve_begin(*hs[i], b[i], u[i]);
        if (st != MG_OK) {
            state[i] = 2;
            if (res) { res[i] = mg_result{}; res[i].status = st; }
            if (first_bad == MG_OK) first_bad = st;
        } else {
            ++active;
        }
    }
    while (active > 0) {
        bool progressed = false;
        for (int i = 0; i < n; ++i) {
            if (state[i] != 0) continue;
            cudaError_t q = cudaEventQuery(hs[i]->ev_state);
            if (q == cudaErrorNotReady) continue;
            int rc;
            if (q != cudaSuccess) {
                mgi_set_error(std::string("batch: ") + cudaGetErrorString(q));
                rc = -MG_ERR_CUDA;
            } else {
                rc = mgi_solve_advance(*hs[i]);
            }
            progressed = true;
            if (rc == 0) continue;
            --active;
            state[i] = rc == 1 ? 1 : 2;
            mg_result r = hs[i]->ctx.res;
            if (rc < 0) r.status = -rc;
            if (res) res[i] = r;
            if (r.status != MG_OK && first_bad == MG_OK) first_bad = (mg_status)r.status;
        }
        if (!progressed) std::this_thread::yield();
    }
    return first_bad;
}

// ---------------------------------------------------------------- serving engine
namespace {

struct Req {
    uint64_t ticket = 0;
    mgi_hier* h = nullptr;
    const double* b = nullptr;
    double* u = nullptr;
    int state = 0;  // 0 queued, 1 running, 2 done
    size_t bytes = 0;
    mg_result res{};
};

struct Engine {
    std::mutex mu;
    std::condition_variable cv;      // wakes the worker (new work)
    std::condition_variable done_cv; // wakes waiters (request finished)
    bool started = false;
    bool configured = false;
    size_t budget = 0;
    int max_inflight = 16;
    size_t used = 0;
    uint64_t next_ticket = 1;
    std::deque<Req*> queue;
    std::vector<Req*> running;
    std::unordered_map<uint64_t, Req*> all;
    std::unordered_map<mgi_hier*, int> pending;
    std::unordered_set<mgi_hier*> busy;
};

Engine& engine() {
    static Engine* e = new Engine();  // never destroyed: the worker thread is detached
    return *e;
}

void finish(Engine& E, Req* r, const mg_result& res) {
    r->res = res;
    r->state = 2;
    E.used -= r->bytes;
    E.busy.erase(r->h);
    E.pending[r->h] -= 1;
    for (size_t i = 0; i < E.running.size(); ++i)
        if (E.running[i] == r) { E.running.erase(E.running.begin() + i); break; }
    E.done_cv.notify_all();
}

void worker() {
    Engine& E = engine();
    for (;;) {
        std::vector<Req*> to_begin, snapshot;
        {
            std::unique_lock<std::mutex> lk(E.mu);
            if (E.queue.empty() && E.running.empty())
                E.cv.wait(lk, [&] { return !E.queue.empty() || !E.running.empty(); });
            for (auto it = E.queue.begin(); it != E.queue.end();) {
                Req* r = *it;
                if ((int)E.running.size() >= E.max_inflight) break;
                if (E.busy.count(r->h) || E.used + r->bytes > E.budget) { ++it; continue; }
                E.used += r->bytes;
                E.busy.insert(r->h);
                r->state = 1;
                E.running.push_back(r);
                to_begin.push_back(r);
                it = E.queue.erase(it);
            }
        }
        for (Req* r : to_begin) {
            cudaSetDevice(r->h->device);
            mg_status st = mgi_solve_begin(*r->h, r->b, r->u);
            if (st != MG_OK) {
                std::lock_guard<std::mutex> lk(E.mu);
                mg_result res{};
                res.status = st;
                finish(E, r, res);
            }
        }
        {
            std::lock_guard<std::mutex> lk(E.mu);
            snapshot = E.running;
        }
        bool progressed = false;
        for (Req* r : snapshot) {
            if (r->state != 1) continue;
            cudaSetDevice(r->h->device);
            cudaError_t q = cudaEventQuery(r->h->ev_state);
            if (q == cudaErrorNotReady) continue;
            int rc = q == cudaSuccess ? mgi_solve_advance(*r->h) : -MG_ERR_CUDA;
            progressed = true;
            if (rc == 0) continue;
            mg_result res = r->h->ctx.res;
            if (rc < 0) res.status = -rc;
            std::lock_guard<std::mutex> lk(E.mu);
            finish(E, r, res);
        }
        if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(5));
    }
}

size_t default_budget() {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
        cudaGetLastError();
        fr = (size_t)8 << 30;
    }
    return fr / 10 * 8;
}

void ensure_started(Engine& E) {
    if (E.started) return;
    if (E.budget == 0) E.budget = default_budget();
    std::thread(worker).detach();
    E.started = true;
}

}  // namespace

extern "C" mg_status mg_serve_configure(size_t budget_bytes, int32_t max_inflight) {
    Engine& E = engine();
    std::lock_guard<std::mutex> lk(E.mu);
    if (max_inflight < 0) { mgi_set_error("max_inflight < 0"); return MG_ERR_INVALID; }
    E.budget = budget_bytes ? budget_bytes : (E.started ? default_budget() : 0);
    E.max_inflight = max_inflight > 0 ? max_inflight : 16;
    E.configured = true;
    return MG_OK;
}

extern "C" mg_status mg_submit(mg_hierarchy* hh, const double* b, double* u, uint64_t* ticket) {
    mgi_hier* h = reinterpret_cast<mgi_hier*>(hh);
    if (!h || !b || !u || !ticket) { mgi_set_error("NULL argument"); return MG_ERR_INVALID; }
    Engine& E = engine();
    std::lock_guard<std::mutex> lk(E.mu);
    ensure_started(E);
    Req* r = new Req();
    r->h = h;
    r->b = b;
    r->u = u;
    r->bytes = h->footprint;
    if (r->bytes > E.budget) {
        delete r;
        mgi_set_error("request working set " + std::to_string(h->footprint) + " B exceeds the serving budget " +
                      std::to_string(E.budget) + " B");
        return MG_ERR_ADMISSION;
    }
    r->ticket = E.next_ticket++;
    E.all[r->ticket] = r;
    E.pending[h] += 1;
    E.queue.push_back(r);
    *ticket = r->ticket;
    E.cv.notify_all();
    return MG_OK;
}

extern "C" mg_status mg_poll(mg_hierarchy* hh, uint64_t ticket, mg_result* res) {
    mgi_hier* h = reinterpret_cast<mgi_hier*>(hh);
    Engine& E = engine();
    std::lock_guard<std::mutex> lk(E.mu);
    auto it = E.all.find(ticket);
    if (it == E.all.end() || it->second->h != h) { mgi_set_error("unknown ticket"); return MG_ERR_INVALID; }
    Req* r = it->second;
    if (r->state != 2) return MG_BUSY;
    if (res) *res = r->res;
    return (mg_status)r->res.status;
}

bool mgi_serve_busy(mgi_hier* h) {
    Engine& E = engine();
    std::lock_guard<std::mutex> lk(E.mu);
    auto it = E.pending.find(h);
    return it != E.pending.end() && it->second > 0;
}

void mgi_serve_forget(mgi_hier* h) {
    Engine& E = engine();
    std::unique_lock<std::mutex> lk(E.mu);
    E.done_cv.wait(lk, [&] {
        auto it = E.pending.find(h);
        return it == E.pending.end() || it->second <= 0;
    });
    E.pending.erase(h);
    for (auto it = E.all.begin(); it != E.all.end();) {
        if (it->second->h == h) {
            delete it->second;
            it = E.all.erase(it);
        } else {
            ++it;
        }
    }
}
