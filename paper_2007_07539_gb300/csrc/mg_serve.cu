// Concurrent batch solves and the serving engine of libmgfp
// (mg_solve_batch, mg_submit, mg_poll, mg_serve_configure).
//
// Both drive the per-solve IR state machine of mg_host.cu without blocking:
// each hierarchy has its own stream, every solve keeps one action in flight,
// and a host loop advances whichever solve's state event has completed.  So
// the kernels of different solves overlap on the device, and in the serving
// engine new requests start while others are running ("continuous
// batching"): a queued request is admitted as soon as its hierarchy is idle,
// a slot is free (max_inflight) and, for a pooled hierarchy, its working arena
// fits the device-memory pool next to the requests already in flight.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
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
        if (st == MG_BUSY) {
            mgi_set_error("the batch's working arenas do not fit the memory pool's budget at once");
            st = MG_ERR_OOM;
        }
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
// Admission.  A queued request is admitted when a slot is free
// (max_inflight), its hierarchy has no other request running, and -- for a
// pooled hierarchy (mg_params.pooled = 1) -- its working arena can be taken
// from the device-memory pool now (mgi_bind: the pool evicts cached arenas of
// idle hierarchies to make room, but never exceeds its budget and never takes
// memory of running solves).  Requests that do not fit wait in the queue in
// arrival order; later, smaller requests may pass a waiting one, but at most
// kMaxBypass times, after which admission stops behind it until it fits.  A
// resident hierarchy (pooled = 0) holds its arena since creation, outside the
// pool, and is admitted by slots alone.  On completion the arena goes back to
// the pool (kept as that hierarchy's cache until another request needs it).
namespace {

constexpr int kMaxBypass = 8;

struct Req {
    uint64_t ticket = 0;
    mgi_hier* h = nullptr;
    const double* b = nullptr;
    double* u = nullptr;
    int state = 0;  // 0 queued, 1 running, 2 done
    int bypassed = 0;
    bool waited_memory = false;
    bool in_group = false;  // runs inside a merged (level-synchronous) group
    mg_result res{};
};

// Requests admitted together that the level-synchronous launches cover run
// as one merged group (mg_serve_options): one CUDA graph whose launches each
// cover the (instance, tile) items of all members.
struct Group {
    MergedRun* run = nullptr;
    std::vector<Req*> reqs;
};

struct Engine {
    std::mutex mu;
    std::condition_variable cv;      // wakes the worker (new work)
    std::condition_variable done_cv; // wakes waiters (request finished)
    bool started = false;
    int max_inflight = 16;
    uint64_t next_ticket = 1;
    std::deque<Req*> queue;
    std::vector<Req*> running;
    std::unordered_map<uint64_t, Req*> all;
    std::unordered_map<mgi_hier*, int> pending;
    std::unordered_set<mgi_hier*> busy;
    uint64_t submitted = 0, completed = 0, memory_waits = 0, merged_groups = 0, merged_requests = 0;
    int peak_inflight = 0;
    bool merge = false;
};

Engine& engine() {
    static Engine* e = new Engine();  // never destroyed: the worker thread is detached
    return *e;
}

void finish(Engine& E, Req* r, const mg_result& res) {
    r->res = res;
    r->state = 2;
    E.busy.erase(r->h);
    E.pending[r->h] -= 1;
    ++E.completed;
    for (size_t i = 0; i < E.running.size(); ++i)
        if (E.running[i] == r) { E.running.erase(E.running.begin() + i); break; }
    E.done_cv.notify_all();
}

// One admission pass over the queue (engine lock held).  Returns the
// requests admitted, their arenas bound.
std::vector<Req*> admit(Engine& E) {
    std::vector<Req*> out;
    std::vector<Req*> waiting;  // queued requests passed over in this pass
    for (auto it = E.queue.begin(); it != E.queue.end();) {
        Req* r = *it;
        if ((int)E.running.size() >= E.max_inflight) break;
        if (E.busy.count(r->h)) { ++it; continue; }
        cudaSetDevice(r->h->device);
        const mg_status st = mgi_bind(*r->h);
        if (st == MG_BUSY) {  // does not fit the pool's budget now
            if (!r->waited_memory) { r->waited_memory = true; ++E.memory_waits; }
            if (r->bypassed >= kMaxBypass) break;  // nothing passes it any more
            waiting.push_back(r);
            ++it;
            continue;
        }
        it = E.queue.erase(it);
        if (st != MG_OK) {  // cannot be admitted at all: complete with the error
            mg_result res{};
            res.status = st;
            E.running.push_back(r);
            finish(E, r, res);
            continue;
        }
        for (Req* w : waiting) ++w->bypassed;
        E.busy.insert(r->h);
        r->state = 1;
        E.running.push_back(r);
        E.peak_inflight = std::max(E.peak_inflight, (int)E.running.size());
        out.push_back(r);
    }
    return out;
}

void worker() {
    Engine& E = engine();
    std::vector<Group> groups;
    for (;;) {
        std::vector<Req*> to_begin, snapshot;
        bool merge = false;
        {
            std::unique_lock<std::mutex> lk(E.mu);
            if (E.queue.empty() && E.running.empty())
                E.cv.wait(lk, [&] { return !E.queue.empty() || !E.running.empty(); });
            to_begin = admit(E);
            merge = E.merge;
        }
        // requests admitted together that the merged launches cover run as one group
        if (merge && to_begin.size() >= 2) {
            std::vector<Req*> cand, rest;
            for (Req* r : to_begin) {
                const bool ok = mgi_batch_mergeable(*r->h) && r->h->device == to_begin[0]->h->device &&
                                mgi_is_device_ptr(r->b) && mgi_is_device_ptr(r->u);
                (ok ? cand : rest).push_back(r);
            }
            if (cand.size() >= 2) {
                std::vector<mgi_hier*> hs;
                std::vector<const double*> bs;
                std::vector<double*> us;
                for (Req* r : cand) { hs.push_back(r->h); bs.push_back(r->b); us.push_back(r->u); }
                cudaSetDevice(cand[0]->h->device);
                mg_status st = MG_OK;
                MergedRun* run = mgi_batch_merged_start(hs, bs.data(), us.data(), &st);
                if (run) {
                    for (Req* r : cand) r->in_group = true;
                    groups.push_back(Group{run, cand});
                    std::lock_guard<std::mutex> lk(E.mu);
                    ++E.merged_groups;
                    E.merged_requests += cand.size();
                    to_begin = rest;
                } else if (st != MG_OK) {
                    for (Req* r : cand) {
                        mgi_unbind(*r->h);
                        std::lock_guard<std::mutex> lk(E.mu);
                        mg_result res{};
                        res.status = st;
                        finish(E, r, res);
                    }
                    to_begin = rest;
                }
            }
        }
        for (Req* r : to_begin) {
            cudaSetDevice(r->h->device);
            mg_status st = mgi_solve_begin(*r->h, r->b, r->u);
            if (st != MG_OK) {
                mgi_unbind(*r->h);
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
        for (size_t gi = 0; gi < groups.size();) {
            Group& g = groups[gi];
            if (!mgi_batch_merged_ready(g.run)) { ++gi; continue; }
            std::vector<mg_result> res(g.reqs.size());
            mgi_batch_merged_finish(g.run, res.data());  // the group's stream has completed
            for (size_t i = 0; i < g.reqs.size(); ++i) {
                mgi_unbind(*g.reqs[i]->h);
                std::lock_guard<std::mutex> lk(E.mu);
                finish(E, g.reqs[i], res[i]);
            }
            groups.erase(groups.begin() + (long)gi);
            progressed = true;
        }
        for (Req* r : snapshot) {
            if (r->state != 1 || r->in_group) continue;
            cudaSetDevice(r->h->device);
            cudaError_t q = cudaEventQuery(r->h->ev_state);
            if (q == cudaErrorNotReady) continue;
            int rc = q == cudaSuccess ? mgi_solve_advance(*r->h) : -MG_ERR_CUDA;
            progressed = true;
            if (rc == 0) continue;
            if (rc < 0) {  // the arena goes back only once nothing of the solve runs
                cudaStreamSynchronize(r->h->stream);
                cudaGetLastError();
                mgi_unbind(*r->h);
            }
            mg_result res = r->h->ctx.res;
            if (rc < 0) res.status = -rc;
            std::lock_guard<std::mutex> lk(E.mu);
            finish(E, r, res);
        }
        if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(5));
    }
}

void ensure_started(Engine& E) {
    if (E.started) return;
    std::thread(worker).detach();
    E.started = true;
}

}  // namespace

extern "C" mg_status mg_serve_configure(size_t budget_bytes, int32_t max_inflight) {
    Engine& E = engine();
    std::lock_guard<std::mutex> lk(E.mu);
    if (max_inflight < 0) { mgi_set_error("max_inflight < 0"); return MG_ERR_INVALID; }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); mgi_set_error("no CUDA device"); return MG_ERR_CUDA; }
    pool_set_budget(dev, budget_bytes);
    E.max_inflight = max_inflight > 0 ? max_inflight : 16;
    return MG_OK;
}

extern "C" mg_status mg_serve_options(int32_t merge_groups) {
    if (merge_groups != 0 && merge_groups != 1) { mgi_set_error("merge_groups must be 0 or 1"); return MG_ERR_INVALID; }
    Engine& E = engine();
    std::lock_guard<std::mutex> lk(E.mu);
    E.merge = merge_groups == 1;
    return MG_OK;
}

extern "C" mg_status mg_serve_stats_get(mg_serve_stats* out) {
    if (!out) { mgi_set_error("NULL argument"); return MG_ERR_INVALID; }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); mgi_set_error("no CUDA device"); return MG_ERR_CUDA; }
    const PoolStats ps = pool_stats(dev);
    Engine& E = engine();
    std::lock_guard<std::mutex> lk(E.mu);
    std::memset(out, 0, sizeof(*out));
    out->budget_bytes = ps.budget;
    out->reserved_bytes = ps.reserved;
    out->in_use_bytes = ps.in_use;
    out->peak_in_use_bytes = ps.peak_in_use;
    out->peak_reserved_bytes = ps.peak_reserved;
    out->arena_acquires = ps.acquires;
    out->arena_reuses = ps.reuses;
    out->arena_evictions = ps.evictions;
    out->submitted = E.submitted;
    out->completed = E.completed;
    out->memory_waits = E.memory_waits;
    out->merged_groups = E.merged_groups;
    out->merged_requests = E.merged_requests;
    out->inflight = (int32_t)E.running.size();
    out->peak_inflight = E.peak_inflight;
    out->queued = (int32_t)E.queue.size();
    return MG_OK;
}

extern "C" mg_status mg_submit(mg_hierarchy* hh, const double* b, double* u, uint64_t* ticket) {
    mgi_hier* h = reinterpret_cast<mgi_hier*>(hh);
    if (!h || !b || !u || !ticket) { mgi_set_error("NULL argument"); return MG_ERR_INVALID; }
    if (h->p.pooled == 1 && h->lay.work_total > pool_budget(h->device)) {
        mgi_set_error("request working arena " + std::to_string(h->lay.work_total) + " B exceeds the serving budget " +
                      std::to_string(pool_budget(h->device)) + " B");
        return MG_ERR_ADMISSION;
    }
    Engine& E = engine();
    std::lock_guard<std::mutex> lk(E.mu);
    ensure_started(E);
    Req* r = new Req();
    r->h = h;
    r->b = b;
    r->u = u;
    r->ticket = E.next_ticket++;
    E.all[r->ticket] = r;
    E.pending[h] += 1;
    E.queue.push_back(r);
    ++E.submitted;
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
    const mg_status st = (mg_status)r->res.status;
    // the final poll retires the ticket (the engine keeps no finished requests)
    E.all.erase(it);
    delete r;
    return st;
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
