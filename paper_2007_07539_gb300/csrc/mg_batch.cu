// Level-synchronous batch solves of libmgfp (mg_solve_batch, 3D).
//
// Many independent instances of different sizes solve in one CUDA graph: the
// initial residuals, then a WHILE node whose body is one IR step of every
// instance, then the final check.  The IR step is merged across instances:
// each step operation (scale-cast, the pre-smoothing and residual-restriction
// of the k-th level below the finest, the coarse tail, the prolongation and
// post-smoothing, the update, the finalisation) is ONE launch whose grid is
// the concatenation of every instance's tiles -- a work list of (instance,
// tile) items: a table maps each CTA to its item, the item carries the
// instance's kernel arguments and TMA descriptors, the tile follows from the
// item's own grid.  Every instance keeps its own residual scale alpha, its
// norms and its convergence state (kernels of an instance that has converged
// return at once), so each instance's arithmetic -- and result -- is the same
// as when it is solved alone.
//
// Alignment: instances have different numbers of levels above their coarse
// tail.  The descending operations are merged by their position counted from
// the finest level, the ascending ones by their position counted back from
// the update, and all tails run in one launch in between, so each instance's
// own operations keep their order.  Members of a merged position with
// different launch shapes (tile rows, rows per warp, precision) form separate
// launches.  Batches this does not cover (2D, W-cycles, no coarse tail, host
// pointers, instances on different devices) use the concurrent path of
// mg_serve.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "mg_host.h"

using namespace mgi;

namespace {

struct MOp {
    enum Type { KBATCH, TAIL, FIN, RES, SINGLE } type = SINGLE;
    int kkind = 0, mode = 0, prec = 0, prec_c = 0, rpw = 1, ty = 1;
    size_t smem = 0;
    int ncta = 0, nitems = 0;
    size_t items_off = 0, cta_off = 0;  // byte offsets in the plan's device buffer
    int fin_kind = 0;
    bool init_copy = false;
    int tail_prec = -1;
    mgi_hier* h = nullptr;  // SINGLE: the instance and its op
    Op op{};
};

struct Plan {
    std::vector<mgi_hier*> hs;
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    void* dbuf = nullptr;
    std::vector<MOp> init, step, guard, report;
    DevState** d_states = nullptr;
    DevState* d_stage = nullptr;  // initial / final states, staged in one copy
    DevState* h_stage = nullptr;  // pinned host mirror
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t edone = nullptr;   // the final states are back on the host
    int launches_init = 0, launches_body = 0, launches_report = 0;
    bool busy = false;             // a run of this plan is in flight
    unsigned long long stamp = 0;  // last use (the plan cache keeps the most recent kMaxPlans)
};

std::mutex g_mu;
std::vector<Plan*> g_plans;
unsigned long long g_tick = 0;
// Plans are cached per list of hierarchies; a serving loop meets many lists,
// so the least recently used idle plans beyond this many are freed.
constexpr size_t kMaxPlans = 64;

void free_plan(Plan* p) {
    if (!p) return;
    cudaSetDevice(p->device);
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->dbuf) cudaFree(p->dbuf);
    if (p->h_stage) cudaFreeHost(p->h_stage);
    if (p->e0) cudaEventDestroy(p->e0);
    if (p->e1) cudaEventDestroy(p->e1);
    if (p->edone) cudaEventDestroy(p->edone);
    if (p->stream) cudaStreamDestroy(p->stream);
    delete p;
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Host image of the plan's device buffer: items and CTA tables appended with
// their alignment, copied once.
struct Image {
    std::vector<unsigned char> bytes;
    size_t put(const void* p, size_t n, size_t align) {
        const size_t off = align_up(bytes.size(), align);
        bytes.resize(off + n);
        std::memcpy(bytes.data() + off, p, n);
        return off;
    }
};

// Launch signature of a step op: members of a merged position with the same
// signature share one launch.
std::tuple<int, int, int, int, int, int, int, size_t> signature(const Op& op) {
    return std::make_tuple(op.kind, op.kkind, op.mode, op.prec, op.prec_c, op.sh.rpw, op.sh.ty, op.sh.smem);
}

// One merged position: the ops of the members (instance index, op), grouped by
// signature into launches appended to `out`.
void merge_position(const std::vector<std::pair<int, const Op*>>& members, const std::vector<mgi_hier*>& hs,
                    Image& img, std::vector<MOp>& out) {
    std::map<std::tuple<int, int, int, int, int, int, int, size_t>, std::vector<std::pair<int, const Op*>>> groups;
    for (const auto& m : members) groups[signature(*m.second)].push_back(m);
    for (auto& g : groups) {
        const Op& o0 = *g.second.front().second;
        MOp mo;
        if (o0.kind == OP_KERNEL && (o0.kkind == K_SWEEP || o0.kkind == K_UPDATE || o0.kkind == K_SCALE ||
                                     o0.kkind == K_PROLONG)) {
            mo.type = MOp::KBATCH;
            mo.kkind = o0.kkind; mo.mode = o0.mode; mo.prec = o0.prec; mo.prec_c = o0.prec_c;
            mo.rpw = o0.sh.rpw; mo.ty = o0.sh.ty; mo.smem = o0.sh.smem;
            std::vector<int> table;
            if (o0.kkind == K_SWEEP && o0.sh.rpw > 0) {  // marching (TMA) sweeps
                std::vector<SweepItem> items(g.second.size());
                for (size_t i = 0; i < g.second.size(); ++i) {
                    const Op& o = *g.second[i].second;
                    SweepItem& it = items[i];
                    std::memset(&it, 0, sizeof(it));
                    it.maps = o.maps;
                    it.a = o.a;
                    it.gx = o.sh.gx; it.gy = o.sh.gy; it.gz = o.sh.gz;
                    it.cta_begin = (int)table.size();
                    const int nb = o.sh.nblocks();
                    for (int c = 0; c < nb; ++c) table.push_back((int)i);
                }
                mo.items_off = img.put(items.data(), items.size() * sizeof(SweepItem), 64);
            } else {
                std::vector<KItem> items(g.second.size());
                for (size_t i = 0; i < g.second.size(); ++i) {
                    const Op& o = *g.second[i].second;
                    KItem& it = items[i];
                    std::memset(&it, 0, sizeof(it));
                    it.a = o.a;
                    it.ncta = o.sh.nblocks();
                    it.cta_begin = (int)table.size();
                    for (int c = 0; c < it.ncta; ++c) table.push_back((int)i);
                }
                mo.items_off = img.put(items.data(), items.size() * sizeof(KItem), 64);
            }
            mo.nitems = (int)g.second.size();
            mo.ncta = (int)table.size();
            mo.cta_off = img.put(table.data(), table.size() * sizeof(int), 16);
            out.push_back(mo);
        } else if (o0.kind == OP_TAIL) {
            mo.type = MOp::TAIL;
            mo.ty = o0.sh.ty;  // CTAs per instance (cluster size; grouped by it)
            std::vector<TailItem> items(g.second.size());
            int prec = hs[g.second.front().first]->tail_prec;
            for (size_t i = 0; i < g.second.size(); ++i) {
                mgi_hier& h = *hs[g.second[i].first];
                const Op& o = *g.second[i].second;
                items[i] = TailItem{h.tail_prog + o.prog_off, h.minv, h.st, o.prog_len, h.m0};
                mo.smem = std::max(mo.smem, h.tail_smem);
                if (h.tail_prec != prec) prec = -1;
            }
            mo.tail_prec = prec;
            mo.nitems = (int)items.size();
            mo.items_off = img.put(items.data(), items.size() * sizeof(TailItem), 16);
            out.push_back(mo);
        } else if (o0.kind == OP_FINALIZE) {
            mo.type = MOp::FIN;
            mo.fin_kind = o0.fin_kind;
            std::vector<FinItem> items(g.second.size());
            for (size_t i = 0; i < g.second.size(); ++i) {
                mgi_hier& h = *hs[g.second[i].first];
                items[i] = FinItem{h.st, h.partials, g.second[i].second->nblocks};
            }
            mo.nitems = (int)items.size();
            mo.items_off = img.put(items.data(), items.size() * sizeof(FinItem), 16);
            out.push_back(mo);
        } else {  // memset or base solve: one op per instance
            for (const auto& m : g.second) {
                MOp s;
                s.type = MOp::SINGLE;
                s.h = hs[m.first];
                s.op = *m.second;
                out.push_back(s);
            }
        }
    }
}

// Residual kernels of all instances (init, true-residual check or report) and
// their finalisation.
void residual_ops(const std::vector<mgi_hier*>& hs, Image& img, int gate, bool copy_u, int fin_kind,
                  std::vector<MOp>& out) {
    for (int pass = 0; pass < 2; ++pass) {  // init: zero initial guesses (r = b) and the others
        const bool init_copy = fin_kind == FIN_INIT && pass == 0;
        if (fin_kind != FIN_INIT && pass == 1) break;
        std::vector<RItem> items;
        std::vector<int> table;
        for (size_t i = 0; i < hs.size(); ++i) {
            mgi_hier& h = *hs[i];
            if (fin_kind == FIN_INIT && (h.p.zero_guess != 0) != init_copy) continue;
            const Geom& g = h.lv[h.nlev - 1].geo;
            RItem it;
            std::memset(&it, 0, sizeof(it));
            it.a.n = g.n; it.a.P = g.P; it.a.S = g.S;
            it.a.u = h.u; it.a.b = nullptr; it.a.partials = h.partials; it.a.st = h.st;
            it.a.r = fin_kind == FIN_REPORT ? nullptr : h.r;
            it.a.use_st_uout = copy_u ? 1 : 0;
            it.a.need_b = fin_kind == FIN_INIT;
            it.a.gate = gate;
            it.a.h2inv = op_alpha(h.p.op, h.dim, g.n);
            it.a.op = h.p.op;
            it.ncta = residual64_ctas(h.dim, g.n);
            it.cta_begin = (int)table.size();
            for (int c = 0; c < it.ncta; ++c) table.push_back((int)items.size());
            items.push_back(it);
        }
        if (items.empty()) continue;
        MOp mo;
        mo.type = MOp::RES;
        mo.init_copy = init_copy;
        mo.nitems = (int)items.size();
        mo.ncta = (int)table.size();
        mo.items_off = img.put(items.data(), items.size() * sizeof(RItem), 16);
        mo.cta_off = img.put(table.data(), table.size() * sizeof(int), 16);
        out.push_back(mo);
    }
    std::vector<FinItem> fins;
    for (mgi_hier* h : hs) fins.push_back(FinItem{h->st, h->partials, residual64_ctas(h->dim, h->lv[h->nlev - 1].geo.n)});
    MOp f;
    f.type = MOp::FIN;
    f.fin_kind = fin_kind;
    f.nitems = (int)fins.size();
    f.items_off = img.put(fins.data(), fins.size() * sizeof(FinItem), 16);
    out.push_back(f);
}

int run(Plan& p, const std::vector<MOp>& ops, cudaStream_t s) {
    const char* base = static_cast<const char*>(p.dbuf);
    for (const MOp& m : ops) {
        int rc = 0;
        switch (m.type) {
            case MOp::KBATCH:
                rc = launch_kernel_batch(m.kkind, m.mode, m.prec, m.prec_c, m.rpw, base + m.items_off,
                                         reinterpret_cast<const int*>(base + m.cta_off), m.ncta, m.ty, m.smem, s);
                break;
            case MOp::TAIL:
                rc = launch_tail_batch(3, m.tail_prec, reinterpret_cast<const TailItem*>(base + m.items_off), m.nitems,
                                       m.smem, m.ty, s);
                break;
            case MOp::FIN:
                rc = launch_finalize_batch(m.fin_kind, reinterpret_cast<const FinItem*>(base + m.items_off), m.nitems, s);
                break;
            case MOp::RES:
                rc = launch_residual64_batch(3, m.init_copy, reinterpret_cast<const RItem*>(base + m.items_off),
                                             reinterpret_cast<const int*>(base + m.cta_off), m.ncta, s);
                break;
            case MOp::SINGLE:
                rc = mgi_run_op(*m.h, m.op, s);
                break;
        }
        if (rc) return rc;
    }
    return 0;
}

int count_kernels(const std::vector<MOp>& ops) {
    int k = 0;
    for (const MOp& m : ops) k += !(m.type == MOp::SINGLE && m.op.kind == OP_ZERO);
    return k;
}

__global__ void k_states_scatter(const DevState* __restrict__ src, DevState* const* dst, int n, int words) {
    // copies the control part of each instance's state (everything before
    // the residual history) between the staging array and the arenas
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        const unsigned long long* a = reinterpret_cast<const unsigned long long*>(src + i);
        unsigned long long* b = reinterpret_cast<unsigned long long*>(dst[i]);
        for (int w = threadIdx.x; w < words; w += blockDim.x) b[w] = a[w];
    }
}
__global__ void k_states_gather(DevState* __restrict__ dst, DevState* const* src, int n, int words) {
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        const unsigned long long* a = reinterpret_cast<const unsigned long long*>(src[i]);
        unsigned long long* b = reinterpret_cast<unsigned long long*>(dst + i);
        for (int w = threadIdx.x; w < words; w += blockDim.x) b[w] = a[w];
    }
}
constexpr int kStateWords = (int)(offsetof(DevState, hist) / 8);
static_assert(offsetof(DevState, hist) % 8 == 0, "state control block is copied as 8-byte words");

}  // namespace

bool mgi_batch_mergeable(const mgi_hier& h) {
    if (h.dim != 3 || h.tail_level < 0 || !h.p.zero_guess) return false;
    int tails = 0;
    for (const Op& op : h.step) tails += op.kind == OP_TAIL;
    return tails == 1;  // a V-cycle (a W-cycle visits the tail more than once)
}

namespace {

// Builds the merged plan and its graph; nullptr (with the reason) when the
// batch is not covered.
Plan* build_plan(const std::vector<mgi_hier*>& hs, std::string& why) {
    const int n = (int)hs.size();
    if (n == 0) { why = "empty"; return nullptr; }
    for (mgi_hier* h : hs) {
        if (h->device != hs[0]->device) { why = "instances on different devices"; return nullptr; }
        if (!mgi_batch_mergeable(*h)) { why = "2D instance, no coarse tail, initial guess or W-cycle"; return nullptr; }
    }
    Plan* p = new Plan();
    p->hs = hs;
    p->device = hs[0]->device;
    Image img;
    // ---- the IR step, merged
    std::vector<std::vector<const Op*>> pre(n), post(n);
    std::vector<std::pair<int, const Op*>> tails;
    for (int i = 0; i < n; ++i) {
        bool after = false;
        for (const Op& op : hs[i]->step) {
            if (op.kind == OP_TAIL) { tails.push_back({i, &op}); after = true; continue; }
            (after ? post[i] : pre[i]).push_back(&op);
        }
    }
    size_t maxpre = 0, maxpost = 0;
    for (int i = 0; i < n; ++i) { maxpre = std::max(maxpre, pre[i].size()); maxpost = std::max(maxpost, post[i].size()); }
    for (size_t k = 0; k < maxpre; ++k) {
        std::vector<std::pair<int, const Op*>> m;
        for (int i = 0; i < n; ++i)
            if (k < pre[i].size()) m.push_back({i, pre[i][k]});
        merge_position(m, hs, img, p->step);
    }
    merge_position(tails, hs, img, p->step);
    for (size_t k = maxpost; k-- > 0;) {  // positions counted back from the end of each instance's step
        std::vector<std::pair<int, const Op*>> m;
        for (int i = 0; i < n; ++i)
            if (k < post[i].size()) m.push_back({i, post[i][post[i].size() - 1 - k]});
        merge_position(m, hs, img, p->step);
    }
    for (mgi_hier* h : hs) {  // u = 0 (the padded array, pads included)
        MOp z;
        z.type = MOp::SINGLE;
        z.h = h;
        z.op.kind = OP_ZERO;
        z.op.ptr = h->u_alloc;
        z.op.zero_base = 0;
        z.op.bytes = (size_t)h->lv[h->nlev - 1].geo.total * 8;
        p->init.push_back(z);
    }
    residual_ops(hs, img, 0, false, FIN_INIT, p->init);
    residual_ops(hs, img, 1, true, FIN_GUARD, p->guard);
    residual_ops(hs, img, 2, true, FIN_REPORT, p->report);
    std::vector<DevState*> sts(n);
    for (int i = 0; i < n; ++i) sts[i] = hs[i]->st;
    const size_t st_off = img.put(sts.data(), n * sizeof(DevState*), 16);
    const size_t stage_off = align_up(img.bytes.size(), 256);
    img.bytes.resize(stage_off + (size_t)n * sizeof(DevState));
    cudaSetDevice(p->device);
    auto bad = [&](const char* what, cudaError_t e) {
        why = std::string(what) + ": " + cudaGetErrorString(e);
        cudaGetLastError();
        free_plan(p);
        return (Plan*)nullptr;
    };
    cudaError_t e = cudaMalloc(&p->dbuf, img.bytes.size());
    if (e != cudaSuccess) return bad("plan allocation", e);
    e = cudaMemcpy(p->dbuf, img.bytes.data(), img.bytes.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return bad("plan upload", e);
    p->d_states = reinterpret_cast<DevState**>(static_cast<char*>(p->dbuf) + st_off);
    p->d_stage = reinterpret_cast<DevState*>(static_cast<char*>(p->dbuf) + stage_off);
    if ((e = cudaMallocHost((void**)&p->h_stage, (size_t)n * sizeof(DevState))) != cudaSuccess) return bad("pinned stage", e);
    if ((e = cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking)) != cudaSuccess) return bad("stream", e);
    if ((e = cudaEventCreate(&p->e0)) != cudaSuccess) return bad("event", e);
    if ((e = cudaEventCreate(&p->e1)) != cudaSuccess) return bad("event", e);
    if ((e = cudaEventCreateWithFlags(&p->edone, cudaEventDisableTiming)) != cudaSuccess) return bad("event", e);
    p->launches_init = count_kernels(p->init) + 1;
    p->launches_body = count_kernels(p->step) + count_kernels(p->guard) + 1;
    p->launches_report = count_kernels(p->report);

    // ---- the graph: scatter states, init, WHILE(any active){step, check, condition}, report, gather states
    cudaStream_t s = p->stream, aux = nullptr;
    if ((e = cudaStreamCreateWithFlags(&aux, cudaStreamNonBlocking)) != cudaSuccess) return bad("stream", e);
    int max_iter = 0;
    for (mgi_hier* h : hs) max_iter = std::max(max_iter, h->p.max_iter);
    cudaGraph_t graph = nullptr;
    int rc = (int)cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (!rc) {
        k_states_scatter<<<std::min(n, 1024), 256, 0, s>>>(p->d_stage, p->d_states, n, kStateWords);
        rc = (int)cudaGetLastError();
        if (!rc) rc = run(*p, p->init, s);
        cudaGraphConditionalHandle handle = 0;
        if (!rc) {
            cudaStreamCaptureStatus cs;
            cudaGraph_t cg = nullptr;
            const cudaGraphNode_t* deps = nullptr;
            size_t nd = 0;
            cudaGraphNode_t cnode = nullptr;
            cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
            rc = (int)cudaStreamGetCaptureInfo(s, &cs, nullptr, &cg, &deps, nullptr, &nd);
            if (!rc) rc = (int)cudaGraphConditionalHandleCreate(&handle, cg, 1, cudaGraphCondAssignDefault);
            if (!rc) {
                cp.conditional.handle = handle;
                cp.conditional.type = cudaGraphCondTypeWhile;
                cp.conditional.size = 1;
                rc = (int)cudaGraphAddNode(&cnode, cg, deps, nullptr, nd, &cp);
            }
            if (!rc) rc = (int)cudaStreamUpdateCaptureDependencies(s, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies);
            if (!rc) {
                rc = (int)cudaStreamBeginCaptureToGraph(aux, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                                        cudaStreamCaptureModeThreadLocal);
                if (!rc) {
                    int rc2 = run(*p, p->step, aux);
                    if (!rc2) rc2 = run(*p, p->guard, aux);
                    if (!rc2) rc2 = launch_loop_condition_batch(p->d_states, n, (unsigned long long)handle, max_iter + 16, aux);
                    cudaGraph_t body = nullptr;
                    cudaError_t e2 = cudaStreamEndCapture(aux, &body);
                    rc = rc2 ? rc2 : (int)e2;
                }
            }
        }
        if (!rc) rc = run(*p, p->report, s);
        if (!rc) {
            k_states_gather<<<std::min(n, 1024), 256, 0, s>>>(p->d_stage, p->d_states, n, kStateWords);
            rc = (int)cudaGetLastError();
        }
        cudaError_t e3 = cudaStreamEndCapture(s, &graph);
        if (!rc) rc = (int)e3;
    }
    if (!rc) rc = (int)cudaGraphInstantiate(&p->exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(aux);
    if (rc) return bad("batch graph", (cudaError_t)rc);
    return p;
}

}  // namespace

namespace mgi {
struct MergedRun {
    Plan* p = nullptr;
    std::vector<mgi_hier*> took;  // pooled instances this run bound (unbound at the finish)
    bool failed = false;
};
}  // namespace mgi

// Starts a level-synchronous batch solve on the plan's own stream.  Returns
// nullptr with *status = MG_OK when the batch is not covered (the caller takes
// the concurrent path), nullptr with an error status when it failed to start.
MergedRun* mgi_batch_merged_start(std::vector<mgi_hier*>& hs, const double* const* b, double* const* u,
                                  mg_status* status) {
    *status = MG_OK;
    for (size_t i = 0; i < hs.size(); ++i)
        if (!mgi_is_device_ptr(b[i]) || !mgi_is_device_ptr(u[i])) return nullptr;
    // pooled instances take their working arenas first (the plan holds their addresses);
    // the whole batch must fit the pool's budget at once
    MergedRun* run = new MergedRun();
    auto unbind_all = [&]() {
        for (mgi_hier* t : run->took) cudaStreamSynchronize(t->stream);
        for (mgi_hier* h : run->took) mgi_unbind(*h);
    };
    for (mgi_hier* h : hs) {
        if (h->bound) continue;
        cudaSetDevice(h->device);
        const mg_status bs = mgi_bind(*h);
        if (bs != MG_OK) {
            unbind_all();
            delete run;
            if (bs == MG_BUSY) mgi_set_error("the batch's working arenas do not fit the memory pool's budget at once");
            *status = bs == MG_BUSY ? MG_ERR_OOM : bs;
            return nullptr;
        }
        run->took.push_back(h);
    }
    Plan* p = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        for (Plan* q : g_plans)
            if (q->hs == hs) { p = q; break; }
        if (!p) {
            std::string why;
            p = build_plan(hs, why);
            if (!p) {
                unbind_all();
                delete run;
                return nullptr;
            }
            g_plans.push_back(p);
            while (g_plans.size() > kMaxPlans) {  // free the least recently used idle plan
                size_t victim = g_plans.size();
                for (size_t i = 0; i < g_plans.size(); ++i)
                    if (!g_plans[i]->busy && g_plans[i] != p &&
                        (victim == g_plans.size() || g_plans[i]->stamp < g_plans[victim]->stamp))
                        victim = i;
                if (victim == g_plans.size()) break;
                free_plan(g_plans[victim]);
                g_plans.erase(g_plans.begin() + (long)victim);
            }
        }
        p->busy = true;
        p->stamp = ++g_tick;
    }
    run->p = p;
    cudaSetDevice(p->device);
    const int n = (int)hs.size();
    // initial control states (as a single solve's start writes them)
    for (int i = 0; i < n; ++i) {
        mgi_hier& h = *hs[i];
        DevState& sh = p->h_stage[i];
        std::memset(&sh, 0, offsetof(DevState, hist));
        sh.alpha = 1.0;
        sh.inv = 1.0;
        sh.sigma = h.sigma;
        sh.tol = h.p.tol;
        sh.max_iter = h.p.max_iter;
        sh.scaling = h.p.scaling;
        sh.tol_mode = h.p.tol_mode;
        sh.guard = h.p.guard;
        sh.scale_ahead = h.scale_ahead_on() ? 1 : 0;
        sh.b = b[i];
        sh.uout = u[i];
    }
    // the caller's pending work on each instance's stream comes first, and the
    // clearing of freshly bound pooled arenas
    for (mgi_hier* h : hs) {
        cudaEventRecord(h->ev_in, h->user_stream);
        cudaStreamWaitEvent(p->stream, h->ev_in, 0);
        cudaStreamWaitEvent(p->stream, h->ev_bind, 0);
    }
    cudaStream_t s = p->stream;
    cudaError_t e = cudaMemcpyAsync(p->d_stage, p->h_stage, (size_t)n * sizeof(DevState), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaEventRecord(p->e0, s);
    if (e == cudaSuccess) e = cudaGraphLaunch(p->exec, s);
    if (e == cudaSuccess) e = cudaEventRecord(p->e1, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p->h_stage, p->d_stage, (size_t)n * sizeof(DevState), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaEventRecord(p->edone, s);
    if (e != cudaSuccess) {
        mgi_set_error(std::string("batch: ") + cudaGetErrorString(e));
        run->failed = true;
    }
    return run;
}

bool mgi_batch_merged_ready(MergedRun* run) {
    if (run->failed) return true;
    return cudaEventQuery(run->p->edone) != cudaErrorNotReady;
}

mg_status mgi_batch_merged_finish(MergedRun* run, mg_result* res) {
    Plan* p = run->p;
    cudaSetDevice(p->device);
    cudaError_t e = run->failed ? cudaErrorLaunchFailure : cudaEventSynchronize(p->edone);
    cudaStreamSynchronize(p->stream);
    for (mgi_hier* h : run->took) mgi_unbind(*h);
    const bool failed = run->failed || e != cudaSuccess;
    if (e != cudaSuccess && !run->failed) mgi_set_error(std::string("batch: ") + cudaGetErrorString(e));
    delete run;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        p->busy = false;
    }
    const int n = (int)p->hs.size();
    if (failed) {
        for (int i = 0; i < n && res; ++i) { res[i] = mg_result{}; res[i].status = MG_ERR_CUDA; res[i].merged = 1; }
        return MG_ERR_CUDA;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, p->e0, p->e1);
    mg_status first_bad = MG_OK;
    for (int i = 0; i < n; ++i) {
        const DevState& st = p->h_stage[i];
        mg_result r{};
        r.iters = st.iter;
        r.status = st.status;
        r.levels = p->hs[i]->nlev;
        r.guard_restarts = st.guard_restarts;
        r.bnorm = st.bnorm2;
        r.rel_res = st.bnorm2 > 0 ? st.rnorm2 / st.bnorm2 : st.rnorm2;
        r.rel_res_true = st.rel_true;
        r.seconds = ms * 1e-3;
        r.launches = p->launches_init + st.loops * p->launches_body + p->launches_report + 2;
        r.merged = 1;
        if (st.kerr) {
            r.status = MG_ERR_TIMEOUT;
            mgi_set_error("a stencil kernel timed out waiting for its TMA tile copies");
        }
        if (res) res[i] = r;
        if (r.status != MG_OK && first_bad == MG_OK) first_bad = (mg_status)r.status;
    }
    return first_bad;
}

// Level-synchronous batch solve; returns false (and the caller takes the
// concurrent path) when the batch is not covered.
bool mgi_batch_merged(std::vector<mgi_hier*>& hs, const double* const* b, double* const* u, mg_result* res,
                      mg_status* status) {
    MergedRun* run = mgi_batch_merged_start(hs, b, u, status);
    if (!run) return *status != MG_OK;
    *status = mgi_batch_merged_finish(run, res);
    return true;
}

// Drops the cached batch plans that contain h (called when h is destroyed).
void mgi_batch_forget(mgi_hier* h) {
    std::lock_guard<std::mutex> lk(g_mu);
    for (size_t i = 0; i < g_plans.size();) {
        if (!g_plans[i]->busy && std::find(g_plans[i]->hs.begin(), g_plans[i]->hs.end(), h) != g_plans[i]->hs.end()) {
            free_plan(g_plans[i]);
            g_plans.erase(g_plans.begin() + i);
        } else {
            ++i;
        }
    }
}
