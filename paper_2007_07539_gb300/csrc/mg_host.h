// Host-side structures of libmgfp shared by the hierarchy/solve code, the
// stage API and the serving engine.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "mg_internal.h"
#include "mg_tail.h"

namespace mgi {

// Evicts L2 by reading `bytes` (> the L2 size) of buf; sink: 4 bytes of device
// scratch (mg_misc.cu).
int launch_l2_evict(const void* buf, size_t bytes, unsigned* sink, void* stream);
// Holds the stream for about ns nanoseconds (bounded; mg_misc.cu), so that work
// enqueued behind it is queued before the device reaches it (per-kernel profiling).
int launch_hold(long long ns, void* stream);

struct Level {
    Geom geo;
    int prec = MG_FP64;
    size_t esz = 8;
    void* c = nullptr;  // correction (points at (0,0,0) of the padded layout)
    void* g = nullptr;  // right-hand side / restricted residual
    void* t = nullptr;  // ping-pong partner of c
    void* alloc[3] = {nullptr, nullptr, nullptr};  // allocation starts of c, g, t
};

// OP_KERNEL covers the fine-level kernels (kernel kind in kkind: sweep,
// IR update, scale-cast, prolongation); the values of `kind` follow
// mg_kernel_time.kind of mg.h.
enum OpKind : int { OP_KERNEL = 0, OP_COARSE = 1, OP_ZERO = 3, OP_FINALIZE = 4, OP_TAIL = 7, OP_RESCALE = 8 };

struct Op {
    int kind = 0, level = 0;
    int kkind = 0, mode = 0, prec = 0, prec_c = 0;
    KArgs a{};
    MarchShape sh{};
    const void* g = nullptr;  // OP_COARSE
    void* c = nullptr;
    void* ptr = nullptr;      // OP_ZERO: padded base pointer; OP_RESCALE: the FP16 level's g
    size_t bytes = 0;
    size_t zero_base = 0;     // bytes between allocation start and ptr
    int fin_kind = 0, nblocks = 0;
    int prog_off = 0, prog_len = 0;  // OP_TAIL: stages in the hierarchy's tail program
    bool has_maps = false;           // 3D sweeps: TMA descriptors of src and g
    SweepMaps maps{};
};

// Device memory of a hierarchy, in two parts.  The working arena (the level
// vectors c, g, t of every level, the finest level's FP64 u and r, the FP32
// scratch of rescaled restrictions: nearly all the bytes) and the persistent
// part (norm partials, control state, base-level inverse, tail program,
// rescale partials).  Offsets are relative to each part's base.
struct HierLayout {
    size_t level_off[MG_MAX_LEVELS][3] = {};
    size_t u_off = 0, r_off = 0, rsc_off = 0;
    bool has_rsc = false;
    size_t work_total = 0;
    size_t part_off = 0, st_off = 0, minv_off = 0, tprog_off = 0, rpart_off = 0;
    size_t pers_total = 0;
    size_t total = 0;  // both parts of a resident hierarchy (one allocation)
    size_t part_cap = 0;
};

struct SolveCtx {
    const double* b_user = nullptr;
    double* u_user = nullptr;
    const double* bd = nullptr;  // device b (caller's or staging)
    double* ud = nullptr;        // device u (caller's or staging)
    bool b_host = false, u_host = false;
    bool finishing = false;
    bool reported = false;
    bool copied_back = false;
    bool active = false;
    bool graph = false;          // the whole solve runs as one graph launch
    int launches = 0;
    mg_result res{};
};

struct mgi_hier {
    mg_params p{};
    int dim = 0, nlev = 0;
    Level lv[MG_MAX_LEVELS];
    double* u = nullptr;  // FP64 solution, padded finest layout
    double* r = nullptr;  // FP64 residual, padded finest layout
    double* u_alloc = nullptr;
    double* r_alloc = nullptr;
    double* partials = nullptr;
    size_t part_cap = 0;
    DevState* st = nullptr;
    DevState* st_host = nullptr;  // pinned mirror
    double* minv = nullptr;       // dense inverse of the base-level operator
    int m0 = 0;
    double sigma = 1.0;
    bool g_alias_r = false;       // finest g is r itself (FP64 finest level, no scaling)
    double* bstage = nullptr;
    double* ustage = nullptr;
    cudaStream_t stream = nullptr;
    cudaStream_t user_stream = nullptr;
    int device = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr, ev_in = nullptr, ev_state = nullptr;
    std::vector<Op> step;
    cudaGraphExec_t graph_exec = nullptr;  // one IR step (host-driven loop)
    cudaGraphExec_t solve_exec = nullptr;  // whole solve with a device-side IR loop
    bool solve_graph_failed = false;
    cudaStream_t aux = nullptr;            // capture stream of the loop body
    int tail_level = -1;                   // coarse levels 0..tail_level run in one single-CTA kernel
    std::vector<TailOp> tail_host;         // tail programs (all visits), mirrored on the device
    size_t step_tail_ops = 0;              // tail stages of the IR step (stage calls append after)
    TailOp* tail_prog = nullptr;           // device copy (capacity kTailMaxOps)
    bool describe_only = false;            // host-only schedule (mg_describe_cycle): no device objects
    int tail_soff[MG_MAX_LEVELS][3] = {};  // shared-memory byte offsets of c, t, g of tail levels
    int tail_rscr = 0;                     // shared-memory byte offset of the tail's residual scratch
    size_t tail_smem = 0;                  // dynamic shared memory of the tail kernel
    int tail_prec = -1;                    // storage type of every tail level, -1 if they differ
    int tail_cs = 1;                       // CTAs of the tail's thread-block cluster (1: one CTA)
    int tail_sh[MG_MAX_LEVELS] = {};       // chunk shift per tail level (points per CTA = 2^sh)
    int tail_sslot = -1;                   // shared-memory byte offset of the rescale slots (8 B per level)
    int tail_scr2 = -1;                    // ... of the coarse scratch of rescaled restrictions
    int tail_cg = -1;                      // ... of the CG scratch of the base level
    int rsig = 0;                          // rescaled FP16 levels: target max-norm 2^rsig
    float* rsc_alloc = nullptr;            // FP32 restriction into a rescaled level above the tail (padded)
    float* rsc_part = nullptr;             // kRescaleCtas partial maxima
    // level l is an FP16 level whose restricted residual is rescaled (rescale16)
    bool rescaled(int l) const {
        return p.rescale16 == 1 && l >= 0 && l + 1 < nlev && lv[l].prec == MG_FP16 && lv[l + 1].prec != MG_FP16;
    }
    int cg_maxit() const { return p.base_maxit > 0 ? p.base_maxit : m0; }
    // the update writes the next step's g (mg_params.scale_ahead; max-norm scaling, non-FP64 finest level)
    bool scale_ahead_on() const {
        return p.scale_ahead == 1 && p.scaling == 1 && nlev > 0 && lv[nlev - 1].prec != MG_FP64 && !g_alias_r;
    }

    void* arena = nullptr;        // persistent part (and, resident hierarchies, the working arena behind it)
    size_t arena_bytes = 0;
    size_t footprint = 0;         // both parts
    HierLayout lay;
    char* work = nullptr;         // working arena the level pointers point into (null: none yet)
    char* built_for = nullptr;    // working arena the step's launches and graphs were built for
    bool bound = false;           // pooled (mg_params.pooled): a working arena from the pool is held
    cudaEvent_t ev_bind = nullptr;  // pooled: recorded on the stream after a fresh arena was zeroed
    SolveCtx ctx;
    // launch accounting and per-kernel profiling of the IR step
    int step_kernels = 0;            // kernels per IR step (memsets excluded)
    bool prof = false;
    bool prof_pending = false;
    std::vector<cudaEvent_t> prof_ev;
    std::vector<double> prof_ms;
    std::vector<int> prof_cnt;
};

}  // namespace mgi

void mgi_set_error(const std::string& s);
// true (once per pending count) when mg_fault_inject asked the next allocation at this site to fail
bool mgi_fault_take(int site);
int mgi_validate(const mg_params* p, std::string& why);
int mgi_run_op(mgi::mgi_hier& h, const mgi::Op& op, cudaStream_t s);
void* mgi_build_cycle(mgi::mgi_hier& h, std::vector<mgi::Op>& ops, bool top_from_r, int gate,
                      const mgi::DevState* st);
mgi::Op mgi_kernel_op(mgi::mgi_hier& h, int level, int kkind, int mode, const void* src, void* dst,
                      const void* g, int gate, const mgi::DevState* st);
bool mgi_is_device_ptr(const void* p);
mgi::Op mgi_update_op(mgi::mgi_hier& h, const void* cL, int gate, const mgi::DevState* st);
mg_status mgi_solve_begin(mgi::mgi_hier& h, const double* b, double* u);
int mgi_solve_advance(mgi::mgi_hier& h);
mg_status mgi_batch_run(std::vector<mgi::mgi_hier*>& hs, const double* const* b, double* const* u,
                        mg_result* res);
bool mgi_batch_merged(std::vector<mgi::mgi_hier*>& hs, const double* const* b, double* const* u, mg_result* res,
                      mg_status* status);
void mgi_batch_forget(mgi::mgi_hier* h);
// Asynchronous form of the level-synchronous batch (mg_batch.cu): start returns
// nullptr with *status = MG_OK when the batch is not covered; ready polls;
// finish fills res (one per instance), hands back the arenas start bound and
// frees the run.
namespace mgi { struct MergedRun; }
mgi::MergedRun* mgi_batch_merged_start(std::vector<mgi::mgi_hier*>& hs, const double* const* b, double* const* u,
                                       mg_status* status);
bool mgi_batch_merged_ready(mgi::MergedRun* run);
mg_status mgi_batch_merged_finish(mgi::MergedRun* run, mg_result* res);
// The batch is one the level-synchronous launches cover (3D, V-cycle, coarse tail, zero initial guess).
bool mgi_batch_mergeable(const mgi::mgi_hier& h);
// serving engine hooks
void mgi_serve_forget(mgi::mgi_hier* h);
bool mgi_serve_busy(mgi::mgi_hier* h);
// Working arena of a pooled hierarchy (mg_pool.cu / mg_host.cu).
//   mgi_bind: takes the arena from the pool (if not held) and points the levels
//   at it, rebuilding the step's launches when its address changed.  Returns
//   MG_OK, MG_BUSY (does not fit the budget now: memory in use by other
//   solves), MG_ERR_ADMISSION (larger than the whole budget), MG_ERR_OOM or
//   MG_ERR_CUDA.  A resident hierarchy is always bound (MG_OK).
//   mgi_unbind: hands the arena back (kept as a cache for this hierarchy until
//   another needs the room); call only once no work on it is in flight.
mg_status mgi_bind(mgi::mgi_hier& h);
void mgi_unbind(mgi::mgi_hier& h);
namespace mgi {
// The device-memory pool of pooled working arenas (one per device).
//   pool_acquire: 0 ok (*base set; *kept: the block this hierarchy held last,
//   contents intact), 1 no room now, 2 never fits the budget, 3 allocation
//   error.
int pool_acquire(int device, mgi_hier* h, size_t bytes, char** base, bool* kept);
void pool_release(int device, mgi_hier* h);
void pool_drop(int device, mgi_hier* h);      // h is destroyed: its block (if any) becomes free
size_t pool_budget(int device);
void pool_set_budget(int device, size_t bytes); // 0: 80% of the device's free memory at the next use
struct PoolStats {
    size_t budget, reserved, in_use, peak_in_use, peak_reserved;
    unsigned long long acquires, reuses, evictions, chunks;
};
PoolStats pool_stats(int device);
}  // namespace mgi
