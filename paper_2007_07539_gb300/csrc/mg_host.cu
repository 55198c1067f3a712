// Host side of libmgfp: hierarchy construction, the launch schedule of one
// iterative-refinement step, the IR control loop and the C ABI of mg.h.
//
// The IR loop (Alg. 2) runs as a small state machine per solve: every action
// (initial residual, one IR step, the true-residual check, the final report)
// is a launch sequence on the hierarchy's stream followed by an asynchronous
// copy of the device control state to pinned host memory and an event.  A
// blocking solve waits on that event; the batch and serving paths poll the
// events of many solves and advance whichever is ready, so their kernels
// overlap on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "mg_host.h"

using namespace mgi;

// mg_solve on a pooled hierarchy: polls of 100 us while the pool is held by other solves
constexpr int kBindWaitPolls = 600000;

namespace mgi {
int residual64_blocks(int dim, int n);
}

// ---------------------------------------------------------------- errors
static thread_local std::string g_err;
void mgi_set_error(const std::string& s) { g_err = s; }
#define FAIL(code, msg)              \
    do {                             \
        mgi_set_error(msg);          \
        return code;                 \
    } while (0)
#define CUCHK(call)                                                                                \
    do {                                                                                           \
        cudaError_t e_ = (cudaError_t)(call);                                                      \
        if (e_ != cudaSuccess) FAIL(MG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

extern "C" const char* mg_last_error(void) { return g_err.c_str(); }

// ---------------------------------------------------------------- host-side fault injection
// Pending injected allocation failures per site (mg_fault_inject).  The
// allocation sites consult mgi_fault_take before calling the allocator and
// take the allocator's own failure path when it returns true.
static std::atomic<int> g_fault[MG_FAULT_SITES];
bool mgi_fault_take(int site) {
    if (site < 0 || site >= MG_FAULT_SITES) return false;
    int v = g_fault[site].load();
    while (v > 0)
        if (g_fault[site].compare_exchange_weak(v, v - 1)) return true;
    return false;
}
extern "C" mg_status mg_fault_inject(int32_t site, int32_t count) {
    if (site < 0 || site >= MG_FAULT_SITES || count < 0) FAIL(MG_ERR_INVALID, "mg_fault_inject: bad site or count");
    g_fault[site].store(count);
    return MG_OK;
}

// ---------------------------------------------------------------- parameters
extern "C" void mg_params_init(mg_params* p, int32_t dim, int32_t n) {
    std::memset(p, 0, sizeof(*p));
    p->dim = dim;
    p->n = n;
    p->levels = 0;
    for (int i = 0; i < MG_MAX_LEVELS; ++i) p->prec[i] = MG_FP64;
    p->nu1 = 2;
    p->nu2 = 2;
    p->omega = 0.8;
    p->gamma = 1;
    p->scaling = 1;
    p->sigma_log2 = -1;
    p->tol_mode = 0;
    p->tol = 1e-10;
    p->max_iter = 100;
    p->zero_guess = 0;
    p->guard = 1;
    p->graph = 1;
    p->rescale16 = 1;
    p->base_solver = 0;
    p->base_maxit = 0;
    p->base_tol = 1e-4;
    p->scale_ahead = 1;
    p->wait_polls = -1;
    p->pooled = 0;
}

extern "C" int32_t mg_level_count(int32_t n, int32_t levels_req, int32_t* sizes) {
    if (n < 1) return 0;
    int tmp[64], cnt = 0, m = n;
    tmp[cnt++] = m;
    while (m % 2 == 1 && m > 3 && cnt < MG_MAX_LEVELS && (levels_req <= 0 || cnt < levels_req)) {
        m = (m - 1) / 2;
        tmp[cnt++] = m;
    }
    if (sizes)
        for (int l = 0; l < cnt; ++l) sizes[l] = tmp[cnt - 1 - l];
    return cnt;
}

static bool prec_ok(int p) { return p >= MG_FP64 && p <= MG_BF16; }

int mgi_validate(const mg_params* p, std::string& why) {
    if (!p) { why = "params is NULL"; return 0; }
    if (p->dim != 2 && p->dim != 3) { why = "dim must be 2 or 3"; return 0; }
    // point indices are 32-bit: n^d < 2^31
    if (p->n < 1 || p->n > (p->dim == 3 ? 1290 : 46340)) { why = "n out of range (3D: n <= 1290, 2D: n <= 46340)"; return 0; }
    if (p->levels < 0 || p->levels > MG_MAX_LEVELS) { why = "levels out of range"; return 0; }
    int sizes[MG_MAX_LEVELS];
    int L = mg_level_count(p->n, p->levels, sizes);
    if (p->levels > 0 && L != p->levels) { why = "levels exceeds what the coarsening rule allows for n"; return 0; }
    long long m0 = 1;
    for (int a = 0; a < p->dim; ++a) m0 *= sizes[0];
    if (m0 > 4096) { why = "coarsest level has more than 4096 unknowns; use more levels"; return 0; }
    for (int l = 0; l < L; ++l)
        if (!prec_ok(p->prec[l])) { why = "invalid precision in prec[]"; return 0; }
    if (p->nu1 < 0 || p->nu1 > 16 || p->nu2 < 0 || p->nu2 > 16) { why = "nu1/nu2 out of range"; return 0; }
    if (!(p->omega > 0.0 && p->omega < 2.0)) { why = "omega must be in (0, 2)"; return 0; }
    if (p->gamma != 1 && p->gamma != 2) { why = "gamma must be 1 or 2"; return 0; }
    if (p->scaling < 0 || p->scaling > 2) { why = "scaling must be 0, 1 or 2"; return 0; }
    if (p->sigma_log2 < -1 || p->sigma_log2 > 60) { why = "sigma_log2 out of range"; return 0; }
    if (p->tol_mode != 0 && p->tol_mode != 1) { why = "tol_mode must be 0 or 1"; return 0; }
    if (!(p->tol >= 0.0) || !std::isfinite(p->tol)) { why = "tol must be finite and >= 0"; return 0; }
    if (p->max_iter < 0 || p->max_iter > kMaxIter) { why = "max_iter out of range"; return 0; }
    if (p->no_tail < 0 || p->no_tail > 2) { why = "no_tail must be 0, 1 or 2"; return 0; }
    if ((p->tune != 0 && p->tune != 1) || p->fuse_pre < 0 || p->fuse_pre > 2) {
        why = "tune must be 0 or 1 and fuse_pre 0, 1 or 2";
        return 0;
    }
    if ((p->rescale16 != 0 && p->rescale16 != 1) || (p->base_solver != 0 && p->base_solver != 1)) {
        why = "rescale16 and base_solver must be 0 or 1";
        return 0;
    }
    if (p->base_maxit < 0 || p->base_maxit > 100000) { why = "base_maxit out of range (0..100000)"; return 0; }
    if (!(p->base_tol >= 0.0) || !std::isfinite(p->base_tol)) { why = "base_tol must be finite and >= 0"; return 0; }
    if (p->op != 0 && p->op != 1) { why = "op must be 0 (finite differences) or 1 (Q1 finite elements)"; return 0; }
    if (p->op == 1 && p->fuse_pre == 1) { why = "fuse_pre is for the finite-difference operator (op = 0)"; return 0; }
    if (p->scale_ahead != 0 && p->scale_ahead != 1) { why = "scale_ahead must be 0 or 1"; return 0; }
    if (p->wait_polls < -1) { why = "wait_polls must be -1 (default) or >= 0"; return 0; }
    if (p->pooled != 0 && p->pooled != 1) { why = "pooled must be 0 or 1"; return 0; }
    for (int i = 0; i < 4; ++i)
        if (p->reserved[i] != 0) { why = "reserved fields must be 0"; return 0; }
    return L;
}

// ---------------------------------------------------------------- footprint
static size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

static size_t update_blocks_max(const mgi_hier& h);

// Working arena: the level vectors, u, r and the FP32 scratch of rescaled
// restrictions; persistent part: partials, control state, base inverse, tail
// program, rescale partials (HierLayout).  A resident hierarchy holds both in
// one allocation, the working arena at total - work_total.
static void compute_layout(mgi_hier& h, HierLayout& lay) {
    size_t off = 0;
    for (int l = 0; l < h.nlev; ++l) {
        size_t b = align_up((size_t)h.lv[l].geo.total * h.lv[l].esz, 256);
        for (int v = 0; v < 3; ++v) { lay.level_off[l][v] = off; off += b; }
    }
    const Geom& gf = h.lv[h.nlev - 1].geo;
    size_t b64 = align_up((size_t)gf.total * 8, 256);
    lay.u_off = off; off += b64;
    lay.r_off = off; off += b64;
    // FP32 restriction into a rescaled FP16 level run as plain kernels (any
    // rescaled level: a W-cycle beyond the tail's program capacity drops the tail)
    size_t rsc = 0;
    for (int l = 0; l < h.nlev; ++l)
        if (h.rescaled(l)) rsc = std::max(rsc, (size_t)h.lv[l].geo.total * 4);
    lay.has_rsc = rsc > 0;
    lay.rsc_off = 0;
    if (rsc) { lay.rsc_off = off; off += align_up(rsc, 256); }
    lay.work_total = align_up(off, 4096);
    off = 0;
    size_t nb = std::max<size_t>((size_t)residual64_blocks(h.dim, gf.n) * 4, update_blocks_max(h) * 2);
    lay.part_cap = nb;
    lay.part_off = off; off += align_up(nb * 8, 256);
    lay.st_off = off; off += align_up(sizeof(DevState), 256);
    lay.minv_off = off; off += align_up((size_t)h.m0 * h.m0 * 8, 256);
    lay.tprog_off = off;
    if (h.tail_level >= 0) off += align_up(sizeof(TailOp) * kTailMaxOps, 256);
    lay.rpart_off = off;
    if (rsc) off += align_up(kRescaleCtas * sizeof(float), 256);
    lay.pers_total = align_up(off, 4096);
    lay.total = lay.pers_total + lay.work_total;
}

// Points the levels, u, r and the rescale scratch at a working arena.
static void bind_work(mgi_hier& h, char* work) {
    const HierLayout& lay = h.lay;
    h.work = work;
    for (int l = 0; l < h.nlev; ++l) {
        const size_t bo = (size_t)h.lv[l].geo.base * h.lv[l].esz;
        h.lv[l].c = work + lay.level_off[l][0] + bo;
        h.lv[l].g = work + lay.level_off[l][1] + bo;
        h.lv[l].t = work + lay.level_off[l][2] + bo;
        h.lv[l].alloc[0] = work + lay.level_off[l][0];
        h.lv[l].alloc[1] = work + lay.level_off[l][1];
        h.lv[l].alloc[2] = work + lay.level_off[l][2];
    }
    const Geom& gf = h.lv[h.nlev - 1].geo;
    h.u_alloc = (double*)(work + lay.u_off);
    h.r_alloc = (double*)(work + lay.r_off);
    h.u = h.u_alloc + gf.base;
    h.r = h.r_alloc + gf.base;
    h.rsc_alloc = lay.has_rsc ? (float*)(work + lay.rsc_off) : nullptr;
}

// ---------------------------------------------------------------- base-level operator inverse
// Dense A0 = alpha (beta I - W) of the base level's operator (op 0: 5/7-point
// finite differences; op 1: Q1, weights 1 on the 8 neighbours in 2D, 2 on
// edges and 1 on corners in 3D), inverted by Gauss-Jordan elimination with
// partial pivoting in FP64 (host, at setup).
static bool coarse_inverse(int dim, int op, int n, std::vector<double>& inv) {
    int m = 1;
    for (int a = 0; a < dim; ++a) m *= n;
    const double alpha = op_alpha(op, dim, n);
    std::vector<double> A((size_t)m * m, 0.0);
    for (int p = 0; p < m; ++p) {
        const int i = p % n, j = (p / n) % n, k = p / (n * n);
        for (int dk = (dim == 3 ? -1 : 0); dk <= (dim == 3 ? 1 : 0); ++dk)
            for (int dj = -1; dj <= 1; ++dj)
                for (int di = -1; di <= 1; ++di) {
                    const int nz = (di != 0) + (dj != 0) + (dk != 0);
                    int w;  // the weight of the offset in beta I - W
                    if (nz == 0) w = op_beta(op, dim);
                    else if (op == 0) w = nz == 1 ? -1 : 0;
                    else w = dim == 2 ? -1 : (nz == 2 ? -2 : nz == 3 ? -1 : 0);
                    if (w == 0) continue;
                    const int ii = i + di, jj = j + dj, kk = k + dk;
                    if (ii < 0 || ii >= n || jj < 0 || jj >= n || kk < 0 || kk >= (dim == 3 ? n : 1)) continue;
                    A[(size_t)p * m + (size_t)(ii + n * jj + n * n * kk)] = alpha * w;
                }
    }
    inv.assign((size_t)m * m, 0.0);
    for (int i = 0; i < m; ++i) inv[(size_t)i * m + i] = 1.0;
    for (int col = 0; col < m; ++col) {
        int piv = col;
        for (int r = col + 1; r < m; ++r)
            if (std::fabs(A[(size_t)r * m + col]) > std::fabs(A[(size_t)piv * m + col])) piv = r;
        if (A[(size_t)piv * m + col] == 0.0) return false;
        if (piv != col)
            for (int c2 = 0; c2 < m; ++c2) {
                std::swap(A[(size_t)piv * m + c2], A[(size_t)col * m + c2]);
                std::swap(inv[(size_t)piv * m + c2], inv[(size_t)col * m + c2]);
            }
        double d = 1.0 / A[(size_t)col * m + col];
        for (int c2 = 0; c2 < m; ++c2) { A[(size_t)col * m + c2] *= d; inv[(size_t)col * m + c2] *= d; }
        for (int r = 0; r < m; ++r) {
            if (r == col) continue;
            double f = A[(size_t)r * m + col];
            if (f == 0.0) continue;
            for (int c2 = 0; c2 < m; ++c2) {
                A[(size_t)r * m + c2] -= f * A[(size_t)col * m + c2];
                inv[(size_t)r * m + c2] -= f * inv[(size_t)col * m + c2];
            }
        }
    }
    return true;
}

// ---------------------------------------------------------------- schedule of one IR step
namespace {
struct Gen {
    mgi_hier* h;
    int cur[MG_MAX_LEVELS];
    int gate;
    const DevState* st;
    bool top_from_r;  // finest g comes from the FP64 residual (solve) or is given (stage)
    std::vector<Op>* out;

    void* cbuf(int l) { return cur[l] ? h->lv[l].t : h->lv[l].c; }
    void* obuf(int l) { return cur[l] ? h->lv[l].c : h->lv[l].t; }
    const void* gbuf(int l) {
        if (l == h->nlev - 1 && top_from_r && h->g_alias_r) return h->r;
        return h->lv[l].g;
    }

    Op kernel(int l, int kkind, int mode, const void* src, void* dst, const void* g) {
        Op op{};
        op.kind = OP_KERNEL;
        op.level = l;
        op.kkind = kkind;
        // stencil kernels of a Q1 hierarchy: the Q1 variants
        if (h->p.op == 1 && (kkind == K_SWEEP || kkind == K_UPDATE)) mode |= M_FEM;
        op.mode = mode;
        op.prec = h->lv[l].prec;
        op.prec_c = l > 0 ? h->lv[l - 1].prec : op.prec;
        const Geom& f = h->lv[l].geo;
        KArgs& a = op.a;
        a.n = f.n; a.P = f.P; a.S = f.S;
        if (l > 0) { const Geom& c = h->lv[l - 1].geo; a.nc = c.n; a.Pc = c.P; a.Sc = c.S; }
        a.src = src; a.dst = dst; a.g = g;
        a.r64 = h->r;
        a.u64 = h->u; a.rw64 = h->r; a.partials = h->partials;
        a.st = st; a.gate = gate;
        a.omega = h->p.omega;
        a.h2inv = op_alpha(h->p.op, h->dim, f.n);
        a.cf = make_sweep_coef(h->dim, h->p.op, a.omega, a.h2inv);
        op.sh = kernel_shape(h->dim, kkind, mode, op.prec, f.n, f.P, 0);
        a.xstep = op.sh.xstep; a.ystep = op.sh.ystep; a.zstep = op.sh.zstep; a.zlen = op.sh.zlen;
        a.err = h->st ? &h->st->kerr : nullptr;
        a.wait_polls = h->p.wait_polls >= 0 ? h->p.wait_polls + 1 : 0;
        if (h->dim == 3 && kkind == K_SWEEP && op.sh.rpw > 0 && !h->describe_only) {  // TMA boxes: TY+2 rows of the swept vector, TY rows of g
            op.has_maps = true;
            const int rows = op.sh.ty * op.sh.rpw;
            // the one-pass pre-smoothing + restriction reads g boxes of TY+4 rows
            if (make_sweep_map(&op.maps.src, op.prec, f, src, rows + (mode == M_PRE ? 4 : 2), true) != 0) op.has_maps = false;
            const void* gm = g ? g : src;  // modes without g never read it
            if (make_sweep_map(&op.maps.g, op.prec, f, gm, rows, false) != 0) op.has_maps = false;
        }
        return op;
    }

    Op rescale_op(int l) {  // max-norm and scaled cast of the FP32 restriction into FP16 level l
        Op op{};
        op.kind = OP_RESCALE;
        op.level = l;
        op.prec = op.prec_c = h->lv[l].prec;
        op.ptr = h->lv[l].g;
        op.a.gate = gate;
        op.a.st = st;
        return op;
    }

    void sweep(int l) {  // one Jacobi sweep on level l, ping-pong
        out->push_back(kernel(l, K_SWEEP, M_JACOBI, cbuf(l), obuf(l), gbuf(l)));
        cur[l] ^= 1;
    }

    // ---- coarse tail: the same recursion on shared-memory copies of levels
    // 0..tail_level, emitted as the stages of one single-CTA kernel
    int sc(int l) const { return h->tail_soff[l][cur[l]]; }
    int so(int l) const { return h->tail_soff[l][cur[l] ^ 1]; }
    int sg(int l) const { return h->tail_soff[l][2]; }
    TailOp tbase(int l, int kind) {
        TailOp t{};
        t.kind = kind;
        t.prec = h->lv[l].prec;
        t.prec_c = l > 0 ? h->lv[l - 1].prec : t.prec;
        const Geom& f = h->lv[l].geo;
        t.n = f.n; t.P = f.P; t.S = (int)f.S;
        t.mn = tail_magic(f.n);
        if (l > 0) { t.nc = h->lv[l - 1].geo.n; t.mnc = tail_magic(t.nc); }
        t.h2inv = op_alpha(h->p.op, h->dim, f.n);
        t.omega = h->p.omega;
        t.cf = make_sweep_coef(h->dim, h->p.op, t.omega, t.h2inv);
        t.op = h->p.op;
        t.sh = h->tail_sh[l];
        t.shc = l > 0 ? h->tail_sh[l - 1] : t.sh;
        t.sslot = -1;
        t.scr2 = -1;
        t.rsig = h->rsig;
        t.cgmax = h->cg_maxit();
        t.cgtol = h->p.base_tol;
        return t;
    }
    void tpush(const TailOp& t) { h->tail_host.push_back(t); }
    void tsweep(int l, int mode, int src, int dst, int g) {
        TailOp t = tbase(l, TK_SWEEP);
        t.mode = mode; t.src = src; t.dst = dst; t.g = g;
        tpush(t);
    }
    void tjacobi(int l) { tsweep(l, M_JACOBI, sc(l), so(l), sg(l)); cur[l] ^= 1; }
    void tcycle(int l, bool first) {
        if (l == 0) {
            TailOp t = tbase(0, TK_COARSE);
            t.mode = h->p.base_solver;
            t.src = h->tail_cg;
            t.g = sg(0);
            t.dst = sc(0);
            tpush(t);
            return;
        }
        if (first) {
            if (h->p.nu1 >= 2) {
                tsweep(l, M_ZERO2, sg(l), sc(l), 0);
                for (int k = 2; k < h->p.nu1; ++k) tjacobi(l);
            } else if (h->p.nu1 == 1) {
                tsweep(l, M_ZERO1, sg(l), sc(l), 0);
            } else {
                TailOp t = tbase(l, TK_ZERO);
                t.dst = sc(l);
                tpush(t);
            }
        } else {
            for (int k = 0; k < h->p.nu1; ++k) tjacobi(l);
        }
        TailOp r = tbase(l, TK_RESID);
        r.src = sc(l); r.g = sg(l); r.dst = h->tail_rscr;
        tpush(r);
        TailOp rs = tbase(l, TK_RESTRICT);
        rs.src = h->tail_rscr; rs.dst = sg(l - 1);
        const int slot = h->rescaled(l - 1) ? h->tail_sslot + 8 * (l - 1) : -1;
        rs.sslot = slot;
        rs.scr2 = h->tail_scr2;
        tpush(rs);
        cur[l - 1] = 0;
        for (int k = 0; k < h->p.gamma; ++k) tcycle(l - 1, k == 0);
        TailOp pr = tbase(l, TK_PROLONG);
        pr.dst = sc(l); pr.coarse = sc(l - 1);
        pr.sslot = slot;
        tpush(pr);
        for (int k = 0; k < h->p.nu2; ++k) tjacobi(l);
    }
    // one visit of level l = tail_level: load its g (and, on later W-cycle
    // visits, its c) from the global level arrays, recurse, store c back
    void tvisit(int l, bool first) {
        TailOp ld = tbase(l, TK_LOAD);
        ld.dst = sg(l); ld.gptr = const_cast<void*>(gbuf(l));
        tpush(ld);
        if (!first) {
            TailOp lc = tbase(l, TK_LOAD);
            lc.dst = sc(l); lc.gptr = cbuf(l);
            tpush(lc);
        }
        tcycle(l, first);
        TailOp stc = tbase(l, TK_STORE);
        stc.src = sc(l); stc.gptr = cbuf(l);
        tpush(stc);
    }

    // Alg. 1 on level l; first = zero initial correction (first visit).
    void cycle(int l, bool first) {
        const int L = h->nlev - 1;
        if (l == L && top_from_r && !h->g_alias_r)  // Alg. 2's residual scaling: g_L = cast(r / alpha)
            out->push_back(kernel(L, K_SCALE, 0, nullptr, h->lv[L].g, nullptr));
        if (l == h->tail_level && (h->tail_prog || h->describe_only)) {
            Op op{};
            op.kind = OP_TAIL;
            op.level = l;
            op.prec = h->lv[l].prec;
            op.prec_c = l > 0 ? h->lv[l - 1].prec : op.prec;
            op.prog_off = (int)h->tail_host.size();
            tvisit(l, first);
            op.prog_len = (int)h->tail_host.size() - op.prog_off;
            op.sh.ty = h->tail_cs;  // tails of different cluster sizes are not merged in batches
            op.a.gate = gate;
            op.a.st = st;
            out->push_back(op);
            return;
        }
        if (l == 0) {
            Op op{};
            op.kind = OP_COARSE;
            op.level = 0;
            op.prec = h->lv[0].prec;
            op.prec_c = op.prec;
            op.g = gbuf(0);
            op.c = cbuf(0);
            op.a.gate = gate;
            op.a.st = st;
            out->push_back(op);
            return;
        }
        // one pass for the two sweeps from zero and the residual-restriction
        const bool resc = h->rescaled(l - 1);
        const bool fused = first && h->p.nu1 == 2 && h->dim == 3 && !resc && h->p.op == 0 &&
                           (h->p.fuse_pre == 1 ||
                            (h->p.fuse_pre == 2 && fuse_choice_get(h->lv[l].prec, h->lv[l - 1].prec, h->lv[l].geo.n) == 1));
        if (fused) {
            Op op = kernel(l, K_SWEEP, M_PRE, gbuf(l), h->lv[l - 1].g, gbuf(l));
            op.a.dst2 = cbuf(l);
            out->push_back(op);
        } else if (first) {
            if (h->p.nu1 >= 2) {
                out->push_back(kernel(l, K_SWEEP, M_ZERO2, gbuf(l), cbuf(l), nullptr));
                for (int s = 2; s < h->p.nu1; ++s) sweep(l);
            } else if (h->p.nu1 == 1) {
                out->push_back(kernel(l, K_SWEEP, M_ZERO1, gbuf(l), cbuf(l), nullptr));
            } else {
                Op z{};
                z.kind = OP_ZERO;
                z.level = l;
                z.prec = z.prec_c = h->lv[l].prec;
                z.ptr = cbuf(l);
                z.bytes = (size_t)h->lv[l].geo.total * h->lv[l].esz;
                z.zero_base = h->lv[l].geo.base * h->lv[l].esz;
                out->push_back(z);
            }
        } else {
            for (int s = 0; s < h->p.nu1; ++s) sweep(l);
        }
        if (resc) {  // restriction into a rescaled FP16 level: FP32 scratch, then max-norm and scaled cast
            Op op = kernel(l, K_SWEEP, M_RESTRICT, cbuf(l), h->rsc_alloc + h->lv[l - 1].geo.base, gbuf(l));
            op.prec_c = MG_FP32;
            out->push_back(op);
            out->push_back(rescale_op(l - 1));
        } else if (!fused) {
            out->push_back(kernel(l, K_SWEEP, M_RESTRICT, cbuf(l), h->lv[l - 1].g, gbuf(l)));
        }
        cur[l - 1] = 0;
        for (int k = 0; k < h->p.gamma; ++k) cycle(l - 1, k == 0);
        Op pr = kernel(l, K_PROLONG, 0, nullptr, cbuf(l), nullptr);
        pr.a.coarse = cbuf(l - 1);
        if (resc) pr.a.cscale = &h->st->lscale[l - 1];
        out->push_back(pr);
        for (int s = 0; s < h->p.nu2; ++s) sweep(l);
    }
};
}  // namespace

// Builds the ops of one MG cycle on the finest level (c_L from g_L) and
// returns where c_L ends up.
void* mgi_build_cycle(mgi_hier& h, std::vector<Op>& ops, bool top_from_r, int gate, const DevState* st) {
    Gen gen{};
    gen.h = &h;
    gen.gate = gate;
    gen.st = st;
    gen.top_from_r = top_from_r;
    gen.out = &ops;
    for (int l = 0; l < MG_MAX_LEVELS; ++l) gen.cur[l] = 0;
    const size_t t0 = h.tail_host.size();
    gen.cycle(h.nlev - 1, true);
    if (h.tail_prog && h.tail_host.size() > t0) {
        if (h.tail_host.size() > (size_t)kTailMaxOps) return nullptr;
        cudaMemcpy(h.tail_prog + t0, h.tail_host.data() + t0, (h.tail_host.size() - t0) * sizeof(TailOp),
                   cudaMemcpyHostToDevice);
    }
    return gen.cbuf(h.nlev - 1);
}

Op mgi_kernel_op(mgi_hier& h, int level, int kkind, int mode, const void* src, void* dst, const void* g,
                 int gate, const DevState* st) {
    Gen gen{};
    gen.h = &h;
    gen.gate = gate;
    gen.st = st;
    gen.top_from_r = false;
    return gen.kernel(level, kkind, mode, src, dst, g);
}

Op mgi_update_op(mgi_hier& h, const void* cL, int gate, const DevState* st) {
    const int L = h.nlev - 1;
    Gen gen{};
    gen.h = &h;
    gen.gate = gate;
    gen.st = st;
    gen.top_from_r = true;
    // scale-ahead: the update also writes the next step's g (the M_SA instantiation)
    Op op = gen.kernel(L, K_UPDATE, 0, cL, h.scale_ahead_on() ? h.lv[L].g : nullptr, nullptr);
    if (op.a.dst && h.lv[L].prec != MG_FP64) op.mode |= M_SA;
    return op;
}

static size_t update_blocks_max(const mgi_hier& h) {
    const Geom& f = h.lv[h.nlev - 1].geo;
    MarchShape s = kernel_shape(h.dim, K_UPDATE, 0, h.lv[h.nlev - 1].prec, f.n, f.P, 0);
    return (size_t)s.nblocks();
}

static void build_step(mgi_hier& h) {
    h.step.clear();
    h.tail_host.clear();
    void* cL = mgi_build_cycle(h, h.step, true, 1, h.st);
    if (!cL) {  // tail programs beyond capacity (deep W-cycles): plain kernels on every level
        h.tail_prog = nullptr;
        h.tail_level = -1;
        h.tail_host.clear();
        h.step.clear();
        cL = mgi_build_cycle(h, h.step, true, 1, h.st);
    }
    h.step_tail_ops = h.tail_host.size();
    Op up = mgi_update_op(h, cL, 1, h.st);
    up.a.fin = 1;  // the update's last CTA runs the step's finalisation (FIN_STEP)
    h.step.push_back(up);
    h.step_kernels = 0;
    for (const Op& op : h.step) h.step_kernels += op.kind == OP_ZERO ? 0 : op.kind == OP_RESCALE ? 2 : 1;
}

int mgi_run_op(mgi_hier& h, const Op& op, cudaStream_t s) {
    switch (op.kind) {
        case OP_KERNEL:
            if (h.dim == 3 && op.kkind == K_SWEEP && op.sh.rpw > 0 && !op.has_maps) return (int)cudaErrorNotSupported;
            return launch_kernel(h.dim, op.kkind, op.mode, op.prec, op.prec_c, op.a, op.sh,
                                 op.has_maps ? &op.maps : nullptr, s);
        case OP_COARSE:
            if (h.p.base_solver == 1)
                return launch_coarse_cg(op.prec, h.p.op, op.g, op.c, h.lv[0].geo, h.p.base_tol, h.cg_maxit(),
                                        op.a.st, op.a.gate, s);
            return launch_coarse_solve(op.prec, h.minv, h.m0, op.g, op.c, h.lv[0].geo, op.a.st, op.a.gate, s);
        case OP_RESCALE:
            if (!h.rsc_alloc) return (int)cudaErrorInvalidValue;
            return launch_rescale(h.rsc_alloc + h.lv[op.level].geo.base, op.ptr, h.lv[op.level].geo, h.rsc_part,
                                  h.rsig, &h.st->lscale[op.level], op.a.st, op.a.gate, s);
        case OP_ZERO:
            return (int)cudaMemsetAsync((char*)op.ptr - op.zero_base, 0, op.bytes, s);
        case OP_FINALIZE:
            return launch_finalize(op.fin_kind, h.st, h.partials, op.nblocks, s);
        case OP_TAIL:
            return launch_tail(h.dim, h.tail_prec, h.tail_prog + op.prog_off, op.prog_len, h.minv, h.m0, op.a.st,
                               op.a.gate, h.tail_smem, h.tail_cs, s,
                               op.prog_len > 0 ? &h.tail_host[op.prog_off] : nullptr);
    }
    return (int)cudaErrorInvalidValue;
}

// ---------------------------------------------------------------- creation
static void free_hier(mgi_hier* h) {
    if (!h) return;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaSetDevice(h->device);
    if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
    if (h->solve_exec) cudaGraphExecDestroy(h->solve_exec);
    if (h->aux) cudaStreamDestroy(h->aux);
    if (h->p.pooled == 1) pool_drop(h->device, h);
    if (h->arena) cudaFree(h->arena);
    if (h->bstage) cudaFree(h->bstage);
    if (h->ustage) cudaFree(h->ustage);
    if (h->st_host) cudaFreeHost(h->st_host);
    if (h->e0) cudaEventDestroy(h->e0);
    if (h->e1) cudaEventDestroy(h->e1);
    if (h->ev_in) cudaEventDestroy(h->ev_in);
    if (h->ev_state) cudaEventDestroy(h->ev_state);
    if (h->ev_bind) cudaEventDestroy(h->ev_bind);
    for (cudaEvent_t e : h->prof_ev) cudaEventDestroy(e);
    if (h->stream) cudaStreamDestroy(h->stream);
    cudaSetDevice(dev);
    delete h;
}

// Shared-memory plan of the coarse tail: the deepest level T >= 1 whose
// levels 0..T (c, t, g in their storage types, one residual scratch in the
// arithmetic type, the scale slots and coarse scratch of rescaled FP16 levels,
// the CG vectors of the base level) fit in kTailMaxSmem bytes per CTA, either
// in one CTA (levels of at most kTailMaxPoints points) or distributed over a
// thread-block cluster of 16 or 8 CTAs (chunks of 2^sh points per CTA; dense
// base solve and no rescaled level inside, as their reductions are CTA-wide);
// tail_level = -1 when no level qualifies.  probe = false (no device query, or
// the cluster tail not requested): single-CTA plans only.
static void plan_tail(mgi_hier& h, bool disabled, bool probe) {
    h.tail_level = -1;
    h.tail_smem = 0;
    h.tail_cs = 1;
    if (disabled) return;
    for (int T = h.nlev - 1; T >= 1; --T) {
        bool resc = false;
        for (int l = 0; l < T; ++l) resc = resc || h.rescaled(l);
        int uprec = h.lv[0].prec;
        for (int l = 1; l <= T; ++l)
            if (h.lv[l].prec != uprec) uprec = -1;
        for (int cs : {16, 8, 1}) {
            if (cs > 1 && (!probe || resc || h.p.base_solver == 1)) continue;
            size_t off = 0, rmax = 0;
            bool ok = true;
            for (int l = 0; l <= T && ok; ++l) {
                const long long n = h.lv[l].geo.n;
                const long long N = h.dim == 3 ? n * n * n : n * n;
                if (N > (cs > 1 ? kTailMaxPointsCl : kTailMaxPoints)) { ok = false; break; }
                int sh = kTailWholeShift;
                long long chunk = N;
                if (cs > 1) {
                    sh = 5;
                    while (((long long)cs << sh) < N) ++sh;
                    chunk = 1LL << sh;
                }
                h.tail_sh[l] = sh;
                for (int v = 0; v < 3; ++v) {
                    h.tail_soff[l][v] = (int)off;
                    off = align_up(off + (size_t)chunk * h.lv[l].esz, 16);
                }
                rmax = std::max(rmax, (size_t)chunk * (h.lv[l].prec == MG_FP64 ? 8 : 4));
            }
            if (!ok) continue;
            h.tail_rscr = (int)off;
            off = align_up(off + rmax, 16);
            h.tail_sslot = h.tail_scr2 = h.tail_cg = -1;
            size_t smax = 0;  // rescaled restrictions inside the tail: coarse values in the arithmetic type
            for (int l = 0; l < T; ++l)
                if (h.rescaled(l)) {
                    const long long n = h.lv[l].geo.n;
                    smax = std::max(smax, (size_t)(h.dim == 3 ? n * n * n : n * n) * 8);
                }
            if (smax) {
                h.tail_sslot = (int)off;
                off = align_up(off + 8 * MG_MAX_LEVELS, 16);
                h.tail_scr2 = (int)off;
                off = align_up(off + smax, 16);
            }
            if (h.p.base_solver == 1) {  // r, p, A p of the base level: 16-byte aligned slots of m0 * 8 bytes
                const long long n = h.lv[0].geo.n;
                h.tail_cg = (int)off;
                off += 3 * align_up((size_t)(h.dim == 3 ? n * n * n : n * n) * 8, 16);
            }
            if (off > kTailMaxSmem) continue;
            if (cs > 1 && tail_cluster_ok(h.dim, uprec, cs, off) < 1) continue;
            h.tail_level = T;
            h.tail_smem = off;
            h.tail_cs = cs;
            h.tail_prec = uprec;
            return;
        }
    }
}

// Autotuner (tune = 1): for every 3D stencil kernel of the step -- sweeps
// from zero, residual-restriction, Jacobi on each level above the coarse
// tail -- time candidate tile shapes (rows per warp 1/2; the model's march
// length, half and double it; best of five runs; a candidate must beat the
// model's shape by 8%) on this hierarchy's level
// arrays (their contents at creation do not matter; pads stay zero) and keep
// the fastest.
// The choice is process-wide per (kernel, type, level size): later
// hierarchies of the same sizes reuse it without timing.
static void autotune(mgi_hier& h) {
    if (h.dim != 3) return;
    cudaStream_t s = h.stream;
    cudaEvent_t ea = nullptr, eb = nullptr;
    if (cudaEventCreate(&ea) != cudaSuccess || cudaEventCreate(&eb) != cudaSuccess) {
        cudaGetLastError();
        if (ea) cudaEventDestroy(ea);
        return;
    }
    // Inside a solve the finest levels stream from DRAM while the small ones
    // stay in L2: kernels on levels whose arrays exceed a quarter of L2 are
    // timed after reading 256 MB (an L2 eviction without write-back), the
    // others warm.
    void* flush = nullptr;
    const size_t kFlush = 256u << 20;
    if (cudaMalloc(&flush, kFlush + 256) != cudaSuccess) {
        cudaGetLastError();
        flush = nullptr;
    } else if (cudaMemsetAsync(flush, 1, kFlush + 256, s) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(flush);
        flush = nullptr;
    }
    unsigned* sink = flush ? reinterpret_cast<unsigned*>(static_cast<char*>(flush) + kFlush) : nullptr;
    bool cold = false;
    auto time_op = [&](const Op& op) -> float {
        float best = 1e30f;
        if (mgi_run_op(h, op, s)) return best;  // warm-up (and launch check)
        for (int rep = 0; rep < 5; ++rep) {
            if (cold && flush) launch_l2_evict(flush, kFlush, sink, s);
            cudaEventRecord(ea, s);
            if (mgi_run_op(h, op, s)) return 1e30f;
            cudaEventRecord(eb, s);
            cudaEventSynchronize(eb);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ea, eb);
            best = std::min(best, ms);
        }
        return best;
    };
    const int lo = h.tail_level >= 0 ? h.tail_level + 1 : 1;
    for (int l = h.nlev - 1; l >= lo; --l) {
        Level& lv = h.lv[l];
        const int n = lv.geo.n;
        cold = 3.0 * (double)lv.geo.total * (double)lv.esz > 32.0 * 1048576.0;
        for (int mode : {M_PRE, M_ZERO2, M_RESTRICT, M_JACOBI}) {
            if (mode == M_PRE && (h.p.fuse_pre == 0 || h.p.op != 0)) continue;
            const int kmode = mode | (h.p.op == 1 ? M_FEM : 0);  // the key of the kernel's shapes
            TileChoice have;
            if (tile_choice_get(3, K_SWEEP, kmode, lv.prec, n, &have)) continue;
            const bool coarse_out = mode == M_RESTRICT || mode == M_PRE;
            const void* src = mode == M_ZERO2 || mode == M_PRE ? lv.g : lv.c;
            void* dst = coarse_out ? h.lv[l - 1].g : (mode == M_ZERO2 ? lv.c : lv.t);
            const void* g = mode == M_ZERO2 ? nullptr : lv.g;
            auto make = [&]() {
                Op op = mgi_kernel_op(h, l, K_SWEEP, mode, src, dst, g, 0, nullptr);
                op.a.dst2 = lv.c;  // M_PRE's smoothed correction
                return op;
            };
            const Op base = make();
            const int z0 = base.sh.rpw == 0 ? std::max(1, std::min(8, coarse_out ? (n - 1) / 2 : n))
                                             : (coarse_out ? (base.sh.zlen - 1) / 2 : base.sh.zlen);
            const int zmax = coarse_out ? (n - 1) / 2 : n;
            TileChoice best{base.sh.rpw, z0};
            float tbest = time_op(base);
            // a candidate replaces the model's shape only when clearly faster:
            // timed alone, shapes within a few percent of each other order
            // differently inside a solve
            tbest *= 0.92f;
            if (h.p.op == 0 && mode != M_PRE && base.sh.rpw != 0 && n <= 255) {  // the direct kernel
                const TileChoice c{0, 0};
                tile_choice_set(3, K_SWEEP, kmode, lv.prec, n, &c);
                const float t = time_op(make());
                if (t < tbest) { tbest = t; best = c; }
            }
            for (int rpw = 1; rpw <= 2; ++rpw) {
                if (rpw == 2 && (coarse_out || n < 16 || h.p.op == 1)) continue;
                for (int z : {z0 / 2, z0, z0 * 2}) {
                    z = std::max(1, std::min(z, zmax));
                    if (rpw == base.sh.rpw && z == z0) continue;  // the model's shape, timed above
                    const TileChoice c{rpw, z};
                    tile_choice_set(3, K_SWEEP, kmode, lv.prec, n, &c);
                    const float t = time_op(make());
                    if (t < tbest) { tbest = t; best = c; }
                }
            }
            tile_choice_set(3, K_SWEEP, kmode, lv.prec, n, &best);
        }
        // sweeps per launch of the pre-smoothing (fuse_pre = 2): the one-pass form
        // (two sweeps from zero and the residual-restriction, M_PRE) against the two
        // launches, each in its tuned shape; kept only when clearly faster
        if (h.p.fuse_pre == 2 && h.p.op == 0 && h.p.nu1 == 2 && !h.rescaled(l - 1) &&
            fuse_choice_get(lv.prec, h.lv[l - 1].prec, n) < 0) {
            Op zero2 = mgi_kernel_op(h, l, K_SWEEP, M_ZERO2, lv.g, lv.c, nullptr, 0, nullptr);
            Op restr = mgi_kernel_op(h, l, K_SWEEP, M_RESTRICT, lv.c, h.lv[l - 1].g, lv.g, 0, nullptr);
            Op pre = mgi_kernel_op(h, l, K_SWEEP, M_PRE, lv.g, h.lv[l - 1].g, lv.g, 0, nullptr);
            pre.a.dst2 = lv.c;
            const float t2 = time_op(zero2) + time_op(restr);
            const float t1 = time_op(pre);
            fuse_choice_set(lv.prec, h.lv[l - 1].prec, n, t1 < 0.97f * t2 ? 1 : 0);
        }
    }
    cudaStreamSynchronize(s);
    cudaGetLastError();
    if (flush) cudaFree(flush);
    cudaEventDestroy(ea);
    cudaEventDestroy(eb);
}

static mg_status plan_hier(const mg_params* p, mgi_hier& h, bool probe) {
    std::string why;
    int L = mgi_validate(p, why);
    if (!L) FAIL(MG_ERR_INVALID, why);
    h.p = *p;
    h.dim = p->dim;
    h.nlev = L;
    int sizes[MG_MAX_LEVELS];
    mg_level_count(p->n, p->levels, sizes);
    bool any16 = false;
    for (int l = 0; l < L; ++l) {
        h.lv[l].geo = make_geom(p->dim, sizes[l]);
        h.lv[l].prec = p->prec[l];
        h.lv[l].esz = elem_size(p->prec[l]);
        any16 = any16 || p->prec[l] == MG_FP16;
    }
    int sl = p->sigma_log2 >= 0 ? p->sigma_log2 : (any16 ? 14 : 0);
    h.sigma = p->scaling == 0 ? 1.0 : std::ldexp(1.0, sl);
    h.g_alias_r = (p->prec[L - 1] == MG_FP64 && p->scaling == 0);
    h.rsig = sl;
    plan_tail(h, p->no_tail == 1, probe && p->no_tail == 2);
    h.m0 = 1;
    for (int a = 0; a < p->dim; ++a) h.m0 *= sizes[0];
    compute_layout(h, h.lay);
    h.footprint = h.lay.total;
    h.part_cap = h.lay.part_cap;
    return MG_OK;
}

extern "C" size_t mg_footprint_bytes(const mg_params* p) {
    mgi_hier h;
    if (plan_hier(p, h, false) != MG_OK) return 0;
    return h.footprint;
}

extern "C" mg_status mg_describe_cycle(const mg_params* p, int* rec, int cap, int* count) {
    if (!count || cap < 0 || (cap > 0 && !rec)) FAIL(MG_ERR_INVALID, "count is NULL or rec / cap inconsistent");
    *count = 0;
    mgi_hier h;
    const mg_status st = plan_hier(p, h, false);
    if (st != MG_OK) return st;
    h.describe_only = true;
    DevState dummy{};  // stands in for the device state (its address is recorded, never read)
    h.st = &dummy;
    std::vector<Op> ops;
    mgi_build_cycle(h, ops, true, 0, nullptr);
    int n = 0;
    auto put = [&](int kind, int level, int kkind, int mode, int prec, int prec_c) {
        if (n < cap) {
            int* r = rec + 6 * (size_t)n;
            r[0] = kind; r[1] = level; r[2] = kkind; r[3] = mode; r[4] = prec; r[5] = prec_c;
        }
        ++n;
    };
    for (const Op& op : ops) {
        put(op.kind, op.level, op.kind == OP_KERNEL ? op.kkind : -1, op.kind == OP_COARSE ? h.p.base_solver : op.mode,
            op.prec, op.prec_c);
        if (op.kind != OP_TAIL) continue;
        for (int k = op.prog_off; k < op.prog_off + op.prog_len; ++k) {
            const TailOp& t = h.tail_host[k];
            int level = -1;
            for (int l = 0; l < h.nlev; ++l)
                if (h.lv[l].geo.n == t.n) level = l;
            put(100 + t.kind, level, -1, t.mode, t.prec, t.prec_c);
        }
    }
    *count = n;
    return MG_OK;
}

extern "C" mg_status mg_create_hierarchy(const mg_params* p, void* cuda_stream, mg_hierarchy** out) {
    if (!out) FAIL(MG_ERR_INVALID, "out is NULL");
    *out = nullptr;
    mgi_hier* h = new mgi_hier();
    mg_status st = plan_hier(p, *h, true);
    if (st != MG_OK) { delete h; return st; }
    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) { delete h; FAIL(MG_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e)); }
    h->user_stream = (cudaStream_t)cuda_stream;
    const HierLayout& lay = h->lay;
    const bool pooled = h->p.pooled == 1;
    // a resident hierarchy holds both parts in one allocation; a pooled one only
    // the persistent part (its working arena comes from the pool per solve)
    const size_t bytes = pooled ? lay.pers_total : lay.total;
    e = (!pooled && mgi_fault_take(MG_FAULT_ARENA)) ? cudaErrorMemoryAllocation : cudaMalloc(&h->arena, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        h->arena = nullptr;
        free_hier(h);
        FAIL(MG_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed");
    }
    h->arena_bytes = bytes;
    char* base = (char*)h->arena;
    h->partials = (double*)(base + lay.part_off);
    if (h->tail_level >= 0) h->tail_prog = (TailOp*)(base + lay.tprog_off);
    h->st = (DevState*)(base + lay.st_off);
    h->minv = (double*)(base + lay.minv_off);
    if (lay.has_rsc) h->rsc_part = (float*)(base + lay.rpart_off);
    if (!pooled) bind_work(*h, base + lay.pers_total);
    std::vector<double> inv;
    if (!coarse_inverse(h->dim, h->p.op, h->lv[0].geo.n, inv)) { free_hier(h); FAIL(MG_ERR_INVALID, "singular base-level operator"); }
#define CK_CREATE(call)                                                                       \
    do {                                                                                      \
        cudaError_t e2 = (call);                                                              \
        if (e2 != cudaSuccess) {                                                              \
            free_hier(h);                                                                     \
            FAIL(MG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e2));            \
        }                                                                                     \
    } while (0)
    CK_CREATE(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
    CK_CREATE(cudaStreamCreateWithFlags(&h->aux, cudaStreamNonBlocking));
    CK_CREATE(cudaEventCreate(&h->e0));
    CK_CREATE(cudaEventCreate(&h->e1));
    CK_CREATE(cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming));
    CK_CREATE(cudaEventCreateWithFlags(&h->ev_state, cudaEventDisableTiming));
    CK_CREATE(cudaEventCreateWithFlags(&h->ev_bind, cudaEventDisableTiming));
    CK_CREATE(cudaMallocHost((void**)&h->st_host, sizeof(DevState)));
    std::memset(h->st_host, 0, sizeof(DevState));
    CK_CREATE(cudaMemsetAsync(h->arena, 0, bytes, h->stream));
    CK_CREATE(cudaMemcpyAsync(h->minv, inv.data(), inv.size() * 8, cudaMemcpyHostToDevice, h->stream));
    CK_CREATE(cudaStreamSynchronize(h->stream));
#undef CK_CREATE
    if (!pooled) {
        if (p->tune == 1) autotune(*h);
        build_step(*h);
        h->built_for = h->work;
        h->bound = true;
    } else if (p->tune == 1) {
        // tile shapes are timed on the hierarchy's own arrays: take an arena from
        // the pool for it if one fits now (it stays cached for the first solve);
        // otherwise the shapes come from the wave model
        if (mgi_bind(*h) == MG_OK) {
            autotune(*h);
            h->built_for = nullptr;  // rebuild the step with the tuned shapes at the next bind
            cudaStreamSynchronize(h->stream);
            mgi_unbind(*h);
        }
        cudaGetLastError();
    }
    *out = reinterpret_cast<mg_hierarchy*>(h);
    return MG_OK;
}

// ---------------------------------------------------------------- pooled working arenas
mg_status mgi_bind(mgi_hier& h) {
    if (h.p.pooled != 1 || h.bound) return MG_OK;
    char* base = nullptr;
    bool kept = false;
    const int rc = pool_acquire(h.device, &h, h.lay.work_total, &base, &kept);
    if (rc == 1) FAIL(MG_BUSY, "the memory pool's budget is held by other solves");
    if (rc == 2)
        FAIL(MG_ERR_ADMISSION, "working arena of " + std::to_string(h.lay.work_total) +
                                   " B exceeds the memory pool's budget of " + std::to_string(pool_budget(h.device)) + " B");
    if (rc == 3) FAIL(MG_ERR_OOM, "device allocation for the memory pool failed");
    h.bound = true;
    if (!kept || base != h.work) {
        // a block that held another hierarchy's arrays (or nothing): the padded
        // layout needs its pads and guards zero, so the whole arena is cleared
        bind_work(h, base);
        cudaError_t e = cudaMemsetAsync(base, 0, h.lay.work_total, h.stream);
        if (e == cudaSuccess) e = cudaEventRecord(h.ev_bind, h.stream);
        if (e != cudaSuccess) {
            pool_release(h.device, &h);
            h.bound = false;
            FAIL(MG_ERR_CUDA, std::string("arena clear: ") + cudaGetErrorString(e));
        }
    }
    if (h.built_for != h.work) {  // launches and graphs hold the arena's addresses
        if (h.graph_exec) { cudaGraphExecDestroy(h.graph_exec); h.graph_exec = nullptr; }
        if (h.solve_exec) { cudaGraphExecDestroy(h.solve_exec); h.solve_exec = nullptr; }
        mgi_batch_forget(&h);
        build_step(h);
        h.built_for = h.work;
    }
    return MG_OK;
}

void mgi_unbind(mgi_hier& h) {
    if (h.p.pooled != 1 || !h.bound) return;
    pool_release(h.device, &h);
    h.bound = false;
}

extern "C" mg_status mg_destroy(mg_hierarchy* hh) {
    mgi_hier* h = reinterpret_cast<mgi_hier*>(hh);
    if (!h) return MG_OK;
    mgi_serve_forget(h);
    mgi_batch_forget(h);
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    free_hier(h);
    return MG_OK;
}

// ---------------------------------------------------------------- the IR state machine
bool mgi_is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device address of a page-locked host allocation that kernels can access in
// place (pinned memory is mapped into the device's address space), else null.
static double* mapped_host_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost && a.devicePointer ? static_cast<double*>(a.devicePointer) : nullptr;
}

static size_t npoints(const mgi_hier& h) {
    size_t n = (size_t)h.lv[h.nlev - 1].geo.n;
    return h.dim == 3 ? n * n * n : n * n;
}

static int ensure_staging(mgi_hier& h) {
    if (h.bstage) return 0;
    size_t bytes = npoints(h) * 8;
    if (mgi_fault_take(MG_FAULT_STAGING)) return 1;
    if (cudaMalloc(&h.bstage, bytes) != cudaSuccess) { cudaGetLastError(); h.bstage = nullptr; return 1; }
    if (cudaMalloc(&h.ustage, bytes) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(h.bstage);
        h.bstage = h.ustage = nullptr;
        return 1;
    }
    return 0;
}

static int run_step_ops(mgi_hier& h, cudaStream_t s) {
    for (const Op& op : h.step) {
        int rc = mgi_run_op(h, op, s);
        if (rc) return rc;
    }
    return 0;
}

static int launch_step(mgi_hier& h) {
    cudaStream_t s = h.stream;
    h.ctx.launches += h.step_kernels;
    if (h.prof) {
        // the device waits while the host enqueues the step (a few us per
        // kernel and event pair): each event pair then brackets its kernel alone
        int rc0 = launch_hold(20000 + 8000 * (long long)h.step.size(), s);
        if (rc0) return rc0;
        for (size_t i = 0; i < h.step.size(); ++i) {
            cudaError_t e = cudaEventRecord(h.prof_ev[2 * i], s);
            if (e != cudaSuccess) return (int)e;
            int rc = mgi_run_op(h, h.step[i], s);
            if (rc) return rc;
            e = cudaEventRecord(h.prof_ev[2 * i + 1], s);
            if (e != cudaSuccess) return (int)e;
        }
        h.prof_pending = true;
        return 0;
    }
    if (h.p.graph) {
        if (!h.graph_exec) {
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) return (int)e;
            int rc = run_step_ops(h, s);
            e = cudaStreamEndCapture(s, &g);
            if (rc) { if (g) cudaGraphDestroy(g); return rc; }
            if (e != cudaSuccess) return (int)e;
            e = cudaGraphInstantiate(&h.graph_exec, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) { h.graph_exec = nullptr; return (int)e; }
        }
        return (int)cudaGraphLaunch(h.graph_exec, s);
    }
    return run_step_ops(h, s);
}

// r = b - A u with b taken from the control state; gate: 0 always, 1 only when
// the true-residual check is pending, 2 only when u must still be copied out.
static int launch_residual(mgi_hier& h, cudaStream_t s, double* r, int copy_u, int gate, int fin_kind) {
    const Geom& g = h.lv[h.nlev - 1].geo;
    RArgs a{};
    a.n = g.n; a.P = g.P; a.S = g.S;
    a.u = h.u; a.b = nullptr; a.r = r; a.partials = h.partials; a.st = h.st;
    a.use_st_uout = copy_u;
    a.need_b = fin_kind == FIN_INIT;
    a.gate = gate;
    a.h2inv = op_alpha(h.p.op, h.dim, g.n);
    a.op = h.p.op;
    int nb = 0;
    int rc = launch_residual64(h.dim, a, &nb, s);
    if (rc) return rc;
    return launch_finalize(fin_kind, h.st, h.partials, nb, s);
}

// Alg. 2's initial residual: r = b - A u0 (or r = b for u0 = 0), then the first stopping test.
static int launch_init(mgi_hier& h, cudaStream_t s) {
    const Geom& g = h.lv[h.nlev - 1].geo;
    if (h.p.zero_guess) {
        cudaError_t e = cudaMemsetAsync(h.u_alloc, 0, (size_t)g.total * 8, s);
        if (e != cudaSuccess) return (int)e;
        int nb = 0;
        int rc = launch_init_rb(h.dim, g, nullptr, h.r, h.partials, h.st, &nb, s);
        if (rc) return rc;
        return launch_finalize(FIN_INIT, h.st, h.partials, nb, s);
    }
    int rc = launch_pack_u0(h.dim, g, h.st, h.u, s);
    if (rc) return rc;
    return launch_residual(h, s, h.r, 0, 0, FIN_INIT);
}
static int init_kernels(const mgi_hier& h) { return h.p.zero_guess ? 2 : 3; }

// The true-residual check (a11): recompute b - A u in FP64, copy u out.
static int launch_guard(mgi_hier& h, cudaStream_t s) { return launch_residual(h, s, h.r, 1, 1, FIN_GUARD); }
// Final report when u changed after the last check: ||b - A u|| and the copy-out.
static int launch_report(mgi_hier& h, cudaStream_t s) { return launch_residual(h, s, nullptr, 1, 2, FIN_REPORT); }

// The whole solve as one graph: init, then a WHILE node whose body is the IR
// step (kernels gated on phase 0), the true-residual check (gated on phase 1)
// and the loop condition; then the report (gated on u not yet copied out).
// No host round trip per IR step.
static int build_solve_graph(mgi_hier& h) {
    cudaStream_t s = h.stream;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return (int)e;
    int rc = launch_init(h, s);
    if (!rc) {
        cudaStreamCaptureStatus cs;
        cudaGraph_t cg = nullptr;
        const cudaGraphNode_t* deps = nullptr;
        size_t nd = 0;
        cudaGraphConditionalHandle handle = 0;
        cudaGraphNode_t cnode = nullptr;
        cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
        rc = (int)cudaStreamGetCaptureInfo(s, &cs, nullptr, &cg, &deps, nullptr, &nd);
        if (!rc) rc = (int)cudaGraphConditionalHandleCreate(&handle, cg, 1, cudaGraphCondAssignDefault);
        if (!rc) {
            cp.type = cudaGraphNodeTypeConditional;
            cp.conditional.handle = handle;
            cp.conditional.type = cudaGraphCondTypeWhile;
            cp.conditional.size = 1;
            rc = (int)cudaGraphAddNode(&cnode, cg, deps, nullptr, nd, &cp);
        }
        if (!rc) rc = (int)cudaStreamUpdateCaptureDependencies(s, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies);
        if (!rc) {
            cudaGraph_t body = cp.conditional.phGraph_out[0];
            rc = (int)cudaStreamBeginCaptureToGraph(h.aux, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
            if (!rc) {
                int rc2 = run_step_ops(h, h.aux);
                if (!rc2) rc2 = launch_guard(h, h.aux);
                if (!rc2) rc2 = launch_loop_condition(h.st, (unsigned long long)handle, h.p.max_iter + 16, h.aux);
                cudaGraph_t out = nullptr;
                cudaError_t e2 = cudaStreamEndCapture(h.aux, &out);
                rc = rc2 ? rc2 : (int)e2;
            }
        }
    }
    if (!rc) rc = launch_report(h, s);
    e = cudaStreamEndCapture(s, &graph);
    if (!rc) rc = (int)e;
    if (!rc) rc = (int)cudaGraphInstantiate(&h.solve_exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (rc) {
        h.solve_exec = nullptr;
        cudaGetLastError();
    }
    return rc;
}

static int push_state(mgi_hier& h) {
    cudaError_t e = cudaMemcpyAsync(h.st_host, h.st, offsetof(DevState, hist), cudaMemcpyDeviceToHost, h.stream);
    if (e != cudaSuccess) return (int)e;
    return (int)cudaEventRecord(h.ev_state, h.stream);
}

// Starts a solve: resolves host/device pointers, writes the control state,
// then launches either the whole-solve graph or the initial residual (the
// host-driven loop, used when graphs are off or for per-kernel profiling).
static mg_status solve_begin_bound(mgi_hier& h, const double* b, double* u);
mg_status mgi_solve_begin(mgi_hier& h, const double* b, double* u) {
    const bool was_bound = h.bound;
    mg_status st = mgi_bind(h);
    if (st != MG_OK) return st;
    if (h.prof) {  // per-kernel events of the step as built for this arena
        const size_t nops = h.step.size();
        if (h.prof_ev.size() != 2 * nops) {
            for (cudaEvent_t e : h.prof_ev) cudaEventDestroy(e);
            h.prof_ev.assign(2 * nops, nullptr);
            for (auto& e : h.prof_ev)
                if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); e = nullptr; }
        }
        h.prof_ms.assign(nops, 0.0);
        h.prof_cnt.assign(nops, 0);
    }
    st = solve_begin_bound(h, b, u);
    if (st != MG_OK && !was_bound) {
        cudaStreamSynchronize(h.stream);
        cudaGetLastError();
        mgi_unbind(h);
    }
    return st;
}

static mg_status solve_begin_bound(mgi_hier& h, const double* b, double* u) {
    SolveCtx& c = h.ctx;
    c = SolveCtx{};
    c.b_user = b;
    c.u_user = u;
    c.b_host = !mgi_is_device_ptr(b);
    c.u_host = !mgi_is_device_ptr(u);
    cudaStream_t s = h.stream;
    const size_t N = npoints(h);
    CUCHK(cudaEventRecord(h.ev_in, h.user_stream));
    CUCHK(cudaStreamWaitEvent(s, h.ev_in, 0));
    CUCHK(cudaEventRecord(h.e0, s));
    c.bd = b;
    c.ud = u;
    if (c.u_host) {
        // a pinned host u is read (initial guess) and written (solution) by the
        // kernels in place over the host link: no staging copy either way
        if (double* um = mapped_host_ptr(u)) {
            c.ud = um;
            c.u_host = false;
        }
    }
    if (c.b_host || c.u_host) {
        if (ensure_staging(h)) FAIL(MG_ERR_OOM, "staging allocation failed");
    }
    if (c.b_host) {
        CUCHK(cudaMemcpyAsync(h.bstage, b, N * 8, cudaMemcpyHostToDevice, s));
        c.bd = h.bstage;
    }
    if (c.u_host) {
        if (!h.p.zero_guess) CUCHK(cudaMemcpyAsync(h.ustage, u, N * 8, cudaMemcpyHostToDevice, s));
        c.ud = h.ustage;
    }
    DevState& sh = *h.st_host;
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
    sh.phase = 0;
    sh.b = c.bd;
    sh.uout = c.ud;
    CUCHK(cudaMemcpyAsync(h.st, &sh, offsetof(DevState, hist), cudaMemcpyHostToDevice, s));
    c.graph = h.p.graph && !h.prof && !h.solve_graph_failed;
    if (c.graph && !h.solve_exec && build_solve_graph(h)) {
        h.solve_graph_failed = true;  // conditional nodes unavailable: host-driven loop
        c.graph = false;
    }
    if (c.graph) {
        CUCHK(cudaGraphLaunch(h.solve_exec, s));
    } else {
        CUCHK(launch_init(h, s));
        c.launches += init_kernels(h);
    }
    CUCHK(push_state(h));
    c.active = true;
    return MG_OK;
}

// Advances a started solve by one action; call once its state event has
// completed.  Returns 1 when the solve has finished (result in h.ctx), 0 when
// a new action was launched, or a negative mg_status on a launch error.
int mgi_solve_advance(mgi_hier& h) {
    SolveCtx& c = h.ctx;
    const DevState& s = *h.st_host;
    int rc = 0;
    if (h.prof_pending) {  // the previous step has completed: collect its kernel times
        for (size_t i = 0; i < h.step.size(); ++i) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, h.prof_ev[2 * i], h.prof_ev[2 * i + 1]) == cudaSuccess) {
                h.prof_ms[i] += ms;
                h.prof_cnt[i] += 1;
            }
        }
        h.prof_pending = false;
    }
    auto fail = [&](int code) {
        mgi_set_error(std::string("launch: ") + cudaGetErrorString((cudaError_t)code));
        c.active = false;
        cudaStreamSynchronize(h.stream);  // nothing of this solve may still run on a released arena
        cudaGetLastError();
        mgi_unbind(h);
        return -MG_ERR_CUDA;
    };
    if (c.graph && !c.finishing) {
        // the graph ran init, loop and report: count its kernel launches
        c.launches += init_kernels(h) + s.loops * (h.step_kernels + 3) + 2;
        c.finishing = true;
        c.reported = true;
    }
    if (!c.finishing) {
        if (s.phase == 0) {
            rc = launch_step(h);
        } else if (s.phase == 1) {
            rc = launch_guard(h, h.stream);
            c.launches += 2;
        } else {
            c.finishing = true;
        }
        if (!c.finishing) {
            if (rc || (rc = push_state(h))) return fail(rc);
            return 0;
        }
    }
    if (!c.reported) {  // ||b - A u|| and the copy-out, unless the last check already did both
        c.reported = true;
        if (s.dirty) {
            rc = launch_report(h, h.stream);
            c.launches += 2;
            if (!rc) rc = push_state(h);
            if (rc) return fail(rc);
            return 0;
        }
    }
    if (c.u_host && !c.copied_back) {
        rc = (int)cudaMemcpyAsync(c.u_user, c.ud, npoints(h) * 8, cudaMemcpyDeviceToHost, h.stream);
        c.copied_back = true;
        if (!rc) rc = (int)cudaEventRecord(h.ev_state, h.stream);
        if (rc) return fail(rc);
        return 0;
    }
    cudaEventRecord(h.e1, h.stream);
    cudaEventSynchronize(h.e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h.e0, h.e1);
    mg_result& r = c.res;
    r.iters = s.iter;
    r.status = s.status;
    r.levels = h.nlev;
    r.guard_restarts = s.guard_restarts;
    r.bnorm = s.bnorm2;
    r.rel_res = s.bnorm2 > 0 ? s.rnorm2 / s.bnorm2 : s.rnorm2;
    r.rel_res_true = s.rel_true;
    r.seconds = ms * 1e-3;
    r.launches = c.launches;
    if (s.kerr) {  // a stencil kernel's bounded wait for its tile copies ran out: results are not valid
        r.status = MG_ERR_TIMEOUT;
        mgi_set_error(s.kerr == 2 ? "a stencil kernel timed out waiting for its TMA tile copies, and a copy "
                                    "had still not completed when it drained them"
                                  : "a stencil kernel timed out waiting for its TMA tile copies");
    }
    c.active = false;
    mgi_unbind(h);  // the last action's event has completed: no work on the arena is in flight
    return 1;
}

extern "C" mg_status mg_solve(mg_hierarchy* hh, const double* b, double* u, mg_result* res) {
    mgi_hier* h = reinterpret_cast<mgi_hier*>(hh);
    if (!h || !b || !u) FAIL(MG_ERR_INVALID, "NULL argument");
    if (mgi_serve_busy(h)) FAIL(MG_ERR_INVALID, "hierarchy has serving requests in flight");
    CUCHK(cudaSetDevice(h->device));
    mg_status st = mgi_solve_begin(*h, b, u);
    // a pooled hierarchy waits while other solves hold the pool's budget
    for (int k = 0; st == MG_BUSY && k < kBindWaitPolls; ++k) {
        std::this_thread::sleep_for(std::chrono::microseconds(100));
        st = mgi_solve_begin(*h, b, u);
    }
    if (st == MG_BUSY) FAIL(MG_ERR_OOM, "the memory pool's budget stayed held by other solves for 60 s");
    if (st != MG_OK) return st;
    for (;;) {
        cudaError_t e = cudaEventSynchronize(h->ev_state);
        if (e != cudaSuccess) FAIL(MG_ERR_CUDA, std::string("solve: ") + cudaGetErrorString(e));
        int rc = mgi_solve_advance(*h);
        if (rc < 0) return (mg_status)(-rc);
        if (rc == 1) break;
    }
    if (res) *res = h->ctx.res;
    return (mg_status)h->ctx.res.status;
}

// ---------------------------------------------------------------- batch (concurrent instances)
extern "C" mg_status mg_solve_batch(int32_t count, mg_hierarchy* const* hs, const double* const* b,
                                    double* const* u, mg_result* res) {
    if (count < 0 || (count > 0 && (!hs || !b || !u))) FAIL(MG_ERR_INVALID, "bad batch arguments");
    std::vector<mgi_hier*> H(count);
    for (int i = 0; i < count; ++i) {
        H[i] = reinterpret_cast<mgi_hier*>(hs[i]);
        if (!H[i] || !b[i] || !u[i]) FAIL(MG_ERR_INVALID, "NULL entry in batch");
        for (int j = 0; j < i; ++j)
            if (H[j] == H[i]) FAIL(MG_ERR_INVALID, "a hierarchy appears twice in the batch");
        if (mgi_serve_busy(H[i])) FAIL(MG_ERR_INVALID, "hierarchy has serving requests in flight");
    }
    // level-synchronous merged launches where the batch allows, else one
    // concurrent state machine per instance
    mg_status st = MG_OK;
    if (count > 0 && mgi_batch_merged(H, b, u, res, &st)) return st;
    return mgi_batch_run(H, b, u, res);
}

// ---------------------------------------------------------------- profiling
static double op_bytes(const mgi_hier& h, const Op& op) {
    auto pts = [&](int l) {
        double n = h.lv[l].geo.n;
        return h.dim == 3 ? n * n * n : n * n;
    };
    const double s = (double)elem_size(op.prec);
    const double sc = (double)elem_size(op.prec_c);
    const double N = pts(op.level);
    const double Nc = op.level > 0 ? pts(op.level - 1) : 0.0;
    switch (op.kind) {
        case OP_KERNEL:
            switch (op.kkind) {
                case K_SWEEP:
                    if ((op.mode & M_BASE) == M_JACOBI) return 3 * s * N;      // read c, g; write c'
                    if ((op.mode & M_BASE) == M_RESTRICT) return 2 * s * N + sc * Nc;  // read c, g; write g_coarse
                    if ((op.mode & M_BASE) == M_PRE) return 2 * s * N + sc * Nc;       // read g; write c, g_coarse
                    return 2 * s * N;                               // read g; write c
                case K_UPDATE: return (32 + s + (op.a.dst ? s : 0)) * N;  // read c; read+write u, r (FP64); g
                case K_SCALE: return (8 + s) * N;                   // read r (FP64); write g
                case K_PROLONG: return 2 * s * N + sc * Nc;         // read+write c; read c_coarse
            }
            return 0.0;
        case OP_COARSE: return 2 * s * N + (h.p.base_solver == 1 ? 0.0 : 8.0 * h.m0 * h.m0);
        case OP_RESCALE: return 10.0 * N;  // read the FP32 restriction twice; write g (FP16)
        case OP_ZERO: return (double)op.bytes;
        case OP_FINALIZE: return 16.0 * op.nblocks;
        case OP_TAIL: {
            double b = 0.0;  // global traffic only: the level arrays of the tail live in shared memory
            for (int i = op.prog_off; i < op.prog_off + op.prog_len; ++i) {
                const TailOp& t = h.tail_host[i];
                const double tn = h.dim == 3 ? (double)t.n * t.n * t.n : (double)t.n * t.n;
                if (t.kind == TK_LOAD || t.kind == TK_STORE) b += (double)elem_size(t.prec) * tn;
                if (t.kind == TK_COARSE && t.mode == 0) b += 8.0 * h.m0 * h.m0;
            }
            return b;
        }
    }
    return 0.0;
}

extern "C" mg_status mg_profile_solve(mg_hierarchy* hh, const double* b, double* u, mg_result* res,
                                      mg_kernel_time* out, int32_t max_out, int32_t* count) {
    mgi_hier* h = reinterpret_cast<mgi_hier*>(hh);
    if (!h) FAIL(MG_ERR_INVALID, "NULL hierarchy");
    CUCHK(cudaSetDevice(h->device));
    h->prof = true;  // the solve sizes the per-kernel events for the step it runs
    mg_result r{};
    mg_status st = mg_solve(hh, b, u, &r);
    h->prof = false;
    h->prof_pending = false;
    const size_t nops = std::min(h->step.size(), h->prof_ms.size());
    if (res) *res = r;
    if (count) *count = (int32_t)nops;
    for (size_t i = 0; i < nops && (int32_t)i < max_out && out; ++i) {
        const Op& op = h->step[i];
        mg_kernel_time& k = out[i];
        std::memset(&k, 0, sizeof(k));
        k.kind = op.kind == OP_KERNEL ? (op.kkind == K_SWEEP ? 0 : op.kkind == K_PROLONG ? 2
                                         : op.kkind == K_UPDATE ? 5 : 6)
                                      : op.kind;  // OP_TAIL = 7, OP_RESCALE = 8
        k.level = op.level;
        k.mode = op.mode & M_BASE;
        k.loader = 0;
        k.prec = op.prec;
        k.prec_coarse = op.prec_c;
        k.launches = h->prof_cnt[i];
        if (op.kind == OP_KERNEL) {
            k.threads = op.sh.tx * op.sh.ty;
            k.grid[0] = op.sh.gx; k.grid[1] = op.sh.gy; k.grid[2] = op.sh.gz;
        }
        k.total_ms = h->prof_ms[i];
        k.bytes = op_bytes(*h, op);
    }
    return st;
}
