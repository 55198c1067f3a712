// Stage-level entry points of libmgfp (mg_level_write / mg_level_read /
// mg_level_info_get / mg_run_stage): run one production kernel of the method
// on one level so that tests can compare it with the CPU oracle.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "mg_host.h"

using namespace mgi;

#define SFAIL(code, msg)      \
    do {                      \
        mgi_set_error(msg);   \
        return code;          \
    } while (0)
#define SCK(call)                                                                                    \
    do {                                                                                             \
        cudaError_t e_ = (cudaError_t)(call);                                                        \
        if (e_ != cudaSuccess) SFAIL(MG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// Stage calls work on the hierarchy's level arrays: a pooled hierarchy holds
// them only while one of its solves runs.
#define NEED_ARENA(h)                                                                                   \
    do {                                                                                                \
        if (!(h)->bound)                                                                                \
            SFAIL(MG_ERR_INVALID, "a pooled hierarchy holds no working arena outside a solve; stage calls " \
                                  "need a resident hierarchy (pooled = 0)");                            \
    } while (0)

static void* vec_ptr(mgi_hier& h, int level, int vec, int& prec, Geom& geo, void** alloc, size_t* bytes) {
    if (level < 0 || level >= h.nlev) return nullptr;
    Level& L = h.lv[level];
    geo = L.geo;
    if (vec >= MG_VEC_C && vec <= MG_VEC_T) {
        prec = L.prec;
        if (alloc) *alloc = L.alloc[vec];
        if (bytes) *bytes = (size_t)geo.total * L.esz;
        return vec == MG_VEC_C ? L.c : (vec == MG_VEC_G ? L.g : L.t);
    }
    if ((vec == MG_VEC_U || vec == MG_VEC_R) && level == h.nlev - 1) {
        prec = MG_FP64;
        if (alloc) *alloc = vec == MG_VEC_U ? (void*)h.u_alloc : (void*)h.r_alloc;
        if (bytes) *bytes = (size_t)geo.total * 8;
        return vec == MG_VEC_U ? (void*)h.u : (void*)h.r;
    }
    return nullptr;
}

static size_t count_pts(const Geom& g) {
    return g.dim == 3 ? (size_t)g.n * g.n * g.n : (size_t)g.n * g.n;
}

static mg_status order_after_user(mgi_hier& h) {
    SCK(cudaEventRecord(h.ev_in, h.user_stream));
    SCK(cudaStreamWaitEvent(h.stream, h.ev_in, 0));
    return MG_OK;
}

extern "C" mg_status mg_level_write(mg_hierarchy* hh, int32_t level, int32_t vec, const void* src) {
    mgi_hier* h = reinterpret_cast<mgi_hier*>(hh);
    if (!h || !src) SFAIL(MG_ERR_INVALID, "NULL argument");
    NEED_ARENA(h);
    int prec = 0;
    Geom geo;
    void* dst = vec_ptr(*h, level, vec, prec, geo, nullptr, nullptr);
    if (!dst) SFAIL(MG_ERR_INVALID, "no such level vector");
    SCK(cudaSetDevice(h->device));
    mg_status st = order_after_user(*h);
    if (st) return st;
    const size_t bytes = count_pts(geo) * elem_size(prec);
    const void* dsrc = src;
    void* tmp = nullptr;
    if (!mgi_is_device_ptr(src)) {
        SCK(cudaMalloc(&tmp, bytes));
        SCK(cudaMemcpyAsync(tmp, src, bytes, cudaMemcpyHostToDevice, h->stream));
        dsrc = tmp;
    }
    int rc = launch_pack(h->dim, prec, geo, dsrc, dst, h->stream);
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (tmp) cudaFree(tmp);
    if (rc) SFAIL(MG_ERR_CUDA, std::string("pack: ") + cudaGetErrorString((cudaError_t)rc));
    SCK(e);
    return MG_OK;
}

extern "C" mg_status mg_level_read(mg_hierarchy* hh, int32_t level, int32_t vec, void* dst) {
    mgi_hier* h = reinterpret_cast<mgi_hier*>(hh);
    if (!h || !dst) SFAIL(MG_ERR_INVALID, "NULL argument");
    NEED_ARENA(h);
    int prec = 0;
    Geom geo;
    void* src = vec_ptr(*h, level, vec, prec, geo, nullptr, nullptr);
    if (!src) SFAIL(MG_ERR_INVALID, "no such level vector");
    SCK(cudaSetDevice(h->device));
    mg_status st = order_after_user(*h);
    if (st) return st;
    const size_t bytes = count_pts(geo) * elem_size(prec);
    void* ddst = dst;
    void* tmp = nullptr;
    const bool host = !mgi_is_device_ptr(dst);
    if (host) {
        SCK(cudaMalloc(&tmp, bytes));
        ddst = tmp;
    }
    int rc = launch_unpack(h->dim, prec, geo, src, ddst, h->stream);
    if (!rc && host) rc = (int)cudaMemcpyAsync(dst, tmp, bytes, cudaMemcpyDeviceToHost, h->stream);
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (tmp) cudaFree(tmp);
    if (rc) SFAIL(MG_ERR_CUDA, std::string("unpack: ") + cudaGetErrorString((cudaError_t)rc));
    SCK(e);
    return MG_OK;
}

// A tile shape fixed from outside, recorded where the autotuner records its
// choices (kernel_shape reads them for solves and stage calls alike).
extern "C" mg_status mg_tile_set(int32_t kernel, int32_t prec, int32_t n, int32_t rows_per_warp, int32_t march_len) {
    static const int kModes[3] = {M_JACOBI, M_ZERO2, M_RESTRICT};
    if (kernel < 0 || kernel > 2) SFAIL(MG_ERR_INVALID, "mg_tile_set: kernel must be 0 (Jacobi), 1 (two sweeps from zero) or 2 (restriction)");
    if (prec < MG_FP64 || prec > MG_BF16) SFAIL(MG_ERR_INVALID, "mg_tile_set: unknown precision");
    if (n < 3 || n > 1290) SFAIL(MG_ERR_INVALID, "mg_tile_set: n out of range (3..1290)");
    const bool restr = kernel == 2;
    if (rows_per_warp < -1 || rows_per_warp > (restr ? 1 : 2) || (rows_per_warp == 2 && n < 16))
        SFAIL(MG_ERR_INVALID, "mg_tile_set: rows_per_warp out of range");
    if (rows_per_warp > 0 && (march_len < 1 || march_len > (restr ? (n - 1) / 2 : n)))
        SFAIL(MG_ERR_INVALID, "mg_tile_set: march_len out of range");
    if (restr && n < 5) SFAIL(MG_ERR_INVALID, "mg_tile_set: the restriction needs n >= 5");
    if (rows_per_warp < 0) {
        tile_choice_set(3, K_SWEEP, kModes[kernel], prec, n, nullptr);
    } else {
        const TileChoice c{rows_per_warp, rows_per_warp > 0 ? march_len : 0};
        tile_choice_set(3, K_SWEEP, kModes[kernel], prec, n, &c);
    }
    return MG_OK;
}

extern "C" mg_status mg_level_info_get(const mg_hierarchy* hh, int32_t level, mg_level_info* out) {
    const mgi_hier* h = reinterpret_cast<const mgi_hier*>(hh);
    if (!h || !out) SFAIL(MG_ERR_INVALID, "NULL argument");
    if (level < 0 || level >= h->nlev) SFAIL(MG_ERR_INVALID, "no such level");
    const Level& L = h->lv[level];
    out->n = L.geo.n;
    out->prec = L.prec;
    out->pitch = L.geo.P;
    out->tail_ctas = h->tail_level >= 0 && level <= h->tail_level ? h->tail_cs : 0;
    out->bytes = 3 * (size_t)L.geo.total * L.esz;
    // the step's first visit of the level: one fused pre-smoothing + restriction pass, or two launches
    bool pre = false, zero = false, restr = false;
    for (const Op& op : h->step) {
        if (op.kind != OP_KERNEL || op.kkind != K_SWEEP || op.level != level) continue;
        const int m = op.mode & M_BASE;
        pre |= m == M_PRE;
        zero |= m == M_ZERO2 || m == M_ZERO1;
        restr |= m == M_RESTRICT;
    }
    out->pre_launches = pre ? 1 : (zero && restr ? 2 : 0);
    out->reserved_ = 0;
    return MG_OK;
}

// Reduces per-CTA norm partials on the host: out[0] = ||r||_2, out[1] = ||r||_inf.
static mg_status host_norms(mgi_hier& h, int nblocks, int stride, double* out) {
    std::vector<double> p((size_t)nblocks * stride);
    SCK(cudaMemcpy(p.data(), h.partials, p.size() * 8, cudaMemcpyDeviceToHost));
    double s = 0.0;
    unsigned long long m = 0;
    for (int b = 0; b < nblocks; ++b) {
        s += p[(size_t)b * stride];
        unsigned long long k;
        std::memcpy(&k, &p[(size_t)b * stride + 1], 8);
        if (k > m) m = k;
    }
    double mx;
    std::memcpy(&mx, &m, 8);
    if (out) { out[0] = std::sqrt(s); out[1] = mx; }
    return MG_OK;
}

static mg_status copy_back(mgi_hier& h, int level, void* from_base) {
    // The result of a sweep lands in T; copy T's allocation over C's.
    Level& L = h.lv[level];
    (void)from_base;
    SCK(cudaMemcpyAsync(L.alloc[0], L.alloc[2], (size_t)L.geo.total * L.esz, cudaMemcpyDeviceToDevice, h.stream));
    return MG_OK;
}

extern "C" mg_status mg_run_stage(mg_hierarchy* hh, int32_t stage, int32_t level, const double* arg,
                                  const void* ptr_arg, double* out) {
    mgi_hier* h = reinterpret_cast<mgi_hier*>(hh);
    if (!h) SFAIL(MG_ERR_INVALID, "NULL hierarchy");
    if (level < 0 || level >= h->nlev) SFAIL(MG_ERR_INVALID, "no such level");
    NEED_ARENA(h);
    SCK(cudaSetDevice(h->device));
    mg_status st0 = order_after_user(*h);
    if (st0) return st0;
    const int L = h->nlev - 1;
    Level& lv = h->lv[level];
    cudaStream_t s = h->stream;
    int rc = 0;
    switch (stage) {
        case MG_STAGE_JACOBI: {
            Op op = mgi_kernel_op(*h, level, K_SWEEP, M_JACOBI, lv.c, lv.t, lv.g, 0, nullptr);
            rc = mgi_run_op(*h, op, s);
            if (!rc) { mg_status e = copy_back(*h, level, nullptr); if (e) return e; }
            break;
        }
        case MG_STAGE_JACOBI_ZERO2: {
            Op op = mgi_kernel_op(*h, level, K_SWEEP, M_ZERO2, lv.g, lv.c, nullptr, 0, nullptr);
            rc = mgi_run_op(*h, op, s);
            break;
        }
        case MG_STAGE_PRE_RESTRICT: {
            if (level < 1 || h->dim != 3 || h->p.op != 0)
                SFAIL(MG_ERR_INVALID, "the one-pass pre-smoothing needs 3D, level >= 1 and the finite-difference operator");
            Op op = mgi_kernel_op(*h, level, K_SWEEP, M_PRE, lv.g, h->lv[level - 1].g, lv.g, 0, nullptr);
            op.a.dst2 = lv.c;
            rc = mgi_run_op(*h, op, s);
            break;
        }
        case MG_STAGE_RESTRICT_RESCALE: {
            if (level < 1 || !h->rescaled(level - 1))
                SFAIL(MG_ERR_INVALID, "rescaled restriction needs an FP16 level below a non-FP16 level, rescale16 = 1");
            Op op = mgi_kernel_op(*h, level, K_SWEEP, M_RESTRICT, lv.c, h->rsc_alloc + h->lv[level - 1].geo.base,
                                  lv.g, 0, nullptr);
            op.prec_c = MG_FP32;
            rc = mgi_run_op(*h, op, s);
            if (!rc) {
                Op r{};
                r.kind = OP_RESCALE;
                r.level = level - 1;
                r.prec = r.prec_c = MG_FP16;
                r.ptr = h->lv[level - 1].g;
                rc = mgi_run_op(*h, r, s);
            }
            if (rc) SFAIL(MG_ERR_CUDA, std::string("stage launch: ") + cudaGetErrorString((cudaError_t)rc));
            double sc = 0.0;
            SCK(cudaMemcpyAsync(&sc, &h->st->lscale[level - 1], sizeof(double), cudaMemcpyDeviceToHost, s));
            SCK(cudaStreamSynchronize(s));
            if (out) { out[0] = sc; out[1] = 0.0; }
            return MG_OK;
        }
        case MG_STAGE_RESTRICT: {
            if (level < 1) SFAIL(MG_ERR_INVALID, "restriction needs level >= 1");
            Op op = mgi_kernel_op(*h, level, K_SWEEP, M_RESTRICT, lv.c, h->lv[level - 1].g, lv.g, 0, nullptr);
            rc = mgi_run_op(*h, op, s);
            break;
        }
        case MG_STAGE_PROLONG:
        case MG_STAGE_JACOBI_PROLONG: {
            if (level < 1) SFAIL(MG_ERR_INVALID, "prolongation needs level >= 1");
            Op op = mgi_kernel_op(*h, level, K_PROLONG, 0, nullptr, lv.c, nullptr, 0, nullptr);
            op.a.coarse = h->lv[level - 1].c;
            if (arg) {  // the coarse correction's scale, staged in the level's scale slot
                double* slot = &h->st->lscale[level - 1];
                SCK(cudaMemcpyAsync(slot, arg, sizeof(double), cudaMemcpyHostToDevice, s));
                op.a.cscale = slot;
            }
            rc = mgi_run_op(*h, op, s);
            if (!rc && stage == MG_STAGE_JACOBI_PROLONG) {
                Op sw = mgi_kernel_op(*h, level, K_SWEEP, M_JACOBI, lv.c, lv.t, lv.g, 0, nullptr);
                rc = mgi_run_op(*h, sw, s);
                if (!rc) { mg_status e = copy_back(*h, level, nullptr); if (e) return e; }
            }
            break;
        }
        case MG_STAGE_COARSE: {
            if (level != 0) SFAIL(MG_ERR_INVALID, "base solve runs on level 0");
            Op op{};
            op.kind = OP_COARSE;
            op.prec = lv.prec;
            op.g = lv.g;
            op.c = lv.c;
            rc = mgi_run_op(*h, op, s);
            break;
        }
        case MG_STAGE_SCALE_ZERO2: {
            if (level != L) SFAIL(MG_ERR_INVALID, "scale-cast runs on the finest level");
            if (!arg) SFAIL(MG_ERR_INVALID, "arg[0] (scale) required");
            Op op = mgi_kernel_op(*h, level, K_SCALE, 0, nullptr, lv.g, nullptr, 0, nullptr);
            op.a.inv_explicit = arg[0];
            rc = mgi_run_op(*h, op, s);
            if (!rc && L > 0) {
                Op sw = mgi_kernel_op(*h, level, K_SWEEP, M_ZERO2, lv.g, lv.c, nullptr, 0, nullptr);
                rc = mgi_run_op(*h, sw, s);
            }
            break;
        }
        case MG_STAGE_IR_UPDATE: {
            if (level != L) SFAIL(MG_ERR_INVALID, "update runs on the finest level");
            if (!arg) SFAIL(MG_ERR_INVALID, "arg[0] (alpha) required");
            Op op = mgi_update_op(*h, lv.c, 0, nullptr);
            op.a.a_step = arg[0];
            // arg[1] > 0 (a power of two): also write G_L = cast(trunc_FP32(R_new arg[1]))
            op.a.dst = lv.prec != MG_FP64 && arg[1] > 0.0 ? lv.g : nullptr;
            op.a.inv_explicit = op.a.dst ? arg[1] : 0.0;
            op.mode = (op.mode & ~M_SA) | (op.a.dst ? M_SA : 0);
            rc = mgi_run_op(*h, op, s);
            if (!rc) {
                SCK(cudaStreamSynchronize(s));
                return host_norms(*h, op.sh.nblocks(), 2, out);
            }
            break;
        }
        case MG_STAGE_RESIDUAL: {
            if (level != L) SFAIL(MG_ERR_INVALID, "residual runs on the finest level");
            if (!ptr_arg || !mgi_is_device_ptr(ptr_arg)) SFAIL(MG_ERR_INVALID, "ptr_arg must be a device pointer to b");
            const Geom& g = lv.geo;
            RArgs a{};
            a.n = g.n; a.P = g.P; a.S = g.S;
            a.u = h->u; a.b = (const double*)ptr_arg; a.r = h->r; a.partials = h->partials;
            a.need_b = 1;
            a.h2inv = op_alpha(h->p.op, h->dim, g.n);
            a.op = h->p.op;
            int nb = 0;
            rc = launch_residual64(h->dim, a, &nb, s);
            if (!rc) {
                SCK(cudaStreamSynchronize(s));
                return host_norms(*h, nb, 4, out);
            }
            break;
        }
        case MG_STAGE_CYCLE: {
            if (level != L) SFAIL(MG_ERR_INVALID, "a cycle starts on the finest level");
            std::vector<Op> ops;
            h->tail_host.resize(h->step_tail_ops);  // stage programs follow the IR step's
            void* cL = mgi_build_cycle(*h, ops, false, 0, nullptr);
            if (!cL) SFAIL(MG_ERR_INVALID, "coarse-tail program capacity exceeded");
            for (const Op& op : ops) {
                rc = mgi_run_op(*h, op, s);
                if (rc) break;
            }
            if (!rc && cL != lv.c) { mg_status e = copy_back(*h, level, nullptr); if (e) return e; }
            break;
        }
        default:
            SFAIL(MG_ERR_INVALID, "unknown stage");
    }
    if (rc) SFAIL(MG_ERR_CUDA, std::string("stage launch: ") + cudaGetErrorString((cudaError_t)rc));
    SCK(cudaStreamSynchronize(s));
    if (out) out[0] = out[1] = 0.0;
    return MG_OK;
}
