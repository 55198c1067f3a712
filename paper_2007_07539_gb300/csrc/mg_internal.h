// Internal declarations shared by the host code and the CUDA kernels of libmgfp.
//
// Padded level layout (every level vector, every storage type):
//   row pitch P = round_up(n + 1, 16) elements; rows y = 0..n per plane, row n
//   all zero; planes z = -1..n (3D), planes -1 and n all zero; a zero guard of
//   2P + 32 elements before plane -1 and after plane n.  Element (x, y, z) sits
//   at base + z*S + y*P + x with S = P*(n+1) (3D; 2D has no z term).
// Only interior points (x, y, z < n) are ever written with non-zero values, so
// every read at x = -1 or x = n (the previous/this row's pad column), y = -1
// or y = n (a pad row) and z = -1 or z = n (a pad plane) returns the zero
// Dirichlet boundary value without a branch.  P is a multiple of 16 elements,
// so x = 0 of every row is 16-byte aligned for all types.
#pragma once
#include <cuda.h>

#include <cstddef>
#include <cstdint>

#include "../../include/mg.h"

namespace mgi {

constexpr int kMaxHist = 1024;
constexpr int kMaxIter = 1000;

struct Geom {
    int dim = 0;
    int n = 0;          // interior points per dimension
    int P = 0;          // row pitch (elements)
    long long S = 0;    // plane stride (elements): P*(n+1)
    long long base = 0; // element offset of (0,0,0) in the allocation
    long long total = 0;// allocated elements
};

inline Geom make_geom(int dim, int n) {
    Geom g;
    g.dim = dim;
    g.n = n;
    g.P = ((n + 1 + 15) / 16) * 16;
    g.S = (long long)g.P * (n + 1);
    long long guard = 2LL * g.P + 32;
    if (dim == 3) {
        g.base = guard + g.S;                         // plane -1 precedes (0,0,0)
        g.total = g.base + (long long)(n + 1) * g.S + guard;
    } else {
        g.base = guard + g.P;                         // row -1 precedes (0,0)
        g.total = g.base + (long long)(n + 1) * g.P + guard;
    }
    g.total = ((g.total + 127) / 128) * 128;
    return g;
}

// Device-side solver state of one solve (one per hierarchy / solve slot).
struct DevState {
    double alpha;     // scale of the current correction: u += alpha c, r -= alpha A c
    double inv;       // sigma/alpha: the scaled residual is r * inv
    double rnorm2;    // ||r||_2 of the current recursive residual
    double rnorminf;  // ||r||_inf
    double bnorm2;    // ||b||_2
    double tol_abs;   // threshold on ||r||_2
    double sigma;     // 2^sigma_log2
    double rel_true;  // last ||b - A u||_2 / ||b||_2
    double tol;
    int iter;         // completed IR steps
    int phase;        // 0 iterate, 1 recursive test passed (guard pending), 2 converged, 3 stopped
    int status;       // mg_status
    int guard_restarts;
    int max_iter;
    int scaling;
    int tol_mode;
    int guard;
    int stag;         // consecutive steps without decrease
    int dirty;        // u changed since it was last copied to the caller's array
    int loops;        // body iterations of the device-side IR loop (bounded)
    int kerr;         // non-zero: a kernel's bounded wait for its tile copies ran out
    int scale_ahead;  // 1: the update writes the next g with inv_pred (mg_params.scale_ahead in effect)
    int g_ready;      // 1: g of the coming step was written by the last update (the scale-cast returns)
    int gover;        // set by the update when a scaled g value overflowed the storage type
    int fin_count;    // IR update CTAs done in this step (the last one finalises)
    double inv_pred;  // scale-ahead: sigma / 2^e, 2^e the power of two above the last ||r||_inf
    double lscale[MG_MAX_LEVELS];  // power-of-two scale of each rescaled FP16 level's residual
    const double* b;  // caller's right-hand side (device, contiguous)
    double* uout;     // caller's solution (device, contiguous): u0 in, u out
    double hist[kMaxHist + 2];
};

// Kernel kinds of the fine-level TUs.
enum Kind : int {
    K_SWEEP = 0,    // stencil sweep (mode below)
    K_UPDATE = 1,   // u += alpha c; r -= alpha A c; norm partials (Alg. 2's solution and residual updates)
    K_SCALE = 2,    // g = cast(r * inv) (Alg. 2's residual scaling)
    K_PROLONG = 3,  // c += P c_coarse (Alg. 1's prolongation and correction)
};

enum Mode : int {
    M_JACOBI = 0,   // dst = c + w D^-1 (g - A c)
    M_ZERO2 = 1,    // dst = two sweeps from zero; the swept vector is g
    M_ZERO1 = 2,    // dst = w D^-1 g
    M_RESTRICT = 3, // coarse dst = R (g - A c)
    M_PRE = 4,      // dst2 = two sweeps from zero of g (src = g); coarse dst = R (g - A dst2): one pass
};
// Flag or'ed into the mode of the stencil kernels (sweeps, IR update) of a
// hierarchy with the Q1 finite-element operator (op = 1); M_BASE masks it off.
constexpr int M_FEM = 16;
constexpr int M_BASE = 15;
// Flag or'ed into the mode of the IR update when it also writes the next
// step's scaled g (scale-ahead, non-FP64 finest levels): that instantiation
// sums the squares of r in FP32, from the scaled FP32 values it forms for g.
constexpr int M_SA = 32;

// The operator of a level, A = alpha (beta I - W), W the sum of neighbour
// values with positive integer weights (Sec. 5):
//   op 0, finite differences: alpha = h^-2, beta = 2d, weight 1 on the 2d axis neighbours;
//   op 1, Q1 elements (stiffness / h^d): 2D alpha = h^-2/3, beta = 8, weight 1 on the 8
//     neighbours; 3D alpha = h^-2/12, beta = 32, weight 2 on the 12 edge neighbours, 1 on
//     the 8 corners, 0 on the 6 faces.
inline double op_alpha(int op, int dim, int n) {
    const double h2inv = (double)(n + 1) * (double)(n + 1);
    return op == 1 ? h2inv / (dim == 3 ? 12.0 : 3.0) : h2inv;
}
inline int op_beta(int op, int dim) { return op == 1 ? (dim == 3 ? 32 : 8) : 2 * dim; }

// Arguments of the fine-level kernels (passed by value).
// Sweep coefficients of A = alpha (beta I - W), computed once on the host in
// the arithmetic type (the same IEEE operations the kernels would do):
// c1 = 1 - w, c2 = w/beta, c3 = w/(beta alpha) = w D^-1, k2 = 2 - w, alpha,
// -beta alpha.  Jacobi: c1 c + c2 W c + c3 g; two sweeps from zero:
// c3 (k2 g + c2 W g); residual: g + alpha W c - beta alpha c.
struct SweepCoef {
    float f[6];
    double d[6];
};
inline SweepCoef make_sweep_coef(int dim, int op, double omega, double alpha) {
    SweepCoef c;
    const float om = (float)omega, h2 = (float)alpha, twod = (float)op_beta(op, dim);
    c.f[0] = 1.0f - om; c.f[1] = om / twod; c.f[2] = om / (twod * h2); c.f[3] = 2.0f - om; c.f[4] = h2; c.f[5] = -twod * h2;
    const double dom = omega, dh2 = alpha, dtwod = (double)op_beta(op, dim);
    c.d[0] = 1.0 - dom; c.d[1] = dom / dtwod; c.d[2] = dom / (dtwod * dh2); c.d[3] = 2.0 - dom; c.d[4] = dh2; c.d[5] = -dtwod * dh2;
    return c;
}

struct KArgs {
    int n, P;            // this level
    long long S;
    int nc, Pc;          // coarser level (restrict target / prolong source)
    long long Sc;
    const void* src;     // swept vector / correction (T)
    const void* g;       // right-hand side (T)
    void* dst;           // output (T, or TC for M_RESTRICT / M_PRE)
    void* dst2;          // M_PRE: the smoothed correction (T)
    const void* coarse;  // coarse correction (TC) for K_PROLONG
    const double* cscale;// K_PROLONG: scale of the coarse correction (a rescaled level), null = 1
    const double* r64;   // FP64 residual for K_SCALE (padded, finest geometry)
    double* u64;         // K_UPDATE: FP64 solution (padded)
    double* rw64;        // K_UPDATE: FP64 residual (padded)
    double* partials;    // per-CTA norm partials (K_UPDATE): 2 doubles each
    const DevState* st;  // alpha / inv, phase (early exit)
    double a_step;       // K_UPDATE explicit alpha when st == nullptr
    double inv_explicit; // K_SCALE explicit scale when st == nullptr
    double omega;
    double h2inv;        // alpha of this level's operator (h^-2 for finite differences)
    int xstep, ystep, zstep, zlen;  // tile strides / march length
    int gate;            // 1: return at once unless st->phase == 0
    int fin;             // K_UPDATE: the last CTA runs the step's finalisation (FIN_STEP)
    int* err;            // set to 1 when a bounded copy wait runs out (3D sweeps), 2 if the drain also did
    int wait_polls;      // 3D sweeps: k + 1 for k polls per wait for a plane's copies; 0: the default bound
    SweepCoef cf;        // sweep coefficients of this level (host-computed)
};

// Arguments of the FP64 residual kernel r = b - A u.
struct RArgs {
    int n, P;
    long long S;
    const double* u;      // padded
    const double* b;      // contiguous interior (n^d); from st->b when null
    double* r;            // padded output (may be null)
    double* uout;         // contiguous interior copy of u (may be null; st->uout with use_st_uout)
    double* partials;     // 4 doubles per CTA: sum r^2, max |r|, sum b^2, unused
    const DevState* st;   // control state (gating, caller pointers); may be null
    double h2inv;         // alpha of the operator (op_alpha)
    int op;               // 0 finite differences, 1 Q1 elements
    int gate;             // 0 always run; 1 only when st->phase == 1; 2 only when st->dirty
    int use_st_uout;      // 1: copy u to st->uout
    int need_b;           // 1: also the partial sums of b^2 (initial residual, stage calls)
};

struct RItem {
    RArgs a;
    int ncta, cta_begin;
};
struct FinItem {
    DevState* st;
    const double* partials;
    int nblocks;
};

struct MarchShape {
    int gx, gy, gz, tx, ty;
    int rpw;  // 3D sweeps: rows per warp (the CTA tile has ty * rpw rows); 0: the direct
              // small-level kernels (k_dsweep3 / k_drestrict3, one thread per vector / coarse point)
    size_t smem;
    int xstep, ystep, zstep, zlen;
    int nblocks() const { return gx * gy * gz; }
};
// Launch geometry of a fine-level kernel over a level of size n (pitch P).
MarchShape kernel_shape(int dim, int kind, int mode, int prec, int n, int P, int tz_hint);

// Autotuned tile shapes of the 3D stencil kernels, per (kind, mode, storage
// type, level size): rows per warp and march length (planes per CTA for the
// sweeps, coarse planes per CTA for the residual-restriction).  kernel_shape
// uses an entry when there is one, else its wave model.
struct TileChoice {
    int rpw, zlen;  // rpw 0: the direct kernel
};
// Default for levels of at most this many points per dimension (3D, finite
// differences, untuned): the direct kernels.
constexpr int kDirectMaxN = 63;
void tile_choice_set(int dim, int kind, int mode, int prec, int n, const TileChoice* c);  // nullptr: erase
bool tile_choice_get(int dim, int kind, int mode, int prec, int n, TileChoice* c);
// Sweeps per launch of a 3D level's pre-smoothing (two sweeps from zero and the
// residual-restriction): 1 = one fused pass (M_PRE), 0 = two launches; -1: not tuned.
void fuse_choice_set(int prec, int prec_c, int n, int fused);
int fuse_choice_get(int prec, int prec_c, int n);

// TMA descriptors of the 3D sweeps: the swept vector (boxes of TY+2 rows with
// a 16-byte x-halo on each side) and the right-hand side (TY rows, no halo).
// Both describe a padded level vector as a 3D tensor of 4-byte units (2-byte
// types) or 8-byte units (4- and 8-byte types): x over the pitch, y over rows
// 0..n (the pad row included), z over planes -1..n.
struct alignas(64) SweepMaps {
    CUtensorMap src;
    CUtensorMap g;
};
// Work items of the batched (level-synchronous) launches: one per instance,
// owning CTAs [cta_begin, cta_begin + its grid size) of the merged grid.
struct alignas(64) SweepItem {
    SweepMaps maps;
    KArgs a;
    int gx, gy, gz, cta_begin;
};
struct KItem {
    KArgs a;
    int ncta, cta_begin;
};

// Encodes one map for level vector `x0` (the address of element (0,0,0)).
int make_sweep_map(CUtensorMap* m, int prec, const Geom& geo, const void* x0, int rows, bool halo);

// Shared-memory plan of the 3D sweep, identical on host and device.
// Ring of kSweepStages stages, each [c box: (R+2) rows x 544 B, 128-aligned]
// [g box: R rows x 512 B] for a tile of R rows, then the restriction's flush
// area, then one mbarrier per stage.
constexpr int kSweepStages = 6;
#ifdef __CUDACC__
__host__ __device__
#endif
constexpr int sweep3_stages(int, int) { return kSweepStages; }
constexpr int kSweepRowBytes = 544;
#ifdef __CUDACC__
__host__ __device__
#endif
inline int sweep3_cbytes(int ty) { return ((ty + 2) * kSweepRowBytes + 127) / 128 * 128; }
#ifdef __CUDACC__
__host__ __device__
#endif
inline int sweep3_stage_bytes(int ty, bool need_g) { return (sweep3_cbytes(ty) + (need_g ? ty * 512 : 0) + 127) / 128 * 128; }
// One-pass pre-smoothing + residual + restriction (M_PRE) on a tile of R
// residual rows: a 6-stage ring of g boxes (R+4 rows), a 3-plane ring of the
// smoothed correction (R+2 rows, in the storage type), the restriction's
// flush area, 6 mbarriers.
constexpr int kPreStagesG = 6;
constexpr int kPreStagesC = 3;
#ifdef __CUDACC__
__host__ __device__
#endif
inline int pre3_gbytes(int r) { return ((r + 4) * kSweepRowBytes + 127) / 128 * 128; }
#ifdef __CUDACC__
__host__ __device__
#endif
inline int pre3_cbytes(int r) { return ((r + 2) * kSweepRowBytes + 127) / 128 * 128; }
#ifdef __CUDACC__
__host__ __device__
#endif
inline int pre3_smem(int r, int flush_bytes) {
    return 128 + kPreStagesG * pre3_gbytes(r) + kPreStagesC * pre3_cbytes(r) + (flush_bytes + 15) / 16 * 16 + kPreStagesG * 8;
}
#ifdef __CUDACC__
__host__ __device__
#endif
inline int sweep3_smem(int ty, bool need_g, int flush_bytes, int stages = kSweepStages) {
    return 128 + stages * sweep3_stage_bytes(ty, need_g) + (flush_bytes + 15) / 16 * 16 + stages * 8;
}

// Launches a fine-level kernel (one translation unit per fine storage type);
// maps: the TMA descriptors of a 3D sweep (nullptr for other kernels).
int launch_kernel(int dim, int kind, int mode, int prec, int prec_c, const KArgs& a, const MarchShape& s,
                  const SweepMaps* maps, void* stream);

// Misc kernels (mg_misc.cu).
// Rescale of a restricted residual into an FP16 level: x is the FP32
// restriction (padded, geometry geo), g the FP16 level vector; s = 2^-k with
// max|x| 2^k in [2^(sig-1), 2^sig) is written to *scale and g = cast(x 2^k).
// part holds kRescaleCtas floats.
constexpr int kRescaleCtas = 304;
int launch_rescale(const float* x, void* g, const Geom& geo, float* part, int sig, double* scale,
                   const DevState* st, int gate, void* stream);
// Conjugate gradients on the base level (one CTA; Sec. 6), in the level's type.
int launch_coarse_cg(int prec, int op, const void* g, void* c, const Geom& geo, double tol, int maxit,
                     const DevState* st, int gate, void* stream);
int launch_coarse_solve(int prec, const double* inv, int m, const void* g, void* c, const Geom& geo,
                        const DevState* st, int gate, void* stream);
int launch_residual64(int dim, const RArgs& a, int* nblocks, void* stream);
int launch_init_rb(int dim, const Geom& geo, const double* b, double* r, double* partials, const DevState* st,
                   int* nblocks, void* stream);
int launch_finalize(int kind, DevState* st, const double* partials, int nblocks, void* stream);
// u (padded) <- st->uout (the caller's initial guess)
int launch_pack_u0(int dim, const Geom& geo, const DevState* st, double* u_padded, void* stream);
// Condition of the device-side IR loop: continue while phase is 0 or 1 and the
// body has run fewer than `limit` times.
int launch_loop_condition(DevState* st, unsigned long long handle, int limit, void* stream);
// Batched counterparts (level-synchronous batch solves): one launch for all
// instances; cta_item maps each CTA of the merged grid to its work item.
int launch_finalize_batch(int kind, const FinItem* items, int nitems, void* stream);
int launch_loop_condition_batch(DevState* const* sts, int n, unsigned long long handle, int limit, void* stream);
int launch_residual64_batch(int dim, bool init_copy, const RItem* items, const int* cta_item, int ncta, void* stream);
int residual64_ctas(int dim, int n);
int launch_kernel_batch(int kind, int mode, int prec, int prec_c, int rpw, const void* items, const int* cta_item,
                        int ncta, int ty, size_t smem, void* stream);
int launch_pack(int dim, int prec, const Geom& geo, const void* src_contig, void* dst_padded,
                void* stream);
int launch_unpack(int dim, int prec, const Geom& geo, const void* src_padded, void* dst_contig,
                  void* stream);

enum FinalizeKind : int { FIN_INIT = 0, FIN_STEP = 1, FIN_GUARD = 2, FIN_REPORT = 3 };

size_t elem_size(int prec);

}  // namespace mgi
