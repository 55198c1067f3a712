/*
 * mg.h - C ABI of libmgfp, a GB300 (sm_103a) solver for finite-difference
 * Poisson problems by mixed-precision iterative refinement preconditioned with
 * one geometric-multigrid cycle per step.
 *
 * Method: K. L. Oo and A. Vogel, "Accelerating Geometric Multigrid
 * Preconditioning with Half-Precision Arithmetic on GPUs", arXiv 2007.07539.
 *   - Iterative refinement (IR), Sec. 4.1: r = b - A u; solve A c = r
 *     approximately; u = u + c.
 *   - Multigrid cycle, Sec. 4.2 and Alg. 1: damped-Jacobi pre-smoothing,
 *     residual, restriction with a precision change, coarse correction,
 *     prolongation with a precision change, post-smoothing; exact solve on the
 *     coarsest (base) level; recursion gives the V-cycle (gamma = 2: W-cycle).
 *   - Per-level precisions, Table 2 and Fig. 1 (D_MG, H_MG, HSD_MG, DSH_MG).
 *   - Mixed-precision IR with residuum scaling, Sec. 4.3 and Alg. 2:
 *     alpha = ||r||; r_low = (1/alpha) r_high; one cycle gives c_low;
 *     u += alpha c_low; r -= alpha A c_low, with r, u and the stopping test in FP64.
 *   - Model problem, Sec. 5 (Eq. 1): -Laplace(u) = f on the unit square/cube,
 *     u = 0 on the boundary, on n interior points per dimension, h = 1/(n+1).
 *     Discretised by the 5-point (2D) / 7-point (3D) finite-difference stencil,
 *     (A u)_p = h^-2 (2d u_p - sum of the 2d axis neighbours) (op = 0), or by
 *     the paper's bilinear / trilinear Q1 finite elements (op = 1, 9/27-point,
 *     the stiffness matrix divided by h^d; see mg_params.op).
 *
 * Conventions for every entry point:
 *   - Grid vectors passed by the caller (b, u) are interior-only, contiguous,
 *     FP64, x fastest: element (i, j[, k]) at i + n*j [+ n*n*k], i.e. the
 *     C-order layout of an array of shape (n, n[, n]) indexed [k][j][i].
 *   - Pointers may be device pointers (cudaMalloc / torch CUDA tensors) or
 *     host pointers (pinned or pageable); the library detects which with
 *     cudaPointerGetAttributes and copies host data through its own device
 *     staging buffers on the hierarchy's stream, except a pinned u, which the
 *     kernels read and write in place over the host link.  The caller keeps
 *     ownership.
 *   - Every call returns an mg_status; nothing throws across the ABI.  On an
 *     error mg_last_error() returns a message for the calling thread.
 *   - A hierarchy is bound to the device that was current at creation and to
 *     the CUDA stream given there.  Calls on one hierarchy must not run
 *     concurrently from several host threads.
 */
#ifndef MG_H
#define MG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MG_ABI_VERSION 2
#define MG_MAX_LEVELS 16

/* Storage precision of one multigrid level (Table 2, Fig. 1).  Arithmetic
 * inside a sweep is FP32 for FP16/BF16/FP32 levels and FP64 for FP64 levels. */
typedef enum { MG_FP64 = 0, MG_FP32 = 1, MG_FP16 = 2, MG_BF16 = 3 } mg_prec;

typedef enum {
    MG_OK = 0,
    MG_BUSY = 1,               /* mg_poll: request still running */
    MG_ERR_INVALID = 2,        /* bad argument or parameter */
    MG_ERR_OOM = 3,            /* device allocation failed */
    MG_ERR_CUDA = 4,           /* a CUDA call failed */
    MG_ERR_NOT_CONVERGED = 5,  /* max_iter reached, or the residual stagnated */
    MG_ERR_NUMERIC = 6,        /* non-finite residual */
    MG_ERR_TIMEOUT = 7,        /* a bounded device wait expired */
    MG_ERR_ADMISSION = 8       /* request can never fit the memory budget */
} mg_status;

/* Solver parameters.  Fill with mg_params_init() and then override fields. */
typedef struct mg_params {
    int32_t dim;        /* 2 or 3 */
    int32_t n;          /* interior points per dimension on the finest level (>= 1) */
    int32_t levels;     /* number of levels; 0 = as many as the coarsening rule allows.
                           Rule: n_{l-1} = (n_l - 1)/2 while n_l is odd and > 3; the
                           coarsest level must have at most 4096 unknowns */
    int32_t prec[MG_MAX_LEVELS]; /* mg_prec per level, prec[0] = coarsest (base level),
                           prec[levels-1] = finest; default all MG_FP64 (D_MG) */
    int32_t nu1, nu2;   /* pre-/post-smoothing sweeps (Alg. 1's pre- and post-smoothing); default 2, 2 */
    double omega;       /* Jacobi damping; default 0.8 (the paper uses 2/3, Sec. 4.2) */
    int32_t gamma;      /* coarse visits per level: 1 = V-cycle (default), 2 = W-cycle */
    int32_t scaling;    /* the scale alpha of Alg. 2's residual scaling: 0 = none (alpha = 1, the paper's
                           choice for D_MG, Sec. 6), 1 = ||r||_inf (default), 2 = ||r||_2 */
    int32_t sigma_log2; /* the scaled residual is r * 2^sigma_log2 / alpha, so its inf-norm
                           is 2^sigma_log2 (scaling = 1); -1 = automatic: 14 when any
                           level is FP16, else 0.  Ignored when scaling = 0 */
    int32_t tol_mode;   /* 0: stop when ||r||_2 <= tol ||b||_2 (default);
                           1: stop when ||r||_2 < tol (the paper's absolute test, Sec. 6) */
    double tol;         /* default 1e-10 */
    int32_t max_iter;   /* IR step limit; default 100, at most 1000 */
    int32_t zero_guess; /* 1: ignore u on entry and start from u0 = 0 (default 0) */
    int32_t guard;      /* 1 (default): when the recursively updated residual passes the
                           test, recompute b - A u in FP64 and continue from it if it fails */
    int32_t graph;      /* 1 (default): run the whole solve as one CUDA graph launch with a
                           device-side IR loop; 0: one launch per kernel from a host loop */
    int32_t no_tail;    /* coarse-tail kernel (the coarsest levels' cycle in one launch with the levels
                           in shared memory): 0 (default) in one CTA; 1: no tail (every level as
                           plain kernels); 2: in one CTA or in a thread-block cluster of 16 or 8
                           CTAs sharing their shared memory (levels up to 2^15 points), whichever
                           covers more levels (same results; measured no faster on GB300 at the
                           benchmark sizes) */
    int32_t tune;       /* 1: autotune at creation: every 3D stencil kernel of the hierarchy
                           (sweeps from zero, residual-restriction, Jacobi; per level) is timed
                           on the device with candidate tile shapes -- rows per warp and march
                           length -- and the fastest is kept for this process (shared by later
                           hierarchies with the same level sizes and types).  Results do not
                           depend on the tile shape.  Default 0: shapes from the wave model */
    int32_t fuse_pre;   /* sweeps per launch of the pre-smoothing: 1: the two sweeps from zero and
                           the residual-restriction in one pass over each level (3D finite
                           differences; temporal blocking: half the bytes and one launch,
                           bit-identical results); 2: per level, whichever of the one pass and
                           the two launches the autotuner (tune = 1) times faster (without tune:
                           two launches); default 0: two launches, which are faster on GB300 at
                           every level size measured (both forms are bound by latency, not DRAM) */
    int32_t rescale16;  /* 1 (default): when a restriction goes from a non-FP16 level into an
                           FP16 level (DSH_MG, Sec. 6), the restricted residual is divided by a
                           power of two s so that its inf-norm lies in [2^(k-1), 2^k), k the
                           sigma_log2 in effect (14 with FP16 levels); the correction
                           prolongated back from that level is multiplied by s.  0: off */
    int32_t base_solver;/* 0 (default): exact base solve with the dense FP64 inverse;
                           1: conjugate gradients in the base level's precision (Sec. 6:
                           x, r, p stored in the level's type, A p and dot products in its
                           arithmetic type), from x = 0, until ||r||_2 <= base_tol ||g||_2
                           or base_maxit steps */
    int32_t base_maxit; /* CG step limit, at most 100000; 0 = the number of base-level unknowns */
    double base_tol;    /* CG relative tolerance; default 1e-4 */
    int32_t op;         /* discretisation of -Laplace (Sec. 5): 0 (default) finite differences,
                           5-point (2D) / 7-point (3D), A = h^-2 (2d I - axis neighbours);
                           1 bilinear / trilinear Q1 finite elements, the stiffness matrix
                           divided by h^d: 2D A = h^-2/3 (8 I - the 8 neighbours), 3D
                           A = h^-2/12 (32 I - 2 x the 12 edge - the 8 corner neighbours).
                           b is then the load vector divided by h^d.  Coarse levels use the
                           same operator at their h (for Q1 this equals the Galerkin
                           product of full weighting, A and interpolation).  op = 1
                           requires fuse_pre = 0 */
    int32_t scale_ahead;/* 1 (default): with scaling = 1 and a non-FP64 finest level, the fused
                           IR update (Alg. 2's solution and residual updates) also writes the next step's g =
                           cast(r * 2^k) (Alg. 2's residual scaling), with 2^k = 2^sigma_log2 / 2^e and 2^e the
                           power of two just above the previous ||r||_inf, so the separate
                           scale-and-cast pass over the FP64 residual is skipped; alpha is
                           then 2^-k, a power of two within a factor of two of the previous
                           residual's norm instead of the current one.  When the scaled
                           values would overflow the storage type, that step falls back to
                           the scale-and-cast with alpha = ||r||_inf.  0: always
                           alpha = ||r||_inf and the separate pass */
    int32_t wait_polls; /* bound on each wait of the 3D stencil kernels for their TMA tile copies,
                           in polls of the copy barrier (each poll may suspend the thread for a
                           short hardware-chosen time): -1 (default) about a second in all;
                           >= 0 that many polls (a diagnostic for the timeout path: 0 gives up at
                           once, while the copies still land).  A wait that gives up stops the
                           solve with MG_ERR_TIMEOUT; the kernel first waits, with the default
                           bound, for every copy it issued, so none is in flight at its exit,
                           and later solves are unaffected */
    int32_t pooled;     /* 0 (default): the hierarchy allocates its working arena (the level
                           vectors and the FP64 u and r, nearly all of mg_footprint_bytes) at
                           creation and holds it until mg_destroy.  1: the hierarchy holds
                           only its plan and small control state; the arena is taken from the
                           library's device-memory pool when a solve is admitted (mg_submit)
                           or started (mg_solve, mg_solve_batch) and handed back to the pool
                           when it completes, so idle hierarchies hold no working memory and
                           the serving budget bounds the memory in use (mg_serve_configure) */
    int32_t reserved[4];/* must be 0 */
} mg_params;

/* Outcome of one solve. */
typedef struct mg_result {
    int32_t iters;          /* IR steps performed */
    int32_t status;         /* mg_status of the solve */
    int32_t levels;         /* levels used */
    int32_t guard_restarts; /* times the true residual replaced the recursive one */
    int32_t launches;       /* kernels of this library launched by the solve */
    int32_t merged;         /* mg_solve_batch: 1 if the level-synchronous merged launches ran */
    double rel_res;         /* recursive ||r||_2 / ||b||_2 at exit */
    double rel_res_true;    /* ||b - A u||_2 / ||b||_2 at exit, computed in FP64 */
    double bnorm;           /* ||b||_2 */
    double seconds;         /* device time of the solve (CUDA events) */
} mg_result;

typedef struct mg_hierarchy mg_hierarchy; /* opaque; owns all device state of a solver */

/* Describes one level of a hierarchy (for tests and diagnostics). */
typedef struct mg_level_info {
    int32_t n;        /* interior points per dimension */
    int32_t prec;     /* mg_prec */
    int32_t pitch;    /* row pitch of the padded device layout, in elements */
    int32_t tail_ctas;/* 0: the level runs as level kernels; else it is in the coarse tail,
                         held by this many CTAs (1, or a thread-block cluster of 8 / 16) */
    size_t bytes;     /* device bytes held for this level */
    int32_t pre_launches; /* launches of the level's pre-smoothing and residual-restriction in
                         the IR step (1: one fused pass, 2: two; 0: none, e.g. coarse tail) */
    int32_t reserved_;
} mg_level_info;

/* ---------------------------------------------------------------- basics */

/* Fills *p with the defaults listed above for the given dim and n. */
void mg_params_init(mg_params* p, int32_t dim, int32_t n);

/* Number of levels the coarsening rule gives for n (levels_req = 0) or the
 * smaller of that and levels_req; fills sizes[0..count-1] (coarsest first)
 * when sizes is not NULL.  Returns 0 for invalid n. */
int32_t mg_level_count(int32_t n, int32_t levels_req, int32_t* sizes);

/* Message describing the last error on this host thread ("" if none). */
const char* mg_last_error(void);

/* Device bytes a hierarchy with these parameters will hold (0 if invalid). */
size_t mg_footprint_bytes(const mg_params* p);

/* The operations of one IR step's multigrid cycle as the library schedules
 * them, computed on the host without a device: the Alg. 1 recursion (nu1
 * pre-smoothing sweeps, residual-restriction, gamma visits of the coarser
 * level, prolongation, nu2 post-smoothing sweeps; base solve on level 0),
 * preceded by the scale-and-cast of Alg. 2's residual scaling, with the coarse tail and
 * the FP16 rescale of Sec. 6 where the hierarchy has them.
 * rec receives records of 6 int32 values (caller-owned, 6 * cap entries):
 *   kind    0 stencil kernel, 1 base solve, 3 zero fill, 7 coarse-tail
 *           launch, 8 rescale into an FP16 level; 100 + stage for a stage of
 *           the preceding coarse-tail launch (0 sweep, 1 residual,
 *           2 restriction, 3 prolongation, 4 base solve, 5 zero, 6 load,
 *           7 store)
 *   level   level index (0 = coarsest)
 *   kernel  for kind 0: 0 sweep, 1 IR update, 2 scale-and-cast,
 *           3 prolongation; else -1
 *   mode    sweep mode (0 Jacobi, 1 two sweeps from zero, 2 one sweep from
 *           zero, 3 residual-restriction, 4 one-pass pre-smoothing and
 *           restriction; + 16 for the Q1 operator); base-solve stages: 0
 *           exact, 1 CG
 *   prec, prec_c  storage types of the level and of the next coarser level
 * Records beyond cap are counted but not written.  The cluster tail's size
 * needs a device; the description shows the plan without that probe.
 * Returns MG_OK with the record count in *count, or MG_ERR_INVALID (invalid
 * parameters, count NULL, rec NULL with cap > 0). */
mg_status mg_describe_cycle(const mg_params* p, int32_t* rec, int32_t cap, int32_t* count);

/* ---------------------------------------------------------------- the five calls */

/* Creates a hierarchy: level geometry, per-level precision ladder, padded
 * device buffers, the dense FP64 inverse of the base-level operator and the
 * launch schedule of one IR step.  `cuda_stream` is a cudaStream_t (NULL =
 * the legacy default stream) on which every later call of this hierarchy
 * runs.  Host-side setup only: nothing here is part of a solve's time.
 * Errors: MG_ERR_INVALID (parameters), MG_ERR_OOM, MG_ERR_CUDA. */
mg_status mg_create_hierarchy(const mg_params* p, void* cuda_stream, mg_hierarchy** out);

/* Solves A u = b (Alg. 2).  b: n^d FP64 values, read only.  u: n^d FP64
 * values, in: initial guess (ignored when zero_guess = 1), out: solution.
 * Blocks until the solve has finished.  Returns the solve status (also in
 * res->status): MG_OK, MG_ERR_NOT_CONVERGED, MG_ERR_NUMERIC, MG_ERR_TIMEOUT
 * (a stencil kernel's bounded wait for its tile copies gave up; see
 * mg_params.wait_polls), MG_ERR_OOM (staging or, for a pooled hierarchy, its
 * arena could not be allocated) or a CUDA error.  A pooled hierarchy takes its
 * working arena from the pool for the solve, waiting up to 60 s while other
 * solves hold the budget (then MG_ERR_OOM), and hands it back at the end;
 * MG_ERR_ADMISSION if the arena exceeds the whole budget.
 * On a failed solve u holds the last iterate.  res may be NULL. */
mg_status mg_solve(mg_hierarchy* h, const double* b, double* u, mg_result* res);

/* Queues a solve of A u = b on hierarchy h and returns at once with a ticket
 * (the serving workload: requests of different sizes arriving over time).  A
 * background worker admits queued requests in arrival order when a slot is
 * free (mg_serve_configure), the hierarchy has no other request running and,
 * for a pooled hierarchy (mg_params.pooled = 1), its working arena fits the
 * device-memory pool's budget now: the arena is then taken from the pool, and
 * returned to it when the request completes.  Requests that do not fit wait;
 * a later request may pass a waiting one at most 8 times.  Admitted requests
 * run concurrently, each as one CUDA graph on its hierarchy's stream, with
 * the requests already running and with new arrivals.  A resident hierarchy
 * (pooled = 0) holds its arena outside the pool and is admitted by slots
 * alone.  b and u must stay valid until mg_poll reports completion.  Errors:
 * MG_ERR_INVALID, MG_ERR_ADMISSION (a pooled hierarchy's working arena
 * exceeds the whole budget, so it can never be admitted). */
mg_status mg_submit(mg_hierarchy* h, const double* b, double* u, uint64_t* ticket);

/* Completion test for a ticket of mg_submit: MG_BUSY while queued or running;
 * otherwise the solve's status, with the result in *res (may be NULL).  The
 * poll that reports completion retires the ticket: polling it again returns
 * MG_ERR_INVALID (unknown ticket), and the engine keeps no finished requests. */
mg_status mg_poll(mg_hierarchy* h, uint64_t ticket, mg_result* res);

/* Waits for outstanding requests of h, then frees all its device and host
 * state.  NULL is accepted. */
mg_status mg_destroy(mg_hierarchy* h);

/* ---------------------------------------------------------------- serving and batching */

/* Sets, for the current device, the budget of the device-memory pool that
 * holds the working arenas of pooled hierarchies (bytes; 0 = 80% of the free
 * device memory at the pool's next use), and the maximum number of serving
 * requests in flight (0 = 16).  The pool never holds more than the budget:
 * lowering it returns empty chunks to the device and evicts cached arenas of
 * idle hierarchies at once, the rest as running solves complete.  The peak
 * counters of mg_serve_stats_get restart from the current values. */
mg_status mg_serve_configure(size_t budget_bytes, int32_t max_inflight);

/* Counters of the current device's memory pool and of the serving engine. */
typedef struct mg_serve_stats {
    uint64_t budget_bytes;        /* the pool's budget */
    uint64_t reserved_bytes;      /* device memory the pool holds now (<= budget) */
    uint64_t in_use_bytes;        /* working arenas of solves running now */
    uint64_t peak_in_use_bytes;   /* maxima since the process started */
    uint64_t peak_reserved_bytes;
    uint64_t arena_acquires;      /* arenas taken from the pool */
    uint64_t arena_reuses;        /* ... that found their hierarchy's cached arena intact */
    uint64_t arena_evictions;     /* cached arenas given up to make room */
    uint64_t submitted, completed;/* serving requests */
    uint64_t memory_waits;        /* requests that waited at least once for the pool */
    uint64_t merged_groups;       /* merged groups run (mg_serve_options) */
    uint64_t merged_requests;     /* requests that ran inside one */
    int32_t inflight, peak_inflight, queued, reserved_;
} mg_serve_stats;
mg_status mg_serve_stats_get(mg_serve_stats* out);

/* merge_groups = 1: requests admitted in the same pass of the serving worker
 * whose hierarchies the level-synchronous launches cover (3D, V-cycle, coarse
 * tail, zero initial guess, device pointers) run together as one merged group,
 * as in mg_solve_batch: one CUDA graph whose every step operation is a single
 * launch over the (instance, tile) items of all members, each member keeping
 * its own scale, norms and stopping test (its result equals its solve alone
 * bit for bit).  A group completes when its last member converges.  The other
 * requests run as before, each as its own graph.  0 (default): no merging.
 * MG_ERR_INVALID for other values. */
mg_status mg_serve_options(int32_t merge_groups);

/* Solves `count` independent problems together, one per hierarchy (each
 * hierarchy at most once; none with serving requests in flight).  b[i], u[i],
 * res[i] as for mg_solve.  When every instance is 3D, uses V-cycles with a
 * coarse tail and a zero initial guess, and b and u are device pointers on
 * one device, the whole batch runs as one CUDA graph of level-synchronous
 * launches: each step operation (scale-cast, the pre-smoothing and
 * residual-restriction of the k-th level below each instance's finest, all
 * coarse tails, the prolongation and post-smoothing, the update, the norms)
 * is one launch over a work list of (instance, tile) items, instances of
 * different sizes included; res[i].merged = 1.  Otherwise the instances run
 * as concurrent solves on their own streams (res[i].merged = 0).  Each
 * instance keeps its own residual scale, norms and stopping test and stops
 * independently; its result equals its solve alone bit for bit.  Pooled
 * hierarchies (mg_params.pooled = 1) take their working arenas from the pool
 * for the batch and hand them back after it (MG_ERR_OOM when they do not fit
 * the budget at once).  Returns MG_OK if every instance converged, else the
 * first failing status. */
mg_status mg_solve_batch(int32_t count, mg_hierarchy* const* hs, const double* const* b,
                         double* const* u, mg_result* res);

/* ---------------------------------------------------------------- vector bandwidth study */

/* y <- a x + y for n values of type prec in caller-owned device arrays x, y
 * (16-byte aligned; n a multiple of 16 bytes of values), asynchronous on
 * `stream`: the AXPY of the bandwidth-versus-size study of Sec. 8.2 (Fig. 6),
 * with the widest vector accesses for every type (FP16/BF16 in half2 /
 * bfloat162 arithmetic).  MG_ERR_INVALID on bad arguments. */
mg_status mg_axpy(int32_t prec, int64_t n, double a, const void* x, void* y, void* stream);

/* ---------------------------------------------------------------- no device allocation */

/* The paper has no counterpart to this entry point; it exists for callers
 * that must not allocate device memory where they need a residual check: a
 * host application that has already reserved (nearly) all device memory for
 * its own pool, or a latency-critical loop where cudaMalloc/cudaFree would
 * synchronise the device and stall other streams.  mg_solve and the stage
 * calls allocate (hierarchy buffers, staging); this call does not.
 *
 * Computes, for the finite-difference operator A (op = 0: 5/7-point, h = 1/(n+1)):
 *   norms[0] = ||b - A u||_2,  norms[1] = ||b - A u||_inf,  norms[2] = ||b||_2
 * b, u: n^d FP64 values, contiguous, x fastest, device memory, read only.
 * norms: 3 doubles of device memory, written.  All three must be memory of
 * the current device (or managed memory), else MG_ERR_INVALID: host memory,
 * and another device's memory, which the kernels could not read without peer
 * access, are rejected before any launch.  Asynchronous: enqueued on cuda_stream
 * (NULL = legacy default stream); the norms are valid once the stream has
 * reached them.
 * Scratch: per-CTA partial sums in one static device array of 2 MiB that
 * every device loading this library keeps until exit; the largest accepted
 * problem is n^d = 536,870,912 points (MG_ERR_INVALID beyond, with a message).
 * All calls share that array: calls whose work overlaps on the GPU (e.g. on
 * different streams) race and must be serialised by the caller.  The first
 * call on a device looks up the array's device address with that device
 * current; make it before any stream capture begins.  The address is kept
 * per device and CUDA context: after cudaDeviceReset the next call on that
 * device looks it up again (also outside any capture). */
mg_status mg_residual_norms_noalloc(int32_t dim, int32_t n, const double* b, const double* u,
                                    double* norms, void* cuda_stream);

/* ---------------------------------------------------------------- host-side fault injection */

/* Allocation sites that mg_fault_inject can make fail. */
typedef enum {
    MG_FAULT_ARENA = 0,   /* the working arena: at mg_create_hierarchy, or for a pooled
                             hierarchy the pool's growth when a solve is admitted */
    MG_FAULT_STAGING = 1, /* the device staging buffers of host b / u at the first solve
                             with host pointers */
    MG_FAULT_SITES = 2
} mg_fault_site;

/* Failure detection without a device fault (the paper has no counterpart; it
 * tests the library's error paths): the next `count` allocations at `site`
 * fail as if the device were out of memory, without calling the allocator,
 * and take the library's own failure path (MG_ERR_OOM; nothing is leaked, the
 * caller's u is left unchanged, later calls are unaffected).  count = 0
 * cancels pending failures.  Process-wide; thread-safe.  Errors:
 * MG_ERR_INVALID for an unknown site or count < 0. */
mg_status mg_fault_inject(int32_t site, int32_t count);

/* ---------------------------------------------------------------- tile shapes (diagnostics) */

/* Fixes the launch shape of one 3D finite-difference stencil kernel for levels
 * of n points per dimension (FD operator, op = 0), process-wide, as the
 * autotuner (mg_params.tune) records its choices; later solves and stage calls
 * on such levels use it.  The results do not depend on the shape (the kernels
 * apply the same operations in the same order); this call lets tests and
 * measurements pin a shape.
 *   kernel         0 Jacobi sweep, 1 two sweeps from zero, 2 residual-restriction
 *   prec           mg_prec of the level
 *   rows_per_warp  -1: forget the shape (the wave model, or the autotuner at the
 *                  next tuned creation, decides again); 0: the direct kernel (one
 *                  thread per vector or coarse point); 1: the marching kernel with
 *                  one row per warp (two planes per step); 2: two rows per warp
 *                  (sweeps only, n >= 16)
 *   march_len      planes per CTA along z (sweeps) or coarse planes per CTA
 *                  (restriction), >= 1; ignored for rows_per_warp 0 and -1
 * Errors: MG_ERR_INVALID for an unknown kernel or precision, n outside
 * 3..1290 (the 3D grid limit of mg_params), or a shape outside those above.
 * Needs no device. */
mg_status mg_tile_set(int32_t kernel, int32_t prec, int32_t n, int32_t rows_per_warp, int32_t march_len);

/* ---------------------------------------------------------------- profiling */

/* Device time of one kernel of the IR step, summed over the steps of a solve. */
typedef struct mg_kernel_time {
    int32_t kind;        /* 0 stencil sweep, 1 base solve, 2 prolongation, 3 zero fill, 4 norm
                            finalise, 5 FP64 IR update, 6 scale and cast of the residual,
                            7 coarse tail (the cycle below `level` in one CTA),
                            8 rescale of a restricted residual into an FP16 level (max-norm
                            and scaled cast; two kernels) */
    int32_t level;       /* level index (0 = coarsest) */
    int32_t mode;        /* sweep mode: 0 Jacobi, 1 two sweeps from zero, 2 one sweep from zero,
                            3 residual + restriction */
    int32_t loader;      /* reserved (0) */
    int32_t prec;        /* mg_prec of the level */
    int32_t prec_coarse; /* mg_prec of the next coarser level */
    int32_t launches;    /* number of launches timed */
    int32_t threads;     /* threads per CTA */
    int32_t grid[3];     /* CTA grid */
    int32_t reserved;
    double total_ms;     /* summed device time (CUDA events around each launch) */
    double bytes;        /* algorithmic bytes per launch: each array touched once */
} mg_kernel_time;

/* Runs mg_solve with one launch per kernel (no CUDA graph) and CUDA events
 * around every kernel of every IR step; fills out[0..min(count, max_out)-1]
 * with one record per kernel of the step schedule (in launch order) and sets
 * *count to the schedule length.  Before each step the stream is held for a
 * few tens of microseconds (a bounded sleep, not timed) so that the host has
 * enqueued the whole step when the device starts it: every event pair then
 * times its kernel, not the host's launch gaps.  Same arguments and result as
 * mg_solve. */
mg_status mg_profile_solve(mg_hierarchy* h, const double* b, double* u, mg_result* res,
                           mg_kernel_time* out, int32_t max_out, int32_t* count);

/* ---------------------------------------------------------------- stages (tests, diagnostics) */

/* Level vectors addressable by mg_level_write / mg_level_read.  C, G, T are
 * stored in the level's precision; U, R are FP64 and exist on the finest
 * level only. */
typedef enum { MG_VEC_C = 0, MG_VEC_G = 1, MG_VEC_T = 2, MG_VEC_U = 3, MG_VEC_R = 4 } mg_vec;

/* Copies n_l^d interior values (contiguous, x fastest, element type = the
 * vector's storage type: double/float/half/bfloat16) into or out of a level
 * vector.  src/dst may be host or device pointers.  These and mg_run_stage
 * need a resident hierarchy (pooled = 0): a pooled one holds no level arrays
 * outside a solve (MG_ERR_INVALID). */
mg_status mg_level_write(mg_hierarchy* h, int32_t level, int32_t vec, const void* src);
mg_status mg_level_read(mg_hierarchy* h, int32_t level, int32_t vec, void* dst);
mg_status mg_level_info_get(const mg_hierarchy* h, int32_t level, mg_level_info* out);

/* One step of the method on one level, run on the hierarchy's stream:
 *   MG_STAGE_JACOBI        C <- C + omega D^-1 (G - A C)          (Sec. 4.2)
 *   MG_STAGE_JACOBI_ZERO2  C <- two damped Jacobi sweeps from C = 0 on G
 *   MG_STAGE_RESTRICT      G_{l-1} <- cast(R (G_l - A_l C_l))     (Alg. 1's residual restriction)
 *   MG_STAGE_PROLONG       C_l <- C_l + cast(s P C_{l-1})         (Alg. 1's prolongation and correction);
 *                          s = arg[0] when arg is not NULL (a rescaled coarse level), else 1
 *   MG_STAGE_JACOBI_PROLONG  C_l <- C_l + P C_{l-1}, then one Jacobi sweep
 *   MG_STAGE_COARSE        C_0 <- A_0^-1 G_0 (level 0 only; the base_solver in effect)
 *   MG_STAGE_SCALE_ZERO2   G_L <- cast(R * s) (Alg. 2's residual scaling), then JACOBI_ZERO2 on
 *                          level L; s = arg[0]
 *   MG_STAGE_IR_UPDATE     U <- U + a C_L;  R <- R - a A C_L;  a = arg[0]  (Alg. 2's solution and residual updates);
 *                          when the finest level is not FP64 and arg[1] > 0 (a power of two s), also
 *                          G_L <- cast(trunc_FP32(R s)) of the updated R (the next step's residual scaling,
 *                          as the solve's update forms it); arg holds 2 doubles
 *   MG_STAGE_RESIDUAL      R <- B - A U with B = arg pointer (n^d FP64, device)
 *   MG_STAGE_CYCLE         C_L <- one full cycle on G_L (Alg. 1, recursive)
 *   MG_STAGE_PRE_RESTRICT  C <- two damped Jacobi sweeps from C = 0 on G, then
 *                          G_{l-1} <- cast(R (G_l - A_l C_l)): one pass (3D)
 *   MG_STAGE_RESTRICT_RESCALE  G_{l-1} <- cast(R (G_l - A_l C_l) / s), level l-1 FP16,
 *                          s the power of two of the rescale16 rule; out[0] = s
 * out (may be NULL) receives, where the stage computes them, ||R||_2 and
 * ||R||_inf (IR_UPDATE, RESIDUAL) or the scale s (RESTRICT_RESCALE).  Synchronous. */
typedef enum {
    MG_STAGE_JACOBI = 0, MG_STAGE_JACOBI_ZERO2 = 1, MG_STAGE_RESTRICT = 2, MG_STAGE_PROLONG = 3,
    MG_STAGE_JACOBI_PROLONG = 4, MG_STAGE_COARSE = 5, MG_STAGE_SCALE_ZERO2 = 6,
    MG_STAGE_IR_UPDATE = 7, MG_STAGE_RESIDUAL = 8, MG_STAGE_CYCLE = 9, MG_STAGE_PRE_RESTRICT = 10,
    MG_STAGE_RESTRICT_RESCALE = 11
} mg_stage;
mg_status mg_run_stage(mg_hierarchy* h, int32_t stage, int32_t level, const double* arg,
                       const void* ptr_arg, double* out);

#ifdef __cplusplus
}
#endif
#endif /* MG_H */
