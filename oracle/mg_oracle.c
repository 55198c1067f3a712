/*
 * CPU oracle for the mixed-precision multigrid-preconditioned iterative
 * refinement of Oo & Vogel, "Accelerating Geometric Multigrid Preconditioning
 * with Half-Precision Arithmetic on GPUs" (arXiv 2007.07539).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain FP64 statement of
 * what the GPU library computes.  Only the test-suite, the package's smoke
 * check and the benchmark's CPU-baseline leg may load it.  It shares no code,
 * header, table or constant with the CUDA path, and imports nothing from it.
 *
 * Every routine is written directly from the paper's text, in FP64 (double),
 * with no blocking, fusion or reordering beyond what the cited definition says:
 *
 *   or_apply_A_op     Poisson's equation (Sec. 5, Eq. 1) on the unit
 *                     square/cube, zero Dirichlet boundary, h = 1/(n+1),
 *                     discretised either by the finite-difference 5-point (2D) /
 *                     7-point (3D) stencil (op 0) or by bilinear / trilinear Q1
 *                     finite elements (op 1, Sec. 5), the element matrix
 *                     assembled from the 1-D element integrals, divided by h^d
 *   or_residual       IR step 1, r = b - A u (Sec. 4.1)
 *   or_jacobi         damped Jacobi smoothing step (Sec. 4.2, smoother paragraph)
 *   or_restrict       restriction of a residual to the next coarser grid
 *                     (Alg. 1's residual restriction): full weighting
 *   or_prolong_add    transfer of the coarse correction to the fine grid and
 *                     update (Alg. 1's prolongation and correction): bi/trilinear interpolation
 *   or_coarse_solve   exact solve on the base level (Sec. 4.2: "an exact solve
 *                     is applied at the coarsest level")
 *   or_cycle          Alg. 1 applied recursively (V-cycle; gamma = 2 gives the
 *                     W-cycle)
 *   or_ir_solve       Alg. 2, mixed-precision IR with residuum scaling; here all
 *                     in FP64
 *   or_round          round-to-nearest-even into FP32, FP16 or BF16 (Sec. 3,
 *                     Table 1), written from the formats' definitions
 *   or_cg_solve_fmt   conjugate gradients on the base level (Sec. 6: the CG
 *                     base solver), optionally with its vectors stored in a
 *                     low-precision format
 *
 * Optional low-precision emulation (params.emulate = 1, a diagnostic: parity
 * of the GPU path is stated against the FP64 oracle): every vector a level
 * stores (the smoother's output, the restricted right-hand side, the base
 * solution, the corrected c after prolongation) is rounded once to that
 * level's format, while each operation itself is evaluated in FP64 (Sec. 6:
 * operations in the precision of the level, results cast on transfer).  The
 * IR loop then scales the residual to max-norm 2^sigma before the cast and
 * divides the correction by it again (Sec. 4.3), and a restriction from a
 * non-FP16 level into an FP16 level is rescaled by a power of two taken from
 * its max-norm and undone on prolongation (Sec. 6, DSH_MG).  With scale_ahead
 * the scale of Alg. 2's residual scaling is instead the power of two 2^sigma / 2^e with
 * 2^(e-1) <= ||r||_inf < 2^e of the previous step's residual (any scale is
 * exact in exact arithmetic), and the scaled residual is truncated to FP32
 * before the cast, as when the update itself forms the next right-hand side.
 *
 * Grid vectors are interior-only, contiguous, x fastest:
 *   index(i, j[, k]) = i + n*j [+ n*n*k], point ((i+1)h, (j+1)h[, (k+1)h]).
 * Levels: level 0 is the coarsest, level L the finest; n_{l-1} = (n_l - 1)/2;
 * fine 0-based index 2I+1 coincides with coarse 0-based index I.
 *
 * Parallelism: the stencil loops may run under OpenMP (each output point is
 * computed independently, so results do not depend on the thread count);
 * every reduction (norms, dot products) runs serially in index order.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAX_LEVELS 24

typedef struct {
    int dim;              /* 2 or 3 */
    int n;                /* interior points per dimension on the finest level */
    int levels;           /* 0 = as many as the coarsening rule allows */
    int nu1, nu2;         /* pre- and post-smoothing steps */
    int gamma;            /* 1 = V-cycle, 2 = W-cycle */
    double omega;         /* Jacobi damping */
    int scaling;          /* 0: alpha = 1; 1: alpha = ||r||_inf; 2: alpha = ||r||_2 */
    int tol_mode;         /* 0: ||r||_2 <= tol*||b||_2; 1: ||r||_2 < tol */
    double tol;
    int max_iter;
    int true_residual_guard; /* 1: confirm convergence with b - A u */
    int nthreads;         /* OpenMP threads for stencil loops (<= 0: 1) */
    int op;               /* 0: finite differences; 1: Q1 finite elements */
    /* low-precision emulation (diagnostic) */
    int emulate;          /* 1: round every stored level vector to prec[l] */
    int prec[OR_MAX_LEVELS]; /* storage format per level, coarsest first (OR_FP64 ...) */
    int sigma_log2;       /* scaled residual max-norm 2^sigma; -1: 14 if a level is FP16, else 0 */
    int rescale16;        /* 1: rescale restrictions from a non-FP16 into an FP16 level */
    /* base solver (Sec. 6) */
    int base_solver;      /* 0: exact (Cholesky); 1: conjugate gradients */
    double base_tol;      /* CG: stop at ||r||_2 <= base_tol ||g||_2 */
    int base_maxit;       /* CG: step limit (<= 0: the number of unknowns) */
    int scale_ahead;      /* emulation, max-norm scaling: the next g scaled by the power of two from the
                             previous residual's max-norm, through an FP32 truncation */
} or_params;

/* storage formats of the emulation (Sec. 3, Table 1) */
enum { OR_FP64 = 0, OR_FP32 = 1, OR_FP16 = 2, OR_BF16 = 3 };

typedef struct {
    int iters;            /* IR iterations performed */
    int converged;        /* 1 if the stopping test held for b - A u */
    int levels;           /* levels used */
    double bnorm;         /* ||b||_2 */
    double rel_res;       /* last recursive ||r||_2 / ||b||_2 */
    double rel_res_true;  /* ||b - A u||_2 / ||b||_2 at exit */
    int guard_restarts;   /* times the true residual replaced the recursive one */
} or_result;

static int g_threads = 1;

static size_t npts(int d, int n) { return d == 2 ? (size_t)n * n : (size_t)n * n * n; }

/*
 * x rounded to the nearest value of a binary floating-point format with p
 * significand bits (the leading bit included), least normal exponent emin and
 * largest finite value maxv, ties to the even significand (Sec. 3; IEEE 754
 * round-to-nearest-even).  In x's binade [2^e, 2^(e+1)) the format's values
 * are the multiples of 2^(e-p+1); below 2^emin (the subnormals) they are the
 * multiples of 2^(emin-p+1).  A rounded magnitude above maxv is an overflow:
 * infinity with x's sign.  x / q and the product by q are exact in FP64
 * (powers of two), and rint rounds to the nearest integer, ties to even, in
 * the default rounding mode.
 */
static double round_bin(double x, int p, int emin, double maxv) {
    if (x == 0.0 || !isfinite(x)) return x;
    int E;
    (void)frexp(x, &E); /* |x| = f 2^E with f in [1/2, 1): binade exponent E - 1 */
    const int e = E - 1 < emin ? emin : E - 1;
    const double q = ldexp(1.0, e - p + 1);
    const double y = rint(x / q) * q;
    return fabs(y) > maxv ? copysign(INFINITY, x) : y;
}

/*
 * x stored in format fmt (Table 1): binary32 (24 significand bits, least
 * normal exponent -126, max (2 - 2^-23) 2^127), binary16 (11, -14, 65504),
 * bfloat16 (8, -126, (2 - 2^-7) 2^127); OR_FP64 returns x.
 */
double or_round(int fmt, double x) {
    switch (fmt) {
    case OR_FP32: return round_bin(x, 24, -126, ldexp(2.0 - ldexp(1.0, -23), 127));
    case OR_FP16: return round_bin(x, 11, -14, 65504.0);
    case OR_BF16: return round_bin(x, 8, -126, ldexp(2.0 - ldexp(1.0, -7), 127));
    default: return x;
    }
}
void or_round_array(int fmt, size_t N, const double *x, double *y) {
    for (size_t p = 0; p < N; ++p) y[p] = or_round(fmt, x[p]);
}
static void round_vec(int fmt, size_t N, double *v) {
    if (fmt != OR_FP64) or_round_array(fmt, N, v, v);
}

/* Value of v at (i, j, k); zero outside the interior (Dirichlet boundary). */
static double at(const double *v, int d, int n, int i, int j, int k) {
    if (i < 0 || i >= n || j < 0 || j >= n) return 0.0;
    if (d == 2) return v[(size_t)j * n + i];
    if (k < 0 || k >= n) return 0.0;
    return v[((size_t)k * n + j) * n + i];
}

/*
 * (A v)_p = h^-2 * (2d v_p - sum of the 2d axis neighbours of p), the standard
 * second-order finite-difference approximation of -Laplace(v) (Sec. 5, Eq. 1).
 * With absmode != 0 the neighbour coefficients are taken as +1: this gives
 * |A| |v|, the magnitude used to scale rounding tolerances.
 */
static void apply_fd(int d, int n, const double *v, double *out, int absmode) {
    const double h = 1.0 / (n + 1);
    const double ih2 = 1.0 / (h * h);
    const double sgn = absmode ? 1.0 : -1.0;
    const int nk = d == 3 ? n : 1;
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int k = 0; k < nk; ++k)
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                double nb = at(v, d, n, i - 1, j, k) + at(v, d, n, i + 1, j, k)
                          + at(v, d, n, i, j - 1, k) + at(v, d, n, i, j + 1, k);
                if (d == 3) nb += at(v, d, n, i, j, k - 1) + at(v, d, n, i, j, k + 1);
                double c = at(v, d, n, i, j, k);
                if (absmode) c = fabs(c), nb = 0.0
                    + fabs(at(v, d, n, i - 1, j, k)) + fabs(at(v, d, n, i + 1, j, k))
                    + fabs(at(v, d, n, i, j - 1, k)) + fabs(at(v, d, n, i, j + 1, k))
                    + (d == 3 ? fabs(at(v, d, n, i, j, k - 1)) + fabs(at(v, d, n, i, j, k + 1)) : 0.0);
                size_t p = d == 2 ? (size_t)j * n + i : ((size_t)k * n + j) * n + i;
                out[p] = ih2 * (2.0 * d * c + sgn * nb);
            }
}

/*
 * Q1 finite elements (Sec. 5: bilinear quadrilaterals in 2D, trilinear
 * hexahedra in 3D) on the uniform grid.  The basis function of node p is the
 * product of 1-D hat functions, so the Galerkin entry between nodes p and
 * p + o (o in {-1, 0, 1}^d) is
 *     int grad phi_p . grad phi_{p+o} = sum_a K1(o_a) prod_{b != a} M1(o_b)
 * with K1, M1 the 1-D stiffness and mass integrals of two hats at offset o,
 * assembled from the element matrices of a linear element of length h.
 */
static double q1_stiff1(int o, double h) {
    const double ke[2][2] = {{1.0 / h, -1.0 / h}, {-1.0 / h, 1.0 / h}};  /* int phi_a' phi_b' over one element */
    return o == 0 ? ke[0][0] + ke[1][1] : ke[0][1];  /* a node's hat spans two elements */
}
static double q1_mass1(int o, double h) {
    const double me[2][2] = {{h / 3.0, h / 6.0}, {h / 6.0, h / 3.0}};      /* int phi_a phi_b over one element */
    return o == 0 ? me[0][0] + me[1][1] : me[0][1];
}
static double q1_entry(int d, double h, const int *o) {
    double s = 0.0;
    for (int a = 0; a < d; ++a) {
        double t = q1_stiff1(o[a], h);
        for (int b = 0; b < d; ++b)
            if (b != a) t *= q1_mass1(o[b], h);
        s += t;
    }
    return s;
}

/*
 * (A v)_p = h^-d sum_o q1_entry(o) v_{p+o}: the Q1 stiffness matrix divided
 * by the element measure h^d, so that, like the finite-difference operator, it
 * approximates -Laplace pointwise and its coarse-grid counterpart at 2h equals
 * the Galerkin product of full weighting, A and interpolation.  absmode: the
 * absolute values of the entries (|A| |v|).
 */
static void apply_q1(int d, int n, const double *v, double *out, int absmode) {
    const double h = 1.0 / (n + 1);
    const double scale = 1.0 / pow(h, d);
    const int nk = d == 3 ? n : 1;
    const int ok0 = d == 3 ? -1 : 0, ok1 = d == 3 ? 1 : 0;
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int k = 0; k < nk; ++k)
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                double s = 0.0;
                for (int ok = ok0; ok <= ok1; ++ok)
                    for (int oj = -1; oj <= 1; ++oj)
                        for (int oi = -1; oi <= 1; ++oi) {
                            const int o[3] = {oi, oj, ok};
                            double w = q1_entry(d, h, o);
                            double x = at(v, d, n, i + oi, j + oj, k + ok);
                            s += absmode ? fabs(w) * fabs(x) : w * x;
                        }
                size_t p = d == 2 ? (size_t)j * n + i : ((size_t)k * n + j) * n + i;
                out[p] = scale * s;
            }
}

/* Diagonal entry of A (the Jacobi D): 2d/h^2 (op 0) or h^-d q1_entry(0). */
static double diag_A(int op, int d, int n) {
    const double h = 1.0 / (n + 1);
    if (op == 0) return 2.0 * d / (h * h);
    const int o[3] = {0, 0, 0};
    return q1_entry(d, h, o) / pow(h, d);
}

void or_apply_A_op(int op, int d, int n, const double *v, double *out, int absmode) {
    if (op == 1) apply_q1(d, n, v, out, absmode);
    else apply_fd(d, n, v, out, absmode);
}
void or_apply_A_mode(int d, int n, const double *v, double *out, int absmode) { or_apply_A_op(0, d, n, v, out, absmode); }
void or_apply_A(int d, int n, const double *v, double *out) { or_apply_A_op(0, d, n, v, out, 0); }

/* IR step 1 (Sec. 4.1): r = b - A u. */
void or_residual_op(int op, int d, int n, const double *b, const double *u, double *r) {
    size_t N = npts(d, n);
    double *au = (double *)malloc(N * sizeof(double));
    or_apply_A_op(op, d, n, u, au, 0);
    for (size_t p = 0; p < N; ++p) r[p] = b[p] - au[p];
    free(au);
}
void or_residual(int d, int n, const double *b, const double *u, double *r) { or_residual_op(0, d, n, b, u, r); }

/*
 * One damped Jacobi step (Sec. 4.2): out = v + omega D^-1 (g - A v), with
 * D = diag(A).  The update is simultaneous: out must not alias v.
 */
void or_jacobi_op(int op, int d, int n, double omega, const double *g, const double *v, double *out) {
    const double dinv = 1.0 / diag_A(op, d, n);
    size_t N = npts(d, n);
    double *av = (double *)malloc(N * sizeof(double));
    or_apply_A_op(op, d, n, v, av, 0);
    for (size_t p = 0; p < N; ++p) out[p] = v[p] + omega * dinv * (g[p] - av[p]);
    free(av);
}
void or_jacobi(int d, int n, double omega, const double *g, const double *v, double *out) {
    or_jacobi_op(0, d, n, omega, g, v, out);
}

/* 1-D full-weighting weight of fine offset o in {-1, 0, 1}: [1/4, 1/2, 1/4]. */
static double fw(int o) { return o == 0 ? 0.5 : 0.25; }

/*
 * Restriction (Alg. 1's residual restriction): full weighting, the tensor product of the 1-D
 * stencil [1/4, 1/2, 1/4] centred on the fine point 2I+1 that coincides with
 * coarse point I.  nf = 2 nc + 1.
 */
void or_restrict(int d, int nf, const double *rf, double *gc) {
    const int nc = (nf - 1) / 2;
    const int nk = d == 3 ? nc : 1;
    const int ok0 = d == 3 ? -1 : 0, ok1 = d == 3 ? 1 : 0;
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int K = 0; K < nk; ++K)
        for (int J = 0; J < nc; ++J)
            for (int I = 0; I < nc; ++I) {
                double s = 0.0;
                for (int ok = ok0; ok <= ok1; ++ok)
                    for (int oj = -1; oj <= 1; ++oj)
                        for (int oi = -1; oi <= 1; ++oi) {
                            double w = fw(oi) * fw(oj) * (d == 3 ? fw(ok) : 1.0);
                            s += w * at(rf, d, nf, 2 * I + 1 + oi, 2 * J + 1 + oj, 2 * K + 1 + ok);
                        }
                size_t p = d == 2 ? (size_t)J * nc + I : ((size_t)K * nc + J) * nc + I;
                gc[p] = s;
            }
}

/*
 * 1-D linear interpolation from coarse to fine at fine 0-based index i:
 * an odd index 2I+1 takes coarse I; an even index 2I lies between coarse I-1
 * and I and takes their mean (coarse values outside the grid are zero).
 * Returns the number of contributing coarse indices (1 or 2) in *cnt and
 * fills idx/wt.
 */
static void lin1d(int i, int *cnt, int idx[2], double wt[2]) {
    if (i % 2 == 1) { *cnt = 1; idx[0] = (i - 1) / 2; wt[0] = 1.0; }
    else { *cnt = 2; idx[0] = i / 2 - 1; idx[1] = i / 2; wt[0] = wt[1] = 0.5; }
}

/*
 * Prolongation and correction (Alg. 1's prolongation and correction): cf += P cc, with P the
 * tensor-product (bi/trilinear) interpolation.  nf = 2 nc + 1.
 */
void or_prolong_add(int d, int nc, const double *cc, double *cf) {
    const int nf = 2 * nc + 1;
    const int nk = d == 3 ? nf : 1;
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int k = 0; k < nk; ++k)
        for (int j = 0; j < nf; ++j)
            for (int i = 0; i < nf; ++i) {
                int ci, cj, ck = 1, ii[2], jj[2], kk[2] = {0, 0};
                double wi[2], wj[2], wk[2] = {1.0, 1.0};
                lin1d(i, &ci, ii, wi);
                lin1d(j, &cj, jj, wj);
                if (d == 3) lin1d(k, &ck, kk, wk);
                double s = 0.0;
                for (int c = 0; c < ck; ++c)
                    for (int b = 0; b < cj; ++b)
                        for (int a = 0; a < ci; ++a)
                            s += wi[a] * wj[b] * wk[c] * at(cc, d, nc, ii[a], jj[b], kk[c]);
                size_t p = d == 2 ? (size_t)j * nf + i : ((size_t)k * nf + j) * nf + i;
                cf[p] += s;
            }
}

/*
 * Exact base-level solve (Sec. 4.2): assemble the dense matrix of A on the
 * n^d grid column by column (A applied to unit vectors), factor it by
 * Cholesky (A is symmetric positive definite) and solve.  Returns 0 on
 * success, -1 if the factorisation breaks down or n^d is too large.
 */
int or_coarse_solve_op(int op, int d, int n, const double *g, double *c) {
    size_t m = npts(d, n);
    if (m > 4096) return -1;
    double *A = (double *)calloc(m * m, sizeof(double));
    double *e = (double *)calloc(m, sizeof(double));
    double *col = (double *)malloc(m * sizeof(double));
    double *y = (double *)malloc(m * sizeof(double));
    int saved = g_threads;
    g_threads = 1;
    for (size_t q = 0; q < m; ++q) {
        e[q] = 1.0;
        or_apply_A_op(op, d, n, e, col, 0);
        for (size_t p = 0; p < m; ++p) A[p * m + q] = col[p];
        e[q] = 0.0;
    }
    g_threads = saved;
    int rc = 0;
    /* Cholesky A = L L^T, L stored in the lower triangle of A. */
    for (size_t j = 0; j < m && rc == 0; ++j) {
        double s = A[j * m + j];
        for (size_t k = 0; k < j; ++k) s -= A[j * m + k] * A[j * m + k];
        if (!(s > 0.0)) { rc = -1; break; }
        double ljj = sqrt(s);
        A[j * m + j] = ljj;
        for (size_t i = j + 1; i < m; ++i) {
            double t = A[i * m + j];
            for (size_t k = 0; k < j; ++k) t -= A[i * m + k] * A[j * m + k];
            A[i * m + j] = t / ljj;
        }
    }
    if (rc == 0) {
        for (size_t i = 0; i < m; ++i) {           /* L y = g */
            double t = g[i];
            for (size_t k = 0; k < i; ++k) t -= A[i * m + k] * y[k];
            y[i] = t / A[i * m + i];
        }
        for (size_t ii = m; ii-- > 0;) {           /* L^T c = y */
            double t = y[ii];
            for (size_t k = ii + 1; k < m; ++k) t -= A[k * m + ii] * c[k];
            c[ii] = t / A[ii * m + ii];
        }
    }
    free(A); free(e); free(col); free(y);
    return rc;
}
int or_coarse_solve(int d, int n, const double *g, double *c) { return or_coarse_solve_op(0, d, n, g, c); }

/*
 * Conjugate gradients for A c = g on an n^d grid (Sec. 6: the base solver),
 * from c = 0, in the textbook order of Hestenes and Stiefel:
 *   r = g, p = r
 *   repeat:  q = A p;  a = r.r / p.q;  c += a p;  r -= a q;
 *            b = r_new.r_new / r.r;  p = r + b p
 * Stops when ||r||_2 <= tol ||g||_2 for the recursively updated r, after
 * maxit steps, or when p.q is not positive (breakdown; g = 0 included).
 * With fmt != OR_FP64 the stored vectors c, r, p are rounded to fmt after
 * each update (the CG of a low-precision base level); A p and the dot
 * products stay in FP64.  Returns the steps taken, or -1 on allocation
 * failure.
 */
int or_cg_solve_fmt(int op, int d, int n, int fmt, const double *g, double *c, double tol, int maxit) {
    size_t N = npts(d, n);
    double *r = (double *)malloc(N * sizeof(double));
    double *p = (double *)malloc(N * sizeof(double));
    double *q = (double *)malloc(N * sizeof(double));
    if (!r || !p || !q) { free(r); free(p); free(q); return -1; }
    double rr = 0.0;
    for (size_t i = 0; i < N; ++i) {
        c[i] = 0.0;
        r[i] = or_round(fmt, g[i]);
        p[i] = r[i];
        rr += r[i] * r[i];
    }
    const double thr = tol * tol * rr;
    int it = 0;
    while (it < maxit && rr > thr) {
        or_apply_A_op(op, d, n, p, q, 0);
        double pq = 0.0;
        for (size_t i = 0; i < N; ++i) pq += p[i] * q[i];
        if (!(pq > 0.0)) break;
        const double a = rr / pq;
        double rn = 0.0;
        for (size_t i = 0; i < N; ++i) {
            c[i] = or_round(fmt, c[i] + a * p[i]);
            r[i] = or_round(fmt, r[i] - a * q[i]);
            rn += r[i] * r[i];
        }
        const double b = rn / rr;
        for (size_t i = 0; i < N; ++i) p[i] = or_round(fmt, r[i] + b * p[i]);
        rr = rn;
        ++it;
    }
    free(r); free(p); free(q);
    return it;
}

/* Coarsening rule: n_{l-1} = (n_l - 1)/2 while n_l is odd and > 3.
 * Fills sizes[0..L] with sizes[L] = n (finest) and returns the level count. */
int or_level_sizes(int n, int levels_req, int *sizes) {
    int tmp[OR_MAX_LEVELS], cnt = 0, m = n;
    tmp[cnt++] = m;
    while (m % 2 == 1 && m > 3 && cnt < OR_MAX_LEVELS && (levels_req <= 0 || cnt < levels_req)) {
        m = (m - 1) / 2;
        tmp[cnt++] = m;
    }
    for (int l = 0; l < cnt; ++l) sizes[l] = tmp[cnt - 1 - l];
    return cnt;
}

typedef struct {
    int d, L;
    int n[OR_MAX_LEVELS];
    double *c[OR_MAX_LEVELS], *g[OR_MAX_LEVELS], *t[OR_MAX_LEVELS];
    int sigma;              /* emulation: log2 of the residual's target max-norm */
} or_hier;

/* format of level l's vectors: FP64 unless emulating */
static int lfmt(const or_params *P, int l) { return P->emulate ? P->prec[l] : OR_FP64; }

/*
 * Power-of-two rescale of a restricted residual into an FP16 level (Sec. 6):
 * k with m 2^k in [2^(sigma-1), 2^sigma) for its max-norm m, |k| <= 126;
 * k = 0 for m = 0.
 */
static int rescale_k(size_t N, const double *v, int sigma) {
    double m = 0.0;
    for (size_t p = 0; p < N; ++p) { double a = fabs(v[p]); if (a > m) m = a; }
    if (!(m > 0.0) || !isfinite(m)) return 0;
    int e;
    (void)frexp(m, &e); /* m = f 2^e, f in [1/2, 1) */
    int k = sigma - e;
    return k > 126 ? 126 : (k < -126 ? -126 : k);
}

/*
 * Alg. 1 applied recursively on level l, with c the initial guess on entry
 * (zero at the first visit) and the approximate solution of A_l c = g on exit.
 *   step 1: nu1 damped Jacobi sweeps
 *   step 2: residual g - A_l c, restricted to level l-1
 *   step 3: coarse correction by gamma visits of the same cycle on level l-1
 *           (gamma = 1: V-cycle); the base level is solved exactly
 *   step 4: prolongation of the coarse correction and update of c
 *   step 5: nu2 damped Jacobi sweeps
 */
static int cycle(or_hier *H, const or_params *P, int l) {
    int d = H->d, n = H->n[l];
    size_t N = npts(d, n);
    double *c = H->c[l], *g = H->g[l], *t = H->t[l];
    const int op = P->op;
    const int f = lfmt(P, l);
    if (l == 0) {
        if (P->base_solver == 1) {
            const int maxit = P->base_maxit > 0 ? P->base_maxit : (int)N;
            return or_cg_solve_fmt(op, d, n, f, g, c, P->base_tol, maxit) < 0 ? -1 : 0;
        }
        int rc = or_coarse_solve_op(op, d, n, g, c);
        round_vec(f, N, c);
        return rc;
    }
    for (int s = 0; s < P->nu1; ++s) {
        or_jacobi_op(op, d, n, P->omega, g, c, t);
        memcpy(c, t, N * sizeof(double));
        round_vec(f, N, c);
    }
    or_residual_op(op, d, n, g, c, t);
    const int nc = H->n[l - 1], fc = lfmt(P, l - 1);
    const size_t Nc = npts(d, nc);
    or_restrict(d, n, t, H->g[l - 1]);
    int k = 0; /* the coarse level's rescale 2^k (emulation, Sec. 6) */
    if (P->emulate && P->rescale16 && fc == OR_FP16 && f != OR_FP16) {
        k = rescale_k(Nc, H->g[l - 1], H->sigma);
        for (size_t p = 0; p < Nc; ++p) H->g[l - 1][p] = ldexp(H->g[l - 1][p], k);
    }
    round_vec(fc, Nc, H->g[l - 1]);
    memset(H->c[l - 1], 0, Nc * sizeof(double));
    for (int v = 0; v < P->gamma; ++v) { int rc = cycle(H, P, l - 1); if (rc) return rc; }
    if (k != 0) {
        /* the correction of the rescaled level, scaled back by 2^-k (exact) */
        double *cs = H->t[l - 1];
        for (size_t p = 0; p < Nc; ++p) cs[p] = ldexp(H->c[l - 1][p], -k);
        or_prolong_add(d, nc, cs, c);
    } else {
        or_prolong_add(d, nc, H->c[l - 1], c);
    }
    round_vec(f, N, c);
    for (int s = 0; s < P->nu2; ++s) {
        or_jacobi_op(op, d, n, P->omega, g, c, t);
        memcpy(c, t, N * sizeof(double));
        round_vec(f, N, c);
    }
    return 0;
}

static int hier_alloc(or_hier *H, const or_params *P) {
    memset(H, 0, sizeof(*H));
    H->d = P->dim;
    int cnt = or_level_sizes(P->n, P->levels, H->n);
    H->L = cnt - 1;
    int any16 = 0;
    for (int l = 0; l < cnt; ++l) any16 |= lfmt(P, l) == OR_FP16;
    H->sigma = P->sigma_log2 >= 0 ? P->sigma_log2 : (any16 ? 14 : 0);
    for (int l = 0; l < cnt; ++l) {
        size_t N = npts(H->d, H->n[l]);
        H->c[l] = (double *)calloc(N, sizeof(double));
        H->g[l] = (double *)calloc(N, sizeof(double));
        H->t[l] = (double *)calloc(N, sizeof(double));
        if (!H->c[l] || !H->g[l] || !H->t[l]) return -1;
    }
    return 0;
}

static void hier_free(or_hier *H) {
    for (int l = 0; l <= H->L; ++l) { free(H->c[l]); free(H->g[l]); free(H->t[l]); }
}

/*
 * One multigrid cycle as a preconditioner: c = MG(g) with zero initial guess
 * on the finest level.  Exposed for the contraction-factor pin and for
 * per-cycle parity checks.  Returns the level count, or -1 on failure.
 */
int or_mg_cycle(const or_params *P, const double *g, double *c) {
    or_hier H;
    g_threads = P->nthreads > 0 ? P->nthreads : 1;
    if (hier_alloc(&H, P)) { hier_free(&H); return -1; }
    size_t N = npts(P->dim, P->n);
    memcpy(H.g[H.L], g, N * sizeof(double));
    memcpy(H.c[H.L], c, N * sizeof(double));
    round_vec(lfmt(P, H.L), N, H.g[H.L]); /* the finest level stores g and c in its format */
    round_vec(lfmt(P, H.L), N, H.c[H.L]);
    int rc = cycle(&H, P, H.L);
    memcpy(c, H.c[H.L], N * sizeof(double));
    int L = H.L;
    hier_free(&H);
    return rc ? -1 : L + 1;
}

double or_norm2(size_t N, const double *v) {
    double s = 0.0;
    for (size_t p = 0; p < N; ++p) s += v[p] * v[p];
    return sqrt(s);
}

double or_norminf(size_t N, const double *v) {
    double m = 0.0;
    for (size_t p = 0; p < N; ++p) { double a = fabs(v[p]); if (a > m) m = a; }
    return m;
}

/*
 * Alg. 2: iterative refinement with residuum scaling and one multigrid cycle
 * per step, all in FP64.
 *   r = b - A u
 *   while the stopping test fails:
 *     alpha = ||r|| (inf-norm, 2-norm, or 1 without scaling)
 *     g = (1/alpha) r                       (Alg. 2's residual scaling)
 *     c = one multigrid cycle for A c = g   (Alg. 2's correction by Alg. 1)
 *     u = u + alpha c                       (Alg. 2's solution update)
 *     r = r - alpha A c                     (Alg. 2's residual update)
 * When the recursive residual passes the test, b - A u is recomputed; if it
 * fails the test the loop continues from that true residual.
 * history (optional, max_iter+1 entries) receives ||r||_2/||b||_2 before each
 * step and after the last.  Returns 0 on convergence, 1 if max_iter was hit,
 * -1 on failure (allocation, base solve, non-finite residual).
 */
/* x truncated toward zero to binary32 precision (0 below its normal range,
   infinity at and above 2^128): the low 29 of FP64's 52 fraction bits cleared */
double or_trunc_f32(double x) {
    if (!isfinite(x)) return x;
    const double a = fabs(x);
    if (a < ldexp(1.0, -126)) return copysign(0.0, x);
    if (a >= ldexp(1.0, 128)) return copysign(INFINITY, x);
    int E;
    const double f = frexp(a, &E);                 /* a = f 2^E, f in [1/2, 1) */
    const double m = floor(ldexp(f, 24));          /* the 24 leading significand bits */
    return copysign(ldexp(m, E - 24), x);
}

/* Scale-ahead cast of the emulation (reading R21 of Alg. 2's residual scaling): g =
   cast_fmt(trunc_f32(r inv)).  Returns 1 when some truncated value lies at or
   beyond the format's overflow threshold (it would round to infinity: 65520
   for FP16, the midpoint above FP16's largest finite value; 3.0e38 as a bound
   below BF16's / FP32's, above any value reached), else 0.  g is written either way. */
int or_scale_ahead_cast(int fmt, size_t N, const double *r, double inv, double *g) {
    const double lim = fmt == OR_FP16 ? 65520.0 : 3.0e38;
    int over = 0;
    for (size_t p = 0; p < N; ++p) {
        const double t = or_trunc_f32(r[p] * inv);
        over |= !(fabs(t) < lim);
        g[p] = or_round(fmt, t);
    }
    return over;
}

int or_ir_solve(const or_params *P, const double *b, double *u, or_result *res, double *history) {
    or_hier H;
    g_threads = P->nthreads > 0 ? P->nthreads : 1;
    memset(res, 0, sizeof(*res));
    if (hier_alloc(&H, P)) { hier_free(&H); return -1; }
    res->levels = H.L + 1;
    const int d = P->dim, n = P->n;
    size_t N = npts(d, n);
    double *r = (double *)malloc(N * sizeof(double));
    double *ac = (double *)malloc(N * sizeof(double));
    int status = 1;
    const int op = P->op;
    or_residual_op(op, d, n, b, u, r);
    double bnorm = or_norm2(N, b);
    res->bnorm = bnorm;
    double scale = P->tol_mode == 0 ? bnorm : 1.0;
    int it = 0;
    const int fL = lfmt(P, H.L);
    const int ahead_on = P->emulate && P->scale_ahead && P->scaling == 1 && fL != OR_FP64;
    double inv_pred = 0.0; /* scale-ahead: 2^sigma / 2^e from the previous residual's max-norm */
    int ahead = 0;         /* the current r is the result of a refinement step */
    for (;;) {
        double rn = or_norm2(N, r);
        if (!isfinite(rn)) { status = -1; break; }
        if (history) history[it] = bnorm > 0 ? rn / bnorm : rn;
        res->rel_res = bnorm > 0 ? rn / bnorm : rn;
        if (rn <= P->tol * scale) {
            if (!P->true_residual_guard) { status = 0; break; }
            or_residual_op(op, d, n, b, u, ac);
            double tn = or_norm2(N, ac);
            if (tn <= P->tol * scale) { status = 0; break; }
            memcpy(r, ac, N * sizeof(double));
            ahead = 0;
            res->guard_restarts++;
            rn = tn;
            res->rel_res = bnorm > 0 ? rn / bnorm : rn;
            if (history) history[it] = res->rel_res;
        }
        if (it >= P->max_iter) { status = 1; break; }
        double alpha = 1.0;
        if (P->scaling == 1) alpha = or_norminf(N, r);
        else if (P->scaling == 2) alpha = rn;
        if (!(alpha > 0.0)) { status = -1; break; }
        double inv = 1.0 / alpha;
        double *g = H.g[H.L], *c = H.c[H.L];
        if (P->emulate && P->scaling != 0) {
            /* g = cast(r 2^sigma / alpha), c = MG(g), and the correction
               taken with alpha 2^-sigma (both powers of two exact) */
            inv = ldexp(inv, H.sigma);
            alpha = ldexp(alpha, -H.sigma);
        }
        int done = 0;
        if (ahead_on && ahead && inv_pred > 0.0) {
            /* scale-ahead: g = cast(trunc_f32(r inv_pred)) unless a value is
               beyond the format's range, then the scale above */
            if (!or_scale_ahead_cast(fL, N, r, inv_pred, g)) { inv = inv_pred; alpha = 1.0 / inv_pred; done = 1; }
        }
        if (ahead_on) {
            int e;
            (void)frexp(or_norminf(N, r), &e); /* 2^(e-1) <= ||r||_inf < 2^e */
            inv_pred = ldexp(1.0, H.sigma - e);
            ahead = 1;
        }
        if (!done) {
            for (size_t p = 0; p < N; ++p) g[p] = inv * r[p];
            round_vec(fL, N, g);
        }
        memset(c, 0, N * sizeof(double));
        if (cycle(&H, P, H.L)) { status = -1; break; }
        for (size_t p = 0; p < N; ++p) u[p] = u[p] + alpha * c[p];
        or_apply_A_op(op, d, n, c, ac, 0);
        for (size_t p = 0; p < N; ++p) r[p] = r[p] - alpha * ac[p];
        ++it;
    }
    res->iters = it;
    res->converged = status == 0;
    or_residual_op(op, d, n, b, u, ac);
    res->rel_res_true = bnorm > 0 ? or_norm2(N, ac) / bnorm : or_norm2(N, ac);
    free(r); free(ac);
    hier_free(&H);
    return status;
}
