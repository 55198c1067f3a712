"""ctypes wrapper of the FP64 CPU oracle (``mg_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the test-suite, the package smoke check
and the benchmark's CPU-baseline leg, never by the library.  It shares no code
with the CUDA path.

Every function takes and returns numpy float64 arrays in the interior-only,
x-fastest layout: shape ``(n, n)`` in 2D or ``(n, n, n)`` in 3D, indexed
``[k, j, i]`` / ``[j, i]`` with ``i`` along x.  The routines follow the paper's
Sec. 4.1 (IR), Alg. 1 (two-grid/V-cycle), Alg. 2 (mixed-precision IR with
residuum scaling) and Sec. 5 (Poisson model problem); see the C source for the
per-routine citations.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mg_oracle.c")
_LIB = os.path.join(_HERE, "libmg_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, -O2, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99",
                               "-fno-fast-math", "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Params(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int), ("levels", ctypes.c_int),
                ("nu1", ctypes.c_int), ("nu2", ctypes.c_int), ("gamma", ctypes.c_int),
                ("omega", ctypes.c_double), ("scaling", ctypes.c_int),
                ("tol_mode", ctypes.c_int), ("tol", ctypes.c_double),
                ("max_iter", ctypes.c_int), ("true_residual_guard", ctypes.c_int),
                ("nthreads", ctypes.c_int), ("op", ctypes.c_int),
                ("emulate", ctypes.c_int), ("prec", ctypes.c_int * 24),
                ("sigma_log2", ctypes.c_int), ("rescale16", ctypes.c_int),
                ("base_solver", ctypes.c_int), ("base_tol", ctypes.c_double),
                ("base_maxit", ctypes.c_int), ("scale_ahead", ctypes.c_int)]


class Result(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("converged", ctypes.c_int), ("levels", ctypes.c_int),
                ("bnorm", ctypes.c_double), ("rel_res", ctypes.c_double),
                ("rel_res_true", ctypes.c_double), ("guard_restarts", ctypes.c_int)]


_D = ctypes.POINTER(ctypes.c_double)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i, d = ctypes.c_int, ctypes.c_double
            lib.or_apply_A_op.argtypes = [i, i, i, _D, _D, i]
            lib.or_residual_op.argtypes = [i, i, i, _D, _D, _D]
            lib.or_jacobi_op.argtypes = [i, i, i, d, _D, _D, _D]
            lib.or_restrict.argtypes = [i, i, _D, _D]
            lib.or_prolong_add.argtypes = [i, i, _D, _D]
            lib.or_coarse_solve_op.argtypes = [i, i, i, _D, _D]
            lib.or_coarse_solve_op.restype = i
            lib.or_level_sizes.argtypes = [i, i, ctypes.POINTER(ctypes.c_int)]
            lib.or_level_sizes.restype = i
            lib.or_mg_cycle.argtypes = [ctypes.POINTER(Params), _D, _D]
            lib.or_mg_cycle.restype = i
            lib.or_ir_solve.argtypes = [ctypes.POINTER(Params), _D, _D, ctypes.POINTER(Result), _D]
            lib.or_ir_solve.restype = i
            lib.or_cg_solve_fmt.argtypes = [i, i, i, i, _D, _D, d, i]
            lib.or_cg_solve_fmt.restype = i
            lib.or_round.argtypes = [i, d]
            lib.or_round.restype = d
            lib.or_round_array.argtypes = [i, ctypes.c_size_t, _D, _D]
            lib.or_trunc_f32.argtypes = [d]
            lib.or_trunc_f32.restype = d
            lib.or_scale_ahead_cast.argtypes = [i, ctypes.c_size_t, _D, d, _D]
            lib.or_scale_ahead_cast.restype = i
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _dn(a: np.ndarray):
    d = a.ndim
    n = a.shape[0]
    assert d in (2, 3) and all(s == n for s in a.shape), a.shape
    return d, n


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def apply_A(v, absmode: bool = False, op: int = 0) -> np.ndarray:
    """A v, or |A||v|: the 5/7-point finite-difference -Laplacian (op 0) or the
    Q1 finite-element operator divided by h^d (op 1) (Sec. 5)."""
    v = _f64(v)
    d, n = _dn(v)
    out = np.empty_like(v)
    _load().or_apply_A_op(int(op), d, n, _p(v), _p(out), 1 if absmode else 0)
    return out


def residual(b, u, op: int = 0) -> np.ndarray:
    """r = b - A u (Sec. 4.1, IR step 1)."""
    b, u = _f64(b), _f64(u)
    d, n = _dn(u)
    r = np.empty_like(u)
    _load().or_residual_op(int(op), d, n, _p(b), _p(u), _p(r))
    return r


def jacobi(g, v, omega: float, op: int = 0) -> np.ndarray:
    """One damped Jacobi step v + omega D^-1 (g - A v) (Sec. 4.2)."""
    g, v = _f64(g), _f64(v)
    d, n = _dn(v)
    out = np.empty_like(v)
    _load().or_jacobi_op(int(op), d, n, float(omega), _p(g), _p(v), _p(out))
    return out


def restrict(r) -> np.ndarray:
    """Full-weighting restriction to the next coarser grid (Alg. 1's residual restriction)."""
    r = _f64(r)
    d, nf = _dn(r)
    nc = (nf - 1) // 2
    out = np.empty((nc,) * d)
    _load().or_restrict(d, nf, _p(r), _p(out))
    return out


def prolong_add(cc, cf) -> np.ndarray:
    """cf + P cc with bi/trilinear interpolation P (Alg. 1's prolongation and correction); returns a new array."""
    cc = _f64(cc)
    out = _f64(cf).copy()
    d, nc = _dn(cc)
    assert out.shape[0] == 2 * nc + 1
    _load().or_prolong_add(d, nc, _p(cc), _p(out))
    return out


def coarse_solve(g, op: int = 0) -> np.ndarray:
    """Exact base-level solve A c = g by dense Cholesky (Sec. 4.2)."""
    g = _f64(g)
    d, n = _dn(g)
    c = np.empty_like(g)
    rc = _load().or_coarse_solve_op(int(op), d, n, _p(g), _p(c))
    if rc != 0:
        raise RuntimeError("oracle coarse solve failed")
    return c


def cg_solve(g, tol: float = 1e-4, maxit: int = 0, op: int = 0, fmt: int = 0):
    """Conjugate gradients for A c = g from c = 0 (Sec. 6 base solver): stops at
    ||r||_2 <= tol ||g||_2, after maxit steps (<= 0: the number of unknowns) or on
    breakdown; fmt rounds the stored vectors (emulation).  Returns (c, steps)."""
    g = _f64(g)
    d, n = _dn(g)
    c = np.zeros_like(g)
    it = _load().or_cg_solve_fmt(int(op), d, n, int(fmt), _p(g), _p(c), float(tol),
                                 int(maxit) if maxit > 0 else g.size)
    if it < 0:
        raise RuntimeError("oracle CG failed")
    return c, it


def level_sizes(n: int, levels: int = 0) -> list[int]:
    """Level sizes, coarsest first: n_{l-1} = (n_l - 1)/2 while n_l is odd and > 3."""
    buf = (ctypes.c_int * 24)()
    cnt = _load().or_level_sizes(int(n), int(levels), buf)
    return [buf[i] for i in range(cnt)]


# storage formats of the emulation (Sec. 3, Table 1)
FP64, FP32, FP16, BF16 = 0, 1, 2, 3


def round_to(fmt: int, x) -> np.ndarray:
    """x (FP64) rounded to nearest, ties to even, into FP32 / FP16 / BF16 (FP64: x)."""
    shape = np.shape(x)
    x = _f64(x).reshape(-1)
    y = np.empty_like(x)
    _load().or_round_array(int(fmt), x.size, _p(x), _p(y))
    return y.reshape(shape)


def trunc_f32(x) -> np.ndarray:
    """x truncated toward zero to FP32 precision (0 below 2^-126, infinity at and
    above 2^128): the truncation of the emulated scale-ahead cast (reading R21)."""
    shape = np.shape(x)
    x = _f64(x).reshape(-1)
    f = _load().or_trunc_f32
    return np.array([f(float(v)) for v in x]).reshape(shape)


def scale_ahead_cast(fmt: int, r, inv: float):
    """The emulated scale-ahead cast g = round_fmt(trunc_f32(r inv)) (reading R21
    of Alg. 2's residual scaling).  Returns (g, over): over is True when a truncated value
    reaches the format's overflow threshold (the step then falls back to the
    plain scale-and-cast)."""
    r = _f64(r)
    shape = r.shape
    r = r.reshape(-1)
    g = np.empty_like(r)
    over = _load().or_scale_ahead_cast(int(fmt), r.size, _p(r), float(inv), _p(g))
    return g.reshape(shape), bool(over)


def make_params(dim: int, n: int, *, levels: int = 0, nu1: int = 2, nu2: int = 2,
                gamma: int = 1, omega: float = 0.8, scaling: int = 1, tol_mode: int = 0,
                tol: float = 1e-10, max_iter: int = 100, guard: bool = True,
                nthreads: int = 1, op: int = 0, prec=None, sigma_log2: int = -1,
                rescale16: int = 1, base_solver: int = 0, base_tol: float = 1e-4,
                base_maxit: int = 0, scale_ahead: int = 0) -> Params:
    """prec: per-level storage formats, coarsest first (one entry per level), to
    run the low-precision emulation; None runs the plain FP64 oracle.
    base_solver 1: CG on the base level (Sec. 6) to base_tol, relative.
    scale_ahead 1 (emulation): the power-of-two scale from the previous residual."""
    P = Params(dim, n, levels, nu1, nu2, gamma, omega, scaling, tol_mode, tol,
               max_iter, 1 if guard else 0, nthreads, op)
    P.sigma_log2 = sigma_log2
    P.rescale16 = rescale16
    P.base_solver = base_solver
    P.base_tol = base_tol
    P.base_maxit = base_maxit
    P.scale_ahead = scale_ahead
    if prec is not None:
        nl = len(level_sizes(n, levels))
        if len(prec) != nl:
            raise ValueError(f"prec has {len(prec)} entries for {nl} levels")
        P.emulate = 1
        for l, f in enumerate(prec):
            P.prec[l] = int(f)
    return P


def mg_cycle(g, c0=None, **kw) -> np.ndarray:
    """One multigrid cycle (Alg. 1, recursive) for A c = g from initial guess c0 (default 0);
    with prec=[...] the low-precision emulation (g and c0 rounded to the finest format)."""
    g = _f64(g)
    d, n = _dn(g)
    c = np.zeros_like(g) if c0 is None else _f64(c0).copy()
    P = make_params(d, n, **kw)
    if _load().or_mg_cycle(ctypes.byref(P), _p(g), _p(c)) < 0:
        raise RuntimeError("oracle cycle failed")
    return c


def ir_solve(b, u0=None, **kw):
    """Alg. 2 in FP64 (with prec=[...] the low-precision emulation of the levels).
    Returns (u, info dict, residual history array)."""
    b = _f64(b)
    d, n = _dn(b)
    u = np.zeros_like(b) if u0 is None else _f64(u0).copy()
    P = make_params(d, n, **kw)
    hist = np.zeros(P.max_iter + 2)
    res = Result()
    status = _load().or_ir_solve(ctypes.byref(P), _p(b), _p(u), ctypes.byref(res), _p(hist))
    info = dict(status=status, iters=res.iters, converged=bool(res.converged), levels=res.levels,
                bnorm=res.bnorm, rel_res=res.rel_res, rel_res_true=res.rel_res_true,
                guard_restarts=res.guard_restarts)
    return u, info, hist[: res.iters + 1].copy()
