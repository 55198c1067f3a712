"""The Q1 finite-element operator of Sec. 5 (op = 1: bilinear 9-point in 2D,
trilinear 27-point in 3D, the stiffness matrix divided by h^d) through every
kernel of the path, against the FP64 oracle with op = 1.

Kernel level: Jacobi sweep, the two sweeps from zero, residual + restriction,
the FP64 IR update and residual, the base solves; bounds as for the
finite-difference kernels (|gpu - oracle| <= tol * M, M the scaled
magnitude).  Solve level: FP64 iteration counts equal to the oracle's, low
precision within two more, FP64 accuracy, the closed-form discrete solution of
the manufactured problem, the paper's k = 20 problem from a random initial
guess in [0, 1), and merged batches equal to alone solves bit for bit."""
import math

import numpy as np
import pytest

from _helpers import TOL, as_f64, check_close, empty_storage, to_storage
from paper_2007_07539_gb300 import inputs as I
from paper_2007_07539_gb300 import mg

pytestmark = pytest.mark.gpu

OMEGA = 0.8
ALLP = [mg.FP64, mg.FP32, mg.FP16, mg.BF16]
Q1 = 1


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    mg.lib()


def hier(dim, n, precs, **kw):
    nlev = len(mg.level_count(n, kw.get("levels", 0)))
    if isinstance(precs, int):
        precs = [precs] * nlev
    return mg.Hierarchy(mg.make_params(dim, n, precs, op=Q1, **kw))


def rnd(dim, n, seed, scale=1.0):
    return I.uniform(seed, (n,) * dim) * scale


def dinv(n):
    """1 / diag(A) = 3 h^2 / 8 in 2D and 3D."""
    h = 1.0 / (n + 1)
    return 3.0 * h * h / 8.0


def gscale(n, prec):
    return 2.0**13 if prec == mg.FP16 else 1.0 / dinv(n)


def cscale(n, prec):
    return 2.0**14 * dinv(n) if prec == mg.FP16 else 1.0


def write(h, level, vec, x, prec):
    buf, x64 = to_storage(x, prec)
    h.level_write(level, vec, buf)
    return x64


def read(h, level, vec, n, dim, prec):
    out = empty_storage((n,) * dim, prec)
    h.level_read(level, vec, out)
    return as_f64(out)


def pname(p):
    return ["fp64", "fp32", "fp16", "bf16"][p]


CASES = [(3, n, p) for n in (7, 15, 47, 95) for p in ALLP] + [(3, 191, mg.FP16), (3, 127, mg.FP32)] + \
        [(2, n, p) for n in (15, 127, 511) for p in ALLP] + [(2, 1023, mg.FP16)]


@pytest.mark.parametrize("dim,n,prec", CASES, ids=lambda c: str(c))
def test_q1_jacobi_sweep(oracle, dim, n, prec):
    with hier(dim, n, prec) as h:
        L = h.nlev - 1
        c = write(h, L, mg.VEC_C, rnd(dim, n, 1, cscale(n, prec)), prec)
        g = write(h, L, mg.VEC_G, rnd(dim, n, 2, gscale(n, prec)), prec)
        h.run_stage(mg.STAGE_JACOBI, L)
        out = read(h, L, mg.VEC_C, n, dim, prec)
    ref = oracle.jacobi(g, c, OMEGA, op=Q1)
    mag = np.abs(c) + OMEGA * dinv(n) * (np.abs(g) + oracle.apply_A(c, absmode=True, op=Q1))
    check_close(out, ref, mag, prec, "q1 jacobi")


@pytest.mark.parametrize("dim,n,prec", CASES, ids=lambda c: str(c))
def test_q1_two_sweeps_from_zero(oracle, dim, n, prec):
    with hier(dim, n, prec) as h:
        L = h.nlev - 1
        g = write(h, L, mg.VEC_G, rnd(dim, n, 3, 2.0**13 if prec == mg.FP16 else 1.0), prec)
        h.run_stage(mg.STAGE_JACOBI_ZERO2, L)
        out = read(h, L, mg.VEC_C, n, dim, prec)
    ref = oracle.jacobi(g, oracle.jacobi(g, np.zeros_like(g), OMEGA, op=Q1), OMEGA, op=Q1)
    c1 = OMEGA * dinv(n) * np.abs(g)
    mag = c1 + OMEGA * dinv(n) * (np.abs(g) + oracle.apply_A(c1, absmode=True, op=Q1))
    check_close(out, ref, mag, prec, "q1 zero2")


RCASES = [(3, n, pf, pc) for n in (7, 15, 47, 95) for pf in ALLP for pc in (pf, mg.FP32)] + \
         [(3, 191, mg.FP16, mg.FP16), (3, 63, mg.FP64, mg.FP16)] + \
         [(2, n, pf, pc) for n in (15, 127, 511) for pf in ALLP for pc in (pf, mg.FP64)]


@pytest.mark.parametrize("dim,n,pf,pc", RCASES, ids=lambda c: str(c))
def test_q1_residual_restriction(oracle, dim, n, pf, pc):
    nlev = len(mg.level_count(n))
    with hier(dim, n, [pc] * (nlev - 1) + [pf]) as h:
        L = h.nlev - 1
        c = write(h, L, mg.VEC_C, rnd(dim, n, 4, cscale(n, pf)), pf)
        g = write(h, L, mg.VEC_G, rnd(dim, n, 5, gscale(n, pf)), pf)
        h.run_stage(mg.STAGE_RESTRICT, L)
        out = read(h, L - 1, mg.VEC_G, (n - 1) // 2, dim, pc)
    ref = oracle.restrict(oracle.residual(g, c, op=Q1))
    mag = oracle.restrict(np.abs(g) + oracle.apply_A(c, absmode=True, op=Q1))
    check_close(out, ref, mag, pf if TOL[pf] > TOL[pc] else pc, "q1 restrict")


@pytest.mark.parametrize("dim,n,prec", [(3, n, p) for n in (15, 95) for p in ALLP] +
                         [(3, 191, mg.FP16), (2, 511, mg.FP16), (2, 127, mg.BF16), (2, 255, mg.FP64),
                          (2, 127, mg.FP32)])
def test_q1_ir_update(oracle, dim, n, prec):
    """u += alpha c, r -= alpha A c in FP64 with the Q1 A c formed exactly (FP16) or as
    a double-float sum (FP32/BF16)."""
    alpha = 3.7e-6
    with hier(dim, n, prec) as h:
        L = h.nlev - 1
        c = write(h, L, mg.VEC_C, rnd(dim, n, 13, 1000.0), prec)
        u = rnd(dim, n, 14)
        r = alpha * oracle.apply_A(c, op=Q1) * (1.0 + 1e-3 * rnd(dim, n, 15))
        h.level_write(L, mg.VEC_U, u)
        h.level_write(L, mg.VEC_R, r)
        n2, ninf = h.run_stage(mg.STAGE_IR_UPDATE, L, arg=alpha)
        uo = read(h, L, mg.VEC_U, n, dim, mg.FP64)
        ro = read(h, L, mg.VEC_R, n, dim, mg.FP64)
    Ac = oracle.apply_A(c, op=Q1)
    uref = u + alpha * c
    rref = r - alpha * Ac
    check_close(uo, uref, np.abs(u) + alpha * np.abs(c), mg.FP64, "q1 update u")
    check_close(ro, rref, np.abs(r) + alpha * oracle.apply_A(c, absmode=True, op=Q1), mg.FP64, "q1 update r")
    assert np.abs(ro - rref).max() <= 1e-9 * np.abs(rref).max()
    assert n2 == pytest.approx(np.linalg.norm(ro), rel=1e-12)
    assert ninf == np.abs(ro).max()


@pytest.mark.parametrize("dim,n", [(3, 15), (3, 95), (2, 127), (2, 1023)])
def test_q1_fp64_residual(oracle, dim, n):
    import torch
    with hier(dim, n, mg.FP64) as h:
        L = h.nlev - 1
        u = rnd(dim, n, 16)
        b = rnd(dim, n, 17, 1e3)
        h.level_write(L, mg.VEC_U, u)
        n2, ninf = h.run_stage(mg.STAGE_RESIDUAL, L, ptr=torch.from_numpy(b).cuda())
        ro = read(h, L, mg.VEC_R, n, dim, mg.FP64)
    ref = oracle.residual(b, u, op=Q1)
    check_close(ro, ref, np.abs(b) + oracle.apply_A(u, absmode=True, op=Q1), mg.FP64, "q1 residual")
    assert n2 == pytest.approx(np.linalg.norm(ro), rel=1e-12)


@pytest.mark.parametrize("dim,n,prec", [(3, 3, p) for p in ALLP] + [(2, 3, mg.FP64), (3, 2, mg.FP16),
                                                                      (3, 5, mg.FP64), (2, 7, mg.FP32)])
def test_q1_base_level_solve(oracle, dim, n, prec):
    with hier(dim, n, prec, levels=1) as h:
        g = write(h, 0, mg.VEC_G, rnd(dim, n, 11), prec)
        h.run_stage(mg.STAGE_COARSE, 0)
        out = read(h, 0, mg.VEC_C, n, dim, prec)
    check_close(out, oracle.coarse_solve(g, op=Q1), oracle.coarse_solve(np.abs(g), op=Q1), prec, "q1 coarse")


@pytest.mark.parametrize("dim,n,prec", [(3, 3, mg.FP64), (3, 15, mg.FP64), (2, 31, mg.FP32), (3, 5, mg.FP16)])
def test_q1_cg_base_solve(oracle, dim, n, prec):
    tol = {mg.FP64: 1e-9, mg.FP32: 1e-5, mg.FP16: 1e-3}[prec]
    with hier(dim, n, prec, levels=1, base_solver=1, base_tol=tol) as h:
        g = write(h, 0, mg.VEC_G, rnd(dim, n, 12), prec)
        h.run_stage(mg.STAGE_COARSE, 0)
        x = read(h, 0, mg.VEC_C, n, dim, prec)
    rr = np.linalg.norm(oracle.residual(g, x, op=Q1)) / np.linalg.norm(g)
    u = {mg.FP64: 2.0**-53, mg.FP32: 2.0**-24, mg.FP16: 2.0**-11}[prec]
    assert rr <= 1.01 * tol + 400 * u, rr


@pytest.mark.parametrize("dim,n,gamma", [(3, 31, 1), (3, 47, 2), (2, 127, 1), (2, 255, 2)])
def test_q1_full_cycle_fp64(oracle, dim, n, gamma):
    g = rnd(dim, n, 18)
    with hier(dim, n, mg.FP64, gamma=gamma) as h:
        L = h.nlev - 1
        h.level_write(L, mg.VEC_G, g)
        h.run_stage(mg.STAGE_CYCLE, L)
        out = read(h, L, mg.VEC_C, n, dim, mg.FP64)
    ref = oracle.mg_cycle(g, gamma=gamma, op=Q1)
    assert np.abs(out - ref).max() <= 1e-11 * np.abs(ref).max()


# ---------------------------------------------------------------- solves

def gpu_solve(dim, n, lad, b, u0=None, **kw):
    import torch
    p = mg.make_params(dim, n, lad, zero_guess=1 if u0 is None else 0, op=Q1, **kw)
    with mg.Hierarchy(p) as h:
        bd = torch.from_numpy(b).cuda()
        ud = torch.zeros_like(bd) if u0 is None else torch.from_numpy(u0).cuda()
        res = h.solve(bd, ud)
        return ud.cpu().numpy(), res


def check_solve(oracle, dim, n, lad, b, u0=None, extra=0, **kw):
    u, res = gpu_solve(dim, n, lad, b, u0, **kw)
    okw = {k: kw[k] for k in ("scaling", "gamma", "tol_mode", "tol") if k in kw}
    uo, info, hist = oracle.ir_solve(b, u0, op=Q1, **okw)
    assert info["converged"]
    assert res["status"] == 0, res
    if kw.get("tol_mode", 0) == 0:
        assert res["rel_res_true"] <= kw.get("tol", 1e-10)
        rt = np.linalg.norm(oracle.residual(b, u, op=Q1)) / np.linalg.norm(b)
        assert rt <= kw.get("tol", 1e-10) and rt == pytest.approx(res["rel_res_true"], rel=1e-6)
    else:
        assert np.linalg.norm(oracle.residual(b, u, op=Q1)) < kw["tol"]
    assert np.linalg.norm(u - uo) <= 1e-6 * np.linalg.norm(uo)
    if extra == 0:
        assert res["iters"] == info["iters"], (res["iters"], info["iters"])
    else:
        assert res["iters"] <= info["iters"] + extra, (res["iters"], info["iters"])
    return u, res, info


@pytest.mark.parametrize("dim,n", [(3, 15), (3, 31), (3, 63), (2, 63), (2, 255), (3, 47)])
def test_q1_fp64_solve_same_iterations(oracle, dim, n):
    check_solve(oracle, dim, n, "D", I.random_rhs(dim, n, 500 + n), scaling=0)


@pytest.mark.parametrize("dim,n,lad", [(3, 63, "H"), (3, 127, "H"), (3, 95, "HSD"), (3, 63, "BSD"),
                                       (2, 255, "H"), (2, 511, "HSD"), (3, 63, "S")])
def test_q1_low_precision_solve(oracle, dim, n, lad):
    check_solve(oracle, dim, n, lad, I.random_rhs(dim, n, 600 + n), extra=2)


@pytest.mark.parametrize("no_tail", [0, 1])
def test_q1_dsh_with_cg_base(oracle, no_tail):
    dim, n = 3, 63
    nlev = len(mg.level_count(n))
    check_solve(oracle, dim, n, mg.ladder("DSH", nlev, nlev - 3, 2), I.random_rhs(dim, n, 700), extra=2,
                base_solver=1, no_tail=no_tail)


@pytest.mark.parametrize("dim,n,gamma,lad", [(3, 63, 2, "H"), (2, 127, 2, "D")])
def test_q1_wcycle(oracle, dim, n, gamma, lad):
    check_solve(oracle, dim, n, lad, I.random_rhs(dim, n, 710), extra=0 if lad == "D" else 2, gamma=gamma,
                **({"scaling": 0} if lad == "D" else {}))


@pytest.mark.parametrize("dim,n,k", [(3, 63, 1), (2, 255, 1), (3, 127, 2)])
def test_q1_manufactured_closed_form(oracle, dim, n, k):
    """The FE load vector of the manufactured sine is an eigenvector of A: the GPU's
    solution equals b / lambda in closed form (FP16 preconditioning)."""
    b = I.manufactured_load(dim, n, k)
    u, res = gpu_solve(dim, n, "H", b)
    assert res["status"] == 0 and res["rel_res_true"] <= 1e-10
    h = 1.0 / (n + 1)
    t = k * math.pi * h
    kk, mm = (2 - 2 * math.cos(t)) / h, h * (4 + 2 * math.cos(t)) / 6
    lam = dim * kk * mm ** (dim - 1) / h ** dim
    assert np.abs(u - b / lam).max() <= 1e-9 * np.abs(b / lam).max()


@pytest.mark.parametrize("dim,n,k", [(3, 63, 20), (2, 255, 20)])
def test_q1_paper_problem_random_guess(oracle, dim, n, k):
    """Sec. 8.1's setting: k = 20, initial guess uniform in [0, 1), absolute tolerance
    on ||r||_2 (of this scaling), FP16-preconditioned."""
    b = I.manufactured_load(dim, n, k)
    u0 = I.random_guess(dim, n, 720)
    check_solve(oracle, dim, n, "HSD", b, u0, extra=2, tol_mode=1, tol=1e-6)


def test_q1_batch_equals_alone():
    import torch
    specs = [(3, 63, "H", 81), (3, 95, "HSD", 82), (3, 47, "H", 83)]
    refs = [gpu_solve(d, n, lad, I.random_rhs(d, n, sd)) for d, n, lad, sd in specs]
    hs = [mg.Hierarchy(mg.make_params(d, n, lad, zero_guess=1, op=Q1)) for d, n, lad, sd in specs]
    bs = [torch.from_numpy(I.random_rhs(d, n, sd)).cuda() for d, n, lad, sd in specs]
    us = [torch.zeros_like(b) for b in bs]
    res = mg.solve_batch(hs, bs, us)
    for (u_ref, r_ref), u, r in zip(refs, us, res):
        assert r["merged"] == 1
        assert r["status"] == 0 and r["iters"] == r_ref["iters"]
        assert np.array_equal(u.cpu().numpy(), u_ref)
    for h in hs:
        h.close()


def test_q1_and_fd_instances_in_one_batch():
    """A batch mixing the two operators keeps them apart (different kernels)."""
    import torch
    specs = [(3, 63, 0, 91), (3, 63, 1, 91), (3, 47, 1, 92)]
    hs, bs, us, refs = [], [], [], []
    for d, n, op, sd in specs:
        b = I.random_rhs(d, n, sd)
        with mg.Hierarchy(mg.make_params(d, n, "H", zero_guess=1, op=op)) as h1:
            bd = torch.from_numpy(b).cuda()
            ud = torch.zeros_like(bd)
            r1 = h1.solve(bd, ud)
            refs.append((ud.cpu().numpy(), r1))
        hs.append(mg.Hierarchy(mg.make_params(d, n, "H", zero_guess=1, op=op)))
        bs.append(torch.from_numpy(b).cuda())
        us.append(torch.zeros_like(bs[-1]))
    res = mg.solve_batch(hs, bs, us)
    for (u_ref, r_ref), u, r in zip(refs, us, res):
        assert r["status"] == 0 and r["iters"] == r_ref["iters"]
        assert np.array_equal(u.cpu().numpy(), u_ref)
    assert not np.array_equal(refs[0][0], refs[1][0])
    for h in hs:
        h.close()
