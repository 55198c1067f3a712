"""DSH_MG pieces of Sec. 6: residual rescaling on restriction into FP16 levels
and the conjugate-gradient base solver in the base level's precision.

Kernel level (stages through the C ABI) against the FP64 oracle on the same
inputs; solve level: the paper's DSH ladder (FP16 base with CG, FP16 level 1,
FP32 level 2, FP64 above) reaches the FP64 accuracy of the oracle within two
extra IR steps, with and without the coarse-tail kernel, and batched
instances with rescaled levels give their alone results bit for bit."""
import math

import numpy as np
import pytest

from _helpers import TOL, as_f64, check_close, empty_storage, to_storage
from paper_2007_07539_gb300 import inputs as I
from paper_2007_07539_gb300 import mg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    mg.lib()


def write(h, level, vec, x, prec):
    buf, x64 = to_storage(x, prec)
    h.level_write(level, vec, buf)
    return x64


def read(h, level, vec, n, dim, prec):
    out = empty_storage((n,) * dim, prec)
    h.level_read(level, vec, out)
    return as_f64(out)


def dinv(dim, n):
    h = 1.0 / (n + 1)
    return h * h / (2 * dim)


def paper_dsh(nlev):
    """Sec. 6: CG base solver in FP16 on level 0, FP16 on level 1, FP32 on level 2,
    FP64 on the rest."""
    return mg.ladder("DSH", nlev, nlev - 3, 2)


# ---------------------------------------------------------------- rescaled restriction

RS_CASES = [(3, n, pf, amp) for n in (7, 15, 47, 95) for pf in (mg.FP32, mg.FP64) for amp in (1.0, 1e-7)] + \
           [(3, 63, mg.FP64, 1e-12), (3, 31, mg.FP32, 1e5), (2, 127, mg.FP32, 1.0), (2, 511, mg.FP64, 1e-9),
            (2, 15, mg.FP64, 1.0)]


@pytest.mark.parametrize("dim,n,pf,amp", RS_CASES)
def test_rescaled_restriction_into_fp16(oracle, dim, n, pf, amp):
    """g_{l-1} = fp16(R (g_l - A c_l) / s), s a power of two that puts the max-norm in
    [2^13, 2^14]: s times the stored values equals the FP64 restriction within FP16
    rounding at any input magnitude (amp), where a plain cast would flush small
    residuals to zero or subnormals."""
    nlev = len(mg.level_count(n))
    precs = [mg.FP16] * (nlev - 1) + [pf]
    nc = (n - 1) // 2
    with mg.Hierarchy(mg.make_params(dim, n, precs)) as h:
        L = h.nlev - 1
        c = write(h, L, mg.VEC_C, I.uniform(31, (n,) * dim) * amp, pf)
        g = write(h, L, mg.VEC_G, I.uniform(32, (n,) * dim) * amp / dinv(dim, n), pf)
        s, _ = h.run_stage(mg.STAGE_RESTRICT_RESCALE, L)
        out = read(h, L - 1, mg.VEC_G, nc, dim, mg.FP16)
    assert s > 0 and math.frexp(s)[0] == 0.5, s  # a power of two
    ref = oracle.restrict(oracle.residual(g, c))
    m = np.abs(out).max()
    assert 2.0**13 <= m <= 2.0**14, m
    assert 2.0**13 * (1 - 1e-5) <= np.abs(ref).max() / s <= 2.0**14 * (1 + 1e-5)
    mag = oracle.restrict(np.abs(g) + oracle.apply_A(c, absmode=True))
    check_close(out * s, ref, mag, mg.FP16, "rescaled restriction")


def test_rescaled_restriction_of_zero(oracle):
    """A zero residual keeps s = 1 and gives zeros."""
    dim, n = 3, 15
    nlev = len(mg.level_count(n))
    with mg.Hierarchy(mg.make_params(dim, n, [mg.FP16] * (nlev - 1) + [mg.FP32])) as h:
        L = h.nlev - 1
        write(h, L, mg.VEC_C, np.zeros((n,) * dim), mg.FP32)
        write(h, L, mg.VEC_G, np.zeros((n,) * dim), mg.FP32)
        s, _ = h.run_stage(mg.STAGE_RESTRICT_RESCALE, L)
        out = read(h, L - 1, mg.VEC_G, 7, dim, mg.FP16)
    assert s == 1.0 and not out.any()


def test_rescaled_restriction_needs_a_transition():
    """The stage is refused where the coarse level is not a rescaled FP16 level."""
    with mg.Hierarchy(mg.make_params(3, 15, "H")) as h:
        with pytest.raises(RuntimeError):
            h.run_stage(mg.STAGE_RESTRICT_RESCALE, h.nlev - 1)
    nlev = len(mg.level_count(15))
    with mg.Hierarchy(mg.make_params(3, 15, [mg.FP16] * (nlev - 1) + [mg.FP32], rescale16=0)) as h:
        with pytest.raises(RuntimeError):
            h.run_stage(mg.STAGE_RESTRICT_RESCALE, h.nlev - 1)


@pytest.mark.parametrize("dim,n,pf,s", [(3, 15, mg.FP32, 2.0**-20), (3, 95, mg.FP64, 2.0**-35),
                                        (2, 127, mg.FP32, 2.0**-3), (3, 47, mg.FP32, 1.0)])
def test_prolongation_of_rescaled_level(oracle, dim, n, pf, s):
    """c_l += s P c_{l-1}: the correction of a rescaled FP16 level returns at scale s."""
    nlev = len(mg.level_count(n))
    nc = (n - 1) // 2
    with mg.Hierarchy(mg.make_params(dim, n, [mg.FP16] * (nlev - 1) + [pf])) as h:
        L = h.nlev - 1
        cf = write(h, L, mg.VEC_C, I.uniform(41, (n,) * dim) * 2.0**14 * s * dinv(dim, n), pf)
        cc = write(h, L - 1, mg.VEC_C, I.uniform(42, (nc,) * dim) * 2.0**14 * dinv(dim, n), mg.FP16)
        h.run_stage(mg.STAGE_PROLONG, L, arg=s)
        out = read(h, L, mg.VEC_C, n, dim, pf)
    ref = oracle.prolong_add(s * cc, cf)
    mag = np.abs(cf) + oracle.prolong_add(s * np.abs(cc), np.zeros_like(cf))
    check_close(out, ref, mag, pf, "prolong (rescaled)")


# ---------------------------------------------------------------- CG base solver

CG_CASES = [(3, 3, p) for p in (mg.FP64, mg.FP32, mg.FP16, mg.BF16)] + \
           [(2, 3, mg.FP64), (3, 2, mg.FP16), (3, 5, mg.FP32), (2, 31, mg.FP64), (3, 15, mg.FP64),
            (3, 15, mg.FP32), (2, 63, mg.FP16), (3, 1, mg.FP64)]
UNIT = {mg.FP64: 2.0**-53, mg.FP32: 2.0**-24, mg.FP16: 2.0**-11, mg.BF16: 2.0**-8}


def laplace_cond(dim, n):
    h = 1.0 / (n + 1)
    return (math.sin(n * math.pi * h / 2) / math.sin(math.pi * h / 2)) ** 2


@pytest.mark.parametrize("dim,n,prec", CG_CASES)
def test_cg_base_solve(oracle, dim, n, prec):
    """CG from x = 0 on the base level stops at ||r||_2 <= tol ||g||_2 (recursive r);
    the true residual of the stored x, in FP64, is within tol plus the storage
    rounding (kappa u), and x is within kappa times that of the exact solve."""
    tol = {mg.FP64: 1e-9, mg.FP32: 1e-5, mg.FP16: 1e-3, mg.BF16: 1e-2}[prec]
    with mg.Hierarchy(mg.make_params(dim, n, [prec], levels=1, base_solver=1, base_tol=tol)) as h:
        g = write(h, 0, mg.VEC_G, I.uniform(51 + n, (n,) * dim), prec)
        h.run_stage(mg.STAGE_COARSE, 0)
        x = read(h, 0, mg.VEC_C, n, dim, prec)
    kappa = laplace_cond(dim, n)
    rr = np.linalg.norm(oracle.residual(g, x)) / np.linalg.norm(g)
    assert rr <= 1.01 * tol + 4 * kappa * UNIT[prec], (rr, tol)
    xs = oracle.coarse_solve(g)
    assert np.linalg.norm(x - xs) <= kappa * (1.01 * tol + 4 * kappa * UNIT[prec]) * np.linalg.norm(xs)


def test_cg_base_solve_of_zero(oracle):
    with mg.Hierarchy(mg.make_params(3, 3, [mg.FP16], levels=1, base_solver=1)) as h:
        write(h, 0, mg.VEC_G, np.zeros((3, 3, 3)), mg.FP16)
        h.run_stage(mg.STAGE_COARSE, 0)
        assert not read(h, 0, mg.VEC_C, 3, 3, mg.FP16).any()


def test_cg_step_limit_one_is_a_steepest_descent_step(oracle):
    """base_maxit = 1: x = (g^T g / g^T A g) g exactly (FP64)."""
    dim, n = 3, 5
    with mg.Hierarchy(mg.make_params(dim, n, [mg.FP64], levels=1, base_solver=1, base_maxit=1,
                                     base_tol=0.0)) as h:
        g = write(h, 0, mg.VEC_G, I.uniform(61, (n,) * dim), mg.FP64)
        h.run_stage(mg.STAGE_COARSE, 0)
        x = read(h, 0, mg.VEC_C, n, dim, mg.FP64)
    Ag = oracle.apply_A(g)
    ref = (g.ravel() @ g.ravel()) / (g.ravel() @ Ag.ravel()) * g
    assert np.abs(x - ref).max() <= 1e-13 * np.abs(ref).max()


# ---------------------------------------------------------------- solves

def gpu_solve(dim, n, lad, b, **kw):
    import torch
    p = mg.make_params(dim, n, lad, zero_guess=1, **kw)
    with mg.Hierarchy(p) as h:
        bd = torch.from_numpy(b).cuda()
        ud = torch.zeros_like(bd)
        res = h.solve(bd, ud)
        return ud.cpu().numpy(), res


def check_solve(oracle, dim, n, lad, b, extra, **kw):
    u, res = gpu_solve(dim, n, lad, b, **kw)
    okw = dict(scaling=kw.get("scaling", 1))
    uo, info, hist = oracle.ir_solve(b, None, **okw)
    assert info["converged"]
    assert res["status"] == 0, res
    assert res["rel_res_true"] <= 1e-10
    rt = np.linalg.norm(oracle.residual(b, u)) / np.linalg.norm(b)
    assert rt <= 1e-10
    assert np.linalg.norm(u - uo) <= 1e-6 * np.linalg.norm(uo)
    assert res["iters"] <= info["iters"] + extra, (res["iters"], info["iters"])
    return u, res, info


@pytest.mark.parametrize("no_tail", [0, 1])
@pytest.mark.parametrize("dim,n,rhs", [(3, 63, "random"), (3, 127, "manufactured"), (2, 255, "random"),
                                       (3, 95, "random")])
def test_dsh_paper_ladder_solve(oracle, dim, n, rhs, no_tail):
    """Sec. 6's DSH_MG: FP16 CG base, FP16 level 1, FP32 level 2, FP64 above, residual
    rescaled into the FP16 levels: FP64 accuracy within two extra IR steps."""
    b = I.random_rhs(dim, n, 300 + n) if rhs == "random" else I.manufactured_rhs(dim, n)
    nlev = len(mg.level_count(n))
    check_solve(oracle, dim, n, paper_dsh(nlev), b, 2, base_solver=1, no_tail=no_tail)


@pytest.mark.parametrize("sigma", [0, 14])
def test_dsh_rescaling_with_unit_scaled_residual(oracle, sigma):
    """With the paper's norm-one IR scaling (sigma_log2 = 0) the restricted residual on
    the FP16 levels is small; the rescale keeps it in FP16's normal range, and the
    wide FP16 range above a big (non-tail) transition level works the same."""
    dim, n = 3, 127
    b = I.random_rhs(dim, n, 77)
    lad = [mg.FP16] * 4 + [mg.FP32, mg.FP64]  # rescaled transition 63^3 (FP32) -> 31^3 (FP16): plain kernels
    for no_tail in (0, 1):
        check_solve(oracle, dim, n, lad, b, 2, sigma_log2=sigma, no_tail=no_tail)


def test_rescale_changes_only_fp16_transitions(oracle):
    """rescale16 has no effect on ladders without a non-FP16 to FP16 restriction."""
    dim, n = 3, 63
    b = I.random_rhs(dim, n, 78)
    for lad in ("H", "HSD", "D"):
        u1, r1 = gpu_solve(dim, n, lad, b)
        u0, r0 = gpu_solve(dim, n, lad, b, rescale16=0)
        assert np.array_equal(u1, u0) and r1["iters"] == r0["iters"]


@pytest.mark.parametrize("lad,extra", [("D", 1), ("H", 2), ("HSD", 2)])
def test_cg_base_in_other_ladders(oracle, lad, extra):
    """The CG base solver (tolerance 1e-4) in place of the exact solve."""
    dim, n = 3, 63
    check_solve(oracle, dim, n, lad, I.random_rhs(dim, n, 79), extra, base_solver=1)


def test_batch_with_rescaled_levels_equals_alone():
    """Merged batches carry the rescale (tail-internal and plain-kernel transitions)
    and the CG base solver: each instance gives its alone result bit for bit."""
    import torch
    specs = [(3, 63, paper_dsh(5), 81, dict(base_solver=1)),
             (3, 127, [mg.FP16] * 4 + [mg.FP32, mg.FP64], 82, {}),
             (3, 95, "H", 83, dict(base_solver=1)),
             (3, 47, paper_dsh(5), 84, {})]
    refs = [gpu_solve(d, n, lad, I.random_rhs(d, n, sd), **kw) for d, n, lad, sd, kw in specs]
    hs = [mg.Hierarchy(mg.make_params(d, n, lad, zero_guess=1, **kw)) for d, n, lad, sd, kw in specs]
    bs = [torch.from_numpy(I.random_rhs(d, n, sd)).cuda() for d, n, lad, sd, kw in specs]
    us = [torch.zeros_like(b) for b in bs]
    res = mg.solve_batch(hs, bs, us)
    for (u_ref, r_ref), u, r in zip(refs, us, res):
        assert r["merged"] == 1
        assert r["status"] == 0 and r["iters"] == r_ref["iters"]
        assert np.array_equal(u.cpu().numpy(), u_ref)
    for h in hs:
        h.close()
