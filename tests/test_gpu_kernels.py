"""Kernel parity: each CUDA kernel of the method, run through the C ABI
(mg_level_write / mg_run_stage / mg_level_read), against the FP64 oracle
evaluated on the same storage-rounded inputs.  Bound per point:
|gpu - oracle| <= tol * M with tol = 1e-12 (FP64), 1e-5 (FP32), 5e-3
(FP16/BF16) and M the componentwise scaled magnitude of the operation.
FP16 and BF16 outputs are also held to one rounding of the exact result:
|gpu - round(oracle)| <= one spacing of the format + the FP32 arithmetic's
error bound (check_rounded).
Sizes span several CTA tiles, multi-chunk rows and ragged (padded) rows."""
import math

import numpy as np
import pytest

from paper_2007_07539_gb300 import inputs as I
from paper_2007_07539_gb300 import mg
from _helpers import TOL, as_f64, check_close, check_rounded, empty_storage, to_storage

pytestmark = pytest.mark.gpu

OMEGA = 0.8
ALLP = [mg.FP64, mg.FP32, mg.FP16, mg.BF16]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    mg.lib()


def hier(dim, n, precs, **kw):
    nlev = len(mg.level_count(n, kw.get("levels", 0)))
    if isinstance(precs, int):
        precs = [precs] * nlev
    return mg.Hierarchy(mg.make_params(dim, n, precs, **kw))


def rnd(dim, n, seed, scale=1.0):
    return I.uniform(seed, (n,) * dim) * scale


def dinv(dim, n):
    h = 1.0 / (n + 1)
    return h * h / (2 * dim)


def gscale(dim, n, prec):
    """Right-hand side scale.  FP16 data are kept at the magnitudes the solver gives them
    (scaled residual of inf-norm 2^14, Alg. 2's residual scaling, so corrections of size 2^14 h^2):
    above FP16's subnormal range and with residuals below its overflow threshold."""
    return 2.0**13 if prec == mg.FP16 else 1.0 / dinv(dim, n)


def cscale(dim, n, prec):
    """Correction scale matching gscale: about D^-1 g."""
    return 2.0**14 * dinv(dim, n) if prec == mg.FP16 else 1.0


def write(h, level, vec, x, prec):
    buf, x64 = to_storage(x, prec)
    h.level_write(level, vec, buf)
    return x64


def read(h, level, vec, n, dim, prec):
    out = empty_storage((n,) * dim, prec)
    h.level_read(level, vec, out)
    return as_f64(out)


CASES3 = [(n, p) for n in (7, 15, 47, 95) for p in ALLP] + [(191, mg.FP32), (287, mg.FP16), (127, mg.BF16)]
CASES2 = [(n, p) for n in (15, 127, 511) for p in ALLP] + [(1023, mg.FP16), (2047, mg.FP64)]
CASES = [(3, n, p) for n, p in CASES3] + [(2, n, p) for n, p in CASES2]


def ids(c):
    return f"{c[0]}d-n{c[1]}-{['fp64', 'fp32', 'fp16', 'bf16'][c[2]]}"


@pytest.mark.parametrize("case", CASES, ids=ids)
def test_jacobi_sweep(oracle, case):
    """Damped Jacobi (Sec. 4.2): c + omega D^-1 (g - A c)."""
    dim, n, prec = case
    with hier(dim, n, prec) as h:
        L = h.nlev - 1
        c = write(h, L, mg.VEC_C, rnd(dim, n, 1, cscale(dim, n, prec)), prec)
        g = write(h, L, mg.VEC_G, rnd(dim, n, 2, gscale(dim, n, prec)), prec)
        h.run_stage(mg.STAGE_JACOBI, L)
        out = read(h, L, mg.VEC_C, n, dim, prec)
    ref = oracle.jacobi(g, c, OMEGA)
    mag = np.abs(c) + OMEGA * dinv(dim, n) * (np.abs(g) + oracle.apply_A(c, absmode=True))
    check_close(out, ref, mag, prec, "jacobi")
    check_rounded(oracle, out, ref, mag, prec, "jacobi")


@pytest.mark.parametrize("case", CASES, ids=ids)
def test_two_sweeps_from_zero(oracle, case):
    """Pre-smoothing from c = 0 (Alg. 1's pre-smoothing), two sweeps fused in one pass."""
    dim, n, prec = case
    with hier(dim, n, prec) as h:
        L = h.nlev - 1
        g = write(h, L, mg.VEC_G, rnd(dim, n, 3, 2.0**13 if prec == mg.FP16 else 1.0), prec)
        h.run_stage(mg.STAGE_JACOBI_ZERO2, L)
        out = read(h, L, mg.VEC_C, n, dim, prec)
    ref = oracle.jacobi(g, oracle.jacobi(g, np.zeros_like(g), OMEGA), OMEGA)
    c1 = OMEGA * dinv(dim, n) * np.abs(g)
    mag = c1 + OMEGA * dinv(dim, n) * (np.abs(g) + oracle.apply_A(c1, absmode=True))
    check_close(out, ref, mag, prec, "zero2")
    check_rounded(oracle, out, ref, mag, prec, "zero2")


RCASES = [(3, n, pf, pc) for n in (7, 15, 47, 95) for pf in ALLP for pc in (pf, mg.FP32)] + \
    [(3, 191, mg.FP32, mg.FP64), (3, 287, mg.FP16, mg.FP16), (3, 95, mg.FP64, mg.FP16)] + \
    [(2, n, pf, pc) for n in (15, 127, 511) for pf in ALLP for pc in (pf, mg.FP64)] + \
    [(2, 1023, mg.FP16, mg.FP32), (2, 2047, mg.FP64, mg.FP64)]


def rids(c):
    nm = ['fp64', 'fp32', 'fp16', 'bf16']
    return f"{c[0]}d-n{c[1]}-{nm[c[2]]}-to-{nm[c[3]]}"


def two_level_precs(n, pf, pc):
    nlev = len(mg.level_count(n))
    return [pc] * (nlev - 1) + [pf]


@pytest.mark.parametrize("case", RCASES, ids=rids)
def test_residual_restriction(oracle, case):
    """Alg. 1's residual restriction: g_{l-1} = cast(R (g_l - A_l c_l)), full weighting, fused."""
    dim, n, pf, pc = case
    with hier(dim, n, two_level_precs(n, pf, pc)) as h:
        L = h.nlev - 1
        c = write(h, L, mg.VEC_C, rnd(dim, n, 4, cscale(dim, n, pf)), pf)
        g = write(h, L, mg.VEC_G, rnd(dim, n, 5, gscale(dim, n, pf)), pf)
        h.run_stage(mg.STAGE_RESTRICT, L)
        nc = (n - 1) // 2
        out = read(h, L - 1, mg.VEC_G, nc, dim, pc)
    ref = oracle.restrict(oracle.residual(g, c))
    mag = oracle.restrict(np.abs(g) + oracle.apply_A(c, absmode=True))
    worst = pf if TOL[pf] > TOL[pc] else pc
    check_close(out, ref, mag, worst, "restrict")
    check_rounded(oracle, out, ref, mag, pc, "restrict", k=64)


TILE_CASES = [(k, n, p) for k in (0, 1, 2) for n in (17, 47, 95) for p in (mg.FP16, mg.FP64)]


@pytest.mark.parametrize("case", TILE_CASES,
                         ids=lambda c: f"{['jacobi', 'zero2', 'restrict'][c[0]]}-n{c[1]}-{['fp64', 'fp32', 'fp16', 'bf16'][c[2]]}")
def test_tile_shapes_give_the_same_bits(oracle, case):
    """Every launch shape of a 3D stencil kernel (mg_tile_set) gives the same bits: the direct
    kernel, one row per warp marching two planes per step (march lengths 1, 2, 3 and whole:
    single-plane last steps, odd and even plane counts), two rows per warp; and the oracle
    (Sec. 4.2 smoother, Alg. 1's residual restriction)."""
    kernel, n, prec = case
    dim, nc = 3, (n - 1) // 2
    zmax = nc if kernel == 2 else n
    shapes = [(0, 0), (1, 1), (1, 2), (1, 3), (1, zmax)]
    if kernel != 2:
        shapes += [(2, 1), (2, 2), (2, 5), (2, zmax)]
    stage = [mg.STAGE_JACOBI, mg.STAGE_JACOBI_ZERO2, mg.STAGE_RESTRICT][kernel]
    outs = []
    try:
        for rpw, z in shapes:
            mg.tile_set(kernel, prec, n, rpw, z)
            with hier(dim, n, prec) as h:
                L = h.nlev - 1
                c = write(h, L, mg.VEC_C, rnd(dim, n, 21, cscale(dim, n, prec)), prec)
                g = write(h, L, mg.VEC_G, rnd(dim, n, 22, gscale(dim, n, prec)), prec)
                h.run_stage(stage, L)
                outs.append(read(h, L - 1, mg.VEC_G, nc, dim, prec) if kernel == 2 else read(h, L, mg.VEC_C, n, dim, prec))
    finally:
        mg.tile_set(kernel, prec, n, -1)
    for (rpw, z), o in zip(shapes[1:], outs[1:]):
        assert np.array_equal(o, outs[0]), (rpw, z, np.count_nonzero(o != outs[0]))
    if kernel == 0:
        ref = oracle.jacobi(g, c, OMEGA)
        mag = np.abs(c) + OMEGA * dinv(dim, n) * (np.abs(g) + oracle.apply_A(c, absmode=True))
    elif kernel == 1:
        ref = oracle.jacobi(g, oracle.jacobi(g, np.zeros_like(g), OMEGA), OMEGA)
        c1 = OMEGA * dinv(dim, n) * np.abs(g)
        mag = c1 + OMEGA * dinv(dim, n) * (np.abs(g) + oracle.apply_A(c1, absmode=True))
    else:
        ref = oracle.restrict(oracle.residual(g, c))
        mag = oracle.restrict(np.abs(g) + oracle.apply_A(c, absmode=True))
    check_close(outs[0], ref, mag, prec, "tile shapes")


@pytest.mark.parametrize("case", [c for c in RCASES if c[0] == 3], ids=rids)
def test_one_pass_presmoothing_and_restriction(oracle, case):
    """Alg. 1's pre-smoothing and residual restriction in one pass (temporal blocking): c = two sweeps from zero on g,
    g_{l-1} = cast(R (g - A c)).  Against the oracle, and bit for bit against the two
    separate kernels."""
    dim, n, pf, pc = case
    precs = two_level_precs(n, pf, pc)
    nc = (n - 1) // 2
    gin = rnd(dim, n, 6, 2.0**13 if pf == mg.FP16 else 1.0)
    outs = []
    for fused in (True, False):
        with hier(dim, n, precs) as h:
            L = h.nlev - 1
            g = write(h, L, mg.VEC_G, gin, pf)
            if fused:
                h.run_stage(mg.STAGE_PRE_RESTRICT, L)
            else:
                h.run_stage(mg.STAGE_JACOBI_ZERO2, L)
                h.run_stage(mg.STAGE_RESTRICT, L)
            outs.append((read(h, L, mg.VEC_C, n, dim, pf), read(h, L - 1, mg.VEC_G, nc, dim, pc)))
    (c, gc), (c2, gc2) = outs
    assert np.array_equal(c, c2) and np.array_equal(gc, gc2)
    ref = oracle.jacobi(g, oracle.jacobi(g, np.zeros_like(g), OMEGA), OMEGA)
    c1 = OMEGA * dinv(dim, n) * np.abs(g)
    mag = c1 + OMEGA * dinv(dim, n) * (np.abs(g) + oracle.apply_A(c1, absmode=True))
    check_close(c, ref, mag, pf, "pre-smoothing")
    refc = oracle.restrict(oracle.residual(g, c))
    magc = oracle.restrict(np.abs(g) + oracle.apply_A(c, absmode=True))
    worst = pf if TOL[pf] > TOL[pc] else pc
    check_close(gc, refc, magc, worst, "restriction")


@pytest.mark.parametrize("case", RCASES, ids=rids)
def test_prolongation_and_correction(oracle, case):
    """Alg. 1's prolongation and correction: c_l += cast(P c_{l-1}), bi/trilinear interpolation."""
    dim, n, pf, pc = case
    nc = (n - 1) // 2
    with hier(dim, n, two_level_precs(n, pf, pc)) as h:
        L = h.nlev - 1
        cf = write(h, L, mg.VEC_C, rnd(dim, n, 6, cscale(dim, n, pf)), pf)
        cc = write(h, L - 1, mg.VEC_C, rnd(dim, nc, 7, cscale(dim, n, pf)), pc)
        h.run_stage(mg.STAGE_PROLONG, L)
        out = read(h, L, mg.VEC_C, n, dim, pf)
    ref = oracle.prolong_add(cc, cf)
    mag = np.abs(cf) + oracle.prolong_add(np.abs(cc), np.zeros_like(cf))
    worst = pf if TOL[pf] > TOL[pc] else pc
    check_close(out, ref, mag, worst, "prolong")
    check_rounded(oracle, out, ref, mag, pf, "prolong")


@pytest.mark.parametrize("case", RCASES, ids=rids)
def test_prolongation_fused_into_sweep(oracle, case):
    """Alg. 1's prolongation and post-smoothing fused: one Jacobi sweep applied to c_l + P c_{l-1}."""
    dim, n, pf, pc = case
    nc = (n - 1) // 2
    with hier(dim, n, two_level_precs(n, pf, pc)) as h:
        L = h.nlev - 1
        cf = write(h, L, mg.VEC_C, rnd(dim, n, 8, cscale(dim, n, pf)), pf)
        cc = write(h, L - 1, mg.VEC_C, rnd(dim, nc, 9, cscale(dim, n, pf)), pc)
        g = write(h, L, mg.VEC_G, rnd(dim, n, 10, gscale(dim, n, pf)), pf)
        h.run_stage(mg.STAGE_JACOBI_PROLONG, L)
        out = read(h, L, mg.VEC_C, n, dim, pf)
    v = oracle.prolong_add(cc, cf)
    ref = oracle.jacobi(g, v, OMEGA)
    vm = np.abs(cf) + oracle.prolong_add(np.abs(cc), np.zeros_like(cf))
    mag = vm + OMEGA * dinv(dim, n) * (np.abs(g) + oracle.apply_A(vm, absmode=True))
    worst = pf if TOL[pf] > TOL[pc] else pc
    check_close(out, ref, mag, worst, "jacobi+prolong")


@pytest.mark.parametrize("dim,n,prec", [(3, 3, p) for p in ALLP] + [(2, 3, mg.FP64), (3, 2, mg.FP16),
                                                                      (3, 5, mg.FP64), (2, 7, mg.FP32),
                                                                      (3, 1, mg.FP64)])
def test_base_level_solve(oracle, dim, n, prec):
    """Exact solve on the coarsest level (Sec. 4.2) with the dense FP64 inverse."""
    with hier(dim, n, prec, levels=1) as h:
        g = write(h, 0, mg.VEC_G, rnd(dim, n, 11), prec)
        h.run_stage(mg.STAGE_COARSE, 0)
        out = read(h, 0, mg.VEC_C, n, dim, prec)
    ref = oracle.coarse_solve(g)
    mag = oracle.coarse_solve(np.abs(g))
    check_close(out, ref, mag, prec, "coarse")
    check_rounded(oracle, out, ref, mag, prec, "coarse")


@pytest.mark.parametrize("dim,n,prec", [(3, 47, mg.FP16), (3, 95, mg.BF16), (3, 63, mg.FP32), (3, 31, mg.FP64),
                                        (2, 511, mg.FP16), (2, 127, mg.FP64), (3, 287, mg.FP16)])
def test_scale_cast_and_first_sweeps(oracle, dim, n, prec):
    """Alg. 2's residual scaling (r_low = cast(r/alpha), here r * 2^14/||r||_inf) fused with the first
    two sweeps.  The residual is tiny (1e-12 scale) to exercise the FP32-free rescaling."""
    r = rnd(dim, n, 12, 3e-12)
    r[tuple([0] * dim)] = 0.0
    s = 2.0**14 / np.abs(r).max()
    with hier(dim, n, prec) as h:
        L = h.nlev - 1
        h.level_write(L, mg.VEC_R, r)
        h.run_stage(mg.STAGE_SCALE_ZERO2, L, arg=s)
        g = read(h, L, mg.VEC_G, n, dim, prec)
        out = read(h, L, mg.VEC_C, n, dim, prec)
    check_close(g, r * s, np.abs(r * s), prec, "scale-cast")
    check_rounded(oracle, g, r * s, np.abs(r * s), prec, "scale-cast")
    assert g[tuple([0] * dim)] == 0.0
    ref = oracle.jacobi(g, oracle.jacobi(g, np.zeros_like(g), OMEGA), OMEGA)
    c1 = OMEGA * dinv(dim, n) * np.abs(g)
    mag = c1 + OMEGA * dinv(dim, n) * (np.abs(g) + oracle.apply_A(c1, absmode=True))
    check_close(out, ref, mag, prec, "scale-cast+zero2")
    check_rounded(oracle, out, ref, mag, prec, "scale-cast+zero2")


@pytest.mark.parametrize("dim,n,prec", [(3, n, p) for n in (15, 95) for p in ALLP] +
                         [(3, 287, mg.FP16), (2, 511, mg.FP16), (2, 127, mg.BF16), (2, 255, mg.FP64),
                          (2, 127, mg.FP32)])
def test_ir_update(oracle, dim, n, prec):
    """Alg. 2's solution and residual updates in one kernel: u += alpha c, r -= alpha A c in FP64, with
    ||r||_2 and ||r||_inf.  r is built so that the update cancels most of it."""
    alpha = 3.7e-6
    with hier(dim, n, prec) as h:
        L = h.nlev - 1
        c = write(h, L, mg.VEC_C, rnd(dim, n, 13, 1000.0), prec)
        u = rnd(dim, n, 14)
        r = alpha * oracle.apply_A(c) * (1.0 + 1e-3 * rnd(dim, n, 15))
        h.level_write(L, mg.VEC_U, u)
        h.level_write(L, mg.VEC_R, r)
        n2, ninf = h.run_stage(mg.STAGE_IR_UPDATE, L, arg=alpha)
        uo = read(h, L, mg.VEC_U, n, dim, mg.FP64)
        ro = read(h, L, mg.VEC_R, n, dim, mg.FP64)
    uref = u + alpha * c
    rref = r - alpha * oracle.apply_A(c)
    check_close(uo, uref, np.abs(u) + alpha * np.abs(c), mg.FP64, "update u")
    check_close(ro, rref, np.abs(r) + alpha * oracle.apply_A(c, absmode=True), mg.FP64, "update r")
    # the update of r is exact up to one FP64 rounding: far tighter than the bound above
    assert np.abs(ro - rref).max() <= 1e-9 * np.abs(rref).max()
    assert n2 == pytest.approx(np.linalg.norm(ro), rel=1e-12)
    assert ninf == np.abs(ro).max()


@pytest.mark.parametrize("dim,n,prec", [(3, 95, mg.FP16), (3, 255, mg.FP16), (3, 95, mg.BF16), (3, 47, mg.FP32),
                                        (2, 511, mg.FP16), (2, 127, mg.BF16)])
def test_ir_update_writes_the_next_scaled_residual(oracle, dim, n, prec):
    """The update's scale-ahead output (reading R21 of Alg. 2's residual scaling): with a power of
    two s it also writes the next step's g = cast(trunc_FP32(r_new s)).  Checked bit for bit
    against the oracle's emulated cast applied to the kernel's own updated r (pinned against
    numpy's FP32 / FP16 conversions on CPU), with s putting max |r_new s| near 2^14, as in a
    solve.  u and r are checked as in test_ir_update."""
    alpha = 3.7e-6
    fmt = {mg.FP16: oracle.FP16, mg.BF16: oracle.BF16, mg.FP32: oracle.FP32}[prec]
    with hier(dim, n, prec) as h:
        L = h.nlev - 1
        c = write(h, L, mg.VEC_C, rnd(dim, n, 23, 1000.0), prec)
        u = rnd(dim, n, 24)
        r = alpha * oracle.apply_A(c) * (1.0 + 1e-3 * rnd(dim, n, 25))
        rref = r - alpha * oracle.apply_A(c)
        _, e = np.frexp(np.abs(rref).max())
        s = 2.0 ** (14 - int(e))  # the power of two of the scale-ahead rule
        h.level_write(L, mg.VEC_U, u)
        h.level_write(L, mg.VEC_R, r)
        h.run_stage(mg.STAGE_IR_UPDATE, L, arg=alpha, arg2=s)
        ro = read(h, L, mg.VEC_R, n, dim, mg.FP64)
        go = read(h, L, mg.VEC_G, n, dim, prec)
        uo = read(h, L, mg.VEC_U, n, dim, mg.FP64)
    check_close(uo, u + alpha * c, np.abs(u) + alpha * np.abs(c), mg.FP64, "update u")
    assert np.abs(ro - rref).max() <= 1e-9 * np.abs(rref).max()
    want, over = oracle.scale_ahead_cast(fmt, ro, s)
    assert not over
    assert np.array_equal(go, want), (np.abs(go - want).max(), np.count_nonzero(go != want))
    assert 2.0**13 <= np.abs(go).max() <= 2.0**14


@pytest.mark.parametrize("dim,n", [(3, 15), (3, 95), (2, 127), (2, 1023)])
def test_fp64_residual(oracle, dim, n):
    """IR step 1 (Sec. 4.1): r = b - A u in FP64, with norms."""
    import torch
    with hier(dim, n, mg.FP64) as h:
        L = h.nlev - 1
        u = rnd(dim, n, 16)
        b = rnd(dim, n, 17, 1e3)
        h.level_write(L, mg.VEC_U, u)
        bd = torch.from_numpy(b).cuda()
        n2, ninf = h.run_stage(mg.STAGE_RESIDUAL, L, ptr=bd)
        ro = read(h, L, mg.VEC_R, n, dim, mg.FP64)
    ref = oracle.residual(b, u)
    check_close(ro, ref, np.abs(b) + oracle.apply_A(u, absmode=True), mg.FP64, "residual")
    assert n2 == pytest.approx(np.linalg.norm(ro), rel=1e-12)
    assert ninf == np.abs(ro).max()


@pytest.mark.parametrize("dim,n,gamma", [(3, 31, 1), (3, 63, 2), (2, 127, 1), (2, 255, 2), (3, 47, 1)])
def test_full_cycle_fp64(oracle, dim, n, gamma):
    """One multigrid cycle (Alg. 1 applied recursively; gamma = 2: W-cycle) in FP64."""
    g = rnd(dim, n, 18)
    with hier(dim, n, mg.FP64, gamma=gamma) as h:
        L = h.nlev - 1
        h.level_write(L, mg.VEC_G, g)
        h.run_stage(mg.STAGE_CYCLE, L)
        out = read(h, L, mg.VEC_C, n, dim, mg.FP64)
    ref = oracle.mg_cycle(g, gamma=gamma)
    assert np.abs(out - ref).max() <= 1e-11 * np.abs(ref).max()


@pytest.mark.parametrize("dim,n,lad,bound", [(3, 63, "H", 3e-2), (3, 63, "HSD", 3e-2), (3, 63, "BSD", 1e-1),
                                             (2, 255, "H", 3e-2), (3, 63, "S", 1e-5)])
def test_full_cycle_low_precision(oracle, dim, n, lad, bound):
    """A low-precision cycle approximates the FP64 cycle to about the storage precision
    of its finest levels (relative 2-norm)."""
    g = rnd(dim, n, 19, 2.0**14)
    with mg.Hierarchy(mg.make_params(dim, n, lad)) as h:
        L = h.nlev - 1
        fp = mg.ladder(lad, h.nlev)[-1]
        gb = write(h, L, mg.VEC_G, g, fp)
        h.run_stage(mg.STAGE_CYCLE, L)
        out = read(h, L, mg.VEC_C, n, dim, fp)
    ref = oracle.mg_cycle(gb)
    assert np.linalg.norm(out - ref) <= bound * np.linalg.norm(ref)


@pytest.mark.parametrize("prec", ALLP)
@pytest.mark.parametrize("n", [8, 4096, 1 << 20, 3 * (1 << 16) + 8])
def test_axpy(prec, n):
    """mg_axpy (Sec. 8.2, Fig. 6): y <- a x + y in the storage type (FP16/BF16 in pairs),
    against the FP64 result on the same rounded inputs."""
    import torch
    tdt = {mg.FP64: torch.float64, mg.FP32: torch.float32, mg.FP16: torch.float16, mg.BF16: torch.bfloat16}[prec]
    x = torch.from_numpy(I.uniform(31, (n,))).to(tdt).cuda()
    y = torch.from_numpy(I.uniform(32, (n,))).to(tdt).cuda()
    a = 0.75
    ref = a * x.double().cpu().numpy() + y.double().cpu().numpy()
    mg.axpy(prec, a, x, y)
    got = y.double().cpu().numpy()
    mag = np.abs(a * x.double().cpu().numpy()) + np.abs(ref)
    check_close(got, ref, mag, prec, "axpy")
