"""Pins of the oracle's low-precision emulation (a diagnostic mode of the oracle).

The rounding into FP32 / FP16 / BF16 is checked against numpy's conversions and
against a brute-force nearest search over every finite value of the format,
built from its bit patterns.  The emulated cycle and refinement loop are checked
against what the arithmetic and the paper fix:

- an all-FP64 emulation with the 2^sigma residual scaling equals the plain
  oracle bit for bit (powers of two commute with every rounding);
- the unit roundoff and range of Table 1;
- FP16 multigrid without residual scaling stalls (Sec. 4.3), while FP32 and
  BF16, which have FP64-like range, do not;
- DSH_MG with an unscaled outer residual needs the rescale into its FP16 levels
  (Sec. 6);
- low-precision ladders take the FP64 iteration count (Sec. 8, Table 3).
"""
import os

import numpy as np
import pytest

from paper_2007_07539_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------- rounding
def _samples(seed, count, lo_log2, hi_log2):
    """Signed values log-uniform in [2^lo, 2^hi), with random FP64 significands."""
    rng = np.random.default_rng(seed)
    mag = np.exp2(rng.uniform(lo_log2, hi_log2, count))
    return np.where(rng.random(count) < 0.5, -mag, mag)


def _finite_table(fmt):
    """Every finite non-negative value of the format in increasing order (index =
    bit pattern), plus the first value past the largest finite one, which stands
    for the overflow to infinity (its pattern is the infinity's)."""
    if fmt == "fp16":
        pats = np.arange(0, 0x7C00, dtype=np.uint16)
        vals = pats.view(np.float16).astype(np.float64)
        return np.append(vals, 65536.0)
    pats = np.arange(0, 0x7F80, dtype=np.uint32) << np.uint32(16)  # bfloat16: the top half of a binary32
    vals = pats.view(np.float32).astype(np.float64)
    return np.append(vals, 2.0**128)


def _nearest_brute(table, x):
    """Nearest table value to |x|, ties to the even bit pattern; the top entry is infinity."""
    a = np.abs(x)
    hi = np.searchsorted(table, a, side="left").clip(1, len(table) - 1)
    lo = hi - 1
    dlo, dhi = a - table[lo], table[hi] - a  # exact: neighbours within a factor two of a
    pick = np.where(dlo < dhi, lo, np.where(dhi < dlo, hi, np.where(lo % 2 == 0, lo, hi)))
    out = table[pick].copy()
    out[pick == len(table) - 1] = np.inf
    out[a >= table[-1]] = np.inf
    return np.copysign(out, x)


def _ties(table, count, seed):
    """Exact midpoints of neighbouring values of the format (representable in FP64), and
    their FP64 neighbours."""
    rng = np.random.default_rng(seed)
    i = rng.integers(0, len(table) - 1, count)
    mid = (table[i] + table[i + 1]) / 2
    return np.concatenate([mid, np.nextafter(mid, 0), np.nextafter(mid, np.inf), -mid])


@pytest.mark.parametrize("fmt", ["fp16", "bf16"])
def test_round_matches_brute_force_nearest(oracle, fmt):
    """Round-to-nearest-even against a search over every finite value of the format:
    normals, subnormals, exact ties, overflow."""
    table = _finite_table(fmt)
    code = oracle.FP16 if fmt == "fp16" else oracle.BF16
    top = 17 if fmt == "fp16" else 129
    low = -27 if fmt == "fp16" else -136
    x = np.concatenate([_samples(1, 20000, low, top), _ties(table, 5000, 2), [0.0, -0.0]])
    got = oracle.round_to(code, x)
    want = _nearest_brute(table, x)
    bad = np.flatnonzero(~((got == want) | (np.isnan(got) & np.isnan(want))))
    assert bad.size == 0, (x[bad[:5]], got[bad[:5]], want[bad[:5]])
    assert np.array_equal(np.signbit(got[-2:]), [False, True])


def test_round_matches_numpy_conversions(oracle):
    """FP16 and FP32 against numpy's float64 -> float16 / float32 conversions."""
    x16 = np.concatenate([_samples(3, 20000, -27, 17), _ties(_finite_table("fp16"), 3000, 4)])
    with np.errstate(over="ignore"):
        assert np.array_equal(oracle.round_to(oracle.FP16, x16), x16.astype(np.float16).astype(np.float64))
        x32 = _samples(5, 20000, -152, 129)
        assert np.array_equal(oracle.round_to(oracle.FP32, x32), x32.astype(np.float32).astype(np.float64))
    x = _samples(6, 100, -40, 40)
    assert np.array_equal(oracle.round_to(oracle.FP64, x), x)


def test_round_table1_limits(oracle):
    """Table 1: largest value, least normal value and unit roundoff of FP16 and FP32,
    and the rounding at their edges."""
    rows = {}
    with open(os.path.join(GOLDEN, "fp_formats.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                name, rmin, rmax, ulog = line.split()
                rows[name] = (float(rmin), float(rmax), int(ulog))
    for name, code, p, emin in (("FP16", oracle.FP16, 11, -14), ("FP32", oracle.FP32, 24, -126)):
        def r(v):
            return float(oracle.round_to(code, v))
        rmin, rmax, ulog = rows[name]
        u = 2.0**ulog
        assert ulog == -p
        top = (2 - 2 * u) * 2.0 ** (1 - emin)  # the largest value: the printed maximum to 3 digits
        assert abs(top / rmax - 1) < 5e-3 and r(top) == top and r(rmax) <= top
        tiny = 2.0**emin
        assert abs(tiny / rmin - 1) < 5e-3 and r(tiny) == tiny
        assert r(1 + u) == 1.0  # a tie at the unit roundoff goes to the even 1
        assert r(1 + u + u * u) == 1 + 2 * u
        assert r(1 + 3 * u) == 1 + 4 * u  # a tie goes to the even neighbour above
        mid = (2 - u) * 2.0 ** (1 - emin)  # halfway from the maximum to the next power of two
        assert r(np.nextafter(mid, 0)) == top and np.isinf(r(mid)) and r(-mid) == -np.inf
        sub = 2.0 ** (emin - p + 1)  # least subnormal
        assert r(sub / 2) == 0.0 and r(sub * 0.75) == sub and r(1.5 * sub) == 2 * sub


# ----------------------------------------------------------------------------- cycles and solves
def _lad(oracle, name, nlev):
    """The per-level formats of the Table 2 variants, coarsest first: H all FP16,
    HSD FP16 on the two finest levels, FP64 base, FP32 between; DSH the reverse;
    S all FP32, B all BF16, D all FP64."""
    H, S, D, B = oracle.FP16, oracle.FP32, oracle.FP64, oracle.BF16
    if name in ("H", "S", "D", "B"):
        return [{"H": H, "S": S, "D": D, "B": B}[name]] * nlev
    fine, coarse = (H, D) if name == "HSD" else (D, H)
    return [coarse] + [S] * (nlev - 3) + [fine, fine]


@pytest.mark.parametrize("dim,n,gamma,op", [(2, 31, 1, 0), (3, 15, 1, 0), (3, 15, 2, 0), (3, 15, 1, 1), (2, 31, 2, 1)])
def test_all_fp64_emulation_is_the_plain_oracle(oracle, dim, n, gamma, op):
    """With every level FP64 and the residual scaled to 2^14 (sigma forced), the
    emulated refinement equals the plain FP64 oracle bit for bit: the scaling by a
    power of two and its compensation in the update are exact (both operators)."""
    b = I.random_rhs(dim, n, 5)
    nl = len(oracle.level_sizes(n))
    u0, i0, h0 = oracle.ir_solve(b, gamma=gamma, op=op)
    u1, i1, h1 = oracle.ir_solve(b, gamma=gamma, op=op, prec=[oracle.FP64] * nl, sigma_log2=14)
    assert i0["iters"] == i1["iters"]
    assert np.array_equal(u0, u1) and np.array_equal(h0, h1)
    c0 = oracle.mg_cycle(b, gamma=gamma, op=op)
    c1 = oracle.mg_cycle(b, gamma=gamma, op=op, prec=[oracle.FP64] * nl)
    assert np.array_equal(c0, c1)


def test_emulated_cycle_stores_level_formats(oracle):
    """One emulated cycle's result is a vector of the finest level's format and lies
    within a few units of that format's roundoff of the FP64 cycle."""
    dim, n = 3, 31
    g = I.random_rhs(dim, n, 6)
    nl = len(oracle.level_sizes(n))
    c64 = oracle.mg_cycle(g)
    for code, u in ((oracle.FP16, 2.0**-11), (oracle.BF16, 2.0**-8), (oracle.FP32, 2.0**-24)):
        c = oracle.mg_cycle(g * 2.0**10, prec=[code] * nl) / 2.0**10
        assert np.array_equal(oracle.round_to(code, c * 2.0**10), c * 2.0**10)
        err = np.linalg.norm(c - c64) / np.linalg.norm(c64)
        assert u / 8 < err < 50 * u, (code, err)


@pytest.mark.parametrize("dim,n", [(3, 31), (2, 127)])
def test_fp16_without_residual_scaling_stalls(oracle, dim, n):
    """Sec. 4.3: without the residual scaling the FP16 correction underflows once the
    residual is small, and the refinement stalls far above 1e-10; FP32 and BF16
    (FP32's exponent range) converge unscaled, so the range is the cause.  With the
    scaling FP16 converges."""
    b = I.random_rhs(dim, n, 2)
    nl = len(oracle.level_sizes(n))
    _, i64, _ = oracle.ir_solve(b)
    _, ih, _ = oracle.ir_solve(b, prec=_lad(oracle, "H", nl), scaling=0, max_iter=30)
    assert not ih["converged"] and ih["rel_res"] > 1e-6
    for name in ("S", "B"):
        _, inf, _ = oracle.ir_solve(b, prec=_lad(oracle, name, nl), scaling=0)
        assert inf["converged"] and inf["iters"] <= i64["iters"] + 1
    _, ihs, _ = oracle.ir_solve(b, prec=_lad(oracle, "H", nl))
    assert ihs["converged"]


@pytest.mark.parametrize("dim,n", [(3, 31), (2, 127)])
def test_dsh_unscaled_needs_the_fp16_rescale(oracle, dim, n):
    """Sec. 6 (DSH_MG): with an unscaled outer residual the restricted residual on the
    FP16 levels shrinks into FP16's subnormals; rescaling it by a power of two on
    restriction restores the FP64 iteration count."""
    b = I.random_rhs(dim, n, 2)
    nl = len(oracle.level_sizes(n))
    lad = [oracle.FP16] * (nl - 2) + [oracle.FP32, oracle.FP64]
    _, i64, _ = oracle.ir_solve(b)
    _, i0, _ = oracle.ir_solve(b, prec=lad, scaling=0, rescale16=0, max_iter=30)
    _, i1, _ = oracle.ir_solve(b, prec=lad, scaling=0, rescale16=1)
    assert not i0["converged"]
    assert i1["converged"] and i1["iters"] == i64["iters"]


@pytest.mark.parametrize("dim,n,rhs", [(3, 31, "random"), (2, 127, "random"), (3, 31, "manufactured")])
def test_low_precision_ladders_keep_the_fp64_iteration_count(oracle, dim, n, rhs):
    """Sec. 8 / Table 3: the multigrid preconditioner in FP16 (all levels, or with FP32 /
    FP64 coarse levels) needs as many refinement steps as in FP64; so does BF16."""
    b = I.random_rhs(dim, n, 2) if rhs == "random" else I.manufactured_rhs(dim, n)
    nl = len(oracle.level_sizes(n))
    _, i64, _ = oracle.ir_solve(b)
    for name in ("H", "HSD", "DSH", "B"):
        _, inf, _ = oracle.ir_solve(b, prec=_lad(oracle, name, nl))
        assert inf["converged"] and inf["rel_res_true"] <= 1e-10
        assert abs(inf["iters"] - i64["iters"]) <= 1, (name, inf["iters"], i64["iters"])


@pytest.mark.parametrize("dim,n,case", [(3, 31, "random"), (2, 127, "random"), (3, 31, "k1"), (2, 63, "k20")])
def test_paper_ladders_with_fp16_cg_base(oracle, dim, n, case):
    """Sec. 8, Table 3 settings: DSH_MG with the CG base solver in FP16 (level 0), FP16
    level 1, FP32 level 2, FP64 above, and H_MG / HSD_MG with the CG base, need as many
    refinement steps as D_MG; the manufactured cases start from u0 uniform in [0, 1)."""
    if case == "random":
        b, u0 = I.random_rhs(dim, n, 2), None
    else:
        b, u0 = I.manufactured_rhs(dim, n, int(case[1:])), I.random_guess(dim, n, 5)
    nl = len(oracle.level_sizes(n))
    H, S, D = oracle.FP16, oracle.FP32, oracle.FP64
    _, i64, _ = oracle.ir_solve(b, u0)
    for lad in ([H, H, S] + [D] * (nl - 3), [H] * nl, [D, D, S] + [H] * (nl - 3)):
        _, inf, _ = oracle.ir_solve(b, u0, prec=lad, base_solver=1)
        assert inf["converged"] and inf["rel_res_true"] <= 1e-10
        assert inf["iters"] <= i64["iters"] + 1, (lad, inf["iters"], i64["iters"])


def test_fp16_finest_level_caps_a_fast_cycle(oracle):
    """When the FP64 cycle contracts much faster than an FP16 correction is accurate
    (Q1 operator, W(2,2)-cycle: 5 steps to 1e-10), the ladders with FP16 finest levels
    need more steps, while DSH_MG (FP64 finest levels, FP16 only on the coarsest)
    keeps the FP64 count: the finest levels' precision bounds the per-step gain."""
    dim, n = 3, 31
    b = I.manufactured_load(dim, n, 1)
    nl = len(oracle.level_sizes(n))
    H, S, D = oracle.FP16, oracle.FP32, oracle.FP64
    kw = dict(op=1, gamma=2)
    _, i64, _ = oracle.ir_solve(b, **kw)
    its = {}
    for name, lad in (("H", [H] * nl), ("HSD", [D, D, S] + [H] * (nl - 3)), ("DSH", [H, H, S] + [D] * (nl - 3))):
        _, inf, _ = oracle.ir_solve(b, prec=lad, **kw)
        assert inf["converged"]
        its[name] = inf["iters"]
    assert i64["iters"] <= 6
    assert its["DSH"] == i64["iters"]
    assert its["H"] >= i64["iters"] + 2 and its["HSD"] >= i64["iters"] + 2, (its, i64["iters"])


def test_emulated_fp16_cg_is_a_low_precision_cg(oracle):
    """The base solver's CG with its vectors stored in FP16: every stored value is an
    FP16 value, and the solution meets the relative 1e-4 test up to FP16's resolution."""
    g = oracle.round_to(oracle.FP16, I.uniform(24, (3, 3, 3)) * 2.0**13)
    c, steps = oracle.cg_solve(g, tol=1e-4, fmt=oracle.FP16)
    assert np.array_equal(oracle.round_to(oracle.FP16, c), c)
    ref = oracle.coarse_solve(g)
    assert 1 <= steps <= 27
    assert np.linalg.norm(c - ref) <= 4e-3 * np.linalg.norm(ref)


@pytest.mark.parametrize("dim,n,case", [(3, 31, "random"), (2, 127, "random"), (2, 255, "fd_k1"), (3, 31, "q1_k1")])
def test_scale_ahead_keeps_the_iteration_count(oracle, dim, n, case):
    """The scale of Alg. 2's residual scaling taken as the power of two from the previous step's
    max-norm, with the scaled residual truncated to FP32 before the cast: a different
    scale (the histories differ) but the same number of refinement steps, for FP16,
    HSD and BF16 ladders."""
    kw = dict(op=1) if case.startswith("q1") else {}
    if case == "random":
        b = I.random_rhs(dim, n, 2)
    elif case == "fd_k1":
        b = I.manufactured_rhs(dim, n, 1)
    else:
        b = I.manufactured_load(dim, n, 1)
    nl = len(oracle.level_sizes(n))
    changed = False
    for name in ("H", "HSD", "B"):
        lad = _lad(oracle, name, nl)
        _, i0, h0 = oracle.ir_solve(b, prec=lad, **kw)
        _, i1, h1 = oracle.ir_solve(b, prec=lad, scale_ahead=1, **kw)
        assert i0["converged"] and i1["converged"]
        assert i1["iters"] == i0["iters"], (name, i0["iters"], i1["iters"])
        changed |= not np.array_equal(h0, h1)
    assert changed


def test_fp16_iteration_count_is_grid_independent(oracle):
    """Sec. 8: the refinement needs a bounded number of steps as the grid is refined;
    with every level in FP16 the counts stay within one step from 15^3 to 63^3 and
    from 31^2 to 511^2."""
    for dim, ns in ((3, (15, 31, 63)), (2, (31, 63, 127, 255, 511))):
        its = []
        for n in ns:
            nl = len(oracle.level_sizes(n))
            _, inf, _ = oracle.ir_solve(I.random_rhs(dim, n, 11), prec=[oracle.FP16] * nl, nthreads=4)
            assert inf["converged"]
            its.append(inf["iters"])
        assert max(its) - min(its) <= 1 and max(its) <= 20, (dim, its)


def test_emulation_parameters_checked(oracle):
    with pytest.raises(ValueError):
        oracle.make_params(3, 15, prec=[oracle.FP16] * 2)


# ----------------------------------------------------------------------------- the kernels' one-rounding check
@pytest.mark.parametrize("prec_name", ["fp16", "bf16"])
def test_one_rounding_check_separates_fp32_arithmetic_from_an_extra_rounding(oracle, prec_name):
    """The GPU kernel tests hold FP16/BF16 outputs to one rounding of the exact result
    (check_rounded).  A Jacobi sweep computed in FP32 (numpy) and rounded once passes;
    the same sweep with one intermediate value rounded to the storage format fails."""
    from _helpers import check_rounded, to_storage
    from paper_2007_07539_gb300 import mg
    prec = mg.FP16 if prec_name == "fp16" else mg.BF16
    dim, n, om = 3, 15, 0.8
    h = 1.0 / (n + 1)
    dinv = h * h / 6
    cs, gs = (2.0**14 * dinv, 2.0**13) if prec == mg.FP16 else (1.0, 1.0 / dinv)
    _, c = to_storage(I.uniform(1, (n,) * dim) * cs, prec)
    _, g = to_storage(I.uniform(2, (n,) * dim) * gs, prec)
    ref = oracle.jacobi(g, c, om)
    mag = np.abs(c) + om * dinv * (np.abs(g) + oracle.apply_A(c, absmode=True))
    c32, g32 = c.astype(np.float32), g.astype(np.float32)
    p = np.pad(c32, 1)
    nb = (p[1:-1, 1:-1, :-2] + p[1:-1, 1:-1, 2:] + p[1:-1, :-2, 1:-1] + p[1:-1, 2:, 1:-1]
          + p[:-2, 1:-1, 1:-1] + p[2:, 1:-1, 1:-1])
    part = np.float32(om * dinv) * g32 + np.float32(om / 6) * nb
    once = to_storage((np.float32(1 - om) * c32 + part).astype(np.float64), prec)[1]
    check_rounded(oracle, once, ref, mag, prec, "fp32 sweep")
    twice = to_storage((1 - om) * c + to_storage(part.astype(np.float64), prec)[1], prec)[1]
    with pytest.raises(AssertionError):
        check_rounded(oracle, twice, ref, mag, prec, "extra rounding")


# ----------------------------------------------------------------------------- scale-ahead truncation
def _trunc_f32_numpy(x):
    """Truncation toward zero to binary32 built from numpy's round-to-nearest
    conversion: a result larger in magnitude than x steps one float32 spacing back
    toward zero; results below the least normal 2^-126 flush to zero (FTZ, as
    the truncation from the bit pattern does), |x| >= 2^128 gives infinity."""
    x = np.asarray(x, dtype=np.float64)
    with np.errstate(over="ignore"):
        f = x.astype(np.float32)
    up = np.abs(f.astype(np.float64)) > np.abs(x)
    f = np.where(up, np.nextafter(f, np.float32(0)), f).astype(np.float64)
    f = np.where(np.abs(f) < 2.0**-126, np.copysign(0.0, x), f)
    f = np.where(np.abs(x) >= 2.0**128, np.copysign(np.inf, x), f)
    return np.where(np.isnan(x), x, f)


def test_trunc_f32_matches_numpy_round_toward_zero(oracle):
    """The FP32 truncation of the emulated scale-ahead cast (reading R21) against
    numpy: random values over binary32's whole range and beyond, exact binary32
    values (unchanged), exact midpoints between neighbouring binary32 values (the
    lower magnitude wins, unlike round-to-nearest) and their FP64 neighbours,
    the underflow edge 2^-126 and the overflow edge 2^128."""
    rng = np.random.default_rng(11)
    f32 = _samples(12, 4000, -125, 127).astype(np.float32)
    nxt = np.nextafter(f32, np.float32(np.inf) * np.sign(f32))
    mid = (f32.astype(np.float64) + nxt.astype(np.float64)) / 2  # exact in FP64
    edges = [2.0**-126, np.nextafter(2.0**-126, 0), 2.0**-126 * (1 + 2.0**-30), 2.0**-149, 2.0**-127,
             2.0**128, np.nextafter(2.0**128, 0), 2.0**128 - 2.0**103, np.nextafter(2.0**128 - 2.0**103, 0),
             float(np.finfo(np.float32).max), 65520.0, np.nextafter(65520.0, 0), 1.0, 1 + 2.0**-24, 0.0]
    x = np.concatenate([_samples(13, 20000, -140, 130), f32.astype(np.float64), mid,
                        np.nextafter(mid, 0), np.nextafter(mid, np.inf), edges, -np.asarray(edges),
                        rng.uniform(-1, 1, 1000)])
    got = oracle.trunc_f32(x)
    want = _trunc_f32_numpy(x)
    bad = np.flatnonzero(~((got == want) & (np.signbit(got) == np.signbit(want))))
    assert bad.size == 0, (x[bad[:5]], got[bad[:5]], want[bad[:5]])
    # every midpoint goes to the neighbour of smaller magnitude
    assert np.array_equal(oracle.trunc_f32(mid), np.where(np.abs(f32) < np.abs(nxt), f32, nxt).astype(np.float64))
    assert oracle.trunc_f32(np.array([np.inf, -np.inf])).tolist() == [np.inf, -np.inf]
    assert np.isnan(oracle.trunc_f32(np.array([np.nan])))[0]


def test_scale_ahead_cast_overflow_flag(oracle):
    """The fallback flag of the emulated scale-ahead cast: for FP16 it is set exactly
    when a truncated value rounds to infinity in FP16 (numpy's conversion), i.e. at
    65520 and above; BF16 and FP32 flag values from 3.0e38, below their overflow
    thresholds.  The cast values are round(trunc(r inv)) in every case."""
    rng = np.random.default_rng(21)
    inv = 2.0**14
    base = rng.uniform(-1, 1, 4096)
    for t in (65504.0, np.nextafter(65520.0, 0), 65519.99, 65520.0, 65535.0, 70000.0):
        for sign in (1.0, -1.0):
            r = base.copy()
            r[17] = sign * t / inv
            g, over = oracle.scale_ahead_cast(oracle.FP16, r, inv)
            tr = _trunc_f32_numpy(r * inv)
            with np.errstate(over="ignore"):
                g16 = tr.astype(np.float16).astype(np.float64)
            assert over == bool(np.isinf(g16).any()), (t, over)
            assert np.array_equal(g, g16)
    g, over = oracle.scale_ahead_cast(oracle.FP16, base, inv)
    assert not over and np.max(np.abs(g)) <= 2.0**14
    for fmt in (oracle.BF16, oracle.FP32):
        for t, want in ((2.9e38, False), (np.nextafter(3.0e38, 0), False), (3.0e38 * (1 + 2.0**-20), True), (3.5e38, True)):
            r = base.copy()
            r[5] = t / 2.0**100
            g, over = oracle.scale_ahead_cast(fmt, r, 2.0**100)
            assert over == want, (fmt, t)
            assert np.array_equal(g, oracle.round_to(fmt, _trunc_f32_numpy(r * 2.0**100)))
