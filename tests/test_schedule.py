"""The library's schedule of one IR step, read through mg_describe_cycle (host
only, no GPU), against the structure of Alg. 1 and Alg. 2:

- the scale-and-cast of Alg. 2's residual scaling first (unless g is the FP64 residual);
- per visit of level l >= 1: nu1 pre-smoothing sweeps (from zero on a first
  visit), one residual-restriction, gamma visits of level l - 1, one
  prolongation, nu2 post-smoothing sweeps; level l is visited gamma^(L - l)
  times, the base level gamma^L times;
- the coarse tail runs the same recursion on its levels;
- a restriction into an FP16 level from a non-FP16 level is followed by the
  rescale (Sec. 6), only there and only with rescale16 = 1."""
from collections import Counter

import pytest

from paper_2007_07539_gb300 import mg

# record kinds (include/mg.h, mg_describe_cycle)
KERNEL, COARSE, ZERO, TAIL, RESCALE = 0, 1, 3, 7, 8
T_SWEEP, T_RESID, T_RESTRICT, T_PROLONG, T_COARSE, T_ZERO, T_LOAD, T_STORE = range(100, 108)
K_SWEEP, K_UPDATE, K_SCALE, K_PROLONG = 0, 1, 2, 3
M_JACOBI, M_ZERO2, M_ZERO1, M_RESTRICT = 0, 1, 2, 3
M_FEM = 16


def describe(dim, n, lad, **kw):
    return mg.describe_cycle(mg.make_params(dim, n, lad, **kw))


def counts(recs):
    """Per level: pre/post sweeps by mode, restrictions, prolongations, base solves,
    whether they ran as level kernels or as tail stages."""
    c = Counter()
    for r in recs:
        k, l, m = r["kind"], r["level"], r["mode"] & ~M_FEM
        if k == KERNEL and r["kernel"] == K_SWEEP:
            c[("restrict" if m == M_RESTRICT else ("sweep", m), l)] += 1
        elif k == KERNEL and r["kernel"] == K_PROLONG:
            c[("prolong", l)] += 1
        elif k == COARSE or k == T_COARSE:
            c[("base", l)] += 1
        elif k == T_SWEEP:
            c[(("sweep", m), l)] += 1
        elif k == T_RESTRICT:
            c[("restrict", l)] += 1
        elif k == T_PROLONG:
            c[("prolong", l)] += 1
        elif k in (ZERO, T_ZERO):
            c[("zero", l)] += 1
    return c


def expected(nlev, gamma, nu1, nu2):
    L = nlev - 1
    e = Counter()
    for l in range(1, L + 1):
        visits = gamma ** (L - l)
        first = 1 if l == L else gamma ** (L - l - 1)
        if nu1 >= 2:
            e[(("sweep", M_ZERO2), l)] += first
            e[(("sweep", M_JACOBI), l)] += first * (nu1 - 2)
        elif nu1 == 1:
            e[(("sweep", M_ZERO1), l)] += first
        else:
            e[("zero", l)] += first
        e[(("sweep", M_JACOBI), l)] += (visits - first) * nu1 + visits * nu2
        e[("restrict", l)] += visits
        e[("prolong", l)] += visits
    e[("base", 0)] += gamma ** L
    return +e


@pytest.mark.parametrize("dim,n,lad,gamma,nu,no_tail", [
    (3, 31, "H", 1, 2, 0), (3, 31, "H", 2, 2, 0), (3, 63, "HSD", 2, 2, 1), (2, 127, "D", 1, 2, 0),
    (2, 255, "H", 2, 2, 0), (3, 47, "S", 1, 3, 1), (3, 31, "D", 1, 1, 1), (2, 63, "H", 2, 0, 0),
    (3, 255, "H", 1, 2, 0), (2, 511, "DSH", 2, 3, 0)])
def test_cycle_follows_alg1(dim, n, lad, gamma, nu, no_tail):
    nlev = len(mg.level_count(n))
    recs = describe(dim, n, lad, gamma=gamma, nu1=nu, nu2=nu, no_tail=no_tail)
    assert counts(recs) == expected(nlev, gamma, nu, nu)
    # Alg. 2's residual scaling first; no IR update inside the cycle
    assert recs[0]["kind"] == KERNEL and recs[0]["kernel"] == K_SCALE and recs[0]["level"] == nlev - 1
    assert not any(r["kind"] == KERNEL and r["kernel"] == K_UPDATE for r in recs)


@pytest.mark.parametrize("gamma", [1, 2])
def test_one_pass_presmoothing_replaces_first_visits(gamma):
    """fuse_pre = 1 (3D, nu1 = 2): each first visit runs the two sweeps from zero and the
    residual-restriction as one pass (mode 4); later visits keep Jacobi sweeps and a
    separate residual-restriction.  Everything else is unchanged."""
    dim, n, nu = 3, 63, 2
    nlev = len(mg.level_count(n))
    L = nlev - 1
    recs = describe(dim, n, "H", gamma=gamma, fuse_pre=1, no_tail=1)
    c = Counter()
    for r in recs:
        if r["kind"] == KERNEL and r["kernel"] == K_SWEEP:
            c[(r["mode"], r["level"])] += 1
    for l in range(1, L + 1):
        visits = gamma ** (L - l)
        first = 1 if l == L else gamma ** (L - l - 1)
        assert c[(4, l)] == first
        assert c[(M_ZERO2, l)] == 0
        assert c[(M_RESTRICT, l)] == visits - first
        assert c[(M_JACOBI, l)] == (visits - first) * nu + visits * nu


def test_fp64_finest_without_scaling_reads_the_residual():
    """D_MG with no scaling: the finest g is the FP64 residual itself, no scale-and-cast."""
    recs = describe(3, 31, "D", scaling=0)
    assert not any(r["kind"] == KERNEL and r["kernel"] == K_SCALE for r in recs)
    assert describe(3, 31, "D")[0]["kernel"] == K_SCALE


@pytest.mark.parametrize("dim,n,lad", [(3, 255, "H"), (3, 127, "HSD"), (2, 511, "H"), (2, 1023, "S"), (3, 63, "D")])
def test_coarse_tail_boundary(dim, n, lad):
    """The tail holds the levels up to the largest with at most 8192 points (one CTA);
    it loads g and stores c of its top level once per visit."""
    sizes = mg.level_count(n)
    recs = describe(dim, n, lad)
    tails = [r for r in recs if r["kind"] == TAIL]
    assert len(tails) == 1
    t = tails[0]["level"]
    assert sizes[t] ** dim <= 8192 and (t + 1 == len(sizes) or sizes[t + 1] ** dim > 8192)
    assert not any(r["kind"] == KERNEL and r["level"] <= t for r in recs)
    assert sum(r["kind"] == T_LOAD for r in recs) == 1 and sum(r["kind"] == T_STORE for r in recs) == 1
    assert not any(r["kind"] == TAIL for r in describe(dim, n, lad, no_tail=1))


def test_wcycle_tail_reloads_the_correction():
    """Later W-cycle visits of the tail's top level start from the current c: the tail
    loads g every visit and c on every visit after the first."""
    dim, n, gamma = 3, 63, 2
    sizes = mg.level_count(n)
    recs = describe(dim, n, "H", gamma=gamma)
    t = next(r["level"] for r in recs if r["kind"] == TAIL)
    visits = gamma ** (len(sizes) - 1 - t)
    first = gamma ** (len(sizes) - 2 - t)
    assert sum(r["kind"] == TAIL for r in recs) == visits
    assert sum(r["kind"] == T_LOAD for r in recs) == visits + (visits - first)
    assert sum(r["kind"] == T_STORE for r in recs) == visits


@pytest.mark.parametrize("lad,rescaled", [
    ([mg.FP16, mg.FP16, mg.FP32, mg.FP64, mg.FP64], [1]),   # DSH: FP32 level 2 -> FP16 level 1
    ([mg.FP16] * 3 + [mg.FP32, mg.FP64], [2]),
    ("H", []), ("HSD", []), ("D", []),
    ([mg.BF16, mg.BF16, mg.FP32, mg.FP64, mg.FP64], [])])     # BF16 has FP32's range: no rescale
def test_rescale_only_into_fp16_from_wider_levels(lad, rescaled):
    dim, n = 3, 63
    nlev = len(mg.level_count(n))
    if isinstance(lad, str):
        lad = mg.ladder(lad, nlev)
    recs = describe(dim, n, lad, no_tail=1)
    got = [r["level"] for r in recs if r["kind"] == RESCALE]
    assert got == rescaled
    for i, r in enumerate(recs):  # each rescale right after the restriction into its level
        if r["kind"] == RESCALE:
            prev = recs[i - 1]
            assert prev["kernel"] == K_SWEEP and prev["mode"] == M_RESTRICT and prev["level"] == r["level"] + 1
            assert prev["prec_c"] == mg.FP32  # the restriction writes an FP32 scratch first
    assert not any(r["kind"] == RESCALE for r in describe(dim, n, lad, no_tail=1, rescale16=0))


def test_precisions_follow_the_ladder():
    dim, n = 3, 63
    nlev = len(mg.level_count(n))
    lad = mg.ladder("HSD", nlev)
    for r in describe(dim, n, lad, no_tail=1):
        if r["kind"] in (KERNEL, COARSE):
            assert r["prec"] == lad[r["level"]]
            if r["kind"] == KERNEL and r["kernel"] == K_SWEEP and r["mode"] == M_RESTRICT:
                assert r["prec_c"] == lad[r["level"] - 1]


def test_q1_operator_marks_the_stencil_kernels():
    recs = describe(3, 31, "H", op=1, fuse_pre=0)
    sweeps = [r for r in recs if r["kind"] == KERNEL and r["kernel"] == K_SWEEP]
    assert sweeps and all(r["mode"] & M_FEM for r in sweeps)
    assert not any(r["mode"] & M_FEM for r in describe(3, 31, "H") if r["kind"] == KERNEL)


def test_cg_base_solver_in_the_schedule():
    recs = describe(3, 31, "H", base_solver=1, no_tail=1)
    base = [r for r in recs if r["kind"] == COARSE]
    assert len(base) == 1 and base[0]["mode"] == 1
    tail_base = [r for r in describe(3, 31, "H", base_solver=1) if r["kind"] == T_COARSE]
    assert len(tail_base) == 1 and tail_base[0]["mode"] == 1


def test_invalid_parameters_are_rejected():
    p = mg.make_params(3, 31, "H")
    p.gamma = 3
    with pytest.raises(mg.MGError):
        mg.describe_cycle(p)
