"""Pins of the FP64 CPU oracle against facts that do not come from the oracle itself.

Each test checks one oracle routine against a closed form, an independent
textbook construction (scipy Kronecker-product matrices), a library routine
(numpy dense solve), an exact Fourier (two-grid) analysis, a printed table of
the paper, or an invariant.  They are chosen so that a dropped term, a wrong
sign, index, weight or level spacing, or a missing scale compensation in the
refinement loop fails at least one of them.
"""
import math
import os
from decimal import Decimal

import numpy as np
import pytest
import scipy.sparse as sp

from paper_2007_07539_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------- helpers
def mode(dim, n, ms):
    """prod_a sin(m_a pi x_a) with ms = (m_x, m_y[, m_z]); array indexed [z, y, x]."""
    x = I.grid_coords(n)
    f = [np.sin(m * math.pi * x) for m in ms]
    if dim == 2:
        return np.multiply.outer(f[1], f[0])
    return np.multiply.outer(np.multiply.outer(f[2], f[1]), f[0])


def lap1d(n):
    h = 1.0 / (n + 1)
    return sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1]) / h**2


def lap(dim, n):
    """Textbook Kronecker-sum FDM Laplacian, C-order flattening (x fastest)."""
    T, Id = lap1d(n), sp.identity(n)
    if dim == 2:
        return (sp.kron(Id, T) + sp.kron(T, Id)).tocsr()
    return (sp.kron(sp.kron(Id, Id), T) + sp.kron(sp.kron(Id, T), Id) + sp.kron(sp.kron(T, Id), Id)).tocsr()


def fw1d(nf):
    nc = (nf - 1) // 2
    R = sp.lil_matrix((nc, nf))
    for c in range(nc):
        R[c, 2 * c], R[c, 2 * c + 1], R[c, 2 * c + 2] = 0.25, 0.5, 0.25
    return R.tocsr()


def fw(dim, nf):
    R = fw1d(nf)
    return sp.kron(R, R) if dim == 2 else sp.kron(sp.kron(R, R), R)


# ----------------------------------------------------------------------------- Table 1
def test_table1_fp_constants():
    """Table 1 (Sec. 1): range and unit roundoff of FP16/FP32/FP64 as printed."""
    rows = {}
    with open(os.path.join(GOLDEN, "fp_formats.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                name, rmin, rmax, ulog = line.split()
                rows[name] = (Decimal(rmin), Decimal(rmax), int(ulog))
    for name, dt in (("FP16", np.float16), ("FP32", np.float32), ("FP64", np.float64)):
        fi = np.finfo(dt)
        rmin, rmax, ulog = rows[name]
        # printed to three digits: compare in decimal (1.80e308 overflows a double)
        assert abs(Decimal(float(fi.tiny)) / rmin - 1) < Decimal("5e-3")
        assert abs(Decimal(float(fi.max)) / rmax - 1) < Decimal("5e-3")
        assert float(fi.eps) / 2 == 2.0**ulog
    assert float(np.finfo(np.float16).tiny) == 2.0**-14  # Sec. 4.3: 2^-14 ~ 6.10e-5


def test_splitmix64_reference_vector():
    with open(os.path.join(GOLDEN, "splitmix64.txt")) as f:
        vals = [int(l, 16) for l in f if l.startswith("0x")]
    assert [int(v) for v in I.splitmix64(0, 3)] == vals
    u = I.uniform(42, (1000,))
    assert u.min() >= -1.0 and u.max() < 1.0 and abs(u.mean()) < 0.1


# ----------------------------------------------------------------------------- operator A
@pytest.mark.parametrize("dim,n,ms", [(2, 7, (1, 1)), (2, 16, (3, 5)), (2, 31, (30, 2)),
                                      (3, 7, (1, 2, 3)), (3, 12, (11, 1, 5))])
def test_A_eigenvector_closed_form(oracle, dim, n, ms):
    """Sampled sines are exact eigenvectors: lambda = (4/h^2) sum_a sin^2(m_a pi h / 2)."""
    h = 1.0 / (n + 1)
    v = mode(dim, n, ms)
    lam = sum(4.0 / h**2 * math.sin(m * math.pi * h / 2) ** 2 for m in ms)
    Av = oracle.apply_A(v)
    assert np.abs(Av - lam * v).max() <= 1e-13 * lam * np.abs(v).max()


@pytest.mark.parametrize("dim,n", [(2, 9), (2, 16), (3, 6), (3, 9)])
def test_A_matches_kronecker_sum(oracle, dim, n):
    v = I.uniform(5, (n,) * dim)
    ref = (lap(dim, n) @ v.ravel()).reshape(v.shape)
    assert np.abs(oracle.apply_A(v) - ref).max() <= 1e-12 * np.abs(ref).max()
    absref = (abs(lap(dim, n)) @ np.abs(v).ravel()).reshape(v.shape)
    assert np.abs(oracle.apply_A(v, absmode=True) - absref).max() <= 1e-12 * absref.max()


@pytest.mark.parametrize("dim,n", [(2, 15), (3, 7)])
def test_A_symmetric(oracle, dim, n):
    x, y = I.uniform(1, (n,) * dim), I.uniform(2, (n,) * dim)
    a, b = np.vdot(oracle.apply_A(x), y), np.vdot(x, oracle.apply_A(y))
    assert abs(a - b) <= 1e-12 * abs(a)


def test_residual(oracle):
    b, u = I.uniform(3, (9, 9, 9)), I.uniform(4, (9, 9, 9))
    ref = b - (lap(3, 9) @ u.ravel()).reshape(u.shape)
    assert np.abs(oracle.residual(b, u) - ref).max() <= 1e-12 * np.abs(ref).max()


# ----------------------------------------------------------------------------- smoother
@pytest.mark.parametrize("dim,n,ms,omega", [(2, 15, (1, 1), 0.8), (2, 15, (14, 9), 2 / 3),
                                            (3, 7, (7, 1, 4), 0.8)])
def test_jacobi_eigen_factor(oracle, dim, n, ms, omega):
    """On an eigenmode with g = 0 the damped Jacobi factor is 1 - omega (2/d) sum sin^2(m pi h/2)."""
    h = 1.0 / (n + 1)
    v = mode(dim, n, ms)
    fac = 1.0 - omega * (2.0 / dim) * sum(math.sin(m * math.pi * h / 2) ** 2 for m in ms)
    out = oracle.jacobi(np.zeros_like(v), v, omega)
    assert np.abs(out - fac * v).max() <= 1e-13


def test_jacobi_matrix_form(oracle):
    n, dim, omega = 11, 3, 0.8
    g, v = I.uniform(6, (n,) * dim), I.uniform(7, (n,) * dim)
    h = 1.0 / (n + 1)
    ref = v.ravel() + omega * h * h / (2 * dim) * (g.ravel() - lap(dim, n) @ v.ravel())
    assert np.abs(oracle.jacobi(g, v, omega).ravel() - ref).max() <= 1e-12 * np.abs(ref).max()


# ----------------------------------------------------------------------------- transfers
@pytest.mark.parametrize("dim,nf,ms", [(2, 15, (1, 1)), (2, 31, (3, 7)), (3, 15, (2, 5, 1))])
def test_restriction_closed_form(oracle, dim, nf, ms):
    """Full weighting of fine mode m (m <= nc) is prod_a cos^2(m_a pi h/2) times coarse mode m."""
    h = 1.0 / (nf + 1)
    nc = (nf - 1) // 2
    fac = np.prod([math.cos(m * math.pi * h / 2) ** 2 for m in ms])
    out = oracle.restrict(mode(dim, nf, ms))
    assert np.abs(out - fac * mode(dim, nc, ms)).max() <= 1e-14


@pytest.mark.parametrize("dim,nf", [(2, 15), (3, 7), (3, 15)])
def test_restriction_matches_kronecker(oracle, dim, nf):
    r = I.uniform(8, (nf,) * dim)
    nc = (nf - 1) // 2
    ref = (fw(dim, nf) @ r.ravel()).reshape((nc,) * dim)
    assert np.abs(oracle.restrict(r) - ref).max() <= 1e-14


@pytest.mark.parametrize("dim,nc,ms", [(2, 7, (1, 1)), (2, 15, (5, 2)), (3, 7, (1, 3, 6))])
def test_prolongation_closed_form(oracle, dim, nc, ms):
    """Linear interpolation of a coarse mode: fine points on coarse nodes keep the value,
    points between two coarse nodes get the mode times cos(m pi h) along that axis."""
    nf = 2 * nc + 1
    h = 1.0 / (nf + 1)
    idx = np.arange(nf)
    facs = [np.where(idx % 2 == 1, 1.0, math.cos(m * math.pi * h)) for m in ms]
    fac = np.multiply.outer(facs[1], facs[0]) if dim == 2 else \
        np.multiply.outer(np.multiply.outer(facs[2], facs[1]), facs[0])
    out = oracle.prolong_add(mode(dim, nc, ms), np.zeros((nf,) * dim))
    assert np.abs(out - fac * mode(dim, nf, ms)).max() <= 1e-14


@pytest.mark.parametrize("dim,nc", [(2, 7), (3, 3), (3, 7)])
def test_restriction_is_scaled_transpose_of_prolongation(oracle, dim, nc):
    """R = 2^-d P^T: 2^d <R x, y>_coarse = <x, P y>_fine."""
    nf = 2 * nc + 1
    x, y = I.uniform(9, (nf,) * dim), I.uniform(10, (nc,) * dim)
    lhs = 2**dim * np.vdot(oracle.restrict(x), y)
    rhs = np.vdot(x, oracle.prolong_add(y, np.zeros((nf,) * dim)))
    assert abs(lhs - rhs) <= 1e-13 * abs(rhs)
    base = I.uniform(11, (nf,) * dim)
    assert np.allclose(oracle.prolong_add(y, base) - base, oracle.prolong_add(y, np.zeros_like(base)),
                       rtol=0, atol=1e-15)


# ----------------------------------------------------------------------------- base solve
@pytest.mark.parametrize("dim,n", [(2, 2), (2, 3), (2, 5), (3, 2), (3, 3), (3, 5), (2, 7)])
def test_coarse_solve_matches_numpy(oracle, dim, n):
    g = I.uniform(12, (n,) * dim)
    ref = np.linalg.solve(lap(dim, n).toarray(), g.ravel()).reshape(g.shape)
    assert np.abs(oracle.coarse_solve(g) - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("dim,n", [(3, 3), (2, 7), (3, 5), (2, 3)])
def test_cg_terminates_after_the_distinct_eigenvalues(oracle, dim, n):
    """CG (Sec. 6 base solver) reaches the exact solution in as many steps as A has
    distinct eigenvalues (g has a component on each).  The eigenvalues are the sums of
    the 1-D ones, (4/h^2) sum_a sin^2(m_a pi h / 2); on the 3^3 grid they are
    (4/h^2)(3/2 + k sqrt(2)/4), k = -3..3: seven values."""
    g = I.uniform(21, (n,) * dim)
    h = 1.0 / (n + 1)
    s1 = np.sin(np.arange(1, n + 1) * math.pi * h / 2) ** 2
    grids = np.meshgrid(*([s1] * dim), indexing="ij")
    lam = 4.0 / h**2 * sum(grids)
    distinct = len(np.unique(np.round(lam.ravel() / lam.max(), 10)))
    if (dim, n) == (3, 3):
        assert distinct == 7
    c, steps = oracle.cg_solve(g, tol=1e-12)
    ref = np.linalg.solve(lap(dim, n).toarray(), g.ravel()).reshape(g.shape)
    assert steps <= distinct
    assert np.abs(c - ref).max() <= 1e-12 * np.abs(ref).max()
    _, early = oracle.cg_solve(g, tol=1e-12, maxit=distinct - 1)
    assert early == distinct - 1 and steps == distinct  # no earlier step reaches 1e-12


def test_cg_first_step_is_steepest_descent(oracle):
    """One CG step from c = 0 is the exact line search along g: c = (g.g / g.Ag) g."""
    g = I.uniform(22, (7, 7, 7))
    c, steps = oracle.cg_solve(g, tol=0.0, maxit=1)
    Ag = lap(3, 7) @ g.ravel()
    assert steps == 1
    assert np.abs(c - (g.ravel() @ g.ravel()) / (g.ravel() @ Ag) * g).max() <= 1e-14 * np.abs(c).max()


def test_cg_stopping_rule(oracle):
    """CG stops at the first step whose residual is at most tol ||g||_2 (Sec. 6: the
    base solver's residual test, relative here)."""
    g = I.uniform(23, (15, 15, 15))
    A = lap(3, 15)
    c, steps = oracle.cg_solve(g, tol=1e-4)
    rel = np.linalg.norm(g.ravel() - A @ c.ravel()) / np.linalg.norm(g)
    assert 1 < steps < g.size and rel <= 1.0001e-4
    cp, _ = oracle.cg_solve(g, tol=1e-4, maxit=steps - 1)
    assert np.linalg.norm(g.ravel() - A @ cp.ravel()) / np.linalg.norm(g) > 1e-4
    _, none = oracle.cg_solve(np.zeros_like(g))
    assert none == 0


def test_level_sizes(oracle):
    assert oracle.level_sizes(127) == [3, 7, 15, 31, 63, 127]        # 6 levels, coarsest 3x3
    assert oracle.level_sizes(511) == [3, 7, 15, 31, 63, 127, 255, 511]
    assert oracle.level_sizes(383) == [2, 5, 11, 23, 47, 95, 191, 383]
    assert oracle.level_sizes(255, 3) == [63, 127, 255]


# ----------------------------------------------------------------------------- two-grid Fourier
def twogrid_prediction(dim, nf, ks, nu1, nu2, omega):
    """Exact two-grid error propagation of fine mode ks (sine basis, Dirichlet): the
    operator couples the 2^d harmonics (m_a or nf+1-m_a per axis).  Returns a list of
    (mode multi-index, coefficient)."""
    h = 1.0 / (nf + 1)
    nc = (nf - 1) // 2
    base = [min(k, nf + 1 - k) for k in ks]
    lam = lambda km: sum(4 / h**2 * math.sin(k * math.pi * h / 2) ** 2 for k in km)
    s = lambda km: 1.0 - omega * h * h / (2 * dim) * lam(km)
    if any(m == nc + 1 for m in base):
        return [(tuple(ks), s(ks) ** (nu1 + nu2))]
    members = []
    for bits in range(2**dim):
        km = tuple(base[a] if not (bits >> a) & 1 else nf + 1 - base[a] for a in range(dim))
        members.append(km)
    rho = lambda km: np.prod([math.cos(base[a] * math.pi * h / 2) ** 2 if km[a] == base[a]
                              else -math.sin(base[a] * math.pi * h / 2) ** 2 for a in range(dim)])
    lam_c = sum(math.sin(m * math.pi * h) ** 2 / h**2 for m in base)
    S = np.diag([s(k) for k in members])
    r = np.array([rho(k) for k in members])
    L = np.array([lam(k) for k in members])
    E = np.linalg.matrix_power(S, nu2) @ (np.eye(len(members)) - np.outer(r, r * L) / lam_c) \
        @ np.linalg.matrix_power(S, nu1)
    j = members.index(tuple(ks))
    return [(members[i], E[i, j]) for i in range(len(members))]


@pytest.mark.parametrize("dim,nf,ks,nu", [(2, 15, (1, 1), 2), (2, 15, (3, 13), 2), (2, 31, (16, 5), 2),
                                          (2, 31, (20, 29), 3), (3, 7, (1, 2, 3), 2),
                                          (3, 15, (14, 3, 9), 2), (3, 15, (8, 2, 2), 1)])
def test_twogrid_matches_fourier_analysis(oracle, dim, nf, ks, nu):
    """Alg. 1 on two levels (exact coarse solve): the error propagation of a single sine
    mode equals the closed-form two-grid symbol.  Pins the smoother, residual,
    restriction, coarse operator (re-discretised at 2h), base solve, prolongation and
    the order of the steps at once."""
    omega = 0.8
    e = mode(dim, nf, ks)
    c = oracle.mg_cycle(oracle.apply_A(e), levels=2, nu1=nu, nu2=nu, omega=omega)
    pred = sum(coef * mode(dim, nf, km) for km, coef in twogrid_prediction(dim, nf, ks, nu, nu, omega))
    assert np.abs((e - c) - pred).max() <= 1e-11


def test_wcycle_equals_vcycle_on_two_levels(oracle):
    """With an exact base solve a second coarse visit changes nothing."""
    g = I.uniform(13, (15, 15, 15))
    v = oracle.mg_cycle(g, levels=2, gamma=1)
    w = oracle.mg_cycle(g, levels=2, gamma=2)
    assert np.abs(v - w).max() <= 1e-13 * np.abs(v).max()
    v3 = oracle.mg_cycle(g, levels=3, gamma=1)
    w3 = oracle.mg_cycle(g, levels=3, gamma=2)
    assert np.abs(v3 - w3).max() > 1e-6 * np.abs(v3).max()


def contraction(oracle, dim, n, gamma=1, its=10):
    e = I.uniform(3, (n,) * dim)
    r = 1.0
    for _ in range(its):
        e2 = e - oracle.mg_cycle(oracle.apply_A(e), gamma=gamma)
        r = np.linalg.norm(e2) / np.linalg.norm(e)
        e = e2 / np.linalg.norm(e2)
    return r


@pytest.mark.parametrize("dim,ns,bound", [(2, (31, 63, 127), 0.2), (3, (15, 31), 0.3)])
def test_vcycle_contraction_h_independent(oracle, dim, ns, bound):
    """Multigrid's defining property (Sec. 1): a grid-independent error reduction per cycle."""
    rs = [contraction(oracle, dim, n) for n in ns]
    assert max(rs) < bound
    assert (max(rs) - min(rs)) / max(rs) < 0.10
    assert contraction(oracle, dim, ns[0], gamma=2) < rs[0]


# ----------------------------------------------------------------------------- IR (Alg. 2)
@pytest.mark.parametrize("dim,scaling", [(2, 0), (2, 1), (3, 0), (3, 1), (3, 2)])
def test_ir_tiny_grid_matches_dense_solve(oracle, dim, scaling):
    """7x7 and 7^3 grids: IR with one MG cycle per step reaches numpy's dense solution."""
    n = 7
    b = I.random_rhs(dim, n, 21)
    ref = np.linalg.solve(lap(dim, n).toarray(), b.ravel()).reshape(b.shape)
    u, info, hist = oracle.ir_solve(b, scaling=scaling)
    assert info["converged"] and info["rel_res_true"] <= 1e-10
    assert np.linalg.norm(u - ref) <= 1e-9 * np.linalg.norm(ref)
    assert np.all(np.diff(hist) < 0)


@pytest.mark.parametrize("dim,n", [(2, 31), (2, 63), (3, 15), (3, 31)])
def test_ir_manufactured_discrete_solution_exact(oracle, dim, n):
    """For f = d pi^2 prod sin(pi x) the discrete solution is known in closed form:
    u_h = (d pi^2 / lambda_1) prod sin(pi x), lambda_1 = (4d/h^2) sin^2(pi h/2).  Its error
    against the continuous solution is the O(h^2) constant d pi^2/lambda_1 - 1."""
    h = 1.0 / (n + 1)
    lam1 = 4 * dim / h**2 * math.sin(math.pi * h / 2) ** 2
    ustar = I.sine_product(dim, n)
    uh = dim * math.pi**2 / lam1 * ustar
    u, info, _ = oracle.ir_solve(I.manufactured_rhs(dim, n), scaling=1)
    assert info["converged"]
    assert np.abs(u - uh).max() <= 1e-9 * np.abs(uh).max()
    err = np.abs(u - ustar).max() / np.abs(ustar).max()
    assert err == pytest.approx(dim * math.pi**2 / lam1 - 1.0, rel=1e-4)
    assert err == pytest.approx(math.pi**2 * h * h / 12, rel=2e-2)


def test_ir_scaling_invariance(oracle):
    """Alg. 2's residual scaling and updates: the scale alpha is compensated, so in FP64 the iterates do not
    depend on the scaling choice beyond rounding (a missing compensation breaks this)."""
    b = I.random_rhs(3, 31, 22)
    u0, i0, h0 = oracle.ir_solve(b, scaling=0)
    u1, i1, h1 = oracle.ir_solve(b, scaling=1)
    u2, i2, h2 = oracle.ir_solve(b, scaling=2)
    assert i0["iters"] == i1["iters"] == i2["iters"]
    for u in (u1, u2):
        assert np.linalg.norm(u - u0) <= 1e-12 * np.linalg.norm(u0)
    assert np.allclose(h0, h1, rtol=1e-9) and np.allclose(h0, h2, rtol=1e-9)


def test_ir_nonzero_initial_guess_and_absolute_tolerance(oracle):
    """The paper's setting (Sec. 6, 8.1): random initial guess in [0, 1), absolute 1e-9 test."""
    n = 31
    b = I.manufactured_rhs(2, n)
    u0 = I.random_guess(2, n, 23)
    u, info, hist = oracle.ir_solve(b, u0, tol_mode=1, tol=1e-9, scaling=1)
    assert info["converged"]
    assert np.linalg.norm(oracle.residual(b, u)) < 1e-9
    assert hist[0] > 1.0


def test_ir_iteration_count_behaviour(oracle):
    """Table 3 reports at most ~15 IR iterations with one cycle per step; the FDM V(2,2)
    variant stays within that and is grid-independent."""
    its = [oracle.ir_solve(I.random_rhs(2, n, 24))[1]["iters"] for n in (31, 63, 127)]
    assert max(its) <= 15 and max(its) - min(its) <= 2
    its3 = [oracle.ir_solve(I.random_rhs(3, n, 25))[1]["iters"] for n in (15, 31)]
    assert max(its3) <= 20 and max(its3) - min(its3) <= 2


def test_ir_max_iter_reports_not_converged(oracle):
    b = I.random_rhs(2, 31, 26)
    _, info, hist = oracle.ir_solve(b, max_iter=2)
    assert info["status"] == 1 and not info["converged"] and info["iters"] == 2 and len(hist) == 3


# ----------------------------------------------------------------------------- Q1 finite elements (op 1)
def q1_assembled(dim, n):
    """The Q1 stiffness matrix assembled element by element, each element matrix
    integrated by 2^d-point Gauss quadrature of grad(phi_i) . grad(phi_j) over the
    bilinear / trilinear shape functions of the reference cell mapped to an h-cube;
    Dirichlet nodes dropped; divided by h^d.  A route independent of the 1-D
    product form the oracle uses."""
    h = 1.0 / (n + 1)
    gp = np.array([-1.0, 1.0]) / math.sqrt(3.0)  # Gauss points on [-1, 1], weights 1
    corners = [tuple((c >> a) & 1 for a in range(dim)) for c in range(2 ** dim)]
    Ke = np.zeros((2 ** dim, 2 ** dim))
    for q in np.array(np.meshgrid(*([gp] * dim), indexing="ij")).reshape(dim, -1).T:
        grads = []
        for c in corners:  # shape function prod_a (1 + s_a xi_a)/2, s = +-1
            s = [2 * ca - 1 for ca in c]
            g = []
            for a in range(dim):
                t = s[a] / 2.0
                for b in range(dim):
                    if b != a:
                        t *= (1 + s[b] * q[b]) / 2.0
                g.append(t * 2.0 / h)  # d xi / d x = 2 / h
            grads.append(g)
        G = np.array(grads)
        Ke += (G @ G.T) * (h / 2.0) ** dim  # Jacobian of the map
    N = n ** dim
    A = np.zeros((N, N))
    for e in np.ndindex(*([n + 1] * dim)):  # element e spans nodes e .. e+1 (node 0 = boundary)
        idx = []
        for c in corners:
            node = [e[a] + c[a] - 1 for a in range(dim)]  # interior index, -1 / n are boundary
            idx.append(None if any(v < 0 or v >= n for v in node) else
                       sum(node[a] * n ** a for a in range(dim)))
        for i, p in enumerate(idx):
            if p is None:
                continue
            for j, q in enumerate(idx):
                if q is not None:
                    A[p, q] += Ke[i, j]
    return A / h ** dim


def q1_symbol(dim, n, ms):
    """Eigenvalue of the h^-d-scaled Q1 operator on the sampled sine mode ms:
    h^-d sum_a k(t_a) prod_{b != a} m(t_b), k(t) = (2 - 2 cos t)/h, m(t) = h (4 + 2 cos t)/6,
    t = m pi h (the Fourier symbols of the 1-D stiffness and mass stencils)."""
    h = 1.0 / (n + 1)
    t = [m * math.pi * h for m in ms]
    k = [(2 - 2 * math.cos(x)) / h for x in t]
    mm = [h * (4 + 2 * math.cos(x)) / 6 for x in t]
    lam = 0.0
    for a in range(dim):
        v = k[a]
        for b in range(dim):
            if b != a:
                v *= mm[b]
        lam += v
    return lam / h ** dim


@pytest.mark.parametrize("dim,n", [(2, 5), (2, 8), (3, 3), (3, 5)])
def test_q1_matches_quadrature_assembly(oracle, dim, n):
    A = q1_assembled(dim, n)
    v = I.uniform(71, (n,) * dim)
    ref = (A @ v.ravel()).reshape(v.shape)
    assert np.abs(oracle.apply_A(v, op=1) - ref).max() <= 1e-12 * np.abs(ref).max()
    absref = (np.abs(A) @ np.abs(v).ravel()).reshape(v.shape)
    assert np.abs(oracle.apply_A(v, absmode=True, op=1) - absref).max() <= 1e-12 * absref.max()
    g = I.uniform(72, (n,) * dim)
    ref = np.linalg.solve(A, g.ravel()).reshape(g.shape)
    assert np.abs(oracle.coarse_solve(g, op=1) - ref).max() <= 1e-11 * np.abs(ref).max()


def test_q1_stencil_weights(oracle):
    """The interior rows: 2D h^-2 [8/3 centre, -1/3 x 8]; 3D h^-2 [8/3 centre, 0 faces,
    -1/6 edges, -1/12 corners] (row sums zero)."""
    for dim, n in ((2, 5), (3, 5)):
        h = 1.0 / (n + 1)
        e = np.zeros((n,) * dim)
        e[(2,) * dim] = 1.0
        col = oracle.apply_A(e, op=1) * h * h
        c = (2,) * dim
        assert col[c] == pytest.approx(8 / 3, rel=1e-14)
        for off in np.ndindex(*([3] * dim)):
            o = tuple(x - 1 for x in off)
            nz = sum(1 for x in o if x)
            if nz == 0:
                continue
            want = -1 / 3 if dim == 2 else {1: 0.0, 2: -1 / 6, 3: -1 / 12}[nz]
            assert col[tuple(ci + oi for ci, oi in zip(c, o))] == pytest.approx(want, abs=1e-14)
        assert abs(col.sum()) <= 1e-13


@pytest.mark.parametrize("dim,n,ms", [(2, 7, (1, 1)), (2, 16, (3, 5)), (3, 7, (1, 2, 3)), (3, 12, (11, 1, 5))])
def test_q1_eigenvector_closed_form(oracle, dim, n, ms):
    v = mode(dim, n, ms)
    lam = q1_symbol(dim, n, ms)
    assert np.abs(oracle.apply_A(v, op=1) - lam * v).max() <= 1e-13 * lam * np.abs(v).max()


@pytest.mark.parametrize("dim,nc", [(2, 3), (2, 7), (3, 3)])
def test_q1_coarse_operator_is_galerkin(oracle, dim, nc):
    """With the h^-d scaling, full weighting R and interpolation P = 2^d R^T, the
    re-discretised coarse operator equals R A_h P exactly."""
    nf = 2 * nc + 1

    def dense(n):
        N = n ** dim
        M = np.zeros((N, N))
        for q in range(N):
            e = np.zeros(N)
            e[q] = 1.0
            M[:, q] = oracle.apply_A(e.reshape((n,) * dim), op=1).ravel()
        return M
    R = fw(dim, nf).toarray()
    RAP = R @ dense(nf) @ (2 ** dim * R.T)
    A2h = dense(nc)
    assert np.abs(RAP - A2h).max() <= 1e-12 * np.abs(A2h).max()


def test_q1_jacobi_eigen_factor(oracle):
    """Damped Jacobi with D = 8/3 h^-2 (both dimensions) multiplies a mode by 1 - omega lambda / D."""
    for dim, n, ms in ((2, 15, (3, 7)), (3, 7, (7, 1, 4))):
        h = 1.0 / (n + 1)
        v = mode(dim, n, ms)
        fac = 1.0 - 0.8 * q1_symbol(dim, n, ms) / (8.0 / 3.0 / h ** 2)
        assert np.abs(oracle.jacobi(np.zeros_like(v), v, 0.8, op=1) - fac * v).max() <= 1e-13


@pytest.mark.parametrize("dim,n,k", [(2, 31, 1), (2, 63, 3), (3, 15, 1), (3, 31, 2)])
def test_q1_ir_manufactured_discrete_solution_exact(oracle, dim, n, k):
    """The Q1 load vector of f = d (k pi)^2 prod sin(k pi x) is a multiple of the
    sampled mode, so the discrete solution is b / lambda in closed form."""
    b = I.manufactured_load(dim, n, k)
    lam = q1_symbol(dim, n, (k,) * dim)
    uh = b / lam
    u, info, _ = oracle.ir_solve(b, op=1)
    assert info["converged"] and info["rel_res_true"] <= 1e-10
    assert np.abs(u - uh).max() <= 1e-9 * np.abs(uh).max()
    ustar = I.sine_product(dim, n, k)
    err = np.abs(u - ustar).max() / np.abs(ustar).max()
    assert err <= (k * math.pi / (n + 1)) ** 2  # O(h^2) nodal error


def test_q1_ir_iteration_count_grid_independent(oracle):
    its = [oracle.ir_solve(I.random_rhs(3, n, 73), op=1)[1]["iters"] for n in (15, 31)]
    assert max(its) <= 25 and max(its) - min(its) <= 2
    its2 = [oracle.ir_solve(I.random_rhs(2, n, 74), op=1)[1]["iters"] for n in (31, 63, 127)]
    assert max(its2) <= 25 and max(its2) - min(its2) <= 2
