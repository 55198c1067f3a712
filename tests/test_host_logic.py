"""Host-side helpers of the CUDA library, compiled from its own headers with the
host compiler (no GPU): the tail's fixed-point division and the sweep
coefficients, checked against brute force and against the oracle.

The kernels evaluate a damped Jacobi sweep as c1 c + c2 W c + c3 g with
A = alpha (beta I - W) (alpha, beta from op_alpha / op_beta, the coefficients
from make_sweep_coef); two sweeps from zero as c3 (k2 g + c2 W g).  With
W v = beta v - A v / alpha these must equal the oracle's sweeps, for the
finite-difference and the Q1 operator (Sec. 4.2, Sec. 5)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2007_07539_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2007_07539_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"

PROGRAM = r'''
#include "mg_tail.h"
#include "mg_noalloc.h"
#include <cstdio>
#include <cstdlib>
#include <cstring>
int main(int argc, char** argv) {
    if (argc > 1 && !std::strcmp(argv[1], "magic")) {  // exact p / n for every tail point
        long long bad = 0;
        for (int n = 1; n < 1024; ++n) {
            const unsigned long long mn = mgi::tail_magic(n);
            for (unsigned p = 0; p < (1u << 15); ++p)
                if ((int)((p * mn) >> 40) != (int)(p / n)) ++bad;
        }
        std::printf("%lld\n", bad);
        return 0;
    }
    if (argc == 6 && !std::strcmp(argv[1], "coef")) {  // dim op n omega
        const int dim = std::atoi(argv[2]), op = std::atoi(argv[3]), n = std::atoi(argv[4]);
        const double omega = std::atof(argv[5]);
        const double alpha = mgi::op_alpha(op, dim, n);
        const mgi::SweepCoef c = mgi::make_sweep_coef(dim, op, omega, alpha);
        std::printf("%.17g %d", alpha, mgi::op_beta(op, dim));
        for (int k = 0; k < 6; ++k) std::printf(" %.17g", c.d[k]);
        for (int k = 0; k < 6; ++k) std::printf(" %.9g", (double)c.f[k]);
        std::printf("\n");
        return 0;
    }
    if (argc == 4 && !std::strcmp(argv[1], "geom")) {  // dim nmax: every level size up to nmax
        const int dim = std::atoi(argv[2]), nmax = std::atoi(argv[3]);
        for (int n = 1; n <= nmax; ++n) {
            const mgi::Geom g = mgi::make_geom(dim, n);
            std::printf("%d %d %lld %lld %lld\n", n, g.P, g.S, g.base, g.total);
        }
        return 0;
    }
    if (argc == 2 && !std::strcmp(argv[1], "ptrclass")) {  // type device current -> class, every combination
        for (int type = 0; type < 4; ++type)
            for (int dev = 0; dev < 3; ++dev)
                for (int cur = 0; cur < 3; ++cur)
                    std::printf("%d %d %d %d\n", type, dev, cur, mgi::noalloc_ptr_class(type, dev, cur));
        return 0;
    }
    return 2;
}
'''


@pytest.fixture(scope="module")
def hostprog(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None or not os.path.exists(os.path.join(CUDA_INC, "cuda.h")):
        pytest.skip("needs g++ and the CUDA headers")
    d = tmp_path_factory.mktemp("host")
    src, exe = d / "host.cpp", d / "host"
    src.write_text(PROGRAM)
    subprocess.check_call([gxx, "-std=c++17", "-O2", "-I", os.path.join(ROOT, "include"), "-I", CSRC,
                           "-I", CUDA_INC, str(src), "-o", str(exe)])
    return str(exe)


def run(exe, *args):
    return subprocess.check_output([exe, *map(str, args)], text=True).split()


def test_tail_division_is_exact(hostprog):
    """q = (p * ceil(2^40 / n)) >> 40 equals p / n for every n < 2^10 and p < 2^15
    (every point of a tail level)."""
    assert run(hostprog, "magic") == ["0"]


@pytest.mark.parametrize("dim,op,n", [(2, 0, 31), (3, 0, 15), (2, 1, 31), (3, 1, 15), (3, 0, 7)])
def test_sweep_coefficients_reproduce_the_oracle_sweeps(oracle, hostprog, dim, op, n):
    omega = 0.8
    out = run(hostprog, "coef", dim, op, n, omega)
    alpha, beta = float(out[0]), int(out[1])
    c1, c2, c3, k2, a4, a5 = map(float, out[2:8])
    f = list(map(float, out[8:14]))
    assert a4 == alpha and a5 == -beta * alpha
    # the FP32 coefficients are the FP64 ones rounded once
    for x, y in zip(f, (c1, c2, c3, k2, a4, a5)):
        assert x == float(np.float32(y)) or abs(x - y) <= 2.0**-23 * abs(y)
    c = I.uniform(3, (n,) * dim)
    g = I.uniform(4, (n,) * dim)

    def W(v):
        return beta * v - oracle.apply_A(v, op=op) / alpha

    ref = oracle.jacobi(g, c, omega, op=op)
    got = c1 * c + c2 * W(c) + c3 * g
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()
    ref2 = oracle.jacobi(g, oracle.jacobi(g, np.zeros_like(g), omega, op=op), omega, op=op)
    got2 = c3 * (k2 * g + c2 * W(g))
    assert np.abs(got2 - ref2).max() <= 1e-13 * np.abs(ref2).max()
    res = g + alpha * W(c) + a5 * c
    assert np.abs(res - oracle.residual(g, c, op=op)).max() <= 1e-12 * np.abs(g).max()


@pytest.mark.parametrize("dim", [2, 3])
def test_padded_layout(hostprog, dim):
    """The padded level layout: row pitch a multiple of 16 elements with room for the
    zero pad column, the interior start (0, 0[, 0]) 16-byte aligned for every storage
    type, and everything a stencil or a vector access of a row can touch inside the
    allocation: from row -1 of plane -1, x = -1 and a 16-byte vector before it, up to
    the last pitch element of row n of plane n and a 16-byte vector after it."""
    rows = [list(map(int, ln.split())) for ln in
            subprocess.check_output([hostprog, "geom", str(dim), "1100"], text=True).splitlines()]
    assert len(rows) == 1100
    for n, P, S, base, total in rows:
        assert P % 16 == 0 and P >= n + 1 and S == P * (n + 1)
        assert base % 16 == 0 and total % 128 == 0  # 16 elements: >= 32 bytes for every type
        lo = base - P - (S if dim == 3 else 0) - 1 - 8
        hi = base + n * P + (n * S if dim == 3 else 0) + (P - 1) + 8
        assert lo >= 0 and hi < total, (n, P, base, total)


def test_noalloc_pointer_checks(hostprog):
    """mg_residual_norms_noalloc's pointer check, on the fields of
    cudaPointerAttributes without a device: memory of the current device and
    managed memory pass; host or unregistered memory is rejected (class 1);
    another device's memory is rejected (class 2) -- the kernels could not
    read it without peer access, which a one-GPU test cannot set up."""
    rows = [list(map(int, ln.split())) for ln in
            subprocess.check_output([hostprog, "ptrclass"], text=True).splitlines()]
    assert len(rows) == 36
    for typ, dev, cur, cls in rows:
        want = 0 if typ == 3 else (1 if typ in (0, 1) else (0 if dev == cur else 2))
        assert cls == want, (typ, dev, cur, cls)
