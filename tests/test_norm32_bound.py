"""The FP32 sum of squares of the scale-ahead IR update, restated in numpy (no GPU).

With FP16 / BF16 / FP32 finest levels the fused update of Alg. 2's solution and
residual updates also forms the next step's g = cast(trunc_FP32(r 2^k)) (reading
R21) and takes ||r||_2^2 as 2^-2k times an FP32 sum of the squares of those
truncated values: each thread sums the squares of its points (about a hundred
at the benchmark size) in FP32, the per-thread sums are added in FP64.  Here
that arithmetic is replayed on residuals of the oracle's emulated FP16 solves
to pin the bound the stopping test relies on (reading R11): relative error
below 1e-5, so a stopping decision can differ from the FP64 norm's only when
||r|| lies within 1e-5 of the tolerance."""
import numpy as np
import pytest

from paper_2007_07539_gb300 import inputs as I


def fp32_norm(oracle, r, per_thread):
    """sqrt of the FP64 sum over threads of sequential FP32 sums of squares of
    trunc_FP32(r 2^k), 2^k the power of two that puts ||r||_inf just below 2^14."""
    _, e = np.frexp(np.abs(r).max())
    k = 14 - int(e)
    g = oracle.trunc_f32(r * 2.0**k).astype(np.float32)
    sq = g * g
    pad = (-sq.size) % per_thread
    sq = np.concatenate([sq, np.zeros(pad, np.float32)]).reshape(-1, per_thread)
    thread_sums = np.cumsum(sq, axis=1, dtype=np.float32)[:, -1]  # sequential FP32 per thread
    return np.sqrt(np.sum(thread_sums.astype(np.float64))) * 2.0**-k


@pytest.mark.parametrize("dim,n,steps", [(3, 31, 1), (3, 31, 6), (2, 127, 4), (3, 63, 9)])
def test_fp32_sum_of_squares_is_within_1e5_of_the_fp64_norm(oracle, dim, n, steps):
    b = I.random_rhs(dim, n, 3)
    nl = len(oracle.level_sizes(n))
    u, info, _ = oracle.ir_solve(b, prec=[oracle.FP16] * nl, max_iter=steps, tol=0.0)
    r = oracle.residual(b, u).reshape(-1)
    ref = np.linalg.norm(r)
    for per_thread in (4, 108, 512):
        got = fp32_norm(oracle, r, per_thread)
        assert abs(got - ref) <= 1e-5 * ref, (per_thread, got / ref - 1)
    # and the typical error at the benchmark's ~108 points per thread is far smaller
    assert abs(fp32_norm(oracle, r, 108) - ref) <= 2e-6 * ref
