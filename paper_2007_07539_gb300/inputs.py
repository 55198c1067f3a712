"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This module holds only input recipes: right-hand sides, initial guesses and
workload draws.  It contains none of the solver's arithmetic and imports
neither the CUDA library nor the oracle.

Recipes (all FP64 on the host, so the oracle and the GPU see identical bits):

* ``uniform(seed, shape)``: value i (C order) is the i-th output of SplitMix64
  started from state ``seed`` (Steele, Lea & Flood, OOPSLA 2014; the
  generator of ``java.util.SplittableRandom``), mapped to [-1, 1) as
  ``(z >> 11) * 2**-53 * 2 - 1``.
* ``manufactured_rhs(dim, n, k)``: f = dim (k pi)^2 prod_a sin(k pi x_a), the
  right-hand side of -Laplace(u) = f for u = prod_a sin(k pi x_a) (Sec. 5,
  Eq. 2 of the paper and its 3-D analogue), sampled at the interior grid
  points x = (i+1) h, h = 1/(n+1).
* ``manufactured_load(dim, n, k)``: the same f integrated against the Q1
  finite-element basis (the load vector of the paper's FEM discretisation,
  Sec. 5), divided by h^d, in closed form.
* ``random_guess``: initial guesses in [0, 1), the paper's choice (Sec. 8.1).
* batched and serving workloads: log-uniform grid sizes snapped to sizes
  n with n+1 in {2^a, 3*2^a}, the shapes of the paper's grids (Sec. 8.1).
"""
from __future__ import annotations

import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Outputs offset .. offset+count-1 of SplitMix64 started from state ``seed``."""
    with np.errstate(over="ignore"):
        idx = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform(seed: int, shape, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """Seeded uniform values in [lo, hi), FP64, C order."""
    shape = tuple(shape)
    cnt = int(np.prod(shape)) if shape else 1
    out = np.empty(cnt, dtype=np.float64)
    step = 1 << 24
    for s in range(0, cnt, step):
        z = splitmix64(seed, min(step, cnt - s), s)
        v = (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
        out[s:s + len(v)] = lo + (hi - lo) * v
    return out.reshape(shape)


def grid_coords(n: int) -> np.ndarray:
    """Interior node coordinates (i+1)/(n+1), i = 0..n-1."""
    return (np.arange(n, dtype=np.float64) + 1.0) / (n + 1)


def sine_product(dim: int, n: int, k: int = 1) -> np.ndarray:
    """prod_a sin(k pi x_a) at the interior nodes, shape (n,)*dim, x fastest."""
    s = np.sin(k * math.pi * grid_coords(n))
    if dim == 2:
        return np.ascontiguousarray(np.multiply.outer(s, s))
    return np.ascontiguousarray(np.multiply.outer(np.multiply.outer(s, s), s))


def manufactured_rhs(dim: int, n: int, k: int = 1) -> np.ndarray:
    """f = -Laplace(u) for u = prod_a sin(k pi x_a): f = dim (k pi)^2 u."""
    return dim * (k * math.pi) ** 2 * sine_product(dim, n, k)


def manufactured_load(dim: int, n: int, k: int = 1) -> np.ndarray:
    """The finite-element load vector of the same f, h^-d times the integral of
    f against each node's Q1 basis function (a product of 1-D hats), in closed
    form: a hat of half-width h centred at x_i integrates sin(k pi x) to
    sin(k pi x_i) * 2 (1 - cos t) / ((k pi)^2 h) with t = k pi h, so
    b = dim (k pi)^2 prod_a sin(k pi x_a) (2 (1 - cos t) / t^2)^dim."""
    t = k * math.pi / (n + 1)
    return manufactured_rhs(dim, n, k) * (2.0 * (1.0 - math.cos(t)) / t ** 2) ** dim


def random_rhs(dim: int, n: int, seed: int) -> np.ndarray:
    """f ~ U[-1, 1) per node from ``seed`` (SplitMix64)."""
    return uniform(seed, (n,) * dim)


def random_guess(dim: int, n: int, seed: int) -> np.ndarray:
    """Initial guess with values in [0, 1), the paper's choice (Sec. 8.1)."""
    return uniform(seed, (n,) * dim, 0.0, 1.0)


def snapped_sizes(lo: int, hi: int) -> list[int]:
    """Sizes n in [lo, hi] with n+1 = 2^a or 3*2^a (odd n, so they coarsen)."""
    out = set()
    a = 1
    while 2 ** a <= hi + 1:
        for m in (2 ** a, 3 * 2 ** (a - 1)):
            if lo <= m - 1 <= hi and (m - 1) % 2 == 1:
                out.add(m - 1)
        a += 1
    return sorted(out)


def snap(n_raw: float, sizes: list[int]) -> int:
    """Nearest allowed size in log space."""
    return min(sizes, key=lambda s: abs(math.log(s) - math.log(n_raw)))


def log_uniform_sizes(seed: int, count: int, lo: int, hi: int) -> list[int]:
    """``count`` sizes drawn log-uniformly in [lo, hi] and snapped."""
    sizes = snapped_sizes(lo, hi)
    u = uniform(seed, (count,), 0.0, 1.0)
    return [snap(math.exp(math.log(lo) + x * (math.log(hi) - math.log(lo))), sizes) for x in u]


def batched_workload(count: int = 64, seed: int = 7, lo: int = 31, hi: int = 255):
    """Independent 3-D instances: list of (n, rhs seed); rhs seeds 1000 + i."""
    return [(n, 1000 + i) for i, n in enumerate(log_uniform_sizes(seed, count, lo, hi))]


def serving_workload(count: int = 512, seed: int = 11, rate_per_s: float = 100.0,
                     lo2: int = 255, hi2: int = 4095, lo3: int = 63, hi3: int = 383):
    """Request stream: list of dicts (arrival_s, dim, n, seed).  Poisson arrivals
    (exponential gaps at ``rate_per_s``), half 2-D and half 3-D, log-uniform sizes."""
    u = uniform(seed, (count, 3), 0.0, 1.0)
    t = 0.0
    out = []
    s2, s3 = snapped_sizes(lo2, hi2), snapped_sizes(lo3, hi3)
    for i in range(count):
        t += -math.log(1.0 - u[i, 0]) / rate_per_s
        dim = 2 if u[i, 1] < 0.5 else 3
        lo, hi, sz = (lo2, hi2, s2) if dim == 2 else (lo3, hi3, s3)
        n = snap(math.exp(math.log(lo) + u[i, 2] * (math.log(hi) - math.log(lo))), sz)
        out.append(dict(arrival_s=t, dim=dim, n=n, seed=5000 + i))
    return out
