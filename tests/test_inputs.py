"""The seeded input recipes (host logic, no solver arithmetic): grid sizes of the
paper's shapes, the batched and serving workloads, initial guesses.

Sizes follow the reading that every draw snaps to an n with n + 1 = 2^a or
3 * 2^a (the paper's grids of 2^a + 1 and 3 * 2^a + 1 nodes, Sec. 8.1), so that
each coarsens by n -> (n - 1) / 2 down to a 2- or 3-point base grid."""
import math

import numpy as np

from paper_2007_07539_gb300 import inputs as I


def test_snapped_size_sets():
    """The batched sizes are {31, 47, ..., 255}; the serving sizes 63..383 (3D) and
    255..4095 (2D)."""
    assert I.snapped_sizes(31, 255) == [31, 47, 63, 95, 127, 191, 255]
    assert I.snapped_sizes(63, 383) == [63, 95, 127, 191, 255, 383]
    assert I.snapped_sizes(255, 4095) == [255, 383, 511, 767, 1023, 1535, 2047, 3071, 4095]


def test_snapped_sizes_coarsen_to_a_small_base(oracle):
    for n in I.snapped_sizes(3, 8191):
        m = n + 1
        assert m & (m - 1) == 0 or (m % 3 == 0 and (m // 3) & (m // 3 - 1) == 0)
        assert oracle.level_sizes(n)[0] in (2, 3), n


def test_snap_is_nearest_in_log_space():
    sizes = I.snapped_sizes(31, 255)
    assert I.snap(40, sizes) == 47 and I.snap(38, sizes) == 31
    for x in np.exp(np.linspace(math.log(31), math.log(255), 50)):
        s = I.snap(float(x), sizes)
        assert all(abs(math.log(s / x)) <= abs(math.log(t / x)) for t in sizes)


def test_batched_workload():
    """64 instances, right-hand-side seeds 1000 + i, every size present, about 172M
    unknowns, and the same list on every call."""
    w = I.batched_workload()
    assert len(w) == 64 and [s for _, s in w] == list(range(1000, 1064))
    assert sorted({n for n, _ in w}) == I.snapped_sizes(31, 255)
    assert sum(n ** 3 for n, _ in w) == 172365440
    assert I.batched_workload() == w


def test_serving_workload():
    """Poisson arrivals at the given rate, about half 2D and half 3D, sizes from the
    snapped sets, per-request seeds 5000 + i."""
    rate = 100.0
    s = I.serving_workload(count=512, rate_per_s=rate)
    t = np.array([r["arrival_s"] for r in s])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    assert abs(gaps.mean() * rate - 1) < 0.15          # exponential gaps of mean 1 / rate
    assert abs(np.std(gaps) / gaps.mean() - 1) < 0.2   # coefficient of variation 1
    d2 = sum(r["dim"] == 2 for r in s)
    assert 200 < d2 < 312
    s2, s3 = set(I.snapped_sizes(255, 4095)), set(I.snapped_sizes(63, 383))
    assert all(r["n"] in (s2 if r["dim"] == 2 else s3) for r in s)
    assert [r["seed"] for r in s] == list(range(5000, 5512))


def test_initial_guess_and_rhs_ranges():
    g = I.random_guess(3, 15, 5)
    assert g.shape == (15, 15, 15) and g.min() >= 0.0 and g.max() < 1.0
    b = I.random_rhs(2, 31, 2)
    assert b.min() >= -1.0 and b.max() < 1.0 and abs(b.mean()) < 0.1
    assert np.array_equal(I.random_rhs(2, 31, 2), b) and not np.array_equal(I.random_rhs(2, 31, 3), b)
