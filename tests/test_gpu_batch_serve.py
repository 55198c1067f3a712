"""Batched solves (mg_solve_batch) and the serving engine (mg_submit / mg_poll):
every instance gives the same result alone and in the mix (bitwise: the
kernels use fixed-order reductions), and the engine admits requests by memory
budget and in-flight slots while others run."""
import time

import numpy as np
import pytest

from paper_2007_07539_gb300 import inputs as I
from paper_2007_07539_gb300 import mg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def alone(dim, n, lad, b):
    import torch
    with mg.Hierarchy(mg.make_params(dim, n, lad, zero_guess=1)) as h:
        u = torch.zeros(b.shape, dtype=torch.float64, device="cuda")
        res = h.solve(torch.from_numpy(b).cuda(), u)
        return u.cpu().numpy(), res


def test_batch_equals_alone(oracle):
    import torch
    work = [(n, s) for n, s in I.batched_workload(count=8, seed=7, lo=31, hi=127)]
    hs, bs, us, refs = [], [], [], []
    for n, seed in work:
        b = I.random_rhs(3, n, seed)
        refs.append(alone(3, n, "H", b))
        hs.append(mg.Hierarchy(mg.make_params(3, n, "H", zero_guess=1)))
        bs.append(torch.from_numpy(b).cuda())
        us.append(torch.zeros_like(bs[-1]))
    res = mg.solve_batch(hs, bs, us)
    for (u_ref, r_ref), u, r, (n, seed) in zip(refs, us, res, work):
        assert r["merged"] == 1  # level-synchronous merged launches
        assert r["status"] == 0 and r["rel_res_true"] <= 1e-10
        assert np.array_equal(u.cpu().numpy(), u_ref), n
        assert r["iters"] == r_ref["iters"]
        uo, info, _ = oracle.ir_solve(I.random_rhs(3, n, seed))
        assert np.linalg.norm(u.cpu().numpy() - uo) <= 1e-6 * np.linalg.norm(uo)
    for h in hs:
        h.close()


@pytest.mark.parametrize("mix", ["ladders", "dims"])
def test_batch_mixed_equals_alone(mix):
    """Instances with different ladders (merged launches split by launch shape) and a
    2D/3D mix (the concurrent path) give their alone results bit for bit; a second call
    reuses the cached plan."""
    import torch
    if mix == "ladders":
        specs = [(3, 63, "H", 11), (3, 95, "HSD", 12), (3, 47, "S", 13), (3, 127, "H", 14), (3, 31, "BSD", 15)]
    else:
        specs = [(3, 63, "H", 21), (2, 255, "H", 22), (3, 47, "H", 23)]
    refs = [alone(d, n, lad, I.random_rhs(d, n, sd)) for d, n, lad, sd in specs]
    hs = [mg.Hierarchy(mg.make_params(d, n, lad, zero_guess=1)) for d, n, lad, sd in specs]
    bs = [torch.from_numpy(I.random_rhs(d, n, sd)).cuda() for d, n, lad, sd in specs]
    for rep in range(2):
        us = [torch.zeros_like(b) for b in bs]
        res = mg.solve_batch(hs, bs, us)
        for (u_ref, r_ref), u, r in zip(refs, us, res):
            assert r["merged"] == (1 if mix == "ladders" else 0)
            assert r["status"] == 0 and r["iters"] == r_ref["iters"]
            assert np.array_equal(u.cpu().numpy(), u_ref)
    for h in hs:
        h.close()


def test_serving_results_equal_alone_and_overlap(oracle):
    """Requests of different sizes submitted while others run: all complete, each equals
    its alone solve bitwise and the FP64 oracle's solution (Alg. 2) within 1e-6 with at
    most 2 more IR steps, and their device work overlaps (the mix finishes faster than
    the sum of the alone times)."""
    import torch
    specs = [(2, 255, 1), (3, 63, 2), (3, 95, 3), (2, 511, 4), (3, 47, 5), (2, 383, 6), (3, 127, 7), (3, 63, 8)]
    refs = [alone(d, n, "HS", I.random_rhs(d, n, s)) for d, n, s in specs]
    mg.serve_configure(0, 8)
    hs = [mg.Hierarchy(mg.make_params(d, n, "HS", zero_guess=1)) for d, n, s in specs]
    bs = [torch.from_numpy(I.random_rhs(d, n, s)).cuda() for d, n, s in specs]
    us = [torch.zeros_like(b) for b in bs]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tickets = [h.submit(b, u) for h, b, u in zip(hs, bs, us)]
    done = [None] * len(tickets)
    deadline = time.time() + 120
    while any(d is None for d in done):
        assert time.time() < deadline, "serving requests did not complete"
        for i, (h, t) in enumerate(zip(hs, tickets)):
            if done[i] is None:
                done[i] = h.poll(t)
        time.sleep(1e-4)
    wall = time.perf_counter() - t0
    for (u_ref, r_ref), u, r, (d, n, sd) in zip(refs, us, done, specs):
        assert r["status"] == 0 and r["rel_res_true"] <= 1e-10
        assert np.array_equal(u.cpu().numpy(), u_ref)
        assert r["iters"] == r_ref["iters"]
        uo, info, _ = oracle.ir_solve(I.random_rhs(d, n, sd))
        assert np.linalg.norm(u.cpu().numpy() - uo) <= 1e-6 * np.linalg.norm(uo), (d, n)
        assert r["iters"] <= info["iters"] + 2, (d, n, r["iters"], info["iters"])
    assert wall < sum(r["seconds"] for _, r in refs) * 1.5
    # the poll that reported completion retired the ticket
    with pytest.raises(mg.MGError) as e:
        hs[0].poll(tickets[0])
    assert e.value.status == 2
    for h in hs:
        h.close()


def test_serving_same_hierarchy_queues():
    """Several requests on one hierarchy run one after another (one working set)."""
    import torch
    n = 47
    with mg.Hierarchy(mg.make_params(3, n, "H", zero_guess=1)) as h:
        bs = [torch.from_numpy(I.random_rhs(3, n, 400 + i)).cuda() for i in range(4)]
        us = [torch.zeros_like(b) for b in bs]
        ts = [h.submit(b, u) for b, u in zip(bs, us)]
        res = [None] * 4
        deadline = time.time() + 60
        while any(r is None for r in res):
            assert time.time() < deadline
            res = [r if r is not None else h.poll(t) for r, t in zip(res, ts)]
            time.sleep(1e-4)
        for i in range(4):
            u_ref, _ = alone(3, n, "H", I.random_rhs(3, n, 400 + i))
            assert np.array_equal(us[i].cpu().numpy(), u_ref)


def test_batch_with_cluster_tails_equals_alone():
    """Instances whose coarse tail runs in a thread-block cluster (no_tail = 2) merge
    into one batched cluster launch and give their alone results bit for bit."""
    import torch
    specs = [(3, 63, "H", 31), (3, 95, "HSD", 32), (3, 127, "H", 33)]
    refs = []
    for d, n, lad, sd in specs:
        with mg.Hierarchy(mg.make_params(d, n, lad, zero_guess=1, no_tail=2)) as h:
            b = torch.from_numpy(I.random_rhs(d, n, sd)).cuda()
            u = torch.zeros_like(b)
            r = h.solve(b, u)
            refs.append((u.cpu().numpy(), r))
    hs = [mg.Hierarchy(mg.make_params(d, n, lad, zero_guess=1, no_tail=2)) for d, n, lad, sd in specs]
    assert all(h.level_info(0)["tail_ctas"] > 1 for h in hs)
    bs = [torch.from_numpy(I.random_rhs(d, n, sd)).cuda() for d, n, lad, sd in specs]
    us = [torch.zeros_like(b) for b in bs]
    res = mg.solve_batch(hs, bs, us)
    for (u_ref, r_ref), u, r in zip(refs, us, res):
        assert r["merged"] == 1 and r["status"] == 0 and r["iters"] == r_ref["iters"]
        assert np.array_equal(u.cpu().numpy(), u_ref)
    for h in hs:
        h.close()
