"""Serving with admission by device memory (pooled hierarchies, mg_params.pooled = 1).

A pooled hierarchy holds only its plan; its working arena comes from the
device-memory pool when a solve is admitted and goes back when it completes.
The tests check that the pool's budget bounds the memory it holds while every
request completes with its alone result (bitwise) and the FP64 oracle's
solution (Alg. 2) within 1e-6, that requests which do not fit wait, and the
error paths of admission."""
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
    yield
    mg.serve_configure(0, 16)  # default budget for later tests


def alone(dim, n, lad, b, **kw):
    import torch
    with mg.Hierarchy(mg.make_params(dim, n, lad, zero_guess=1, **kw)) as h:
        u = torch.zeros(b.shape, dtype=torch.float64, device="cuda")
        res = h.solve(torch.from_numpy(b).cuda(), u)
        return u.cpu().numpy(), res


def work_bytes(dim, n, lad):
    """The working arena of a hierarchy: its footprint minus the persistent part
    (norm partials, control state, base inverse, tail program), which is small."""
    return mg.footprint_bytes(mg.make_params(dim, n, lad, pooled=1))


def wait_all(hs, tickets, limit=180):
    done = [None] * len(tickets)
    deadline = time.time() + limit
    while any(d is None for d in done):
        assert time.time() < deadline, "serving requests did not complete"
        for i, (h, t) in enumerate(zip(hs, tickets)):
            if done[i] is None:
                done[i] = h.poll(t)
        time.sleep(1e-4)
    return done


def test_pooled_solve_equals_resident_and_reuses_its_arena():
    import torch
    n = 95
    b = I.random_rhs(3, n, 61)
    u_ref, r_ref = alone(3, n, "H", b)
    mg.serve_configure(0, 16)
    with mg.Hierarchy(mg.make_params(3, n, "H", zero_guess=1, pooled=1)) as h:
        s0 = mg.serve_stats()
        bd = torch.from_numpy(b).cuda()
        for rep in range(2):
            ud = torch.zeros_like(bd)
            r = h.solve(bd, ud)
            assert r["status"] == 0 and r["iters"] == r_ref["iters"]
            assert np.array_equal(ud.cpu().numpy(), u_ref)
            assert mg.serve_stats()["in_use_bytes"] == s0["in_use_bytes"]  # handed back after the solve
        s1 = mg.serve_stats()
        assert s1["arena_acquires"] - s0["arena_acquires"] == 2
        assert s1["arena_reuses"] - s0["arena_reuses"] == 1  # the second solve found its arena intact
        # outside a solve a pooled hierarchy holds no level arrays: stage calls are refused
        with pytest.raises(mg.MGError) as e:
            h.run_stage(mg.STAGE_JACOBI, h.nlev - 1)
        assert e.value.status == 2 and "pooled" in str(e.value)


def test_serving_within_a_budget_smaller_than_the_inflight_arenas(oracle):
    """Eight requests whose working arenas add up to about three times the budget:
    the pool never holds more than the budget, requests wait for memory, and every
    result equals its alone solve bitwise and the oracle within 1e-6."""
    import torch
    specs = [(3, 127, 1), (2, 511, 2), (3, 95, 3), (3, 127, 4), (2, 383, 5), (3, 63, 6), (3, 95, 7), (2, 255, 8)]
    lad = "HS"
    sizes = [work_bytes(d, n, lad) for d, n, _ in specs]
    budget = int(max(sizes) * 1.3)
    assert sum(sizes) > 2.5 * budget
    refs = [alone(d, n, lad, I.random_rhs(d, n, s)) for d, n, s in specs]
    mg.serve_configure(budget, 8)
    try:
        hs = [mg.Hierarchy(mg.make_params(d, n, lad, zero_guess=1, pooled=1)) for d, n, s in specs]
        bs = [torch.from_numpy(I.random_rhs(d, n, s)).cuda() for d, n, s in specs]
        us = [torch.zeros_like(x) for x in bs]
        torch.cuda.synchronize()
        s0 = mg.serve_stats()
        assert s0["budget_bytes"] == budget
        tickets = [h.submit(x, u) for h, x, u in zip(hs, bs, us)]
        done = wait_all(hs, tickets)
        s1 = mg.serve_stats()
        assert s1["peak_reserved_bytes"] <= budget and s1["peak_in_use_bytes"] <= budget, s1
        assert s1["memory_waits"] - s0["memory_waits"] >= 1, s1  # some requests waited for memory
        assert s1["completed"] - s0["completed"] == len(specs) and s1["in_use_bytes"] == 0
        for (u_ref, r_ref), u, r, (d, n, sd) in zip(refs, us, done, specs):
            assert r["status"] == 0 and r["rel_res_true"] <= 1e-10
            assert r["iters"] == r_ref["iters"]
            assert np.array_equal(u.cpu().numpy(), u_ref), (d, n)
            uo, info, _ = oracle.ir_solve(I.random_rhs(d, n, sd))
            assert np.linalg.norm(u.cpu().numpy() - uo) <= 1e-6 * np.linalg.norm(uo), (d, n)
            assert r["iters"] <= info["iters"] + 2
        # the final poll retired each ticket
        with pytest.raises(mg.MGError) as e:
            hs[0].poll(tickets[0])
        assert e.value.status == 2
        # a second round on the same hierarchies: cached arenas are reused where they survived
        us2 = [torch.zeros_like(x) for x in bs]
        done2 = wait_all(hs, [h.submit(x, u) for h, x, u in zip(hs, bs, us2)])
        for (u_ref, _), u, r in zip(refs, us2, done2):
            assert r["status"] == 0 and np.array_equal(u.cpu().numpy(), u_ref)
        s2 = mg.serve_stats()
        assert s2["peak_reserved_bytes"] <= budget and s2["arena_evictions"] >= s1["arena_evictions"]
        for h in hs:
            h.close()
    finally:
        mg.serve_configure(0, 16)


def test_admission_rejects_a_request_larger_than_the_budget():
    import torch
    n = 63
    mg.serve_configure(1 << 20, 4)  # 1 MiB: smaller than the working arena
    try:
        with mg.Hierarchy(mg.make_params(3, n, "H", zero_guess=1, pooled=1)) as h:
            b = torch.zeros(n, n, n, dtype=torch.float64, device="cuda")
            with pytest.raises(mg.MGError) as e:
                h.submit(b, torch.zeros_like(b))
            assert e.value.status == 8
            with pytest.raises(mg.MGError) as e:  # a blocking solve cannot take the arena either
                h.solve(b, torch.zeros_like(b))
            assert e.value.status == 8
    finally:
        mg.serve_configure(0, 16)


def test_batch_of_pooled_hierarchies_equals_alone():
    """mg_solve_batch takes every instance's arena from the pool for the merged
    level-synchronous launches and hands them back afterwards."""
    import torch
    specs = [(3, 63, "H", 71), (3, 95, "H", 72), (3, 127, "HSD", 73)]
    refs = [alone(d, n, lad, I.random_rhs(d, n, sd)) for d, n, lad, sd in specs]
    mg.serve_configure(0, 16)
    hs = [mg.Hierarchy(mg.make_params(d, n, lad, zero_guess=1, pooled=1)) for d, n, lad, sd in specs]
    bs = [torch.from_numpy(I.random_rhs(d, n, sd)).cuda() for d, n, lad, sd in specs]
    for rep in range(2):
        us = [torch.zeros_like(x) for x in bs]
        res = mg.solve_batch(hs, bs, us)
        for (u_ref, r_ref), u, r in zip(refs, us, res):
            assert r["merged"] == 1 and r["status"] == 0 and r["iters"] == r_ref["iters"]
            assert np.array_equal(u.cpu().numpy(), u_ref)
    assert mg.serve_stats()["in_use_bytes"] == 0
    for h in hs:
        h.close()


def test_injected_pool_growth_failure():
    """The pool's chunk allocation fails (host-side injection): the solve reports
    MG_ERR_OOM, and the next one succeeds."""
    import torch
    n = 63
    mg.serve_configure(0, 16)
    b = torch.from_numpy(I.random_rhs(3, n, 9)).cuda()
    with mg.Hierarchy(mg.make_params(3, n, "H", zero_guess=1, pooled=1)) as h:
        # a tiny budget returns every idle chunk to the device, so the next solve must grow the pool
        mg.serve_configure(1 << 20, 16)
        assert mg.serve_stats()["reserved_bytes"] == 0
        mg.serve_configure(work_bytes(3, n, "H") * 2, 16)
        mg.fault_inject(mg.FAULT_ARENA, 1)
        with pytest.raises(mg.MGError) as e:
            h.solve(b, torch.zeros_like(b))
        assert e.value.status == 3
        mg.fault_inject(mg.FAULT_ARENA, 0)
        u = torch.zeros_like(b)
        assert h.solve(b, u)["status"] == 0
    mg.serve_configure(0, 16)


def test_serving_merges_requests_admitted_together(oracle):
    """With mg_serve_options(1), requests admitted in the same pass whose hierarchies the
    level-synchronous launches cover run as one merged group.  One slot is held by a long
    request while six others queue; opening the slots admits the six together.  Every
    result equals its alone solve bitwise (the merged launches keep each instance's own
    scale, norms and stopping test) and the oracle within 1e-6."""
    import torch
    specs = [(3, 63, "H", 81), (3, 95, "H", 82), (3, 127, "HSD", 83), (3, 63, "H", 84), (3, 47, "H", 85),
             (3, 95, "H", 86)]
    refs = [alone(d, n, lad, I.random_rhs(d, n, sd)) for d, n, lad, sd in specs]
    mg.serve_configure(0, 1)
    mg.serve_options(True)
    try:
        big = mg.Hierarchy(mg.make_params(3, 255, "H", zero_guess=1, pooled=1))
        hs = [mg.Hierarchy(mg.make_params(d, n, lad, zero_guess=1, pooled=1)) for d, n, lad, sd in specs]
        bb = torch.from_numpy(I.random_rhs(3, 255, 80)).cuda()
        ub = torch.zeros_like(bb)
        bs = [torch.from_numpy(I.random_rhs(d, n, sd)).cuda() for d, n, lad, sd in specs]
        us = [torch.zeros_like(x) for x in bs]
        torch.cuda.synchronize()
        s0 = mg.serve_stats()
        tb = big.submit(bb, ub)  # holds the only slot for a few milliseconds
        time.sleep(2e-3)
        tickets = [h.submit(x, u) for h, x, u in zip(hs, bs, us)]
        mg.serve_configure(0, 16)  # the six queued requests are admitted in one pass
        done = wait_all(hs + [big], tickets + [tb])
        s1 = mg.serve_stats()
        assert s1["merged_requests"] - s0["merged_requests"] >= 2, s1
        assert s1["merged_groups"] - s0["merged_groups"] >= 1
        for (u_ref, r_ref), u, r, (d, n, lad, sd) in zip(refs, us, done[:-1], specs):
            assert r["status"] == 0 and r["iters"] == r_ref["iters"]
            assert np.array_equal(u.cpu().numpy(), u_ref), (n, lad)
            uo, info, _ = oracle.ir_solve(I.random_rhs(d, n, sd))
            assert np.linalg.norm(u.cpu().numpy() - uo) <= 1e-6 * np.linalg.norm(uo)
        assert done[-1]["status"] == 0
        assert sum(r["merged"] for r in done[:-1]) >= 2
        for h in hs + [big]:
            h.close()
    finally:
        mg.serve_options(False)
        mg.serve_configure(0, 16)
