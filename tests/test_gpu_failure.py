"""Failure detection without a device fault.

- Timeout path of the 3D stencil kernels' bounded waits for their TMA tile
  copies: a hierarchy made with wait_polls = 0 gives up on the first wait at
  once, while the copies it issued still land; the kernel stops issuing,
  drains those copies with the default bound and stops the solve.  The solve
  returns MG_ERR_TIMEOUT with u untouched, and the CUDA context stays usable:
  the next solves (same process, other hierarchies, a batch) are correct.
- Host-side fault injection (mg_fault_inject): allocations of the working
  arena and of the staging buffers fail as if the device were out of memory.
"""
import numpy as np
import pytest

from paper_2007_07539_gb300 import inputs as I
from paper_2007_07539_gb300 import mg

pytestmark = pytest.mark.gpu

MG_ERR_OOM, MG_ERR_TIMEOUT = 3, 7


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def _solve_ok(oracle, dim, n, lad, b):
    import torch
    with mg.Hierarchy(mg.make_params(dim, n, lad, zero_guess=1)) as h:
        bd = torch.from_numpy(b).cuda()
        ud = torch.zeros_like(bd)
        res = h.solve(bd, ud)
    uo, info, _ = oracle.ir_solve(b)
    u = ud.cpu().numpy()
    assert res["status"] == 0 and res["rel_res_true"] <= 1e-10, res
    assert np.linalg.norm(u - uo) <= 1e-6 * np.linalg.norm(uo)
    return u, res


@pytest.mark.parametrize("graph", [1, 0])
def test_wait_timeout_stops_the_solve_and_the_context_stays_usable(oracle, graph):
    import torch
    n = 127  # the finest level runs the marching TMA kernels (levels above 63^3)
    b = I.random_rhs(3, n, 7)
    p = mg.make_params(3, n, "H", zero_guess=1, wait_polls=0, graph=graph)
    with mg.Hierarchy(p) as h:
        bd = torch.from_numpy(b).cuda()
        for rep in range(2):  # the same hierarchy fails the same way again
            ud = torch.full_like(bd, 7.0)
            with pytest.raises(mg.MGError) as e:
                h.solve(bd, ud)
            assert e.value.status == MG_ERR_TIMEOUT, str(e.value)
            assert "timed out" in str(e.value) and "still not completed" not in str(e.value)
            # zero initial guess: the stopped solve leaves its last iterate, u = 0
            assert torch.count_nonzero(ud).item() == 0
    torch.cuda.synchronize()
    # the context is intact: a plain torch op and a normal solve of the same problem
    x = torch.arange(1000, device="cuda", dtype=torch.float64)
    assert float(x.sum()) == 499500.0
    _solve_ok(oracle, 3, n, "H", b)


def test_wait_timeout_in_a_batch_stops_only_its_instance(oracle):
    """In the level-synchronous batch each instance keeps its own control state:
    the instance whose waits give up stops with MG_ERR_TIMEOUT, the others
    complete with their alone results."""
    import torch
    specs = [(127, 0, 31), (95, -1, 32), (127, -1, 33)]
    refs = {}
    for n, wp, sd in specs:
        if wp < 0:
            refs[sd] = _solve_ok(oracle, 3, n, "H", I.random_rhs(3, n, sd))
    hs = [mg.Hierarchy(mg.make_params(3, n, "H", zero_guess=1, wait_polls=wp)) for n, wp, sd in specs]
    bs = [torch.from_numpy(I.random_rhs(3, n, sd)).cuda() for n, wp, sd in specs]
    us = [torch.zeros_like(x) for x in bs]
    with pytest.raises(mg.MGError) as e:
        mg.solve_batch(hs, bs, us)
    assert e.value.status == MG_ERR_TIMEOUT
    # per-instance results through the C ABI
    import ctypes
    n = len(hs)
    H = (ctypes.c_void_p * n)(*[h.handle.value for h in hs])
    B = (ctypes.c_void_p * n)(*[x.data_ptr() for x in bs])
    us = [torch.zeros_like(x) for x in bs]
    U = (ctypes.c_void_p * n)(*[x.data_ptr() for x in us])
    R = (mg.Result * n)()
    st = mg.lib().mg_solve_batch(n, H, B, U, R)
    assert st == MG_ERR_TIMEOUT
    for i, (nn, wp, sd) in enumerate(specs):
        assert R[i].merged == 1
        if wp == 0:
            assert R[i].status == MG_ERR_TIMEOUT
        else:
            assert R[i].status == 0 and R[i].iters == refs[sd][1]["iters"]
            assert np.array_equal(us[i].cpu().numpy(), refs[sd][0])
    for h in hs:
        h.close()


def test_injected_arena_allocation_failure():
    """mg_create_hierarchy reports MG_ERR_OOM when its arena allocation fails, and
    the next creation succeeds (nothing left behind)."""
    import torch
    p = mg.make_params(3, 63, "H", zero_guess=1)
    free0 = torch.cuda.mem_get_info()[0]
    mg.fault_inject(mg.FAULT_ARENA, 1)
    with pytest.raises(mg.MGError) as e:
        mg.Hierarchy(p)
    assert e.value.status == MG_ERR_OOM and "allocation" in str(e.value)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] >= free0 - (8 << 20)  # no arena held
    with mg.Hierarchy(p) as h:
        b = torch.from_numpy(I.random_rhs(3, 63, 3)).cuda()
        u = torch.zeros_like(b)
        assert h.solve(b, u)["status"] == 0


def test_injected_staging_allocation_failure(oracle):
    """A solve with host b and u needs device staging buffers; when their
    allocation fails the solve returns MG_ERR_OOM and leaves u unchanged; the
    next solve on the same hierarchy allocates them and is correct."""
    n = 31
    b = I.random_rhs(3, n, 4)
    u = np.full_like(b, 3.0)  # pageable host memory: staged
    with mg.Hierarchy(mg.make_params(3, n, "H")) as h:
        mg.fault_inject(mg.FAULT_STAGING, 1)
        with pytest.raises(mg.MGError) as e:
            h.solve(b, u)
        assert e.value.status == MG_ERR_OOM
        assert np.all(u == 3.0)
        u[...] = 0.0
        res = h.solve(b, u)
    uo, info, _ = oracle.ir_solve(b)
    assert res["status"] == 0 and res["iters"] <= info["iters"] + 2
    assert np.linalg.norm(u - uo) <= 1e-6 * np.linalg.norm(uo)
    mg.fault_inject(mg.FAULT_STAGING, 0)
