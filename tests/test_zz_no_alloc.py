"""mg_residual_norms_noalloc: residual norms for callers that cannot allocate device
memory (a host application that has reserved the device memory for its own pool, or
a latency-critical loop where an allocation would synchronise the device).  Checked
on two calls in a row against the existing stage entry point (MG_STAGE_RESIDUAL) and
against the FP64 oracle's residual b - A u with numpy's norms, within the FP64
tolerance of the other tests.  Collected last on purpose."""
import numpy as np
import pytest

from paper_2007_07539_gb300 import inputs as I
from paper_2007_07539_gb300 import mg

pytestmark = pytest.mark.gpu

REL = 1e-12  # the FP64 tolerance used by the kernel parity tests


def reference_norms(dim, n, b, u):
    """||b - A u||_2, ||b - A u||_inf through the existing entry point, and ||b||_2."""
    import torch
    with mg.Hierarchy(mg.make_params(dim, n, "D")) as h:
        h.level_write(h.nlev - 1, mg.VEC_U, u)
        n2, ninf = h.run_stage(mg.STAGE_RESIDUAL, h.nlev - 1, ptr=torch.from_numpy(b).cuda())
    return n2, ninf, float(np.linalg.norm(b))


def oracle_norms(oracle, b, u):
    """The oracle's r = b - A u (Sec. 4.1) and numpy's norms of r and b."""
    r = oracle.residual(b, u)
    return float(np.linalg.norm(r)), float(np.abs(r).max()), float(np.linalg.norm(b))


def test_noalloc_residual_norms_match_stage_entry_point_twice(oracle):
    import torch
    assert torch.cuda.is_available()
    cases = [(3, 95, 41), (2, 511, 42)]  # two calls in a row, the second smaller than the first
    for dim, n, seed in cases:
        u = I.uniform(seed, (n,) * dim)
        b = I.uniform(seed + 100, (n,) * dim, -1e3, 1e3)
        ref = reference_norms(dim, n, b, u)
        ora = oracle_norms(oracle, b, u)
        out = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
        mg.residual_norms_noalloc(dim, n, torch.from_numpy(b).cuda(), torch.from_numpy(u).cuda(), out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        for g, r, o in zip(got, ref, ora):
            assert abs(g - r) <= REL * abs(r), (dim, n, got, ref)
            assert abs(g - o) <= REL * abs(o), (dim, n, got, ora)


def test_noalloc_rejects_oversized_and_host_pointers():
    import torch
    b = torch.zeros(8, dtype=torch.float64, device="cuda")
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    with pytest.raises(mg.MGError) as e:
        mg.residual_norms_noalloc(3, 1000, b, b, out)  # 1e9 points > the static scratch limit
    assert e.value.status == 2 and "scratch" in mg.last_error()
    with pytest.raises(mg.MGError):
        mg.residual_norms_noalloc(2, 2, np.zeros(4), np.zeros(4), out)
