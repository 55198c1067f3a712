"""The GPU solve against the oracle's low-precision emulation: every stored level
vector rounded to the level's format, operations in FP64, the residual scaling
of Sec. 4.3 and the FP16 rescale of Sec. 6.  The emulation rounds where the GPU
path stores, so iteration counts agree to one step, and the failures the
emulation predicts (FP16 without residual scaling, DSH_MG without the rescale)
happen on the GPU too."""
import numpy as np
import pytest

from paper_2007_07539_gb300 import inputs as I
from paper_2007_07539_gb300 import mg

pytestmark = pytest.mark.gpu

NOT_CONVERGED = 5  # MG_ERR_NOT_CONVERGED


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def gpu_solve(dim, n, lad, b, **kw):
    import torch
    p = mg.make_params(dim, n, lad, zero_guess=1, **kw)
    with mg.Hierarchy(p) as h:
        bd = torch.from_numpy(b).cuda()
        ud = torch.zeros_like(bd)
        res = h.solve(bd, ud)
        return ud.cpu().numpy(), res


def emulated(oracle, lad, b, **kw):
    """The oracle's emulation of the GPU ladder lad (library precision codes)."""
    fmt = {mg.FP64: oracle.FP64, mg.FP32: oracle.FP32, mg.FP16: oracle.FP16, mg.BF16: oracle.BF16}
    return oracle.ir_solve(b, prec=[fmt[p] for p in lad], **kw)


@pytest.mark.parametrize("dim,n,seed", [(3, 31, 2), (3, 63, 2), (2, 127, 2), (2, 255, 9)])
def test_iteration_counts_match_the_emulation(oracle, dim, n, seed):
    """H_MG, HSD_MG, DSH_MG and the BF16 ladder: the GPU's iteration count is the
    emulation's to one step."""
    b = I.random_rhs(dim, n, seed)
    nl = len(mg.level_count(n))
    for name in ("H", "HSD", "DSH", "B"):
        lad = mg.ladder(name, nl)
        _, res = gpu_solve(dim, n, lad, b)
        _, info, _ = emulated(oracle, lad, b)
        assert res["status"] == 0 and info["converged"], (name, res, info)
        assert abs(res["iters"] - info["iters"]) <= 1, (name, res["iters"], info["iters"])


@pytest.mark.parametrize("dim,n", [(3, 31), (2, 127)])
def test_fp16_without_residual_scaling_stalls_as_emulated(oracle, dim, n):
    """Sec. 4.3: all-FP16 multigrid with the unscaled residual stalls far above the
    tolerance on the GPU as in the emulation, at a residual of the same order."""
    b = I.random_rhs(dim, n, 2)
    nl = len(mg.level_count(n))
    lad = mg.ladder("H", nl)
    _, res = gpu_solve(dim, n, lad, b, scaling=0, max_iter=30)
    _, info, _ = emulated(oracle, lad, b, scaling=0, max_iter=30)
    assert not info["converged"] and info["rel_res"] > 1e-6
    assert res["status"] == NOT_CONVERGED, res
    assert info["rel_res"] / 10 < res["rel_res"] < info["rel_res"] * 10, (res["rel_res"], info["rel_res"])


@pytest.mark.parametrize("dim,n", [(3, 31), (2, 127)])
def test_dsh_unscaled_needs_the_rescale_as_emulated(oracle, dim, n):
    """Sec. 6: FP64 / FP32 fine levels over FP16 coarse levels with the unscaled outer
    residual converge at the emulation's count with the rescale into the FP16
    levels, and take clearly more steps (or stall) without it."""
    b = I.random_rhs(dim, n, 2)
    nl = len(mg.level_count(n))
    lad = [mg.FP16] * (nl - 2) + [mg.FP32, mg.FP64]
    _, res1 = gpu_solve(dim, n, lad, b, scaling=0, rescale16=1)
    _, info1, _ = emulated(oracle, lad, b, scaling=0, rescale16=1)
    assert res1["status"] == 0 and info1["converged"]
    assert abs(res1["iters"] - info1["iters"]) <= 1, (res1["iters"], info1["iters"])
    _, res0 = gpu_solve(dim, n, lad, b, scaling=0, rescale16=0, max_iter=30)
    assert res0["status"] == NOT_CONVERGED or res0["iters"] >= res1["iters"] + 4, (res0, res1)
