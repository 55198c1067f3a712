"""The C-ABI library: builds, loads, exports every symbol of include/mg.h, and
its host-side logic (coarsening rule, parameter validation, footprint) -- no
GPU needed."""
import ctypes
import os
import re

import pytest

from paper_2007_07539_gb300 import mg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "mg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mg_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = mg.lib()
    decl = declared_functions()
    assert len(decl) >= 15
    for name in decl:
        assert hasattr(L, name), name
    assert sorted(mg.EXPORTS) == decl


def test_level_count_matches_oracle(oracle):
    for n in (1, 2, 3, 5, 7, 31, 47, 63, 127, 255, 383, 511, 4095):
        assert mg.level_count(n) == oracle.level_sizes(n)
    for n, L in ((255, 3), (511, 2), (127, 6)):
        assert mg.level_count(n, L) == oracle.level_sizes(n, L)
    assert mg.level_count(0) == []


def test_params_defaults():
    p = mg.make_params(3, 255)
    assert (p.nu1, p.nu2, p.gamma, p.scaling, p.tol_mode, p.max_iter) == (2, 2, 1, 1, 0, 100)
    assert p.omega == 0.8 and p.tol == 1e-10
    assert list(p.prec)[:7] == [mg.FP64] * 7
    assert (p.rescale16, p.base_solver, p.base_maxit, p.base_tol, p.op) == (1, 0, 0, 1e-4, 0)


def test_ladders():
    assert mg.ladder("HSD", 8) == [0, 1, 1, 1, 1, 1, 2, 2]
    assert mg.ladder("DSH", 6, 2, 1) == [2, 1, 1, 1, 0, 0]
    assert mg.ladder("BSD", 7)[-2:] == [mg.BF16, mg.BF16]
    assert mg.ladder("H", 3) == [2, 2, 2]


@pytest.mark.parametrize("bad", [dict(dim=4), dict(n=0), dict(omega=2.5), dict(gamma=3), dict(scaling=7),
                                 dict(max_iter=5000), dict(nu1=-1), dict(levels=9), dict(tol=-1.0), dict(tune=2),
                                 dict(no_tail=5), dict(fuse_pre=3), dict(rescale16=2), dict(base_solver=2),
                                 dict(base_maxit=-1), dict(base_tol=-1.0), dict(base_tol=float("nan")),
                                 dict(op=2), dict(op=1, fuse_pre=1), dict(scale_ahead=2), dict(no_tail=3),
                                 dict(base_maxit=100001), dict(wait_polls=-2), dict(pooled=2)])
def test_invalid_params_rejected_without_gpu(bad):
    p = mg.make_params(3, 63)
    for k, v in bad.items():
        setattr(p, k, v)
    h = ctypes.c_void_p()
    st = mg.lib().mg_create_hierarchy(ctypes.byref(p), None, ctypes.byref(h))
    assert st == 2 and not h.value
    assert mg.last_error()
    assert mg.footprint_bytes(p) == 0


def test_coarsest_level_limit():
    p = mg.make_params(3, 33)  # 33 -> 16: 4096 unknowns on the base level: allowed
    assert mg.footprint_bytes(p) > 0
    p = mg.make_params(3, 34)  # one level of 34^3 unknowns: too large for the dense base solve
    assert mg.footprint_bytes(p) == 0


def test_footprint_scales_with_precision():
    d = mg.footprint_bytes(mg.make_params(3, 255, "D"))
    h = mg.footprint_bytes(mg.make_params(3, 255, "H"))
    assert 0 < h < d
    # FP64 u, r plus three level vectors per level: about 2*8 + 3*8*8/7 bytes/DOF for D_MG
    assert 40 * 255**3 < d < 56 * 255**3


def test_footprint_of_options():
    """The operator, the tail layout, scale-ahead and the base solver do not change
    the device arrays; a rescaled FP16 level adds only its FP32 restriction scratch."""
    base = mg.footprint_bytes(mg.make_params(3, 127, "H"))
    assert base > 0
    for kw in (dict(op=1), dict(no_tail=2), dict(scale_ahead=0), dict(base_solver=1)):
        assert mg.footprint_bytes(mg.make_params(3, 127, "H", **kw)) == base, kw
    # no tail: no stage program on the device
    assert mg.footprint_bytes(mg.make_params(3, 127, "H", no_tail=1)) < base
    nlev = len(mg.level_count(127))
    dsh = [mg.FP16] * 2 + [mg.FP32] * (nlev - 2)
    with_rescale = mg.footprint_bytes(mg.make_params(3, 127, dsh))
    without = mg.footprint_bytes(mg.make_params(3, 127, dsh, rescale16=0))
    assert with_rescale > without > 0


def test_fault_inject_validates_its_arguments_without_gpu():
    """mg_fault_inject is host-side: bad sites and counts are rejected, valid
    requests are accepted and cancelled with count 0 (no device needed)."""
    L = mg.lib()
    assert L.mg_fault_inject(-1, 1) == 2 and L.mg_fault_inject(2, 1) == 2 and L.mg_fault_inject(0, -1) == 2
    assert L.mg_fault_inject(mg.FAULT_ARENA, 3) == 0 and L.mg_fault_inject(mg.FAULT_ARENA, 0) == 0
    assert L.mg_fault_inject(mg.FAULT_STAGING, 0) == 0


@pytest.mark.parametrize("bad", [(3, mg.FP16, 95, 1, 1), (0, 9, 95, 1, 1), (0, mg.FP16, 2, 1, 1),
                                 (0, mg.FP16, 1291, 1, 1), (2, mg.FP16, 95, 2, 1), (0, mg.FP16, 15, 2, 1),
                                 (0, mg.FP16, 95, 1, 0), (0, mg.FP16, 95, 1, 96), (2, mg.FP16, 95, 1, 48),
                                 (1, mg.FP16, 95, 3, 1), (1, mg.FP16, 95, -2, 1), (2, mg.FP16, 4, 0, 0)])
def test_tile_set_validates_its_arguments_without_gpu(bad):
    """mg_tile_set rejects unknown kernels and precisions, grid sizes outside 3..1290 and shapes
    the kernels do not have (two rows per warp for the restriction or below 16 rows, march
    lengths outside 1..n, or 1..(n-1)/2 coarse planes), with MG_ERR_INVALID and no device."""
    with pytest.raises(mg.MGError) as e:
        mg.tile_set(*bad)
    assert e.value.status == 2  # MG_ERR_INVALID


def test_tile_set_accepts_and_forgets_shapes_without_gpu():
    """Valid shapes are recorded and forgotten (rows_per_warp = -1) without a device."""
    for shape in [(0, mg.FP16, 95, 0, 0), (0, mg.FP64, 95, 1, 95), (1, mg.BF16, 17, 2, 1),
                  (2, mg.FP32, 95, 1, 47), (2, mg.FP16, 5, 0, 0)]:
        mg.tile_set(*shape)
        mg.tile_set(shape[0], shape[1], shape[2], -1)


def test_params_struct_matches_the_header():
    """The binding's mg_params mirrors include/mg.h: the C size (compiled with gcc)
    equals ctypes' size, and the defaults of the new fields."""
    import subprocess
    import tempfile
    src = '#include <stdio.h>\n#include "mg.h"\nint main(void){printf("%zu %zu", sizeof(mg_params), sizeof(mg_result));return 0;}\n'
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "s.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "s")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), "-o", exe, c])
        out = subprocess.check_output([exe]).decode().split()
    assert int(out[0]) == ctypes.sizeof(mg.Params) and int(out[1]) == ctypes.sizeof(mg.Result)
    p = mg.make_params(3, 31)
    assert p.wait_polls == -1 and p.pooled == 0 and list(p.reserved) == [0, 0, 0, 0]
