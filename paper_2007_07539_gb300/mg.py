"""ctypes binding of libmgfp (include/mg.h).

Argument marshalling only: every step of the solve runs in the library's CUDA
kernels.  Vectors may be torch CUDA tensors (device pointers), pinned or
pageable host memory (torch CPU tensors or numpy arrays); they must be
contiguous FP64 arrays of n^d values, x fastest (shape (n, n) or (n, n, n)).
The library is loaded from this package directory and nothing falls back to
another implementation: if libmgfp.so is missing, every entry point raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmgfp.so")
MAX_LEVELS = 16

FP64, FP32, FP16, BF16 = 0, 1, 2, 3
PREC = {"fp64": FP64, "fp32": FP32, "fp16": FP16, "bf16": BF16}
STATUS = {0: "MG_OK", 1: "MG_BUSY", 2: "MG_ERR_INVALID", 3: "MG_ERR_OOM", 4: "MG_ERR_CUDA",
          5: "MG_ERR_NOT_CONVERGED", 6: "MG_ERR_NUMERIC", 7: "MG_ERR_TIMEOUT", 8: "MG_ERR_ADMISSION"}
MG_OK, MG_BUSY = 0, 1
VEC_C, VEC_G, VEC_T, VEC_U, VEC_R = range(5)
(STAGE_JACOBI, STAGE_JACOBI_ZERO2, STAGE_RESTRICT, STAGE_PROLONG, STAGE_JACOBI_PROLONG, STAGE_COARSE,
 STAGE_SCALE_ZERO2, STAGE_IR_UPDATE, STAGE_RESIDUAL, STAGE_CYCLE, STAGE_PRE_RESTRICT,
 STAGE_RESTRICT_RESCALE) = range(12)

# Every symbol declared in include/mg.h.
EXPORTS = ["mg_params_init", "mg_level_count", "mg_last_error", "mg_footprint_bytes",
           "mg_create_hierarchy", "mg_solve", "mg_submit", "mg_poll", "mg_destroy",
           "mg_serve_configure", "mg_solve_batch", "mg_profile_solve", "mg_level_write", "mg_level_read",
           "mg_level_info_get", "mg_run_stage", "mg_residual_norms_noalloc", "mg_axpy", "mg_describe_cycle",
           "mg_fault_inject", "mg_serve_stats_get", "mg_serve_options", "mg_tile_set"]
FAULT_ARENA, FAULT_STAGING = 0, 1


class Params(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("n", ctypes.c_int32), ("levels", ctypes.c_int32),
                ("prec", ctypes.c_int32 * MAX_LEVELS), ("nu1", ctypes.c_int32), ("nu2", ctypes.c_int32),
                ("omega", ctypes.c_double), ("gamma", ctypes.c_int32), ("scaling", ctypes.c_int32),
                ("sigma_log2", ctypes.c_int32), ("tol_mode", ctypes.c_int32), ("tol", ctypes.c_double),
                ("max_iter", ctypes.c_int32), ("zero_guess", ctypes.c_int32), ("guard", ctypes.c_int32),
                ("graph", ctypes.c_int32), ("no_tail", ctypes.c_int32), ("tune", ctypes.c_int32),
                ("fuse_pre", ctypes.c_int32), ("rescale16", ctypes.c_int32), ("base_solver", ctypes.c_int32),
                ("base_maxit", ctypes.c_int32), ("base_tol", ctypes.c_double), ("op", ctypes.c_int32),
                ("scale_ahead", ctypes.c_int32), ("wait_polls", ctypes.c_int32), ("pooled", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 4)]


class Result(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("status", ctypes.c_int32), ("levels", ctypes.c_int32),
                ("guard_restarts", ctypes.c_int32), ("launches", ctypes.c_int32), ("merged", ctypes.c_int32),
                ("rel_res", ctypes.c_double),
                ("rel_res_true", ctypes.c_double), ("bnorm", ctypes.c_double), ("seconds", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class ServeStats(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_uint64), ("reserved_bytes", ctypes.c_uint64),
                ("in_use_bytes", ctypes.c_uint64), ("peak_in_use_bytes", ctypes.c_uint64),
                ("peak_reserved_bytes", ctypes.c_uint64), ("arena_acquires", ctypes.c_uint64),
                ("arena_reuses", ctypes.c_uint64), ("arena_evictions", ctypes.c_uint64),
                ("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("memory_waits", ctypes.c_uint64),
                ("merged_groups", ctypes.c_uint64), ("merged_requests", ctypes.c_uint64),
                ("inflight", ctypes.c_int32), ("peak_inflight", ctypes.c_int32), ("queued", ctypes.c_int32),
                ("reserved_", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved_"}


class LevelInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("prec", ctypes.c_int32), ("pitch", ctypes.c_int32),
                ("tail_ctas", ctypes.c_int32), ("bytes", ctypes.c_size_t), ("pre_launches", ctypes.c_int32),
                ("reserved_", ctypes.c_int32)]


class KernelTime(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("level", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("loader", ctypes.c_int32), ("prec", ctypes.c_int32), ("prec_coarse", ctypes.c_int32),
                ("launches", ctypes.c_int32), ("threads", ctypes.c_int32), ("grid", ctypes.c_int32 * 3),
                ("reserved", ctypes.c_int32), ("total_ms", ctypes.c_double), ("bytes", ctypes.c_double)]

    KIND = ["sweep", "base_solve", "prolong", "zero", "finalize", "ir_update", "scale_cast", "coarse_tail",
            "rescale16"]
    MODE = ["jacobi", "jacobi_x2_from_zero", "jacobi_from_zero", "residual_restrict", "pre_smooth_restrict"]

    def name(self) -> str:
        p = ["fp64", "fp32", "fp16", "bf16"]
        if self.kind == 0:
            nm = self.MODE[self.mode]
            if self.mode in (3, 4):
                return nm + f"_{p[self.prec]}_to_{p[self.prec_coarse]}"
            return nm + f"_{p[self.prec]}"
        if self.kind == 2:
            return f"prolong_{p[self.prec_coarse]}_to_{p[self.prec]}"
        return self.KIND[self.kind] + f"_{p[self.prec]}"

    def as_dict(self) -> dict:
        d = {f: getattr(self, f) for f, _ in self._fields_ if f not in ("grid", "reserved")}
        d["grid"] = list(self.grid)
        d["name"] = self.name()
        return d


class MGError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None
_lock = threading.Lock()


def lib() -> ctypes.CDLL:
    """Loads libmgfp.so from the package directory (raises if it was not built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libmgfp.so not built ({LIB_PATH}); run __graft_entry__.build()")
            L = ctypes.CDLL(LIB_PATH)
            P, R, H = ctypes.POINTER(Params), ctypes.POINTER(Result), ctypes.c_void_p
            i32, vp, dp = ctypes.c_int32, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)
            L.mg_params_init.argtypes = [P, i32, i32]
            L.mg_params_init.restype = None
            L.mg_level_count.argtypes = [i32, i32, ctypes.POINTER(i32)]
            L.mg_level_count.restype = i32
            L.mg_last_error.restype = ctypes.c_char_p
            L.mg_footprint_bytes.argtypes = [P]
            L.mg_footprint_bytes.restype = ctypes.c_size_t
            L.mg_describe_cycle.argtypes = [P, ctypes.POINTER(i32), i32, ctypes.POINTER(i32)]
            L.mg_create_hierarchy.argtypes = [P, vp, ctypes.POINTER(H)]
            L.mg_solve.argtypes = [H, vp, vp, R]
            L.mg_submit.argtypes = [H, vp, vp, ctypes.POINTER(ctypes.c_uint64)]
            L.mg_poll.argtypes = [H, ctypes.c_uint64, R]
            L.mg_destroy.argtypes = [H]
            L.mg_serve_configure.argtypes = [ctypes.c_size_t, i32]
            L.mg_solve_batch.argtypes = [i32, ctypes.POINTER(H), ctypes.POINTER(vp), ctypes.POINTER(vp), R]
            L.mg_level_write.argtypes = [H, i32, i32, vp]
            L.mg_level_read.argtypes = [H, i32, i32, vp]
            L.mg_level_info_get.argtypes = [H, i32, ctypes.POINTER(LevelInfo)]
            L.mg_run_stage.argtypes = [H, i32, i32, dp, vp, dp]
            L.mg_profile_solve.argtypes = [H, vp, vp, R, ctypes.POINTER(KernelTime), i32, ctypes.POINTER(i32)]
            L.mg_residual_norms_noalloc.argtypes = [i32, i32, vp, vp, vp, vp]
            L.mg_residual_norms_noalloc.restype = ctypes.c_int
            L.mg_axpy.argtypes = [i32, ctypes.c_int64, ctypes.c_double, vp, vp, vp]
            L.mg_axpy.restype = ctypes.c_int
            L.mg_serve_stats_get.argtypes = [ctypes.POINTER(ServeStats)]
            L.mg_serve_stats_get.restype = ctypes.c_int
            L.mg_serve_options.argtypes = [i32]
            L.mg_serve_options.restype = ctypes.c_int
            L.mg_fault_inject.argtypes = [i32, i32]
            L.mg_fault_inject.restype = ctypes.c_int
            L.mg_tile_set.argtypes = [i32, i32, i32, i32, i32]
            L.mg_tile_set.restype = ctypes.c_int
            for f in ("mg_create_hierarchy", "mg_solve", "mg_submit", "mg_poll", "mg_destroy",
                      "mg_serve_configure", "mg_solve_batch", "mg_level_write", "mg_level_read",
                      "mg_level_info_get", "mg_run_stage", "mg_profile_solve"):
                getattr(L, f).restype = ctypes.c_int
            _lib = L
    return _lib


def last_error() -> str:
    return lib().mg_last_error().decode()


def _check(status: int, where: str, ok=(MG_OK,)) -> int:
    if status not in ok:
        raise MGError(status, where, last_error())
    return status


def level_count(n: int, levels: int = 0) -> list[int]:
    """Level sizes, coarsest first (the library's coarsening rule)."""
    buf = (ctypes.c_int32 * 64)()
    cnt = lib().mg_level_count(int(n), int(levels), buf)
    return [buf[i] for i in range(cnt)]


def ladder(name: str, nlev: int, n_fine: int = 2, n_coarse: int = 1) -> list[int]:
    """Per-level precisions, coarsest first, for the variants of Table 2 and the
    ladders used in the benchmarks:
      D      all FP64 (D_MG)           H    all FP16, FP16 base (H_MG)
      S      all FP32                  HSD  FP16 on the n_fine finest levels, FP32 between,
                                            FP64 on the n_coarse coarsest (HSD_MG)
      DSH    FP64 on the n_fine finest, FP32 between, FP16 on the n_coarse coarsest (DSH_MG)
      BSD    as HSD with BF16 on the finest levels
      HS     FP16 on the n_fine finest, FP32 below"""
    name = name.upper()
    if name == "D":
        return [FP64] * nlev
    if name == "H":
        return [FP16] * nlev
    if name == "S":
        return [FP32] * nlev
    if name == "B":
        return [BF16] * nlev
    fine, coarse = {"HSD": (FP16, FP64), "DSH": (FP64, FP16), "BSD": (BF16, FP64), "HS": (FP16, FP32)}[name]
    out = []
    for l in range(nlev):
        if l >= nlev - n_fine:
            out.append(fine)
        elif l < n_coarse:
            out.append(coarse)
        else:
            out.append(FP32)
    return out


def make_params(dim: int, n: int, ladder_name: str | list[int] = "D", **kw) -> Params:
    """mg_params_init plus overrides; ladder_name is a ladder() name or an explicit
    per-level list (coarsest first)."""
    p = Params()
    lib().mg_params_init(ctypes.byref(p), int(dim), int(n))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    nlev = len(level_count(n, p.levels))
    precs = ladder(ladder_name, nlev) if isinstance(ladder_name, str) else list(ladder_name)
    if len(precs) != nlev:
        raise ValueError(f"ladder has {len(precs)} entries, hierarchy has {nlev} levels")
    for i, v in enumerate(precs):
        p.prec[i] = v
    return p


def footprint_bytes(p: Params) -> int:
    return int(lib().mg_footprint_bytes(ctypes.byref(p)))


CYCLE_FIELDS = ("kind", "level", "kernel", "mode", "prec", "prec_c")


def describe_cycle(p: Params) -> list[dict]:
    """The operations of one IR step's cycle as the library schedules them
    (mg_describe_cycle; no device needed): one dict per record."""
    cnt = ctypes.c_int32(0)
    _check(lib().mg_describe_cycle(ctypes.byref(p), None, 0, ctypes.byref(cnt)), "mg_describe_cycle")
    buf = (ctypes.c_int32 * (6 * max(cnt.value, 1)))()
    _check(lib().mg_describe_cycle(ctypes.byref(p), buf, cnt.value, ctypes.byref(cnt)), "mg_describe_cycle")
    return [dict(zip(CYCLE_FIELDS, buf[6 * k: 6 * k + 6])) for k in range(cnt.value)]


def _ptr(x) -> int:
    """Address of a torch tensor or numpy array (no copy)."""
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    import numpy as np
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    raise TypeError(f"unsupported buffer type {type(x)}")


def _stream_handle(stream) -> int:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return 0
    return int(getattr(stream, "cuda_stream", stream))


class Hierarchy:
    """Owner of one mg_hierarchy (all device state of a solver)."""

    def __init__(self, params: Params, stream=None):
        self.params = params
        self.dim, self.n = params.dim, params.n
        h = ctypes.c_void_p()
        _check(lib().mg_create_hierarchy(ctypes.byref(params), ctypes.c_void_p(_stream_handle(stream)),
                                         ctypes.byref(h)), "mg_create_hierarchy")
        self._h = h
        self.nlev = len(level_count(params.n, params.levels))

    @property
    def handle(self) -> ctypes.c_void_p:
        if self._h is None:
            raise RuntimeError("hierarchy destroyed")
        return self._h

    def solve(self, b, u) -> dict:
        """mg_solve: u (in: initial guess, out: solution).  Returns the mg_result as a dict;
        a failed solve raises MGError except for MG_ERR_NOT_CONVERGED (status in the dict)."""
        r = Result()
        st = lib().mg_solve(self.handle, ctypes.c_void_p(_ptr(b)), ctypes.c_void_p(_ptr(u)), ctypes.byref(r))
        _check(st, "mg_solve", ok=(MG_OK, 5))
        return r.as_dict()

    def profile_solve(self, b, u):
        """mg_profile_solve: (result dict, list of per-kernel timing dicts in launch order)."""
        r = Result()
        buf = (KernelTime * 512)()
        cnt = ctypes.c_int32()
        st = lib().mg_profile_solve(self.handle, ctypes.c_void_p(_ptr(b)), ctypes.c_void_p(_ptr(u)),
                                    ctypes.byref(r), buf, 512, ctypes.byref(cnt))
        _check(st, "mg_profile_solve", ok=(MG_OK, 5))
        return r.as_dict(), [buf[i].as_dict() for i in range(min(cnt.value, 512))]

    def submit(self, b, u) -> int:
        t = ctypes.c_uint64()
        _check(lib().mg_submit(self.handle, ctypes.c_void_p(_ptr(b)), ctypes.c_void_p(_ptr(u)),
                               ctypes.byref(t)), "mg_submit")
        return t.value

    def poll(self, ticket: int):
        """None while running, else the result dict."""
        r = Result()
        st = lib().mg_poll(self.handle, ctypes.c_uint64(ticket), ctypes.byref(r))
        if st == MG_BUSY:
            return None
        _check(st, "mg_poll", ok=(MG_OK, 5, 6))
        return r.as_dict()

    def level_info(self, level: int) -> dict:
        li = LevelInfo()
        _check(lib().mg_level_info_get(self.handle, int(level), ctypes.byref(li)), "mg_level_info_get")
        return dict(n=li.n, prec=li.prec, pitch=li.pitch, tail_ctas=li.tail_ctas, bytes=li.bytes,
                    pre_launches=li.pre_launches)

    def level_write(self, level: int, vec: int, src) -> None:
        _check(lib().mg_level_write(self.handle, int(level), int(vec), ctypes.c_void_p(_ptr(src))),
               "mg_level_write")

    def level_read(self, level: int, vec: int, dst) -> None:
        _check(lib().mg_level_read(self.handle, int(level), int(vec), ctypes.c_void_p(_ptr(dst))),
               "mg_level_read")

    def run_stage(self, stage: int, level: int, arg: float | None = None, ptr=None, arg2: float = 0.0):
        a = (ctypes.c_double * 2)(arg if arg is not None else 0.0, arg2)
        out = (ctypes.c_double * 2)()
        _check(lib().mg_run_stage(self.handle, int(stage), int(level), a if arg is not None else None,
                                  ctypes.c_void_p(_ptr(ptr)) if ptr is not None else None, out),
               "mg_run_stage")
        return out[0], out[1]

    def close(self) -> None:
        if self._h is not None:
            lib().mg_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_batch(hs: list[Hierarchy], bs: list, us: list) -> list[dict]:
    """mg_solve_batch over hierarchies hs with right-hand sides bs and solutions us."""
    n = len(hs)
    H = (ctypes.c_void_p * n)(*[h.handle.value for h in hs])
    B = (ctypes.c_void_p * n)(*[_ptr(b) for b in bs])
    U = (ctypes.c_void_p * n)(*[_ptr(u) for u in us])
    R = (Result * n)()
    st = lib().mg_solve_batch(n, H, B, U, R)
    _check(st, "mg_solve_batch", ok=(MG_OK, 5))
    return [R[i].as_dict() for i in range(n)]


def serve_configure(budget_bytes: int = 0, max_inflight: int = 0) -> None:
    _check(lib().mg_serve_configure(int(budget_bytes), int(max_inflight)), "mg_serve_configure")


def serve_options(merge_groups: bool) -> None:
    """mg_serve_options: run requests admitted together as merged level-synchronous groups."""
    _check(lib().mg_serve_options(1 if merge_groups else 0), "mg_serve_options")


def serve_stats() -> dict:
    """mg_serve_stats_get: the current device's memory pool and serving counters."""
    st = ServeStats()
    _check(lib().mg_serve_stats_get(ctypes.byref(st)), "mg_serve_stats_get")
    return st.as_dict()


def residual_norms_noalloc(dim: int, n: int, b, u, norms, stream=None) -> None:
    """mg_residual_norms_noalloc: writes ||b - A u||_2, ||b - A u||_inf and ||b||_2 into the
    3-element device array `norms`, enqueued on `stream` (default: torch's current stream).
    Allocates no device memory (a static 2 MiB scratch array inside the library), for
    callers that cannot allocate at that point; calls that overlap on the GPU race."""
    _check(lib().mg_residual_norms_noalloc(int(dim), int(n), ctypes.c_void_p(_ptr(b)), ctypes.c_void_p(_ptr(u)),
                                           ctypes.c_void_p(_ptr(norms)), ctypes.c_void_p(_stream_handle(stream))),
           "mg_residual_norms_noalloc")


def axpy(prec: int, a: float, x, y, stream=None) -> None:
    """mg_axpy: y <- a x + y on device tensors of the storage type prec (Sec. 8.2, Fig. 6)."""
    n = x.numel()
    _check(lib().mg_axpy(int(prec), ctypes.c_int64(n), ctypes.c_double(a), ctypes.c_void_p(_ptr(x)),
                         ctypes.c_void_p(_ptr(y)), ctypes.c_void_p(_stream_handle(stream))), "mg_axpy")


TILE_JACOBI, TILE_ZERO2, TILE_RESTRICT = 0, 1, 2


def tile_set(kernel: int, prec: int, n: int, rows_per_warp: int, march_len: int = 0) -> None:
    """mg_tile_set: pin the launch shape of a 3D finite-difference stencil kernel on levels of
    n points (rows_per_warp -1 forgets it, 0 the direct kernel, 1 or 2 marching; march_len
    planes, or coarse planes for the restriction, per CTA).  Process-wide."""
    _check(lib().mg_tile_set(int(kernel), int(prec), int(n), int(rows_per_warp), int(march_len)), "mg_tile_set")


def fault_inject(site: int, count: int) -> None:
    """mg_fault_inject: the next `count` allocations at `site` (FAULT_ARENA,
    FAULT_STAGING) fail as if the device were out of memory (host-side; 0 cancels)."""
    _check(lib().mg_fault_inject(int(site), int(count)), "mg_fault_inject")
