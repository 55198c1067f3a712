#!/usr/bin/env python3
"""Benchmark of the mixed-precision multigrid-preconditioned iterative refinement.

Workload (one "step" = one complete solve to relative FP64 residual 1e-10):
3D Poisson, 7-point finite differences, zero Dirichlet boundary, 255^3
interior points (16,581,375 DOF), f ~ U[-1, 1) from SplitMix64 seed 2 (seed
2 + rank on other ranks), u0 = 0.  Preconditioner: one V(2,2) cycle per IR
step, damped Jacobi omega = 0.8, full weighting / trilinear transfers, exact
3^3 base solve, every level stored in FP16 with FP32 sweep arithmetic (H_MG),
residual scaled by 2^14/||r||_inf before the cast; FP64 refinement.  The same
solve with all levels in FP64 (D_MG, no scaling) is timed beside it.

Metric: DOF/s to relative residual 1e-10 (whole job: DOF solved by all ranks
per second of the slowest rank).  Each step flushes L2 (256 MiB write) before
it starts; the inputs (b, u: 133 MB each in FP64) are also larger than L2.

JSON line keys follow the benchmark contract: value / ms_per_step from the
library's CUDA events around each solve (device time, inputs resident in
HBM), e2e through the same C-ABI call with pinned host buffers (H2D of b and
D2H of u inside the timed region), roofline of the dominant kernel from CUDA
events around every kernel of a profiled solve, cpu_baseline from the FP64
oracle on the host cores, clocks sampled with nvidia-smi during the timed
region.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DIM, N, SEED, TOL = 3, 255, 2, 1e-10
METRIC = "DOF/s to rel. residual 1e-10: mixed-FP16 MG-IR vs FP64 MG; stencil HBM % peak"
WORKLOAD = ("3D Poisson 7-point FDM, zero Dirichlet, 255^3 interior (16,581,375 DOF), f~U[-1,1) seed 2; "
            "H_MG: V(2,2) damped-Jacobi (omega 0.8) MG preconditioner with all 7 levels in FP16 "
            "(FP32 in-sweep accumulation), residual scaled by 2^14/||r||_inf before the FP16 cast, "
            "FP64 iterative refinement to rel. residual 1e-10; compared with all-FP64 MG (D_MG)")
# --op 1: the same line for the paper's trilinear Q1 finite-element operator (27-point)
WORKLOAD_Q1 = WORKLOAD.replace("3D Poisson 7-point FDM", "3D Poisson trilinear Q1 FEM (27-point, stiffness / h^3)")
GOLDEN_KEY = {0: "3d_n255_random_seed2", 1: "3d_n255_random_seed2_q1"}


def env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.rows, self.proc = [], None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(device)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def oracle_iters(name: str) -> int:
    with open(os.path.join(ROOT, "tests", "golden", "oracle_solves.json")) as f:
        return int(json.load(f)[name]["iters"])


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith(("model name", "cpu model")):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def cpu_oracle_sample(b, steps: int = 1, op: int = 0):
    """The FP64 oracle, as it stands, on the same 255^3 workload: one complete solve to
    relative residual 1e-10 (about 5 s on 16 host cores), timed; DOF/s = n^3 / time."""
    from oracle import oracle as O
    O.build()
    cores = os.cpu_count() or 1
    ts, iters = [], None
    for _ in range(steps):
        t = time.perf_counter()
        _, info, _ = O.ir_solve(b, nthreads=cores, op=op)
        ts.append(time.perf_counter() - t)
        iters = info["iters"]
        if not info["converged"]:
            raise RuntimeError(f"oracle solve did not converge: {info}")
    t_solve = min(ts)
    dofs = b.size / t_solve
    sample = (f"one complete FP64 oracle solve of the 255^3 workload ({iters} IR steps to 1e-10) on "
              f"{cores} threads of {cpu_model()}: {t_solve:.2f} s")
    return dofs, cores, sample, t_solve


def reference_arm(args):
    """--impl reference: the FP64 CPU oracle timed on the host cores (rank 0 only)."""
    import numpy as np  # noqa: F401
    from paper_2007_07539_gb300 import inputs as I
    rank = env_int("RANK", 0)
    if rank != 0:
        return 0
    b = I.random_rhs(DIM, N, SEED)
    for _ in range(args.warmup):
        cpu_oracle_sample(b, 1)
    vals, walls = [], []
    sample = cores = None
    for _ in range(args.steps):
        v, cores, sample, wall = cpu_oracle_sample(b, 1)
        vals.append(v)
        walls.append(wall)
    value = statistics.median(vals)
    line = {"metric": METRIC, "value": value, "unit": "DOF/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median(walls), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD.replace("H_MG", "reference: FP64 CPU oracle of the same method; H_MG")},
            "cpu_baseline": {"value": value, "unit": "DOF/s", "cores": cores, "kind": "oracle", "sample": sample,
                             "cpu_model": cpu_model()},
            "e2e": {"value": value, "unit": "DOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# The dominant kernel's DRAM traffic per launch comes from an ncu capture
# summarised in profiles/; it stands only while the kernel's sources are the
# ones that capture measured (their SHA-256 is recorded in the summary).
TRAFFIC_SUMMARY = os.path.join(ROOT, "profiles", "k_update_fp16_255cubed.md")
TRAFFIC_SOURCES = [os.path.join(ROOT, "paper_2007_07539_gb300", "csrc", f)
                   for f in ("mg_march.cuh", "mg_device.cuh", "mg_internal.h")]


def kernel_sources_sha256() -> str:
    import hashlib
    h = hashlib.sha256()
    for p in TRAFFIC_SOURCES:
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def profiled_traffic():
    """(bytes per launch, note): DRAM read + write bytes of the update kernel from
    the committed ncu summary, or (None, why) when absent or stale."""
    try:
        with open(TRAFFIC_SUMMARY) as f:
            kv = dict(ln.split(":", 1) for ln in f.read().splitlines() if ln.startswith(("source_sha256:", "dram_bytes_per_launch:")))
        if kv.get("source_sha256", "").strip() != kernel_sources_sha256():
            return None, "kernel sources changed since the ncu capture"
        return float(kv["dram_bytes_per_launch"]), os.path.relpath(TRAFFIC_SUMMARY, ROOT)
    except (OSError, KeyError, ValueError):
        return None, "no ncu summary"


def rank_max(x: float, world: int, device: str) -> float:
    """Max of x over the ranks of the default process group (the slowest rank's time)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, seconds: float, world: int, device: str) -> float:
    """Whole-job throughput: the units of all ranks (each rank solves its own
    instance of the same size, no data-path collective) over the slowest
    rank's time."""
    return world * units_per_rank / rank_max(seconds, world, device)


def extra_workloads(mg, I, torch, flush, quick=False):
    """Secondary measurements reported inside config (not the headline): the
    511^3 manufactured problem with the FP16/FP32/FP64 ladder against all-FP64
    MG, the four precision variants of Table 2 at 255^3, the batched workload (64 independent 3D instances, n log-uniform in
    [31, 255]) through mg_solve_batch against the same instances one by one,
    and a serving stream (Poisson arrivals at 0.8x the serial FP16 capacity,
    half 2D / half 3D) through mg_submit / mg_poll with p50 / p99 latency
    against serial all-FP64 solves of the same stream."""
    import numpy as np
    out = {}

    def solve_ms(h, b, u, k):
        ts, res = [], None
        for _ in range(k):
            flush.fill_(1)
            torch.cuda.synchronize()
            res = h.solve(b, u)
            if res["status"] != 0:
                raise RuntimeError(f"solve failed: {res}")
            ts.append(1e3 * res["seconds"])
        return statistics.median(ts), res

    # ---- 511^3, manufactured u = prod sin(pi x): HSD ladder vs D
    n = 511
    b = torch.from_numpy(I.manufactured_rhs(3, n)).cuda()
    u = torch.zeros_like(b)
    with mg.Hierarchy(mg.make_params(3, n, "HSD", zero_guess=1, tune=1)) as h:
        solve_ms(h, b, u, 1)
        t_h, r_h = solve_ms(h, b, u, 1 if quick else 3)
    with mg.Hierarchy(mg.make_params(3, n, "D", zero_guess=1, scaling=0, tune=1)) as h:
        solve_ms(h, b, u, 1)
        t_d, r_d = solve_ms(h, b, u, 1 if quick else 2)
    out["n511_manufactured"] = {"dof": n ** 3, "ladder": "FP16 on 511, 255; FP32 on 127..7; FP64 on 3",
                                "hsd_ms": t_h, "hsd_dofs": n ** 3 / (t_h * 1e-3), "hsd_iters": r_h["iters"],
                                "hsd_rel_res_true": r_h["rel_res_true"], "fp64_mg_ms": t_d,
                                "fp64_mg_iters": r_d["iters"], "speedup_vs_fp64_mg": t_d / t_h}
    del b, u
    torch.cuda.empty_cache()

    # ---- Table 2's four variants on the 255^3 random problem: D_MG (no scaling), H_MG,
    # HSD_MG and DSH_MG with the level split of Sec. 6 (HSD: FP64 base and level 1, FP32
    # level 2, FP16 above; DSH: the reverse, CG base solver in FP16, residual rescaled
    # into the FP16 levels)
    n = 255
    b = torch.from_numpy(I.random_rhs(3, n, 2)).cuda()
    u = torch.zeros_like(b)
    nlev = len(mg.level_count(n))
    variants = {"D_MG": ("D", dict(scaling=0)), "H_MG": ("H", {}),
                "HSD_MG": (mg.ladder("HSD", nlev, nlev - 3, 2), {}),
                "DSH_MG": (mg.ladder("DSH", nlev, nlev - 3, 2), dict(base_solver=1))}
    t2 = {}
    for name, (lad, kw) in variants.items():
        with mg.Hierarchy(mg.make_params(3, n, lad, zero_guess=1, tune=1, **kw)) as h:
            solve_ms(h, b, u, 1)
            t, r = solve_ms(h, b, u, 1 if quick else 3)
        t2[name] = {"ms": t, "iters": r["iters"], "dofs": n ** 3 / (t * 1e-3), "rel_res_true": r["rel_res_true"]}
    for name in t2:
        t2[name]["speedup_vs_D_MG"] = t2["D_MG"]["ms"] / t2[name]["ms"]
    out["table2_variants_255"] = t2
    del b, u
    torch.cuda.empty_cache()

    # ---- the paper's discretisation (Sec. 5): Q1 finite elements (27-point), 255^3.
    # (a) Table 2's variants on the random right-hand side from u0 = 0; (b) Table 3's
    # setting: manufactured load with k = 1 and 20, initial guess uniform in [0, 1),
    # IR steps to ||r||_2 <= 1e-10 ||b||_2 per variant
    n = 255
    b = torch.from_numpy(I.random_rhs(3, n, 2)).cuda()
    u = torch.zeros_like(b)
    q1 = {}
    for name, (lad, kw) in variants.items():
        with mg.Hierarchy(mg.make_params(3, n, lad, zero_guess=1, tune=1, op=1, **kw)) as h:
            solve_ms(h, b, u, 1)
            t, r = solve_ms(h, b, u, 1 if quick else 3)
        q1[name] = {"ms": t, "iters": r["iters"], "dofs": n ** 3 / (t * 1e-3), "rel_res_true": r["rel_res_true"]}
    for name in q1:
        q1[name]["speedup_vs_D_MG"] = q1["D_MG"]["ms"] / q1[name]["ms"]
    iters = {}
    u0 = torch.from_numpy(I.random_guess(3, n, 3)).cuda()
    for k in (1, 20):
        bk = torch.from_numpy(I.manufactured_load(3, n, k)).cuda()
        for name, (lad, kw) in variants.items():
            with mg.Hierarchy(mg.make_params(3, n, lad, op=1, **kw)) as h:
                u.copy_(u0)
                r = h.solve(bk, u)
            iters[f"k{k}_{name}"] = r["iters"]
    out["q1_fem_255"] = {"operator": "trilinear Q1 elements, 27-point, stiffness / h^3", "variants": q1,
                         "iters_manufactured_random_u0": iters}
    del b, u, u0
    torch.cuda.empty_cache()

    # ---- batched: 64 independent instances in one mg_solve_batch call
    work = I.batched_workload(count=16 if quick else 64)
    hs = [mg.Hierarchy(mg.make_params(3, nn, "H", zero_guess=1, tune=1)) for nn, _ in work]
    bs = [torch.from_numpy(I.random_rhs(3, nn, sd)).cuda() for nn, sd in work]
    us = [torch.zeros_like(x) for x in bs]
    dof = sum(nn ** 3 for nn, _ in work)
    t_one = 0.0
    for h, bb, uu in zip(hs, bs, us):  # one by one (also the warm-up)
        t_one += solve_ms(h, bb, uu, 1)[0]
    mg.solve_batch(hs, bs, us)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rb = mg.solve_batch(hs, bs, us)
    torch.cuda.synchronize()
    t_b = time.perf_counter() - t0
    for h in hs:
        h.close()
    del hs, bs, us
    out["batched_64"] = {"instances": len(work), "dof": dof, "sizes": sorted({nn for nn, _ in work}),
                         "batch_wall_ms": 1e3 * t_b, "batch_dofs": dof / t_b,
                         "one_by_one_device_ms": t_one, "one_by_one_dofs": dof / (t_one * 1e-3),
                         "all_converged": all(r["status"] == 0 for r in rb),
                         "level_synchronous_merged_launches": all(r["merged"] == 1 for r in rb),
                         "launches_per_solve": rb[0]["launches"],
                         "max_iters": max(r["iters"] for r in rb)}

    # ---- serving stream: Poisson arrivals of 2D / 3D requests.  The server keeps up to
    # four pooled hierarchies per request shape (plans and graphs resident; working arenas
    # from the device-memory pool per request, cached while memory allows); a request goes
    # to its shape's hierarchies in turn and queues behind a busy one.  The pool's budget
    # bounds the working memory of everything admitted.
    reqs = I.serving_workload(count=48 if quick else 512)
    shapes = sorted({(q["dim"], q["n"]) for q in reqs})
    t16, t64 = {}, {}
    for d, nn in shapes:  # serial references per request shape (median of the shape's solves)
        bb = torch.from_numpy(I.random_rhs(d, nn, 5000)).cuda()
        uu = torch.zeros_like(bb)
        with mg.Hierarchy(mg.make_params(d, nn, "HS", zero_guess=1)) as h:
            solve_ms(h, bb, uu, 1)
            t16[(d, nn)] = solve_ms(h, bb, uu, 3)[0]
        with mg.Hierarchy(mg.make_params(d, nn, "D", zero_guess=1, scaling=0)) as h:
            solve_ms(h, bb, uu, 1)
            t64[(d, nn)] = solve_ms(h, bb, uu, 1)[0]
        del bb, uu
    t_fp16 = sum(t16[(q["dim"], q["n"])] for q in reqs)
    t_fp64 = sum(t64[(q["dim"], q["n"])] for q in reqs)
    rate = 0.8 * len(reqs) / (t_fp16 * 1e-3)
    mean_gap = reqs[-1]["arrival_s"] / len(reqs)  # the workload's exponential gaps rescaled to this rate
    arr = [q["arrival_s"] / (mean_gap * rate) for q in reqs]
    budget = 4 << 30
    mg.serve_configure(budget, 16)
    per_shape = 4
    pool_h = {sh: [mg.Hierarchy(mg.make_params(sh[0], sh[1], "HS", zero_guess=1, pooled=1))
                   for _ in range(per_shape)] for sh in shapes}
    turn = {sh: 0 for sh in shapes}
    served = []
    for q in reqs:
        sh = (q["dim"], q["n"])
        served.append(pool_h[sh][turn[sh] % per_shape])
        turn[sh] += 1
    bufs = [torch.from_numpy(I.random_rhs(q["dim"], q["n"], q["seed"])).cuda() for q in reqs]
    us = [torch.zeros_like(bb) for bb in bufs]
    for sh, hl in pool_h.items():  # warm-up: one solve per hierarchy builds its graph
        bb = torch.from_numpy(I.random_rhs(sh[0], sh[1], 1)).cuda()
        for h in hl:
            h.solve(bb, torch.zeros_like(bb))
        del bb
    torch.cuda.synchronize()
    dof_s = sum(q["n"] ** q["dim"] for q in reqs)

    def stream(merge):
        """One pass of the request stream; returns its latency / throughput / pool record."""
        mg.serve_options(merge)
        torch.cuda.synchronize()
        st0 = mg.serve_stats()
        t0 = time.perf_counter()
        pending, lat, slow, statuses = {}, [], [], []
        i = 0
        while i < len(reqs) or pending:
            now = time.perf_counter() - t0
            while i < len(reqs) and arr[i] <= now:
                pending[i] = served[i].submit(bufs[i], us[i])
                i += 1
            for j in list(pending):
                r = served[j].poll(pending[j])
                if r is not None:
                    lat.append(time.perf_counter() - t0 - arr[j])
                    slow.append(lat[-1] / (1e-3 * t16[(reqs[j]["dim"], reqs[j]["n"])]))
                    statuses.append(r["status"])
                    del pending[j]
            time.sleep(0.0002)
        t_s = time.perf_counter() - t0
        st1 = mg.serve_stats()
        mg.serve_options(False)
        lat_ms = sorted(1e3 * x for x in lat)
        return {"p50_ms": float(np.percentile(lat_ms, 50)), "p99_ms": float(np.percentile(lat_ms, 99)),
                "slowdown_p50": float(np.percentile(slow, 50)), "slowdown_p99": float(np.percentile(slow, 99)),
                "slowdown": "latency over the request shape's serial device time",
                "served_dofs": dof_s / t_s, "wall_s": t_s, "all_ok": all(x == 0 for x in statuses),
                "pool_peak_reserved_bytes": st1["peak_reserved_bytes"], "pool_peak_in_use_bytes": st1["peak_in_use_bytes"],
                "requests_that_waited_for_memory": st1["memory_waits"] - st0["memory_waits"],
                "arena_reuses": st1["arena_reuses"] - st0["arena_reuses"],
                "arena_evictions": st1["arena_evictions"] - st0["arena_evictions"],
                "merged_requests": st1["merged_requests"] - st0["merged_requests"],
                "merged_groups": st1["merged_groups"] - st0["merged_groups"], "peak_inflight": st1["peak_inflight"]}

    plain = stream(False)
    merged = stream(True)  # requests admitted together run as level-synchronous groups
    out["serving"] = dict(plain, requests=len(reqs), ladder="FP16 fine / FP32 coarse (HS)", rate_per_s=rate,
                          serial_fp16_device_ms=t_fp16, serial_fp64_device_ms=t_fp64,
                          serial_fp64_dofs=dof_s / (t_fp64 * 1e-3),
                          serial_times="per request shape, median of 3 FP16 / 1 FP64 device-timed solves, summed "
                                       "over the stream",
                          pool_budget_bytes=budget, hierarchies=per_shape * len(shapes), shapes=len(shapes),
                          with_merged_groups=merged)
    for hl in pool_h.values():
        for h in hl:
            h.close()
    del served, pool_h, bufs, us
    mg.serve_configure(0, 16)
    torch.cuda.empty_cache()

    # ---- vector bandwidth versus size (Sec. 8.2, Fig. 6): y <- a x + y, 3 bytes-moved
    # vectors per value (read x, read y, write y), event-timed on torch's stream
    dtypes = {mg.FP16: torch.float16, mg.BF16: torch.bfloat16, mg.FP32: torch.float32, mg.FP64: torch.float64}
    axpy = {}
    for prec, tdt in dtypes.items():
        pts = []
        for lg in range(12, 29, 2):
            nv = 1 << lg
            xv = torch.ones(nv, dtype=tdt, device="cuda")
            yv = torch.zeros(nv, dtype=tdt, device="cuda")
            reps = 20 if nv < (1 << 24) else 5
            mg.axpy(prec, 0.5, xv, yv)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                mg.axpy(prec, 0.5, xv, yv)
            e1.record()
            e1.synchronize()
            sec = e0.elapsed_time(e1) * 1e-3 / reps
            pts.append([nv, round(3 * nv * xv.element_size() / sec / 1e9, 1)])
            del xv, yv
        axpy[["fp64", "fp32", "fp16", "bf16"][prec]] = pts
    out["axpy_gbs_vs_n"] = axpy
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the 511^3, batched and serving measurements")
    ap.add_argument("--no-tune", action="store_true", help="tile shapes from the wave model instead of the autotuner")
    ap.add_argument("--kernel-dump", default=None, help="write every kernel's profiled time to this JSON file")
    ap.add_argument("--ncu-case", action="store_true",
                    help="only two solves of the workload, kernel by kernel (a small launch list for ncu captures)")
    ap.add_argument("--ncu-ladder", default="H", choices=["H", "D"],
                    help="with --ncu-case: H (FP16 levels, the default) or D (all-FP64 MG, no scaling)")
    ap.add_argument("--op", type=int, default=0, choices=[0, 1],
                    help="operator: 0 the 7-point finite-difference stencil (the headline workload), "
                         "1 the trilinear Q1 finite elements of Sec. 5")
    ap.add_argument("--graph", type=int, default=1,
                    help="1: each solve is one CUDA graph with a device-side IR loop; 0: kernels launched one "
                         "by one from the host loop (ncu cannot profile kernels inside conditional graphs)")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)

    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2007_07539_gb300 import inputs as I
    from paper_2007_07539_gb300 import mg

    world = env_int("WORLD_SIZE", 1)
    rank = env_int("RANK", 0)
    local = env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    def allmax(x: float) -> float:
        return rank_max(x, world, "cuda")

    ndof = N**DIM
    b = I.random_rhs(DIM, N, SEED + rank)
    bd = torch.from_numpy(b).cuda()
    ud = torch.zeros_like(bd)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    graph = 0 if args.ncu_case else args.graph
    # tile shapes of the stencil kernels autotuned at creation (results do not depend on them)
    tune = 0 if args.no_tune else 1
    # fuse_pre = 2: the autotuner also picks, per level, one fused pre-smoothing + restriction
    # pass or two launches (sweeps per launch)
    hH = mg.Hierarchy(mg.make_params(DIM, N, "H", zero_guess=1, graph=graph, tune=tune, op=args.op,
                                     fuse_pre=2 if tune and args.op == 0 else 0))
    hD = mg.Hierarchy(mg.make_params(DIM, N, "D", zero_guess=1, scaling=0, graph=graph, tune=tune, op=args.op))

    def run(h, bb, uu, k):
        secs, res = [], None
        for _ in range(k):
            flush.fill_(1)
            torch.cuda.synchronize()
            res = h.solve(bb, uu)
            if res["status"] != 0:
                raise RuntimeError(f"solve failed: {res}")
            secs.append(res["seconds"])
        return secs, res

    if args.ncu_case:
        run(hD if args.ncu_ladder == "D" else hH, bd, ud, 2)
        torch.cuda.synchronize()
        print(json.dumps({"ncu_case": f"2 {'FP64' if args.ncu_ladder == 'D' else 'FP16'} solves done"}), flush=True)
        return 0
    run(hH, bd, ud, args.warmup)
    run(hD, bd, ud, max(1, min(args.warmup, 2)))

    # timed region: H_MG solves, device time from the library's CUDA events
    barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    t_wall = time.perf_counter()
    secs, resH = run(hH, bd, ud, args.steps)
    torch.cuda.synchronize()
    barrier()
    wall = time.perf_counter() - t_wall
    clocks = clk.stop()
    launches = resH["launches"] * args.steps
    t_dev = allmax(sum(secs))
    value = whole_job_rate(ndof * args.steps, sum(secs), world, "cuda")
    uH = ud.cpu().numpy().copy()

    # all-FP64 MG on the same grid
    secsD, resD = run(hD, bd, ud, max(1, min(args.steps, 3)))
    tD = allmax(sum(secsD) / len(secsD))
    valueD = world * ndof / tD
    uD = ud.cpu().numpy()
    rel_diff = float(np.linalg.norm(uH - uD) / np.linalg.norm(uD))

    # end to end: the same C-ABI call on pinned host buffers (H2D of b, D2H of u timed)
    bh = torch.from_numpy(b).pin_memory()
    uh = torch.zeros_like(bh).pin_memory()
    run(hH, bh, uh, 1)
    secsE, _ = run(hH, bh, uh, args.steps)
    e2e = whole_job_rate(ndof * args.steps, sum(secsE), world, "cuda")

    # per-kernel device times of one profiled solve (events around every kernel)
    resP, ktimes = hH.profile_solve(bd, ud)
    if args.kernel_dump and rank == 0:
        with open(args.kernel_dump, "w") as f:
            json.dump({"result": resP, "kernels": ktimes}, f, indent=1)
    top = max(ktimes, key=lambda k: k["total_ms"])
    if args.op != 0:
        traffic, traffic_note = None, "the ncu summary covers the finite-difference workload"
    else:
        traffic, traffic_note = profiled_traffic() if top["kind"] == 5 else (None, "dominant kernel is not the update")
    tot_ms = sum(k["total_ms"] for k in ktimes)
    peak, peak_kind = measured_peaks()
    ach = top["bytes"] * top["launches"] / (top["total_ms"] * 1e-3) / 1e9
    finest = max(k["level"] for k in ktimes)
    sweeps = [k for k in ktimes if k["kind"] == 0 and k["level"] == finest and k["mode"] in (0, 1, 3)]
    sweep_bytes = sum(k["bytes"] * k["launches"] for k in sweeps)
    sweep_ms = sum(k["total_ms"] for k in sweeps)
    byshare = sorted(ktimes, key=lambda k: -k["total_ms"])[:8]

    def finest_frac(kind, mode=None):
        """Algorithmic GB/s of a finest-level kernel over the measured peak (CUDA events)."""
        ks = [k for k in ktimes if k["level"] == finest and k["kind"] == kind and (mode is None or k["mode"] == mode)]
        ms = sum(k["total_ms"] for k in ks)
        if not ks or ms <= 0:
            return None
        return round(sum(k["bytes"] * k["launches"] for k in ks) / (ms * 1e-3) / 1e9 / peak, 3)

    line = {
        "metric": METRIC, "value": value, "unit": "DOF/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_dev / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f16 storage / f32 sweeps / f64 refinement",
        "data": "synthetic",
        "config": {"workload": WORKLOAD_Q1 if args.op == 1 else WORKLOAD, "dof": ndof,
                   "iters_fp16": resH["iters"], "iters_fp64": resD["iters"],
                   "oracle_iters": oracle_iters(GOLDEN_KEY[args.op]),
                   "rel_res_true_fp16": resH["rel_res_true"], "rel_res_true_fp64": resD["rel_res_true"],
                   "fp64_mg_dofs": valueD, "fp64_mg_ms": 1e3 * tD, "speedup_fp16_vs_fp64": value / valueD,
                   "rel_diff_u_fp16_vs_fp64": rel_diff, "l2": "256 MiB L2 flush before every step; "
                   "b and u (133 MB each) exceed the 129 MB L2", "wall_s_timed_region": wall,
                   "parallelism": f"{world} independent instance(s), one per GPU, no collective on the data path",
                   "tile_shapes": "autotuned at creation" if tune else "wave model",
                   "pre_smoothing_launches_per_level": {hH.level_info(l)["n"]: hH.level_info(l)["pre_launches"]
                                                        for l in range(hH.nlev) if hH.level_info(l)["tail_ctas"] == 0},
                   "hbm_frac_finest_jacobi": finest_frac(0, 0), "hbm_frac_finest_zero_start": finest_frac(0, 1),
                   "hbm_frac_finest_residual_restrict": finest_frac(0, 3), "hbm_frac_finest_prolong": finest_frac(2),
                   "hbm_frac_ir_update": finest_frac(5),
                   "finest_sweeps_gbs": sweep_bytes / (sweep_ms * 1e-3) / 1e9 if sweep_ms else None,
                   "kernel_shares": [{"kernel": f"{k['name']}@L{k['level']}", "ms": round(k["total_ms"], 4),
                                      "share": round(k["total_ms"] / tot_ms, 4),
                                      "gbs": round(k["bytes"] * k["launches"] / max(k["total_ms"], 1e-9) / 1e6, 1)}
                                     for k in byshare]},
        "roofline": {"bound": "hbm", "kernel": f"{top['name']} level {top['level']}", "achieved": ach,
                     "peak": peak, "peak_source": peak_kind, "unit": "GB/s", "frac": ach / peak,
                     "traffic": traffic, "traffic_source": traffic_note, "bytes_per_launch": top["bytes"],
                     "avg_launch_ms": top["total_ms"] / max(top["launches"], 1)},
        "e2e": {"value": e2e, "unit": "DOF/s", "h2d_bytes_per_step": ndof * 8, "d2h_bytes_per_step": ndof * 8},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    if rank == 0 and world == 1 and not args.no_extras and args.op == 0:
        hH.close()
        hD.close()
        ex = extra_workloads(mg, I, torch, flush)
        # the headline secondary figures as short top-level keys (the full records follow in extras)
        c, e5 = line["config"], ex["n511_manufactured"]
        c.update({"n511_hsd_ms": e5["hsd_ms"], "n511_fp64_ms": e5["fp64_mg_ms"],
                  "n511_speedup": e5["speedup_vs_fp64_mg"], "n511_iters": e5["hsd_iters"],
                  "n511_fp64_iters": e5["fp64_mg_iters"], "n511_oracle_iters": oracle_iters("3d_n511_manufactured"),
                  "batched_dofs": ex["batched_64"]["batch_dofs"],
                  "serving_p50_ms": ex["serving"]["p50_ms"], "serving_p99_ms": ex["serving"]["p99_ms"],
                  "serving_dofs": ex["serving"]["served_dofs"],
                  "serving_merged_p50_ms": ex["serving"]["with_merged_groups"]["p50_ms"],
                  "serving_merged_p99_ms": ex["serving"]["with_merged_groups"]["p99_ms"],
                  "serving_merged_dofs": ex["serving"]["with_merged_groups"]["served_dofs"],
                  "serving_pool_peak_bytes": ex["serving"]["pool_peak_reserved_bytes"],
                  "serving_pool_budget_bytes": ex["serving"]["pool_budget_bytes"]})
        c["extras"] = ex
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, cores, sample, _ = cpu_oracle_sample(b, 1, args.op)
        line["cpu_baseline"] = {"value": v, "unit": "DOF/s", "cores": cores, "kind": "oracle", "sample": sample,
                                "cpu_model": cpu_model()}
    if rank == 0:
        print(json.dumps(line), flush=True)
    hH.close()
    hD.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
