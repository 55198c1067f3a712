"""Writes tests/golden/oracle_solves.json: iteration counts and residual histories
of the FP64 oracle (oracle/) on the benchmark workloads.  Calls only the oracle
and the seeded input recipes; run it after any change to either:

    python tests/golden/make_golden.py [name ...]   (only the named entries; the others are kept)
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2007_07539_gb300 import inputs as I  # noqa: E402

WORKLOADS = {
    "3d_n255_random_seed2": dict(dim=3, n=255, rhs=("random", 2)),
    "2d_n127_manufactured": dict(dim=2, n=127, rhs=("manufactured", 1)),
    "3d_n63_random_seed2": dict(dim=3, n=63, rhs=("random", 2)),
    "3d_n511_manufactured": dict(dim=3, n=511, rhs=("manufactured", 1)),
    "3d_n255_random_seed2_q1": dict(dim=3, n=255, rhs=("random", 2), op=1),
    "3d_n511_manufactured_w": dict(dim=3, n=511, rhs=("manufactured", 1), gamma=2),
    # the oracle's low-precision emulation (a diagnostic of the FP64 oracle, Sec. 6 ladders):
    # HSD_MG with FP16 on the two finest levels, FP32 between, FP64 base, W-cycle, with the
    # power-of-two scale of the previous step (reading R21), as the library runs it by default
    "3d_n511_manufactured_w_hsd_emulated": dict(dim=3, n=511, rhs=("manufactured", 1), gamma=2,
                                                ladder="HSD", scale_ahead=1),
}

FP64, FP32, FP16 = 0, 1, 2


def ladder(name, nlev):
    """Per-level storage formats, coarsest first: HSD = FP64 base, FP32 between, FP16 on
    the two finest levels (Table 2)."""
    assert name == "HSD"
    return [FP64] + [FP32] * (nlev - 3) + [FP16, FP16]


def rhs(w):
    kind, arg = w["rhs"]
    if kind == "random":
        return I.random_rhs(w["dim"], w["n"], arg)
    return I.manufactured_rhs(w["dim"], w["n"], arg)


def main(only=None):
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_solves.json")
    out = {}
    if only and os.path.exists(path):
        with open(path) as f:
            out = json.load(f)
    for name, w in WORKLOADS.items():
        if only and name not in only:
            continue
        t = time.time()
        op, gamma = w.get("op", 0), w.get("gamma", 1)
        kw = {}
        if "ladder" in w:
            kw = dict(prec=ladder(w["ladder"], len(O.level_sizes(w["n"]))), scale_ahead=w.get("scale_ahead", 0))
        _, info, hist = O.ir_solve(rhs(w), scaling=1, nthreads=os.cpu_count() or 1, op=op, gamma=gamma, **kw)
        out[name] = dict(dim=w["dim"], n=w["n"], rhs=list(w["rhs"]), iters=info["iters"],
                         rel_res_true=info["rel_res_true"], history=[float(x) for x in hist],
                         params=(f"emulated {w['ladder']} ladder, " if "ladder" in w else "")
                         + ("W(2,2)" if gamma == 2 else "V(2,2)")
                         + ", omega 0.8, damped Jacobi, FW/linear transfers, exact base solve, "
                                "alpha = ||r||_inf, rel. tol 1e-10, u0 = 0, operator "
                                + ("Q1 finite elements / h^d" if op == 1 else "finite differences"))
        print(name, info["iters"], f"{time.time() - t:.1f}s", flush=True)
    with open(path, "w") as f:
        json.dump({k: out[k] for k in WORKLOADS if k in out}, f, indent=1)


if __name__ == "__main__":
    main(sys.argv[1:] or None)
