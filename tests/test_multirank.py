"""The N > 1 path of the benchmark on CPU: gloo ranks (world size 2) run the
same whole-job aggregation the GPU ranks run over NCCL.  Each rank solves an
independent instance, so the only collective is the max of the ranks' times
(and the barrier around the timed region)."""
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    dist.barrier()
    secs = [1.0, 3.0][rank]                    # the second rank is the slow one
    rate = bench.whole_job_rate(100.0, secs, world, "cpu")
    tmax = bench.rank_max(secs, world, "cpu")
    dist.barrier()
    out.put((rank, rate, tmax))
    dist.destroy_process_group()


def test_whole_job_rate_over_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, rate, tmax in res:
        assert tmax == 3.0                      # slowest rank's time on every rank
        assert rate == pytest.approx(2 * 100.0 / 3.0)  # units of all ranks / slowest time


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.rank_max(2.5, 1, "cpu") == 2.5
    assert bench.whole_job_rate(10.0, 2.0, 1, "cpu") == 5.0


def test_reference_arm_other_ranks_exit_without_work(monkeypatch):
    """Under torchrun only rank 0 runs the CPU oracle; other ranks return 0 at once."""
    import bench
    monkeypatch.setenv("RANK", "1")

    class A:
        warmup, steps, gpus = 3, 1, 2
    assert bench.reference_arm(A()) == 0
