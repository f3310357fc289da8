"""The benchmark's multi-rank host logic on CPU with the gloo backend and two
ranks (no GPU): the slowest rank's time is what every rank reports, the
whole-job rate counts every rank's replica, and the reference arm runs on rank
0 only."""
import contextlib
import io
import multiprocessing as mp
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, world, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, ms))


def test_max_over_ranks_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == {0: 15.0, 1: 15.0}


def test_single_rank_and_rate():
    import bench
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    # two replicas of 300,763 dofs in 0.1 ms each: 6.015 GDoF/s for the job
    assert abs(bench.whole_job_rate(300763, 2, 1e-4) - 6.01526) < 1e-4


def test_reference_arm_runs_on_rank_0_only(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    out = io.StringIO()
    with contextlib.redirect_stdout(out):
        bench.run_reference(bench.argparse.Namespace(p=4, elements=64, op="stiffness", steps=1,
                                                     warmup=0, gpus=2, prec="fp32"))
    assert out.getvalue() == ""
