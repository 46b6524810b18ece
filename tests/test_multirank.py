"""The N > 1 path of the benchmark on CPU ranks (gloo, world size 2): every rank runs its own replica of
the workload (tracers are independent, Sec. 3), the timing is the MAX over ranks, the reported value is
the work of all ranks over that time, and only rank 0 prints; the reference arm runs on rank 0 alone."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    slowest = bench.max_over_ranks(1.5 + rank, world, device="cpu")   # rank 1 is the slow one
    nan_ok = bench.max_over_ranks(0.25 * (rank + 1), world, device="cpu")
    dist.barrier()
    out.put((rank, slowest, nan_ok))
    dist.destroy_process_group()


def test_max_over_ranks_on_two_gloo_ranks():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, 2.5, 0.5), (1, 2.5, 0.5)]


def test_single_rank_is_the_identity():
    import bench

    assert bench.max_over_ranks(3.25, 1) == 3.25


def test_reference_arm_runs_on_rank_zero_only(capsys):
    import argparse

    import bench

    ns = argparse.Namespace(steps=1, warmup=0, config="c2", gpus=2)
    bench.reference_arm(ns, rank=1, world=2)      # rank 1: no work, no output
    assert capsys.readouterr().out == ""
