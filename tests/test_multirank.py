"""Multi-rank logic of bench.py on the CPU (gloo, world size 2, spawned processes).  Under torchrun
every rank advances its own replica (the time step has no data-path exchange), and each timed
duration is reduced with MAX so that the reported throughput is that of the slowest replica; the
reference arm runs on rank 0 only."""
import argparse
import multiprocessing as mp
import os
import socket

import pytest


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    import bench
    a = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")   # rank 1 is the slowest
    b = bench.max_over_ranks(7.0 - rank, dist, "cpu")          # rank 0 is the slowest
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, a, b))


def test_durations_are_reduced_to_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        res = sorted(q.get(timeout=180) for _ in procs)
    finally:
        for p in procs:
            p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    assert res == [(0, 15.0, 7.0), (1, 15.0, 7.0)]


def test_single_process_reduction_is_identity():
    import bench
    assert bench.max_over_ranks(3.25) == 3.25


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    args = argparse.Namespace(config="ricker128", steps=3, warmup=1, gpus=2)
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""
