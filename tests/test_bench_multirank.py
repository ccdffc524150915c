"""The multi-rank (replica) logic of bench.py on the CPU: two gloo ranks, as the
benchmark runs under torchrun with one rank per GPU.  The timing reduction takes
the maximum over ranks, the whole-job rate counts every rank's units over that
time, each rank draws its own inputs, and the reference arm does its work on rank
0 only (other ranks return without work)."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    times = [10.0 + rank, 5.0 - rank]          # rank 1 is slower on the first, faster on the second
    red = bench._max_over_ranks(times, world, "cpu")
    rate = bench._job_rate(world, 1000, 4, red[0])
    pos, _ = bench._inputs("open_uniform_n4096_mesh8_p4_fp64", rank)

    class A:
        workload = "open_uniform_n4096_mesh8_p4_fp64"
        steps, warmup = 1, 0
    ref = bench.run_reference(A(), rank, world) if rank == 1 else None
    dist.barrier()
    out[rank] = (red, rate, float(pos[0, 0]), ref)
    dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    world = 2
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(world, _port(), out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    for r in range(world):
        red, rate, _, _ = res[r]
        assert red == [11.0, 5.0]
        assert rate == pytest.approx(world * 1000 * 4 / (11.0e-3))
    assert res[0][2] != res[1][2]     # each replica draws its own inputs
    assert res[1][3] == 0             # the reference arm does nothing on rank 1
