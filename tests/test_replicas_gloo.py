"""The multi-GPU form is replicas (every rank runs its own PCAs, no data-path exchange):
the job's time is the slowest rank's and its throughput counts every rank's PCAs.  The
host logic of that reduction runs here as two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 100.0 + 7.0 * rank                       # rank 1 is the slower one
        slowest = bench.max_over_ranks(ms, dist, world, torch.device("cpu"))
        value = bench.job_throughput(world, 50, slowest)
        dist.barrier()
        with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
            f.write(f"{slowest!r} {value!r}\n")
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    rows = [open(tmp_path / f"rank{r}.txt").read().split() for r in range(world)]
    for slowest, value in rows:
        assert float(slowest) == 107.0                         # max over ranks, seen by every rank
        assert abs(float(value) - world * 50 / 0.107) < 1e-9   # every rank's PCAs over that time


def test_one_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, None, 1, None) == 3.25
    assert bench.job_throughput(1, 200, 684.0) == 200 / 0.684
