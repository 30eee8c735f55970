"""Multi-process (N > 1) path of bench.py on CPU: two gloo ranks, each timing
its own replica; the job's time is the slowest rank's and its work the sum."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, results):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dist.barrier()
    ms = [120.0, 150.0][rank]
    units = [1000.0, 1000.0][rank]
    results[rank] = bench.over_ranks(ms, units, dist)
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_slowest_time_and_sum_work():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        results = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, results)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        for r in range(2):
            ms_max, units, value = results[r]
            assert ms_max == 150.0
            assert units == 2000.0
            assert value == pytest.approx(2000.0 / 0.150)


def test_single_process_is_unchanged():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.over_ranks(200.0, 500.0) == (200.0, 500.0, 2500.0)
