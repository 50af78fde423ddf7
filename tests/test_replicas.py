"""The N > 1 path of bench.py: one replica per GPU, no data exchange; the job's
time is the slowest rank's (a max all-reduce) and its throughput the units of
every rank over that time.  Two gloo ranks on the CPU exercise the same calls
the NCCL ranks make."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 100.0 + 25.0 * rank            # rank 1 is the slow one
    total = bench.reduce_max(local_ms, dist)
    dist.barrier()
    q.put((rank, total, bench.job_value(world, 20, total)))
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    world, port = 2, _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, total, value in got:
        assert total == 125.0
        assert value == pytest.approx(2 * 20 / 0.125)


def test_single_process_helpers():
    assert bench.reduce_max(3.5, None) == 3.5
    assert bench.job_value(1, 200, 680.0) == pytest.approx(200 / 0.68)
