"""The multi-rank bookkeeping of bench.py on CPU: two gloo ranks, the job
time is the slowest rank's and the job value counts every rank's replica
(weak scaling, no data-path collective)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [12.5, 20.0][rank]
    out[rank] = bench.max_over_ranks(ms, dist, device="cpu")
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world = 2
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    assert out[0] == 20.0 and out[1] == 20.0


def test_job_value_counts_every_replica():
    import bench
    one = bench.job_value(1000, 5, 10, 1, 50.0)
    two = bench.job_value(1000, 5, 10, 2, 50.0)
    assert two == 2 * one
    assert bench.max_over_ranks(7.0, None) == 7.0
