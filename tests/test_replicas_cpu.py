"""The replica path of bench.py (one independent model per rank, no data-path
collective): the job time is the slowest rank's and the throughput counts every
rank's evaluations.  Two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, v = bench.job_throughput(100.0 * (rank + 1), 6.6e11, 5, world, dist)
    out[rank] = (t, v)
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    world = 2
    # spawn, not fork: this process already runs torch's threads
    out = mp.get_context("spawn").Manager().dict()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        t, v = out[r]
        assert t == 200.0
        assert v == pytest.approx(world * 6.6e11 * 5 / 0.2)
