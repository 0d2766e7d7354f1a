"""The multi-GPU path is replicas only: every rank runs its own solves, the
job time is the slowest rank's and the job's points are the sum over ranks.
Exercised here with two gloo ranks on CPU (no GPU, no collective in the data
path)."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, pts = bench.reduce_over_ranks(10.0 + 5.0 * rank, 1000.0 * (rank + 1), torch.device("cpu"))
    out[rank] = (ms, pts)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_timing_is_max_and_points_are_summed():
    import torch.multiprocessing as mp
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        assert out[r] == (15.0, 3000.0)


def test_single_process_passes_through():
    import torch
    import bench
    assert bench.reduce_over_ranks(3.5, 42.0, torch.device("cpu")) == (3.5, 42.0)
