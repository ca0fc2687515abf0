"""The N > 1 path of the benchmark on CPU: two gloo ranks, each a replica (no data-path collective);
the job time is the slowest rank's and the throughput counts both ranks' points."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    total = 100.0 if rank == 0 else 150.0   # rank 1 is the slow one
    res = bench.aggregate_replicas(total, pts=1e6, K=10, world=world, dist=dist, device="cpu")
    out[rank] = res
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank():
    import torch.multiprocessing as mp
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
    for r in (0, 1):
        total, ms, value = out[r]
        assert total == 150.0 and ms == 15.0
        assert abs(value - 2 * 1e6 * 10 / 0.150 / 1e6) < 1e-9
