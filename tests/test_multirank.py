"""N > 1 path of bench.py on CPU ranks (gloo, world size 2): every rank works on
its own instance, the job total sums the nonzeros and takes the slowest rank."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    nnz = 1000 * (rank + 1)
    t = 0.5 + rank
    tot, tmax = bench.aggregate(nnz, t, world, "cpu")
    dist.barrier()
    out[rank] = (tot, tmax)
    dist.destroy_process_group()


def test_aggregate_two_gloo_ranks():
    import torch.multiprocessing as mp
    mgr = mp.Manager()
    out = mgr.dict()
    port = _free_port()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    assert out[0] == (3000.0, 1.5) and out[1] == (3000.0, 1.5)


def test_aggregate_single_rank():
    import bench
    assert bench.aggregate(7, 0.25, 1, "cpu") == (7.0, 0.25)
