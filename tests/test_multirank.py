"""Replica ranks (bench.py under torchrun): the whole-job number takes the
slowest rank's time and the DoFs of all ranks.  Two gloo ranks on CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 10.0 + 5.0 * rank           # rank 1 is slower
    dofs = 1000 * (rank + 1)
    t, n = bench.aggregate_ranks(ms, dofs, dist, torch.device("cpu"))
    out[rank] = (t, n)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate():
    mgr = mp.Manager()
    out = mgr.dict()
    port = _free_port()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    assert out[0] == out[1] == (15.0, 3000.0)


def test_single_rank_passthrough():
    import bench
    assert bench.aggregate_ranks(7.5, 123) == (7.5, 123.0)
