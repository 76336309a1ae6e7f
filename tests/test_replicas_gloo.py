"""Host logic of bench.py's multi-GPU mode on CPU ranks (gloo, world size 2).

The solve does not exchange data across ranks: each rank runs its own replica
and only the timing is combined (maximum over ranks); value = total
iterations / that maximum.  These tests run that logic with two CPU processes.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    w, r, l = bench.dist_env()
    assert (w, r, l) == (world, rank, rank)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    elapsed = 1.0 + rank           # rank 1 is the slowest
    t_max = bench.max_over_ranks(elapsed, dist, torch.device("cpu"))
    out[rank] = t_max
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_weak_scaling_value():
    world = 2
    port = _free_port()
    manager = mp.get_context("spawn").Manager()   # no fork of this multi-threaded process
    out = manager.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    assert out[0] == out[1] == 2.0
    iters_per_rank = 256
    value = iters_per_rank * world / out[0]      # what bench.py reports
    assert value == 256.0


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, None) == 3.5
    assert bench.init_dist(1, "gloo") is None
