"""Host logic of bench.py's multi-GPU mode on CPU ranks (gloo, world size 2).

The solve does not exchange data across ranks: for one LP each rank runs its
own replica and only the timing is combined (maximum over ranks); value =
total iterations / that maximum.  The sweep's independent LPs are dealt out
whole (deal_lps) and only the timing and the status counts are combined.
These tests run that logic with two CPU processes.
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


def test_deal_lps_partitions_and_balances():
    """The sweep's independent LPs are dealt out whole: every LP to exactly one
    rank, the same answer on every rank, loads within the largest LP of each
    other (greedy largest-first)."""
    import bench
    from synthetic.targets import sweep_workloads
    work = [w.n ** 3 * w.n_angles for w in sweep_workloads()]
    for world in (1, 2, 3, 4, 8):
        shares = [bench.deal_lps(work, world, r) for r in range(world)]
        flat = sorted(i for s in shares for i in s)
        assert flat == list(range(len(work)))
        loads = [sum(work[i] for i in s) for s in shares]
        assert max(loads) - min(loads) <= max(work)
    assert bench.deal_lps(work, 1, 0) == list(range(len(work)))


def _sweep_worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local = {"optimal": 3, "iteration_limit": 1} if rank == 0 else {"optimal": 1, "primal_infeasible": 2}
    t, counts, iters = bench.combine_sweep(10.0 + 5.0 * rank, local, 1000 * (rank + 1), dist,
                                           torch.device("cpu"))
    out[rank] = (t, counts, iters)
    dist.barrier()
    dist.destroy_process_group()


def test_sweep_figures_combine_over_ranks():
    """Two CPU ranks each solving their share of the sweep: the sweep's time is
    the slowest rank's, the status counts and iterations are summed."""
    world = 2
    port = _free_port()
    manager = mp.get_context("spawn").Manager()
    out = manager.dict()
    mp.spawn(_sweep_worker, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        t, counts, iters = out[r]
        assert t == 15.0 and iters == 3000
        assert counts == {"optimal": 4, "primal_infeasible": 2, "iteration_limit": 1}
    import bench
    assert bench.combine_sweep(2.5, {"optimal": 2, "iteration_limit": 0}, 7, None) == (2.5, {"optimal": 2}, 7)
