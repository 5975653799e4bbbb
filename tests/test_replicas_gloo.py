"""Multi-GPU is replicas only (no data-path collective): the N-rank launch of
bench.py, its barrier and the max-over-ranks timing, checked with two gloo
ranks on CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    r, w, l = bench.dist_env()
    assert (r, w, l) == (rank, world, rank)
    local_ms = 100.0 * (rank + 1)  # rank 1 is the slow one
    local_flop = 1e9 * (rank + 1)
    dist.barrier()
    ms, gflops = bench.replica_aggregate(local_ms, local_flop, dist)
    out[rank] = (ms, gflops)
    dist.destroy_process_group()


def test_replica_aggregate_two_ranks():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()  # no fork of a multi-threaded process
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    # every rank sees the same job figures: the slowest rank's time, all FLOPs
    for rank in range(world):
        ms, gflops = out[rank]
        assert ms == pytest.approx(200.0)
        assert gflops == pytest.approx(3e9 / 0.2 / 1e9)


def test_replica_aggregate_single():
    import bench

    ms, g = bench.replica_aggregate(50.0, 1e9, None)
    assert ms == 50.0 and g == pytest.approx(20.0)
