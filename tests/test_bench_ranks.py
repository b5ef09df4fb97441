"""The bench's multi-rank host logic on CPU with gloo (world size 2): each
rank runs an independent replica, the job time is the slowest rank's, and the
value counts every rank's work (weak scaling, no collective on the data path)."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


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

    ms_local = 10.0 + 5.0 * rank  # rank 1 is the slower one
    ms = bench.max_over_ranks(ms_local, dist, device="cpu")
    value = bench.job_value(1000, 20, world, ms)
    out[rank] = (ms, value)
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_job_value_gloo():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        ms, value = out[r]
        assert ms == 15.0
        assert value == pytest.approx(1000 * 20 * 2 / 0.015)


def test_single_rank_needs_no_collective():
    import bench

    assert bench.max_over_ranks(3.5, None) == 3.5
    assert bench.job_value(10, 4, 1, 2.0) == pytest.approx(10 * 4 / 0.002)
