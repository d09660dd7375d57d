"""Replicas-only multi-GPU path of bench.py, host logic on CPU with gloo ranks.

Each rank runs an independent replica; the whole-job value is the DoF-cycles
of all ranks over the slowest rank's time (max over ranks).
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = [100.0, 250.0][rank]
    value, ms_max = bench.aggregate_throughput(1000, 10, local_ms, dist, "cpu")
    out[rank] = (value, ms_max)
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    for rank in range(2):
        value, ms_max = out[rank]
        assert ms_max == 250.0
        assert value == pytest.approx(1000 * 10 * 2 / 0.25)


def test_single_rank_has_no_collective():
    import bench
    value, ms_max = bench.aggregate_throughput(1000, 10, 100.0, None, "cpu")
    assert ms_max == 100.0 and value == pytest.approx(1e5)
