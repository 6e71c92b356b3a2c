"""The benchmark's multi-rank path on CPU: two gloo ranks, each timing its own replica; the
job's time is the slowest rank's and its throughput counts both ranks' units."""
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
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    # rank r pretends its filter took (1 + r) s and its step (2 + r) s for 100 units
    value, fs, ss = bench.aggregate(1.0 + rank, 2.0 + rank, 100.0, world)
    out[rank] = (value, fs, ss)
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_aggregate_takes_the_slowest_rank(world):
    mgr = mp.Manager()
    out = mgr.dict()
    port = _free_port()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        value, fs, ss = out[r]
        assert fs == float(world) and ss == float(world + 1)
        assert value == pytest.approx(world * 100.0 / world)
