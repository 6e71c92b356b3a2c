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


def _rr_worker(rank, world, port, out):
    """Rank r holds rows r::world of Y, HY and SY (plane waves dealt round-robin); the
    subspace matrices are sums of per-rank partial products, reduced with all_reduce."""
    import numpy as np
    import scipy.linalg
    import torch
    import torch.distributed as dist
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from oracle.planewave import PWOperator
    from synth import make_cell
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    cell = make_cell(6.0, 12, 3.0, 2, 8, 6, True, 17)
    op = PWOperator.from_cell(cell)
    Y = cell.Y0
    HY, SY = op.apply_H(Y), op.apply_S(Y)
    rows = slice(rank, None, world)
    part = np.stack([Y[rows].conj().T @ HY[rows], Y[rows].conj().T @ SY[rows]])
    t = torch.from_numpy(part)
    dist.all_reduce(t)  # the one exchange step of a row-sharded Rayleigh-Ritz
    Hs, Ss = t.numpy()
    w = scipy.linalg.eigh(0.5 * (Hs + Hs.conj().T), 0.5 * (Ss + Ss.conj().T), eigvals_only=True)
    out[rank] = w
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_row_sharded_rayleigh_ritz_reduction(world):
    """CPU simulation of the exchange step a row-sharded Rayleigh-Ritz would need (sum of
    partial Gram matrices): every rank gets the unsharded Ritz values."""
    import numpy as np
    import scipy.linalg
    from oracle.planewave import PWOperator
    from synth import make_cell
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rr_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    cell = make_cell(6.0, 12, 3.0, 2, 8, 6, True, 17)
    op = PWOperator.from_cell(cell)
    Y = cell.Y0
    Hs, Ss = Y.conj().T @ op.apply_H(Y), Y.conj().T @ op.apply_S(Y)
    ref = scipy.linalg.eigh(0.5 * (Hs + Hs.conj().T), 0.5 * (Ss + Ss.conj().T), eigvals_only=True)
    for r in range(world):
        np.testing.assert_allclose(out[r], ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    np.testing.assert_array_equal(out[0], out[1])
