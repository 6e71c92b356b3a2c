"""The multi-rank paths on CPU with two gloo ranks: the job's time is the slowest rank's; one
problem's bands split over the ranks (paper_1406_4350_gb300.parallel) reproduce the unsplit
sweep of Algorithm 2; the row-sharded reduction of the subspace matrices gives the unsharded
Ritz values; k-point and band ranges partition their index sets."""
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
    from paper_1406_4350_gb300.parallel import row_sharded_gram
    rows = slice(rank, None, world)
    part = np.stack([Y[rows].conj().T @ HY[rows], Y[rows].conj().T @ SY[rows]])
    Hs, Ss = row_sharded_gram(torch.from_numpy(part), Y.shape[1]).numpy()  # the exchange step
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


def _band_worker(rank, world, port, out):
    """One sweep of Algorithm 2 with the bands split over the ranks: rank r filters its band
    range, the block is gathered on every rank for Rayleigh-Ritz, each rank keeps its bands.
    The oracle stands in for the library as the local arithmetic (no GPU here)."""
    import numpy as np
    import torch
    import torch.distributed as dist
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from oracle import chebyshev as ch
    from oracle.planewave import PWOperator
    from paper_1406_4350_gb300.parallel import band_range, gather_bands
    from synth import make_cell
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    cell = make_cell(6.0, 12, 3.0, 2, 8, 7, True, 19)
    op = PWOperator.from_cell(cell)
    nb = cell.Y0.shape[1]
    b0, b1 = band_range(nb, world, rank)
    lo = float(ch.rayleigh_quotients(op, cell.Y0).max())
    hi = ch.upper_bound(op, "rigorous")
    mine = ch.filter_reuse(op, cell.Y0[:, b0:b1], 5, lo, hi)
    full = gather_bands(torch.from_numpy(np.ascontiguousarray(mine.T)).T, nb, world).numpy()
    w, Yr = ch.rayleigh_ritz(op, full)
    out[rank] = (w, Yr[:, b0:b1], b0, b1)
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_band_split_sweep_matches_the_unsplit_one(world):
    import numpy as np
    from oracle import chebyshev as ch
    from oracle.planewave import PWOperator
    from synth import make_cell
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_band_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    cell = make_cell(6.0, 12, 3.0, 2, 8, 7, True, 19)
    op = PWOperator.from_cell(cell)
    lo = float(ch.rayleigh_quotients(op, cell.Y0).max())
    hi = ch.upper_bound(op, "rigorous")
    w_ref, _ = ch.rayleigh_ritz(op, ch.filter_reuse(op, cell.Y0, 5, lo, hi))
    covered = []
    for r in range(world):
        w, Yr, b0, b1 = out[r]
        np.testing.assert_allclose(w, w_ref, rtol=0, atol=1e-11 * np.abs(w_ref).max())
        covered += list(range(b0, b1))
        assert Yr.shape[1] == b1 - b0
    assert covered == list(range(cell.Y0.shape[1]))  # 7 bands over 2 ranks: 4 + 3


def test_band_and_kpoint_ranges_partition_their_sets():
    from paper_1406_4350_gb300.parallel import band_range, kpoint_range
    for n in (0, 1, 7, 64, 2048, 2049):
        for world in (1, 2, 3, 4, 8):
            got = []
            for r in range(world):
                a, b = band_range(n, world, r)
                assert 0 <= a <= b <= n
                got += list(range(a, b))
            assert got == list(range(n))
            assert [kpoint_range(n, world, r) for r in range(world)] == [band_range(n, world, r) for r in range(world)]
    with pytest.raises(ValueError):
        band_range(10, 2, 2)
