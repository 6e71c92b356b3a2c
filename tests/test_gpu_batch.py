"""Batched k-points (chebfi_batch_*): Algorithm 2's filter for many Bloch vectors of one
cell in grouped launches, against the oracle's filter of each k-point on its own."""
import dataclasses

import numpy as np
import pytest
import torch

from oracle import chebyshev as ch
from oracle.planewave import PWOperator
from synth import kpoint_cells

pytestmark = pytest.mark.gpu

TOL64 = 1e-11  # the FP64 parity tolerance of the single-problem tests
TOL32 = 2e-5   # the FP32 one
TOLMIX = 1e-4  # the mixed one, per filter step


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1406_4350_gb300 import build
    build.build()


def _small(nk=5, nb=8, seed=1204):
    return kpoint_cells(nk=nk, nbands=nb, seed=seed, npw_range=(300, 900), L=8.0, grid=24, natoms=3)


def _intervals(cells):
    lo, hi = [], []
    for c in cells:
        op = PWOperator.from_cell(c)
        l, h, _, _ = ch.bounds(op, c.Y0, mode="rigorous")
        lo.append(l)
        hi.append(h)
    return lo, hi


def _batch(cells):
    from paper_1406_4350_gb300.chebfi import ChebFI, ChebFIBatch
    ctxs = [ChebFI.from_cell(c) for c in cells]
    return ChebFIBatch(ctxs, cells[0].nbands)


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("prec, tol", [(0, TOL64), (1, TOL32), (2, TOLMIX * 6)])
def test_batch_filter_matches_oracle_per_kpoint(prec, tol):
    from paper_1406_4350_gb300.chebfi import fortran
    cells = _small()
    assert len({c.npw for c in cells}) == len(cells)  # uneven spheres
    lo, hi = _intervals(cells)
    bt = _batch(cells)
    Ys = [fortran(c.Y0) for c in cells]
    deg = 6
    bt.cheb_filter(Ys, deg, lo, hi, prec=prec)
    torch.cuda.synchronize()
    for c, Y, l, h in zip(cells, Ys, lo, hi):
        ref = ch.filter_plain(PWOperator.from_cell(c), c.Y0, deg, l, h)
        assert _rel(Y.cpu().numpy(), ref) <= tol


def test_batch_graph_replay_takes_new_blocks_and_intervals():
    """The second call replays the captured graph with other blocks and other intervals."""
    from paper_1406_4350_gb300.chebfi import fortran
    cells = _small(seed=1205)
    lo, hi = _intervals(cells)
    bt = _batch(cells)
    deg = 4
    first = [fortran(c.Y0) for c in cells]
    bt.cheb_filter(first, deg, lo, hi, prec=0)
    n1 = bt.kernel_launches
    rng = np.random.default_rng(3)
    Y2 = [np.asfortranarray(rng.normal(size=c.Y0.shape) + 1j * rng.normal(size=c.Y0.shape)) for c in cells]
    lo2 = [l - 0.3 for l in lo]
    hi2 = [h + 1.0 for h in hi]
    second = [fortran(y) for y in Y2]
    bt.cheb_filter(second, deg, lo2, hi2, prec=0)
    torch.cuda.synchronize()
    assert bt.kernel_launches == 2 * n1 > 0
    for c, Y, y0, l, h in zip(cells, second, Y2, lo2, hi2):
        ref = ch.filter_plain(PWOperator.from_cell(c), y0, deg, l, h)
        assert _rel(Y.cpu().numpy(), ref) <= TOL64


def test_batch_norm_conserving_and_degree_zero():
    from paper_1406_4350_gb300.chebfi import fortran
    cells = [dataclasses.replace(c, Q=None) for c in _small(nk=3, seed=1206)]
    lo, hi = _intervals(cells)
    bt = _batch(cells)
    Ys = [fortran(c.Y0) for c in cells]
    bt.cheb_filter(Ys, 0, lo, hi, prec=0)
    torch.cuda.synchronize()
    for c, Y in zip(cells, Ys):
        assert np.array_equal(Y.cpu().numpy(), c.Y0)
    bt.cheb_filter(Ys, 3, lo, hi, prec=0)
    torch.cuda.synchronize()
    for c, Y, l, h in zip(cells, Ys, lo, hi):
        ref = ch.filter_plain(PWOperator.from_cell(c), c.Y0, 3, l, h)
        assert _rel(Y.cpu().numpy(), ref) <= TOL64


def test_batch_autotune_reports_every_shape():
    cells = _small(nk=3, seed=1207)
    bt = _batch(cells)
    shapes, split, ms, split_ms = bt.autotune(1)
    assert len(shapes) == 3 and all(0 <= s < 4 for s in shapes) and split in (1, 2, 4, 8)
    assert np.all(np.isfinite(ms)) and np.all(ms > 0) and np.all(split_ms > 0)
    for gc in (1, 2):
        assert ms[gc, shapes[gc]] == ms[gc].min()
    # the P^H Z choice is the fastest (shape, split) pair
    assert split_ms[[1, 2, 4, 8].index(split)] == split_ms.min()


@pytest.mark.parametrize("shapes, split", [([0, 1, 2], 1), ([3, 0, 3], 2), ([1, 2, 0], 4), ([2, 3, 1], 8)])
def test_batch_every_tile_shape_and_split(shapes, split):
    """Forced tiles (every shape in some class, every split-K factor of P^H Z): FP64 parity."""
    from paper_1406_4350_gb300.chebfi import fortran
    cells = _small(nk=4, seed=1209)
    lo, hi = _intervals(cells)
    bt = _batch(cells)
    bt.set_tiles(shapes, split, prec=0)
    Ys = [fortran(c.Y0) for c in cells]
    bt.cheb_filter(Ys, 5, lo, hi, prec=0)
    torch.cuda.synchronize()
    for c, Y, l, h in zip(cells, Ys, lo, hi):
        ref = ch.filter_plain(PWOperator.from_cell(c), c.Y0, 5, l, h)
        assert _rel(Y.cpu().numpy(), ref) <= TOL64


def test_batch_rejects_incompatible_contexts():
    from paper_1406_4350_gb300.chebfi import ChebFI, ChebFIBatch, ChebFIError
    cells = _small(nk=2, seed=1208)
    other = dataclasses.replace(cells[1], vloc=cells[1].vloc * 1.01)
    with pytest.raises(ChebFIError):
        ChebFIBatch([ChebFI.from_cell(cells[0]), ChebFI.from_cell(other)], cells[0].nbands)
    nc = dataclasses.replace(cells[1], Q=None)
    with pytest.raises(ChebFIError):
        ChebFIBatch([ChebFI.from_cell(cells[0]), ChebFI.from_cell(nc)], cells[0].nbands)
    bt = _batch(cells)
    from paper_1406_4350_gb300.chebfi import fortran
    Ys = [fortran(c.Y0) for c in cells]
    with pytest.raises(ChebFIError):
        bt.cheb_filter(Ys, 2, [1.0, 1.0], [0.0, 2.0], prec=1)  # lambda_hi <= lambda_lo at k = 0
    with pytest.raises(ChebFIError):
        bt.cheb_filter(Ys, 2, [0.0, 0.0], [1.0, 1.0], prec=3)  # no such form


def test_batch_kpoint_workload_sampled():
    """The batched k-point workload (64 k-points of a 48^3 PAW cell, spheres of 3000 to 12000
    plane waves, 128 bands, FP32 filter of degree 8): three k-points (the smallest, the
    largest and one between) against the oracle, every element."""
    from paper_1406_4350_gb300.chebfi import fortran
    cells = kpoint_cells()
    npw = np.array([c.npw for c in cells])
    assert npw.min() >= 3000 and npw.max() <= 12300
    bt = _batch(cells)
    picks = [int(np.argmin(npw)), int(np.argmax(npw)), len(cells) // 2]
    lo = [float(ch.rayleigh_quotients(PWOperator.from_cell(c), c.Y0).max()) if i in picks else 0.5
          for i, c in enumerate(cells)]
    hi = [40.0] * len(cells)
    Ys = [fortran(c.Y0) for c in cells]
    bt.cheb_filter(Ys, 8, lo, hi, prec=1)
    Ym = [fortran(cells[i].Y0) if i in picks else Y.clone() for i, Y in enumerate(Ys)]
    bt.cheb_filter(Ym, 8, lo, hi, prec=2)
    torch.cuda.synchronize()
    for i in picks:
        c = cells[i]
        ref = ch.filter_reuse(PWOperator.from_cell(c), c.Y0, 8, lo[i], hi[i])
        assert _rel(Ys[i].cpu().numpy(), ref) <= 1e-4
        assert _rel(Ym[i].cpu().numpy(), ref) <= TOLMIX * 8


@pytest.mark.parametrize("paw", [True, False])
def test_batch_mixed_replay_ragged_band_tiles(paw):
    """Mixed form: 136 bands (a full and a ragged 128-band tile of the grouped tensor-core
    GEMMs), spheres of several 512-real chunks, PAW and norm-conserving; the second call
    replays the graph with new blocks and intervals (the 1/r_k of P W is refreshed)."""
    from paper_1406_4350_gb300.chebfi import fortran
    cells = kpoint_cells(nk=3, nbands=136, seed=1210, npw_range=(400, 1100), L=8.0, grid=24, natoms=3)
    if not paw:
        cells = [dataclasses.replace(c, Q=None) for c in cells]
    lo, hi = _intervals(cells)
    bt = _batch(cells)
    deg = 5
    Ys = [fortran(c.Y0) for c in cells]
    bt.cheb_filter(Ys, deg, lo, hi, prec=2)
    torch.cuda.synchronize()
    n1 = bt.kernel_launches
    for c, Y, l, h in zip(cells, Ys, lo, hi):
        ref = ch.filter_plain(PWOperator.from_cell(c), c.Y0, deg, l, h)
        assert _rel(Y.cpu().numpy(), ref) <= TOLMIX * deg
    rng = np.random.default_rng(5)
    Y2 = [np.asfortranarray(rng.normal(size=c.Y0.shape) + 1j * rng.normal(size=c.Y0.shape)) for c in cells]
    lo2 = [l - 0.2 for l in lo]
    hi2 = [h + 2.0 for h in hi]
    second = [fortran(y) for y in Y2]
    bt.cheb_filter(second, deg, lo2, hi2, prec=2)
    torch.cuda.synchronize()
    assert bt.kernel_launches == 2 * n1 > 0
    for c, Y, y0, l, h in zip(cells, second, Y2, lo2, hi2):
        ref = ch.filter_plain(PWOperator.from_cell(c), y0, deg, l, h)
        assert _rel(Y.cpu().numpy(), ref) <= TOLMIX * deg
