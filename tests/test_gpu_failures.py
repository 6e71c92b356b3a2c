"""Failure detection through the C ABI, with no GPU fault: bad inputs are refused on the host,
Inf/NaN blocks are reported as CHEBFI_ERR_NONFINITE, bounded device waits that nothing
satisfies run out and record their error, and the context stays usable after each."""
import dataclasses

import numpy as np
import pytest
import torch

from synth import make_cell

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1406_4350_gb300 import build
    build.build()


def _cell():
    return make_cell(8.0, 16, 3.0, 3, 8, 7, True, 21)


def _ctx(cell):
    from paper_1406_4350_gb300.chebfi import ChebFI
    return ChebFI.from_cell(cell)


def _F(x):
    from paper_1406_4350_gb300.chebfi import fortran
    return fortran(x)


def _still_works(g, cell):
    Y = _F(cell.Y0)
    HY = g.apply_H(Y)
    torch.cuda.synchronize()
    assert torch.isfinite(torch.view_as_real(HY)).all()


def test_non_finite_setup_data_is_refused():
    from paper_1406_4350_gb300._lib import ERR_NONFINITE
    from paper_1406_4350_gb300.chebfi import ChebFI, ChebFIError
    cell = _cell()
    g = ChebFI(0)
    g.set_cell(cell.lattice, cell.grid, cell.kpt)
    g.set_sphere(cell.miller)
    v = cell.vloc.copy()
    v[1, 2, 3] = np.nan
    with pytest.raises(ChebFIError) as e:
        g.set_vloc(v)
    assert e.value.code == ERR_NONFINITE
    g.set_vloc(cell.vloc)
    D = cell.D.copy()
    D[5] = np.inf
    with pytest.raises(ChebFIError) as e:
        g.set_projectors(cell.P, cell.proj_offsets, D, cell.Q)
    assert e.value.code == ERR_NONFINITE
    P = cell.P.copy()
    P[4, 2] = np.nan
    with pytest.raises(ChebFIError) as e:
        g.set_projectors(P, cell.proj_offsets, cell.D, cell.Q)
    assert e.value.code == ERR_NONFINITE
    g.set_projectors(cell.P, cell.proj_offsets, cell.D, cell.Q)
    with pytest.raises(ChebFIError) as e:
        g.set_D(np.full(cell.D.shape, np.inf))
    assert e.value.code == ERR_NONFINITE
    _still_works(g, cell)


def test_non_finite_block_in_rayleigh_ritz_and_solve():
    from paper_1406_4350_gb300._lib import ERR_NONFINITE
    from paper_1406_4350_gb300.chebfi import ChebFIError
    cell = _cell()
    g = _ctx(cell)
    Y0 = cell.Y0.copy()
    Y0[3, 2] = np.nan
    with pytest.raises(ChebFIError) as e:
        g.rayleigh_ritz(_F(Y0))
    assert e.value.code == ERR_NONFINITE
    with pytest.raises(ChebFIError) as e:
        g.orthonormalise(_F(Y0))
    assert e.value.code == ERR_NONFINITE
    with pytest.raises(ChebFIError) as e:
        g.solve(_F(Y0), degree=4, sweeps=2)
    assert e.value.code == ERR_NONFINITE
    _still_works(g, cell)
    ev, _ = g.rayleigh_ritz(_F(cell.Y0))
    assert torch.isfinite(ev).all()


@pytest.mark.parametrize("which", [0, 1])
def test_bounded_waits_run_out_and_record_their_error(which):
    from paper_1406_4350_gb300._lib import ERR_CUDA
    cell = _cell()
    g = _ctx(cell)
    code, ms = g.selftest_bounded_wait(which, 20.0)
    assert code == ERR_CUDA
    assert 15.0 <= ms <= 2000.0
    _still_works(g, cell)
    assert g.lib.chebfi_sync_status(g.h) == 0  # the self-test used its own status word
