"""The refined dense eigensolver of Rayleigh-Ritz (FP32 Jacobi + FP64 Ogita-Aishima
refinement on the tensor-core GEMMs) through the C ABI.

Fixed independently of its code: the oracle's Rayleigh-Ritz (LAPACK) on the same block;
exactly degenerate Ritz values of a free-electron subspace, whose values are the shells
(2 pi^2 / L^2) s with multiplicities 1, 6, 12, 8; and the FP64 Jacobi eigensolver.
"""
import dataclasses

import numpy as np
import pytest
import torch

from oracle import chebyshev as ch
from oracle.planewave import PWOperator
from synth import config_cell, make_cell

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1406_4350_gb300 import build
    build.build()


def _F(x):
    from paper_1406_4350_gb300.chebfi import fortran
    return fortran(x)


def _np(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _ctx(cell):
    from paper_1406_4350_gb300.chebfi import ChebFI
    return ChebFI.from_cell(cell)


def test_refined_rayleigh_ritz_matches_oracle():
    from paper_1406_4350_gb300._lib import EIG_REFINED
    cell = config_cell("paw48", nbands=37)
    op = PWOperator.from_cell(cell)
    g = _ctx(cell)
    g.set_eigensolver(EIG_REFINED)
    lo = float(ch.rayleigh_quotients(op, cell.Y0).max())
    hi = ch.upper_bound(op, "rigorous")
    ref = ch.filter_reuse(op, cell.Y0, 10, lo, hi)
    w_ref, X_ref = ch.rayleigh_ritz(op, ref)
    Y = _F(ref)
    ev, rs = g.rayleigh_ritz(Y)
    assert g.eigensolver_steps >= 1
    assert np.abs(_np(ev) - w_ref).max() <= 1e-9
    r_ref = ch.residuals(op, X_ref, w_ref)
    assert np.abs(_np(rs) - r_ref).max() <= 1e-6 * r_ref.max()
    Yn = _np(Y)
    G = Yn.conj().T @ op.apply_S(Yn)
    assert np.abs(G - np.eye(G.shape[0])).max() <= 1e-11


def test_refined_eigensolver_near_convergence_skips_the_fp32_stage():
    """Ritz vectors turned by 1e-6: the projected matrix is nearly diagonal, the refinement
    starts from the identity and no FP32 Jacobi sweep of the whole matrix runs (only cluster
    blocks may be diagonalised); Ritz values as the oracle's on the same block."""
    from paper_1406_4350_gb300._lib import EIG_REFINED
    cell = config_cell("paw48", nbands=37)
    op = PWOperator.from_cell(cell)
    g = _ctx(cell)
    g.set_eigensolver(EIG_REFINED)
    lo = float(ch.rayleigh_quotients(op, cell.Y0).max())
    hi = ch.upper_bound(op, "rigorous")
    ref = ch.filter_reuse(op, cell.Y0, 10, lo, hi)
    Y = _F(ref)
    g.rayleigh_ritz(Y)
    rng = np.random.default_rng(9)
    Y2 = _np(Y) + 1e-6 * (rng.normal(size=ref.shape) + 1j * rng.normal(size=ref.shape))
    w_ref, _ = ch.rayleigh_ritz(op, Y2)
    Yg = _F(Y2)
    g.profile(True)
    ev, _ = g.rayleigh_ritz(Yg)
    tot = g.profile_totals()
    g.profile(False)
    n = Y2.shape[1]
    jac_work = sum(v[2] for k, v in tot.items() if k.startswith("k_jac"))
    assert jac_work < 33.0 * n ** 3  # less than one sweep of the full matrix
    assert 1 <= g.eigensolver_steps <= 6
    assert np.abs(_np(ev) - w_ref).max() <= 1e-9


def test_refined_eigensolver_resolves_exactly_degenerate_shells():
    """V = 0, no projectors: the plane waves of the first four shells (27 of them) mixed by a
    random unitary span an invariant subspace with eigenvalues 0, (2 pi^2/L^2) x {1 (6-fold),
    2 (12-fold), 3 (8-fold)}; the refinement meets exact ties and must hand them to the
    cluster step."""
    from paper_1406_4350_gb300._lib import EIG_REFINED
    L = 10.0
    base = make_cell(L, 24, 7.6, 2, 1, 27, False, 5)
    cell = dataclasses.replace(base, vloc=np.zeros_like(base.vloc), D=np.zeros_like(base.D))
    m = cell.miller.astype(float)
    s = np.sum(m * m, 1).round().astype(int)
    idx = np.concatenate([np.nonzero(s == k)[0] for k in range(4)])
    assert idx.size == 27
    rng = np.random.default_rng(2)
    Q, _ = np.linalg.qr(rng.normal(size=(27, 27)) + 1j * rng.normal(size=(27, 27)))
    Y0 = np.zeros((cell.npw, 27), complex)
    Y0[idx, :] = Q
    g = _ctx(cell)
    g.set_eigensolver(EIG_REFINED)
    Y = _F(Y0)
    ev, rs = g.rayleigh_ritz(Y)
    assert g.eigensolver_steps >= 1
    expect = 2 * np.pi ** 2 / L ** 2 * np.repeat([0, 1, 2, 3], [1, 6, 12, 8])
    assert np.abs(_np(ev) - expect).max() <= 1e-12
    assert _np(rs).max() <= 1e-12
    Yn = _np(Y)
    assert np.abs(Yn.conj().T @ Yn - np.eye(27)).max() <= 1e-13


def test_refined_and_jacobi_agree_on_600_bands():
    from paper_1406_4350_gb300._lib import EIG_JACOBI, EIG_REFINED
    cell = config_cell("paw48", nbands=600)
    g = _ctx(cell)
    Y1 = _F(cell.Y0)
    g.set_eigensolver(EIG_JACOBI)
    e1, r1 = g.rayleigh_ritz(Y1)
    assert g.eigensolver_steps == 0
    Y2 = _F(cell.Y0)
    g.set_eigensolver(EIG_REFINED)
    e2, r2 = g.rayleigh_ritz(Y2)
    steps = g.eigensolver_steps
    assert 1 <= steps <= 8
    e1, e2 = _np(e1), _np(e2)
    assert np.abs(e1 - e2).max() <= 1e-10 * max(1.0, np.abs(e1).max())
    r1, r2 = _np(r1), _np(r2)
    assert np.abs(r1 - r2).max() <= 1e-8 * r1.max()
