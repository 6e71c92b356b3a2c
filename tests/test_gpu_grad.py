"""Derivatives of Algorithm 1's H application (chebfi_apply_H_backward, the autograd
binding) against the FP64 oracle: central differences of the oracle's own H application,
and the Hellmann-Feynman theorem for exact eigenpairs of a tiny cell."""
import dataclasses

import numpy as np
import pytest
import torch

from oracle.exact import exact_eigs
from oracle.planewave import PWOperator
from synth import make_cell

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1406_4350_gb300 import build
    build.build()


def _cell(nb=3, paw=True, seed=31):
    return make_cell(8.0, 16, 3.0, 3, 8, nb, paw, seed)


def _loss_oracle(cell, W, Y=None, vloc=None, D=None):
    c = dataclasses.replace(cell, vloc=cell.vloc if vloc is None else vloc, D=cell.D if D is None else D)
    HY = PWOperator.from_cell(c).apply_H(cell.Y0 if Y is None else Y)
    return float(np.sum(np.conj(W) * HY).real)


def test_apply_H_backward_against_oracle_differences():
    from paper_1406_4350_gb300.chebfi import ChebFI, fortran
    cell = _cell()
    rng = np.random.default_rng(0)
    W = rng.normal(size=cell.Y0.shape) + 1j * rng.normal(size=cell.Y0.shape)
    g = ChebFI.from_cell(cell)
    gY, gV, gD = g.apply_H_backward(fortran(cell.Y0), fortran(W), cell.vloc.shape, cell.D.size)
    torch.cuda.synchronize()
    gY, gV, gD = gY.cpu().numpy(), gV.cpu().numpy(), gD.cpu().numpy()
    # L is linear in V, D and Y, so central differences are exact up to rounding
    h = 1e-3
    for idx in [(0, 0, 0), (3, 7, 11), (15, 2, 9)]:
        vp = cell.vloc.copy()
        vm = cell.vloc.copy()
        vp[idx] += h
        vm[idx] -= h
        fd = (_loss_oracle(cell, W, vloc=vp) - _loss_oracle(cell, W, vloc=vm)) / (2 * h)
        assert abs(gV[idx] - fd) <= 1e-9 * max(1.0, abs(fd)), (idx, gV[idx], fd)
    for e in [0, 5, 64 + 9, cell.D.size - 1]:
        dp = cell.D.copy()
        dm = cell.D.copy()
        dp[e] += h
        dm[e] -= h
        fd = (_loss_oracle(cell, W, D=dp) - _loss_oracle(cell, W, D=dm)) / (2 * h)
        assert abs(gD[e] - fd) <= 1e-9 * max(1.0, abs(fd)), (e, gD[e], fd)
    # Y: the directional derivative along a random direction E is Re sum conj(gY) E
    E = rng.normal(size=cell.Y0.shape) + 1j * rng.normal(size=cell.Y0.shape)
    fd = (_loss_oracle(cell, W, Y=cell.Y0 + h * E) - _loss_oracle(cell, W, Y=cell.Y0 - h * E)) / (2 * h)
    an = float(np.sum(np.conj(gY) * E).real)
    assert abs(an - fd) <= 1e-9 * max(1.0, abs(fd))


def test_hellmann_feynman_for_exact_eigenpairs():
    """d lambda_n / d V_loc(r) from chebfi_apply_H_backward with Y = G = psi_n (an S-normalised
    exact eigenvector of the pencil) equals the central difference of the exact eigenvalue."""
    from paper_1406_4350_gb300.chebfi import ChebFI, fortran
    cell = _cell(nb=1, seed=5)
    op = PWOperator.from_cell(cell)
    w, Psi = exact_eigs(op, vectors=True)
    n = int(np.argmax(np.minimum(np.diff(w)[:-1], np.diff(w)[1:])[:10])) + 1  # a well-separated level
    psi = np.asfortranarray(Psi[:, n:n + 1])
    g = ChebFI.from_cell(cell)
    _, gV, _ = g.apply_H_backward(fortran(psi), fortran(psi), cell.vloc.shape, cell.D.size, want_Y=False,
                                  want_D=False)
    torch.cuda.synchronize()
    gV = gV.cpu().numpy()
    # Parseval: the grid sum of (1/N^3)|psi(r)|^2 is the coefficient norm sum_G |c_G|^2
    assert abs(gV.sum() - np.vdot(psi, psi).real) <= 1e-12
    # a single-point change of V moves lambda_n by ~1e-6 h; the second-order term cancels in the
    # central difference and higher orders are negligible, while the eigenvalues' own
    # rounding (~1e-14) enters divided by 2h, so a large step is the accurate one
    h = 1e-2
    for idx in [(0, 0, 0), (4, 9, 2), (12, 12, 12)]:
        vp = cell.vloc.copy()
        vm = cell.vloc.copy()
        vp[idx] += h
        vm[idx] -= h
        lp = exact_eigs(PWOperator.from_cell(dataclasses.replace(cell, vloc=vp)))[n]
        lm = exact_eigs(PWOperator.from_cell(dataclasses.replace(cell, vloc=vm)))[n]
        fd = (lp - lm) / (2 * h)
        assert abs(gV[idx] - fd) <= 1e-6 * abs(fd) + 1e-12, (idx, gV[idx], fd)


def test_autograd_function_matches_backward():
    from paper_1406_4350_gb300.autograd import apply_H
    from paper_1406_4350_gb300.chebfi import ChebFI
    cell = _cell(nb=2)
    g = ChebFI.from_cell(cell)
    Y = torch.tensor(cell.Y0, dtype=torch.complex128, device="cuda", requires_grad=True)
    V = torch.tensor(cell.vloc, dtype=torch.float64, device="cuda", requires_grad=True)
    D = torch.tensor(cell.D, dtype=torch.float64, device="cuda", requires_grad=True)
    rng = np.random.default_rng(3)
    W = torch.tensor(rng.normal(size=cell.Y0.shape) + 1j * rng.normal(size=cell.Y0.shape), device="cuda")
    out = apply_H(g, Y, V, D)
    ref = PWOperator.from_cell(cell).apply_H(cell.Y0)
    assert np.abs(out.detach().cpu().numpy() - ref).max() <= 1e-11 * np.abs(ref).max()
    loss = (torch.conj(W) * out).real.sum()
    loss.backward()
    h = 1e-3
    idx = (5, 6, 7)
    vp = cell.vloc.copy()
    vm = cell.vloc.copy()
    vp[idx] += h
    vm[idx] -= h
    fd = (_loss_oracle(cell, W.cpu().numpy(), vloc=vp) - _loss_oracle(cell, W.cpu().numpy(), vloc=vm)) / (2 * h)
    assert abs(V.grad[idx].item() - fd) <= 1e-9 * max(1.0, abs(fd))
    assert Y.grad is not None and D.grad is not None
    e = 3
    dp = cell.D.copy()
    dm = cell.D.copy()
    dp[e] += h
    dm[e] -= h
    fd = (_loss_oracle(cell, W.cpu().numpy(), D=dp) - _loss_oracle(cell, W.cpu().numpy(), D=dm)) / (2 * h)
    assert abs(D.grad[e].item() - fd) <= 1e-9 * max(1.0, abs(fd))
