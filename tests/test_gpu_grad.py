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


# ----------------------------------------------------------------------------- filter backward
def _interval(cell):
    from oracle import chebyshev as ch
    op = PWOperator.from_cell(cell)
    lo, hi, _, _ = ch.bounds(op, cell.Y0, mode="rigorous")
    return lo, hi


def _rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


@pytest.mark.parametrize("paw", [True, False])
@pytest.mark.parametrize("every", [0, 1, 2, 5])
def test_filter_backward_matches_oracle(paw, every):
    """chebfi_cheb_filter_backward (FP64) against the oracle's adjoint recurrence, element by
    element, for every checkpoint interval (1: every iterate kept; 5 = degree: one segment)."""
    from oracle.gradients import filter_backward
    from paper_1406_4350_gb300.chebfi import ChebFI, fortran
    cell = _cell(nb=3, paw=paw)
    deg = 5
    lo, hi = _interval(cell)
    rng = np.random.default_rng(4)
    W = rng.normal(size=cell.Y0.shape) + 1j * rng.normal(size=cell.Y0.shape)
    g = ChebFI.from_cell(cell)
    gY, gV, gD = g.cheb_filter_backward(fortran(cell.Y0), fortran(W), deg, lo, hi, cell.vloc.shape, cell.D.size,
                                        checkpoint_every=every)
    torch.cuda.synchronize()
    rY, rV, rD = filter_backward(PWOperator.from_cell(cell), cell.Y0, W, deg, lo, hi)
    assert _rel(gY.cpu().numpy(), rY) <= 1e-11
    assert _rel(gV.cpu().numpy(), rV) <= 1e-11
    assert _rel(gD.cpu().numpy(), rD) <= 1e-11


def test_filter_backward_degree_zero_and_one():
    from oracle.gradients import filter_backward
    from paper_1406_4350_gb300.chebfi import ChebFI, fortran
    cell = _cell(nb=2)
    lo, hi = _interval(cell)
    rng = np.random.default_rng(5)
    W = rng.normal(size=cell.Y0.shape) + 1j * rng.normal(size=cell.Y0.shape)
    g = ChebFI.from_cell(cell)
    for deg in (0, 1):
        gY, gV, gD = g.cheb_filter_backward(fortran(cell.Y0), fortran(W), deg, lo, hi, cell.vloc.shape, cell.D.size)
        torch.cuda.synchronize()
        rY, rV, rD = filter_backward(PWOperator.from_cell(cell), cell.Y0, W, deg, lo, hi)
        assert _rel(gY.cpu().numpy(), rY) <= 1e-11
        assert np.abs(gV.cpu().numpy() - rV).max() <= 1e-11 * max(np.abs(rV).max(), 1.0)
        assert np.abs(gD.cpu().numpy() - rD).max() <= 1e-11 * max(np.abs(rD).max(), 1.0)


def test_filter_backward_rejects_mixed_and_bad_arguments():
    from paper_1406_4350_gb300.chebfi import ChebFI, ChebFIError, fortran
    cell = _cell(nb=1)
    g = ChebFI.from_cell(cell)
    Y = fortran(cell.Y0)
    with pytest.raises(ChebFIError):
        g.cheb_filter_backward(Y, Y, 3, 0.0, 1.0, cell.vloc.shape, cell.D.size, prec=2)
    with pytest.raises(ChebFIError):
        g.cheb_filter_backward(Y, Y, 3, 1.0, 0.0, cell.vloc.shape, cell.D.size)
    with pytest.raises(ChebFIError):
        g.cheb_filter_backward(Y, Y, 3, 0.0, 1.0, cell.vloc.shape, cell.D.size, checkpoint_every=-1)


def test_filter_backward_eigenvector_closed_form():
    """Y_0 = psi_n (S-normalised exact eigenvector), gY_n = S psi_n: the filter acts as the
    scalar p(lambda_n) = T_n((lambda_n - c)/r), so gY_0 = p S psi_n and gV = p' |psi_n(r)|^2/N^3
    with p' = n U_{n-1}((lambda_n - c)/r)/r (numpy's Chebyshev derivative)."""
    from paper_1406_4350_gb300.chebfi import ChebFI, fortran
    cell = _cell(nb=1, seed=5)
    op = PWOperator.from_cell(cell)
    w, Psi = exact_eigs(op, vectors=True)
    n = 3
    psi = np.asfortranarray(Psi[:, n:n + 1])
    deg, lo, hi = 7, w[6], float(w[-1]) + 1.0
    c, r = 0.5 * (hi + lo), 0.5 * (hi - lo)
    Tn = np.polynomial.chebyshev.Chebyshev.basis(deg)
    x = (w[n] - c) / r
    p, dp = Tn(x), Tn.deriv()(x) / r
    Spsi = op.apply_S(psi)
    g = ChebFI.from_cell(cell)
    gY, gV, _ = g.cheb_filter_backward(fortran(psi), fortran(Spsi), deg, lo, hi, cell.vloc.shape, cell.D.size,
                                       want_D=False)
    torch.cuda.synchronize()
    assert np.abs(gY.cpu().numpy() - p * Spsi).max() <= 1e-10 * abs(p)
    grid = np.zeros(op.grid, dtype=np.complex128)
    grid[tuple(op.miller[:, i] % op.grid[i] for i in range(3))] = psi[:, 0]
    dens = np.abs(np.fft.ifftn(grid) * op.vloc.size) ** 2 / op.vloc.size
    assert np.abs(gV.cpu().numpy() - dp * dens).max() <= 1e-9 * abs(dp) * dens.max()


@pytest.fixture(scope="module")
def _cfg5():
    """The differentiation workload: 48^3 grid, 8025 plane waves, 32 atoms x 8 projectors (PAW),
    128 bands, degree 8, with the oracle's gradients of L = Re <W, Y_8>."""
    from oracle.gradients import filter_backward
    from synth import config_cell
    cell = config_cell("paw48", nbands=128)
    lo, hi = _interval(cell)
    rng = np.random.default_rng(8)
    W = np.asfortranarray(rng.normal(size=cell.Y0.shape) + 1j * rng.normal(size=cell.Y0.shape))
    ref = filter_backward(PWOperator.from_cell(cell), cell.Y0, W, 8, lo, hi)
    return cell, lo, hi, W, ref


@pytest.mark.parametrize("prec, tol", [(0, 1e-10), (1, 2e-4)])
def test_filter_backward_differentiation_workload(_cfg5, prec, tol):
    """FP64 and FP32 forms at the differentiation workload against the oracle, every element of
    gY_0, gV and gD (the FP32 tolerance covers FP32 iterates amplified by the degree-8 filter)."""
    from paper_1406_4350_gb300.chebfi import ChebFI, fortran
    cell, lo, hi, W, (rY, rV, rD) = _cfg5
    g = ChebFI.from_cell(cell)
    gY, gV, gD = g.cheb_filter_backward(fortran(cell.Y0), fortran(W), 8, lo, hi, cell.vloc.shape, cell.D.size,
                                        prec=prec)
    torch.cuda.synchronize()
    assert _rel(gY.cpu().numpy(), rY) <= tol
    assert _rel(gV.cpu().numpy(), rV) <= tol
    assert _rel(gD.cpu().numpy(), rD) <= tol


def test_autograd_filter_matches_oracle():
    from oracle.gradients import filter_backward
    from paper_1406_4350_gb300.autograd import cheb_filter
    from paper_1406_4350_gb300.chebfi import ChebFI
    from oracle import chebyshev as ch
    cell = _cell(nb=2)
    lo, hi = _interval(cell)
    g = ChebFI.from_cell(cell)
    Y = torch.tensor(cell.Y0, dtype=torch.complex128, device="cuda", requires_grad=True)
    V = torch.tensor(cell.vloc, dtype=torch.float64, device="cuda", requires_grad=True)
    D = torch.tensor(cell.D, dtype=torch.float64, device="cuda", requires_grad=True)
    rng = np.random.default_rng(6)
    W = rng.normal(size=cell.Y0.shape) + 1j * rng.normal(size=cell.Y0.shape)
    out = cheb_filter(g, Y, V, D, 4, lo, hi)
    ref = ch.filter_plain(PWOperator.from_cell(cell), cell.Y0, 4, lo, hi)
    assert _rel(out.detach().cpu().numpy(), ref) <= 1e-11
    loss = (torch.conj(torch.tensor(W, device="cuda")) * out).real.sum()
    loss.backward()
    rY, rV, rD = filter_backward(PWOperator.from_cell(cell), cell.Y0, W, 4, lo, hi)
    assert _rel(Y.grad.cpu().numpy(), rY) <= 1e-11
    assert _rel(V.grad.cpu().numpy(), rV) <= 1e-11
    assert _rel(D.grad.cpu().numpy(), rD) <= 1e-11
