"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on seeded cells.

Tolerances, from the arithmetic: FP64 results are compared elementwise against
``1e-11 * max|reference|`` (FP64 unit roundoff 1.1e-16 times the length of the longest
sum, sqrt(6e4) ~ 250, and the FFT's log N growth, with a 100x margin).  The FP32 form
uses ``2e-5 * max|reference|`` (unit roundoff 6e-8, same growth).  Eigenvalues are
compared in Hartree: 1e-8 against the exact pencil, 1e-9 against the oracle's own run of
Algorithm 2 from the same start.
"""
import ctypes
import dataclasses
import os

import numpy as np
import pytest
import torch

from oracle import chebyshev as ch
from oracle.planewave import PWOperator
from synth import config_cell, make_cell

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
TOL64 = 1e-11
TOL32 = 2e-5
# mixed form: projector products from bf16 (hi, lo) pairs (about 16 significant bits, unit
# roundoff 2^-17 = 7.6e-6) with FP32 accumulation over up to 1.2e5 terms
TOLMIX = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1406_4350_gb300 import build
    build.build()


def _ctx(cell):
    from paper_1406_4350_gb300.chebfi import ChebFI
    return ChebFI.from_cell(cell)


def _F(x):
    from paper_1406_4350_gb300.chebfi import fortran
    return fortran(x)


def _np(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _close(got, ref, tol):
    ref = np.asarray(ref)
    scale = max(np.abs(ref).max(), 1e-300)
    err = np.abs(np.asarray(got) - ref).max() / scale
    assert err <= tol, "relative error %.3e > %.1e" % (err, tol)
    return err


def _tiny_paw(nb=7, seed=21, natoms=3):
    return make_cell(8.0, 16, 3.0, natoms, 8, nb, True, seed)


CELLS = {
    "tiny_paw": lambda: _tiny_paw(),
    "tiny_nc": lambda: make_cell(8.0, 16, 3.0, 2, 1, 5, False, 5),
    "nc24": lambda: config_cell("nc24"),
    "paw48_37": lambda: config_cell("paw48", nbands=37),
}


@pytest.mark.parametrize("name", list(CELLS))
def test_apply_H_S_Sinv_fp64(name):
    cell = CELLS[name]()
    op = PWOperator.from_cell(cell)
    g = _ctx(cell)
    Y = _F(cell.Y0)
    _close(_np(g.apply_H(Y)), op.apply_H(cell.Y0), TOL64)
    _close(_np(g.apply_S(Y)), op.apply_S(cell.Y0), TOL64)
    _close(_np(g.apply_Sinv(Y)), op.apply_Sinv(cell.Y0), TOL64)


@pytest.mark.parametrize("name", ["nc24", "paw48_37"])
def test_fp64_fft_double_float_and_native(name):
    """The FP64 path's FFT in double-float (initial) and on the FP64 units: both within the FP64
    tolerance of the oracle for apply_H and a degree-8 filter, and within 1e-12 of each other."""
    from paper_1406_4350_gb300._lib import FFT64_DOUBLE_FLOAT, FFT64_NATIVE
    cell = CELLS[name]()
    op = PWOperator.from_cell(cell)
    g = _ctx(cell)
    lo = float(ch.rayleigh_quotients(op, cell.Y0).max())
    hi = ch.upper_bound(op, "rigorous")
    ref_f = ch.filter_reuse(op, cell.Y0, 8, lo, hi)
    out = {}
    for mode in (FFT64_DOUBLE_FLOAT, FFT64_NATIVE):
        g.set_fft64(mode)
        h = _np(g.apply_H(_F(cell.Y0)))
        _close(h, op.apply_H(cell.Y0), TOL64)
        Y = _F(cell.Y0)
        g.cheb_filter(Y, 8, lo, hi)
        f = _np(Y)
        _close(f, ref_f, TOL64)
        out[mode] = (h, f)
    _close(out[FFT64_DOUBLE_FLOAT][0], out[FFT64_NATIVE][0], 1e-12)
    _close(out[FFT64_DOUBLE_FLOAT][1], out[FFT64_NATIVE][1], 1e-12)
    with pytest.raises(Exception):
        g.set_fft64(7)


def test_plane_pass_with_a_wide_sphere():
    """A sphere spanning 43 of the 48 x rows: the first y pass of the plane kernel has
    43 x 6 items, more than a 256-thread block (NB = 6 does not divide 256, so each item takes
    its own twiddles); apply_H in the FP64 form (double-float and FP64-unit FFTs), FP32 and
    mixed against the oracle."""
    from paper_1406_4350_gb300 import F32, MIXED
    from paper_1406_4350_gb300._lib import FFT64_DOUBLE_FLOAT, FFT64_NATIVE
    cell = make_cell(8.0, 48, 140.0, 2, 8, 3, True, 7)
    xs = (cell.miller[:, 0] + 24) % 48
    assert xs.max() - xs.min() + 1 == 43
    op = PWOperator.from_cell(cell)
    ref = op.apply_H(cell.Y0)
    g = _ctx(cell)
    for mode in (FFT64_DOUBLE_FLOAT, FFT64_NATIVE):
        g.set_fft64(mode)
        _close(_np(g.apply_H(_F(cell.Y0))), ref, TOL64)
    _close(_np(g.apply_H(_F(cell.Y0), prec=F32)), ref, TOL32)
    _close(_np(g.apply_H(_F(cell.Y0), prec=MIXED)), ref, TOLMIX)
    g.sync_status()


@pytest.mark.parametrize("name", ["tiny_paw", "nc24", "paw48_37"])
def test_apply_H_fp32(name):
    from paper_1406_4350_gb300 import F32
    cell = CELLS[name]()
    op = PWOperator.from_cell(cell)
    g = _ctx(cell)
    _close(_np(g.apply_H(_F(cell.Y0), prec=F32)), op.apply_H(cell.Y0), TOL32)


@pytest.mark.parametrize("name", ["tiny_paw", "nc24", "paw48_37"])
def test_apply_H_mixed_tensor_cores(name):
    from paper_1406_4350_gb300 import MIXED
    cell = CELLS[name]()
    op = PWOperator.from_cell(cell)
    g = _ctx(cell)
    _close(_np(g.apply_H(_F(cell.Y0), prec=MIXED)), op.apply_H(cell.Y0), TOLMIX)
    g.sync_status()


@pytest.mark.parametrize("name,degree", [("tiny_paw", 5), ("nc24", 8), ("paw48_37", 10)])
def test_cheb_filter_mixed(name, degree):
    from paper_1406_4350_gb300 import MIXED
    cell = CELLS[name]()
    op = PWOperator.from_cell(cell)
    lo = float(ch.rayleigh_quotients(op, cell.Y0).max())
    hi = ch.upper_bound(op, "rigorous")
    ref = ch.filter_reuse(op, cell.Y0, degree, lo, hi)
    g = _ctx(cell)
    Y = _F(cell.Y0)
    g.cheb_filter(Y, degree, lo, hi, prec=MIXED)
    g.sync_status()
    _close(_np(Y), ref, TOLMIX * degree)


@pytest.mark.parametrize("name,degree", [("tiny_paw", 5), ("tiny_nc", 3), ("nc24", 8), ("paw48_37", 10)])
def test_cheb_filter_fp64(name, degree):
    cell = CELLS[name]()
    op = PWOperator.from_cell(cell)
    lo = float(ch.rayleigh_quotients(op, cell.Y0).max())
    hi = ch.upper_bound(op, "rigorous")
    ref = ch.filter_reuse(op, cell.Y0, degree, lo, hi)
    g = _ctx(cell)
    Y = _F(cell.Y0)
    g.cheb_filter(Y, degree, lo, hi)
    _close(_np(Y), ref, TOL64)


@pytest.mark.parametrize("name,degree", [("tiny_paw", 5), ("paw48_37", 10)])
def test_cheb_filter_fp32(name, degree):
    from paper_1406_4350_gb300 import F32
    cell = CELLS[name]()
    op = PWOperator.from_cell(cell)
    lo = float(ch.rayleigh_quotients(op, cell.Y0).max())
    hi = ch.upper_bound(op, "rigorous")
    ref = ch.filter_reuse(op, cell.Y0, degree, lo, hi)
    g = _ctx(cell)
    Y = _F(cell.Y0)
    g.cheb_filter(Y, degree, lo, hi, prec=F32)
    # the recurrence amplifies FP32 rounding by about the degree
    _close(_np(Y), ref, TOL32 * degree)


@pytest.mark.parametrize("name", ["tiny_paw", "nc24", "paw48_37"])
def test_rayleigh_quotients_and_ritz(name):
    cell = CELLS[name]()
    op = PWOperator.from_cell(cell)
    g = _ctx(cell)
    Y = _F(cell.Y0)
    rq = _np(g.rayleigh_quotients(Y))
    _close(rq, ch.rayleigh_quotients(op, cell.Y0), TOL64)
    w_ref, Y_ref = ch.rayleigh_ritz(op, cell.Y0)
    ev, rs = g.rayleigh_ritz(Y)
    ev, rs, Yg = _np(ev), _np(rs), _np(Y)
    _close(ev, w_ref, TOL64)
    nb = cell.nbands
    np.testing.assert_allclose(Yg.conj().T @ op.apply_S(Yg), np.eye(nb), atol=1e-10)
    np.testing.assert_allclose(Yg.conj().T @ op.apply_H(Yg), np.diag(ev), atol=1e-9 * max(1, np.abs(ev).max()))
    _close(rs, ch.residuals(op, Yg, ev), 1e-8)


def test_orthonormalise():
    cell = CELLS["paw48_37"]()
    op = PWOperator.from_cell(cell)
    g = _ctx(cell)
    Y = _F(cell.Y0)
    g.orthonormalise(Y)
    Yg = _np(Y)
    np.testing.assert_allclose(Yg.conj().T @ op.apply_S(Yg), np.eye(cell.nbands), atol=1e-10)
    # same span: the projector onto span(Y0) reproduces Y
    Q, _ = np.linalg.qr(cell.Y0)
    np.testing.assert_allclose(Q @ (Q.conj().T @ Yg), Yg, atol=1e-9)


def _golden(name):
    return np.loadtxt(os.path.join(HERE, "golden", "%s_exact_eigs.txt" % name))


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_solve_nc24_reaches_exact_eigenvalues(prec):
    """Config nc24 (degree 8; 7 sweeps, the count that reaches the target from the random
    start): lowest 75 % of the bands within 1e-8 Ha of the exact pencil eigenvalues
    (oracle O1, stored by tests/golden/make_golden.py)."""
    cell = config_cell("nc24")
    exact = _golden("nc24")
    g = _ctx(cell)
    Y = _F(cell.Y0)
    ev, rs = g.solve(Y, degree=8, sweeps=7, prec=prec)
    ev = _np(ev)
    k = (3 * cell.nbands) // 4
    assert np.abs(ev[:k] - exact[:k]).max() <= 1e-8


def test_solve_parity_with_oracle_algorithm_paw():
    """Same start, same lambda_+, same degree and sweeps: the CUDA run of Algorithm 2 and
    the oracle's agree on every Ritz value (rounding-level differences only)."""
    cell = _tiny_paw(nb=10, seed=4, natoms=4)
    op = PWOperator.from_cell(cell)
    hi = ch.upper_bound(op, "rigorous")
    ref = ch.solve(op, cell.Y0, degree=6, sweeps=4, lam_hi=hi)
    g = _ctx(cell)
    Y = _F(cell.Y0)
    ev, rs = g.solve(Y, degree=6, sweeps=4, lambda_hi=hi)
    ev = _np(ev)
    assert np.abs(ev - ref["w"]).max() <= 1e-9
    _close(_np(rs), ref["resid"], 1e-6)


def test_upper_bounds_match_oracle():
    from paper_1406_4350_gb300 import BOUND_PAPER, BOUND_RIGOROUS
    cell = _tiny_paw()
    op = PWOperator.from_cell(cell)
    g = _ctx(cell)
    assert abs(g.upper_bound(BOUND_PAPER) - ch.upper_bound(op, "paper")) <= 1e-12
    assert abs(g.upper_bound(BOUND_RIGOROUS) - ch.upper_bound(op, "rigorous")) <= 1e-9


# ------------------------------------------------------------------ edge cases
def test_empty_and_single_band_and_padded_ld():
    cell = _tiny_paw(nb=3)
    op = PWOperator.from_cell(cell)
    g = _ctx(cell)
    empty = torch.empty((cell.npw, 0), dtype=torch.complex128, device="cuda")
    assert g.apply_H(empty).shape == (cell.npw, 0)
    one = _F(cell.Y0[:, :1])
    _close(_np(g.apply_H(one)), op.apply_H(cell.Y0[:, :1]), TOL64)
    # leading dimension larger than npw
    big = torch.zeros((3, cell.npw + 13), dtype=torch.complex128, device="cuda")
    Yp = big.T[: cell.npw]
    Yp.copy_(_F(cell.Y0))
    out = torch.zeros_like(big).T[: cell.npw]
    g.apply_H(Yp, out=out)
    _close(_np(out), op.apply_H(cell.Y0), TOL64)


def test_plane_wave_order_is_the_callers():
    cell = _tiny_paw(nb=4)
    rng = np.random.default_rng(0)
    perm = rng.permutation(cell.npw)
    shuffled = dataclasses.replace(cell, miller=cell.miller[perm], P=np.asfortranarray(cell.P[perm]),
                                   Y0=np.asfortranarray(cell.Y0[perm]))
    a = _np(_ctx(cell).apply_H(_F(cell.Y0)))
    b = _np(_ctx(shuffled).apply_H(_F(shuffled.Y0)))
    _close(b, a[perm], TOL64)


def test_projectors_from_device_memory():
    cell = _tiny_paw(nb=4)
    from paper_1406_4350_gb300.chebfi import ChebFI
    g = ChebFI()
    g.set_cell(cell.lattice, cell.grid, cell.kpt)
    g.set_sphere(cell.miller)
    g.set_vloc(torch.as_tensor(cell.vloc, device="cuda"))
    g.set_projectors(_F(cell.P), cell.proj_offsets, cell.D, cell.Q)
    _close(_np(g.apply_H(_F(cell.Y0))), PWOperator.from_cell(cell).apply_H(cell.Y0), TOL64)


def test_errors_are_reported_not_raised_on_the_device():
    from paper_1406_4350_gb300.chebfi import ChebFI, ChebFIError
    from paper_1406_4350_gb300 import _lib
    cell = _tiny_paw(nb=2)
    g = ChebFI()
    with pytest.raises(ChebFIError) as e:
        g.set_sphere(cell.miller)
    assert e.value.code == _lib.ERR_STATE
    g.set_cell(cell.lattice, cell.grid, cell.kpt)
    bad = cell.miller.copy()
    bad[0] = (8, 0, 0)  # |m| must stay below N/2 = 8
    with pytest.raises(ChebFIError) as e:
        g.set_sphere(bad)
    assert e.value.code == _lib.ERR_ARG
    dup = cell.miller.copy()
    dup[1] = dup[0]
    with pytest.raises(ChebFIError) as e:
        g.set_sphere(dup)
    assert e.value.code == _lib.ERR_ARG
    g.set_sphere(cell.miller)
    g.set_vloc(cell.vloc)
    with pytest.raises(ChebFIError) as e:  # S = I - 5 P P^H is not positive definite
        g.set_projectors(cell.P, cell.proj_offsets, cell.D, -5.0 * np.concatenate(
            [np.eye(8).ravel()] * cell.natoms))
    assert e.value.code == _lib.ERR_NOT_SPD
    g.set_projectors(cell.P, cell.proj_offsets, cell.D, cell.Q)
    Y = _F(cell.Y0)
    with pytest.raises(ChebFIError) as e:
        g.cheb_filter(Y, 4, 2.0, 1.0)
    assert e.value.code == _lib.ERR_ARG
    with pytest.raises(ChebFIError) as e:  # T_n grows past 1/(100 eps) of FP32
        g.solve(Y, degree=200, sweeps=1, prec=1, bound_mode=1)
    assert e.value.code == _lib.ERR_FILTER_OVERFLOW
    g.sync_status()


# ------------------------------------------------------------------ full-size samples
@pytest.fixture(scope="module")
def paw96():
    return config_cell("paw96")


def test_full_size_apply_H_sampled_bands(paw96):
    """The 96^3 / 60005-plane-wave / 2048-projector workload: a sample of bands against
    the oracle, through the same entry points the benchmark uses."""
    from paper_1406_4350_gb300 import MIXED
    cols = [0, 777, 2047]
    Ys = np.asfortranarray(paw96.Y0[:, cols])
    op = PWOperator.from_cell(paw96)
    g = _ctx(paw96)
    ref = op.apply_H(Ys)
    _close(_np(g.apply_H(_F(Ys))), ref, TOL64)
    _close(_np(g.apply_Sinv(_F(Ys))), op.apply_Sinv(Ys), TOL64)
    _close(_np(g.apply_H(_F(Ys), prec=MIXED)), ref, TOLMIX)
    g.sync_status()


def test_paw48_forms_agree_after_convergence():
    """Config paw48 (PAW via Woodbury, 8025 plane waves, 256 bands): after convergence the FP32
    and mixed filters give the FP64 filter's Ritz values on the lowest 75 % of the bands to
    1e-8 Ha.  Degree 8 keeps T_n((lambda_1 - c)/r) below the FP32 guard (degree 10 trips it
    at this cell's lambda_1 = -5.2 Ha)."""
    from paper_1406_4350_gb300 import BOUND_RIGOROUS
    cell = config_cell("paw48")
    g = _ctx(cell)
    hi = g.upper_bound(BOUND_RIGOROUS)
    k = (3 * cell.nbands) // 4
    evs = {}
    for prec in (0, 1, 2):
        Y = _F(cell.Y0)
        ev, rs = g.solve(Y, degree=8, sweeps=40, prec=prec, lambda_hi=hi)
        evs[prec] = (_np(ev), _np(rs))
    ref, res = evs[0]
    assert res[:k].max() < 1e-7, res[:k].max()
    for prec in (1, 2):
        assert np.abs(evs[prec][0][:k] - ref[:k]).max() <= 1e-8, (prec, np.abs(evs[prec][0][:k] - ref[:k]).max())


# ----------------------------------------------------------------------------- Woodbury by refinement
def test_apply_Sinv_refined_matches_oracle_and_direct():
    """Section 5.1's iterative refinement on the device: the same S^{-1} x as the direct
    Woodbury form, in the same number of updates as the oracle's refinement."""
    from paper_1406_4350_gb300.chebfi import ChebFI, fortran
    cell = config_cell("paw48", nbands=16)
    op = PWOperator.from_cell(cell)
    g = ChebFI.from_cell(cell)
    X = fortran(cell.Y0)
    out, its = g.apply_Sinv_refined(X, tol=1e-12)
    torch.cuda.synchronize()
    ref, its_ref = op.apply_Sinv_refined(cell.Y0, tol=1e-12)
    got = out.cpu().numpy()
    scale = np.abs(cell.Y0).max()
    assert np.abs(got - ref).max() <= TOL64 * scale
    assert np.abs(got - op.apply_Sinv(cell.Y0)).max() <= TOL64 * scale
    assert abs(its - its_ref) <= 1 and 1 <= its <= 30
    # too few updates for the tolerance: an error, with the partial result written
    from paper_1406_4350_gb300.chebfi import ChebFIError
    with pytest.raises(ChebFIError):
        g.apply_Sinv_refined(X, tol=1e-12, maxit=2)


def test_apply_Sinv_refined_norm_conserving_and_singular_Q():
    from paper_1406_4350_gb300.chebfi import ChebFI, ChebFIError, fortran
    cell = make_cell(8.0, 16, 3.0, 3, 8, 2, True, 21)
    g = ChebFI.from_cell(dataclasses.replace(cell, Q=None))
    out, its = g.apply_Sinv_refined(fortran(cell.Y0))
    torch.cuda.synchronize()
    assert its == 0 and np.abs(out.cpu().numpy() - cell.Y0).max() == 0.0
    Q = cell.Q.copy()
    Q[:64] = 0.0  # first atom's D_S block is zero: no D_S^{-1}
    g = ChebFI.from_cell(dataclasses.replace(cell, Q=Q))
    with pytest.raises(ChebFIError):
        g.apply_Sinv_refined(fortran(cell.Y0))


# ----------------------------------------------------------------------------- locking (Section 5.4)
@pytest.mark.parametrize("prec, tol", [(0, TOL64), (1, TOL32), (2, TOLMIX)])
def test_cheb_filter_adaptive_matches_oracle(prec, tol):
    """Band j filtered to its own degree (0 = left alone), against the oracle band by band."""
    cell = _tiny_paw(nb=7, seed=9)
    op = PWOperator.from_cell(cell)
    hi = ch.upper_bound(op, "rigorous")
    lo = float(ch.rayleigh_quotients(op, cell.Y0).max())
    deg = np.array([4, 0, 7, 1, 4, 2, 0], dtype=np.int32)
    g = _ctx(cell)
    Y = _F(cell.Y0)
    g.cheb_filter_adaptive(Y, deg, lo, hi, prec=prec)
    ref = ch.filter_adaptive(op, cell.Y0, deg, lo, hi)
    got = _np(Y)
    for j in range(len(deg)):
        scale = np.abs(ref[:, j]).max()
        assert np.abs(got[:, j] - ref[:, j]).max() <= tol * scale, (j, deg[j])
    assert np.array_equal(got[:, 1], cell.Y0[:, 1]) and np.array_equal(got[:, 6], cell.Y0[:, 6])


@pytest.mark.parametrize("prec, lock_tol", [(0, 1e-7), (2, 3e-6)])
def test_locked_solve_nc24_reaches_exact_eigenvalues_with_less_work(prec, lock_tol):
    """Locking: after the first sweep each band gets the degree its residual estimate needs
    for the tolerance; the lowest 75 % still reach 1e-8 Ha of the exact eigenvalues (oracle
    O1) while the filters apply fewer band-H-applications than full-degree sweeps."""
    cell = config_cell("nc24")
    exact = _golden("nc24")
    g = _ctx(cell)
    Y = _F(cell.Y0)
    ev, rs = g.solve(Y, degree=8, sweeps=12, prec=prec, lock_tol=lock_tol)
    sweeps, applies = g.solve_stats()
    ev = _np(ev)
    k = (3 * cell.nbands) // 4
    assert np.abs(ev[:k] - exact[:k]).max() <= 1e-8
    assert applies < 0.8 * 8 * cell.nbands * sweeps
    assert _np(rs)[:k].max() <= 10 * lock_tol


# ----------------------------------------------------------------------------- host-block filter
@pytest.mark.parametrize("prec, tol, nchunks", [(0, TOL64, 1), (0, TOL64, 2), (0, TOL64, 3), (2, TOLMIX, 2),
                                                (1, TOL32, 0)])
def test_cheb_filter_host_block_in_chunks(prec, tol, nchunks):
    """The filter on a pinned host block, copied through the GPU in band chunks whose copies
    overlap the neighbouring chunks' filters, against the oracle (degree 5, 7 bands)."""
    cell = _tiny_paw(nb=7, seed=14)
    op = PWOperator.from_cell(cell)
    hi = ch.upper_bound(op, "rigorous")
    lo = float(ch.rayleigh_quotients(op, cell.Y0).max())
    g = _ctx(cell)
    host = torch.empty((cell.nbands, cell.npw), dtype=torch.complex128, pin_memory=True).T
    host.copy_(torch.from_numpy(cell.Y0))
    g.cheb_filter_host(host, 5, lo, hi, prec=prec, nchunks=nchunks)
    torch.cuda.synchronize()
    ref = ch.filter_reuse(op, cell.Y0, 5, lo, hi)
    _close(host.numpy(), ref, tol * 5)


def test_cheb_filter_host_block_tapered_chunks():
    """From 2048 bands up the automatic split of the host-block filter makes the first and the
    last chunk half as wide (nb/8, nb/4, nb/4, nb/4, rest): every band against the oracle."""
    cell = make_cell(8.0, 16, 3.0, 3, 8, 2049, True, 33)
    op = PWOperator.from_cell(cell)
    hi = ch.upper_bound(op, "rigorous")
    lo = float(ch.rayleigh_quotients(op, cell.Y0).max())
    g = _ctx(cell)
    host = torch.empty((cell.nbands, cell.npw), dtype=torch.complex128, pin_memory=True).T
    host.copy_(torch.from_numpy(cell.Y0))
    g.cheb_filter_host(host, 3, lo, hi, nchunks=0)
    torch.cuda.synchronize()
    _close(host.numpy(), ch.filter_reuse(op, cell.Y0, 3, lo, hi), TOL64 * 3)


# ----------------------------------------------------------------------------- projections handed over
def _proj_buf(nq, nb):
    return torch.empty((nb, nq), dtype=torch.complex128, device="cuda").T


@pytest.mark.parametrize("name", ["tiny_paw", "paw48_37"])
def test_rayleigh_ritz_returns_projections_of_the_rotated_block(name):
    """chebfi_rayleigh_ritz_proj writes P^H Y of the rotated block (the rotation's p R): against
    the oracle's P^H Y of the returned block, and the Ritz pairs unchanged."""
    cell = CELLS[name]()
    op = PWOperator.from_cell(cell)
    g = _ctx(cell)
    Y = _F(cell.Y0)
    proj = _proj_buf(cell.nproj, cell.nbands)
    ev, rs = g.rayleigh_ritz(Y, proj=proj)
    Yg = _np(Y)
    _close(_np(proj), op.projections(Yg), TOL64)
    w_ref, _ = ch.rayleigh_ritz(op, cell.Y0)
    _close(_np(ev), w_ref, TOL64)
    # a padded leading dimension
    proj2 = torch.zeros((cell.nbands, cell.nproj + 5), dtype=torch.complex128, device="cuda").T
    Y2 = _F(cell.Y0)
    g.rayleigh_ritz(Y2, proj=proj2[: cell.nproj])
    _close(_np(proj2[: cell.nproj]), op.projections(_np(Y2)), TOL64)
    assert float(proj2[cell.nproj:].abs().max()) == 0.0


@pytest.mark.parametrize("prec, tol", [(0, TOL64), (1, TOL32), (2, TOLMIX)])
@pytest.mark.parametrize("name,degree", [("tiny_paw", 5), ("paw48_37", 6)])
def test_filter_from_handed_projections_matches_oracle(name, degree, prec, tol):
    """The filter that starts from the projections Rayleigh-Ritz handed over gives the oracle's
    filter of the rotated block (Algorithm 2's loop: Rayleigh-Ritz, then the next filter)."""
    cell = CELLS[name]()
    op = PWOperator.from_cell(cell)
    hi = ch.upper_bound(op, "rigorous")
    g = _ctx(cell)
    Y = _F(cell.Y0)
    proj = _proj_buf(cell.nproj, cell.nbands)
    ev, _ = g.rayleigh_ritz(Y, proj=proj)
    lo = float(_np(ev).max())
    Yr = _np(Y)
    ref = ch.filter_reuse(op, Yr, degree, lo, hi)
    g.cheb_filter(Y, degree, lo, hi, prec=prec, proj=proj)
    g.sync_status()
    _close(_np(Y), ref, tol * degree)
    # through the host-block path, the projections in host memory, two chunks
    host = torch.empty((cell.nbands, cell.npw), dtype=torch.complex128, pin_memory=True).T
    host.copy_(torch.from_numpy(Yr))
    host_p = torch.empty((cell.nbands, cell.nproj), dtype=torch.complex128, pin_memory=True).T
    host_p.copy_(proj.cpu())
    g.cheb_filter_host(host, degree, lo, hi, prec=prec, nchunks=2, proj=host_p)
    torch.cuda.synchronize()
    _close(host.numpy(), ref, tol * degree)


def test_handed_projections_argument_checks():
    """A projection leading dimension below nproj is an argument error; projections of the
    wrong shape are refused by the binding."""
    from paper_1406_4350_gb300.chebfi import ChebFIError, _block
    cell = _tiny_paw(nb=3, seed=2)
    g = _ctx(cell)
    Y = _F(cell.Y0)
    proj = _proj_buf(cell.nproj, cell.nbands)
    y, nb, ld = _block(Y)
    pp = ctypes.c_void_p(proj.data_ptr())
    with pytest.raises(ChebFIError, match="projection leading dimension"):
        g._check(g.lib.chebfi_cheb_filter_proj(g.h, y, pp, cell.nproj - 1, nb, ld, 2, 0.0, 10.0, 0, None))
    ev = torch.empty(cell.nbands, dtype=torch.float64, device="cuda")
    with pytest.raises(ChebFIError, match="projection leading dimension"):
        g._check(g.lib.chebfi_rayleigh_ritz_proj(g.h, y, ctypes.c_void_p(ev.data_ptr()), None, pp, cell.nproj - 1,
                                                 nb, ld, None))
    with pytest.raises(ValueError):
        g.cheb_filter(Y, 2, 0.0, 10.0, proj=_proj_buf(cell.nproj + 1, cell.nbands))
    # norm-conserving projectors (S = I): the handed projections give the filter computed
    # from scratch
    nc = make_cell(8.0, 16, 3.0, 2, 1, 3, False, 5)
    h = _ctx(nc)
    Yn = _F(nc.Y0)
    pn = _proj_buf(nc.nproj, nc.nbands)
    h.rayleigh_ritz(Yn, proj=pn)
    Yn2 = Yn.clone()
    h.cheb_filter(Yn, 3, 0.0, 30.0, proj=pn)
    h.cheb_filter(Yn2, 3, 0.0, 30.0)
    _close(_np(Yn), _np(Yn2), TOL64)
