"""FP64 complex GEMMs on the tensor cores (the modular emulation) through the C ABI.

The emulation scales every row of op(A) and column of op(B) by a power of two to a 2-norm
in [2^(E-1), 2^E), rounds to integers, multiplies their residues modulo 8-15 coprime
moduli exactly on the bf16 tensor pipe and rebuilds the integer product by the Chinese
remainder theorem.  What fixes its results independently of its own code:

* integer matrices whose scaled entries need no rounding give the exact integer product,
  bit for bit (this pins the exact FP32 chunk sums, the modular reductions and the CRT);
* for real data the error of entry (m, n) is at most a small multiple of
  2^-E ||a_m|| ||b_n|| (E = 53 for 14 moduli), measured against a product evaluated in
  numpy's extended precision;
* the error falls by about 2^(E2 - E1) from one modulus count to the next;
* Algorithm 2's FP64 steps (filter, Rayleigh-Ritz, Cholesky-QR, solve) with every GEMM
  forced onto the tensor cores agree with the FP64 oracle at the FP64 tolerance used for
  the CUDA-core path.
"""
import numpy as np
import pytest
import torch

from oracle import chebyshev as ch
from oracle.planewave import PWOperator
from synth import config_cell, make_cell

pytestmark = pytest.mark.gpu

TOL64 = 1e-11


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1406_4350_gb300 import build
    build.build()


def _F(x):
    from paper_1406_4350_gb300.chebfi import fortran
    return fortran(x)


def _ctx(cell=None):
    from paper_1406_4350_gb300.chebfi import ChebFI
    return ChebFI.from_cell(cell) if cell is not None else ChebFI(0)


def _np(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _rand(rng, m, n):
    return rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))


def _op(X, conj):
    return X.conj().T if conj else X


def _ref(A, B, conjA, conjB):
    """The product in numpy's extended precision (64 or 113 significand bits)."""
    a = _op(A, conjA)
    b = _op(B, conjB)
    ar, ai = a.real.astype(np.longdouble), a.imag.astype(np.longdouble)
    br, bi = b.real.astype(np.longdouble), b.imag.astype(np.longdouble)
    return (ar @ br - ai @ bi), (ar @ bi + ai @ br)


def _bound(A, B, conjA, conjB):
    """||row m of op(A)|| ||column n of op(B)|| for every entry."""
    ra = np.linalg.norm(_op(A, conjA), axis=1)
    cb = np.linalg.norm(_op(B, conjB), axis=0)
    return ra[:, None] * cb[None, :]


def test_integer_products_are_exact():
    from paper_1406_4350_gb300._lib import GEMM_TENSOR
    rng = np.random.default_rng(7)
    m, n, k = 200, 131, 3001  # ragged against the 64 x 128 complex tiles and the 512-product chunks
    A = rng.integers(-1000, 1001, (m, k)) + 1j * rng.integers(-1000, 1001, (m, k))
    B = rng.integers(-1000, 1001, (k, n)) + 1j * rng.integers(-1000, 1001, (k, n))
    exact_re = A.real.astype(np.int64) @ B.real.astype(np.int64) - A.imag.astype(np.int64) @ B.imag.astype(np.int64)
    exact_im = A.real.astype(np.int64) @ B.imag.astype(np.int64) + A.imag.astype(np.int64) @ B.real.astype(np.int64)
    g = _ctx()
    g.set_fp64_gemm(GEMM_TENSOR, 14)
    C = _np(g.gemm_fp64(_F(A), _F(B)))
    assert np.array_equal(C.real, exact_re.astype(np.float64))
    assert np.array_equal(C.imag, exact_im.astype(np.float64))


@pytest.mark.parametrize("conjA,conjB", [(False, False), (True, False), (False, True), (True, True)])
def test_random_products_within_fp64_bound(conjA, conjB):
    from paper_1406_4350_gb300._lib import GEMM_CUDA_CORES, GEMM_TENSOR
    rng = np.random.default_rng(11 + 2 * conjA + conjB)
    m, n, k = 96, 70, 1500
    A = _rand(rng, k, m) if conjA else _rand(rng, m, k)
    B = _rand(rng, n, k) if conjB else _rand(rng, k, n)
    # entries spread over six decades, as plane-wave coefficients are
    A *= np.exp(rng.uniform(-7, 7, A.shape))
    ref_re, ref_im = _ref(A, B, conjA, conjB)
    bound = _bound(A, B, conjA, conjB)
    g = _ctx()
    E = g.set_fp64_gemm(GEMM_TENSOR, 14)
    assert E == 53
    C = _np(g.gemm_fp64(_F(A), _F(B), conjA, conjB))
    err = np.maximum(np.abs(C.real - ref_re), np.abs(C.imag - ref_im)).astype(np.float64) / bound
    # scaling error about 2 x 2^-E, plus the rounding of the FP64 result itself
    assert err.max() <= 4.0 * 2.0 ** -E + 2.0 ** -52, "tensor-core error %.3e x ||a|| ||b||" % err.max()
    # the CUDA-core FP64 product of the same operands: same order of error
    g.set_fp64_gemm(GEMM_CUDA_CORES)
    C2 = _np(g.gemm_fp64(_F(A), _F(B), conjA, conjB))
    err2 = np.maximum(np.abs(C2.real - ref_re), np.abs(C2.imag - ref_im)).astype(np.float64) / bound
    assert err2.max() <= 64.0 * 2.0 ** -53
    assert np.abs(C - C2).max() <= 1e-13 * bound.max()


def test_precision_follows_the_modulus_count():
    from paper_1406_4350_gb300._lib import GEMM_TENSOR
    rng = np.random.default_rng(3)
    A, B = _rand(rng, 64, 777), _rand(rng, 777, 40)
    ref_re, ref_im = _ref(A, B, False, False)
    bound = _bound(A, B, False, False)
    g = _ctx()
    errs = {}
    for nmod in (8, 10, 12, 14, 15):
        E = g.set_fp64_gemm(GEMM_TENSOR, nmod)
        C = _np(g.gemm_fp64(_F(A), _F(B)))
        err = (np.maximum(np.abs(C.real - ref_re), np.abs(C.imag - ref_im)).astype(np.float64) / bound).max()
        errs[nmod] = (E, err)
        assert err <= 4.0 * 2.0 ** -E + 2.0 ** -52, (nmod, E, err)
        if E < 50:  # above the rounding of the FP64 output itself the bound is reached, not beaten by far
            assert err >= 2.0 ** -(E + 12), (nmod, E, err)
    assert errs[8][1] > errs[10][1] > errs[12][1] > errs[14][1]


def test_beta_zero_rows_nan_rows_and_tiny_shapes():
    from paper_1406_4350_gb300._lib import GEMM_TENSOR
    rng = np.random.default_rng(5)
    A, B = _rand(rng, 70, 300), _rand(rng, 300, 9)
    A[3] = 0.0
    A[5, 17] = np.nan
    C0 = _rand(rng, 70, 9)
    g = _ctx()
    g.set_fp64_gemm(GEMM_TENSOR, 14)
    C = _np(g.gemm_fp64(_F(A), _F(B), alpha=-0.5, beta=2.0, C=_F(C0)))
    ok = np.ones(70, bool)
    ok[5] = False
    ref = -0.5 * (A[ok] @ B) + 2.0 * C0[ok]
    assert np.abs(C[ok] - ref).max() <= 1e-13 * np.abs(ref).max()
    assert np.array_equal(C[3], 2.0 * C0[3])
    assert np.isnan(C[5]).all()
    # K below one k-tile, one row, one column
    for (m, n, k) in [(1, 1, 1), (1, 5, 3), (7, 1, 40), (129, 2, 63)]:
        a, b = _rand(rng, m, k), _rand(rng, k, n)
        c = _np(g.gemm_fp64(_F(a), _F(b)))
        assert np.abs(c - a @ b).max() <= 1e-14 * max(np.abs(a @ b).max(), 1.0), (m, n, k)


@pytest.fixture(scope="module")
def paw48():
    return config_cell("paw48", nbands=37)


@pytest.mark.parametrize("name", ["tiny_paw", "paw48_37"])
def test_fp64_steps_with_tensor_gemms_match_oracle(name, paw48):
    from paper_1406_4350_gb300._lib import GEMM_TENSOR
    cell = make_cell(8.0, 16, 3.0, 3, 8, 7, True, 21) if name == "tiny_paw" else paw48
    op = PWOperator.from_cell(cell)
    g = _ctx(cell)
    g.set_fp64_gemm(GEMM_TENSOR, 14)
    Y = _F(cell.Y0)

    def close(got, ref):
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err <= TOL64, "relative error %.3e" % err

    close(_np(g.apply_H(Y)), op.apply_H(cell.Y0))
    close(_np(g.apply_S(Y)), op.apply_S(cell.Y0))
    close(_np(g.apply_Sinv(Y)), op.apply_Sinv(cell.Y0))
    lo = float(ch.rayleigh_quotients(op, cell.Y0).max())
    hi = ch.upper_bound(op, "rigorous")
    degree = 5 if name == "tiny_paw" else 10
    ref = ch.filter_reuse(op, cell.Y0, degree, lo, hi)
    Yf = _F(cell.Y0)
    g.cheb_filter(Yf, degree, lo, hi)
    close(_np(Yf), ref)
    # Rayleigh-Ritz (Hermitian lower-triangle products, rotations) against the oracle
    w_ref, X_ref = ch.rayleigh_ritz(op, ref)
    ev, rs = g.rayleigh_ritz(Yf)
    assert np.abs(_np(ev) - w_ref).max() <= 1e-9
    r_ref = ch.residuals(op, X_ref, w_ref)
    assert np.abs(_np(rs) - r_ref).max() <= 1e-6 * max(r_ref.max(), 1e-3)
    # Cholesky-QR: Y^H S Y = I with the oracle's S
    Yo = _F(cell.Y0)
    g.orthonormalise(Yo)
    Yn = _np(Yo)
    G = Yn.conj().T @ op.apply_S(Yn)
    assert np.abs(G - np.eye(G.shape[0])).max() <= 1e-11


def test_solve_with_tensor_gemms_matches_oracle_algorithm(paw48):
    """Same start, lambda_+, degree and sweeps as the oracle's Algorithm 2: every Ritz value
    agrees at the rounding level with every FP64 GEMM on the tensor cores."""
    from paper_1406_4350_gb300._lib import GEMM_TENSOR
    cell = paw48
    op = PWOperator.from_cell(cell)
    hi = ch.upper_bound(op, "rigorous")
    ref = ch.solve(op, cell.Y0, degree=10, sweeps=2, lam_hi=hi)
    g = _ctx(cell)
    g.set_fp64_gemm(GEMM_TENSOR, 14)
    Y = _F(cell.Y0)
    ev, rs = g.solve(Y, degree=10, sweeps=2, lambda_hi=hi)
    assert np.abs(_np(ev) - ref["w"]).max() <= 1e-9
    r = _np(rs)
    assert np.abs(r - ref["resid"]).max() <= 1e-6 * ref["resid"].max()
