"""Pins of the FP64 oracle to facts that do not come from the oracle itself.

Each check compares the oracle against a closed form, a brute-force definition, a
library routine on a special case, or an invariant of the mathematics; the last test
plants plausible mistakes in the oracle and checks that some pin catches each one.
"""
import dataclasses

import numpy as np
import pytest

from oracle import chebyshev as ch
from oracle import planewave as pw
from oracle.exact import exact_eigs
from oracle.jacobi import jacobi_eigh
from synth import make_cell

# number of integer triples m with m.m = s (sums of three squares), s = 0..10
R3 = [1, 6, 12, 8, 6, 24, 24, 0, 12, 30, 24]


def _tiny(L=6.0, N=12, ecut=3.0, natoms=2, nlmn=8, nb=8, paw=True, seed=11):
    return make_cell(L, N, ecut, natoms, nlmn, nb, paw, seed)


def _free(cell, v0=0.0):
    return dataclasses.replace(cell, vloc=np.full_like(cell.vloc, v0), D=np.zeros_like(cell.D), Q=None)


# ----------------------------------------------------------------------------- pins
def _pin_free_electron():
    """V = 0, D = 0: eigenvalues are the shells (2 pi^2 / L^2) s with multiplicity r3(s)."""
    L, ecut = 6.0, 3.0
    cell = _free(_tiny(L=L, ecut=ecut))
    w = exact_eigs(pw.PWOperator.from_cell(cell))
    smax = int(np.floor(2 * ecut * L * L / (4 * np.pi ** 2)))
    expect = np.concatenate([np.full(R3[s], 2 * np.pi ** 2 / L ** 2 * s) for s in range(smax + 1)])
    assert w.shape == expect.shape
    np.testing.assert_allclose(w, expect, rtol=0, atol=1e-12)


def _pin_constant_shift():
    """V = V0 everywhere shifts every free-electron eigenvalue by exactly V0."""
    L, ecut, v0 = 6.0, 3.0, -0.7310
    cell = _free(_tiny(L=L, ecut=ecut), v0)
    w = exact_eigs(pw.PWOperator.from_cell(cell))
    smax = int(np.floor(2 * ecut * L * L / (4 * np.pi ** 2)))
    expect = np.concatenate([np.full(R3[s], 2 * np.pi ** 2 / L ** 2 * s) for s in range(smax + 1)]) + v0
    np.testing.assert_allclose(w, expect, rtol=0, atol=1e-12)


def _pin_cosine_potential():
    """V(j) = 2A cos(2 pi n0.j/N + phi) has V~(n0) = A e^{i phi}: the local matrix element
    <e_G|V|e_G'> equals A e^{i phi} when m - m' = n0, A e^{-i phi} when m - m' = -n0."""
    cell = _tiny(N=12)
    N = 12
    A, phi, n0 = 0.37, 0.9, np.array([1, 2, 0])
    j = np.stack(np.meshgrid(*[np.arange(N)] * 3, indexing="ij"), -1)
    v = 2 * A * np.cos(2 * np.pi * (j @ n0) / N + phi)
    cell = dataclasses.replace(cell, vloc=v, D=np.zeros_like(cell.D), Q=None)
    op = pw.PWOperator.from_cell(cell)
    H = pw.dense_H(op) - np.diag(op.K)
    m = cell.miller.astype(int)
    diff = m[:, None, :] - m[None, :, :]
    plus = np.all(diff == n0, axis=-1)
    minus = np.all(diff == -n0, axis=-1)
    assert plus.sum() > 10
    np.testing.assert_allclose(H[plus], A * np.exp(1j * phi), atol=1e-13)
    np.testing.assert_allclose(H[minus], A * np.exp(-1j * phi), atol=1e-13)
    np.testing.assert_allclose(H[~(plus | minus)], 0.0, atol=1e-13)
    # the matrix-free FFT path agrees with the brute-force matrix on random vectors
    rng = np.random.default_rng(3)
    x = rng.normal(size=(cell.npw, 3)) + 1j * rng.normal(size=(cell.npw, 3))
    np.testing.assert_allclose(op.apply_local(x), H @ x, atol=1e-12)


def _pin_vtilde_bruteforce():
    """V~(n) = (1/N^3) sum_j V(j) e^{-2 pi i n.j/N} by explicit sums on a 6^3 grid."""
    rng = np.random.default_rng(5)
    N = 6
    v = rng.normal(size=(N, N, N))
    vt = pw.vtilde(v)
    j = np.stack(np.meshgrid(*[np.arange(N)] * 3, indexing="ij"), -1).reshape(-1, 3)
    for n in [(0, 0, 0), (1, 0, 0), (0, 2, 5), (3, 1, 4), (5, 5, 5)]:
        brute = sum(v[tuple(jj)] * np.exp(-2j * np.pi * np.dot(n, jj) / N) for jj in j) / N ** 3
        assert abs(vt[n] - brute) < 1e-14


def _pin_hermitian():
    """<x, H y> = conj <y, H x> and the same for S, S^{-1} (Eq. KS: H, S Hermitian)."""
    cell = _tiny(N=12, natoms=3)
    op = pw.PWOperator.from_cell(cell)
    rng = np.random.default_rng(7)
    x = rng.normal(size=(cell.npw, 2)) + 1j * rng.normal(size=(cell.npw, 2))
    y = rng.normal(size=(cell.npw, 2)) + 1j * rng.normal(size=(cell.npw, 2))
    for f in (op.apply_H, op.apply_S, op.apply_Sinv):
        a = np.einsum("gn,gn->n", x.conj(), f(y))
        b = np.einsum("gn,gn->n", y.conj(), f(x)).conj()
        np.testing.assert_allclose(a, b, rtol=1e-12)
    Hd = pw.dense_H(op)
    np.testing.assert_allclose(Hd, Hd.conj().T, atol=1e-13)
    np.testing.assert_allclose(op.apply_H(x), Hd @ x, atol=1e-12)
    np.testing.assert_allclose(op.apply_S(x), pw.dense_S(op) @ x, atol=1e-12)


def _pin_secular_rank1():
    """V = 0 and one projector p with coefficient d: every eigenvalue lambda off the
    kinetic values solves 1 = d sum_G |p_G|^2 / (lambda - K_G) (rank-one update)."""
    L = 6.0
    cell = _tiny(L=L, natoms=1, nlmn=1, paw=False)
    d = 0.8
    cell = dataclasses.replace(cell, vloc=np.zeros_like(cell.vloc), D=np.array([d]))
    op = pw.PWOperator.from_cell(cell)
    w = exact_eigs(op)
    m = cell.miller.astype(float)
    K = 2 * np.pi ** 2 / L ** 2 * np.sum(m * m, 1)
    p2 = np.abs(cell.P[:, 0]) ** 2
    shells = np.unique(np.round(K, 10))
    off = [lam for lam in w if np.min(np.abs(shells - lam)) > 1e-6]
    # one secular root per distinct shell the projector touches
    assert len(off) == len(shells)
    for lam in off:
        f = 1.0 - d * np.sum(p2 / (lam - K))
        assert abs(f) < 1e-9, (lam, f)


def _pin_woodbury():
    """S (S^{-1} x) = x with S applied directly, and S^{-1} x equals a dense solve."""
    cell = _tiny(N=12, natoms=3)
    op = pw.PWOperator.from_cell(cell)
    rng = np.random.default_rng(9)
    x = rng.normal(size=(cell.npw, 4)) + 1j * rng.normal(size=(cell.npw, 4))
    np.testing.assert_allclose(op.apply_S(op.apply_Sinv(x)), x, atol=1e-12)
    np.testing.assert_allclose(op.apply_Sinv(x), np.linalg.solve(pw.dense_S(op), x), atol=1e-12)


def _pin_chebyshev_closed_forms():
    """T_n(cos t) = cos(n t) inside [a, b] and T_n(cosh t) = cosh(n t) above it."""
    a, b = -1.3, 2.9
    c, r = 0.5 * (a + b), 0.5 * (b - a)
    t = np.linspace(0.0, np.pi, 37)
    for n in range(0, 12):
        x = c + r * np.cos(t)
        np.testing.assert_allclose(ch.cheb_T(n, x, a, b), np.cos(n * t), atol=1e-12)
        s = np.linspace(0.0, 2.0, 9)
        np.testing.assert_allclose(ch.cheb_T(n, c + r * np.cosh(s), a, b), np.cosh(n * s), rtol=1e-12)
        np.testing.assert_allclose(ch.cheb_T(n, c - r * np.cosh(s), a, b), (-1) ** n * np.cosh(n * s),
                                   rtol=1e-12)


def _pin_filter_on_eigenvectors():
    """With V = V0 and no projectors every plane wave e_G is an eigenvector with
    lambda = K_G + V0, so the filter of Algorithm 2 returns T_n((lambda - c)/r) e_G, with T_n
    from its cosh / cos closed form."""
    L, v0 = 6.0, 0.25
    cell = _free(_tiny(L=L), v0)
    op = pw.PWOperator.from_cell(cell)
    m = cell.miller.astype(float)
    lam = 2 * np.pi ** 2 / L ** 2 * np.sum(m * m, 1) + v0
    cols = [0, 3, 9, 20, 40]
    Y = np.zeros((cell.npw, len(cols)), complex)
    Y[cols, range(len(cols))] = 1.0
    lo, hi, n = 0.9, 3.2, 7
    c, r = 0.5 * (hi + lo), 0.5 * (hi - lo)
    y = (lam[cols] - c) / r
    tn = np.where(np.abs(y) <= 1, np.cos(n * np.arccos(np.clip(y, -1, 1))),
                  np.sign(y) ** n * np.cosh(n * np.arccosh(np.maximum(np.abs(y), 1))))
    for f in (ch.filter_plain, ch.filter_reuse):
        out = f(op, Y, n, lo, hi)
        np.testing.assert_allclose(out[cols, range(len(cols))], tn, rtol=1e-11)
        out[cols, range(len(cols))] = 0
        assert np.abs(out).max() < 1e-10


def _pencil_eigenpairs(cell):
    """Eigenpairs of the dense pencil (H, S) from LAPACK, S-normalised: x^H S x = 1."""
    import scipy.linalg
    op = pw.PWOperator.from_cell(cell)
    H, S = pw.dense_H(op), pw.dense_S(op)
    w, X = scipy.linalg.eigh(H, S)
    return op, H, S, w, X


def _pin_rayleigh_quotients():
    """Rayleigh quotients (Algorithm 2's first step): an exact eigenvector of the pencil gives
    its eigenvalue whatever its scale; a plane wave e_G with V = V0 and no projectors gives
    K_G + V0 = 2 pi^2 |m|^2 / L^2 + V0."""
    cell = _tiny(N=12, natoms=3, nb=6, seed=13)
    op, H, S, w, X = _pencil_eigenpairs(cell)
    cols = [0, 1, 5, 17, len(w) - 1]
    scale = np.array([1.0, -3.0, 0.5j, 2.0 + 1.0j, 1e-3])
    rq = ch.rayleigh_quotients(op, X[:, cols] * scale[None, :])
    np.testing.assert_allclose(rq, w[cols], rtol=0, atol=1e-11)
    L, v0 = 6.0, -0.41
    free = _free(_tiny(L=L), v0)
    fop = pw.PWOperator.from_cell(free)
    m = free.miller.astype(float)
    pick = [0, 2, 11, 30]
    E = np.zeros((free.npw, len(pick)), complex)
    E[pick, range(len(pick))] = 1.0
    np.testing.assert_allclose(ch.rayleigh_quotients(fop, E),
                               2 * np.pi ** 2 / L ** 2 * np.sum(m[pick] ** 2, 1) + v0, atol=1e-12)


def _pin_residuals():
    """Residual norms ||H y - w S y||: zero for exact eigenpairs of the pencil; for
    y = x_i + eps e_G with w = lambda_i, exactly eps ||(H - lambda_i S) e_G||, the norm of
    column G of the dense H - lambda_i S; and x_i with w = lambda_i + delta gives
    |delta| ||S x_i||."""
    cell = _tiny(N=12, natoms=3, nb=6, seed=13)
    op, H, S, w, X = _pencil_eigenpairs(cell)
    cols = [0, 3, 8, 21]
    r = ch.residuals(op, X[:, cols], w[cols])
    assert np.abs(r).max() <= 1e-10 * max(1.0, np.abs(w).max())
    eps, g = 1e-3, 7
    Y = X[:, cols].copy()
    Y[g, :] += eps
    expect = eps * np.linalg.norm(H[:, g][:, None] - S[:, g][:, None] * w[cols][None, :], axis=0)
    np.testing.assert_allclose(ch.residuals(op, Y, w[cols]), expect, rtol=1e-8)
    delta = 0.125
    expect2 = delta * np.linalg.norm(S @ X[:, cols], axis=0)
    np.testing.assert_allclose(ch.residuals(op, X[:, cols], w[cols] + delta), expect2, rtol=1e-8)


# ----------------------------------------------------------------------------- tests
def test_free_electron_shells():
    _pin_free_electron()


def test_constant_potential_shift():
    _pin_constant_shift()


def test_cosine_potential_matrix_elements():
    _pin_cosine_potential()


def test_vtilde_against_explicit_sums():
    _pin_vtilde_bruteforce()


def test_hermiticity():
    _pin_hermitian()


def test_rank_one_secular_equation():
    _pin_secular_rank1()


def test_woodbury_inverse():
    _pin_woodbury()


def test_chebyshev_closed_forms():
    _pin_chebyshev_closed_forms()


def test_filter_scales_eigenvectors_by_Tn():
    _pin_filter_on_eigenvectors()


@pytest.mark.parametrize("n", [1, 2, 3, 7, 40, 121])
def test_jacobi_matches_lapack(n):
    rng = np.random.default_rng(n)
    X = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    A = X + X.conj().T
    w, V = jacobi_eigh(A)
    np.testing.assert_allclose(w, np.linalg.eigvalsh(A), atol=1e-11 * max(1, np.abs(w).max()))
    np.testing.assert_allclose(A @ V, V * w, atol=1e-10)
    np.testing.assert_allclose(V.conj().T @ V, np.eye(n), atol=1e-12)


def test_jacobi_degenerate_and_diagonal():
    rng = np.random.default_rng(1)
    d = np.array([1.0, 1.0, 1.0, -2.0, 5.0, 5.0])
    Q, _ = np.linalg.qr(rng.normal(size=(6, 6)) + 1j * rng.normal(size=(6, 6)))
    A = Q @ np.diag(d) @ Q.conj().T
    w, V = jacobi_eigh(A)
    np.testing.assert_allclose(w, np.sort(d), atol=1e-13)
    w2, _ = jacobi_eigh(np.diag(d))
    np.testing.assert_array_equal(w2, np.sort(d))


def test_filter_reuse_equals_plain_and_projections_track():
    """The projection-reuse identity of Section 5.1 changes no result: the carried
    projections equal freshly computed P^H psi."""
    cell = _tiny(N=12, natoms=3, nb=6)
    op = pw.PWOperator.from_cell(cell)
    lo, hi = 0.5, ch.upper_bound(op, "rigorous")
    a = ch.filter_plain(op, cell.Y0, 6, lo, hi)
    b, p = ch.filter_reuse(op, cell.Y0, 6, lo, hi, return_proj=True)
    scale = np.abs(a).max()
    np.testing.assert_allclose(b, a, atol=1e-11 * scale)
    np.testing.assert_allclose(p, op.projections(b), atol=1e-11 * scale)


def test_norm_conserving_is_paw_limit():
    """S = I is the D_S -> 0 limit of the PAW operators."""
    cell = _tiny(N=12, natoms=2, nb=4)
    tiny_q = dataclasses.replace(cell, Q=cell.Q * 1e-10)
    nc = dataclasses.replace(cell, Q=None)
    a = pw.PWOperator.from_cell(tiny_q)
    b = pw.PWOperator.from_cell(nc)
    x = cell.Y0
    np.testing.assert_allclose(a.apply_Sinv(x), b.apply_Sinv(x), atol=1e-9)
    np.testing.assert_allclose(ch.filter_reuse(a, x, 4, 0.5, 9.0), ch.filter_reuse(b, x, 4, 0.5, 9.0),
                               rtol=1e-8, atol=1e-8)


def test_rayleigh_ritz_invariants_and_interlacing():
    """After Rayleigh-Ritz Y^H S Y = I, Y^H H Y = diag(w), and each Ritz value is at
    least the exact eigenvalue of the same index (Cauchy interlacing)."""
    cell = _tiny(N=12, natoms=3, nb=10)
    op = pw.PWOperator.from_cell(cell)
    w, Y = ch.rayleigh_ritz(op, cell.Y0)
    np.testing.assert_allclose(Y.conj().T @ op.apply_S(Y), np.eye(10), atol=1e-12)
    np.testing.assert_allclose(Y.conj().T @ op.apply_H(Y), np.diag(w), atol=1e-11)
    exact = exact_eigs(op)
    assert np.all(w >= exact[:10] - 1e-12)


def test_solve_converges_to_exact_and_residual_bounds_hold():
    cell = _tiny(L=8.0, N=16, ecut=3.0, natoms=4, nb=16, seed=7)
    op = pw.PWOperator.from_cell(cell)
    exact = exact_eigs(op)
    res = ch.solve(op, cell.Y0, degree=8, sweeps=9, mode="rigorous")
    k = 12  # lowest 75 %
    assert np.abs(res["w"][:k] - exact[:k]).max() < 1e-8
    bnd = ch.residual_bound(op, res["Y"], res["w"])
    for wi, bi in zip(res["w"], bnd):
        # rounding of the exact eigenvalues themselves is ~ n eps ||H||
        assert np.min(np.abs(exact - wi)) <= bi * (1 + 1e-6) + 1e-12 * np.abs(exact).max()


def test_rigorous_upper_bound_is_an_upper_bound():
    cell = _tiny(L=8.0, N=16, ecut=3.0, natoms=4, nb=4, seed=7)
    op = pw.PWOperator.from_cell(cell)
    exact = exact_eigs(op)
    assert exact.max() <= ch.upper_bound(op, "rigorous")


def test_rayleigh_quotients_of_exact_eigenpairs_and_plane_waves():
    _pin_rayleigh_quotients()


def test_residuals_of_exact_and_perturbed_eigenpairs():
    _pin_residuals()


# --------------------------------------------------------------- planted mistakes
def _mut_kinetic(monkeypatch):
    orig = pw.kinetic
    monkeypatch.setattr(pw, "kinetic", lambda *a: 2.0 * orig(*a))


def _mut_vtilde_conj(monkeypatch):
    orig = pw.vtilde
    monkeypatch.setattr(pw, "vtilde", lambda v: np.conj(orig(v)))


def _mut_projection_transpose(monkeypatch):
    monkeypatch.setattr(pw.PWOperator, "projections", lambda self, Y: self.P.T @ Y)


def _mut_woodbury_sign(monkeypatch):
    orig = pw.PWOperator.apply_Sinv
    monkeypatch.setattr(pw.PWOperator, "apply_Sinv", lambda self, X: 2 * np.asarray(X) - orig(self, X))


def _mut_recurrence(monkeypatch):
    def bad(op, Y, degree, lo, hi):
        c, r = 0.5 * (hi + lo), 0.5 * (hi - lo)
        prev = np.array(Y, complex)
        cur = (op.apply_Sinv(op.apply_H(prev)) - c * prev) / r
        for _ in range(2, degree + 1):
            cur, prev = 1.0 / r * (op.apply_Sinv(op.apply_H(cur)) - c * cur) - prev, cur
        return cur
    monkeypatch.setattr(ch, "filter_plain", bad)


def _mut_rq_without_S(monkeypatch):
    def bad(op, Y):
        Y = np.asarray(Y)
        return (np.einsum("gn,gn->n", Y.conj(), op.apply_H(Y)).real
                / np.einsum("gn,gn->n", Y.conj(), Y).real)
    monkeypatch.setattr(ch, "rayleigh_quotients", bad)


def _mut_residual_without_S(monkeypatch):
    monkeypatch.setattr(ch, "residuals",
                        lambda op, Y, w: np.linalg.norm(op.apply_H(Y) - np.asarray(Y) * np.asarray(w)[None, :],
                                                        axis=0))


def _mut_residual_sign(monkeypatch):
    monkeypatch.setattr(ch, "residuals",
                        lambda op, Y, w: np.linalg.norm(op.apply_H(Y) + op.apply_S(Y) * np.asarray(w)[None, :],
                                                        axis=0))


@pytest.mark.parametrize("mutation, pins", [
    (_mut_kinetic, [_pin_free_electron]),
    (_mut_vtilde_conj, [_pin_cosine_potential]),
    (_mut_projection_transpose, [_pin_hermitian]),
    (_mut_woodbury_sign, [_pin_woodbury]),
    (_mut_recurrence, [_pin_filter_on_eigenvectors]),
    (_mut_rq_without_S, [_pin_rayleigh_quotients]),
    (_mut_residual_without_S, [_pin_residuals]),
    (_mut_residual_sign, [_pin_residuals]),
])
def test_pins_catch_planted_mistakes(monkeypatch, mutation, pins):
    mutation(monkeypatch)
    for pin in pins:
        with pytest.raises(AssertionError):
            pin()


def test_woodbury_iterative_refinement_reaches_the_direct_solve():
    """Section 5.1's solve of the reduced system by block-diagonally preconditioned
    iterative refinement converges to the direct Woodbury result (and hence to S^{-1} x)."""
    cell = _tiny(N=12, natoms=3)
    op = pw.PWOperator.from_cell(cell)
    rng = np.random.default_rng(12)
    x = rng.normal(size=(cell.npw, 3)) + 1j * rng.normal(size=(cell.npw, 3))
    y, its = op.apply_Sinv_refined(x, tol=1e-14)
    assert 1 <= its < 200
    np.testing.assert_allclose(y, op.apply_Sinv(x), atol=1e-12)
    np.testing.assert_allclose(op.apply_S(y), x, atol=1e-11)
    # the update count follows the contraction factor: the residual shrinks by about rho
    # per update, so reaching 1e-14 takes about log(1e-14)/log(rho) updates
    rho, kappa = op.refinement_diagnostics()
    assert 0.0 < rho < 1.0 and kappa >= 1.0
    assert its <= np.ceil(np.log(1e-14) / np.log(rho)) + 8
    # a tolerance of 1 is met before any update; maxit = 0 makes no update either
    assert op.apply_Sinv_refined(x, tol=1.0)[1] == 0
    y0, its0 = op.apply_Sinv_refined(x, tol=1e-14, maxit=0)
    assert its0 == 0 and np.allclose(y0, x)


def test_filter_setup_and_threaded_ffts_do_not_change_the_filter():
    """The CPU baseline forms Section 5.1's G = P^H P and the reduced matrix's factors once and
    runs the FFTs on several threads: the filter's result is the same to rounding."""
    cell = _tiny(N=12, natoms=3, nb=5, seed=17)
    op = pw.PWOperator.from_cell(cell)
    lo, hi = 0.4, ch.upper_bound(op, "rigorous")
    ref = ch.filter_reuse(op, cell.Y0, 6, lo, hi)
    setup = ch.filter_setup(op)
    op.fft_workers = 4
    got = ch.filter_reuse(op, cell.Y0, 6, lo, hi, setup=setup)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * np.abs(ref).max())
