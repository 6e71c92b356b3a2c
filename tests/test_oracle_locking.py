"""Locking with per-band degrees (Section 5.4): pins of the oracle's degree rule and
locked solve, and the library's host-side degree rule against the oracle's (no GPU)."""
import dataclasses

import numpy as np
import pytest

from oracle import chebyshev as ch
from oracle.exact import exact_eigs
from oracle.planewave import PWOperator
from synth import make_cell


def _closed_form_degree(lam, res, lo, hi, tol, nmax):
    """|T_n(x)| = cosh(n arccosh |x|) for |x| >= 1, so the smallest n with res <= tol |T_n| is
    ceil(arccosh(res / tol) / arccosh |x|); inside the interval |T_n| <= 1 never gets there."""
    if res <= tol:
        return 0
    x = abs((lam - 0.5 * (hi + lo)) / (0.5 * (hi - lo)))
    if x <= 1.0:
        return nmax
    n = int(np.ceil(np.arccosh(res / tol) / np.arccosh(x)))
    return min(max(n, 1), nmax)


def test_degree_rule_matches_the_closed_form():
    rng = np.random.default_rng(0)
    lo, hi, tol, nmax = 0.3, 25.0, 1e-9, 40
    lam = rng.uniform(-6.0, 2.0, size=400)
    res = 10.0 ** rng.uniform(-12, -1, size=400)
    got = ch.adaptive_degrees(lam, res, lo, hi, tol, nmax)
    want = np.array([_closed_form_degree(l, r, lo, hi, tol, nmax) for l, r in zip(lam, res)])
    # the two evaluations of T_n may straddle the threshold only when the ratio is within
    # rounding of an integer; none of these draws is
    assert np.array_equal(got, want)
    assert np.all(got[res <= tol] == 0)


def test_filter_adaptive_is_the_per_band_filter():
    cell = make_cell(6.0, 12, 3.0, 2, 8, 5, True, 11)
    op = PWOperator.from_cell(cell)
    deg = np.array([3, 0, 5, 3, 1])
    lo, hi = 0.5, 12.0
    out = ch.filter_adaptive(op, cell.Y0, deg, lo, hi)
    for j, d in enumerate(deg):
        np.testing.assert_allclose(out[:, j], ch.filter_plain(op, cell.Y0[:, j:j + 1], int(d), lo, hi)[:, 0],
                                   rtol=0, atol=1e-12 * np.abs(out[:, j]).max())
    np.testing.assert_array_equal(out[:, 1], cell.Y0[:, 1])


def test_residual_estimate_predicts_the_next_sweep():
    """Near convergence the estimate ||r_i|| / |T_n((lambda_i - c)/r)| is close to the residual
    actually reached after filtering band i to degree n and Rayleigh-Ritz."""
    cell = make_cell(8.0, 16, 3.0, 3, 8, 12, True, 31)
    op = PWOperator.from_cell(cell)
    hi = ch.upper_bound(op, "rigorous")
    Y = cell.Y0
    lo = float(ch.rayleigh_quotients(op, Y).max())
    for _ in range(6):
        w, Y = ch.rayleigh_ritz(op, ch.filter_plain(op, Y, 6, lo, hi))
        lo = float(w.max())
    res = ch.residuals(op, Y, w)
    deg = ch.adaptive_degrees(w, res, lo, hi, 1e-9, 20)
    assert 0 < (deg == 0).sum() < len(deg) and (deg == 20).sum() < len(deg)
    pred = np.array([r / abs(float(ch.cheb_T(int(d), l, lo, hi))) for l, r, d in zip(w, res, deg)])
    w2, Y2 = ch.rayleigh_ritz(op, ch.filter_adaptive(op, Y, deg, lo, hi))
    res2 = ch.residuals(op, Y2, w2)
    ratio = res2 / pred
    assert np.all(ratio > 0.3) and np.all(ratio < 1.5), ratio


def test_locked_solve_reaches_exact_eigenvalues_with_less_work():
    cell = make_cell(6.0, 12, 3.0, 2, 8, 8, True, 13)
    op = PWOperator.from_cell(cell)
    exact = exact_eigs(op)[:8]
    Y, w, res, used = ch.solve_locked(op, cell.Y0, 10, 12, 1e-8, mode="rigorous")
    k = 6  # the lowest 75% of the bands
    assert np.abs(w[:k] - exact[:k]).max() <= 1e-8
    full = 10 * 8 * len(used)
    assert sum(int(u.sum()) for u in used) < 0.8 * full
    assert any((u == 0).any() for u in used[1:])  # some bands were locked


def test_library_degree_rule_equals_the_oracle():
    """chebfi_adaptive_degrees is host code: it runs here without a GPU."""
    from paper_1406_4350_gb300 import build
    from paper_1406_4350_gb300.chebfi import ChebFI
    build.build()
    rng = np.random.default_rng(1)
    for trial in range(5):
        lo, hi = rng.uniform(-1, 1), rng.uniform(5, 40)
        lam = rng.uniform(-8.0, hi, size=300)
        res = 10.0 ** rng.uniform(-14, 0, size=300)
        tol = 10.0 ** rng.uniform(-12, -6)
        nmax = int(rng.integers(1, 60))
        got = ChebFI.adaptive_degrees(lam, res, lo, hi, tol, nmax)
        want = ch.adaptive_degrees(lam, res, lo, hi, tol, nmax)
        assert np.array_equal(got, want)
