"""Pins of the oracle's derivatives (oracle.gradients) to facts outside the oracle: central
differences of the oracle's own forward maps (the H application of Algorithm 1 and the
filter of Algorithm 2), and the closed form for an exact eigenvector, where the filter acts
as the scalar T_n((lambda - c)/r) and the derivative of T_n is n U_{n-1} (numpy's Chebyshev
routines); the last test plants mistakes in the derivative code and checks that a pin
catches each one."""
import dataclasses

import numpy as np
import pytest

from oracle import chebyshev as ch
from oracle import gradients as gr
from oracle.exact import exact_eigs
from oracle.planewave import PWOperator
from synth import make_cell


def _cell(nb=3, paw=True, seed=41):
    return make_cell(6.0, 12, 3.0, 2, 8, nb, paw, seed)


def _rand(rng, shape):
    return rng.normal(size=shape) + 1j * rng.normal(size=shape)


def _op(cell, vloc=None, D=None):
    c = dataclasses.replace(cell, vloc=cell.vloc if vloc is None else vloc, D=cell.D if D is None else D)
    return PWOperator.from_cell(c)


def _sym_dir(cell, rng):
    """A random direction in the packed D coordinates (each entry independent)."""
    return rng.normal(size=cell.D.shape)


# ----------------------------------------------------------------------------- pins
def _pin_h_gradients_by_differences():
    """L = Re <W, H Y> is linear in V, D and Y: central differences are exact up to rounding."""
    cell = _cell()
    rng = np.random.default_rng(1)
    W = _rand(rng, cell.Y0.shape)
    gY, gV, gD = gr.h_gradients(PWOperator.from_cell(cell), cell.Y0, W)
    loss = lambda **kw: float(np.sum(np.conj(W) * _op(cell, **{k: v for k, v in kw.items() if k != "Y"})
                                     .apply_H(kw.get("Y", cell.Y0))).real)
    h = 1e-3
    dV = rng.normal(size=cell.vloc.shape)
    fd = (loss(vloc=cell.vloc + h * dV) - loss(vloc=cell.vloc - h * dV)) / (2 * h)
    assert abs(np.sum(gV * dV) - fd) <= 1e-10 * max(1.0, abs(fd))
    dD = _sym_dir(cell, rng)
    fd = (loss(D=cell.D + h * dD) - loss(D=cell.D - h * dD)) / (2 * h)
    assert abs(np.sum(gD * dD) - fd) <= 1e-10 * max(1.0, abs(fd))
    E = _rand(rng, cell.Y0.shape)
    fd = (loss(Y=cell.Y0 + h * E) - loss(Y=cell.Y0 - h * E)) / (2 * h)
    assert abs(np.sum(np.conj(gY) * E).real - fd) <= 1e-10 * max(1.0, abs(fd))


def _fd4(f, h):
    """Fourth-order central difference of a scalar function at t = 0."""
    return (8 * (f(h) - f(-h)) - (f(2 * h) - f(-2 * h))) / (12 * h)


def _pin_filter_backward_by_differences(paw=True):
    """The filter output is a polynomial of degree n in V and D and linear in Y_0."""
    cell = _cell(paw=paw)
    rng = np.random.default_rng(2)
    deg, lo, hi = 5, -0.5, 9.0
    W = _rand(rng, cell.Y0.shape)
    op = PWOperator.from_cell(cell)
    gY, gV, gD = gr.filter_backward(op, cell.Y0, W, deg, lo, hi)

    def loss(vloc=None, D=None, Y=None):
        out = ch.filter_plain(_op(cell, vloc, D), cell.Y0 if Y is None else Y, deg, lo, hi)
        return float(np.sum(np.conj(W) * out).real)

    dV = rng.normal(size=cell.vloc.shape)
    fd = _fd4(lambda t: loss(vloc=cell.vloc + t * dV), 1e-3)
    assert abs(np.sum(gV * dV) - fd) <= 1e-8 * abs(fd), (np.sum(gV * dV), fd)
    dD = _sym_dir(cell, rng)
    fd = _fd4(lambda t: loss(D=cell.D + t * dD), 1e-3)
    assert abs(np.sum(gD * dD) - fd) <= 1e-8 * abs(fd), (np.sum(gD * dD), fd)
    E = _rand(rng, cell.Y0.shape)
    fd = (loss(Y=cell.Y0 + 1e-3 * E) - loss(Y=cell.Y0 - 1e-3 * E)) / 2e-3
    assert abs(np.sum(np.conj(gY) * E).real - fd) <= 1e-10 * abs(fd)


def _pin_filter_backward_nc():
    _pin_filter_backward_by_differences(paw=False)


def _pin_filter_backward_eigenvector():
    """Y_0 = psi (an S-normalised eigenvector, eigenvalue lambda) and L = Re <S psi, Y_n>:
    the filter gives Y_n = p(lambda) psi with p(x) = T_n((x - c)/r), so L = p(lambda), and
    gY_0 = p(lambda) S psi, gV(r) = p'(lambda) |psi(r)|^2 / N^3 (Hellmann-Feynman),
    gD_ij = p'(lambda) Re conj((P^H psi)_i) (P^H psi)_j, with p'(x) = n U_{n-1}((x - c)/r) / r."""
    cell = _cell(nb=1, seed=7)
    op = PWOperator.from_cell(cell)
    w, Psi = exact_eigs(op, vectors=True)
    n_ev = 2
    psi = Psi[:, n_ev:n_ev + 1]
    lam = w[n_ev]
    deg, lo, hi = 6, w[5], 12.0
    c, r = 0.5 * (hi + lo), 0.5 * (hi - lo)
    x = (lam - c) / r
    Tn = np.polynomial.chebyshev.Chebyshev.basis(deg)
    p, dp = Tn(x), Tn.deriv()(x) / r
    Spsi = op.apply_S(psi)
    gY, gV, gD = gr.filter_backward(op, psi, Spsi, deg, lo, hi)
    scale = max(1.0, abs(p))
    assert np.abs(gY - p * Spsi).max() <= 1e-10 * scale
    grid = np.zeros(op.grid, dtype=np.complex128)
    grid[tuple(op.miller[:, i] % op.grid[i] for i in range(3))] = psi[:, 0]
    dens = np.abs(np.fft.ifftn(grid) * op.vloc.size) ** 2 / op.vloc.size  # |psi(r)|^2 / N^3
    assert np.abs(gV - dp * dens).max() <= 1e-10 * abs(dp) * dens.max()
    pp = op.projections(psi)[:, 0]
    full = (np.conj(pp)[:, None] * pp[None, :]).real
    o = 0
    parts = []
    for s in np.diff(op.offsets):
        parts.append(full[o:o + s, o:o + s].reshape(-1))
        o += s
    assert np.abs(gD - dp * np.concatenate(parts)).max() <= 1e-10 * abs(dp) * np.abs(full).max()


PINS = {
    "h_differences": _pin_h_gradients_by_differences,
    "filter_differences": _pin_filter_backward_by_differences,
    "filter_differences_nc": _pin_filter_backward_nc,
    "filter_eigenvector": _pin_filter_backward_eigenvector,
}


@pytest.mark.parametrize("name", sorted(PINS))
def test_gradient_pin(name):
    PINS[name]()


# ----------------------------------------------------------------------------- planted mistakes
def _reflected_real_space(orig):
    """Grid values at -r instead of r (the sign of the transform's exponent flipped)."""
    def f(op, Y):
        out = orig(op, Y)
        for ax, n in enumerate(op.grid):
            out = np.take(out, (-np.arange(n)) % n, axis=ax + 1)
        return out
    return f


def _transposed_D(orig):
    return lambda op, q, p: orig(op, p, q)


MUTATIONS = [
    ("real_space", _reflected_real_space, ["h_differences", "filter_eigenvector"]),
    ("_packed_D_grad", _transposed_D, ["h_differences"]),
]


@pytest.mark.parametrize("attr, mutate, pins", MUTATIONS)
def test_gradient_pins_catch_planted_mistakes(monkeypatch, attr, mutate, pins):
    monkeypatch.setattr(gr, attr, mutate(getattr(gr, attr)))
    for name in pins:
        with pytest.raises(AssertionError):
            PINS[name]()


def test_dropped_sinv_in_adjoint_is_caught(monkeypatch):
    """The adjoint uses S^{-1} explicitly; replacing it by the identity inside the derivative
    code only (the forward map keeps the true S^{-1}) must fail the difference pin."""
    orig_fb = gr.filter_backward

    def broken(op, Y0, Gn, degree, lo, hi):
        class NoSinv:
            def __init__(self, base):
                self._b = base

            def __getattr__(self, k):
                return getattr(self._b, k)

            def apply_Sinv(self, X):
                return np.asarray(X).reshape(self._b.npw, -1).copy()

        return orig_fb(NoSinv(op), Y0, Gn, degree, lo, hi)

    monkeypatch.setattr(gr, "filter_backward", broken)
    with pytest.raises(AssertionError):
        _pin_filter_backward_by_differences(paw=True)
