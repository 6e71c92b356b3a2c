"""Derivatives of the H application (Algorithm 1) and of the Chebyshev filter (Algorithm 2's
inner loop) with respect to the wavefunctions, the local potential V_loc(r) and the nonlocal
coefficients D, in FP64.

Test infrastructure: only the tests, the smoke check and the benchmark's CPU-baseline leg use
this module.

Conventions: a real loss L of a complex block Z has the gradient g = dL/dZ in PyTorch's
convention, dL = Re sum conj(g) dZ.  H = K + V_loc + P D P^H with

  (V_loc c)_G = sum_G' V~(G - G') c_G',    V~(m) = (1/N^3) sum_r V(r) exp(-2 pi i m.r/N)

(Section 2.1), so for L = Re <G, H Y> the derivative with respect to the grid value V(r) is
(1/N^3) Re sum_b conj(g_b(r)) y_b(r), with g_b(r), y_b(r) the unnormalised inverse transforms
of the columns; with respect to the packed entry D_ij of an atom block it is
Re sum_b conj((P^H G)_ib) (P^H Y)_jb; with respect to Y it is H G (H is Hermitian).

The filter is Y_{k+1} = a_k (S^{-1} H Y_k - c Y_k) - b_k Y_{k-1} (a_0 = 1/r, a_k = 2/r,
b_0 = 0, b_k = 1).  Its adjoint runs the same recurrence backwards with (S^{-1} H)^H =
H S^{-1}: L_n = g, L_k = a_k (H S^{-1} L_{k+1} - c L_{k+1}) - L_{k+2}, and the V and D
derivatives are the sums over k of the H derivatives of the pairs (Y_k, a_k S^{-1} L_{k+1}).
This is the plain form: every iterate is stored.
"""
from __future__ import annotations

import numpy as np

from .planewave import PWOperator

__all__ = ["real_space", "h_gradients", "filter_backward"]


def real_space(op: PWOperator, Y) -> np.ndarray:
    """Columns of Y on the grid: psi_b(r_j) = sum_G c_Gb exp(+2 pi i m.j/N), shape (nb, N1, N2, N3)."""
    Y = np.asarray(Y, dtype=np.complex128).reshape(op.npw, -1)
    grid = np.zeros((Y.shape[1],) + op.grid, dtype=np.complex128)
    idx = tuple(op.miller[:, i] % op.grid[i] for i in range(3))
    grid[(slice(None),) + idx] = Y.T
    return np.fft.ifftn(grid, axes=(1, 2, 3)) * op.vloc.size


def _packed_D_grad(op: PWOperator, q, p) -> np.ndarray:
    """Packed per-atom row-major blocks of Re sum_b conj(q_ib) p_jb."""
    full = (np.conj(q) @ p.T).real
    out = []
    o = 0
    for s in np.diff(op.offsets):
        out.append(full[o:o + s, o:o + s].reshape(-1))
        o += s
    return np.concatenate(out) if out else np.zeros(0)


def h_gradients(op: PWOperator, Y, G):
    """(gY, gV, gD) of L = Re <G, H Y>: gY = H G, gV on the grid, gD packed like D."""
    Y = np.asarray(Y, dtype=np.complex128).reshape(op.npw, -1)
    G = np.asarray(G, dtype=np.complex128).reshape(op.npw, -1)
    gY = op.apply_H(G)
    yr = real_space(op, Y)
    gr = real_space(op, G)
    gV = (np.conj(gr) * yr).real.sum(axis=0) / op.vloc.size
    gD = _packed_D_grad(op, op.projections(G), op.projections(Y))
    return gY, gV, gD


def filter_backward(op: PWOperator, Y0, Gn, degree: int, lam_lo: float, lam_hi: float):
    """(gY0, gV, gD) of a real loss of the filter output Y_degree given Gn = dL/dY_degree."""
    c = 0.5 * (lam_hi + lam_lo)
    r = 0.5 * (lam_hi - lam_lo)
    Y0 = np.array(Y0, dtype=np.complex128).reshape(op.npw, -1)
    Gn = np.array(Gn, dtype=np.complex128).reshape(op.npw, -1)
    gV = np.zeros(op.grid)
    gD = np.zeros(sum(int(s) * int(s) for s in np.diff(op.offsets)))
    if degree == 0:
        return Gn, gV, gD
    a = [(1.0 if k == 0 else 2.0) / r for k in range(degree)]
    # forward: every iterate kept
    Ys = [Y0]
    for k in range(degree - 1):
        nxt = a[k] * (op.apply_Sinv(op.apply_H(Ys[k])) - c * Ys[k])
        if k > 0:
            nxt = nxt - Ys[k - 1]
        Ys.append(nxt)
    # adjoint
    lam_next, lam_next2 = Gn, None
    for k in range(degree - 1, -1, -1):
        u = op.apply_Sinv(lam_next)
        lam = a[k] * (op.apply_H(u) - c * lam_next)
        if lam_next2 is not None:
            lam = lam - lam_next2
        _, dV, dD = h_gradients(op, Ys[k], a[k] * u)
        gV += dV
        gD += dD
        lam_next, lam_next2 = lam, lam_next
    return lam_next, gV, gD
