"""Chebyshev-filtered subspace iteration, Algorithm 2 of the paper, in FP64 (oracle part O2).

Test infrastructure only.  Everything here follows the paper's order and notation:

* ``cheb_T`` -- the scaled Chebyshev recurrence of Section 4.2:
  ``T_0 = 1``, ``T_1(x) = (x - c)/r``, ``T_{n+1}(x) = 2 (x - c)/r T_n(x) - T_{n-1}(x)``,
  ``c = (a + b)/2``, ``r = (b - a)/2``;
* ``filter_plain`` -- the inner loop of Algorithm 2 with ``S^{-1} H`` applied as written
  (``H`` by Algorithm 1, ``S^{-1}`` by the Woodbury formula of Section 5.1);
* ``filter_reuse`` -- the same loop with the projection-reuse identity of Section 5.1,
  ``P^H S^{-1} psi = P^H psi - (P^H P) q``, so ``P^H`` is applied once, before the loop;
* ``bounds`` -- the first three steps of Algorithm 2 (maximum Rayleigh quotient for
  ``lambda_-``; the kinetic upper bound of Section 5.3 for ``lambda_+``, or a rigorous bound);
* ``rayleigh_ritz`` -- the last three steps of Algorithm 2 (subspace matrices
  ``H_Psi = Psi^H H Psi``, ``S_Psi = Psi^H S Psi``, dense generalized eigenproblem
  ``H_Psi X = S_Psi X Lambda``, rotation ``Psi <- Psi X``) after rescaling the columns
  (Section 5.3 mentions the rescaling);
* ``solve`` -- Algorithm 2 repeated for a number of sweeps;
* ``adaptive_degrees`` / ``filter_adaptive`` -- locking with a per-band degree (Section 5.4):
  the degree of band i is the smallest n with ``||r_i|| / |T_n((lambda_i - c)/r)| <= tol``,
  0 (locked) when the residual already meets the tolerance.

Readings of the paper (it leaves these open): degree ``n`` means ``n`` applications of
``S^{-1} H`` (``psi^1`` uses ``1/r``, later steps ``2/r``); the recurrence is unscaled;
the Rayleigh quotients are the generalized ones ``y^H H y / y^H S y``.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from .planewave import PWOperator

__all__ = [
    "cheb_T", "filter_plain", "filter_setup", "filter_reuse", "rayleigh_quotients", "upper_bound", "bounds",
    "rayleigh_ritz", "residuals", "residual_bound", "solve", "adaptive_degrees", "filter_adaptive",
    "solve_locked",
]


def cheb_T(n: int, x, a: float, b: float):
    """T_n((x - c)/r) on the interval [a, b] by the recurrence of Section 4.2."""
    c = 0.5 * (a + b)
    r = 0.5 * (b - a)
    x = np.asarray(x, dtype=np.float64)
    t_prev = np.ones_like(x)
    if n == 0:
        return t_prev
    t = (x - c) / r
    for _ in range(1, n):
        t, t_prev = 2.0 * (x - c) / r * t - t_prev, t
    return t


def filter_plain(op: PWOperator, Y, degree: int, lam_lo: float, lam_hi: float):
    """Inner loop of Algorithm 2: psi^1 = (S^{-1}H psi^0 - c psi^0)/r,
    psi^i = 2/r (S^{-1}H psi^{i-1} - c psi^{i-1}) - psi^{i-2}; returns psi^degree."""
    c = 0.5 * (lam_hi + lam_lo)
    r = 0.5 * (lam_hi - lam_lo)
    psi_prev = np.array(Y, dtype=np.complex128)
    if degree == 0:
        return psi_prev
    psi = (op.apply_Sinv(op.apply_H(psi_prev)) - c * psi_prev) / r
    for _ in range(2, degree + 1):
        psi, psi_prev = 2.0 / r * (op.apply_Sinv(op.apply_H(psi)) - c * psi) - psi_prev, psi
    return psi


def _woodbury_reduced(op: PWOperator):
    """(D_S^{-1} + P^H P): the reduced N_projs x N_projs matrix of Section 5.1."""
    sizes = np.diff(op.offsets)
    Dinv = np.zeros_like(op.Ds)
    o = 0
    for s in sizes:
        Dinv[o:o + s, o:o + s] = np.linalg.inv(op.Ds[o:o + s, o:o + s])
        o += s
    return Dinv + op.P.conj().T @ op.P


def filter_setup(op: PWOperator):
    """The quantities of Section 5.1 that depend only on P and D_S, formed once:
    G = P^H P and the LU factors of the reduced matrix D_S^{-1} + P^H P (None for S = I)."""
    G = op.P.conj().T @ op.P
    lu = None if op.Ds is None else scipy.linalg.lu_factor(_woodbury_reduced(op))
    return {"G": G, "lu": lu}


def filter_reuse(op: PWOperator, Y, degree: int, lam_lo: float, lam_hi: float,
                 return_proj: bool = False, setup=None):
    """Algorithm 2's inner loop with the projection-reuse identity of Section 5.1.

    For one step with current iterate psi and its carried projections p = P^H psi:
      Z      = K psi + V_loc psi                      (local part of Algorithm 1)
      P^H H psi = P^H Z + G D_V p                     (G = P^H P, precomputed)
      q      = (D_S^{-1} + G)^{-1} P^H H psi          (Woodbury reduced solve)
      S^{-1} H psi = Z + P D_V p - P q
      P^H S^{-1} H psi = P^H H psi - G q              (the identity of Section 5.1)
    and both psi and p follow the Chebyshev recurrence.  ``setup`` (from filter_setup) holds
    G and the reduced matrix's LU factors when they are formed once for many calls.
    """
    c = 0.5 * (lam_hi + lam_lo)
    r = 0.5 * (lam_hi - lam_lo)
    psi_prev = np.array(Y, dtype=np.complex128)
    p_prev = op.projections(psi_prev)
    if degree == 0:
        return (psi_prev, p_prev) if return_proj else psi_prev
    if setup is None:
        setup = filter_setup(op)
    G, lu = setup["G"], setup["lu"]

    def sinv_h(psi, p):
        Z = op.K[:, None] * psi + op.apply_local(psi)
        Dp = op.Dv @ p
        pHpsi = op.P.conj().T @ Z + G @ Dp
        if lu is None:
            q = np.zeros_like(pHpsi)
        else:
            q = scipy.linalg.lu_solve(lu, pHpsi)
        u = Z + op.P @ (Dp - q)
        pu = pHpsi - G @ q
        return u, pu

    u, pu = sinv_h(psi_prev, p_prev)
    psi = (u - c * psi_prev) / r
    p = (pu - c * p_prev) / r
    for _ in range(2, degree + 1):
        u, pu = sinv_h(psi, p)
        psi, psi_prev = 2.0 / r * (u - c * psi) - psi_prev, psi
        p, p_prev = 2.0 / r * (pu - c * p) - p_prev, p
    return (psi, p) if return_proj else psi


def rayleigh_quotients(op: PWOperator, Y):
    """Generalized Rayleigh quotients y^H H y / y^H S y of every column."""
    Y = np.asarray(Y)
    num = np.einsum("gn,gn->n", Y.conj(), op.apply_H(Y)).real
    den = np.einsum("gn,gn->n", Y.conj(), op.apply_S(Y)).real
    return num / den


def upper_bound(op: PWOperator, mode: str = "paper") -> float:
    """Upper end lambda_+ of the filtered interval.

    ``paper``: the kinetic bound of Section 5.3 (E_cut, here the largest |k+G|^2/2 of the
    sphere; the paper notes it is not a proven bound).
    ``rigorous``: max(0, max K + max V + max(0, l_max(L^H D_V L))) / (1 + min(0, l_min(L^H D_S L)))
    with P^H P = L L^H.  The nonzero eigenvalues of P X P^H are those of L^H X L, which
    bounds the nonlocal term and the smallest eigenvalue of S.
    """
    kmax = float(op.K.max())
    if mode == "paper":
        return kmax
    if mode != "rigorous":
        raise ValueError(mode)
    G = op.P.conj().T @ op.P
    L = np.linalg.cholesky(G)
    lv = np.linalg.eigvalsh(L.conj().T @ op.Dv @ L).max()
    num = kmax + float(op.vloc.max()) + max(0.0, lv)
    smin = 1.0
    if op.Ds is not None:
        smin = 1.0 + min(0.0, np.linalg.eigvalsh(L.conj().T @ op.Ds @ L).min())
    return max(0.0, num) / smin


def bounds(op: PWOperator, Y, mode: str = "paper", lam_hi=None):
    """First three steps of Algorithm 2: (lambda_-, lambda_+, c, r)."""
    lam_lo = float(rayleigh_quotients(op, Y).max())
    if lam_hi is None:
        lam_hi = upper_bound(op, mode)
    return lam_lo, lam_hi, 0.5 * (lam_hi + lam_lo), 0.5 * (lam_hi - lam_lo)


def rayleigh_ritz(op: PWOperator, Y):
    """Last three steps of Algorithm 2.

    Columns are first scaled to unit S-norm; then H_Psi = Psi^H H Psi,
    S_Psi = Psi^H S Psi, the dense generalized problem H_Psi X = S_Psi X Lambda is solved
    (LAPACK through scipy; X is S_Psi-orthonormal) and Psi <- Psi X.
    Returns (Lambda ascending, rotated Psi).
    """
    Y = np.array(Y, dtype=np.complex128)
    SY = op.apply_S(Y)
    nrm = np.sqrt(np.einsum("gn,gn->n", Y.conj(), SY).real)
    Y = Y / nrm[None, :]
    HY = op.apply_H(Y)
    SY = SY / nrm[None, :]
    Hs = Y.conj().T @ HY
    Ss = Y.conj().T @ SY
    Hs = 0.5 * (Hs + Hs.conj().T)
    Ss = 0.5 * (Ss + Ss.conj().T)
    w, X = scipy.linalg.eigh(Hs, Ss)
    return w, Y @ X


def residuals(op: PWOperator, Y, w):
    """Residual 2-norms ||H y_n - w_n S y_n|| of every column."""
    R = op.apply_H(Y) - op.apply_S(Y) * np.asarray(w)[None, :]
    return np.linalg.norm(R, axis=0)


def residual_bound(op: PWOperator, Y, w):
    """||r_n||_{S^{-1}} = sqrt(r^H S^{-1} r) for S-normalised y_n: some eigenvalue of the
    pencil lies within this distance of w_n."""
    R = op.apply_H(Y) - op.apply_S(Y) * np.asarray(w)[None, :]
    return np.sqrt(np.maximum(np.einsum("gn,gn->n", R.conj(), op.apply_Sinv(R)).real, 0.0))


def solve(op: PWOperator, Y0, degree: int, sweeps: int, mode: str = "paper", lam_hi=None,
          reuse: bool = True, history: bool = False):
    """Algorithm 2 repeated ``sweeps`` times from Y0.

    Returns dict(w=Ritz values, Y=Ritz vectors, resid=residual norms, lam=(lambda_-, lambda_+)
    per sweep, hist=Ritz values per sweep if requested).
    """
    Y = np.array(Y0, dtype=np.complex128)
    if lam_hi is None:
        lam_hi = upper_bound(op, mode)
    hist = []
    lams = []
    w = None
    for _ in range(sweeps):
        lam_lo = float(rayleigh_quotients(op, Y).max())
        lams.append((lam_lo, lam_hi))
        f = filter_reuse if reuse else filter_plain
        Y = f(op, Y, degree, lam_lo, lam_hi)
        w, Y = rayleigh_ritz(op, Y)
        if history:
            hist.append(w.copy())
    out = dict(w=w, Y=Y, resid=residuals(op, Y, w), lam=lams)
    if history:
        out["hist"] = hist
    return out


def adaptive_degrees(ritz, resid, lam_lo: float, lam_hi: float, tol: float, max_degree: int):
    """Per-band polynomial degrees for locking (Section 5.4).

    One Chebyshev iteration of degree n scales the eigencomponent of eigenvalue lambda_i by
    T_n((lambda_i - c)/r) while unwanted components grow by at most 1, so the residual of
    band i after filter + Rayleigh-Ritz is estimated by ||r_i|| / |T_n((lambda_i - c)/r)|
    (the paper prints lambda_1 in the argument; the per-band reading lambda_i is the one that
    gives each band its own degree).  Band i gets the smallest n in 1..max_degree meeting
    tol, max_degree if none does, and 0 (locked, not filtered) if ||r_i|| <= tol already.
    T_n is evaluated by the recurrence of Section 4.2 (``cheb_T``).
    """
    out = np.zeros(len(ritz), dtype=np.int64)
    for i, (lam, res) in enumerate(zip(ritz, resid)):
        if res <= tol:
            continue
        n_i = max_degree
        for n in range(1, max_degree + 1):
            if res <= tol * abs(float(cheb_T(n, lam, lam_lo, lam_hi))):
                n_i = n
                break
        out[i] = n_i
    return out


def filter_adaptive(op: PWOperator, Y, degrees, lam_lo: float, lam_hi: float):
    """Algorithm 2's inner loop with band i filtered to its own degree degrees[i]."""
    Y = np.array(Y, dtype=np.complex128)
    out = Y.copy()
    for n in sorted(set(int(d) for d in degrees)):
        cols = [i for i, d in enumerate(degrees) if int(d) == n]
        out[:, cols] = filter_plain(op, Y[:, cols], n, lam_lo, lam_hi)
    return out


def solve_locked(op: PWOperator, Y, max_degree: int, sweeps: int, tol: float, mode: str = "paper",
                 lam_hi=None):
    """Algorithm 2 with locking (Section 5.4): after the first full-degree sweep, every sweep
    filters band i to the degree ``adaptive_degrees`` predicts from its Ritz value and
    residual (the filter interval being that sweep's [lambda_-, lambda_+]).  Returns
    (Y, eigenvalues, residuals, the degrees used in each sweep)."""
    _, lam_hi, _, _ = bounds(op, Y, mode, lam_hi)
    Psi = np.array(Y, dtype=np.complex128)
    lam_lo = float(rayleigh_quotients(op, Psi).max())
    degrees = np.full(Psi.shape[1], max_degree, dtype=np.int64)
    used = []
    w = res = None
    for _ in range(sweeps):
        Psi = filter_adaptive(op, Psi, degrees, lam_lo, lam_hi)
        used.append(degrees.copy())
        w, Psi = rayleigh_ritz(op, Psi)
        res = residuals(op, Psi, w)
        lam_lo = float(w.max())
        degrees = adaptive_degrees(w, res, lam_lo, lam_hi, tol, max_degree)
    return Psi, w, res, used
