"""Exact eigenpairs of the pencil (H, S) for tiny cells (oracle part O1).

Test infrastructure only.  ``H`` and ``S`` are assembled explicitly (``planewave.dense_H``,
``planewave.dense_S``) and the generalized problem ``H psi = lambda S psi`` of the paper's
Eq. (KS) is reduced to a standard one with the Cholesky factor ``S = L L^H``:
``C = L^{-1} H L^{-H}``, ``C z = lambda z``, ``psi = L^{-H} z``.  ``C`` is diagonalised by
the self-written Jacobi method; the Cholesky factor and the triangular solves are
library primitives.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from .jacobi import jacobi_eigh
from .planewave import PWOperator, dense_H, dense_S

__all__ = ["exact_eigs"]


def exact_eigs(op: PWOperator, vectors: bool = False):
    """All eigenvalues (ascending) of the pencil (H, S), and S-orthonormal eigenvectors."""
    H = dense_H(op)
    S = dense_S(op)
    L = np.linalg.cholesky(S)
    X = scipy.linalg.solve_triangular(L, H, lower=True)
    C = scipy.linalg.solve_triangular(L, X.conj().T, lower=True).conj().T
    C = 0.5 * (C + C.conj().T)
    w, Z = jacobi_eigh(C, vectors=vectors)
    if not vectors:
        return w
    Psi = scipy.linalg.solve_triangular(L.conj().T, Z, lower=False)
    return w, Psi
