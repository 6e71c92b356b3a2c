"""Plane-wave operators of the Kohn-Sham eigenproblem (paper Section 2.1), in FP64.

Test infrastructure: only the tests, the smoke check and the benchmark's CPU-baseline
leg use this module.

Conventions (the paper leaves them open; the reading used everywhere in this project):

* complex wavefunctions throughout, so the paper's ``P^T`` becomes ``P^H`` and
  ``Psi^T`` becomes ``Psi^H`` (Section 2.1 notes that the periodic, k-sampled case needs
  complex eigenproblems);
* a plane wave ``G(m) = m1 b1 + m2 b2 + m3 b3`` with ``a_i . b_j = 2 pi delta_ij``;
* real-space values ``psi(r_j) = sum_G c_G exp(+2 pi i m . j / N)`` on grid index ``j``
  (unnormalised inverse transform) and the forward transform
  ``c_G = (1/N^3) sum_j f(r_j) exp(-2 pi i m . j / N)``; only their composition enters
  the operator;
* the local operator is therefore the convolution
  ``(V_loc c)_G = sum_G' V~((m - m') mod N) c_G'`` with
  ``V~(n) = (1/N^3) sum_j V(r_j) exp(-2 pi i n . j / N)``.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "reciprocal", "kinetic", "vtilde", "blockdiag", "PWOperator", "dense_H", "dense_S",
]


def reciprocal(lattice: np.ndarray) -> np.ndarray:
    """Rows b1, b2, b3 with a_i . b_j = 2 pi delta_ij (lattice rows are a1, a2, a3)."""
    return 2.0 * np.pi * np.linalg.inv(lattice).T


def kinetic(lattice, kpt, miller) -> np.ndarray:
    """Diagonal of the kinetic operator K: |k + G|^2 / 2 (Section 2.1, "a simple diagonal matrix")."""
    kg = np.asarray(kpt)[None, :] + np.asarray(miller, dtype=np.float64) @ reciprocal(lattice)
    return 0.5 * np.sum(kg * kg, axis=1)


def vtilde(vloc: np.ndarray) -> np.ndarray:
    """Fourier coefficients V~(n) = (1/N^3) sum_j V(r_j) exp(-2 pi i n.j/N), indexed by n mod N."""
    return np.fft.fftn(vloc) / vloc.size


def blockdiag(blocks_flat: np.ndarray, offsets: np.ndarray) -> np.ndarray:
    """Dense block-diagonal matrix from concatenated row-major per-atom blocks (Section 2.1:
    D_V and D_S "do not couple the different atoms")."""
    sizes = np.diff(np.asarray(offsets))
    n = int(sizes.sum())
    out = np.zeros((n, n), dtype=np.asarray(blocks_flat).dtype)
    f = 0
    o = 0
    for s in sizes:
        out[o:o + s, o:o + s] = blocks_flat[f:f + s * s].reshape(s, s)
        f += s * s
        o += s
    return out


class PWOperator:
    """Matrix-free H and S of one cell, following Algorithm 1 (computation of H psi, S psi).

    ``H = K + V_loc + P D_V P^H`` and ``S = I + P D_S P^H`` (Section 2.1); ``D_S = 0``
    (``Q is None``) is the norm-conserving case ``S = I``.
    """

    def __init__(self, lattice, grid, kpt, miller, vloc, P, proj_offsets, D, Q=None):
        self.grid = tuple(int(g) for g in grid)
        self.miller = np.asarray(miller, dtype=np.int64)
        self.K = kinetic(lattice, kpt, self.miller)
        self.vloc = np.asarray(vloc, dtype=np.float64).reshape(self.grid)
        self.P = np.asarray(P, dtype=np.complex128)
        self.Dv = blockdiag(np.asarray(D, dtype=np.float64), proj_offsets)
        self.Ds = None if Q is None else blockdiag(np.asarray(Q, dtype=np.float64), proj_offsets)
        self.offsets = np.asarray(proj_offsets)
        self._idx = tuple((self.miller[:, i] % self.grid[i]) for i in range(3))
        # threads for the 3-D FFTs (None: numpy's single-threaded FFT; an int: scipy.fft with
        # that many workers -- the same transform definition, only the speed differs)
        self.fft_workers = None

    @classmethod
    def from_cell(cls, cell):
        return cls(cell.lattice, cell.grid, cell.kpt, cell.miller, cell.vloc, cell.P,
                   cell.proj_offsets, cell.D, cell.Q)

    @property
    def npw(self):
        return self.miller.shape[0]

    # -- Algorithm 1, step by step ---------------------------------------------------
    def apply_local(self, Y):
        """V_loc Y: inverse FFT to real space, multiply by V_loc(r), forward FFT back."""
        Y = np.asarray(Y).reshape(self.npw, -1)
        nb = Y.shape[1]
        n3 = self.vloc.size
        grid = np.zeros((nb,) + self.grid, dtype=np.complex128)
        grid[(slice(None),) + self._idx] = Y.T
        if self.fft_workers is None:
            psi_r = np.fft.ifftn(grid, axes=(1, 2, 3)) * n3
            psi_r *= self.vloc[None]
            out = np.fft.fftn(psi_r, axes=(1, 2, 3)) / n3
        else:
            import scipy.fft
            psi_r = scipy.fft.ifftn(grid, axes=(1, 2, 3), workers=self.fft_workers) * n3
            psi_r *= self.vloc[None]
            out = scipy.fft.fftn(psi_r, axes=(1, 2, 3), workers=self.fft_workers) / n3
        return out[(slice(None),) + self._idx].T

    def projections(self, Y):
        """p_psi = P^H psi."""
        return self.P.conj().T @ Y

    def apply_H(self, Y, return_proj=False):
        """H psi = K psi + V_loc psi + P D_V p_psi."""
        Y = np.asarray(Y).reshape(self.npw, -1)
        p = self.projections(Y)
        HY = self.K[:, None] * Y + self.apply_local(Y) + self.P @ (self.Dv @ p)
        return (HY, p) if return_proj else HY

    def apply_S(self, Y):
        """S psi = psi + P D_S p_psi."""
        Y = np.asarray(Y).reshape(self.npw, -1)
        if self.Ds is None:
            return Y.copy()
        return Y + self.P @ (self.Ds @ self.projections(Y))

    def apply_Sinv(self, X):
        """S^{-1} x by the Woodbury formula of Section 5.1:
        S^{-1} = I - P (D_S^{-1} + P^H P)^{-1} P^H.

        The reduced system is solved by a dense LU solve (the paper uses iterative
        refinement; both reach the same vector).  D_S^{-1} is formed block by block.
        """
        X = np.asarray(X).reshape(self.npw, -1)
        if self.Ds is None:
            return X.copy()
        Dinv = np.zeros_like(self.Ds)
        sizes = np.diff(self.offsets)
        o = 0
        for s in sizes:
            Dinv[o:o + s, o:o + s] = np.linalg.inv(self.Ds[o:o + s, o:o + s])
            o += s
        reduced = Dinv + self.P.conj().T @ self.P
        q = np.linalg.solve(reduced, self.projections(X))
        return X - self.P @ q

    def apply_Sinv_refined(self, X, tol: float = 1e-12, maxit: int = 200):
        """S^{-1} x with the reduced system of Section 5.1 solved the paper's way: iterative
        refinement q <- q + B^{-1} (b - A q) from q = 0 on A = D_S^{-1} + P^H P, b = P^H x,
        preconditioned by B = the per-atom diagonal blocks of A; it stops when every column
        has ||b - A q|| <= tol ||b||, or after maxit updates.
        Returns (S^{-1} x, number of updates of q)."""
        X = np.asarray(X).reshape(self.npw, -1)
        if self.Ds is None:
            return X.copy(), 0
        sizes = np.diff(self.offsets)
        G = self.P.conj().T @ self.P
        A = np.zeros_like(G)
        Binv = np.zeros_like(G)
        o = 0
        for s in sizes:
            A[o:o + s, o:o + s] = np.linalg.inv(self.Ds[o:o + s, o:o + s])
            o += s
        A = A + G
        o = 0
        for s in sizes:
            Binv[o:o + s, o:o + s] = np.linalg.inv(A[o:o + s, o:o + s])
            o += s
        b = self.projections(X)
        q = np.zeros_like(b)
        bnorm = np.linalg.norm(b, axis=0)
        it = 0
        while True:
            r = b - A @ q
            if np.all(np.linalg.norm(r, axis=0) <= tol * bnorm) or it == maxit:
                break
            q = q + Binv @ r
            it += 1
        return X - self.P @ q, it

    def refinement_diagnostics(self):
        """The convergence figures of the refinement above: (rho, kappa) with rho the spectral
        radius of I - B^{-1} A (the error shrinks by about rho per update; the iteration
        converges when rho < 1) and kappa = |mu|_max / |mu|_min over the eigenvalues mu of
        B^{-1} A (the preconditioned condition number Section 5.1 reports)."""
        if self.Ds is None:
            return 0.0, 1.0
        sizes = np.diff(self.offsets)
        A = self.P.conj().T @ self.P
        o = 0
        for s in sizes:
            A[o:o + s, o:o + s] += np.linalg.inv(self.Ds[o:o + s, o:o + s])
            o += s
        Binv = np.zeros_like(A)
        o = 0
        for s in sizes:
            Binv[o:o + s, o:o + s] = np.linalg.inv(A[o:o + s, o:o + s])
            o += s
        mu = np.linalg.eigvals(Binv @ A)
        return float(np.abs(1.0 - mu).max()), float(np.abs(mu).max() / np.abs(mu).min())

    # -- dense forms (oracle part O1) -------------------------------------------------
    def dense_H(self):
        return dense_H(self)

    def dense_S(self):
        return dense_S(self)


def dense_H(op: PWOperator) -> np.ndarray:
    """Explicit N_pw x N_pw Hamiltonian:
    H_GG' = K_G delta_GG' + V~((m - m') mod N) + sum_ij P_Gi D_ij conj(P_G'j)."""
    vt = vtilde(op.vloc)
    m = op.miller
    diff = m[:, None, :] - m[None, :, :]
    H = vt[diff[..., 0] % op.grid[0], diff[..., 1] % op.grid[1], diff[..., 2] % op.grid[2]]
    H = H + np.diag(op.K)
    H = H + op.P @ op.Dv @ op.P.conj().T
    return H


def dense_S(op: PWOperator) -> np.ndarray:
    """Explicit overlap S_GG' = delta_GG' + sum_ij P_Gi Q_ij conj(P_G'j) (identity if Q is None)."""
    S = np.eye(op.npw, dtype=np.complex128)
    if op.Ds is not None:
        S = S + op.P @ op.Ds @ op.P.conj().T
    return S
