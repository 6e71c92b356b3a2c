"""Self-written cyclic Jacobi eigensolver for complex Hermitian matrices (oracle part O1).

Test infrastructure only.  Used to diagonalise the explicitly assembled
``C = L^{-1} H L^{-H}`` of tiny cells, giving exact eigenpairs of the pencil (H, S)
(paper Section 2.1, Eq. (KS)) independently of LAPACK.

Method (Jacobi 1846; the 2x2 step is the symmetric Schur decomposition of Golub & Van
Loan, "Matrix Computations", Section 8.5): each rotation removes one off-diagonal
entry ``A[p, q] = |h| e^{i phi}``.  A phase ``diag(1, e^{-i phi})`` makes the 2x2
block real, then the real rotation ``[[c, s], [-s, c]]`` with
``zeta = (A_qq - A_pp) / (2|h|)``, ``t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2))``,
``c = 1/sqrt(1 + t^2)``, ``s = t c`` diagonalises it.  The pairs of one step come
from a round-robin tournament, so they are disjoint and are applied together; one
sweep is ``n - 1`` steps and visits every pair once.

The matrix is kept in the tournament's current seating order (first half of the
rows pairs with the second half), so one step is a handful of whole-array plain
PyTorch CPU operations; between steps the seating is permuted.
"""
from __future__ import annotations

import numpy as np
import torch

__all__ = ["jacobi_eigh", "round_robin_pairs"]


def round_robin_pairs(n: int):
    """Yield n-1 rounds of n/2 disjoint pairs covering all pairs of range(n) (n even)."""
    assert n % 2 == 0
    players = list(range(n))
    for _ in range(n - 1):
        half = n // 2
        yield np.array(players[:half]), np.array(players[half:][::-1])
        players = [players[0], players[-1]] + players[1:-1]


def _seating(players):
    h = len(players) // 2
    return players[:h] + players[h:][::-1]


def jacobi_eigh(A, tol: float = 1e-15, max_sweeps: int = 40, vectors: bool = True):
    """Eigenvalues (ascending) and eigenvectors of a complex Hermitian matrix.

    Returns ``(w, V)`` as numpy arrays with ``A V = V diag(w)``; ``V`` is None when
    ``vectors`` is False.  Stops when the off-diagonal Frobenius norm is below
    ``tol * ||A||_F`` or when a whole sweep finds every off-diagonal entry negligible
    against its diagonal pair (``|A_pq| <= eps sqrt(|A_pp A_qq|)``).
    """
    A0 = np.asarray(A)
    n0 = A0.shape[0]
    if n0 == 0:
        return np.zeros(0), (np.zeros((0, 0), np.complex128) if vectors else None)
    n = n0 + (n0 % 2)
    M = torch.zeros((n, n), dtype=torch.complex128)
    # for odd n an isolated zero row/column (never coupled) makes n even
    M[:n0, :n0] = torch.from_numpy(np.ascontiguousarray(A0, dtype=np.complex128))
    h = n // 2
    V = torch.eye(n, dtype=torch.complex128) if vectors else None
    scale = float(torch.linalg.norm(M)) or 1.0
    eps = float(np.finfo(np.float64).eps)
    players = list(range(n))
    seat = _seating(players)           # seat[i] = logical index stored at physical i
    perm_phys = torch.tensor(seat)
    M = M[perm_phys][:, perm_phys]
    if vectors:
        V = V[:, perm_phys]
    # moving from one round's seating to the next is the same permutation of physical
    # positions every round: list position j of the next round holds list position
    # rot(j) of this one, and physical seat i shows list position pos(i).
    pos = list(range(h)) + list(range(n - 1, h - 1, -1))
    pos_inv = {p: i for i, p in enumerate(pos)}
    rot = [0, n - 1] + list(range(1, n - 1))
    step_perm = torch.tensor([pos_inv[rot[pos[i]]] for i in range(n)])
    converged = False
    for _sweep in range(max_sweeps):
        off = float(torch.linalg.norm(M - torch.diag(torch.diagonal(M))))
        if off <= tol * scale:
            converged = True
            break
        rotated = 0
        for _step in range(n - 1):
            a = torch.diagonal(M)[:h].real
            b = torch.diagonal(M)[h:].real
            hq = torch.diagonal(M[:h, h:])
            g = hq.abs()
            active = (g > 1e-300) & (g > eps * torch.sqrt((a * b).abs()))
            na = int(active.sum())
            if na:
                rotated += na
                gs = torch.where(active, g, torch.ones_like(g))
                zeta = (b - a) / (2.0 * gs)
                sgn = torch.where(zeta >= 0.0, 1.0, -1.0).to(torch.float64)
                t = sgn / (zeta.abs() + torch.hypot(torch.ones_like(zeta), zeta))
                t = torch.where(active, t, torch.zeros_like(t))
                c = 1.0 / torch.sqrt(1.0 + t * t)
                s = t * c
                ph = torch.where(active, hq / gs, torch.ones_like(hq))
                u00 = c.to(torch.complex128)
                u01 = s.to(torch.complex128)
                u10 = -s * ph.conj()
                u11 = c * ph.conj()
                # rows: M <- U^H M
                top = M[:h].clone()
                bot = M[h:]
                M[:h] = u00.conj()[:, None] * top + u10.conj()[:, None] * bot
                M[h:] = u01.conj()[:, None] * top + u11.conj()[:, None] * bot
                # columns: M <- M U
                left = M[:, :h].clone()
                right = M[:, h:]
                M[:, :h] = left * u00[None, :] + right * u10[None, :]
                M[:, h:] = left * u01[None, :] + right * u11[None, :]
                if vectors:
                    left = V[:, :h].clone()
                    right = V[:, h:]
                    V[:, :h] = left * u00[None, :] + right * u10[None, :]
                    V[:, h:] = left * u01[None, :] + right * u11[None, :]
            # next round of the tournament: move to its seating
            players = [players[0], players[-1]] + players[1:-1]
            M = M[step_perm][:, step_perm]
            if vectors:
                V = V[:, step_perm]
        seat = _seating(players)
        if rotated == 0:
            converged = True
            break
    if not converged:
        raise RuntimeError("Jacobi did not converge in %d sweeps" % max_sweeps)
    seat_t = torch.tensor(seat)
    w = torch.empty(n, dtype=torch.float64)
    w[seat_t] = torch.diagonal(M).real
    w = w.numpy()[:n0]
    order = np.argsort(w, kind="stable")
    if vectors:
        Vl = torch.empty_like(V)
        Vl[:, seat_t] = V
        Vn = Vl.numpy()[:n0, :n0][:, order]
        return w[order], Vn
    return w[order], None
