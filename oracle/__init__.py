"""FP64 CPU oracle for the Chebyshev-filtered subspace iteration (test infrastructure).

This package is the reference the CUDA path is checked against.  It is test
infrastructure only: the tests, the smoke check and the benchmark's timed CPU
baseline may import it; the product library never does, and nothing here imports
the product package.  It is plain numpy/scipy in float64/complex128, slow and
written to be checked against the paper by eye:

* ``planewave``  -- the operators of Section 2.1: kinetic diagonal, local potential
  through an inverse/forward FFT pair, nonlocal ``P D_V P^H``, overlap
  ``S = I + P D_S P^H`` (Algorithm 1), the Woodbury inverse of Section 5.1, and the
  explicit dense ``H`` and ``S`` for tiny cells (oracle part O1).
* ``jacobi``     -- a self-written cyclic Jacobi eigensolver for complex Hermitian
  matrices (used by O1).
* ``exact``      -- exact eigenpairs of the pencil (H, S) of a tiny cell: dense H and S,
  Cholesky reduction, Jacobi (oracle part O1).
* ``chebyshev``  -- the Chebyshev polynomials of Section 4.2, Algorithm 2 step by step
  (bounds, filter with the projection-reuse identity of Section 5.1, subspace matrices,
  dense generalized eigenproblem, rotation) and the residuals (oracle part O2).
"""
from . import planewave, jacobi, chebyshev, exact  # noqa: F401
