"""GB300 (sm_103a) Chebyshev-filtered subspace iteration for H psi = lambda S psi.

The compute path is libchebfi.so (CUDA kernels behind a C ABI, include/chebfi.h); this
package only builds it and marshals torch tensors to it.
"""
from ._lib import (BOUND_PAPER, BOUND_RIGOROUS, F32, F64, MIXED)  # noqa: F401

__all__ = ["ChebFI", "ChebFIError", "F64", "F32", "MIXED", "BOUND_PAPER", "BOUND_RIGOROUS"]


def __getattr__(name):
    if name in ("ChebFI", "ChebFIError", "fortran"):
        from . import chebfi as _c
        return getattr(_c, name)
    raise AttributeError(name)
