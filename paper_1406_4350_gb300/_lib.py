"""ctypes declarations of libchebfi's C ABI (include/chebfi.h).  Argument marshalling only."""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libchebfi.so")

c_int, c_int64, c_double, c_void_p, c_char_p = (ctypes.c_int, ctypes.c_int64, ctypes.c_double,
                                                 ctypes.c_void_p, ctypes.c_char_p)
P_int32 = ctypes.POINTER(ctypes.c_int32)
P_double = ctypes.POINTER(ctypes.c_double)
P_int = ctypes.POINTER(ctypes.c_int)

# error codes (chebfi.h)
OK, ERR_ARG, ERR_STATE, ERR_CUDA, ERR_NOT_SPD, ERR_NO_CONVERGENCE, ERR_FILTER_OVERFLOW, ERR_NOMEM, ERR_NONFINITE = \
    0, -1, -2, -3, -4, -5, -6, -7, -8
F64, F32, MIXED = 0, 1, 2
GEMM_AUTO, GEMM_CUDA_CORES, GEMM_TENSOR = 0, 1, 2
EIG_AUTO, EIG_JACOBI, EIG_REFINED = 0, 1, 2
FFT64_NATIVE, FFT64_DOUBLE_FLOAT = 0, 1
BOUND_PAPER, BOUND_RIGOROUS = 0, 1


class Params(ctypes.Structure):
    _fields_ = [("degree", c_int), ("sweeps", c_int), ("prec", c_int), ("bound_mode", c_int),
                ("lambda_hi", c_double), ("tol", c_double), ("lock", c_int)]


SIGNATURES = {
    "chebfi_create": (c_int, [ctypes.POINTER(c_void_p), c_int]),
    "chebfi_destroy": (c_int, [c_void_p]),
    "chebfi_last_error": (c_char_p, [c_void_p]),
    "chebfi_set_cell": (c_int, [c_void_p, P_double, P_int, P_double]),
    "chebfi_set_sphere": (c_int, [c_void_p, c_int64, P_int32]),
    "chebfi_set_vloc": (c_int, [c_void_p, c_void_p, c_int]),
    "chebfi_set_projectors": (c_int, [c_void_p, c_int64, c_void_p, c_int64, c_int, c_int, P_int32,
                                      P_double, P_double]),
    "chebfi_upper_bound": (c_int, [c_void_p, c_int, P_double]),
    "chebfi_overlap_lower_bound": (c_int, [c_void_p, P_double]),
    "chebfi_apply_H": (c_int, [c_void_p, c_void_p, c_void_p, c_int64, c_int64, c_int, c_void_p]),
    "chebfi_apply_H_noalloc": (c_int, [c_void_p, c_void_p, c_void_p, c_int64, c_int64, c_void_p]),
    "chebfi_set_D": (c_int, [c_void_p, c_void_p, c_int]),
    "chebfi_apply_H_backward": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int64,
                                        c_int64, c_void_p]),
    "chebfi_batch_create": (c_int, [c_void_p, c_void_p, c_int, c_int64]),
    "chebfi_batch_destroy": (c_int, [c_void_p]),
    "chebfi_batch_last_error": (c_char_p, [c_void_p]),
    "chebfi_batch_kernel_launches": (c_int64, [c_void_p]),
    "chebfi_batch_autotune": (c_int, [c_void_p, c_int, c_void_p, c_void_p]),
    "chebfi_batch_set_tiles": (c_int, [c_void_p, c_int, c_void_p, c_int]),
    "chebfi_batch_cheb_filter": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_int, c_void_p]),
    "chebfi_cheb_filter_host": (c_int, [c_void_p, c_void_p, c_int64, c_int64, c_int, c_double, c_double, c_int, c_int,
                                        c_void_p]),
    "chebfi_cheb_filter_adaptive": (c_int, [c_void_p, c_void_p, c_int64, c_int64, c_void_p, c_double, c_double,
                                            c_int, c_void_p]),
    "chebfi_adaptive_degrees": (c_int, [c_void_p, c_void_p, c_int64, c_double, c_double, c_double, c_int, c_void_p]),
    "chebfi_solve_stats": (c_int, [c_void_p, c_void_p, c_void_p]),
    "chebfi_apply_Sinv_refined": (c_int, [c_void_p, c_void_p, c_void_p, c_int64, c_int64, c_double, c_int,
                                          c_void_p, c_void_p]),
    "chebfi_cheb_filter_backward": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int64,
                                            c_int64, c_int, c_double, c_double, c_int, c_int, c_void_p]),
    "chebfi_apply_S": (c_int, [c_void_p, c_void_p, c_void_p, c_int64, c_int64, c_void_p]),
    "chebfi_apply_Sinv": (c_int, [c_void_p, c_void_p, c_void_p, c_int64, c_int64, c_void_p]),
    "chebfi_cheb_filter": (c_int, [c_void_p, c_void_p, c_int64, c_int64, c_int, c_double, c_double,
                                   c_int, c_void_p]),
    "chebfi_cheb_filter_host_proj": (c_int, [c_void_p, c_void_p, c_void_p, c_int64, c_int64, c_int64, c_int,
                                             c_double, c_double, c_int, c_int, c_void_p]),
    "chebfi_cheb_filter_proj": (c_int, [c_void_p, c_void_p, c_void_p, c_int64, c_int64, c_int64, c_int, c_double,
                                        c_double, c_int, c_void_p]),
    "chebfi_orthonormalise": (c_int, [c_void_p, c_void_p, c_int64, c_int64, c_void_p]),
    "chebfi_rayleigh_ritz": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_int64,
                                     c_void_p]),
    "chebfi_rayleigh_ritz_proj": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_int64,
                                          c_int64, c_void_p]),
    "chebfi_rayleigh_quotients": (c_int, [c_void_p, c_void_p, c_void_p, c_int64, c_int64, c_void_p]),
    "chebfi_solve": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_int64,
                             ctypes.POINTER(Params), c_void_p]),
    "chebfi_set_fp64_gemm": (c_int, [c_void_p, c_int, c_int, P_int]),
    "chebfi_gemm_fp64": (c_int, [c_void_p, c_int, c_int, c_int64, c_int64, c_int64, c_double, c_void_p, c_int64,
                                 c_void_p, c_int64, c_double, c_void_p, c_int64, c_void_p]),
    "chebfi_gemm_mixed": (c_int, [c_void_p, c_int, c_int64, c_int64, c_int64, ctypes.c_float, c_void_p, c_int64,
                                  c_void_p, c_int64, ctypes.c_float, c_void_p, c_int64, c_void_p]),
    "chebfi_set_eigensolver": (c_int, [c_void_p, c_int]),
    "chebfi_set_fft64": (c_int, [c_void_p, c_int]),
    "chebfi_eigensolver_steps": (c_int, [c_void_p]),
    "chebfi_selftest_bounded_wait": (c_int, [c_void_p, c_int, c_double, P_int, P_double]),
    "chebfi_probe_fma_rate": (c_int, [c_void_p, c_int, P_double, P_double]),
    "chebfi_sync_status": (c_int, [c_void_p]),
    "chebfi_kernel_launches": (c_int64, [c_void_p]),
    "chebfi_profile_enable": (c_int, [c_void_p, c_int]),
    "chebfi_profile_count": (c_int, [c_void_p]),
    "chebfi_profile_entry": (c_int, [c_void_p, c_int, ctypes.c_char_p, c_int, P_double,
                                     ctypes.POINTER(c_int64), P_double]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load the in-tree library; raises if it has not been built (there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libchebfi.so is not built (%s); run paper_1406_4350_gb300.build.build()" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib
