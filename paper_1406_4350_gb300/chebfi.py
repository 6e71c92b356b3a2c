"""Python binding of libchebfi: the same operations as the C ABI, on torch CUDA tensors.

Wavefunction blocks are complex128 CUDA tensors of shape (npw, nb) in column-major
(Fortran) layout: ``Y.stride(0) == 1`` and ``Y.stride(1) = ld >= npw``; ``fortran(x)``
converts.  Every computation runs in libchebfi's kernels; this module only passes
pointers, sizes and the current CUDA stream.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import F32, F64, BOUND_PAPER, GEMM_AUTO, GEMM_CUDA_CORES, GEMM_TENSOR, Params

__all__ = ["ChebFI", "ChebFIBatch", "ChebFIError", "fortran"]


class ChebFIError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("chebfi error %d: %s" % (code, msg))
        self.code = code


def fortran(x, device="cuda") -> torch.Tensor:
    """(npw, nb) complex128 CUDA tensor in column-major layout from a numpy array or tensor."""
    t = torch.as_tensor(np.asarray(x) if not isinstance(x, torch.Tensor) else x)
    t = t.to(device=device, dtype=torch.complex128)
    if t.dim() == 1:
        t = t[:, None]
    return t.T.contiguous().T


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _block(Y):
    if not (isinstance(Y, torch.Tensor) and Y.is_cuda and Y.dtype == torch.complex128 and Y.dim() == 2):
        raise TypeError("expected a 2-D complex128 CUDA tensor")
    if Y.shape[1] > 0 and Y.stride(0) != 1:
        raise ValueError("wavefunction block must be column-major (use fortran())")
    ld = Y.stride(1) if Y.shape[1] > 1 else max(Y.shape[0], 1)
    return ctypes.c_void_p(Y.data_ptr() if Y.numel() else 0), int(Y.shape[1]), int(max(ld, Y.shape[0]))


class ChebFI:
    """One plane-wave problem on one GPU (a libchebfi context)."""

    def __init__(self, device: int = 0):
        self.lib = _lib.load()
        self.device = device
        h = ctypes.c_void_p()
        with torch.cuda.device(device):
            rc = self.lib.chebfi_create(ctypes.byref(h), device)
        if rc != 0:
            raise ChebFIError(rc, "chebfi_create failed")
        self.h = h
        self.npw = 0
        self.nproj = 0

    def close(self):
        if getattr(self, "h", None):
            self.lib.chebfi_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != 0:
            raise ChebFIError(rc, self.lib.chebfi_last_error(self.h).decode())

    # -- setup ---------------------------------------------------------------------
    def set_cell(self, lattice, grid, kpt=(0.0, 0.0, 0.0)):
        lat = np.ascontiguousarray(np.asarray(lattice, dtype=np.float64).reshape(9))
        g = np.ascontiguousarray(np.asarray(grid, dtype=np.int32).reshape(3))
        k = np.ascontiguousarray(np.asarray(kpt, dtype=np.float64).reshape(3))
        self._check(self.lib.chebfi_set_cell(self.h, lat.ctypes.data_as(_lib.P_double),
                                             g.ctypes.data_as(_lib.P_int), k.ctypes.data_as(_lib.P_double)))

    def set_sphere(self, miller):
        m = np.ascontiguousarray(np.asarray(miller, dtype=np.int32).reshape(-1, 3))
        self._check(self.lib.chebfi_set_sphere(self.h, m.shape[0], m.ctypes.data_as(_lib.P_int32)))
        self.npw = m.shape[0]

    def set_vloc(self, vloc):
        if isinstance(vloc, torch.Tensor) and vloc.is_cuda:
            v = vloc.to(torch.float64).contiguous()
            self._check(self.lib.chebfi_set_vloc(self.h, ctypes.c_void_p(v.data_ptr()), 1))
            torch.cuda.synchronize()
        else:
            v = np.ascontiguousarray(np.asarray(vloc, dtype=np.float64))
            self._check(self.lib.chebfi_set_vloc(self.h, ctypes.c_void_p(v.ctypes.data), 0))

    def set_projectors(self, P, proj_offsets, D, Q=None):
        offs = np.ascontiguousarray(np.asarray(proj_offsets, dtype=np.int32))
        Dn = np.ascontiguousarray(np.asarray(D, dtype=np.float64))
        Qn = None if Q is None else np.ascontiguousarray(np.asarray(Q, dtype=np.float64))
        natoms = len(offs) - 1
        if isinstance(P, torch.Tensor) and P.is_cuda:
            Pt = P if (P.stride(0) == 1 and P.dtype == torch.complex128) else fortran(P)
            ptr, ld, on_dev = ctypes.c_void_p(Pt.data_ptr()), Pt.stride(1), 1
            nproj = Pt.shape[1]
            keep = Pt
        else:
            Pn = np.asfortranarray(np.asarray(P, dtype=np.complex128))
            nproj = Pn.shape[1]
            ptr, ld, on_dev = ctypes.c_void_p(Pn.ctypes.data), Pn.shape[0], 0
            keep = Pn
        self._check(self.lib.chebfi_set_projectors(
            self.h, nproj, ptr, ld, on_dev, natoms, offs.ctypes.data_as(_lib.P_int32),
            Dn.ctypes.data_as(_lib.P_double),
            None if Qn is None else Qn.ctypes.data_as(_lib.P_double)))
        del keep
        self.nproj = nproj

    def set_D(self, D):
        """Replace the nonlocal coefficient blocks D (packed like set_projectors' D)."""
        if isinstance(D, torch.Tensor) and D.is_cuda:
            d = D.detach().to(torch.float64).contiguous()
            self._check(self.lib.chebfi_set_D(self.h, ctypes.c_void_p(d.data_ptr()), 1))
        else:
            d = np.ascontiguousarray(np.asarray(D, dtype=np.float64))
            self._check(self.lib.chebfi_set_D(self.h, ctypes.c_void_p(d.ctypes.data), 0))

    @classmethod
    def from_cell(cls, cell, device: int = 0):
        """Context set up from a ``synth.Cell``-like object (lattice, grid, kpt, miller, vloc,
        P, proj_offsets, D, Q)."""
        c = cls(device)
        c.set_cell(cell.lattice, cell.grid, cell.kpt)
        c.set_sphere(cell.miller)
        c.set_vloc(cell.vloc)
        c.set_projectors(cell.P, cell.proj_offsets, cell.D, cell.Q)
        return c

    def upper_bound(self, mode: int = BOUND_PAPER) -> float:
        out = ctypes.c_double()
        self._check(self.lib.chebfi_upper_bound(self.h, mode, ctypes.byref(out)))
        return out.value

    def overlap_lower_bound(self) -> float:
        """Proven lower bound of the smallest eigenvalue of S (1 for S = I)."""
        out = ctypes.c_double()
        self._check(self.lib.chebfi_overlap_lower_bound(self.h, ctypes.byref(out)))
        return out.value

    # -- operators -------------------------------------------------------------------
    def _out_like(self, Y):
        return torch.empty((Y.shape[1], Y.shape[0]), dtype=torch.complex128, device=Y.device).T

    def apply_H(self, Y, prec: int = F64, out=None):
        out = self._out_like(Y) if out is None else out
        y, nb, ld = _block(Y)
        o, _, ldo = _block(out)
        if ldo != ld:
            raise ValueError("Y and out must share a leading dimension")
        self._check(self.lib.chebfi_apply_H(self.h, y, o, nb, ld, prec, _stream()))
        return out

    def apply_H_backward(self, Y, G, grid, nD, want_Y=True, want_V=True, want_D=True):
        """Gradients of a real loss through HY = H Y given G = dL/d(HY) (PyTorch convention):
        returns (gY = H G, gV on the grid, gD packed like D); entries not wanted are None."""
        y, nb, ld = _block(Y)
        g, nbg, ldg = _block(G)
        if nbg != nb or ldg != ld:
            raise ValueError("Y and G must have the same shape and leading dimension")
        gY = self._out_like(Y) if want_Y else None
        gV = torch.empty(tuple(int(x) for x in grid), dtype=torch.float64, device=Y.device) if want_V else None
        gD = torch.empty(int(nD), dtype=torch.float64, device=Y.device) if want_D else None
        ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
        if gY is not None:
            _, _, ldo = _block(gY)
            if ldo != ld:
                gY = torch.empty((nb, ld), dtype=torch.complex128, device=Y.device).T[: Y.shape[0]]
        self._check(self.lib.chebfi_apply_H_backward(self.h, y, g, ptr(gY), ptr(gV), ptr(gD), nb, ld, _stream()))
        return gY, gV, gD

    def cheb_filter_backward(self, Y0, gYn, degree: int, lambda_lo: float, lambda_hi: float, grid, nD,
                             prec: int = F64, checkpoint_every: int = 0, want_Y=True, want_V=True, want_D=True):
        """Gradients of a real loss through the filter Y_n = cheb_filter(Y0) given gYn = dL/dY_n
        (PyTorch convention): returns (gY0, gV on the grid, gD packed like D); entries not
        wanted are None.  The iterates are recomputed from checkpoints every
        ``checkpoint_every`` steps (0: ceil(sqrt(degree)))."""
        y, nb, ld = _block(Y0)
        g, nbg, ldg = _block(gYn)
        if nbg != nb or ldg != ld:
            raise ValueError("Y0 and gYn must have the same shape and leading dimension")
        gY = None
        if want_Y:
            gY = self._out_like(Y0)
            if _block(gY)[2] != ld:
                gY = torch.empty((nb, ld), dtype=torch.complex128, device=Y0.device).T[: Y0.shape[0]]
        gV = torch.empty(tuple(int(x) for x in grid), dtype=torch.float64, device=Y0.device) if want_V else None
        gD = torch.empty(int(nD), dtype=torch.float64, device=Y0.device) if want_D else None
        ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
        self._check(self.lib.chebfi_cheb_filter_backward(self.h, y, g, ptr(gY), ptr(gV), ptr(gD), nb, ld, degree,
                                                         lambda_lo, lambda_hi, prec, checkpoint_every, _stream()))
        return gY, gV, gD

    def apply_S(self, Y, out=None):
        out = self._out_like(Y) if out is None else out
        y, nb, ld = _block(Y)
        o, _, _ = _block(out)
        self._check(self.lib.chebfi_apply_S(self.h, y, o, nb, ld, _stream()))
        return out

    def apply_Sinv(self, X, out=None):
        out = self._out_like(X) if out is None else out
        x, nb, ld = _block(X)
        o, _, _ = _block(out)
        self._check(self.lib.chebfi_apply_Sinv(self.h, x, o, nb, ld, _stream()))
        return out

    def apply_Sinv_refined(self, X, tol: float = 1e-12, maxit: int = 200, out=None):
        """S^{-1} X with the Woodbury reduced system solved by preconditioned iterative
        refinement; returns (out, iterations)."""
        out = self._out_like(X) if out is None else out
        x, nb, ld = _block(X)
        o, _, _ = _block(out)
        its = ctypes.c_int(0)
        self._check(self.lib.chebfi_apply_Sinv_refined(self.h, x, o, nb, ld, tol, maxit, ctypes.byref(its),
                                                       _stream()))
        return out, its.value

    def cheb_filter(self, Y, degree: int, lambda_lo: float, lambda_hi: float, prec: int = F64, proj=None):
        """In place on Y; returns Y.  proj: P^H Y (nproj x nb complex128 CUDA tensor, column-major)
        as rayleigh_ritz(..., proj=...) wrote it for this Y, which saves the filter's first P^H Y."""
        y, nb, ld = _block(Y)
        if proj is None:
            self._check(self.lib.chebfi_cheb_filter(self.h, y, nb, ld, degree, lambda_lo, lambda_hi, prec,
                                                    _stream()))
            return Y
        p, pnb, ldp = self._proj_block(proj, nb)
        self._check(self.lib.chebfi_cheb_filter_proj(self.h, y, p, ldp, nb, ld, degree, lambda_lo, lambda_hi, prec,
                                                     _stream()))
        return Y

    def _proj_block(self, proj, nb):
        p, pnb, ldp = _block(proj)
        if pnb != nb or proj.shape[0] != self.nproj:
            raise ValueError("projections must be nproj x nb")
        return p, pnb, max(ldp, self.nproj)

    @staticmethod
    def _host_block(Y):
        if not (isinstance(Y, torch.Tensor) and not Y.is_cuda and Y.dtype == torch.complex128 and Y.dim() == 2):
            raise TypeError("expected a 2-D complex128 CPU tensor")
        if Y.shape[1] > 0 and Y.stride(0) != 1:
            raise ValueError("host block must be column-major")
        nb = int(Y.shape[1])
        ld = int(Y.stride(1)) if nb > 1 else max(int(Y.shape[0]), 1)
        return ctypes.c_void_p(Y.data_ptr() if Y.numel() else 0), nb, max(ld, int(Y.shape[0]))

    def cheb_filter_host(self, Y, degree: int, lambda_lo: float, lambda_hi: float, prec: int = F64,
                         nchunks: int = 0, proj=None):
        """chebfi_cheb_filter on a host block (complex128 CPU tensor, column-major, ideally pinned),
        in place; the copies overlap the filter of neighbouring band chunks.  proj: P^H Y as an
        nproj x nb host tensor (column-major), copied in chunk by chunk.  Returns Y."""
        y, nb, ld = self._host_block(Y)
        if proj is None:
            self._check(self.lib.chebfi_cheb_filter_host(self.h, y, nb, ld, degree, lambda_lo, lambda_hi, prec,
                                                         nchunks, _stream()))
            return Y
        p, pnb, ldp = self._host_block(proj)
        if pnb != nb or proj.shape[0] != self.nproj:
            raise ValueError("projections must be nproj x nb")
        self._check(self.lib.chebfi_cheb_filter_host_proj(self.h, y, p, max(ldp, self.nproj), nb, ld, degree,
                                                          lambda_lo, lambda_hi, prec, nchunks, _stream()))
        return Y

    def orthonormalise(self, Y):
        y, nb, ld = _block(Y)
        self._check(self.lib.chebfi_orthonormalise(self.h, y, nb, ld, _stream()))
        return Y

    def rayleigh_ritz(self, Y, residuals: bool = True, proj=None):
        """Returns (Ritz values, residual norms or None).  proj: an nproj x nb complex128 CUDA
        tensor (column-major) that receives P^H Y of the rotated block."""
        y, nb, ld = _block(Y)
        ev = torch.empty(nb, dtype=torch.float64, device=Y.device)
        rs = torch.empty(nb, dtype=torch.float64, device=Y.device) if residuals else None
        rsp = ctypes.c_void_p(rs.data_ptr()) if rs is not None else None
        if proj is None:
            self._check(self.lib.chebfi_rayleigh_ritz(self.h, y, ctypes.c_void_p(ev.data_ptr()), rsp, nb, ld,
                                                      _stream()))
        else:
            p, _, ldp = self._proj_block(proj, nb)
            self._check(self.lib.chebfi_rayleigh_ritz_proj(self.h, y, ctypes.c_void_p(ev.data_ptr()), rsp, p, ldp,
                                                           nb, ld, _stream()))
        return ev, rs

    def rayleigh_quotients(self, Y):
        y, nb, ld = _block(Y)
        rq = torch.empty(nb, dtype=torch.float64, device=Y.device)
        self._check(self.lib.chebfi_rayleigh_quotients(self.h, y, ctypes.c_void_p(rq.data_ptr()), nb, ld,
                                                       _stream()))
        return rq

    def solve(self, Y, degree: int, sweeps: int, prec: int = F64, bound_mode: int = BOUND_PAPER,
              lambda_hi: float = 0.0, lock_tol: float = 0.0):
        """Algorithm 2 repeated `sweeps` times in place on Y; returns (evals, residual norms).
        lock_tol > 0 turns on locking with per-band degrees (Section 5.4)."""
        y, nb, ld = _block(Y)
        ev = torch.empty(nb, dtype=torch.float64, device=Y.device)
        rs = torch.empty(nb, dtype=torch.float64, device=Y.device)
        p = Params(degree, sweeps, prec, bound_mode, float(lambda_hi), float(lock_tol), 1 if lock_tol > 0 else 0)
        self._check(self.lib.chebfi_solve(self.h, y, ctypes.c_void_p(ev.data_ptr()), ctypes.c_void_p(rs.data_ptr()),
                                          nb, ld, ctypes.byref(p), _stream()))
        return ev, rs

    def set_fp64_gemm(self, engine: int = GEMM_AUTO, nmod: int = 0) -> int:
        """Engine of the FP64 complex GEMMs (GEMM_AUTO, GEMM_CUDA_CORES, GEMM_TENSOR) and the
        modulus count of the tensor-core emulation (0 keeps it); returns its precision E."""
        e = ctypes.c_int(0)
        self._check(self.lib.chebfi_set_fp64_gemm(self.h, engine, nmod, ctypes.byref(e)))
        return e.value

    def selftest_bounded_wait(self, which: int, limit_ms: float):
        """Run a wait that nothing satisfies (0: grid barrier, 1: mbarrier); returns (code the
        kernel recorded, elapsed ms)."""
        code = ctypes.c_int(0)
        ms = ctypes.c_double(0.0)
        self._check(self.lib.chebfi_selftest_bounded_wait(self.h, which, limit_ms, ctypes.byref(code),
                                                          ctypes.byref(ms)))
        return code.value, ms.value

    def probe_fma_rate(self, prec: int = F64):
        """Measured FMA throughput of the CUDA cores: (TFLOP/s, ms of the timed run)."""
        tf = ctypes.c_double(0.0)
        ms = ctypes.c_double(0.0)
        self._check(self.lib.chebfi_probe_fma_rate(self.h, prec, ctypes.byref(tf), ctypes.byref(ms)))
        return tf.value, ms.value

    def set_fft64(self, mode: int):
        """Arithmetic of the FP64 path's FFT passes: FFT64_DOUBLE_FLOAT (initial; pairs of
        floats on the FP32 units) or FFT64_NATIVE (the FP64 units)."""
        self._check(self.lib.chebfi_set_fft64(self.h, mode))

    def set_eigensolver(self, mode: int):
        """Dense eigensolver of Rayleigh-Ritz: EIG_AUTO, EIG_JACOBI (FP64) or EIG_REFINED (FP32
        Jacobi + FP64 refinement)."""
        self._check(self.lib.chebfi_set_eigensolver(self.h, mode))

    @property
    def eigensolver_steps(self) -> int:
        """Refinement steps of the last dense eigensolve (0: FP64 Jacobi ran)."""
        return int(self.lib.chebfi_eigensolver_steps(self.h))

    def gemm_fp64(self, A, B, conjA: bool = False, conjB: bool = False, alpha: float = 1.0, beta: float = 0.0,
                  C=None):
        """C = alpha op(A) op(B) + beta C for column-major complex128 CUDA matrices."""
        def mat(X):
            if not (isinstance(X, torch.Tensor) and X.is_cuda and X.dtype == torch.complex128 and X.dim() == 2):
                raise TypeError("expected a 2-D complex128 CUDA tensor")
            if X.shape[0] > 1 and X.shape[1] > 1 and X.stride(0) != 1:
                raise ValueError("matrices must be column-major (use fortran())")
            ld = X.stride(1) if X.shape[1] > 1 else X.shape[0]  # a size-1 dimension's stride is free
            return ctypes.c_void_p(X.data_ptr()), int(max(ld, X.shape[0], 1))
        m = A.shape[1] if conjA else A.shape[0]
        k = A.shape[0] if conjA else A.shape[1]
        n = B.shape[0] if conjB else B.shape[1]
        if (B.shape[1] if conjB else B.shape[0]) != k:
            raise ValueError("inner dimensions differ")
        if C is None:
            C = torch.zeros((n, m), dtype=torch.complex128, device=A.device).T
        a, lda = mat(A)
        b, ldb = mat(B)
        c, ldc = mat(C)
        self._check(self.lib.chebfi_gemm_fp64(self.h, int(conjA), int(conjB), m, n, k, alpha, a, lda, b, ldb, beta,
                                              c, ldc, _stream()))
        return C

    def gemm_mixed(self, A, B, conjA: bool = False, alpha: float = 1.0, beta: float = 0.0, C=None):
        """C = alpha op(A) B + beta C for column-major complex64 CUDA matrices, on the tensor
        cores (bf16 pairs, three real products; the mixed form's projector GEMMs)."""
        def mat(X):
            if not (isinstance(X, torch.Tensor) and X.is_cuda and X.dtype == torch.complex64 and X.dim() == 2):
                raise TypeError("expected a 2-D complex64 CUDA tensor")
            if X.shape[0] > 1 and X.shape[1] > 1 and X.stride(0) != 1:
                raise ValueError("matrices must be column-major")
            ld = X.stride(1) if X.shape[1] > 1 else X.shape[0]
            return ctypes.c_void_p(X.data_ptr()), int(max(ld, X.shape[0], 1))
        m = A.shape[1] if conjA else A.shape[0]
        k = A.shape[0] if conjA else A.shape[1]
        n = B.shape[1]
        if B.shape[0] != k:
            raise ValueError("inner dimensions differ")
        if C is None:
            C = torch.zeros((n, m), dtype=torch.complex64, device=A.device).T
        a, lda = mat(A)
        b, ldb = mat(B)
        c, ldc = mat(C)
        self._check(self.lib.chebfi_gemm_mixed(self.h, int(conjA), m, n, k, alpha, a, lda, b, ldb, beta, c, ldc,
                                               _stream()))
        return C

    def solve_stats(self):
        """(sweeps performed, band-H-applications of the filters) of the last solve."""
        sw = ctypes.c_int(0)
        ap = ctypes.c_int64(0)
        self._check(self.lib.chebfi_solve_stats(self.h, ctypes.byref(sw), ctypes.byref(ap)))
        return sw.value, ap.value

    def cheb_filter_adaptive(self, Y, degrees, lambda_lo: float, lambda_hi: float, prec: int = F64):
        """In place on Y: band j filtered to degree degrees[j] (Section 5.4); returns Y."""
        y, nb, ld = _block(Y)
        d = np.ascontiguousarray(np.asarray(degrees, dtype=np.int32))
        if d.shape != (nb,):
            raise ValueError("one degree per band")
        self._check(self.lib.chebfi_cheb_filter_adaptive(self.h, y, nb, ld, ctypes.c_void_p(d.ctypes.data),
                                                         lambda_lo, lambda_hi, prec, _stream()))
        return Y

    @staticmethod
    def adaptive_degrees(ritz, resid, lambda_lo: float, lambda_hi: float, tol: float, max_degree: int):
        """Section 5.4's per-band degree for a residual tolerance (host computation)."""
        lib = _lib.load()
        r = np.ascontiguousarray(np.asarray(ritz, dtype=np.float64))
        s_ = np.ascontiguousarray(np.asarray(resid, dtype=np.float64))
        out = np.zeros(r.shape[0], dtype=np.int32)
        rc = lib.chebfi_adaptive_degrees(ctypes.c_void_p(r.ctypes.data), ctypes.c_void_p(s_.ctypes.data), r.shape[0],
                                         lambda_lo, lambda_hi, tol, max_degree, ctypes.c_void_p(out.ctypes.data))
        if rc != 0:
            raise ChebFIError(rc, "chebfi_adaptive_degrees: bad arguments")
        return out

    def sync_status(self):
        self._check(self.lib.chebfi_sync_status(self.h))

    def profile(self, enable: bool = True):
        """Start (clearing totals) or stop per-kernel CUDA-event timing in the library."""
        self._check(self.lib.chebfi_profile_enable(self.h, 1 if enable else 0))

    def profile_totals(self):
        """{kernel name: (total ms, launches, algorithmic work)} recorded while profiling was on."""
        n = self.lib.chebfi_profile_count(self.h)
        if n < 0:
            self._check(n)
        out = {}
        buf = ctypes.create_string_buffer(128)
        for i in range(n):
            ms = ctypes.c_double()
            cnt = ctypes.c_int64()
            wk = ctypes.c_double()
            self._check(self.lib.chebfi_profile_entry(self.h, i, buf, 128, ctypes.byref(ms), ctypes.byref(cnt),
                                                      ctypes.byref(wk)))
            out[buf.value.decode()] = (ms.value, cnt.value, wk.value)
        return out

    @property
    def kernel_launches(self) -> int:
        return int(self.lib.chebfi_kernel_launches(self.h))


class ChebFIBatch:
    """Algorithm 2's filter for many k-points of one cell in grouped launches (libchebfi
    chebfi_batch_*).  ``contexts``: set-up ChebFI objects sharing grid, V_loc, atoms, D and
    Q; they are kept alive by the batch."""

    def __init__(self, contexts, nbands: int):
        self.lib = _lib.load()
        self.contexts = list(contexts)
        self.nbands = int(nbands)
        arr = (ctypes.c_void_p * len(self.contexts))(*[c.h.value for c in self.contexts])
        h = ctypes.c_void_p()
        with torch.cuda.device(self.contexts[0].device):
            rc = self.lib.chebfi_batch_create(ctypes.byref(h), arr, len(self.contexts), self.nbands)
        if rc != 0:
            raise ChebFIError(rc, "chebfi_batch_create failed (contexts not compatible or not set up)")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.chebfi_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != 0:
            raise ChebFIError(rc, self.lib.chebfi_batch_last_error(self.h).decode())

    @property
    def kernel_launches(self) -> int:
        return int(self.lib.chebfi_batch_kernel_launches(self.h))

    def autotune(self, prec: int = F32):
        """(tile shape per GEMM class, split-K factor of P^H Z, ms per (class, shape) at split 1
        (3 x 4), best ms per split factor 1, 2, 4, 8)."""
        shapes = (ctypes.c_int * 4)()
        ms = (ctypes.c_double * 16)()
        self._check(self.lib.chebfi_batch_autotune(self.h, prec, shapes, ms))
        m = np.array(ms[:])
        return list(shapes[:3]), int(shapes[3]), m[:12].reshape(3, 4), m[12:]

    def set_tiles(self, shapes, split: int, prec: int = F32):
        """Override the autotuner's tile shapes (3 indices) and P^H Z split-K factor."""
        arr = (ctypes.c_int * 3)(*[int(x) for x in shapes])
        self._check(self.lib.chebfi_batch_set_tiles(self.h, prec, arr, int(split)))

    def cheb_filter(self, Ys, degree: int, lambda_lo, lambda_hi, prec: int = F32):
        """In place on every block of ``Ys`` (one complex128 column-major tensor per k-point);
        returns Ys."""
        nk = len(self.contexts)
        if len(Ys) != nk:
            raise ValueError("one block per k-point")
        ptrs, lds = [], []
        for Y, c in zip(Ys, self.contexts):
            y, nb, ld = _block(Y)
            if nb != self.nbands or Y.shape[0] != c.npw:
                raise ValueError("block shape does not match its k-point")
            ptrs.append(y.value)
            lds.append(ld)
        P = (ctypes.c_void_p * nk)(*ptrs)
        L = (ctypes.c_int64 * nk)(*lds)
        lo = (ctypes.c_double * nk)(*[float(x) for x in lambda_lo])
        hi = (ctypes.c_double * nk)(*[float(x) for x in lambda_hi])
        self._check(self.lib.chebfi_batch_cheb_filter(self.h, P, L, degree, lo, hi, prec, _stream()))
        return Ys
