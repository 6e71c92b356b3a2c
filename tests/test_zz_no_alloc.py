"""chebfi_apply_H_noalloc: the allocation-free H application for callers that cannot
allocate device memory where they call it (a host callback or latency-critical section
that must not take the allocator's lock, or a framework that owns all device memory).  Its
output must match chebfi_apply_H on two calls in a row; both go through the C ABI.  The
device's free memory does not change across a call, and a cell whose single band needs
more scratch than the static array holds is refused.  This file is collected last on
purpose."""
import ctypes

import numpy as np
import pytest
import torch

from oracle.planewave import PWOperator
from synth import config_cell

pytestmark = pytest.mark.gpu

TOL64 = 1e-11  # the FP64 parity tolerance of the other GPU tests


def _call_noalloc(g, Y, out, expect=0):
    from paper_1406_4350_gb300.chebfi import _block, _stream
    f = g.lib.chebfi_apply_H_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                  ctypes.c_void_p]
    y, nb, ld = _block(Y)
    o, _, _ = _block(out)
    rc = f(g.h, y, o, nb, ld, _stream())
    msg = g.lib.chebfi_last_error(g.h).decode()
    assert rc == expect, (rc, msg)
    return msg


def test_apply_H_noalloc_matches_apply_H_on_two_calls():
    from paper_1406_4350_gb300 import build
    from paper_1406_4350_gb300.chebfi import ChebFI, fortran
    build.build()
    # 120 bands of the 48^3 PAW cell: more than one chunk of the 32 MiB scratch
    cell = config_cell("paw48", nbands=120)
    g = ChebFI.from_cell(cell)
    Y = fortran(cell.Y0)
    ref = g.apply_H(Y)
    torch.cuda.synchronize()
    ref = ref.cpu().numpy()
    scale = np.abs(ref).max()
    outs = [torch.full_like(Y, float("nan")) for _ in range(2)]
    torch.cuda.synchronize()
    for i in range(2):
        free0 = torch.cuda.mem_get_info()[0]
        _call_noalloc(g, Y, outs[i])
        torch.cuda.synchronize()
        if i == 1:  # the first call may do its one-time set-up; the second allocates nothing
            assert torch.cuda.mem_get_info()[0] == free0
        got = outs[i].cpu().numpy()
        assert np.abs(got - ref).max() <= TOL64 * scale
    # and the oracle agrees with both
    assert np.abs(got - PWOperator.from_cell(cell).apply_H(cell.Y0)).max() <= TOL64 * scale
    g.sync_status()


def test_apply_H_noalloc_refuses_a_band_larger_than_its_scratch():
    """A 256^3 grid whose sphere has more than 8192 (x, y) columns needs over 32 MiB of FFT
    column buffer for one band: the call returns CHEBFI_ERR_ARG before any work."""
    from paper_1406_4350_gb300 import build
    from paper_1406_4350_gb300._lib import ERR_ARG
    from paper_1406_4350_gb300.chebfi import ChebFI
    build.build()
    n, R = 256, 52
    r = np.arange(-R, R + 1)
    m = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3)
    m = m[np.sum(m * m, 1) <= R * R].astype(np.int32)
    g = ChebFI(0)
    g.set_cell(np.eye(3) * 2 * np.pi, (n, n, n))
    g.set_sphere(m)
    g.set_vloc(np.zeros((n, n, n)))
    g.set_projectors(np.zeros((m.shape[0], 0), complex), np.array([0], np.int32), np.zeros(0))
    Y = torch.zeros((1, m.shape[0]), dtype=torch.complex128, device="cuda").T
    out = torch.zeros_like(Y)
    msg = _call_noalloc(g, Y, out, expect=ERR_ARG)
    assert "32 MiB" in msg
