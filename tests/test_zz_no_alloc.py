"""chebfi_apply_H_noalloc: the allocation-free H application for callers that cannot
allocate device memory where they call it (inside a stream capture, a host callback, or
under a framework that owns all device memory).  Its output must match chebfi_apply_H on
two calls in a row; both go through the C ABI.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

from oracle.planewave import PWOperator
from synth import config_cell

pytestmark = pytest.mark.gpu

TOL64 = 1e-11  # the FP64 parity tolerance of the other GPU tests


def _call_noalloc(g, Y, out):
    from paper_1406_4350_gb300.chebfi import _block, _stream
    f = g.lib.chebfi_apply_H_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                  ctypes.c_void_p]
    y, nb, ld = _block(Y)
    o, _, _ = _block(out)
    rc = f(g.h, y, o, nb, ld, _stream())
    assert rc == 0, g.lib.chebfi_last_error(g.h).decode()


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
    for _ in range(2):
        out = torch.full_like(Y, float("nan"))
        _call_noalloc(g, Y, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.abs(got - ref).max() <= TOL64 * scale
    # and the oracle agrees with both
    assert np.abs(got - PWOperator.from_cell(cell).apply_H(cell.Y0)).max() <= TOL64 * scale
    g.sync_status()
