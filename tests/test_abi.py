"""The C-ABI library builds for sm_103a, loads, and exports every function that
include/chebfi.h declares (no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "chebfi.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(chebfi_[A-Za-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1406_4350_gb300 import build as b
    path = b.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for required in ["chebfi_create", "chebfi_set_cell", "chebfi_set_sphere", "chebfi_set_vloc",
                     "chebfi_set_projectors", "chebfi_apply_H", "chebfi_apply_Sinv", "chebfi_cheb_filter",
                     "chebfi_orthonormalise", "chebfi_rayleigh_ritz"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_signatures_cover_the_header():
    from paper_1406_4350_gb300 import _lib
    assert set(_declared()) <= set(_lib.SIGNATURES)


def test_null_context_is_rejected_without_a_gpu(lib):
    f = lib.chebfi_destroy
    f.argtypes = [ctypes.c_void_p]
    f.restype = ctypes.c_int
    assert f(None) == -1
    g = lib.chebfi_apply_H
    g.restype = ctypes.c_int
    assert g(None, None, None, ctypes.c_int64(0), ctypes.c_int64(0), 0, None) == -1


def test_create_fails_cleanly_without_a_device(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    h = ctypes.c_void_p()
    f = lib.chebfi_create
    f.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int]
    f.restype = ctypes.c_int
    assert f(ctypes.byref(h), 0) != 0
    assert not h.value


def test_product_package_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1406_4350_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
