"""The mixed form's tensor-core complex GEMM (chebfi_gemm_mixed: bf16 pairs, three real
products of the (Re, Im, Re -+ Im) planes), against a plain PyTorch complex128 product of the
same FP32 operands.  Bound per element: 1e-4 * (|op(A)| |B|)_ij, the size of the terms it sums
(each operand carries about 16 significant bits; the third product's planes are at most
sqrt(2) times larger)."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1406_4350_gb300 import build
    build.build()
    from paper_1406_4350_gb300.chebfi import ChebFI
    return ChebFI()


def _cmat(rng, r, c, scale=1.0):
    x = (rng.normal(size=(r, c)) + 1j * rng.normal(size=(r, c))) * scale
    return torch.from_numpy(np.asfortranarray(x.astype(np.complex64))).cuda()


def _check(ctx, A, B, conjA, alpha=1.0, beta=0.0, C0=None):
    C = None if C0 is None else C0.clone()
    out = ctx.gemm_mixed(A, B, conjA=conjA, alpha=alpha, beta=beta, C=C)
    torch.cuda.synchronize()
    a = A.cpu().numpy().astype(np.complex128)
    b = B.cpu().numpy().astype(np.complex128)
    opa = a.conj().T if conjA else a
    ref = alpha * (opa @ b)
    if C0 is not None and beta != 0.0:
        ref = ref + beta * C0.cpu().numpy().astype(np.complex128)
    scale = np.abs(alpha) * (np.abs(opa) @ np.abs(b))
    if C0 is not None and beta != 0.0:
        scale = scale + np.abs(beta * C0.cpu().numpy())
    err = np.abs(out.cpu().numpy() - ref)
    assert np.all(err <= 1e-4 * scale + 1e-30), "max err / scale %.3e" % (err / (scale + 1e-30)).max()
    return err.max() / scale.max()


@pytest.mark.parametrize("conjA", [True, False])
@pytest.mark.parametrize("m, n, k", [(1, 1, 1), (37, 5, 3), (130, 129, 700), (300, 200, 1500)])
def test_gemm_mixed_shapes(ctx, conjA, m, n, k):
    rng = np.random.default_rng(m * 1000 + n + k)
    A = _cmat(rng, k, m) if conjA else _cmat(rng, m, k)
    B = _cmat(rng, k, n)
    _check(ctx, A, B, conjA)


def test_gemm_mixed_long_contraction_split(ctx):
    """k long enough for the K split and its reduction (the P^H psi shape, smaller)."""
    rng = np.random.default_rng(11)
    A = _cmat(rng, 40000, 256)
    B = _cmat(rng, 40000, 256)
    _check(ctx, A, B, True)


def test_gemm_mixed_alpha_beta_in_place(ctx):
    rng = np.random.default_rng(12)
    A = _cmat(rng, 500, 64)
    B = _cmat(rng, 64, 40)
    C0 = _cmat(rng, 500, 40)
    _check(ctx, A, B, False, alpha=-0.75, beta=1.0, C0=C0)


def test_gemm_mixed_wide_dynamic_range(ctx):
    """Entries spread over 2^-20 .. 2^20 (the bound is per element, so small products must
    come out small-error too)."""
    rng = np.random.default_rng(13)
    A = _cmat(rng, 200, 96) * torch.from_numpy(2.0 ** rng.uniform(-20, 20, size=(200, 1))).cuda().to(torch.complex64)
    B = _cmat(rng, 96, 72) * torch.from_numpy(2.0 ** rng.uniform(-20, 20, size=(1, 72))).cuda().to(torch.complex64)
    _check(ctx, A, B, False)


def test_gemm_mixed_rejects_bad_arguments(ctx):
    import ctypes
    rng = np.random.default_rng(14)
    A = _cmat(rng, 8, 4)
    B = _cmat(rng, 5, 3)
    with pytest.raises(ValueError):
        ctx.gemm_mixed(A, B)
    with pytest.raises(TypeError):
        ctx.gemm_mixed(A.to(torch.complex128), _cmat(rng, 4, 3))
    rc = ctx.lib.chebfi_gemm_mixed(ctx.h, 0, 8, 3, 0, 1.0, ctypes.c_void_p(A.data_ptr()), 8,
                               ctypes.c_void_p(B.data_ptr()), 5, 0.0, ctypes.c_void_p(B.data_ptr()), 8, None)
    assert rc != 0  # k = 0
