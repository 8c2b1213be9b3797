"""The tensor-core GEMM (tcgen05 kind::tf32, TMA-fed) against an FP64 torch
reference: complex and real, every conjugation mode, plain TF32 and 3xTF32
products (B expanded inside the GEMM, or beforehand: mode 2), shapes
spanning several 128-row tiles with ragged M, N and K tails.

Normwise bound |C - C_ref|_F <= tol |A|_F |B|_F: TF32 keeps 10+1 mantissa
bits (relative rounding ~2^-11 per operand), 3xTF32 ~2^-21.
"""
import pytest
import torch

from paper_2006_15234_gb300 import libpeps

pytestmark = pytest.mark.gpu

# N chosen to reach every MMA width: complex tiles of 32 / 64 / 96 / 128 columns
SHAPES = [(128, 64, 16), (300, 200, 90), (257, 129, 1000), (64, 70, 34), (130, 272, 48), (64, 20, 34)]


def _ref(A, B, cA, cB):
    A64, B64 = A.to(torch.complex128 if A.is_complex() else torch.float64), \
        B.to(torch.complex128 if B.is_complex() else torch.float64)
    if cA:
        A64 = A64.conj()
    if cB:
        B64 = B64.conj()
    return A64 @ B64.T


@pytest.mark.parametrize("split3,tol", [(False, 2e-3), (True, 2e-6), (2, 2e-6)])
@pytest.mark.parametrize("cA,cB", [(False, False), (True, False), (False, True), (True, True)])
@pytest.mark.parametrize("shape", SHAPES)
def test_complex(shape, cA, cB, split3, tol):
    M, N, K = shape
    g = torch.Generator(device="cuda").manual_seed(M * 7 + N)
    A = torch.randn(M, K, dtype=torch.complex64, device="cuda", generator=g)
    B = torch.randn(N, K, dtype=torch.complex64, device="cuda", generator=g)
    C = libpeps.debug_tc_gemm(A, B, cA, cB, split3)
    torch.cuda.synchronize()
    R = _ref(A, B, cA, cB)
    err = (C.to(torch.complex128) - R).norm() / (A.norm().double() * B.norm().double())
    assert err <= tol, float(err)


@pytest.mark.parametrize("split3,tol", [(False, 2e-3), (True, 2e-6), (2, 2e-6)])
@pytest.mark.parametrize("shape", [(128, 64, 32), (300, 200, 92), (257, 129, 1000), (150, 190, 64),
                                   (100, 40, 36)])
def test_real(shape, split3, tol):
    M, N, K = shape
    g = torch.Generator(device="cuda").manual_seed(M + N)
    A = torch.randn(M, K, dtype=torch.float32, device="cuda", generator=g)
    B = torch.randn(N, K, dtype=torch.float32, device="cuda", generator=g)
    C = libpeps.debug_tc_gemm(A, B, False, False, split3)
    torch.cuda.synchronize()
    R = _ref(A, B, False, False)
    err = (C.double() - R).norm() / (A.norm().double() * B.norm().double())
    assert err <= tol, float(err)


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("K", [4096, 16384])
def test_split3_long_sums_unbiased(cplx, K, mode):
    """Same-sign data, long K: an accumulator that truncates the low bits of
    every addend drifts by a relative ~1e-8 per K value (1.6e-4 at K = 16384);
    3xTF32 products accumulated with round-to-nearest stay at FP32 level.
    Elementwise bound against sum |a||b|: 2e-6 (K-independent)."""
    M, N = 200, 136
    g = torch.Generator(device="cuda").manual_seed(K + cplx)
    dt = torch.complex64 if cplx else torch.float32
    A = (torch.rand(M, K, device="cuda", generator=g) + 0.5).to(dt)
    B = (torch.rand(N, K, device="cuda", generator=g) + 0.5).to(dt)
    if cplx:
        A = A * torch.exp(0.3j * torch.rand(M, K, device="cuda", generator=g))
        B = B * torch.exp(-0.3j * torch.rand(N, K, device="cuda", generator=g))
    C = libpeps.debug_tc_gemm(A, B, False, False, mode)
    torch.cuda.synchronize()
    R = _ref(A, B, False, False)
    S = A.abs().double() @ B.abs().double().T
    err = ((C.to(R.dtype) - R).abs() / S).max()
    assert err <= 2e-6, float(err)
