"""Tensor-core products of the mixed form, through the C ABI self-tests
(standard-normal operands; the reference is the library's FP64 DGEMM):
the 3+3-slice bf16 product must be FP32-accurate, the 7+7-digit product
(Ozaki scheme) FP64-accurate, on shapes that cover one tile, several tiles,
ragged edges and the full N = 2048 x 514 x 2048 size of the benchmark."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SHAPES = [(128, 128, 64), (128, 64, 128), (256, 130, 256), (64, 20, 64), (512, 70, 1024), (2048, 514, 2048)]


@pytest.fixture(scope="module")
def ww():
    from paper_1210_5672_gb300 import build as B
    B.build()
    import paper_1210_5672_gb300 as m
    return m


def operands(M, Nn, K, seed):
    import torch
    g = torch.Generator(device="cuda").manual_seed(seed)
    A = torch.randn(M, K, dtype=torch.float64, device="cuda", generator=g)
    B = torch.randn(K, Nn, dtype=torch.float64, device="cuda", generator=g)
    return A, B


@pytest.mark.parametrize("M,Nn,K", SHAPES)
def test_sliced_product_is_fp32_accurate(ww, M, Nn, K):
    A, B = operands(M, Nn, K, 1)
    err = ww.selftest("f32gemm", A, B)
    # 24-bit operands; the tensor cores accumulate in fp32 once per K = 16 MMA
    # and pair (6 K/16 roundings), ~1e-5 of max |C| at K = 2048 -- ample for
    # a preconditioner, whose error is squared away by the refinement
    assert err < 3e-5, err


@pytest.mark.parametrize("M,Nn,K", SHAPES)
def test_digit_product_is_fp64_accurate(ww, M, Nn, K):
    A, B = operands(M, Nn, K, 2)
    err = ww.selftest("ozaki", A, B)
    # the kept pairs end at g = 6; the first dropped group (g = 7, weight
    # 2^-61 of 2^(ea + fb)) is ~5e-14 of max|C| for Gaussian operands (the
    # same digits emulated exactly on the CPU give the same figure).  For the
    # kernel matrices it is far smaller relative to the result, whose row
    # maxima are O(1/N) of the operator norm.
    assert err < 1.5e-13, err


def test_assembly_reciprocal_within_one_ulp(ww):
    """The Newton-Raphson reciprocal of the kernel assembly against the division
    operator, over 16 decades of positive normal doubles (the denominators of
    the cotangent quotients lie between ~1e-7 and ~1e5)."""
    import torch
    g = torch.Generator(device="cuda").manual_seed(7)
    d = torch.pow(10.0, torch.empty(1 << 16, dtype=torch.float64, device="cuda").uniform_(-8, 8, generator=g))
    d = torch.cat([d, torch.tensor([1.0, 2.0, 0.5, 3.0, 1e-7, 1e5], dtype=torch.float64, device="cuda")])
    assert ww.selftest_recip(d) <= 2.3e-16   # one ulp of the quotient
