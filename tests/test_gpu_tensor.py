"""Tensor-core products of the mixed form, through the C ABI self-tests:
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
    # entries spanning several binades, as the kernel matrices and solutions do
    A = torch.randn(M, K, dtype=torch.float64, device="cuda", generator=g) * torch.exp(
        torch.randn(M, K, dtype=torch.float64, device="cuda", generator=g))
    B = torch.randn(K, Nn, dtype=torch.float64, device="cuda", generator=g)
    return A, B


@pytest.mark.parametrize("M,Nn,K", SHAPES)
def test_sliced_product_is_fp32_accurate(ww, M, Nn, K):
    A, B = operands(M, Nn, K, 1)
    err = ww.selftest("f32gemm", A, B)
    assert err < 2e-6, err


@pytest.mark.parametrize("M,Nn,K", SHAPES)
def test_digit_product_is_fp64_accurate(ww, M, Nn, K):
    A, B = operands(M, Nn, K, 2)
    err = ww.selftest("ozaki", A, B)
    assert err < 1e-14, err
