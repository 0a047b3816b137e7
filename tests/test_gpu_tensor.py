"""Dense products of both forms, through the C ABI self-tests, against an
independent host product (numpy FP64 matmul of the same operands, copied to
the CPU): the 3+3-slice bf16 tensor-core product must be FP32-accurate, the
7+7-digit tensor-core product (Ozaki scheme) and the FP64 DGEMM of the plain
form FP64-accurate, on shapes that cover one tile, several tiles, ragged
edges and the full N = 2048 x 514 x 2048 size of the benchmark.  Standard-
normal operands; the error is max|C - C_host| / max|C_host|."""
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


def rel_err(ww, kind, M, Nn, K, seed):
    A, B = operands(M, Nn, K, seed)
    C = ww.selftest(kind, A, B).cpu().numpy()
    ref = A.cpu().numpy() @ B.cpu().numpy()
    return float(np.abs(C - ref).max() / np.abs(ref).max())


@pytest.mark.parametrize("M,Nn,K", SHAPES)
def test_sliced_product_is_fp32_accurate(ww, M, Nn, K):
    err = rel_err(ww, "f32gemm", M, Nn, K, 1)
    # 24-bit operands; the tensor cores accumulate in fp32 once per K = 16 MMA
    # and pair (6 K/16 roundings), ~1e-5 of max |C| at K = 2048 -- ample for
    # a preconditioner, whose error is squared away by the refinement
    assert err < 3e-5, err


@pytest.mark.parametrize("M,Nn,K", SHAPES)
def test_digit_product_is_fp64_accurate(ww, M, Nn, K):
    err = rel_err(ww, "ozaki", M, Nn, K, 2)
    # the kept pairs end at g = 6; the first dropped group (g = 7, weight
    # 2^-61 of 2^(ea + fb)) is ~5e-14 of max|C| for Gaussian operands.  The
    # host product's own rounding (~1e-15 of max|C|) is far below.  For the
    # kernel matrices the dropped group is far smaller relative to the result,
    # whose row maxima are O(1/N) of the operator norm.
    assert err < 1.5e-13, err


@pytest.mark.parametrize("M,Nn,K", SHAPES)
def test_fp64_dgemm_is_fp64_accurate(ww, M, Nn, K):
    err = rel_err(ww, "dgemm", M, Nn, K, 3)
    # two FP64 sums of K products in different orders: ~sqrt(K) eps of max|C|
    assert err < 1e-14, err


def test_assembly_reciprocal_within_one_ulp(ww):
    """The Newton-Raphson reciprocal of the kernel assembly against the division
    operator, over 16 decades of positive normal doubles (the denominators of
    the cotangent quotients lie between ~1e-7 and ~1e5)."""
    import torch
    g = torch.Generator(device="cuda").manual_seed(7)
    d = torch.pow(10.0, torch.empty(1 << 16, dtype=torch.float64, device="cuda").uniform_(-8, 8, generator=g))
    d = torch.cat([d, torch.tensor([1.0, 2.0, 0.5, 3.0, 1e-7, 1e5], dtype=torch.float64, device="cuda")])
    assert ww.selftest_recip(d) <= 2.3e-16   # one ulp of the quotient
