"""The TF32 tensor-core GEMM D = A B^T (the kernel behind the mixed-precision
ridge sketch) against FP64 products of the same inputs.

Small integers are exact in TF32 and their products and sums are exact in
FP32 here, so for integer inputs the tensor-core result must equal the FP64
reference bit for bit: any wrong descriptor, swizzle, K step or tile offset
shows up as a mismatch."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ny():
    from paper_2110_02820_gb300 import build, nyspcg
    build.build()
    nyspcg.lib()
    return nyspcg


SHAPES = [
    (128, 256, 32),       # one tile, one slab
    (128, 256, 4096),     # one tile, long K
    (512, 1000, 256),     # ragged N (BN = 256)
    (200, 300, 96),       # ragged M and N
    (512, 4096, 20000),   # small output, long K: split-K
    (256, 100, 64),       # N < 256 (BN = 128)
]


@pytest.mark.parametrize("M,N,K", SHAPES)
def test_tf32_gemm_integer_inputs_are_exact(ny, M, N, K):
    g = torch.Generator(device="cpu").manual_seed(M * 7 + N * 3 + K)
    A = torch.randint(-4, 5, (M, K), generator=g).float().cuda()
    B = torch.randint(-4, 5, (N, K), generator=g).float().cuda()
    D = ny.nys_gemm_tf32_tn(A, B)
    ref = (A.double() @ B.double().T)
    assert float(ref.abs().max()) < 2 ** 24
    assert torch.equal(D.double(), ref)


@pytest.mark.parametrize("M,N,K", SHAPES[:4])
def test_tf32_gemm_random_inputs_within_tf32_error(ny, M, N, K):
    g = torch.Generator(device="cpu").manual_seed(11)
    A = torch.randn((M, K), generator=g).cuda()
    B = torch.randn((N, K), generator=g).cuda()
    D = ny.nys_gemm_tf32_tn(A, B).double()
    ref = A.double() @ B.double().T
    # TF32 keeps 10 explicit mantissa bits: per-product relative error < 2^-9;
    # random signs give ~ 2^-10 sqrt(K) * |a||b| / sqrt(K) norm-wise
    err = float((D - ref).norm() / ref.norm())
    assert err < 2e-3


def test_tf32_gemm_rejects_unsupported(ny):
    A = torch.zeros((64, 30), device="cuda")  # row stride 30 floats = 120 B: not 16-byte multiple
    B = torch.zeros((64, 30), device="cuda")
    with pytest.raises(ny.NysError) as e:
        ny.nys_gemm_tf32_tn(A, B)
    assert e.value.status == ny.NYS_ERR_ARG
