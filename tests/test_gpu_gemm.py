"""tcgen05 BF16 GEMM (C = A B^T, FP32 accumulation) vs exact products of the same BF16 values."""
import numpy as np
import pytest
import torch

from paper_2303_05455_gb300 import ivhd

pytestmark = pytest.mark.gpu


def bf16(x):
    b = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


@pytest.mark.parametrize("M,N,K", [(128, 64, 64), (128, 128, 128), (300, 200, 72),
                                   (256, 512, 832), (4096, 512, 512), (1000, 64, 4096)])
def test_gemm_matches_exact_products(M, N, K):
    rng = np.random.default_rng(M + N + K)
    A = bf16(rng.standard_normal((M, K)))
    B = bf16(rng.standard_normal((N, K)))
    C = ivhd.gemm_bf16_tn(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()).cpu().numpy()
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    scale = np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64).T
    # FP32 accumulation of K exact BF16 x BF16 products: |err| <= K u sum|a b|
    assert np.all(np.abs(C - ref) <= K * 2 ** -24 * scale + 1e-30)
    assert np.abs(C - ref).max() <= 1e-5 * np.abs(ref).max()
