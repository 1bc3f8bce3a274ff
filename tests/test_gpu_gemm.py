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


# shapes below and above one tile, ragged M / N / K, 128- and 256-column tiles,
# one and several tiles per persistent CTA
@pytest.mark.parametrize("M,N,K", [(128, 64, 64), (128, 128, 128), (300, 200, 72),
                                   (256, 512, 832), (4096, 512, 512), (1000, 64, 4096),
                                   (5000, 1000, 200), (4864, 1024, 192)])
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


def test_gemm_many_tiles_per_cta_sampled_rows():
    """4096^3: 512 tiles of 128 x 256 on the persistent grid (several per CTA, both
    tensor-memory accumulators in use), checked on sampled rows of every tile row."""
    M = N = K = 4096
    g = torch.Generator(device="cuda").manual_seed(7)
    A = torch.randn((M, K), device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn((N, K), device="cuda", generator=g).to(torch.bfloat16)
    C = ivhd.gemm_bf16_tn(A, B)
    rows = torch.arange(5, M, 127, device="cuda")
    ref = A[rows].double() @ B.double().T
    scale = A[rows].double().abs() @ B.double().abs().T
    err = (C[rows].double() - ref).abs()
    assert bool((err <= K * 2 ** -24 * scale + 1e-30).all())
    C2 = ivhd.gemm_bf16_tn(A, B)
    assert torch.equal(C, C2)                       # deterministic
