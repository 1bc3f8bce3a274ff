"""kNN build on the tensor cores vs the oracle's exact brute force (``-m gpu``).

Both methods must return the oracle's graph bit for bit (same FP32 chain or
exact integer distances, ties to the lower index), at sizes that span several
256-column tiles and a ragged tail, for list lengths up to the 32 candidates
the tensor-core pass keeps.  Float rows whose candidate list cannot be
certified (large norms against small distance gaps) are recomputed exactly.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2303_05455_gb300 import ivhd, synth
from paper_2303_05455_gb300._lib import IvhdError

pytestmark = pytest.mark.gpu


def gmm(M, N, seed, offset=0.0):
    X, _ = synth.gaussian_mixture(M, N, 7, seed)
    return (X + np.float32(offset)).astype(np.float32)


@pytest.mark.parametrize("method", ["tensor_cores", "cuda_cores"])
@pytest.mark.parametrize("M,N,k", [(300, 37, 5), (1000, 50, 1), (1000, 50, 32), (2000, 100, 5),
                                   (777, 129, 7)])
def test_knn_f32_methods_bit_exact(method, M, N, k):
    X = gmm(M, N, M + N)
    got, st = ivhd.knn_build(torch.from_numpy(X).cuda(), k, method=method, return_stats=True)
    assert st["method"] == method
    assert np.array_equal(got.cpu().numpy(), oracle.knn_f32(X, k))
    if method == "tensor_cores":
        assert st["max_rel_err"] <= st["eps_coef"] / 8


@pytest.mark.parametrize("method", ["tensor_cores", "cuda_cores"])
@pytest.mark.parametrize("M,N,k", [(300, 64, 5), (1500, 784, 5), (600, 100, 32), (513, 1024, 3),
                                   (3000, 64, 12)])
def test_knn_u8_methods_bit_exact(method, M, N, k):
    X, _ = synth.mnist_like(M, 3, N=N)
    got, st = ivhd.knn_build(torch.from_numpy(X).cuda(), k, method=method, return_stats=True)
    assert st["method"] == method and st["fallback_rows"] == 0
    assert np.array_equal(got.cpu().numpy(), oracle.knn_u8(X, k))


@pytest.mark.parametrize("dtype", ["f32", "u8"])
def test_knn_tc_ties_to_lower_index(dtype):
    rng = np.random.default_rng(4)
    base = rng.integers(0, 256, size=(40, 48))
    X = np.concatenate([base, base, base[:7]])      # every row has exact twins
    X = X.astype(np.float32) if dtype == "f32" else X.astype(np.uint8)
    ref = oracle.knn_f32(X, 4) if dtype == "f32" else oracle.knn_u8(X, 4)
    got = ivhd.knn_build(torch.from_numpy(X).cuda(), 4, method="tensor_cores")
    assert np.array_equal(got.cpu().numpy(), ref)


def test_knn_tc_uncertified_rows_are_recomputed():
    # a large common offset inflates the norms, so the bound cannot separate the
    # k-th neighbour from the 32nd candidate: those rows take the exact path
    X = gmm(1200, 20, 5, offset=3000.0)
    got, st = ivhd.knn_build(torch.from_numpy(X).cuda(), 5, method="tensor_cores",
                             return_stats=True)
    assert st["fallback_rows"] > 0
    assert np.array_equal(got.cpu().numpy(), oracle.knn_f32(X, 5))


def test_knn_auto_picks_tensor_cores_and_rejects_out_of_range():
    X = gmm(500, 16, 1)
    Xd = torch.from_numpy(X).cuda()
    _, st = ivhd.knn_build(Xd, 5, return_stats=True)
    assert st["method"] == "tensor_cores"
    _, st = ivhd.knn_build(Xd, 40, return_stats=True)  # k > 32: CUDA cores
    assert st["method"] == "cuda_cores"
    with pytest.raises(IvhdError):
        ivhd.knn_build(Xd, 40, method="tensor_cores")
    Xu = torch.from_numpy(synth.mnist_like(300, 1, N=1100)[0]).cuda()
    _, st = ivhd.knn_build(Xu, 5, return_stats=True)    # N > 1024: sums could leave FP32's exact range
    assert st["method"] == "cuda_cores"


def test_uncertified_rows_in_column_segments():
    # 12,000 points with a large common offset: many rows fail the certificate
    # and the exact kernel sweeps their candidates in parallel column segments
    X = gmm(12_000, 20, 8, offset=3000.0)
    got, st = ivhd.knn_build(torch.from_numpy(X).cuda(), 5, method="tensor_cores",
                             return_stats=True)
    assert st["fallback_rows"] > 100
    assert np.array_equal(got.cpu().numpy(), oracle.knn_f32(X, 5))
