"""kNN of new points against a base set and their placement (``-m gpu``).

ivhd_knn_query must return the oracle's lists bit for bit (the FP32 chain or
exact integer distances of the graph build, ties to the lower index, nothing
excluded) for both methods, at query counts with ragged 128-row tails and
base sets spanning several 256-column tiles; ivhd_place_nn must give the
neighbours' mean embedding (exactly for k = 1, the Progressive UMAP
placement of Sec. 2.4.3).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2303_05455_gb300 import ivhd, synth
from paper_2303_05455_gb300._lib import IvhdError

pytestmark = pytest.mark.gpu


def split_gmm(Mq, M, N, seed, offset=0.0):
    Z, _ = synth.gaussian_mixture(Mq + M, N, 7, seed)
    Z = (Z + np.float32(offset)).astype(np.float32)
    return Z[:Mq], Z[Mq:]


@pytest.mark.parametrize("method", ["tensor_cores", "cuda_cores"])
@pytest.mark.parametrize("Mq,M,N,k", [(1000, 3000, 50, 5), (129, 2000, 100, 1), (300, 777, 37, 32),
                                      (1, 600, 20, 7)])
def test_knn_query_f32_bit_exact(method, Mq, M, N, k):
    Q, X = split_gmm(Mq, M, N, Mq + M + N)
    got, st = ivhd.knn_query(torch.from_numpy(Q).cuda(), torch.from_numpy(X).cuda(), k,
                             method=method, return_stats=True)
    assert st["method"] == method
    assert np.array_equal(got.cpu().numpy(), oracle.knn_query(Q, X, k))
    if method == "tensor_cores":
        assert st["max_rel_err"] <= st["eps_coef"] / 8


@pytest.mark.parametrize("method", ["tensor_cores", "cuda_cores"])
@pytest.mark.parametrize("Mq,M,N,k", [(777, 2000, 784, 5), (200, 600, 100, 20), (130, 513, 1024, 3)])
def test_knn_query_u8_bit_exact(method, Mq, M, N, k):
    Z, _ = synth.mnist_like(Mq + M, 5, N=N)
    Q, X = Z[:Mq], Z[Mq:]
    got, st = ivhd.knn_query(torch.from_numpy(Q).cuda(), torch.from_numpy(X).cuda(), k,
                             method=method, return_stats=True)
    assert st["method"] == method and st["fallback_rows"] == 0
    assert np.array_equal(got.cpu().numpy(), oracle.knn_query(Q, X, k))


@pytest.mark.parametrize("dtype", ["f32", "u8"])
def test_query_equal_to_base_rows_and_ties(dtype):
    # queries that are base rows (distance 0, nothing excluded) and base rows
    # with exact twins (ties to the lower index)
    rng = np.random.default_rng(6)
    base = rng.integers(0, 256, size=(300, 48))
    X = np.concatenate([base, base[:50]])
    Q = np.concatenate([base[::7], rng.integers(0, 256, size=(20, 48))])
    cast = (lambda a: a.astype(np.float32)) if dtype == "f32" else (lambda a: a.astype(np.uint8))
    X, Q = cast(X), cast(Q)
    ref = oracle.knn_query(Q, X, 4)
    assert np.array_equal(ref[:43, 0], np.arange(0, 300, 7))
    for method in ("tensor_cores", "cuda_cores"):
        got = ivhd.knn_query(torch.from_numpy(Q).cuda(), torch.from_numpy(X).cuda(), 4,
                             method=method)
        assert np.array_equal(got.cpu().numpy(), ref), method


@pytest.mark.parametrize("k", [1, 8, 32])
@pytest.mark.parametrize("dtype", ["f32", "u8"])
def test_short_query_set_split_into_column_segments(dtype, k):
    # 64 queries against 40,000 base rows: one row block, so the columns are
    # split into 32 segments whose lists are merged per row
    if dtype == "f32":
        Q, X = split_gmm(64, 40_000, 24, 3)
    else:
        Z, _ = synth.mnist_like(40_064, 9, N=96)
        Q, X = Z[:64], Z[64:]
    got = ivhd.knn_query(torch.from_numpy(Q).cuda(), torch.from_numpy(X).cuda(), k,
                         method="tensor_cores")
    assert np.array_equal(got.cpu().numpy(), oracle.knn_query(Q, X, k))


def test_query_uncertified_rows_are_recomputed():
    Q, X = split_gmm(500, 1200, 20, 5, offset=3000.0)
    got, st = ivhd.knn_query(torch.from_numpy(Q).cuda(), torch.from_numpy(X).cuda(), 5,
                             method="tensor_cores", return_stats=True)
    assert st["fallback_rows"] > 0
    assert np.array_equal(got.cpu().numpy(), oracle.knn_query(Q, X, 5))


def test_query_uncertified_rows_in_column_segments():
    Q, X = split_gmm(300, 20_000, 20, 6, offset=3000.0)
    got, st = ivhd.knn_query(torch.from_numpy(Q).cuda(), torch.from_numpy(X).cuda(), 7,
                             method="tensor_cores", return_stats=True)
    assert st["fallback_rows"] > 10
    assert np.array_equal(got.cpu().numpy(), oracle.knn_query(Q, X, 7))


@pytest.mark.parametrize("dtype", ["f32", "u8"])
def test_index_queries_equal_single_queries(dtype):
    if dtype == "f32":
        Q, X = split_gmm(900, 5000, 40, 12)
    else:
        Z, _ = synth.mnist_like(5900, 13, N=200)
        Q, X = Z[:900], Z[900:]
    Qd, Xd = torch.from_numpy(Q).cuda(), torch.from_numpy(X).cuda()
    idx = ivhd.KnnIndex(Xd)
    Xd.zero_()                                  # the index holds its own copy
    for method in ("tensor_cores", "cuda_cores"):
        for lo, hi, k in ((0, 900, 5), (0, 64, 1), (300, 900, 20)):
            got = idx.query(Qd[lo:hi], k, method=method).cpu().numpy()
            assert np.array_equal(got, oracle.knn_query(Q[lo:hi], X, k)), (method, lo, k)
    with pytest.raises(IvhdError):
        idx.query(Qd, 5001)
    idx.close()


def test_query_edge_sizes_and_errors():
    Q, X = split_gmm(40, 64, 16, 2)
    Qd, Xd = torch.from_numpy(Q).cuda(), torch.from_numpy(X).cuda()
    # k = M lists the whole base set (CUDA cores; the tensor-core lists hold 32)
    got = ivhd.knn_query(Qd, Xd, 64)
    assert np.array_equal(got.cpu().numpy(), oracle.knn_query(Q, X, 64))
    one = ivhd.knn_query(Qd, Xd[:1], 1)                    # a base set of one row
    assert torch.all(one == 0)
    with pytest.raises(IvhdError):
        ivhd.knn_query(Qd, Xd, 65)                         # k > M
    with pytest.raises(IvhdError):
        ivhd.knn_query(Qd, Xd, 33, method="tensor_cores")  # beyond the candidate lists


def test_knn_query_full_size_sampled_rows():
    # the warm-start workload's shape: 200,000 uint8 base images of 784 pixels
    # and 100,000 new ones (the held-out set is 1.4e6; same kernel, more rows)
    Z, _ = synth.mnist_like(300_000, 11)
    X, Q = Z[:200_000], Z[200_000:]
    got = ivhd.knn_query(torch.from_numpy(Q).cuda(), torch.from_numpy(X).cuda(), 5).cpu().numpy()
    rows = np.random.default_rng(1).choice(Q.shape[0], 12, replace=False)
    assert np.array_equal(got[rows], oracle.knn_query(Q[rows], X, 5))


@pytest.mark.parametrize("k", [1, 3, 10])
def test_place_nn_matches_oracle(k):
    rng = np.random.default_rng(k)
    Y = rng.normal(size=(5000, 2)).astype(np.float32) * 3
    ids = rng.integers(0, 5000, size=(1234, k)).astype(np.int32)
    got = ivhd.place_nn(torch.from_numpy(Y).cuda(), torch.from_numpy(ids).cuda()).cpu().numpy()
    ref = oracle.place_nn(Y, ids)
    if k == 1:
        assert np.array_equal(got, Y[ids[:, 0]])
    assert np.abs(got - ref).max() <= 1e-6 * np.abs(Y).max()


def test_place_nn_rejects_bad_ids_and_accepts_empty():
    Y = torch.zeros((10, 2), device="cuda")
    assert ivhd.place_nn(Y, torch.zeros((0, 3), dtype=torch.int32, device="cuda")).shape == (0, 2)
    for bad in (10, -1):
        ids = torch.tensor([[1, 2], [3, bad]], dtype=torch.int32, device="cuda")
        with pytest.raises(IvhdError) as ex:
            ivhd.place_nn(Y, ids)
        assert ex.value.status == -2
