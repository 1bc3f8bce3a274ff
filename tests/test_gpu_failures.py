"""Failure paths without a GPU fault (``-m gpu``).

A device-side wait that nothing completes ends with IVHD_ERR_TIMEOUT after its
poll limit and leaves the library usable.  Allocation failures are injected
on the host (ivhd_test_fail_alloc) at every allocation an entry point makes:
each one surfaces as IVHD_ERR_OOM, frees everything the call had taken
(ivhd_test_live_allocs returns to its value before the call), and the next
call succeeds.
"""
import numpy as np
import pytest
import torch

from paper_2303_05455_gb300 import _lib, ivhd, synth
from paper_2303_05455_gb300._lib import IvhdError

pytestmark = pytest.mark.gpu

OOM = -3


@pytest.fixture
def L():
    lib = _lib.load()
    lib.ivhd_test_fail_alloc(-1)
    yield lib
    lib.ivhd_test_fail_alloc(-1)


def live(L):
    torch.cuda.synchronize()
    return L.ivhd_test_live_allocs()


def test_wait_timeout_returns_status_and_library_stays_usable(L):
    s = torch.cuda.current_stream().cuda_stream
    assert L.ivhd_probe_wait_timeout(0, s) == -1
    for polls in (1, 1000, 100000):
        assert L.ivhd_probe_wait_timeout(polls, s) == -6
    emb = ivhd.Embedding(synth.random_knn_graph(500, 3, 2), r=1, c=0.1, seed=1)
    emb.step(10)
    assert np.all(np.isfinite(emb.positions(host=True)))
    emb.close()


def test_grid_barrier_timeout_returns_status_and_library_stays_usable(L):
    s = torch.cuda.current_stream().cuda_stream
    for polls in (1, 1000, 100000):
        assert L.ivhd_probe_grid_barrier_timeout(polls, s) == -6
    emb = ivhd.Embedding(synth.random_knn_graph(3000, 3, 2), r=1, c=0.1, seed=1, resident="grid")
    emb.step(20)
    assert np.all(np.isfinite(emb.positions(host=True)))
    emb.close()


def test_knn_index_frees_everything_on_allocation_failure(L):
    X = torch.randn(3000, 24, generator=torch.Generator().manual_seed(4)).cuda()
    Q = X[:500].contiguous()
    base = live(L)

    def one():
        idx = ivhd.KnnIndex(X)
        try:
            idx.query(Q, 5)
        finally:
            idx.close()

    n = _each_failure(L, one)
    assert n >= 3
    assert live(L) == base


def _each_failure(L, call, limit=400):
    """Runs call() with the n-th allocation failing, n = 0, 1, ... until call()
    completes without reaching the injected failure; returns that n."""
    for n in range(limit):
        before = live(L)
        L.ivhd_test_fail_alloc(n)
        try:
            call()
        except IvhdError as e:
            assert e.status == OOM, (n, e)
            L.ivhd_test_fail_alloc(-1)
            assert live(L) == before, n
            continue
        L.ivhd_test_fail_alloc(-1)
        return n
    raise AssertionError("no successful call")


def test_create_and_batch_create_free_everything_on_allocation_failure(L):
    knn = synth.random_knn_graph(3000, 5, 3, hub_frac=0.2, n_hubs=10)
    base = live(L)

    def one():
        emb = ivhd.Embedding(knn, r=2, c=0.05, seed=4, opt="adadelta")
        try:
            emb.step(70)
            emb.stress()
            emb.positions(host=True)
        finally:
            emb.close()

    n = _each_failure(L, one)
    assert n > 10
    assert live(L) == base

    graphs = [synth.random_knn_graph(m, 3, m) for m in (300, 700, 50)]

    def batch():
        emb = ivhd.Embedding.batch(graphs, r=1, seeds=7, c=0.1, adaptive=True)
        try:
            emb.step(5)
            emb.resample_random_neighbors(3)
        finally:
            emb.close()

    assert _each_failure(L, batch) > 10
    assert live(L) == base
    emb = ivhd.Embedding(knn, r=2, c=0.05, seed=4)  # the library still works
    emb.step(3)
    emb.close()
    assert live(L) == base


@pytest.mark.parametrize("dtype", ["f32", "u8"])
def test_knn_build_frees_everything_on_allocation_failure(L, dtype):
    if dtype == "f32":
        X = torch.from_numpy(synth.gaussian_mixture(900, 24, 5, 1)[0]).cuda()
    else:
        X = torch.from_numpy(synth.mnist_like(900, 1, N=64)[0]).cuda()
    base = live(L)
    ref = ivhd.knn_build(X, 5)
    assert _each_failure(L, lambda: ivhd.knn_build(X, 5)) >= 2
    assert torch.equal(ivhd.knn_build(X, 5), ref)
    assert live(L) == base


def test_mlp_frees_everything_on_allocation_failure(L):
    x = torch.randint(0, 256, (256, 784), dtype=torch.uint8, device="cuda")
    t = torch.randn(256, 2, device="cuda")
    base = live(L)

    def run():
        net = ivhd.MLP(784, 512, max_batch=256)
        try:
            net.init_params(1)
            net.train_step(x, t, x_scale=1 / 255)
            net.forward(x, x_scale=1 / 255)
        finally:
            net.close()

    assert _each_failure(L, run) > 5
    assert live(L) == base


def test_eval_rejects_sampled_row_ids_out_of_range(L):
    """A row id outside [0, M) is reported as IVHD_ERR_INDEX, never dereferenced."""
    M, k = 2000, 3
    knn = torch.from_numpy(synth.random_knn_graph(M, k, 5)).cuda()
    Y = torch.from_numpy(synth.uniform_positions(M, 6)).cuda()
    lab = torch.arange(M, dtype=torch.int32, device="cuda") % 5
    for bad in (M, -1, 1 << 40):
        rows = torch.arange(300, dtype=torch.int64, device="cuda")
        rows[211] = bad
        with pytest.raises(IvhdError) as e:
            ivhd.eval_qnx(Y, knn, rows)
        assert e.value.status == -2
        with pytest.raises(IvhdError) as e:
            ivhd.eval_cf(Y, lab, 10, rows)
        assert e.value.status == -2
    rows = torch.arange(300, dtype=torch.int64, device="cuda")
    assert 0.0 <= ivhd.eval_qnx(Y, knn, rows) <= 1.0
