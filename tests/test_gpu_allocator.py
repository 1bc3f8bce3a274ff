"""ivhd_set_allocator on the GPU (``-m gpu``).

With PyTorch's caching allocator behind the library, an embedding, a kNN
build and a warm-start network step give results bitwise equal to those made
with the library's own pool; every block handed out is given back through the
allocator that made it (also after the setting changes while a context
lives); an allocator that fails or returns a misaligned block surfaces as
IVHD_ERR_OOM with nothing leaked.
"""
import numpy as np
import pytest
import torch

from paper_2303_05455_gb300 import _lib, ivhd, synth
from paper_2303_05455_gb300._lib import IvhdError

pytestmark = pytest.mark.gpu

OOM = -3


class Counting:
    """Torch's caching allocator with a record of what the library holds."""

    def __init__(self, fail_after=None, offset=0):
        self.held = {}          # address given to the library -> torch block
        self.n_alloc = 0
        self.n_free = 0
        self.fail_after = fail_after
        self.offset = offset
        self.streams = set()

    def alloc(self, nbytes, stream):
        if self.fail_after is not None and self.n_alloc >= self.fail_after:
            return 0
        base = torch.cuda.caching_allocator_alloc(nbytes + self.offset, None, stream)
        self.n_alloc += 1
        self.held[base + self.offset] = base
        self.streams.add(stream)
        return base + self.offset

    def free(self, ptr, nbytes, stream):
        torch.cuda.caching_allocator_delete(self.held.pop(ptr))
        self.n_free += 1


@pytest.fixture
def restore():
    yield
    ivhd.set_allocator()


def _embed(knn, steps):
    emb = ivhd.Embedding(knn, r=2, c=0.05, seed=9, opt="adadelta")
    try:
        emb.step(steps)
        return emb.positions(host=True), emb.stress()
    finally:
        emb.close()


def test_torch_allocator_gives_identical_embedding(restore):
    knn = synth.random_knn_graph(6000, 5, 11, hub_frac=0.2, n_hubs=12)
    y0, e0 = _embed(knn, 130)
    a = Counting()
    ivhd.set_allocator(a.alloc, a.free)
    before = torch.cuda.memory_allocated()
    emb = ivhd.Embedding(knn, r=2, c=0.05, seed=9, opt="adadelta")
    assert a.n_alloc > 5 and a.held
    assert torch.cuda.memory_allocated() > before      # the state lives in torch's pool
    emb.step(130)
    y1, e1 = emb.positions(host=True), emb.stress()
    emb.close()
    torch.cuda.synchronize()
    assert a.n_free == a.n_alloc and not a.held
    np.testing.assert_array_equal(y0, y1)
    assert e0 == e1


def test_use_torch_allocator_knn_and_mlp(restore):
    g = torch.Generator().manual_seed(3)
    X = torch.randn(3000, 40, generator=g).cuda()
    xb = torch.from_numpy(synth.mnist_like(512, 4)[0]).cuda()
    tb = torch.randn(512, 2, generator=g).cuda()

    def run():
        knn = ivhd.knn_build(X, 5)
        net = ivhd.MLP(784, 512, max_batch=512)
        net.init_params(2)
        loss = [net.train_step(xb, tb, x_scale=1 / 255, want_loss=True) for _ in range(3)]
        p = net.get_params()
        net.close()
        return knn, loss, p

    knn0, l0, p0 = run()
    ivhd.use_torch_allocator()
    before = torch.cuda.memory_allocated()
    knn1, l1, p1 = run()
    torch.cuda.synchronize()
    # everything but the returned graph went back to torch's pool
    assert 0 <= torch.cuda.memory_allocated() - before <= knn1.numel() * 4 + 1024
    assert torch.equal(knn0, knn1)
    assert l0 == l1
    np.testing.assert_array_equal(p0, p1)


def test_blocks_return_to_their_allocator_after_a_switch(restore):
    a = Counting()
    ivhd.set_allocator(a.alloc, a.free)
    emb = ivhd.Embedding(synth.random_knn_graph(2000, 3, 4), r=1, c=0.1, seed=1)
    ivhd.set_allocator()                     # later allocations: the library's pool
    emb.step(70)
    n = a.n_alloc
    emb.close()
    torch.cuda.synchronize()
    assert a.n_free == n and not a.held


@pytest.mark.parametrize("kind", ["fails", "misaligned"])
def test_failing_allocator_reports_oom_and_leaks_nothing(restore, kind):
    L = _lib.load()
    knn = synth.random_knn_graph(2000, 3, 5)
    base = L.ivhd_test_live_allocs()
    for n in (0, 1, 3, 7):
        a = Counting(fail_after=n) if kind == "fails" else Counting(offset=16)
        ivhd.set_allocator(a.alloc, a.free)
        with pytest.raises(IvhdError) as ex:
            ivhd.Embedding(knn, r=1, c=0.1, seed=2)
        assert ex.value.status == OOM
        torch.cuda.synchronize()
        assert not a.held and a.n_free == a.n_alloc
        assert L.ivhd_test_live_allocs() == base
        if kind == "misaligned":
            break
    ivhd.set_allocator()
    y, _ = _embed(knn, 10)                   # the library's pool still serves
    assert np.all(np.isfinite(y))
