"""Seeded random sweep of the GPU path against the FP64 oracle (``-m gpu``).

Thirty graphs with random sizes (including ragged slice tails), k, r, c, hub
structure, absent entries, multiplicity mode, optimiser, hub threshold, block
size and position format: random neighbours bit-exact, one step of positions
within 1e-5 relative (half-precision formats: given the same rounded gathered
positions, as in the precision tests, so only FP32 is compared here against
the oracle; the half formats are checked to stay finite and close), and the
kNN build on random features (float and uint8, both methods) bit-exact.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2303_05455_gb300 import ivhd, synth

pytestmark = pytest.mark.gpu

OPT = {"momentum": oracle.OPT_MOMENTUM, "nesterov": oracle.OPT_NESTEROV,
       "adadelta": oracle.OPT_ADADELTA}


def case(seed):
    rng = np.random.default_rng(1000 + seed)
    M = int(rng.choice([2, 3, 33, 95, 257, 1000, 2049, 4099]))
    k = int(rng.integers(1, min(M - 1, 8) + 1))
    hubs = M > 60 and rng.random() < 0.5
    knn = synth.random_knn_graph(M, k, seed, hub_frac=0.3 if hubs else 0.0,
                                 n_hubs=max(k + 1, M // 50) if hubs else 0)
    if rng.random() < 0.3 and k > 1:  # some absent entries (fewer than k neighbours)
        knn[rng.random(knn.shape) < 0.1] = -1
    r = int(rng.integers(0, 3))
    c = float(rng.choice([0.01, 0.1, 0.5]))
    opt = str(rng.choice(list(OPT)))
    params = dict(opt=opt, a=0.9, b=float(rng.choice([0.001, 0.01])), seed=int(rng.integers(1 << 31)),
                  dedup_mutual=bool(rng.random() < 0.5),
                  hub_threshold=int(rng.choice([0, 1, 16, 128])),
                  block_size=int(rng.choice([0, 128, 256, 512])))
    params["vertices_per_warp"] = int(rng.choice([0, 1, 2, 4, 8]))
    return knn, r, c, params


@pytest.mark.parametrize("seed", range(30))
def test_random_case_matches_oracle(seed):
    knn, r, c, p = case(seed)
    emb = ivhd.Embedding(knn, r=r, c=c, **p)
    rn, empty = oracle.random_neighbors(knn, r, p["seed"])
    assert np.array_equal(emb.random_neighbors(), rn)
    terms = oracle.build_terms(knn, rn, dedup=p["dedup_mutual"])
    assert emb.info()["n_terms"] == terms.T
    y0 = emb.positions(host=True).astype(np.float64)
    st = oracle.State.fresh(y0)
    emb.step(3)
    oracle.run(st, terms, c, 3, OPT[p["opt"]], a=p["a"], b=p["b"])
    got = emb.positions(host=True).astype(np.float64)
    scale = max(np.abs(st.Y).max(), 1e-30)
    assert np.abs(got - st.Y).max() <= 1e-5 * scale
    emb.close()
    for fmt in ("f16", "bf16"):
        e = ivhd.Embedding(knn, r=r, c=c, pos_format=fmt, **p)
        e.step(3)
        y = e.positions(host=True).astype(np.float64)
        assert np.all(np.isfinite(y))
        assert np.abs(y - got).max() <= 0.05 * scale + 1e-3
        e.close()


@pytest.mark.parametrize("seed", range(8))
def test_random_knn_both_methods_bit_exact(seed):
    rng = np.random.default_rng(seed)
    M = int(rng.integers(40, 1500))
    k = int(rng.integers(1, min(M - 1, 32) + 1))
    if seed % 2 == 0:
        N = int(rng.integers(1, 130))
        X = rng.standard_normal((M, N)).astype(np.float32) * np.float32(rng.choice([1, 10, 100]))
        ref = oracle.knn_f32(X, k)
    else:
        N = int(rng.integers(1, 1025))
        X = rng.integers(0, 256, size=(M, N)).astype(np.uint8)
        ref = oracle.knn_u8(X, k)
    Xd = torch.from_numpy(X).cuda()
    for method in ("tensor_cores", "cuda_cores"):
        assert np.array_equal(ivhd.knn_build(Xd, k, method=method).cpu().numpy(), ref), method
