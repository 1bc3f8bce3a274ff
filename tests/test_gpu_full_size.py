"""Parity at the benchmark's full sizes, in the configuration bench.py times.

kNN graphs are checked on sampled rows that the oracle computes one by one.
The embedding step is checked element by element on a 1.4e6-vertex
kNN-shaped graph from the input generators (the oracle never receives a
graph built by the CUDA path).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2303_05455_gb300 import ivhd, synth
from step_bounds import close_elem, force_error_bound, step_bound

pytestmark = pytest.mark.gpu


def close(got, ref, rtol=1e-5):
    err = np.abs(np.asarray(got, np.float64) - ref).max()
    assert err <= rtol * np.abs(ref).max(), (err, np.abs(ref).max())


def test_knn_gmm1p4m_sampled_rows():
    w = synth.WORKLOADS["gmm1p4m"]
    X, _ = synth.workload_features(w)
    knn = ivhd.knn_build(torch.from_numpy(X).cuda(), w.k).cpu().numpy()
    rows = synth.sample_rows(w.M, 24, 5)
    rows[0], rows[-1] = 0, w.M - 1       # first and last query tile (ragged tail)
    assert np.array_equal(knn[rows], oracle.knn_f32(X, w.k, rows))
    assert knn.min() >= 0 and knn.max() < w.M
    assert not np.any(knn == np.arange(w.M)[:, None])


def test_knn_mnist70k_sampled_rows():
    w = synth.WORKLOADS["mnist70k"]
    X, _ = synth.workload_features(w)
    knn = ivhd.knn_build(torch.from_numpy(X).cuda(), w.k).cpu().numpy()
    rows = synth.sample_rows(w.M, 150, 6)
    rows[-1] = w.M - 1
    assert np.array_equal(knn[rows], oracle.knn_u8(X, w.k, rows))


@pytest.mark.parametrize("opt", ["momentum", "adadelta"])
def test_steps_at_full_size(opt):
    w = synth.WORKLOADS["gmm1p4m"]
    knn = synth.random_knn_graph(w.M, w.k, 77, hub_frac=0.02, n_hubs=1400)
    emb = ivhd.Embedding(torch.from_numpy(knn).cuda(), r=w.r, c=w.c, opt=opt, a=w.a, b=w.b,
                         seed=w.seed)
    rn, _ = oracle.random_neighbors(knn, w.r, w.seed)
    assert np.array_equal(emb.random_neighbors(), rn)
    terms = oracle.build_terms(knn, rn)
    assert emb.info()["n_terms"] == terms.T
    y0 = emb.positions(host=True)
    assert np.array_equal(y0, oracle.init_positions(w.M, w.seed).astype(np.float32))
    oid = oracle.OPT_MOMENTUM if opt == "momentum" else oracle.OPT_ADADELTA
    st = oracle.State.fresh(y0)
    F0 = oracle.forces(y0, terms, w.c)
    emb.step(1)
    oracle.step(st, terms, w.c, oid, a=w.a, b=w.b)
    y1 = emb.positions(host=True)
    close(y1, st.Y)
    d_ref = st.Y - y0     # the displacement of the step, element by element at its own scale
    close_elem(y1 - y0, d_ref,
               step_bound(opt, st.Y, d_ref, F0, force_error_bound(y0, terms, w.c), w.a, w.b),
               "displacement")
    emb.step(4)
    oracle.run(st, terms, w.c, 4, oid, a=w.a, b=w.b)
    close(emb.positions(host=True), st.Y)
    y5 = emb.positions(host=True).astype(np.float64)
    close(emb.forces(host=True), oracle.forces(y5, terms, w.c))
    assert emb.stress() == pytest.approx(oracle.stress(y5, terms, w.c), rel=1e-5)
