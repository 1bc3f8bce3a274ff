"""Resident whole-run kernel vs one launch per step (``-m gpu``).

Small embeddings run all steps of an ivhd_step call in one single-block
launch with positions and optimiser state in shared memory (and the id rows
too when they fit).  Its traversal and arithmetic are those of the step
kernel, so positions and optimiser state must agree bit for bit with the
multi-launch path, for every optimiser and both metrics, with the id rows in
shared memory (2,000-vertex mixture) and read through L1 (5,000-vertex hub
graph).
"""
import numpy as np
import pytest

import oracle
from paper_2303_05455_gb300 import ivhd, synth

pytestmark = pytest.mark.gpu


def graphs():
    w = synth.WORKLOADS["gmm2k"]
    X, _ = synth.workload_features(w)
    return {"gmm2k": (oracle.knn_f32(X, w.k), w.r, w.c),
            "hubs5k": (synth.random_knn_graph(5000, 5, 21, hub_frac=0.3, n_hubs=20), 2, 0.05),
            "pair": (np.array([[1], [0]], np.int32), 1, 0.1),
            "ragged37": (synth.random_knn_graph(37, 3, 4), 1, 0.1)}


GRAPHS = graphs()


@pytest.mark.parametrize("vpw", [1, 4])
@pytest.mark.parametrize("kind", [True, "cluster", "grid"])
@pytest.mark.parametrize("name", sorted(GRAPHS))
@pytest.mark.parametrize("opt", ["momentum", "nesterov", "adadelta"])
@pytest.mark.parametrize("metric", ["l2", "l1"])
def test_resident_equals_multi_launch_bitwise(name, opt, metric, kind, vpw):
    knn, r, c = GRAPHS[name]
    runs = []
    for resident in (kind, False):
        e = ivhd.Embedding(knn, r=r, c=c, opt=opt, b=0.002, seed=9, resident=resident,
                           hub_threshold=16, vertices_per_warp=vpw)
        if metric == "l1":
            e.set_metric("l1")
        out = []
        for n in (1, 7, 64, 130):
            e.step(n)
            out.append(e.positions(host=True))
        st = e.get_state()
        runs.append((out, st, e.info()))
        e.close()
    (pa, sa, ia), (pb, sb, ib) = runs
    for x, y in zip(pa, pb):
        assert np.array_equal(x, y)
    assert sa == sb
    assert ia["steps_done"] == ib["steps_done"] == 202
    assert ia["kernel_launches"] == 4 and ib["kernel_launches"] == 202


def test_resident_not_used_for_rows_of_512_entries_or_more():
    # the whole-call kernels give a row at most a warp; such graphs run one step
    # kernel per step (and the persistent grid), with equal results
    M = 3000
    knn = synth.random_knn_graph(M, 3, 12)
    knn[1:, 0] = 0                         # vertex 0: a neighbour of every other vertex
    knn[0] = [1, 2, 3]
    bad = (knn[:, 1] == 0) | (knn[:, 2] == 0) | (knn[:, 1] == knn[:, 2])
    knn[bad, 1], knn[bad, 2] = (np.arange(M)[bad] + 1) % M, (np.arange(M)[bad] + 2) % M
    knn[0] = [1, 2, 3]
    runs = []
    for resident in (True, "cluster", "grid", False):
        e = ivhd.Embedding(knn, r=1, c=0.02, seed=3, b=5e-4, resident=resident)
        e.step(40)
        runs.append((e.positions(host=True), e.info()))
        e.close()
    for (y, inf), resident in zip(runs, (True, "cluster", "grid", False)):
        assert np.array_equal(y, runs[-1][0])
        assert inf["launch_form"] == (3 if resident == "grid" else 0)


def test_resident_not_used_when_state_does_not_fit_or_not_asked():
    knn = synth.random_knn_graph(20000, 5, 3)
    e = ivhd.Embedding(knn, r=1, c=0.01, seed=1, resident=True)
    e.step(10)
    assert e.info()["kernel_launches"] == 10
    e.close()
    small = synth.random_knn_graph(4000, 5, 4)  # ~46k entries: above the automatic limit
    e = ivhd.Embedding(small, r=1, c=0.01, seed=1)
    e.step(10)
    assert e.info()["nnz_sym"] > 40000 and e.info()["kernel_launches"] == 10
    e.close()
    tiny = synth.random_knn_graph(1000, 3, 4)  # automatic: the cluster kernel
    e = ivhd.Embedding(tiny, r=1, c=0.01, seed=1)
    e.step(10)
    assert e.info()["kernel_launches"] == 1
    e.close()
    e = ivhd.Embedding(tiny, r=1, c=0.01, seed=1, resident=False)
    e.step(10)
    assert e.info()["kernel_launches"] == 10
    e.close()
    e = ivhd.Embedding(small, r=1, c=0.01, seed=1, resident=True, adaptive=True)
    e.step(10)
    assert e.info()["kernel_launches"] == 20  # step kernel + controller per step
    e.close()


@pytest.mark.parametrize("opt", ["momentum", "adadelta"])
def test_persistent_grid_with_several_step_blocks_per_block(opt):
    # 300,000 vertices: more step-grid blocks than resident blocks, so every
    # resident block takes several; the positions must equal the multi-launch
    # path bit for bit
    knn = synth.random_knn_graph(300_000, 5, 8, hub_frac=0.02, n_hubs=300)
    out = []
    for resident in ("grid", False):
        e = ivhd.Embedding(knn, r=1, c=0.01, opt=opt, b=0.001, seed=2, resident=resident)
        e.step(3)
        e.step(40)
        out.append((e.positions(host=True), e.info()["kernel_launches"]))
        e.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1] == 2 and out[1][1] == 43
