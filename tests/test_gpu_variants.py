"""Paper variants of the iteration (Sec. 3.3.3, 3.4) on the GPU vs the FP64 oracle.

L1 late stage, random-neighbour redraws, the reverse-neighbour restriction,
the self-adaptive b controller, and kNN rows with absent entries.  Same
tolerances as the core parity tests (1e-5 relative on forces and positions,
exact on integer outputs and on the controller's accept/reject decisions).
"""
import numpy as np
import pytest

import oracle
from paper_2303_05455_gb300 import ivhd, synth

pytestmark = pytest.mark.gpu


def close(got, ref, rtol=1e-5):
    got = np.asarray(got, np.float64)
    err = np.abs(got - ref).max()
    assert err <= rtol * np.abs(ref).max(), (err, np.abs(ref).max())


def hub_graph():
    return synth.random_knn_graph(5000, 5, 21, hub_frac=0.3, n_hubs=20), 2, 0.05


@pytest.mark.parametrize("opt", ["momentum", "nesterov"])
def test_l1_late_stage(opt):
    knn, r, c = hub_graph()
    a, b = 0.9, 0.01
    emb = ivhd.Embedding(knn, r=r, c=c, opt=opt, a=a, b=b, seed=4, init_uniform=False)
    y0 = synth.uniform_positions(5000, 2, scale=4.0)
    emb.set_positions(y0)
    rn, _ = oracle.random_neighbors(knn, r, 4)
    t = oracle.build_terms(knn, rn)
    emb.set_metric("l1")
    y64 = y0.astype(np.float64)
    close(emb.forces(host=True), oracle.forces(y64, t, c, metric="l1"))
    assert emb.stress() == pytest.approx(oracle.stress(y64, t, c, "l1"), rel=1e-5)
    st = oracle.State.fresh(y0)
    oid = oracle.OPT_MOMENTUM if opt == "momentum" else oracle.OPT_NESTEROV
    for n in (1, 4):
        emb.step(n)
        for _ in range(n):
            oracle.step_l1(st, t, c, oid, a=a, b=b)
        close(emb.positions(host=True), st.Y)
    emb.set_metric("l2")
    y5 = emb.positions(host=True).astype(np.float64)
    close(emb.forces(host=True), oracle.forces(y5, t, c))


def test_random_neighbour_redraw_keeps_state():
    w = synth.WORKLOADS["gmm2k"]
    X, _ = synth.workload_features(w)
    knn = oracle.knn_f32(X, w.k)
    emb = ivhd.Embedding(knn, r=2, c=w.c, a=w.a, b=w.b, seed=w.seed)
    rn0, _ = oracle.random_neighbors(knn, 2, w.seed)
    t0 = oracle.build_terms(knn, rn0)
    st = oracle.State.fresh(oracle.init_positions(w.M, w.seed))
    emb.step(10)
    oracle.run(st, t0, w.c, 10, a=w.a, b=w.b)
    y10 = emb.positions(host=True)
    emb.resample_random_neighbors(7)
    assert np.array_equal(emb.positions(host=True), y10)        # the rebuild moves nothing
    rn7, _ = oracle.random_neighbors(knn, 2, w.seed, epoch=7)
    assert np.array_equal(emb.random_neighbors(), rn7)
    t7 = oracle.build_terms(knn, rn7)
    assert emb.info()["n_terms"] == t7.T
    close(emb.forces(host=True), oracle.forces(y10.astype(np.float64), t7, w.c))
    emb.step(70)                                                  # graph replay + tail
    oracle.run(st, t7, w.c, 70, a=w.a, b=w.b)
    close(emb.positions(host=True), st.Y)
    emb.resample_random_neighbors(0)                              # epoch 0 = the first draw
    assert np.array_equal(emb.random_neighbors(), rn0)


def test_reverse_neighbour_restriction_and_restore():
    w = synth.WORKLOADS["gmm2k"]
    X, _ = synth.workload_features(w)
    knn = oracle.knn_f32(X, w.k)
    helper = oracle.knn_f32(X, 4 * w.k)
    emb = ivhd.Embedding(knn, r=w.r, c=w.c, a=w.a, b=w.b, seed=w.seed)
    rn, _ = oracle.random_neighbors(knn, w.r, w.seed)
    t_full = oracle.build_terms(knn, rn)
    st = oracle.State.fresh(oracle.init_positions(w.M, w.seed))
    emb.step(20)
    oracle.run(st, t_full, w.c, 20, a=w.a, b=w.b)
    emb.restrict_nn(helper)
    kr = oracle.restrict(knn, helper)
    t_r = oracle.build_terms(kr, rn)
    assert (kr < 0).any() and emb.info()["n_terms"] == t_r.T < t_full.T
    assert np.array_equal(emb.random_neighbors(), rn)
    close(emb.forces(host=True), oracle.forces(emb.positions(host=True).astype(np.float64), t_r, w.c))
    emb.step(10)
    oracle.run(st, t_r, w.c, 10, a=w.a, b=w.b)
    close(emb.positions(host=True), st.Y)
    emb.restrict_nn(None)
    assert emb.info()["n_terms"] == t_full.T
    bad = helper.copy()
    bad[3, 0] = w.M
    with pytest.raises(ivhd.IvhdError) as e:
        emb.restrict_nn(bad)
    assert e.value.status == -2
    assert emb.info()["n_terms"] == t_full.T


@pytest.mark.parametrize("opt", ["momentum", "nesterov"])
def test_adaptive_b_controller(opt):
    w = synth.WORKLOADS["gmm2k"]
    X, _ = synth.workload_features(w)
    knn = oracle.knn_f32(X, w.k)
    b0, tau, g1, g2 = 0.05, 0.5, 1.1, 0.5
    emb = ivhd.Embedding(knn, r=w.r, c=w.c, opt=opt, a=w.a, b=b0, seed=w.seed, adaptive=True,
                         tau=tau, gamma1=g1, gamma2=g2)
    rn, _ = oracle.random_neighbors(knn, w.r, w.seed)
    t = oracle.build_terms(knn, rn)
    st = oracle.State.fresh(oracle.init_positions(w.M, w.seed))
    oid = oracle.OPT_MOMENTUM if opt == "momentum" else oracle.OPT_NESTEROV
    box = [b0]
    acc = rej = 0
    for _ in range(40):
        emb.step(1)
        ok = oracle.step_adaptive(st, t, w.c, box, oid, a=w.a, tau=tau, gamma1=g1, gamma2=g2)
        acc += ok
        rej += not ok
        s = emb.adaptive_state()
        assert (s["accepted"], s["rejected"]) == (acc, rej)
        assert s["b"] == pytest.approx(box[0], rel=1e-6)
    assert rej > 0 and acc > 0
    close(emb.positions(host=True), st.Y)


def test_adaptive_graph_replay_equals_single_steps():
    knn, r, c = hub_graph()
    a = ivhd.Embedding(knn, r=r, c=c, b=0.02, seed=3, adaptive=True)
    b = ivhd.Embedding(knn, r=r, c=c, b=0.02, seed=3, adaptive=True)
    a.step(130)
    for _ in range(130):
        b.step(1)
    assert np.array_equal(a.positions(host=True), b.positions(host=True))
    assert a.adaptive_state() == b.adaptive_state()
    state = a.get_state()
    a.step(20)
    b.set_state(state)
    b.step(20)
    assert np.array_equal(a.positions(host=True), b.positions(host=True))


def test_absent_knn_entries():
    knn = synth.random_knn_graph(3000, 6, 5)
    rng = np.random.default_rng(1)
    knn[rng.random(knn.shape) < 0.3] = -1                        # vertices with fewer neighbours
    knn[7] = -1                                                  # and one with none
    emb = ivhd.Embedding(knn, r=2, c=0.1, seed=8)
    rn, _ = oracle.random_neighbors(knn, 2, 8)
    assert np.array_equal(emb.random_neighbors(), rn)
    t = oracle.build_terms(knn, rn)
    assert emb.info()["n_terms"] == t.T
    y0 = emb.positions(host=True).astype(np.float64)
    close(emb.forces(host=True), oracle.forces(y0, t, 0.1))
    st = oracle.State.fresh(y0)
    emb.step(3)
    oracle.run(st, t, 0.1, 3)
    close(emb.positions(host=True), st.Y)
