"""Many embeddings in one context (one launch per step) and the launch-shape autotuner."""
import numpy as np
import pytest

import oracle
from paper_2303_05455_gb300 import ivhd, synth

pytestmark = pytest.mark.gpu

SPECS = [  # (M, k, r, seed)
    (300, 2, 1, 11), (1000, 3, 2, 12), (37, 5, 0, 13), (2000, 2, 1, 14), (513, 4, 2, 15),
]


def graphs():
    out = []
    for M, k, r, s in SPECS:
        X, _ = synth.gaussian_mixture(M, 12, 3, s)
        out.append(oracle.knn_f32(X, k))
    return out


def close(got, ref, rtol=1e-5):
    err = np.abs(np.asarray(got, np.float64) - ref).max()
    assert err <= rtol * np.abs(ref).max(), (err, np.abs(ref).max())


def test_batch_matches_independent_oracle_runs():
    gs = graphs()
    a, b, c = 0.9, 0.01, 0.05
    emb = ivhd.Embedding.batch(gs, r=[s[2] for s in SPECS], seeds=[s[3] for s in SPECS], c=c,
                               a=a, b=b)
    lo = np.concatenate([[0], np.cumsum([s[0] for s in SPECS])])
    rn_all = emb.random_neighbors()
    y0 = emb.positions(host=True)
    states, terms = [], []
    E = 0.0
    for e, (M, k, r, s) in enumerate(SPECS):
        rows = rn_all[lo[e]:lo[e + 1]]
        rn_ref, _ = oracle.random_neighbors(gs[e], r, s)
        local = np.where(rows[:, :r] >= 0, rows[:, :r] - lo[e], -1)
        assert np.array_equal(local, rn_ref)
        assert np.all(rows[:, r:] == -1)
        assert np.array_equal(y0[lo[e]:lo[e + 1]], oracle.init_positions(M, s).astype(np.float32))
        t = oracle.build_terms(gs[e], rn_ref)
        terms.append(t)
        states.append(oracle.State.fresh(oracle.init_positions(M, s)))
        E += oracle.stress(states[-1].Y, t, c)
    assert emb.info()["n_terms"] == sum(t.T for t in terms)
    assert emb.stress() == pytest.approx(E, rel=1e-5)
    for n in (1, 9):
        emb.step(n)
        y = emb.positions(host=True)
        for e in range(len(SPECS)):
            oracle.run(states[e], terms[e], c, n, a=a, b=b)
            close(y[lo[e]:lo[e + 1]], states[e].Y)


def test_batch_equals_separate_contexts_and_autotune_keeps_state():
    gs = graphs()
    rs = [s[2] for s in SPECS]
    sd = [s[3] for s in SPECS]
    emb = ivhd.Embedding.batch(gs, r=rs, seeds=sd, c=0.05, pos_format="bf16")
    emb.step(30)
    y = emb.positions(host=True)
    lo = np.concatenate([[0], np.cumsum([s[0] for s in SPECS])])
    for e, g in enumerate(gs):
        one = ivhd.Embedding(g, r=rs[e], c=0.05, seed=sd[e], pos_format="bf16")
        one.step(30)
        close(y[lo[e]:lo[e + 1]], one.positions(host=True).astype(np.float64), rtol=1e-4)
    before = emb.positions(host=True)
    cfg = emb.autotune(trial_steps=5)
    assert cfg["block"] in (128, 256, 512) and cfg["hub_threshold"] in (16, 32, 64, 128, 256, 512)
    assert cfg["vertices_per_warp"] in (1, 2, 4, 8) and cfg["us_per_step"] > 0
    assert np.array_equal(emb.positions(host=True), before)
    assert emb.info()["steps_done"] == 30
    emb.step(64)  # graph replay with the tuned shape
    assert np.all(np.isfinite(emb.positions(host=True)))


@pytest.mark.parametrize("opt", ["momentum", "adadelta"])
def test_autotuned_single_embedding_keeps_parity(opt):
    knn = synth.random_knn_graph(20000, 5, 3, hub_frac=0.05, n_hubs=200)
    emb = ivhd.Embedding(knn, r=1, c=0.01, opt=opt, b=0.002, seed=1)
    rn, _ = oracle.random_neighbors(knn, 1, 1)
    t = oracle.build_terms(knn, rn)
    st = oracle.State.fresh(oracle.init_positions(20000, 1))
    oid = oracle.OPT_MOMENTUM if opt == "momentum" else oracle.OPT_ADADELTA
    emb.step(3)
    oracle.run(st, t, 0.01, 3, oid, b=0.002)
    emb.autotune(trial_steps=3)
    emb.step(7)
    oracle.run(st, t, 0.01, 7, oid, b=0.002)
    close(emb.positions(host=True), st.Y)
