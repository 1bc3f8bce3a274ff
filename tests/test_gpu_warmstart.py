"""What the learned warm start gains over IVHD from a random start (``-m gpu``).

A small instance of the warm-start workload: MNIST-shaped training points and
their IVHD embedding teach the MLP (the library's tensor-core forward and
backward kernels, Adam); the MLP then places a held-out set of the same
distribution, and IVHD refines from that placement.  Against plain IVHD from
the uniform random start on the same held-out kNN graph, the warm start must
reach a lower stress with a tenth of the steps, and end at the same kNN
precision (Q_NX(k) within 0.01) and class neighbourhood (cf_10 no worse than
0.01 below) after the same number of steps.  The nearest-neighbour placement
(each held-out point at the embedding of its nearest training point, the
Progressive UMAP initialisation of Sec. 2.4.3) is run beside it as the
comparator.
"""
import numpy as np
import pytest
import torch

from paper_2303_05455_gb300 import ivhd, synth

pytestmark = pytest.mark.gpu

K, R, C, A, B = 5, 1, 0.01, 0.9, 0.001
N_TRAIN = N_HOLD = 40000
STEPS = 1000


def _curve(knn, lab, rows, init=None, seed=13):
    e = ivhd.Embedding(knn, r=R, c=C, a=A, b=B, seed=seed, init_uniform=init is None)
    if init is not None:
        e.set_positions(init)
    out = {}
    done = 0
    for st in (0, 50, 100, 200, STEPS):
        e.step(st - done)
        done = st
        y = e.positions()
        out[st] = {"stress": e.stress(), "qnx": ivhd.eval_qnx(y, knn, rows),
                   "cf10": ivhd.eval_cf(y, lab, 10, rows)}
    e.close()
    return out


def test_warm_start_gains_over_random_start():
    dev = torch.device("cuda")
    Xtr, _ = synth.mnist_like(N_TRAIN, 7, noise_seed=1)
    Xtr_d = torch.from_numpy(Xtr).to(dev)
    knn_tr = ivhd.knn_build(Xtr_d, K)
    emb = ivhd.Embedding(knn_tr, r=R, c=C, a=A, b=B, seed=11)
    emb.step(STEPS)
    Ytr = emb.positions()
    emb.close()
    mu, sd = Ytr.mean(0), Ytr.std(0)
    T = ((Ytr - mu) / sd).contiguous()

    net = ivhd.MLP(784, 512, max_batch=4096)
    net.init_params(5)
    rng = np.random.Generator(np.random.PCG64(6))
    bs = 4096
    first = last = None
    for ep in range(8):
        perm = torch.from_numpy(rng.permutation(N_TRAIN)).to(dev)
        Xs, Ts = Xtr_d[perm].contiguous(), T[perm].contiguous()
        for bi in range(N_TRAIN // bs):
            sl = slice(bi * bs, (bi + 1) * bs)
            l = net.train_step(Xs[sl], Ts[sl], lr=1e-3, x_scale=1 / 255, want_loss=True)
            first = l if first is None else first
            last = l
    assert last < 0.5 * first

    Xh, Lh = synth.mnist_like(N_HOLD, 7, noise_seed=2)
    Xh_d = torch.from_numpy(Xh).to(dev)
    Yp = (net.forward(Xh_d, x_scale=1 / 255) * sd + mu).contiguous()
    net.close()
    # the comparator: each held-out point at the embedding of its nearest
    # training point (Progressive UMAP initialisation)
    Ynn = ivhd.place_nn(Ytr, ivhd.knn_query(Xh_d, Xtr_d, 1))
    knn_h = ivhd.knn_build(Xh_d, K)
    rows = torch.from_numpy(synth.sample_rows(N_HOLD, 5000, 9)).to(dev)
    lab = torch.from_numpy(Lh).to(dev)
    plain = _curve(knn_h, lab, rows)
    warm = _curve(knn_h, lab, rows, init=Yp)
    nn = _curve(knn_h, lab, rows, init=Ynn)
    # plain IVHD is the placement's fallback: a good placement is taken, a
    # non-finite or far worse one leaves the seeded uniform start in place
    e = ivhd.Embedding(knn_h, r=R, c=C, a=A, b=B, seed=13)
    y_uniform = e.positions(host=True)
    bad = Yp.clone()
    bad[7, 0] = float("nan")
    assert not e.warm_start(bad)
    assert np.array_equal(e.positions(host=True), y_uniform)
    assert not e.warm_start(Yp * 1e4)
    assert np.array_equal(e.positions(host=True), y_uniform)
    assert e.warm_start(Yp)
    assert np.allclose(e.positions(host=True), Yp.cpu().numpy())
    e.close()
    print({"plain": plain, "warm": warm, "nn_placement": nn, "loss": (first, last)})
    # both placements start far below the uniform start and keep the classes apart
    assert nn[0]["stress"] < 0.1 * plain[0]["stress"]
    assert nn[0]["cf10"] >= plain[STEPS]["cf10"] - 0.01
    # a tenth of the steps reaches a lower stress than plain IVHD after all of them
    assert warm[STEPS // 10]["stress"] < plain[STEPS]["stress"]
    # the placement alone already keeps the classes apart as well as the full plain run
    assert warm[0]["cf10"] >= plain[STEPS]["cf10"] - 0.01
    # same kNN precision after the same number of steps
    assert abs(warm[STEPS]["qnx"] - plain[STEPS]["qnx"]) <= 0.01
    assert warm[STEPS]["cf10"] >= plain[STEPS]["cf10"] - 0.01


def test_warm_start_rule_through_the_c_abi():
    """ivhd_warm_start as a C caller sees it: a better placement is kept, a non-finite
    or worse one leaves the current positions bit for bit; the state is zeroed."""
    import ctypes

    import oracle
    from paper_2303_05455_gb300 import _lib

    L = _lib.load()
    w = synth.WORKLOADS["gmm2k"]
    X, _ = synth.workload_features(w)
    knn = oracle.knn_f32(X, w.k)
    rn, _ = oracle.random_neighbors(knn, w.r, w.seed)
    terms = oracle.build_terms(knn, rn)
    st = oracle.State.fresh(oracle.init_positions(w.M, w.seed))
    oracle.run(st, terms, w.c, 200, oracle.OPT_MOMENTUM, a=w.a, b=w.b)
    good = st.Y.astype(np.float32)                       # the oracle's own partial embedding
    e = ivhd.Embedding(knn, r=w.r, c=w.c, a=w.a, b=w.b, seed=w.seed)
    e.step(3)                                            # non-zero velocity to be cleared
    y_cur = e.positions(host=True)
    taken = ctypes.c_int32(-1)
    nan = good.copy()
    nan[5, 1] = np.nan
    for bad in (nan, good * 1e3):
        assert L.ivhd_warm_start(e._h, bad.ctypes.data, 0, ctypes.byref(taken)) == 0
        assert taken.value == 0
        assert np.array_equal(e.positions(host=True), y_cur)
    good_d = torch.from_numpy(good).cuda()
    assert L.ivhd_warm_start(e._h, good_d.data_ptr(), 1, ctypes.byref(taken)) == 0
    assert taken.value == 1
    assert np.array_equal(e.positions(host=True), good)
    assert e.stress() == pytest.approx(oracle.stress(good.astype(np.float64), terms, w.c), rel=1e-5)
    # the optimiser state was zeroed: the next step is a first step from the placement
    ref = oracle.State.fresh(good)
    oracle.step(ref, terms, w.c, oracle.OPT_MOMENTUM, a=w.a, b=w.b)
    e.step(1)
    got = e.positions(host=True)
    assert np.abs(got - ref.Y).max() <= 1e-5 * np.abs(ref.Y).max()
    e.close()
