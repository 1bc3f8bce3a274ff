"""Half-precision gathered positions (FP16 / BF16 copies, FP32 master and accumulation).

One step is exact up to FP32 rounding once the oracle is given the same
rounded positions the kernel gathers (the rounding is an input transform,
done here with numpy).  Full runs report the error of each storage format
against the FP64 oracle's run: Q_NX (kNN precision) and stress.
"""
import numpy as np
import pytest

import oracle
from paper_2303_05455_gb300 import ivhd, synth

pytestmark = pytest.mark.gpu


def bf16_round(x):
    b = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def rounded(y, fmt):
    y = np.asarray(y, np.float32)
    return y.astype(np.float16).astype(np.float32) if fmt == "f16" else bf16_round(y)


@pytest.mark.parametrize("fmt", ["f16", "bf16"])
@pytest.mark.parametrize("opt", ["momentum", "nesterov", "adadelta"])
@pytest.mark.parametrize("hub_threshold", [0, 1])
def test_one_step_with_rounded_gathers(fmt, opt, hub_threshold):
    knn = synth.random_knn_graph(5000, 5, 21, hub_frac=0.3, n_hubs=20)
    r, c, a, b = 2, 0.05, 0.9, 0.5
    emb = ivhd.Embedding(knn, r=r, c=c, opt=opt, a=a, b=b, seed=11, pos_format=fmt,
                         hub_threshold=hub_threshold, init_uniform=False)
    y0 = synth.uniform_positions(5000, 4, scale=6.0)
    emb.set_positions(y0)
    rn, _ = oracle.random_neighbors(knn, r, 11)
    terms = oracle.build_terms(knn, rn)
    F_ref = oracle.forces(rounded(y0, fmt).astype(np.float64), terms, c)
    emb.step(1)
    y1 = emb.positions(host=True).astype(np.float64)
    st = oracle.State.fresh(y0)
    # the update of one step from zero state, with the force taken at the rounded positions
    if opt == "adadelta":
        g = -F_ref
        eg = 0.05 * g * g
        want = y0 - np.sqrt(1e-6) / np.sqrt(eg + 1e-6) * g
    else:
        want = y0 + b * F_ref
    err = np.abs(y1 - want).max()
    assert err <= 1e-5 * max(np.abs(want).max(), 1.0), err
    # forces / stress / positions report the FP32 master positions
    np.testing.assert_array_equal(emb.positions(host=True), y1.astype(np.float32))


# BF16 keeps 8 significant bits: at |y| ~ 20 its spacing is 0.125, coarser than
# the within-cluster distances the nn terms pull towards 0, so the 2-D
# neighbour sets of the 2,000-point run differ (Q_NX 0.069 against the
# oracle's 0.085).  It does not reach equal kNN precision here; the test keeps
# the 0.01 bar and is expected to fail for BF16.
@pytest.mark.parametrize("fmt", [
    "f32", "f16",
    pytest.param("bf16", marks=pytest.mark.xfail(strict=True, reason="BF16 gathered positions "
                                                 "miss the 0.01 Q_NX band on this workload"))])
def test_full_run_error_vs_oracle(fmt, record_property):
    w = synth.WORKLOADS["gmm2k"]
    X, _ = synth.workload_features(w)
    knn = oracle.knn_f32(X, w.k)
    rn, _ = oracle.random_neighbors(knn, w.r, w.seed)
    terms = oracle.build_terms(knn, rn)
    st = oracle.State.fresh(oracle.init_positions(w.M, w.seed))
    oracle.run(st, terms, w.c, w.n_iter, oracle.OPT_MOMENTUM, a=w.a, b=w.b)
    q_ref = oracle.qnx(st.Y.astype(np.float32), knn)
    E_ref = oracle.stress(st.Y, terms, w.c)
    emb = ivhd.Embedding(knn, r=w.r, c=w.c, a=w.a, b=w.b, seed=w.seed, pos_format=fmt)
    emb.step(w.n_iter)
    Y = emb.positions(host=True)
    q = oracle.qnx(Y, knn)
    E = oracle.stress(Y.astype(np.float64), terms, w.c)
    record_property("qnx", q)
    record_property("qnx_oracle", q_ref)
    record_property("stress_rel_err", (E - E_ref) / E_ref)
    print(f"{fmt}: Q_NX {q:.4f} (oracle {q_ref:.4f}), stress {E:.5g} (oracle {E_ref:.5g})")
    assert abs(q - q_ref) <= 0.01      # the equal-kNN-precision bar, every format
