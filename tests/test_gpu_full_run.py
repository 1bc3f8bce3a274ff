"""Full runs at the benchmark's sizes against the oracle's own full runs.

The method is the iteration of Sec. 3.3.3 (Eq. 3.34 and the optimiser
variants of Sec. 3.3.2) run for the whole schedule; an embedding is assessed by
the criteria of Sec. 4.1.  The dynamics amplify rounding, so after 2,000 steps
the FP32 GPU run and the FP64 oracle run are different embeddings of the same
graph: they are compared through the criteria a run is evaluated by.

* Q_NX(k) within 0.01 of the oracle's (the equal-kNN-precision bar).
* cf_2 / cf_10 / cf_100 within 0.01 of the oracle's.  On these inputs Q_NX is
  near its random level (isotropic clusters carry no within-cluster structure
  a 2-D map could keep), so the neighbour hit and the stress are the
  discriminating checks.
* Final stress E (Eq. 3.16) within 0.5 % (relative) of the oracle's.

Inputs (never built by the CUDA path):

* mnist70k: the 70,000 MNIST-shaped uint8 images, their exact kNN graph from
  the oracle (``oracle.knn_u8_gemm``, pinned equal to the serial definition),
  k = 5, r = 1, c = 0.01, 2,000 steps of momentum (a = 0.9, b = 1e-3), of
  Nesterov (same a and b; b lambda_max ~ 0.93 is inside its stability limit
  2 (1 + a) / (1 + 2 a) ~ 1.36) and of Adadelta.  The GPU's own kNN build is also compared with that graph, every
  row, bit for bit.
* 1.4e6 vertices: a kNN-shaped graph with 50 planted clusters whose sizes are
  the power law of the gmm1p4m mixture (``synth.planted_knn_graph``), k = 5,
  r = 1, c = 0.01, 2,000 momentum steps (a = 0.9, b = 1e-3); Q_NX and cf on a
  seeded sample of 10,000 rows.

The oracle runs on all host cores (``oracle.run_threads``, whose per-thread
force sums agree with the serial loop to 1e-12 and keep its pins).  Half
precision gathered positions (FP16 / BF16, FP32 accumulation and master copy)
are held to the same bars against the same oracle run.
"""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2303_05455_gb300 import ivhd, synth

pytestmark = pytest.mark.gpu

THREADS = max(1, len(os.sched_getaffinity(0)))
QNX_BAND = 0.01     # the equal-kNN-precision bar
CF_BAND = 0.01
STRESS_BAND = 0.005  # relative; the final stress of two runs from the same start that
#                     differ in rounding (FP32 or half-precision gathers vs FP64)
OPT_ID = {"momentum": oracle.OPT_MOMENTUM, "nesterov": oracle.OPT_NESTEROV,
          "adadelta": oracle.OPT_ADADELTA}

_cache = {}


def _mnist70k():
    if "c2" not in _cache:
        w = synth.WORKLOADS["mnist70k"]
        X, labels = synth.workload_features(w)
        _cache["c2"] = (w, X, labels, oracle.knn_u8_gemm(X, w.k),
                        np.arange(w.M, dtype=np.int64))
    return _cache["c2"]


def _planted1p4m():
    if "c3" not in _cache:
        w = synth.WORKLOADS["gmm1p4m"]
        knn, labels = synth.planted_knn_graph(w.M, w.k, 1401, sizes=synth.powerlaw_sizes(w.M, 50, 1.5))
        _cache["c3"] = (w, None, labels, knn, synth.sample_rows(w.M, 10_000, 1402))
    return _cache["c3"]


def _criteria_oracle(Y, knn, labels, rows):
    Yf = np.ascontiguousarray(Y, dtype=np.float32)
    out = {"qnx": oracle.qnx(Yf, knn, rows, threads=THREADS)}
    for nn in (2, 10, 100):
        out[f"cf{nn}"] = oracle.cf(Yf, labels, nn, rows, threads=THREADS)
    return out


def _criteria_gpu(Y, knn, labels, rows):
    Yd = torch.as_tensor(np.ascontiguousarray(Y, dtype=np.float32)).cuda() \
        if isinstance(Y, np.ndarray) else Y
    kd = torch.from_numpy(knn).cuda()
    rd = torch.from_numpy(rows).cuda()
    out = {"qnx": ivhd.eval_qnx(Yd, kd, rd)}
    for nn in (2, 10, 100):
        out[f"cf{nn}"] = ivhd.eval_cf(Yd, labels, nn, rd)
    return out


def _oracle_run(key, data, opt):
    ck = (key, opt)
    if ck not in _cache:
        w, _, labels, knn, rows = data
        rn, _ = oracle.random_neighbors(knn, w.r, w.seed)
        terms = oracle.build_terms(knn, rn)
        st = oracle.State.fresh(oracle.init_positions(w.M, w.seed))
        oracle.run_threads(st, terms, w.c, w.n_iter, OPT_ID[opt], a=w.a, b=w.b, threads=THREADS)
        crit = _criteria_oracle(st.Y, knn, labels, rows)
        crit["stress"] = oracle.stress(st.Y, terms, w.c)
        _cache[ck] = (st.Y, crit)
    return _cache[ck]


def _gpu_run(data, opt, pos_format, order="degree"):
    w, _, labels, knn, rows = data
    emb = ivhd.Embedding(torch.from_numpy(knn).cuda(), r=w.r, c=w.c, opt=opt, a=w.a, b=w.b,
                         seed=w.seed, pos_format=pos_format, order=order)
    emb.step(w.n_iter)
    Y = emb.positions()
    crit = _criteria_gpu(Y, knn, labels, rows)
    crit["stress"] = emb.stress()
    emb.close()
    return Y.cpu().numpy(), crit


def _compare(got, ref):
    report = {k: (got[k], ref[k]) for k in ref}
    assert abs(got["qnx"] - ref["qnx"]) <= QNX_BAND, report
    for nn in (2, 10, 100):
        assert abs(got[f"cf{nn}"] - ref[f"cf{nn}"]) <= CF_BAND, report
    assert abs(got["stress"] - ref["stress"]) <= STRESS_BAND * ref["stress"], report
    print("full run", report)


def test_knn_build_mnist70k_equals_the_oracle_graph_on_every_row():
    w, X, _, knn_ref, _ = _mnist70k()
    got = ivhd.knn_build(torch.from_numpy(X).cuda(), w.k).cpu().numpy()
    assert np.array_equal(got, knn_ref)


@pytest.mark.parametrize("opt", ["momentum", "nesterov", "adadelta"])
def test_full_run_mnist70k_matches_oracle(opt):
    data = _mnist70k()
    Y_ref, ref = _oracle_run("c2", data, opt)
    # the GPU evaluators on the oracle's embedding give the oracle's numbers exactly
    assert _criteria_gpu(Y_ref, data[3], data[2], data[4]) == \
        {k: v for k, v in ref.items() if k != "stress"}
    _, got = _gpu_run(data, opt, "f32")
    _compare(got, ref)


def test_full_run_planted_1p4m_matches_oracle():
    data = _planted1p4m()
    Y_ref, ref = _oracle_run("c3", data, "momentum")
    assert _criteria_gpu(Y_ref, data[3], data[2], data[4]) == \
        {k: v for k, v in ref.items() if k != "stress"}
    _, got = _gpu_run(data, "momentum", "f32")
    _compare(got, ref)


# Adadelta with half-precision gathered positions is not equal precision: its
# per-coordinate step sqrt(E[dx^2] + eps) / sqrt(E[g^2] + eps) normalises the
# gradient, so near convergence the rounding noise of the half-precision
# differences keeps the steps from shrinking, and the run ends at a higher
# stress than the oracle's (measured at mnist70k: FP16 1,554 and BF16 2,481
# against 1,480; Q_NX and cf stay within 0.01, as they do for any embedding
# that keeps the clusters apart).  Momentum and Nesterov scale the noise by b.
def _adadelta_half(fmt, gap):
    return pytest.param("c2", "adadelta", marks=pytest.mark.xfail(
        strict=True, reason=f"{fmt} gathers with Adadelta: final stress {gap} above the "
                            "oracle's, outside the 0.5 % band (not equal precision)"))


HALF_CASES = [("c2", "momentum"), ("c2", "nesterov"), ("c3", "momentum")]


@pytest.mark.parametrize("where,opt", HALF_CASES + [_adadelta_half("FP16", "5 %")])
def test_full_run_fp16_positions_match_oracle(where, opt):
    data = _mnist70k() if where == "c2" else _planted1p4m()
    _, ref = _oracle_run(where, data, opt)
    _, got = _gpu_run(data, opt, "f16")
    _compare(got, ref)


@pytest.mark.parametrize("where,opt", HALF_CASES + [_adadelta_half("BF16", "68 %")])
def test_full_run_bf16_positions_match_oracle(where, opt):
    data = _mnist70k() if where == "c2" else _planted1p4m()
    _, ref = _oracle_run(where, data, opt)
    _, got = _gpu_run(data, opt, "bf16")
    _compare(got, ref)


@pytest.mark.parametrize("pos_format", ["f32", "f16"])
def test_full_run_cluster_grouped_order_matches_oracle(pos_format):
    """The cluster-grouped layout order changes only where rows sit and so the
    summation order of the steps; the full run is held to the same bars."""
    data = _planted1p4m()
    _, ref = _oracle_run("c3", data, "momentum")
    _, got = _gpu_run(data, "momentum", pos_format, order="degree_cluster")
    _compare(got, ref)
