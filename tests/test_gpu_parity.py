"""GPU path vs the FP64 oracle through the C ABI (``-m gpu``).

Tolerances.  One step of forces and positions must agree within 1e-5
relative, measured against the largest magnitude of the oracle array
(the FP32 rounding of a vertex force is a few units of 2^-24 of the sum of
its term magnitudes, far inside 1e-5).  Integer work (random neighbours, kNN
ids, neighbour sets of the quality criteria, layout counters) must match
exactly: every such decision is made in the same precision on both sides.

The update is also checked at its own scale: the displacement y' - y of one
step, element by element, within 1e-5 of the largest oracle displacement
plus what FP32 arithmetic allows for that element (``step_bound``): the
force's FP32 summation bound, gamma(n) times the sum of the magnitudes of its
n terms, carried through the optimiser's sensitivity d(y')/dF, a few
roundings of the update itself and the roundings of storing y' in FP32.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2303_05455_gb300 import ivhd, synth
from paper_2303_05455_gb300._lib import IvhdError
from step_bounds import close_elem, force_error_bound, step_bound

pytestmark = pytest.mark.gpu

RTOL = 1e-5
OPT_ID = {"momentum": oracle.OPT_MOMENTUM, "nesterov": oracle.OPT_NESTEROV,
          "adadelta": oracle.OPT_ADADELTA}


def close(got, ref, rtol=RTOL):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    assert got.shape == ref.shape
    assert np.all(np.isfinite(got))
    err = np.abs(got - ref).max() if ref.size else 0.0
    scale = np.abs(ref).max() if ref.size else 0.0
    assert err <= rtol * scale, f"max err {err:.3e} > {rtol:g} * {scale:.3e}"


def graph_case(name):
    if name == "gmm2k":
        w = synth.WORKLOADS["gmm2k"]
        X, _ = synth.workload_features(w)
        return oracle.knn_f32(X, w.k), w.r, w.c
    if name == "hubs5k":
        return synth.random_knn_graph(5000, 5, 21, hub_frac=0.3, n_hubs=20), 2, 0.05
    if name == "ragged37":
        return synth.random_knn_graph(37, 3, 4), 1, 0.1
    if name == "pair":
        return np.array([[1], [0]], np.int32), 1, 0.1      # no eligible random neighbour
    if name == "triangle":
        return np.array([[1, 2], [0, 2], [0, 1]], np.int32), 2, 0.3
    if name == "star":
        M = 300                                            # vertex 0 has degree ~M
        rng = np.random.default_rng(8)
        g = np.empty((M, 3), np.int32)
        g[0] = [1, 2, 3]
        for i in range(1, M):
            others = rng.choice(np.setdiff1d(np.arange(1, M), [i]), 2, replace=False)
            g[i] = [0, *others]
        return g, 1, 0.02
    if name == "star3k":
        # vertex 0 is a neighbour of every other vertex (degree ~3,000): one of the
        # rows long enough to be processed by 4 warps
        M = 3000
        rng = np.random.default_rng(10)
        g = np.empty((M, 3), np.int32)
        g[0] = [1, 2, 3]
        i = np.arange(1, M)
        a = rng.integers(1, M, size=M - 1)
        b = rng.integers(1, M, size=M - 1)
        bad = (a == i) | (b == i) | (a == b)
        while bad.any():
            a[bad] = rng.integers(1, M, size=int(bad.sum()))
            b[bad] = rng.integers(1, M, size=int(bad.sum()))
            bad = (a == i) | (b == i) | (a == b)
        g[1:, 0], g[1:, 1], g[1:, 2] = 0, a, b
        return g, 1, 0.02
    raise KeyError(name)


CASES = ["gmm2k", "hubs5k", "ragged37", "pair", "triangle", "star", "star3k"]


def stable_b(case):
    # momentum is stable only while b lambda_max < 2 (1 + a); star3k's hub has degree
    # ~3,000 (lambda_max ~ 6,000), where b = 0.01 would blow up within a few steps
    return 5e-4 if case == "star3k" else 0.01


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("seed", [0, 77])
def test_random_neighbors_bit_exact(case, seed):
    knn, r, c = graph_case(case)
    emb = ivhd.Embedding(knn, r=r, c=c, seed=seed)
    got = emb.random_neighbors()
    ref, empty = oracle.random_neighbors(knn, r, seed)
    assert np.array_equal(got, ref)
    assert emb.info()["empty_rn"] == empty


@pytest.mark.parametrize("case", CASES)
def test_init_positions_bit_exact(case):
    knn, r, c = graph_case(case)
    emb = ivhd.Embedding(knn, r=r, c=c, seed=123)
    assert np.array_equal(emb.positions(host=True),
                          oracle.init_positions(knn.shape[0], 123).astype(np.float32))


@pytest.mark.parametrize("dedup", [False, True])
@pytest.mark.parametrize("case", CASES)
def test_layout_counts_match_term_list(case, dedup):
    knn, r, c = graph_case(case)
    emb = ivhd.Embedding(knn, r=r, c=c, seed=3, dedup_mutual=dedup)
    rn, _ = oracle.random_neighbors(knn, r, 3)
    terms = oracle.build_terms(knn, rn, dedup=dedup)
    inf = emb.info()
    assert inf["n_terms"] == terms.T
    # stored row entries: out-nn, kept rn, in-nn from non-mutual sources, in-rn
    M, k = knn.shape
    out_sets = [set(row) for row in knn.tolist()]
    deg = np.full(M, k, np.int64) + (rn >= 0).sum(axis=1)
    for i in range(M):
        for j in knn[i]:
            if i not in out_sets[j]:
                deg[j] += 1
        for j in rn[i]:
            if j >= 0:
                deg[j] += 1
    assert inf["nnz_sym"] == deg.sum()
    assert inf["max_degree"] == deg.max()
    mutual_pairs = sum(1 for i in range(M) for j in knn[i] if j < i and i in out_sets[j])
    assert deg.sum() == 2 * terms.T - (0 if dedup else 2 * mutual_pairs)


@pytest.mark.parametrize("hub_threshold", [0, 1, 65535])
@pytest.mark.parametrize("dedup", [False, True])
@pytest.mark.parametrize("opt", ["momentum", "nesterov", "adadelta"])
@pytest.mark.parametrize("case", CASES)
def test_one_step_and_ten_steps(case, opt, dedup, hub_threshold):
    knn, r, c = graph_case(case)
    a, b = 0.9, stable_b(case)
    emb = ivhd.Embedding(knn, r=r, c=c, opt=opt, a=a, b=b, seed=11, dedup_mutual=dedup,
                         hub_threshold=hub_threshold)
    rn, _ = oracle.random_neighbors(knn, r, 11)
    terms = oracle.build_terms(knn, rn, dedup=dedup)
    y0 = emb.positions(host=True).astype(np.float64)
    F0 = oracle.forces(y0, terms, c)
    close(emb.forces(host=True), F0)
    st = oracle.State.fresh(y0)
    emb.step(1)
    oracle.step(st, terms, c, OPT_ID[opt], a=a, b=b)
    y1 = emb.positions(host=True)
    close(y1, st.Y)
    # the displacement of the step, element by element at its own scale
    d_ref = st.Y - y0
    close_elem(y1 - y0, d_ref,
               step_bound(opt, st.Y, d_ref, F0, force_error_bound(y0, terms, c), a, b),
               "displacement")
    emb.step(9)
    oracle.run(st, terms, c, 9, OPT_ID[opt], a=a, b=b)
    close(emb.positions(host=True), st.Y)
    # force and stress kernels at the evolved GPU positions (same input on both sides)
    y10 = emb.positions(host=True).astype(np.float64)
    close(emb.forces(host=True), oracle.forces(y10, terms, c))
    assert emb.stress() == pytest.approx(oracle.stress(y10, terms, c), rel=1e-5)


@pytest.mark.parametrize("opt", ["momentum", "nesterov", "adadelta"])
def test_one_step_from_a_given_state_at_the_step_scale(opt):
    """One step from a chosen optimiser state: the momentum term a v, Nesterov's
    look-ahead and Adadelta's accumulators all enter the displacement."""
    # every vertex has the same symmetric degree (circulant graph, no random
    # neighbours), so the internal vertex order is the input order and a
    # checkpoint's arrays can be written directly
    M, a, b, c = 3000, 0.9, 0.01, 0.01
    i = np.arange(M)
    knn = np.stack([(i + 1) % M, (i + 7) % M, (i + 100) % M], axis=1).astype(np.int32)
    emb = ivhd.Embedding(knn, r=0, c=c, opt=opt, a=a, b=b, seed=3)
    rng = np.random.default_rng(5)
    y = (rng.random((M, 2)) * 3.0).astype(np.float32)
    s1 = (rng.standard_normal((M, 2)) * 0.02).astype(np.float32)
    s2 = None
    if opt == "adadelta":
        s1 = (rng.random((M, 2)) * 0.5).astype(np.float32)        # E[g^2]
        s2 = (rng.random((M, 2)) * 1e-4).astype(np.float32)       # E[dx^2]
    blob = bytearray(emb.get_state())
    arrays = [y, s1] + ([s2] if s2 is not None else [])
    head = len(blob) - len(arrays) * M * 8
    stored_y = y
    if opt == "nesterov":        # the state holds the look-ahead point y + a v
        stored_y = (y.astype(np.float64) + np.float32(a) * s1.astype(np.float64)).astype(np.float32)
    for q, arr in enumerate([stored_y] + arrays[1:]):
        blob[head + q * M * 8: head + (q + 1) * M * 8] = arr.tobytes()
    emb.set_state(bytes(blob))
    y_gpu0 = emb.positions(host=True).astype(np.float64)
    if opt != "nesterov":
        assert np.array_equal(y_gpu0, y)                     # input order == internal order
    rn = np.zeros((M, 0), np.int32)
    terms = oracle.build_terms(knn, rn)
    st = oracle.State(y_gpu0.copy(), s1.astype(np.float64),
                      np.zeros((M, 2)) if s2 is None else s2.astype(np.float64))
    if opt == "nesterov":        # the oracle's look-ahead y + a v must be the GPU's stored point
        st.Y = stored_y.astype(np.float64) - a * st.S1
    y_start = st.Y.copy()
    F_at = oracle.forces(y_start + (a * st.S1 if opt == "nesterov" else 0.0), terms, c)
    F_err = force_error_bound(y_start + (a * st.S1 if opt == "nesterov" else 0.0), terms, c)
    v0 = st.S1.copy() if opt != "adadelta" else None
    oracle.step(st, terms, c, OPT_ID[opt], a=a, b=b)
    emb.step(1)
    y1 = emb.positions(host=True)
    d_ref = st.Y - y_start
    bound = step_bound(opt, st.Y, d_ref, F_at, F_err, a, b, v0=v0,
                       s1=None if opt != "adadelta" else s1.astype(np.float64),
                       s2=None if s2 is None else s2.astype(np.float64))
    close_elem(y1 - y_start, d_ref, bound, "displacement from a given state")
    # the momentum term is a large part of this step: a wrong coefficient would show
    if opt == "momentum":
        assert np.abs(a * v0).max() > 100 * bound.max()


@pytest.mark.parametrize("vpw", [1, 2, 4, 8])
@pytest.mark.parametrize("opt", ["momentum", "adadelta"])
def test_rows_shared_by_a_warp_match_oracle(opt, vpw):
    # hub threshold 16 makes most rows warp-per-vertex rows; with vpw > 1 the
    # rows below 512 / vpw entries share a warp, 32 / vpw lanes each
    knn, r, c = graph_case("hubs5k")
    a, b = 0.9, 0.002
    emb = ivhd.Embedding(knn, r=r, c=c, opt=opt, a=a, b=b, seed=5, hub_threshold=16,
                         vertices_per_warp=vpw, resident=False)
    rn, _ = oracle.random_neighbors(knn, r, 5)
    terms = oracle.build_terms(knn, rn)
    y0 = emb.positions(host=True).astype(np.float64)
    close(emb.forces(host=True), oracle.forces(y0, terms, c))
    st = oracle.State.fresh(y0)
    emb.step(10)
    oracle.run(st, terms, c, 10, OPT_ID[opt], a=a, b=b)
    close(emb.positions(host=True), st.Y)
    y10 = emb.positions(host=True).astype(np.float64)
    assert emb.stress() == pytest.approx(oracle.stress(y10, terms, c), rel=1e-5)


def test_given_positions_and_zero_distance_pairs():
    # all vertices start at one point: every rn pair has d = 0 (zero force),
    # nn forces vanish too; then a spread start through ivhd_set_positions
    knn, r, c = graph_case("hubs5k")
    M = knn.shape[0]
    emb = ivhd.Embedding(knn, r=r, c=c, seed=2, init_uniform=False)
    rn, _ = oracle.random_neighbors(knn, r, 2)
    terms = oracle.build_terms(knn, rn)
    assert np.all(emb.positions(host=True) == 0)
    assert np.all(emb.forces(host=True) == 0)
    y = synth.uniform_positions(M, 9, scale=3.0)
    y[:100] = y[100]                                      # coincident points
    emb.set_positions(y)
    close(emb.forces(host=True), oracle.forces(y.astype(np.float64), terms, c))
    yt = torch.from_numpy(y).cuda()
    emb.set_positions(yt)
    torch.cuda.synchronize()
    close(emb.forces(host=True), oracle.forces(y.astype(np.float64), terms, c))


def test_deterministic_bitwise():
    knn, r, c = graph_case("hubs5k")
    out = []
    for _ in range(2):
        emb = ivhd.Embedding(knn, r=r, c=c, seed=9)
        emb.step(150)   # crosses the CUDA-graph path (64-step graphs) and the tail
        out.append(emb.positions(host=True))
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("opt", ["momentum", "nesterov", "adadelta"])
def test_bitwise_equal_across_block_sizes(opt):
    # the layout (hub threshold) fixes every vertex's summation order; the
    # block size only groups rows into blocks, so results must not move
    knn, r, c = graph_case("hubs5k")
    out = []
    for bs in (128, 256, 512):
        emb = ivhd.Embedding(knn, r=r, c=c, seed=9, opt=opt, b=0.002, block_size=bs,
                             hub_threshold=32, vertices_per_warp=4, resident=False)
        emb.step(70)
        out.append(emb.positions(host=True))
        emb.close()
    assert np.all(np.isfinite(out[0]))
    assert np.array_equal(out[0], out[1]) and np.array_equal(out[0], out[2])


@pytest.mark.parametrize("opt", ["momentum", "adadelta"])
def test_long_rows_bitwise_equal_across_block_sizes(opt):
    # rows of 512 entries or more take 4 warps whatever the block size, so the
    # block size still only groups rows into blocks
    knn, r, c = graph_case("star3k")
    out = []
    for bs in (128, 256, 512):
        emb = ivhd.Embedding(knn, r=r, c=c, seed=9, opt=opt, b=stable_b("star3k"),
                             block_size=bs, resident=False)
        emb.step(70)
        out.append(emb.positions(host=True))
        emb.close()
    assert np.all(np.isfinite(out[0]))
    assert np.array_equal(out[0], out[1]) and np.array_equal(out[0], out[2])


def test_graph_replay_equals_single_launches():
    knn, r, c = graph_case("gmm2k")
    a = ivhd.Embedding(knn, r=r, c=c, seed=4, resident=False)
    b = ivhd.Embedding(knn, r=r, c=c, seed=4, resident=False)
    a.step(130)
    for _ in range(130):
        b.step(1)
    assert np.array_equal(a.positions(host=True), b.positions(host=True))
    assert a.info()["steps_done"] == 130 and a.info()["kernel_launches"] == 130


def test_checkpoint_resume_bitwise_and_mismatch():
    knn, r, c = graph_case("hubs5k")
    ref = ivhd.Embedding(knn, r=r, c=c, opt="adadelta", seed=5)
    ref.step(40)
    state = ref.get_state()
    ref.step(30)
    y_ref = ref.positions(host=True)
    other = ivhd.Embedding(knn, r=r, c=c, opt="adadelta", seed=5)
    other.set_state(state)
    assert other.info()["steps_done"] == 40
    other.step(30)
    assert np.array_equal(other.positions(host=True), y_ref)
    wrong = ivhd.Embedding(knn, r=r, c=c, opt="adadelta", seed=6)
    with pytest.raises(IvhdError) as e:
        wrong.set_state(state)
    assert e.value.status == -7


def test_nonfinite_detected():
    knn, r, c = graph_case("ragged37")
    emb = ivhd.Embedding(knn, r=r, c=c)
    y = synth.uniform_positions(37, 1)
    y[5, 1] = np.nan
    emb.set_positions(y)
    with pytest.raises(IvhdError) as e:
        emb.stress()
    assert e.value.status == -5


@pytest.mark.parametrize("bad", ["range", "negative", "self", "dup"])
def test_invalid_graph_rejected_on_device(bad):
    knn = synth.random_knn_graph(50, 3, 1)
    if bad == "range":
        knn[7, 1] = 50
    elif bad == "negative":
        knn[7, 1] = -2      # -1 is an absent entry, any other negative id is invalid
    elif bad == "self":
        knn[7, 1] = 7
    else:
        knn[7, 1] = knn[7, 0]
    for dev in (False, True):
        src = torch.from_numpy(knn).cuda() if dev else knn
        with pytest.raises(IvhdError) as e:
            ivhd.Embedding(src, r=1, c=0.1)
        assert e.value.status == -2


# ------------------------------------------------------------------- kNN


@pytest.mark.parametrize("M,N,k", [(1007, 50, 5), (300, 33, 1), (513, 100, 16), (129, 7, 64)])
def test_knn_f32_bit_exact(M, N, k):
    X, _ = synth.gaussian_mixture(M, N, 4, M + N)
    got = ivhd.knn_build(torch.from_numpy(X).cuda(), k).cpu().numpy()
    assert np.array_equal(got, oracle.knn_f32(X, k))


def test_knn_f32_ties_to_lower_index():
    # duplicated rows: equal distances must resolve to the lower index
    X, _ = synth.gaussian_mixture(200, 8, 2, 3)
    X[100:150] = X[:50]
    got = ivhd.knn_build(torch.from_numpy(X).cuda(), 6).cpu().numpy()
    assert np.array_equal(got, oracle.knn_f32(X, 6))


@pytest.mark.parametrize("M,N,k", [(777, 784, 5), (260, 30, 3)])
def test_knn_u8_bit_exact(M, N, k):
    X, _ = synth.mnist_like(M, 5, N=N)
    got = ivhd.knn_build(torch.from_numpy(X).cuda(), k).cpu().numpy()
    assert np.array_equal(got, oracle.knn_u8(X, k))


# --------------------------------------------------------------- quality


def test_eval_qnx_cf_bit_exact():
    M, k = 5000, 5
    knn = synth.random_knn_graph(M, k, 12)
    Y = synth.uniform_positions(M, 3)
    Y[:500] = np.round(Y[:500] * 8) / 8   # many exact ties
    rows = synth.sample_rows(M, 1200, 5)
    q, low = ivhd.eval_qnx(torch.from_numpy(Y).cuda(), torch.from_numpy(knn).cuda(),
                           torch.from_numpy(rows).cuda(), return_lowd=True)
    q_ref, low_ref = oracle.qnx(Y, knn, rows, return_lowd=True)
    assert np.array_equal(low.cpu().numpy(), low_ref)
    assert q == q_ref
    lab = (np.arange(M) % 7).astype(np.int32)
    for nn in (2, 10, 100):
        got = ivhd.eval_cf(torch.from_numpy(Y).cuda(), lab, nn, torch.from_numpy(rows).cuda())
        assert got == oracle.cf(Y, lab, nn, rows)


# ------------------------------------------------------------- full runs


@pytest.mark.parametrize("opt", ["momentum", "adadelta"])
def test_full_run_gmm2k_precision_matches_oracle(opt):
    w = synth.WORKLOADS["gmm2k"]
    X, labels = synth.workload_features(w)
    knn = oracle.knn_f32(X, w.k)
    emb = ivhd.Embedding(knn, r=w.r, c=w.c, opt=opt, a=w.a, b=w.b, seed=w.seed)
    emb.step(w.n_iter)
    Y = emb.positions(host=True)
    rn, _ = oracle.random_neighbors(knn, w.r, w.seed)
    terms = oracle.build_terms(knn, rn)
    st = oracle.State.fresh(oracle.init_positions(w.M, w.seed))
    oracle.run(st, terms, w.c, w.n_iter, OPT_ID[opt], a=w.a, b=w.b)
    q_gpu = oracle.qnx(Y, knn)
    q_ref = oracle.qnx(st.Y.astype(np.float32), knn)
    assert abs(q_gpu - q_ref) <= 0.01, (q_gpu, q_ref)
    E_gpu, E_ref = emb.stress(), oracle.stress(st.Y, terms, w.c)
    assert abs(E_gpu - E_ref) <= 0.05 * E_ref, (E_gpu, E_ref)
    if opt == "momentum":  # Adadelta starts with sqrt(eps)-sized steps and is still far from converged
        assert q_gpu > 10 * w.k / (w.M - 1)   # far above a random embedding


def test_probe_gather_rate_is_plausible():
    rate = ivhd.probe_gather(1_400_000, 1 << 22, 3)
    assert 1e9 < rate < 1e13


def test_probe_launch_floor_is_plausible_and_below_the_step_of_the_same_grid():
    small = ivhd.probe_launch(152, 128, 500)
    large = ivhd.probe_launch(152 * 30, 128, 500)
    assert 0.05 < small < 50 and small < large        # more blocks take longer to dispatch
    M = 70_000
    knn = synth.random_knn_graph(M, 5, 7)
    emb = ivhd.Embedding(torch.from_numpy(knn).cuda(), r=1, c=0.01, a=0.9, b=1e-3, seed=1)
    emb.step(50)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    emb.step(500)
    e1.record()
    torch.cuda.synchronize()
    inf = emb.info()
    emb.close()
    step_us = 1e3 * e0.elapsed_time(e1) / 500
    floor = ivhd.probe_launch(inf["step_blocks"], inf["step_threads"], 500)
    assert inf["launch_form"] == 0 and inf["step_blocks"] > 0 and inf["step_threads"] == 128
    assert step_us >= 0.8 * floor, (step_us, floor)


@pytest.mark.parametrize("opt", ["momentum", "nesterov", "adadelta"])
@pytest.mark.parametrize("case", ["gmm2k", "hubs5k", "ragged37", "star"])
def test_cluster_order_matches_oracle(case, opt):
    """The cluster-grouped vertex order changes only where rows are stored (and so the
    FP32 summation order): forces, steps and stress still match the oracle."""
    knn, r, c = graph_case(case)
    a, b = 0.9, 0.01
    emb = ivhd.Embedding(knn, r=r, c=c, opt=opt, a=a, b=b, seed=11, order="degree_cluster",
                         resident=False)
    rn, _ = oracle.random_neighbors(knn, r, 11)
    assert np.array_equal(emb.random_neighbors(), rn)
    terms = oracle.build_terms(knn, rn)
    y0 = emb.positions(host=True).astype(np.float64)
    F0 = oracle.forces(y0, terms, c)
    close(emb.forces(host=True), F0)
    st = oracle.State.fresh(y0)
    emb.step(1)
    oracle.step(st, terms, c, OPT_ID[opt], a=a, b=b)
    y1 = emb.positions(host=True)
    close(y1, st.Y)
    d_ref = st.Y - y0
    close_elem(y1 - y0, d_ref,
               step_bound(opt, st.Y, d_ref, F0, force_error_bound(y0, terms, c), a, b),
               "displacement")
    emb.step(9)
    oracle.run(st, terms, c, 9, OPT_ID[opt], a=a, b=b)
    close(emb.positions(host=True), st.Y)
    y10 = emb.positions(host=True).astype(np.float64)
    assert emb.stress() == pytest.approx(oracle.stress(y10, terms, c), rel=1e-5)


def test_cluster_order_in_a_batch_matches_separate_contexts():
    """Several embeddings in one context form separate components; the cluster order
    keeps each embedding's results equal to its own context's within FP32 rounding."""
    graphs = [graph_case("gmm2k")[0], synth.random_knn_graph(3000, 4, 9),
              synth.random_knn_graph(500, 3, 10)]
    seeds = [5, 6, 7]
    emb = ivhd.Embedding.batch(graphs, r=1, seeds=seeds, c=0.01, a=0.9, b=0.01,
                               order="degree_cluster")
    emb.step(10)
    Y = emb.positions(host=True)
    lo = 0
    for g, sd in zip(graphs, seeds):
        one = ivhd.Embedding(g, r=1, c=0.01, a=0.9, b=0.01, seed=sd, resident=False)
        one.step(10)
        close(Y[lo:lo + g.shape[0]], one.positions(host=True).astype(np.float64))
        lo += g.shape[0]
