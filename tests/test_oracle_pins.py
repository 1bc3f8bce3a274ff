"""Pins of the FP64 oracle against closed forms, invariants and brute force.

None of these compare the oracle with itself: each expected value comes from
mathematics the paper fixes (a 2x2 linear recurrence, the gradient of the
stress, symmetry of the stress, textbook kNN on a line, published generator
vectors), so a dropped term, a wrong sign or a swapped index fails one of them.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2303_05455_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _terms(pairs, M):
    ti = np.array([p[0] for p in pairs], np.int64)
    tj = np.array([p[1] for p in pairs], np.int64)
    kind = np.array([p[2] for p in pairs], np.int8)
    return oracle.Terms(ti, tj, kind, M)


# ---------------------------------------------------------------- generator


def test_splitmix64_published_vectors():
    for line in open(os.path.join(GOLD, "splitmix64.txt")):
        if line.startswith("#") or not line.strip():
            continue
        seed, t, val = (int(x) for x in line.split())
        assert oracle.splitmix64(seed, t) == val


def test_init_positions_grid_and_uniformity():
    Y = oracle.init_positions(20000, 7)
    assert Y.shape == (20000, 2)
    assert np.all((Y >= 0) & (Y < 1))
    assert np.all(Y * 2 ** 24 == np.floor(Y * 2 ** 24))   # exact 24-bit grid, fits FP32
    assert abs(Y.mean() - 0.5) < 0.01
    assert abs(Y.var() - 1 / 12) < 0.003
    assert abs(np.corrcoef(Y[:, 0], Y[:, 1])[0, 1]) < 0.03
    assert not np.array_equal(Y, oracle.init_positions(20000, 8))


# ------------------------------------------------------------ random neighbours


def _connected(knn, i, j):
    return i == j or j in knn[i] or i in knn[j]


def test_random_neighbors_rules_and_uniformity():
    M, k, r = 3000, 5, 2
    knn = synth.random_knn_graph(M, k, 11, hub_frac=0.2, n_hubs=10)
    rn, empty = oracle.random_neighbors(knn, r, 123)
    assert empty == 0
    for i in range(M):
        assert len(set(rn[i].tolist())) == r
        for j in rn[i]:
            assert 0 <= j < M and not _connected(knn, i, int(j))
    # draws are uniform over vertices: chi-square over 30 bins of the id range
    h = np.bincount(rn.ravel() * 30 // M, minlength=30)
    exp = rn.size / 30
    chi2 = ((h - exp) ** 2 / exp).sum()
    assert chi2 < 70  # 29 dof, p ~ 1e-4
    # deterministic in the seed, different across seeds
    assert np.array_equal(rn, oracle.random_neighbors(knn, r, 123)[0])
    assert not np.array_equal(rn, oracle.random_neighbors(knn, r, 124)[0])


def test_random_neighbors_fallback_and_empty_slots():
    # vertex 0 is connected to every other vertex: no random neighbour exists
    M = 5
    knn = np.array([[1, 2], [0, 2], [0, 1], [0, 1], [0, 1]], np.int32)
    knn[0] = [1, 2]
    knn[3] = [0, 4]
    knn[4] = [0, 3]
    rn, empty = oracle.random_neighbors(knn, 2, 5)
    # 0 is joined to 1, 2 (out) and 3, 4 (in): both slots empty
    assert rn[0].tolist() == [-1, -1]
    # 1 is joined to 0, 2 only: its eligible set is exactly {3, 4}
    assert sorted(rn[1].tolist()) == [3, 4]
    # 3 is joined to 0, 4: eligible {1, 2}
    assert sorted(rn[3].tolist()) == [1, 2]
    assert empty == 2


# ---------------------------------------------------------------- terms


def test_term_counts_multiplicity_and_dedup():
    M, k, r = 400, 4, 1
    knn = synth.random_knn_graph(M, k, 3)  # ~k^2/2 mutual pairs expected
    rn, _ = oracle.random_neighbors(knn, r, 9)
    t_mult = oracle.build_terms(knn, rn, dedup=False)
    t_dedup = oracle.build_terms(knn, rn, dedup=True)
    mutual = sum(1 for i in range(M) for j in knn[i] if j < i and i in knn[j])
    assert mutual >= 1
    assert t_mult.T == M * k + M * r
    assert t_dedup.T == M * k - mutual + M * r
    undirected = {(min(i, int(j)), max(i, int(j))) for i in range(M) for j in knn[i]}
    got = {(min(a, b), max(a, b)) for a, b, t in zip(t_dedup.ti, t_dedup.tj, t_dedup.kind) if t == 0}
    assert got == undirected and (t_dedup.kind == 0).sum() == len(undirected)


# ---------------------------------------------------------------- stress


def test_stress_hand_example():
    Y = np.array([[0.0, 0.0], [3.0, 4.0], [0.0, 1.0]])
    c = 0.1
    t = _terms([(0, 1, 0), (0, 2, 1), (1, 2, 1)], 3)
    want = 25.0 + c * (1 - 1.0) ** 2 + c * (1 - np.sqrt(18.0)) ** 2
    assert oracle.stress(Y, t, c) == pytest.approx(want, rel=1e-15)


def _random_case(M, k, r, seed, dedup=False):
    knn = synth.random_knn_graph(M, k, seed)
    rn, _ = oracle.random_neighbors(knn, r, seed + 1)
    t = oracle.build_terms(knn, rn, dedup=dedup)
    Y = np.random.default_rng(seed).random((M, 2)) * 2.0
    return knn, rn, t, Y


@pytest.mark.parametrize("dedup", [False, True])
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_force_is_half_negative_gradient(seed, dedup):
    M = 12 + seed * 2
    _, _, t, Y = _random_case(M, 3, 2, seed, dedup)
    c = 0.3
    F = oracle.forces(Y, t, c)
    h = 1e-6
    G = np.zeros_like(Y)
    for i in range(M):
        for q in range(2):
            Yp = Y.copy()
            Ym = Y.copy()
            Yp[i, q] += h
            Ym[i, q] -= h
            G[i, q] = (oracle.stress(Yp, t, c) - oracle.stress(Ym, t, c)) / (2 * h)
    err = np.abs(F - (-0.5 * G)).max() / np.abs(F).max()
    assert err < 1e-7


def test_net_force_zero_and_centroid_fixed():
    _, _, t, Y = _random_case(300, 5, 1, 7)
    F = oracle.forces(Y, t, 0.01)
    scale = np.abs(F).sum()
    assert np.abs(F.sum(axis=0)).max() <= 1e-12 * scale
    st = oracle.State.fresh(Y)
    c0 = st.Y.mean(axis=0)
    oracle.run(st, t, 0.01, 50, oracle.OPT_MOMENTUM, a=0.9, b=0.01)
    assert np.abs(st.Y.mean(axis=0) - c0).max() < 1e-12
    st2 = oracle.State.fresh(Y)
    oracle.run(st2, t, 0.01, 50, oracle.OPT_NESTEROV, a=0.9, b=0.01)
    assert np.abs(st2.Y.mean(axis=0) - c0).max() < 1e-12


def test_rigid_motion_invariance():
    _, _, t, Y = _random_case(60, 4, 2, 5)
    c = 0.05
    th = 0.7
    R = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
    Refl = np.array([[1.0, 0.0], [0.0, -1.0]])
    shift = np.array([3.0, -2.0])
    E0 = oracle.stress(Y, t, c)
    F0 = oracle.forces(Y, t, c)
    for Q in (R, Refl, R @ Refl):
        Y2 = Y @ Q.T + shift
        assert oracle.stress(Y2, t, c) == pytest.approx(E0, rel=1e-12)
        np.testing.assert_allclose(oracle.forces(Y2, t, c), F0 @ Q.T, atol=1e-12)


def test_gradient_descent_decreases_stress():
    _, _, t, Y = _random_case(200, 3, 1, 9)
    st = oracle.State.fresh(Y)
    c = 0.1
    E = [oracle.stress(st.Y, t, c)]
    for _ in range(40):
        oracle.step(st, t, c, oracle.OPT_MOMENTUM, a=0.0, b=0.002)
        E.append(oracle.stress(st.Y, t, c))
    assert all(e1 < e0 for e0, e1 in zip(E, E[1:]))


# ------------------------------------------------------- closed-form dynamics


def _recurrence(s0, w0, kstiff, a, b, n):
    """[s; w]_{n+1} = [[1 - b K, a], [-b K, a]] [s; w]_n for relative coordinate s."""
    A = np.array([[1 - b * kstiff, a], [-b * kstiff, a]])
    return np.linalg.matrix_power(A, n) @ np.array([s0, w0])


@pytest.mark.parametrize("dedup,stiff", [(False, 4.0), (True, 2.0)])
def test_single_nn_pair_collapses(dedup, stiff):
    # M = 2, k = 1: a mutual pair -> two nn terms (multiplicity) or one (dedup)
    knn = np.array([[1], [0]], np.int32)
    rn = np.full((2, 0), -1, np.int32)
    t = oracle.build_terms(knn, rn, dedup=dedup)
    a, b = 0.9, 0.01
    Y0 = np.array([[0.3, -0.2], [1.1, 0.5]])
    st = oracle.State.fresh(Y0)
    for n in (1, 5, 37, 200):
        st = oracle.State.fresh(Y0)
        oracle.run(st, t, 0.01, n, oracle.OPT_MOMENTUM, a=a, b=b)
        s = st.Y[0] - st.Y[1]
        for q in range(2):
            want = _recurrence(Y0[0, q] - Y0[1, q], 0.0, stiff, a, b, n)[0]
            assert s[q] == pytest.approx(want, abs=1e-12)
    st = oracle.State.fresh(Y0)
    oracle.run(st, t, 0.01, 3000, oracle.OPT_MOMENTUM, a=a, b=b)
    assert np.linalg.norm(st.Y[0] - st.Y[1]) < 1e-9


def test_single_rn_pair_settles_at_unit_distance():
    # one rn term: along the joining line the force is exactly c (1 - d), so the
    # separation error e = d - 1 follows the same recurrence with stiffness 2c.
    t = _terms([(0, 1, 1)], 2)
    c, a, b = 0.5, 0.9, 0.05
    Y0 = np.array([[0.0, 0.0], [0.24, 0.32]])  # d0 = 0.4 on a fixed direction
    u = Y0[1] / np.linalg.norm(Y0[1])
    for n in (1, 10, 60):
        st = oracle.State.fresh(Y0)
        oracle.run(st, t, c, n, oracle.OPT_MOMENTUM, a=a, b=b)
        d = np.linalg.norm(st.Y[1] - st.Y[0])
        want = 1.0 + _recurrence(0.4 - 1.0, 0.0, 2 * c, a, b, n)[0]
        assert d == pytest.approx(want, abs=1e-12)
        # motion stays on the line through the initial pair
        dirv = (st.Y[1] - st.Y[0]) / d
        assert np.abs(dirv - u).max() < 1e-12
    st = oracle.State.fresh(Y0)
    oracle.run(st, t, c, 2000, oracle.OPT_MOMENTUM, a=a, b=b)
    assert np.linalg.norm(st.Y[1] - st.Y[0]) == pytest.approx(1.0, abs=1e-9)


def test_rn_pair_at_zero_distance_has_no_force():
    t = _terms([(0, 1, 1), (1, 2, 0)], 3)
    Y = np.array([[0.5, 0.5], [0.5, 0.5], [1.0, 2.0]])
    F = oracle.forces(Y, t, 0.1)
    np.testing.assert_allclose(F[0], [0.0, 0.0], atol=0)
    np.testing.assert_allclose(F[1], Y[2] - Y[1], atol=1e-15)


def test_nesterov_matches_lookahead_definition():
    # on a single nn pair Nesterov is the linear map with the force taken at
    # s + a w:  w' = a w - bK (s + a w), s' = s + w'.
    knn = np.array([[1], [0]], np.int32)
    t = oracle.build_terms(knn, np.full((2, 0), -1, np.int32), dedup=True)
    a, b, K = 0.8, 0.05, 2.0
    A = np.array([[1 - b * K, a - b * K * a], [-b * K, a - b * K * a]])
    Y0 = np.array([[0.0, 0.0], [1.0, 0.0]])
    st = oracle.State.fresh(Y0)
    oracle.run(st, t, 0.01, 25, oracle.OPT_NESTEROV, a=a, b=b)
    want = (np.linalg.matrix_power(A, 25) @ np.array([-1.0, 0.0]))[0]
    assert (st.Y[0] - st.Y[1])[0] == pytest.approx(want, abs=1e-12)


def test_adadelta_first_steps_closed_form():
    # one nn pair (dedup): per coordinate g = -F; with zero accumulators the
    # first update is -sqrt(eps)/sqrt((1-rho) g^2 + eps) * g.
    knn = np.array([[1], [0]], np.int32)
    t = oracle.build_terms(knn, np.full((2, 0), -1, np.int32), dedup=True)
    rho, eps = 0.95, 1e-6
    Y0 = np.array([[0.0, 0.0], [2.0, -1.0]])
    st = oracle.State.fresh(Y0)
    oracle.step(st, t, 0.01, oracle.OPT_ADADELTA, rho=rho, eps=eps)
    g0 = -(Y0[1] - Y0[0])  # g for vertex 0 = (y0 - y1)
    dx = -np.sqrt(eps) / np.sqrt((1 - rho) * g0 ** 2 + eps) * g0
    np.testing.assert_allclose(st.Y[0], Y0[0] + dx, rtol=1e-14)
    np.testing.assert_allclose(st.S1[0], (1 - rho) * g0 ** 2, rtol=1e-14)
    np.testing.assert_allclose(st.S2[0], (1 - rho) * dx ** 2, rtol=1e-14)
    # Adadelta descends on a single pair
    E0 = oracle.stress(Y0, t, 0.01)
    oracle.run(st, t, 0.01, 200, oracle.OPT_ADADELTA, rho=rho, eps=eps)
    assert oracle.stress(st.Y, t, 0.01) < E0


# ---------------------------------------------------------------- kNN


def test_knn_on_a_line_textbook():
    # points 0, 1, ..., M-1 on a line: neighbours alternate left/right, the
    # left one first on ties (lower index), edges clipped at the ends.
    M, k = 40, 4
    X = np.arange(M, dtype=np.float32)[:, None] * 1.0
    out = oracle.knn_f32(X, k)
    for i in range(M):
        cand = sorted((abs(i - j), j) for j in range(M) if j != i)
        assert out[i].tolist() == [j for _, j in cand[:k]]
    assert out[10].tolist() == [9, 11, 8, 12]
    Xu = (np.arange(M, dtype=np.int64)[:, None] * 3).clip(0, 255).astype(np.uint8)
    assert np.array_equal(oracle.knn_u8(Xu, k), out)


def test_knn_matches_float64_brute_force_when_gaps_are_large():
    X, _ = synth.gaussian_mixture(300, 20, 3, 5)
    out = oracle.knn_f32(X, 6)
    D = ((X.astype(np.float64)[:, None, :] - X.astype(np.float64)[None, :, :]) ** 2).sum(-1)
    np.fill_diagonal(D, np.inf)
    ref = np.argsort(D, axis=1, kind="stable")[:, :6]
    srt = np.sort(D, axis=1)
    safe = (srt[:, 6] - srt[:, 5]) > 1e-3 * srt[:, 5]  # rows with no FP32 near-tie at the cut
    assert safe.mean() > 0.9
    for i in np.nonzero(safe)[0]:
        assert set(out[i].tolist()) == set(ref[i].tolist())
    rows = np.array([3, 77, 150], np.int64)
    assert np.array_equal(oracle.knn_f32(X, 6, rows), out[rows])


def test_knn_u8_integer_exact():
    X, _ = synth.mnist_like(200, 3, N=64)
    out = oracle.knn_u8(X, 5)
    D = ((X.astype(np.int64)[:, None, :] - X.astype(np.int64)[None, :, :]) ** 2).sum(-1)
    np.fill_diagonal(D, np.iinfo(np.int64).max)
    order = np.lexsort((np.broadcast_to(np.arange(200), D.shape), D), axis=1)[:, :5]
    assert np.array_equal(out, order)


@pytest.mark.parametrize("M,N,block", [(200, 64, 1024), (337, 784, 64), (97, 10, 13)])
def test_knn_u8_gemm_is_the_integer_exact_graph(M, N, block):
    """The GEMM form gives the serial definition's graph, ties and ragged blocks included."""
    X, _ = synth.mnist_like(M, 11, N=N)
    X[M // 2:M // 2 + 9] = X[3]                    # exact duplicates: ties decided by index
    X[M - 5:] = X[:5]
    k = 7
    D = ((X.astype(np.int64)[:, None, :] - X.astype(np.int64)[None, :, :]) ** 2).sum(-1)
    np.fill_diagonal(D, np.iinfo(np.int64).max)
    order = np.lexsort((np.broadcast_to(np.arange(M), D.shape), D), axis=1)[:, :k]
    got = oracle.knn_u8_gemm(X, k, block=block)
    assert np.array_equal(got, order)
    assert np.array_equal(got, oracle.knn_u8(X, k))


def test_knn_u8_gemm_on_a_line_textbook():
    M, k = 30, 4
    Xu = (np.arange(M, dtype=np.int64)[:, None] * 3).clip(0, 255).astype(np.uint8)
    out = oracle.knn_u8_gemm(Xu, k, block=7)
    assert out[10].tolist() == [9, 11, 8, 12]
    assert out[0].tolist() == [1, 2, 3, 4]
    assert out[M - 1].tolist() == [M - 2, M - 3, M - 4, M - 5]


# ---------------------------------------------------------------- metrics


@pytest.mark.parametrize("threads", [2, 3, 7, 64])
def test_threaded_qnx_and_cf_equal_the_serial_ones(threads):
    """Integer hit counts over row shares: exactly the serial value, ties included."""
    M, k = 1500, 6
    knn = synth.random_knn_graph(M, k, 21)
    Y = synth.uniform_positions(M, 22)
    Y[:400] = np.round(Y[:400] * 8) / 8           # exact ties in the 2-D neighbour search
    rows = synth.sample_rows(M, 41, 3)            # fewer rows than some thread counts
    for r in (rows, None):
        q, low = oracle.qnx(Y, knn, r, return_lowd=True)
        qt, lowt = oracle.qnx(Y, knn, r, return_lowd=True, threads=threads)
        assert qt == q and np.array_equal(lowt, low)
    lab = (np.arange(M) * 7 % 5).astype(np.int32)
    for nn in (2, 10, 100):
        assert oracle.cf(Y, lab, nn, rows, threads=threads) == oracle.cf(Y, lab, nn, rows)
        assert oracle.cf(Y, lab, nn, None, threads=threads) == oracle.cf(Y, lab, nn)


def test_qnx_identity_embedding_is_one():
    X = synth.uniform_positions(500, 4)
    knn = oracle.knn_f32(X, 5)
    assert oracle.qnx(X, knn) == 1.0


def test_qnx_random_embedding_is_k_over_m_minus_1():
    M, k = 3000, 10
    knn = synth.random_knn_graph(M, k, 6)
    Y = synth.uniform_positions(M, 99)
    rows = synth.sample_rows(M, 1500, 1)
    q = oracle.qnx(Y, knn, rows)
    mean = k / (M - 1)
    sd = np.sqrt(mean / (k * len(rows)))
    assert abs(q - mean) < 5 * sd


def test_qnx_ties_prefer_lower_index():
    # a 3x3 unit grid: the centre (id 4) has four neighbours at distance 1
    Y = np.array([[x, y] for y in range(3) for x in range(3)], np.float32)
    knn = np.tile(np.arange(2, dtype=np.int32), (9, 1))
    _, low = oracle.qnx(Y, knn, rows=np.array([4]), return_lowd=True)
    assert low[0].tolist() == [1, 3]


def test_cf_separated_and_mixed_labels():
    rng = np.random.default_rng(0)
    M = 600
    lab = np.repeat(np.arange(3), 200).astype(np.int32)
    Y = (rng.standard_normal((M, 2)) * 0.1 + lab[:, None] * 10.0).astype(np.float32)
    assert oracle.cf(Y, lab, 10) == 1.0
    lab_rand = rng.integers(0, 3, M).astype(np.int32)
    assert abs(oracle.cf(Y, lab_rand, 10) - 1 / 3) < 0.05


# ------------------------------------------------- late-stage and paper variants


@pytest.mark.parametrize("seed", [1, 4])
def test_l1_force_is_half_negative_gradient(seed):
    _, _, t, Y = _random_case(14, 3, 2, seed)
    c = 0.2
    F = oracle.forces(Y, t, c, metric="l1")
    h = 1e-7  # random coordinates: no |u| kink within h of any term
    G = np.zeros_like(Y)
    for i in range(t.M):
        for q in range(2):
            Yp, Ym = Y.copy(), Y.copy()
            Yp[i, q] += h
            Ym[i, q] -= h
            G[i, q] = (oracle.stress(Yp, t, c, "l1") - oracle.stress(Ym, t, c, "l1")) / (2 * h)
    assert np.abs(F + 0.5 * G).max() <= 1e-6 * np.abs(F).max()


def test_l1_symmetries_and_hand_value():
    _, _, t, Y = _random_case(40, 3, 1, 6)
    F = oracle.forces(Y, t, 0.1, metric="l1")
    assert np.abs(F.sum(axis=0)).max() <= 1e-12 * np.abs(F).sum()
    E = oracle.stress(Y, t, 0.1, "l1")
    swap = np.array([[0.0, 1.0], [1.0, 0.0]])       # symmetries of the l1 ball
    rot90 = np.array([[0.0, -1.0], [1.0, 0.0]])
    for Q in (swap, rot90, -np.eye(2)):
        assert oracle.stress(Y @ Q.T + 5.0, t, 0.1, "l1") == pytest.approx(E, rel=1e-12)
        np.testing.assert_allclose(oracle.forces(Y @ Q.T, t, 0.1, "l1"), F @ Q.T, atol=1e-12)
    # nn pair at (0,0)-(3,-4): d = 7, E = 49; force on 0 = d * sign(y_1 - y_0) = (7, -7)
    tt = _terms([(0, 1, 0)], 2)
    Yp = np.array([[0.0, 0.0], [3.0, -4.0]])
    assert oracle.stress(Yp, tt, 0.1, "l1") == 49.0
    np.testing.assert_array_equal(oracle.forces(Yp, tt, 0.1, "l1")[0], [7.0, -7.0])


def test_redraw_epoch_is_a_first_draw_with_a_mixed_seed():
    M, k, r, s = 500, 4, 2, 77
    knn = synth.random_knn_graph(M, k, 9)
    rn0, _ = oracle.random_neighbors(knn, r, s)
    assert np.array_equal(oracle.random_neighbors(knn, r, s, epoch=0)[0], rn0)
    gamma = 0x9E3779B97F4A7C15
    for e in (1, 2, 12345):
        mixed = oracle.splitmix64((e - gamma) % 2 ** 64, 0)   # = mix(e), pinned generator
        rn_e, _ = oracle.random_neighbors(knn, r, s, epoch=e)
        assert np.array_equal(rn_e, oracle.random_neighbors(knn, r, s ^ mixed)[0])
        assert (rn_e != rn0).mean() > 0.9


def test_absent_knn_entries():
    knn = np.array([[1, -1], [0, 2], [-1, -1], [2, 0]], np.int32)
    rn, _ = oracle.random_neighbors(knn, 1, 3)
    # vertex 2 has no own nn but is connected to 1 and 3 through their rows
    assert rn[2, 0] == 0
    t = oracle.build_terms(knn, np.full((4, 0), -1, np.int32))
    assert sorted(zip(t.ti.tolist(), t.tj.tolist())) == [(0, 1), (1, 0), (1, 2), (3, 0), (3, 2)]


def test_reverse_neighbour_restriction():
    knn = np.array([[1, 2], [0, 3], [3, 0], [2, 1]], np.int32)
    helper = np.array([[1, 2, 3], [0, 2, 3], [3, 1, 0], [2, 1, 0]], np.int32)
    out = oracle.restrict(knn, helper)
    # (i, j) survives iff i is in helper[j]
    want = [[j if (j >= 0 and i in helper[j]) else -1 for j in row] for i, row in enumerate(knn)]
    assert out.tolist() == want
    assert out.tolist() == [[1, 2], [0, 3], [3, 0], [2, 1]]
    helper2 = np.array([[1, 3, 3], [0, 0, 0], [3, 3, 3], [2, 2, 2]], np.int32)
    assert oracle.restrict(knn, helper2).tolist() == [[1, -1], [0, -1], [3, -1], [2, -1]]
    assert np.array_equal(oracle.restrict(knn, np.tile(np.arange(4), (4, 1)).astype(np.int32)),
                          knn)


def test_adaptive_b_rule_on_a_single_pair():
    # one nn pair (dedup): relative coordinate s, velocity w; F_0 - F_1 = -2 s
    knn = np.array([[1], [0]], np.int32)
    t = oracle.build_terms(knn, np.full((2, 0), -1, np.int32), dedup=True)
    st = oracle.State.fresh(np.array([[0.0, 0.0], [1.0, 0.0]]))
    box = [0.1]
    a, tau, g1, g2 = 0.9, 0.5, 1.1, 0.5
    assert oracle.step_adaptive(st, t, 0.01, box, a=a, tau=tau, gamma1=g1, gamma2=g2)  # T_old = 0
    v1 = st.S1.copy()
    np.testing.assert_allclose(v1, [[0.1, 0.0], [-0.1, 0.0]])
    # second attempt: F0 = y1 - y0 = 0.8, v' = 0.9 * 0.1 + 0.1 * 0.8 = 0.17 per particle
    # T_old = 2 * 0.01, T_new = 2 * 0.0289, dT / T_old = 1.89 > tau: rejected, b *= gamma2
    y_before = st.Y.copy()
    assert not oracle.step_adaptive(st, t, 0.01, box, a=a, tau=tau, gamma1=g1, gamma2=g2)
    assert box[0] == pytest.approx(0.05)
    np.testing.assert_array_equal(st.Y, y_before)
    np.testing.assert_array_equal(st.S1, v1)
    # third: v' = 0.09 + 0.05 * 0.8 = 0.13, dT / T_old = 0.69 > 0.5: rejected again -> b = 0.025
    assert not oracle.step_adaptive(st, t, 0.01, box, a=a, tau=tau, gamma1=g1, gamma2=g2)
    assert box[0] == pytest.approx(0.025)
    # fourth: v' = 0.09 + 0.02 = 0.11, dT / T_old = 0.21 < 0.5: accepted
    assert oracle.step_adaptive(st, t, 0.01, box, a=a, tau=tau, gamma1=g1, gamma2=g2)
    np.testing.assert_allclose(st.S1[0], [0.11, 0.0])
    np.testing.assert_allclose(st.Y[0], [0.21, 0.0])


# ---------------------------------------------------------------- MLP oracle


def test_mlp_bf16_rounding_values():
    from oracle import mlp

    x = np.array([1.0, 1.00390625, 1.005859375, 3.14159265, -2.0 ** -130, 65504.0])
    # BF16 keeps 8 significant bits: 1 + 2^-8 is a tie between 1 and 1 + 2^-7 -> even (1.0)
    want = np.array([1.0, 1.0, 1.0078125, 3.140625, -2.0 ** -130, 65536.0])
    np.testing.assert_array_equal(mlp.bf16(x), want)


def test_mlp_gradients_match_finite_differences():
    from oracle import mlp

    rng = np.random.default_rng(0)
    p = mlp.init_params(7, 5, 2, 3)
    p.b1 = rng.standard_normal(5) * 0.1
    p.b2 = rng.standard_normal(5) * 0.1
    X = rng.standard_normal((6, 7))
    T = rng.standard_normal((6, 2))
    L, g = mlp.loss_and_grads(p, X, T)
    h = 1e-6
    for n in p.names():
        w = getattr(p, n)
        num = np.zeros_like(w)
        for idx in np.ndindex(w.shape):
            q1, q2 = p.copy(), p.copy()
            getattr(q1, n)[idx] += h
            getattr(q2, n)[idx] -= h
            num[idx] = (mlp.loss_and_grads(q1, X, T)[0] - mlp.loss_and_grads(q2, X, T)[0]) / (2 * h)
        assert np.abs(num - g[n]).max() <= 1e-7 * max(1.0, np.abs(g[n]).max()), n


def test_mlp_gelu_and_adam_closed_forms():
    from oracle import mlp

    assert mlp.gelu(0.0) == 0.0
    assert mlp.gelu(1.0) == pytest.approx(0.8413447460685429)   # Phi(1)
    assert mlp.gelu_grad(0.0) == pytest.approx(0.5)
    # first Adam step moves every weight by lr * sign(g) (bias-corrected m / sqrt(v) = g / |g|)
    p = mlp.init_params(3, 2, 2, 1)
    g = {n: np.full_like(getattr(p, n), -0.3) for n in p.names()}
    before = p.copy()
    opt = mlp.Adam(lr=1e-3)
    opt.step(p, g)
    for n in p.names():
        np.testing.assert_allclose(getattr(p, n) - getattr(before, n), 1e-3 * (0.3 / (0.3 + 1e-8)),
                                   rtol=1e-12)


# ---------------------------------------------------------------- new points


def test_knn_query_on_a_line_textbook():
    # base points 0, 2, 4, ..., 38 on a line; a query at 5 is 1 from 4 and 6,
    # then 3 from 2 and 8: ties go to the lower index; a query on a base
    # point finds it first (nothing is excluded).
    X = (np.arange(20, dtype=np.float32) * 2)[:, None]
    Q = np.array([[5.0], [0.0], [38.5], [-7.0]], np.float32)
    out = oracle.knn_query(Q, X, 4)
    assert out[0].tolist() == [2, 3, 1, 4]
    assert out[1].tolist() == [0, 1, 2, 3]
    assert out[2].tolist() == [19, 18, 17, 16]
    assert out[3].tolist() == [0, 1, 2, 3]
    Xu = (np.arange(20) * 2).astype(np.uint8)[:, None]
    Qu = np.array([[5], [0], [38], [1]], np.uint8)
    assert oracle.knn_query(Qu, Xu, 3).tolist() == [[2, 3, 1], [0, 1, 2], [19, 18, 17],
                                                   [0, 1, 2]]


def test_knn_query_matches_float64_brute_force_and_integer_lexsort():
    Z, _ = synth.gaussian_mixture(490, 16, 4, 7)
    X, Q = Z[:400], Z[400:]
    out = oracle.knn_query(Q, X, 5)
    D = ((Q.astype(np.float64)[:, None, :] - X.astype(np.float64)[None, :, :]) ** 2).sum(-1)
    ref = np.argsort(D, axis=1, kind="stable")[:, :5]
    srt = np.sort(D, axis=1)
    safe = (srt[:, 5] - srt[:, 4]) > 1e-3 * srt[:, 4]
    assert safe.mean() > 0.9
    for i in np.nonzero(safe)[0]:
        assert set(out[i].tolist()) == set(ref[i].tolist())
    Zu, _ = synth.mnist_like(370, 3, N=48)
    Xu, Qu = Zu[:300], Zu[300:]
    Du = ((Qu.astype(np.int64)[:, None, :] - Xu.astype(np.int64)[None, :, :]) ** 2).sum(-1)
    order = np.lexsort((np.broadcast_to(np.arange(300), Du.shape), Du), axis=1)[:, :6]
    assert np.array_equal(oracle.knn_query(Qu, Xu, 6), order)


def test_knn_query_of_the_base_itself_is_self_then_the_knn_graph():
    X, _ = synth.gaussian_mixture(250, 12, 3, 2)
    q = oracle.knn_query(X, X, 5)
    assert np.array_equal(q[:, 0], np.arange(250))
    assert np.array_equal(q[:, 1:], oracle.knn_f32(X, 4))


def test_place_nn_is_the_neighbour_mean():
    Y = np.array([[0, 0], [2, 0], [0, 4], [6, 6]], np.float32)
    ids = np.array([[0, 1], [1, 2], [3, 3], [2, 0]], np.int32)
    assert oracle.place_nn(Y, ids).tolist() == [[1, 0], [1, 2], [6, 6], [0, 2]]
    # k = 1 is the embedding of the nearest neighbour itself
    assert oracle.place_nn(Y, ids[:, :1]).tolist() == Y[ids[:, 0]].tolist()


# ---------------------------------------------------------------- threaded timing mode


@pytest.mark.parametrize("opt", [oracle.OPT_MOMENTUM, oracle.OPT_NESTEROV, oracle.OPT_ADADELTA])
def test_run_threads_matches_serial_run(opt):
    _, _, t, Y = _random_case(400, 5, 1, 3)
    ref = oracle.State.fresh(Y)
    oracle.run(ref, t, 0.01, 20, opt, a=0.9, b=0.01)
    one = oracle.State.fresh(Y)
    oracle.run_threads(one, t, 0.01, 20, opt, a=0.9, b=0.01, threads=1)
    assert np.array_equal(one.Y, ref.Y) and np.array_equal(one.S1, ref.S1)
    for nt in (2, 3, 8):
        st = oracle.State.fresh(Y)
        oracle.run_threads(st, t, 0.01, 20, opt, a=0.9, b=0.01, threads=nt)
        assert np.abs(st.Y - ref.Y).max() <= 1e-12 * np.abs(ref.Y).max()
        assert np.abs(st.Y.mean(axis=0) - Y.mean(axis=0)).max() < 1e-12 or opt == 2


def test_run_threads_single_pair_recurrence():
    # two nn terms over five threads (three of them without a term) follow the
    # closed-form 2x2 recurrence of the pair's separation
    knn = np.array([[1], [0]], np.int32)
    t = oracle.build_terms(knn, np.full((2, 0), -1, np.int32))
    Y0 = np.array([[0.3, -0.2], [1.1, 0.5]])
    st = oracle.State.fresh(Y0)
    oracle.run_threads(st, t, 0.01, 37, oracle.OPT_MOMENTUM, a=0.9, b=0.01, threads=5)
    s = st.Y[0] - st.Y[1]
    for q in range(2):
        want = _recurrence(Y0[0, q] - Y0[1, q], 0.0, 4.0, 0.9, 0.01, 37)[0]
        assert s[q] == pytest.approx(want, abs=1e-12)


# ---------------------------------------------------------------- toy example


def test_two_hypertetrahedra_separate():
    # Sec. 3.3.1's toy: two regular 18-simplices (19 vertices each, all
    # pairwise distances equal) in 18-D, one rotated and translated away from
    # the other; with nn = 2, rn = 1, c = 0.1 the kNN graph has no edge
    # between them and the random neighbours push them apart, so every
    # vertex's 2 nearest embedded points lie in its own simplex
    rng = np.random.default_rng(3)
    simplex = np.eye(19)                              # regular, in a 18-D affine subspace
    Rm, _ = np.linalg.qr(rng.standard_normal((19, 19)))
    X = np.concatenate([simplex, simplex @ Rm + 10.0]).astype(np.float32)
    labels = np.repeat([0, 1], 19).astype(np.int32)
    knn = oracle.knn_f32(X, 2)
    assert np.all((knn // 19) == (np.arange(38) // 19)[:, None])   # no cross-simplex kNN edge
    rn, _ = oracle.random_neighbors(knn, 1, 7)
    terms = oracle.build_terms(knn, rn)
    st = oracle.State.fresh(oracle.init_positions(38, 7))
    oracle.run(st, terms, 0.1, 3000, oracle.OPT_MOMENTUM, a=0.9, b=0.01)
    assert oracle.cf(st.Y.astype(np.float32), labels, 2) == 1.0
    # the two simplices end apart: centroid distance above the largest radius
    c0, c1 = st.Y[:19].mean(0), st.Y[19:].mean(0)
    radius = max(np.linalg.norm(st.Y[:19] - c0, axis=1).max(),
                 np.linalg.norm(st.Y[19:] - c1, axis=1).max())
    assert np.linalg.norm(c0 - c1) > radius
