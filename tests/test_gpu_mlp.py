"""Learned warm start: the MLP's forward pass, gradients and Adam step vs the FP64 oracle.

Layer by layer, element by element: every intermediate array of the GPU
network (read back with ``ivhd_mlp_activations``) and every gradient is
compared with the oracle's formula evaluated on the GPU's own inputs to that
layer, within the bound its arithmetic allows (``mlp_bounds``: the FP32
accumulation bound of a K-term dot product, FP32 GELU error, and a BF16 store
that may round either way only where its interval straddles a rounding
boundary).  The input conversion is bit-exact.

The whole network is also compared with the oracle run from the original
inputs (BF16 rounding emulated at the same points).  There a BF16 store
whose FP32 value lies next to a rounding boundary may land on the other side
and move one element by a BF16 step (2^-8 relative), which then propagates;
that composition is checked norm-wise.
"""
import numpy as np
import pytest
import torch

from mlp_bounds import U, assert_bf16_store, assert_within, dot_radius, gamma, gelu_fp32_radius
from oracle import mlp as omlp
from paper_2303_05455_gb300 import ivhd, synth

pytestmark = pytest.mark.gpu


def flat(p):
    return np.concatenate([getattr(p, n).ravel() for n in p.names()]).astype(np.float32)


def unflat(v, n_in, H):
    sizes = [(H, n_in), (H,), (H, H), (H,), (2, H), (2,)]
    out, o = [], 0
    for s in sizes:
        n = int(np.prod(s))
        out.append(v[o:o + n].reshape(s).astype(np.float64))
        o += n
    return omlp.Params(*out)


def setup(B=256, n_in=784, H=512, seed=5):
    X, _ = synth.mnist_like(B, seed, N=n_in)
    p = omlp.init_params(n_in, H, 2, seed)
    rng = np.random.default_rng(seed)
    p.b1 = rng.standard_normal(H) * 0.1
    p.b2 = rng.standard_normal(H) * 0.1
    p.b3 = rng.standard_normal(2) * 0.1
    T = rng.standard_normal((B, 2))
    net = ivhd.MLP(n_in, H, max_batch=4096)
    net.set_params(flat(p))
    p32 = unflat(flat(p), n_in, H)      # the FP32 master values, as the GPU holds them
    return X, T, net, p32


def rel(a, b):
    return np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b)


def test_forward_matches_oracle():
    X, T, net, p = setup()
    y = net.forward(torch.from_numpy(X).cuda(), x_scale=1 / 255).cpu().numpy()
    y_ref, _ = omlp.forward(p, X.astype(np.float32) / np.float32(255), emulate_bf16=True)
    assert rel(y, y_ref) < 1e-3


def test_gradients_and_loss_match_oracle():
    X, T, net, p = setup()
    loss, g = net.loss_grad(torch.from_numpy(X).cuda(), torch.from_numpy(T).float().cuda(),
                            x_scale=1 / 255)
    L_ref, g_ref = omlp.loss_and_grads(p, X.astype(np.float32) / np.float32(255), T,
                                       emulate_bf16=True)
    assert loss == pytest.approx(L_ref, rel=1e-4)
    gp = unflat(g.cpu().numpy(), 784, 512)
    for n in p.names():
        assert rel(getattr(gp, n), g_ref[n]) < 5e-3, n


def test_each_layer_matches_oracle_at_its_own_inputs():
    B, n_in, H = 256, 784, 512
    X, T, net, p = setup(B, n_in, H)
    T32 = T.astype(np.float32).astype(np.float64)
    loss, g = net.loss_grad(torch.from_numpy(X).cuda(), torch.from_numpy(T).float().cuda(),
                            x_scale=1 / 255)
    a = {n: net.activations(n).astype(np.float64)
         for n in ("x", "z1", "h1", "z2", "h2", "y", "dy", "dz2", "dz1")}
    # input rows: x * fl32(1/255) in FP32, rounded to BF16 -- bit-exact
    x_ref = omlp.bf16(X.astype(np.float32) * np.float32(1 / 255))
    assert np.array_equal(a["x"], x_ref)
    W1, W2 = omlp.bf16(p.W1), omlp.bf16(p.W2)          # the BF16 weight copies
    # forward: pre-activations are K-term FP32 dot products, activations BF16 stores
    z1 = a["x"] @ W1.T + p.b1
    assert_within(a["z1"], z1, dot_radius(a["x"], W1.T, bias=p.b1), "z1")
    assert_bf16_store(a["h1"], omlp.gelu(a["z1"]), gelu_fp32_radius(a["z1"]), "h1")
    z2 = a["h1"] @ W2.T + p.b2
    assert_within(a["z2"], z2, dot_radius(a["h1"], W2.T, bias=p.b2), "z2")
    assert_bf16_store(a["h2"], omlp.gelu(a["z2"]), gelu_fp32_radius(a["z2"]), "h2")
    y = a["h2"] @ p.W3.T + p.b3
    assert_within(a["y"], y, dot_radius(a["h2"], p.W3.T, bias=p.b3), "y")
    # loss and backward
    dy = 2.0 * (a["y"] - T32) / B
    assert_within(a["dy"], dy, 4 * U * np.abs(dy), "dY")
    assert loss == pytest.approx(((a["y"] - T32) ** 2).sum() / B, rel=1e-6)
    gp = unflat(g.cpu().numpy(), n_in, H)
    assert_within(gp.W3, a["dy"].T @ a["h2"], dot_radius(a["dy"].T, a["h2"]), "dW3")
    assert_within(gp.b3, a["dy"].sum(axis=0), gamma(B) * np.abs(a["dy"]).sum(axis=0), "db3")
    dh2 = a["dy"] @ p.W3
    gg2 = omlp.gelu_grad(a["z2"])
    pre2 = dh2 * gg2
    r2 = (dot_radius(a["dy"], p.W3) * np.abs(gg2) + np.abs(dh2) * gelu_fp32_radius(a["z2"])
          + 2 * U * np.abs(pre2))
    assert_bf16_store(a["dz2"], pre2, r2, "dZ2")
    assert_within(gp.W2, a["dz2"].T @ a["h1"], dot_radius(a["dz2"].T, a["h1"], 8), "dW2")
    assert_within(gp.b2, a["dz2"].sum(axis=0), gamma(B) * np.abs(a["dz2"]).sum(axis=0), "db2")
    dh1 = a["dz2"] @ W2
    gg1 = omlp.gelu_grad(a["z1"])
    pre1 = dh1 * gg1
    r1 = (dot_radius(a["dz2"], W2) * np.abs(gg1) + np.abs(dh1) * gelu_fp32_radius(a["z1"])
          + 2 * U * np.abs(pre1))
    assert_bf16_store(a["dz1"], pre1, r1, "dZ1")
    assert_within(gp.W1, a["dz1"].T @ a["x"], dot_radius(a["dz1"].T, a["x"], 8), "dW1")
    assert_within(gp.b1, a["dz1"].sum(axis=0), gamma(B) * np.abs(a["dz1"]).sum(axis=0), "db1")
    # the bounds are tight enough to mean something: a few BF16 stores at most may round
    # the other way, and the FP32 accumulation radius stays far below the values
    for n, pre, rr in (("dz1", pre1, r1), ("dz2", pre2, r2)):
        assert (a[n] != omlp.bf16(pre)).mean() < 0.01, n
    assert np.median(dot_radius(a["x"], W1.T, bias=p.b1) / (np.abs(z1) + 1e-30)) < 1e-2


def test_adam_step_matches_closed_form():
    X, T, net, p = setup(B=128)
    xt = torch.from_numpy(X).cuda()
    tt = torch.from_numpy(T).float().cuda()
    _, g = net.loss_grad(xt, tt, x_scale=1 / 255)
    w0 = net.get_params().astype(np.float64)
    net.train_step(xt, tt, lr=1e-3, x_scale=1 / 255)
    w1 = net.get_params().astype(np.float64)
    gg = g.cpu().numpy().astype(np.float64)
    m = 0.1 * gg
    v = 0.001 * gg * gg
    want = w0 - 1e-3 * (m / 0.1) / (np.sqrt(v / 0.001) + 1e-8)
    # the update itself (~lr) is exact to 1e-5; the FP32 weight it is added to rounds
    # to a few units in its last place
    ulp = np.spacing(np.abs(w0).astype(np.float32)).astype(np.float64)
    assert np.all(np.abs(w1 - want) <= 4 * ulp + 1e-5 * np.abs(want - w0))


def test_training_fits_and_chunked_forward_is_consistent():
    n_in, H = 64, 128
    rng = np.random.default_rng(3)
    X = rng.standard_normal((8192, n_in)).astype(np.float32)
    P = rng.standard_normal((n_in, 2)) / np.sqrt(n_in)
    T = np.tanh(X @ P) * 3.0
    net = ivhd.MLP(n_in, H, max_batch=1024)
    net.set_params(flat(omlp.init_params(n_in, H, 2, 1)))
    xt = torch.from_numpy(X).cuda()
    tt = torch.from_numpy(T).float().cuda()
    first = net.train_step(xt[:1024], tt[:1024], lr=3e-3, want_loss=True)
    for it in range(400):
        b = (it % 8) * 1024
        net.train_step(xt[b:b + 1024], tt[b:b + 1024], lr=3e-3)
    last = net.train_step(xt[:1024], tt[:1024], lr=3e-3, want_loss=True)
    assert last < 0.1 * first
    y = net.forward(xt[:3000])
    y_parts = torch.cat([net.forward(xt[:1000]), net.forward(xt[1000:3000])])
    assert torch.equal(y, y_parts)


def test_forward_rows_do_not_depend_on_the_chunking():
    """Rows are independent: each output element's K sum runs in the same order
    whatever the number of rows or the tile width, so a row's output is the
    same bits in any chunk, including a ragged last chunk (8,197 rows, not a
    multiple of 8) and a slice that crosses a chunk boundary, and with a
    network whose chunks are 16 times larger."""
    n_in, H = 784, 512
    X, _ = synth.mnist_like(8197, 11, N=n_in)
    p = flat(omlp.init_params(n_in, H, 2, 4))
    xd = torch.from_numpy(X).cuda()
    small = ivhd.MLP(n_in, H, max_batch=512)
    large = ivhd.MLP(n_in, H, max_batch=8192)
    small.set_params(p)
    large.set_params(p)
    y = small.forward(xd, x_scale=1 / 255)
    assert y.shape == (8197, 2) and torch.isfinite(y).all()
    assert torch.equal(y, large.forward(xd, x_scale=1 / 255))
    assert torch.equal(y[500:1037], small.forward(xd[500:1037], x_scale=1 / 255))
    assert torch.equal(y[8190:], large.forward(xd[8190:], x_scale=1 / 255))
    small.close()
    large.close()


def test_replayed_training_steps_follow_adam():
    """From the second step at a batch size on, the step is a replayed CUDA graph whose
    input, target and learning-rate nodes are patched per call: with new batches at new
    addresses every step, each update still equals Adam's closed form from that batch's
    gradient (computed by the direct path)."""
    B = 256
    X, T, net, p = setup(B=4 * B)
    xs = [torch.from_numpy(X[i * B:(i + 1) * B].copy()).cuda() for i in range(4)]
    ts = [torch.from_numpy(T[i * B:(i + 1) * B].copy()).float().cuda() for i in range(4)]
    m = v = None
    w = net.get_params().astype(np.float64)
    lrs = [1e-3, 2e-3, 5e-4, 1e-3]
    u = 2.0 ** -24
    for t in range(1, 5):
        loss_g, g = net.loss_grad(xs[t - 1], ts[t - 1], x_scale=1 / 255)
        g = g.cpu().numpy().astype(np.float64)
        loss = net.train_step(xs[t - 1], ts[t - 1], lr=lrs[t - 1], x_scale=1 / 255, want_loss=True)
        assert loss == loss_g
        m_prev = np.zeros_like(g) if m is None else m
        m = 0.1 * g if m is None else 0.9 * m + 0.1 * g
        v = 0.001 * g * g if v is None else 0.999 * v + 0.001 * g * g
        c1, c2 = 1 - 0.9 ** t, 1 - 0.999 ** t
        den = np.sqrt(v / c2) + 1e-8
        want = w - lrs[t - 1] * (m / c1) / den
        w_new = net.get_params().astype(np.float64)
        ulp = np.spacing(np.abs(w).astype(np.float32)).astype(np.float64)
        # FP32 state and arithmetic: the weight's own rounding, a relative error of the
        # update, and the first moment's rounding relative to its terms (0.9 m + 0.1 g
        # may cancel), carried over the steps
        mom = lrs[t - 1] / c1 * 32 * t * u * (0.9 * np.abs(m_prev) + 0.1 * np.abs(g)) / den
        assert np.all(np.abs(w_new - want) <= 4 * ulp + 1e-5 * np.abs(want - w) + mom), t
        w = w_new
