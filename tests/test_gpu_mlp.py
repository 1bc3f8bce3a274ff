"""Learned warm start: the MLP's forward pass, gradients and Adam step vs the FP64 oracle.

The oracle rounds to BF16 at the points where the GPU stores BF16 (inputs,
W1/W2 copies, h1, h2, dz1, dz2), so the comparison isolates FP32 accumulation
order; a BF16 rounding that lands on the other side of a tie moves one element
by 2^-8 relative, hence the norm-wise tolerances below.
"""
import numpy as np
import pytest
import torch

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
