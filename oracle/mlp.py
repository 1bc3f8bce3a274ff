"""FP64 reference of the learned warm start -- TEST INFRASTRUCTURE ONLY.

A multilayer perceptron  x -> GELU(W1 x + b1) -> GELU(W2 h1 + b2) -> W3 h2 + b3
(784 -> 512 -> 512 -> 2 for the MNIST-shaped data) regressing the 2-D IVHD
embedding of each point with the mean squared error
    L = (1/B) sum_b |y_b - t_b|^2,
trained with Adam (Kingma and Ba, 2015: bias corrections 1 - beta^t; the
paper's Adam formula in Sec. 3.3.2 prints (1 - gamma)^(i-1), read as garbled).
The paper has no such network for IVHD; its closest passages are the
parametric t-SNE / UMAP maps of Sec. 2 and IVHD as an initial configuration
(Sec. 3.4).  GELU is the exact form x Phi(x).

With ``emulate_bf16`` the values the GPU keeps in BF16 (inputs, weights, the
activations h1 and h2, and the back-propagated dz1 and dz2) are rounded to
BF16 (round to nearest even) at the same points, so that a comparison with
the GPU isolates the order of FP32 accumulation.
"""
from __future__ import annotations

import dataclasses

import numpy as np
from scipy.special import erf


def bf16(x) -> np.ndarray:
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    f = np.ascontiguousarray(x, np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


@dataclasses.dataclass
class Params:
    W1: np.ndarray
    b1: np.ndarray
    W2: np.ndarray
    b2: np.ndarray
    W3: np.ndarray
    b3: np.ndarray

    def names(self):
        return ["W1", "b1", "W2", "b2", "W3", "b3"]

    def copy(self):
        return Params(*[getattr(self, n).copy() for n in self.names()])


def init_params(n_in: int, hidden: int, n_out: int, seed: int) -> Params:
    """He-uniform weights (bound sqrt(6 / fan_in)), zero biases, from numpy PCG64."""
    rng = np.random.Generator(np.random.PCG64(seed))

    def u(fo, fi):
        lim = np.sqrt(6.0 / fi)
        return rng.uniform(-lim, lim, size=(fo, fi))

    return Params(u(hidden, n_in), np.zeros(hidden), u(hidden, hidden), np.zeros(hidden),
                  u(n_out, hidden) * 0.1, np.zeros(n_out))


def forward(p: Params, X, emulate_bf16: bool = False):
    r = bf16 if emulate_bf16 else (lambda a: np.asarray(a, np.float64))
    X = r(X)
    W1, W2 = r(p.W1), r(p.W2)
    Z1 = X @ W1.T + p.b1
    H1 = r(gelu(Z1))
    Z2 = H1 @ W2.T + p.b2
    H2 = r(gelu(Z2))
    Y = H2 @ p.W3.T + p.b3
    return Y, (X, Z1, H1, Z2, H2, W1, W2)


def loss_and_grads(p: Params, X, T, emulate_bf16: bool = False):
    """Mean squared error and its gradient with respect to every parameter."""
    r = bf16 if emulate_bf16 else (lambda a: np.asarray(a, np.float64))
    B = X.shape[0]
    Y, (Xr, Z1, H1, Z2, H2, W1, W2) = forward(p, X, emulate_bf16)
    D = Y - T
    L = float((D * D).sum() / B)
    dY = 2.0 * D / B
    g = {}
    g["W3"] = dY.T @ H2
    g["b3"] = dY.sum(axis=0)
    dZ2 = r((dY @ p.W3) * gelu_grad(Z2))
    g["W2"] = dZ2.T @ H1
    g["b2"] = dZ2.sum(axis=0)
    dZ1 = r((dZ2 @ W2) * gelu_grad(Z1))
    g["W1"] = dZ1.T @ Xr
    g["b1"] = dZ1.sum(axis=0)
    return L, g


@dataclasses.dataclass
class Adam:
    lr: float = 1e-3
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8
    t: int = 0
    m: dict = dataclasses.field(default_factory=dict)
    v: dict = dataclasses.field(default_factory=dict)

    def step(self, p: Params, g: dict):
        self.t += 1
        for n in p.names():
            w = getattr(p, n)
            m = self.m.get(n, np.zeros_like(w))
            v = self.v.get(n, np.zeros_like(w))
            m = self.beta1 * m + (1 - self.beta1) * g[n]
            v = self.beta2 * v + (1 - self.beta2) * g[n] ** 2
            mh = m / (1 - self.beta1 ** self.t)
            vh = v / (1 - self.beta2 ** self.t)
            setattr(p, n, w - self.lr * mh / (np.sqrt(vh) + self.eps))
            self.m[n], self.v[n] = m, v
