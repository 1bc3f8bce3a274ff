"""Element-wise bounds for one layer of the warm-start network at given inputs.

Each layer of the GPU network is checked against the FP64 oracle's formula
(``oracle/mlp.py``) evaluated on the GPU's own inputs to that layer, which are
exact BF16 or FP32 values read back with ``ivhd_mlp_activations``.  What can
differ is then only the arithmetic of that layer, and it is bounded element by
element:

* A K-term dot product of exact operands accumulated in FP32 in any order is
  within gamma(K) * sum |a_k| |b_k| of the exact sum (gamma(K) =
  K u / (1 - K u) for round-to-nearest, u = 2^-24; taken as 2 K u, which also
  covers accumulators that round by truncation).
* GELU and its derivative in FP32 (erff / expf and a few roundings) are within
  8 u (1 + |z|) of the exact functions.
* A BF16 store rounds an FP32 value v that lies within r of the exact value:
  the stored value is bf16(exact) unless [exact - r, exact + r] contains a
  BF16 rounding boundary, in which case it may be the rounding of either end.

Composed over the whole network these bounds cascade (every BF16 store whose
interval straddles a boundary passes a full BF16 step on), which is why the
whole network is compared with the oracle norm-wise and each layer element by
element.
"""
from __future__ import annotations

import numpy as np

from oracle import mlp as omlp

U = 2.0 ** -24


def gamma(K: int) -> float:
    return 2.0 * K * U


def bf16_interval(pre, r):
    """Largest |bf16(v) - bf16(pre)| over |v - pre| <= r."""
    lo, hi, mid = omlp.bf16(pre - r), omlp.bf16(pre + r), omlp.bf16(pre)
    return np.maximum(np.abs(hi - mid), np.abs(lo - mid))


def gelu_fp32_radius(z):
    return 8 * U * (1.0 + np.abs(z))


def dot_radius(A, B, extra_terms: int = 0, bias=None):
    """gamma(K) * (|A| @ |B| + |bias|) for A @ B + bias with inner dimension K."""
    acc = np.abs(A) @ np.abs(B)
    if bias is not None:
        acc = acc + np.abs(bias)
    return gamma(A.shape[1] + 1 + extra_terms) * acc


def assert_within(got, ref, rad, what):
    got = np.asarray(got, np.float64)
    assert got.shape == ref.shape, (what, got.shape, ref.shape)
    err = np.abs(got - ref)
    bad = err > rad
    assert not bad.any(), (what, int(bad.sum()), float(err[bad].max()), float(rad[bad].min()))


def assert_bf16_store(got, pre, r, what):
    """got = a BF16 store of an FP32 value within r of the exact pre-store value."""
    assert_within(got, omlp.bf16(pre), bf16_interval(pre, r), what)
