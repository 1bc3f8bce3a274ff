"""Per-element bound on the displacement of one IVHD step, GPU (FP32) vs oracle (FP64).

The step's displacement y' - y is compared element by element within

    1e-5 * max |y'_ref - y|                 (the relative bar of the one-step tests)
  + d(y')/dF * force_error_bound            (the force's FP32 summation error, carried
                                             through the optimiser's sensitivity)
  + a few roundings of the update itself
  + 2^-21 (|y'| + a |v| + |y' - y|)          (storing y', and Nesterov's look-ahead point,
                                             in FP32)

force_error_bound: the FP32 sum of n terms in any order is within gamma(n) times
the sum of their magnitudes (gamma(n) taken as 2 n u, u = 2^-24), with 8 extra
terms' worth for the rounding inside each term.  Sensitivities: b for momentum
and Nesterov; for Adadelta (Sec. 3.3.2, Zeiler's form) |d dx / d g| =
sqrt(E[dx^2] + eps) (rho E[g^2] + eps) / (E[g^2]' + eps)^(3/2).
"""
import numpy as np

U32 = 2.0 ** -24


def force_error_bound(y, terms, c):
    """Per element: 2 (n + 8) u * sum of |term| over the n terms acting on it, with each
    rn term's magnitude taken as c (2 + 4 d) / d |u| (covers its own FP32 evaluation)."""
    y = np.asarray(y, np.float64)
    u = y[terms.ti] - y[terms.tj]
    d = np.sqrt((u * u).sum(axis=1))
    mag = np.abs(u)
    rn = terms.kind == 1
    safe = np.where(d > 0, d, 1.0)
    mag[rn] *= np.where(d[rn] > 0, c * (2.0 + 4.0 * d[rn]) / safe[rn], 0.0)[:, None]
    M = y.shape[0]
    ends = np.concatenate([terms.ti, terms.tj])
    A = np.stack([np.bincount(ends, np.concatenate([mag[:, q], mag[:, q]]), minlength=M)
                  for q in (0, 1)], axis=1)
    n = np.bincount(ends, minlength=M).astype(np.float64)
    return 2.0 * (n[:, None] + 8.0) * U32 * A


def step_bound(opt, y_ref1, d_ref, F_ref, F_err, a, b, v0=None, s1=None, s2=None,
               rho=0.95, eps=1e-6):
    """Per-element bound on |(y'_gpu - y) - (y'_ref - y)| for one step (see module docstring).

    v0 / s1, s2: the optimiser state the step starts from (zeros if None)."""
    if opt in ("momentum", "nesterov"):
        sens = b
        own = 4 * U32 * (np.abs(d_ref) + (0 if v0 is None else a * np.abs(v0)))
    else:
        g = -F_ref
        Eg0 = 0.0 if s1 is None else s1
        Ex0 = 0.0 if s2 is None else s2
        Eg = rho * Eg0 + (1 - rho) * g * g
        sens = np.sqrt(Ex0 + eps) * (rho * Eg0 + eps) / (Eg + eps) ** 1.5
        own = 10 * U32 * np.abs(d_ref)
    store = 2.0 ** -21 * (np.abs(y_ref1) + (0 if v0 is None else a * np.abs(v0)) + np.abs(d_ref))
    return 1e-5 * np.abs(d_ref).max() + sens * F_err + own + store


def close_elem(got, ref, bound, what=""):
    got = np.asarray(got, np.float64)
    err = np.abs(got - ref)
    bad = err > bound
    assert not bad.any(), (what, int(bad.sum()), float(err[bad].max()), float(bound[bad].min()))
