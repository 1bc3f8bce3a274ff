"""FP64 CPU oracle for the IVHD embedding iteration -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never calls it, and it
never calls the CUDA library.  The arithmetic lives in ``ivhd_oracle.c``; this
module marshals numpy arrays through ctypes and adds nothing to the method.

Functions mirror the paper's steps (see the C file's header for citations and
the readings taken where the paper is ambiguous):

* ``random_neighbors`` -- fixed random neighbours O_rn(i), SplitMix64 draws.
* ``init_positions``   -- y0 ~ U(0,1)^2 from SplitMix64.
* ``build_terms``      -- the nn / rn term list of the stress (Eq. 3.16).
* ``stress``, ``forces`` -- E and F = -1/2 grad E.
* ``step`` / ``run``   -- momentum (force-directed), Nesterov, Adadelta.
* ``run_threads``      -- ``run`` on several host threads (CPU timing).
* ``knn_f32`` / ``knn_u8`` -- exact brute-force kNN.
* ``knn_u8_gemm``      -- the same uint8 kNN graph as ``knn_u8`` for full-size
  inputs, its integer distances formed with a float64 matrix product.
* ``knn_query``, ``place_nn`` -- kNN of new points in a base set and their
  placement at the mean embedding of those neighbours (Progressive UMAP).
* ``qnx``, ``cf``      -- Q_NX(k) and neighbour hit cf_nn (``threads`` > 1
  splits the sampled rows over host threads; integer hit counts, so the
  result is the serial one exactly).
"""
from __future__ import annotations

import ctypes
import dataclasses

import numpy as np

from .build import build_oracle

OPT_MOMENTUM, OPT_NESTEROV, OPT_ADADELTA = 0, 1, 2

_lib = None


def _L():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build_oracle())
        P = ctypes.c_void_p
        i64, i32, u64, dbl = ctypes.c_int64, ctypes.c_int, ctypes.c_uint64, ctypes.c_double
        lib.ivo_splitmix64.argtypes = [u64, u64]
        lib.ivo_splitmix64.restype = u64
        lib.ivo_random_neighbors.argtypes = [P, i64, i32, i32, u64, P]
        lib.ivo_random_neighbors.restype = i64
        lib.ivo_random_neighbors_epoch.argtypes = [P, i64, i32, i32, u64, u64, P]
        lib.ivo_random_neighbors_epoch.restype = i64
        lib.ivo_restrict.argtypes = [P, P, i64, i32, i32, P]
        lib.ivo_restrict.restype = None
        lib.ivo_stress_l1.argtypes = [P, P, P, P, i64, dbl]
        lib.ivo_stress_l1.restype = dbl
        lib.ivo_forces_l1.argtypes = [P, i64, P, P, P, i64, dbl, P]
        lib.ivo_forces_l1.restype = None
        lib.ivo_step_l1.argtypes = [i32, P, P, i64, P, P, P, i64, dbl, dbl, dbl, P, P]
        lib.ivo_step_l1.restype = None
        lib.ivo_step_adaptive.argtypes = [i32, i32, P, P, i64, P, P, P, i64, dbl, dbl, P, dbl,
                                          dbl, dbl, P, P, P, P]
        lib.ivo_step_adaptive.restype = i32
        lib.ivo_init_positions.argtypes = [i64, u64, P]
        lib.ivo_init_positions.restype = None
        lib.ivo_build_terms.argtypes = [P, P, i64, i32, i32, i32, P, P, P]
        lib.ivo_build_terms.restype = i64
        lib.ivo_stress.argtypes = [P, P, P, P, i64, dbl]
        lib.ivo_stress.restype = dbl
        lib.ivo_forces.argtypes = [P, i64, P, P, P, i64, dbl, P]
        lib.ivo_forces.restype = None
        lib.ivo_step.argtypes = [i32, P, P, P, i64, P, P, P, i64, dbl, dbl, dbl, dbl, dbl, P, P]
        lib.ivo_step.restype = None
        lib.ivo_run.argtypes = [i32, P, P, P, i64, P, P, P, i64, dbl, dbl, dbl, dbl, dbl, i64]
        lib.ivo_run.restype = i32
        lib.ivo_run_threads.argtypes = [i32, P, P, P, i64, P, P, P, i64, dbl, dbl, dbl, dbl, dbl,
                                        i64, i32]
        lib.ivo_run_threads.restype = i32
        lib.ivo_knn_f32.argtypes = [P, i64, i32, i32, P, i64, P]
        lib.ivo_knn_f32.restype = i32
        lib.ivo_knn_u8.argtypes = [P, i64, i32, i32, P, i64, P]
        lib.ivo_knn_u8.restype = i32
        lib.ivo_knn_query_f32.argtypes = [P, i64, P, i64, i32, i32, P]
        lib.ivo_knn_query_f32.restype = i32
        lib.ivo_knn_query_u8.argtypes = [P, i64, P, i64, i32, i32, P]
        lib.ivo_knn_query_u8.restype = i32
        lib.ivo_place_nn.argtypes = [P, P, i64, i32, P]
        lib.ivo_place_nn.restype = None
        lib.ivo_qnx.argtypes = [P, i64, P, i32, P, i64, P]
        lib.ivo_qnx.restype = dbl
        lib.ivo_cf.argtypes = [P, i64, P, i32, P, i64]
        lib.ivo_cf.restype = dbl
        lib.ivo_qnx_threads.argtypes = [P, i64, P, i32, P, i64, P, i32]
        lib.ivo_qnx_threads.restype = dbl
        lib.ivo_cf_threads.argtypes = [P, i64, P, i32, P, i64, i32]
        lib.ivo_cf_threads.restype = dbl
        _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def splitmix64(seed: int, t: int) -> int:
    return int(_L().ivo_splitmix64(seed & 0xFFFFFFFFFFFFFFFF, t))


def random_neighbors(knn, r: int, seed: int, epoch: int = 0):
    """Returns (rn int32 [M, r] with -1 for unfillable slots, number of -1 slots).

    epoch > 0 is a redraw with the seed replaced by seed ^ mix(epoch)."""
    knn = _c(knn, np.int32)
    M, k = knn.shape
    rn = np.empty((M, max(r, 1)), dtype=np.int32)[:, :r]
    rn = np.ascontiguousarray(rn)
    empty = _L().ivo_random_neighbors_epoch(_p(knn), M, k, r, seed & 0xFFFFFFFFFFFFFFFF,
                                            epoch & 0xFFFFFFFFFFFFFFFF, _p(rn))
    return rn, int(empty)


def restrict(knn, helper) -> np.ndarray:
    """Reverse-neighbour restriction: keep (i, j) iff i is in helper row j, else -1."""
    knn = _c(knn, np.int32)
    helper = _c(helper, np.int32)
    M, k = knn.shape
    out = np.empty_like(knn)
    _L().ivo_restrict(_p(knn), _p(helper), M, k, helper.shape[1], _p(out))
    return out


def init_positions(M: int, seed: int) -> np.ndarray:
    Y = np.empty((M, 2), dtype=np.float64)
    _L().ivo_init_positions(M, seed & 0xFFFFFFFFFFFFFFFF, _p(Y))
    return Y


@dataclasses.dataclass
class Terms:
    ti: np.ndarray
    tj: np.ndarray
    kind: np.ndarray
    M: int

    @property
    def T(self) -> int:
        return int(self.ti.shape[0])


def build_terms(knn, rn, dedup: bool = False) -> Terms:
    knn = _c(knn, np.int32)
    M, k = knn.shape
    rn = _c(rn, np.int32).reshape(M, -1)
    r = rn.shape[1]
    cap = max(1, M * (k + r))
    ti = np.empty(cap, np.int64)
    tj = np.empty(cap, np.int64)
    kind = np.empty(cap, np.int8)
    T = _L().ivo_build_terms(_p(knn), _p(rn), M, k, r, int(dedup), _p(ti), _p(tj), _p(kind))
    return Terms(ti[:T].copy(), tj[:T].copy(), kind[:T].copy(), M)


def stress(Y, terms: Terms, c: float, metric: str = "l2") -> float:
    Y = _c(Y, np.float64)
    fn = _L().ivo_stress_l1 if metric == "l1" else _L().ivo_stress
    return float(fn(_p(Y), _p(terms.ti), _p(terms.tj), _p(terms.kind), terms.T, c))


def forces(Y, terms: Terms, c: float, metric: str = "l2") -> np.ndarray:
    Y = _c(Y, np.float64)
    F = np.empty_like(Y)
    fn = _L().ivo_forces_l1 if metric == "l1" else _L().ivo_forces
    fn(_p(Y), terms.M, _p(terms.ti), _p(terms.tj), _p(terms.kind), terms.T, c, _p(F))
    return F


@dataclasses.dataclass
class State:
    """Oracle optimiser state: positions Y, S1 (velocity or E[g^2]), S2 (E[dx^2])."""
    Y: np.ndarray
    S1: np.ndarray
    S2: np.ndarray

    @classmethod
    def fresh(cls, Y):
        Y = np.array(Y, dtype=np.float64, copy=True).reshape(-1, 2)
        return cls(Y, np.zeros_like(Y), np.zeros_like(Y))


def step(state: State, terms: Terms, c: float, opt: int = OPT_MOMENTUM, a: float = 0.9,
         b: float = 0.01, rho: float = 0.95, eps: float = 1e-6) -> State:
    M = terms.M
    F = np.empty((M, 2))
    W = np.empty((M, 2))
    _L().ivo_step(opt, _p(state.Y), _p(state.S1), _p(state.S2), M, _p(terms.ti), _p(terms.tj),
                  _p(terms.kind), terms.T, c, a, b, rho, eps, _p(F), _p(W))
    return state


def step_l1(state: State, terms: Terms, c: float, opt: int = OPT_MOMENTUM, a: float = 0.9,
            b: float = 0.01) -> State:
    """Momentum / Nesterov step with the L1 forces of the late stage."""
    assert opt in (OPT_MOMENTUM, OPT_NESTEROV)
    M = terms.M
    F = np.empty((M, 2))
    W = np.empty((M, 2))
    _L().ivo_step_l1(opt, _p(state.Y), _p(state.S1), M, _p(terms.ti), _p(terms.tj),
                     _p(terms.kind), terms.T, c, a, b, _p(F), _p(W))
    return state


def step_adaptive(state: State, terms: Terms, c: float, b_box: list, opt: int = OPT_MOMENTUM,
                  a: float = 0.9, tau: float = 0.5, gamma1: float = 1.1, gamma2: float = 0.5,
                  metric: str = "l2") -> bool:
    """One attempt with self-adaptive b; b_box[0] holds b.  Returns True if accepted."""
    M = terms.M
    scratch = [np.empty((M, 2)) for _ in range(4)]
    b = ctypes.c_double(b_box[0])
    ok = _L().ivo_step_adaptive(opt, 1 if metric == "l1" else 0, _p(state.Y), _p(state.S1), M,
                                _p(terms.ti), _p(terms.tj), _p(terms.kind), terms.T, c, a,
                                ctypes.byref(b), tau, gamma1, gamma2, *[_p(x) for x in scratch])
    b_box[0] = b.value
    return bool(ok)


def run(state: State, terms: Terms, c: float, n_iter: int, opt: int = OPT_MOMENTUM,
        a: float = 0.9, b: float = 0.01, rho: float = 0.95, eps: float = 1e-6) -> State:
    rc = _L().ivo_run(opt, _p(state.Y), _p(state.S1), _p(state.S2), terms.M, _p(terms.ti),
                      _p(terms.tj), _p(terms.kind), terms.T, c, a, b, rho, eps, n_iter)
    if rc != 0:
        raise MemoryError("oracle run")
    return state


def run_threads(state: State, terms: Terms, c: float, n_iter: int, opt: int = OPT_MOMENTUM,
                a: float = 0.9, b: float = 0.01, rho: float = 0.95, eps: float = 1e-6,
                threads: int = 1) -> State:
    """run() on `threads` host threads: per-thread force sums added in thread order."""
    rc = _L().ivo_run_threads(opt, _p(state.Y), _p(state.S1), _p(state.S2), terms.M,
                              _p(terms.ti), _p(terms.tj), _p(terms.kind), terms.T, c, a, b, rho,
                              eps, n_iter, int(threads))
    if rc != 0:
        raise MemoryError("oracle run_threads")
    return state


def knn_f32(X, k: int, rows=None) -> np.ndarray:
    X = _c(X, np.float32)
    M, N = X.shape
    rows_a = None if rows is None else _c(rows, np.int64)
    n = M if rows_a is None else rows_a.shape[0]
    out = np.empty((n, k), dtype=np.int32)
    if _L().ivo_knn_f32(_p(X), M, N, k, _p(rows_a), n, _p(out)) != 0:
        raise ValueError("oracle knn: need 1 <= k <= M-1")
    return out


def knn_u8(X, k: int, rows=None) -> np.ndarray:
    X = _c(X, np.uint8)
    M, N = X.shape
    rows_a = None if rows is None else _c(rows, np.int64)
    n = M if rows_a is None else rows_a.shape[0]
    out = np.empty((n, k), dtype=np.int32)
    if _L().ivo_knn_u8(_p(X), M, N, k, _p(rows_a), n, _p(out)) != 0:
        raise ValueError("oracle knn: need 1 <= k <= M-1")
    return out


def knn_query(Q, X, k: int) -> np.ndarray:
    """The k base rows of X nearest to each query row of Q (float32 or uint8)."""
    u8 = np.asarray(X).dtype == np.uint8
    Q = _c(Q, np.uint8 if u8 else np.float32)
    X = _c(X, np.uint8 if u8 else np.float32)
    (Mq, N), M = Q.shape, X.shape[0]
    assert X.shape[1] == N
    out = np.empty((Mq, k), dtype=np.int32)
    fn = _L().ivo_knn_query_u8 if u8 else _L().ivo_knn_query_f32
    if fn(_p(Q), Mq, _p(X), M, N, k, _p(out)) != 0:
        raise ValueError("oracle knn_query: need 1 <= k <= M")
    return out


def place_nn(Y, ids) -> np.ndarray:
    """y_q = mean of Y over the base neighbours ids[q] (FP64)."""
    Y = _c(Y, np.float32)
    ids = _c(ids, np.int32)
    n, k = ids.shape
    out = np.empty((n, 2), dtype=np.float64)
    _L().ivo_place_nn(_p(Y), _p(ids), n, k, _p(out))
    return out


def qnx(Y, knn, rows=None, return_lowd: bool = False, threads: int = 1):
    Y = _c(Y, np.float32)
    knn = _c(knn, np.int32)
    M, k = knn.shape
    rows_a = None if rows is None else _c(rows, np.int64)
    n = M if rows_a is None else rows_a.shape[0]
    low = np.empty((n, k), dtype=np.int32) if return_lowd else None
    if threads > 1:
        q = float(_L().ivo_qnx_threads(_p(Y), M, _p(knn), k, _p(rows_a), n, _p(low), int(threads)))
    else:
        q = float(_L().ivo_qnx(_p(Y), M, _p(knn), k, _p(rows_a), n, _p(low)))
    if q < 0:
        raise MemoryError("oracle qnx")
    return (q, low) if return_lowd else q


def cf(Y, labels, nn: int, rows=None, threads: int = 1) -> float:
    Y = _c(Y, np.float32)
    labels = _c(labels, np.int32)
    M = Y.shape[0]
    rows_a = None if rows is None else _c(rows, np.int64)
    n = M if rows_a is None else rows_a.shape[0]
    if threads > 1:
        v = float(_L().ivo_cf_threads(_p(Y), M, _p(labels), nn, _p(rows_a), n, int(threads)))
    else:
        v = float(_L().ivo_cf(_p(Y), M, _p(labels), nn, _p(rows_a), n))
    if v < 0:
        raise MemoryError("oracle cf")
    return v


def knn_u8_gemm(X, k: int, block: int = 1024) -> np.ndarray:
    """The exact kNN graph of uint8 rows (R10 of the C oracle), for full-size inputs.

    Same definition as ``knn_u8``: for every row q the k other rows with the
    smallest exact integer squared distance, ascending, ties to the lower
    index.  Only the way the integers are formed differs: by the identity
    ||x_q - x_j||^2 = ||x_q||^2 + ||x_j||^2 - 2 x_q . x_j with a float64 matrix
    product (PyTorch on the host cores).  Every product and partial sum is an
    integer below 784 * 255^2 * 2 < 2^53, so the product is exact whatever
    order the library sums in.  The k smallest (distance, index) pairs are
    picked by a library top-k on the key distance * M + index, which is exact
    (below 2^53) and distinct per row, so the selection is unique.  Rows are
    processed ``block`` queries at a time to bound the memory of the distance
    block; each row's result depends on nothing but that row.
    """
    import torch

    X = _c(X, np.uint8)
    M, N = X.shape
    if not 1 <= k <= M - 1:
        raise ValueError("oracle knn: need 1 <= k <= M-1")
    if N * 255 * 255 * 2 * M >= 2 ** 53:
        raise ValueError("oracle knn_u8_gemm: integer keys would exceed 2^53")
    Xd = torch.from_numpy(X).to(torch.float64)
    nrm = (Xd * Xd).sum(dim=1)                  # exact integers
    idx = torch.arange(M, dtype=torch.float64)
    out = np.empty((M, k), dtype=np.int32)
    for s in range(0, M, block):
        e = min(M, s + block)
        G = Xd[s:e] @ Xd.T                      # exact integer dot products
        D = nrm[s:e, None] + nrm[None, :] - 2.0 * G
        key = D * float(M) + idx[None, :]
        key[torch.arange(e - s), torch.arange(s, e)] = float("inf")   # no self
        _, j = torch.topk(key, k, dim=1, largest=False, sorted=True)
        out[s:e] = j.numpy().astype(np.int32)
    return out
