"""Python binding of the IVHD C ABI (argument marshalling only).

Every computation runs in libivhd's CUDA kernels.  Tensors are torch tensors
(device memory and streams come from PyTorch); numpy arrays are accepted for
host inputs.  The names follow the C entry points:

    emb = Embedding(knn, r=1, c=0.01, opt="momentum", a=0.9, b=0.01, seed=0)
    emb.step(2000)
    y = emb.positions()          # torch.float32 [M, 2] on the device

plus ``knn_build`` (exact brute-force kNN graph) and ``eval_qnx`` / ``eval_cf``
(Sec. 4.1 quality criteria on sampled rows).
"""
from __future__ import annotations

import atexit
import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import IvhdError, Info, Params, check

OPTS = {"momentum": 0, "nesterov": 1, "adadelta": 2}
POS_FORMATS = {"f32": 0, "f16": 1, "bf16": 2}
METRICS = {"l2": 0, "l1": 1}
ORDERS = {"degree": 0, "degree_cluster": 1}


def _stream_ptr(stream) -> int | None:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream or None


def _dev_i32(a, device) -> torch.Tensor:
    if isinstance(a, np.ndarray):
        a = torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32))
    return a.to(device=device, dtype=torch.int32).contiguous()


class Embedding:
    """One IVHD embedding context (``ivhd_create`` .. ``ivhd_destroy``).

    knn: int32 [M, k] kNN rows (torch CUDA tensor, torch CPU tensor or numpy);
    host inputs are copied by the library itself.
    """

    def __init__(self, knn, r: int = 1, c: float = 0.01, *, opt: str = "momentum",
                 a: float = 0.9, b: float = 0.01, rho: float = 0.95, eps: float = 1e-6,
                 seed: int = 0, dedup_mutual: bool = False, init_uniform: bool = True,
                 hub_threshold: int = 0, pos_format: str = "f32", adaptive: bool = False,
                 tau: float = 0.5, gamma1: float = 1.1, gamma2: float = 0.5, block_size: int = 0,
                 resident=None, vertices_per_warp: int = 0, order: str = "degree",
                 stream=None, device=None, batch=None):
        self._L = _lib.load()
        if device is None:
            device = torch.device("cuda", torch.cuda.current_device())
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        if isinstance(knn, np.ndarray):
            knn_t = torch.from_numpy(np.ascontiguousarray(knn, dtype=np.int32))
        else:
            knn_t = knn.to(dtype=torch.int32).contiguous()
        if batch is None:
            if knn_t.dim() != 2:
                raise ValueError("knn must be [M, k]")
            self.M, self.k = int(knn_t.shape[0]), int(knn_t.shape[1])
        self.r, self.c = int(r), float(c)
        p = Params()
        self._L.ivhd_default_params(ctypes.byref(p))
        p.opt = OPTS[opt]
        p.a, p.b, p.rho, p.eps = a, b, rho, eps
        p.seed = seed & 0xFFFFFFFFFFFFFFFF
        p.dedup_mutual = int(dedup_mutual)
        p.init_uniform = int(init_uniform)
        p.hub_threshold = int(hub_threshold)
        p.pos_format = POS_FORMATS[pos_format]
        p.adaptive = int(adaptive)
        p.tau, p.gamma1, p.gamma2 = tau, gamma1, gamma2
        p.block_size = int(block_size)
        # resident: None (automatic), False (one launch per step), True (one block),
        # "cluster" (8-block cluster), "grid" (persistent cooperative grid)
        p.resident = {None: 0, False: -1, True: 1, "cluster": 2, "grid": 3}[resident]
        p.vertices_per_warp = int(vertices_per_warp)
        p.order = ORDERS[order]
        p.stream = self.stream.cuda_stream or None
        self.opt = opt
        self.params = p
        h = ctypes.c_void_p()
        on_dev = int(knn_t.is_cuda)
        if batch is None:
            check(self._L.ivhd_create(knn_t.data_ptr(), self.M, self.k, self.r, self.c,
                                      ctypes.byref(p), on_dev, ctypes.byref(h)), "ivhd_create")
        else:
            Ms = np.ascontiguousarray(batch["M"], dtype=np.int64)
            ks = np.ascontiguousarray(batch["k"], dtype=np.int32)
            rs = np.ascontiguousarray(batch["r"], dtype=np.int32)
            seeds = np.ascontiguousarray(np.asarray(batch["seed"], dtype=np.uint64))
            self.M, self.k, self.r = int(Ms.sum()), int(ks.max()), int(rs.max())
            self.sizes = Ms
            check(self._L.ivhd_create_batch(knn_t.data_ptr(), Ms.ctypes.data, ks.ctypes.data,
                                            rs.ctypes.data, seeds.ctypes.data, len(Ms), self.c,
                                            ctypes.byref(p), on_dev, ctypes.byref(h)),
                  "ivhd_create_batch")
        self._h = h

    # -- lifetime ---------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._L.ivhd_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- steps and state ----------------------------------------------------
    def step(self, n_iter: int = 1):
        check(self._L.ivhd_step(self._h, int(n_iter)), "ivhd_step")

    def set_positions(self, xy):
        if isinstance(xy, np.ndarray):
            arr = np.ascontiguousarray(xy, dtype=np.float32)
            check(self._L.ivhd_set_positions(self._h, arr.ctypes.data, 0), "ivhd_set_positions")
            return
        t = xy.to(dtype=torch.float32).contiguous()
        check(self._L.ivhd_set_positions(self._h, t.data_ptr(), int(t.is_cuda)),
              "ivhd_set_positions")
        if not t.is_cuda:
            return
        self._keep = t  # the copy is stream-ordered; keep the source alive until then

    def positions(self, out: torch.Tensor | None = None, host: bool = False):
        if host:
            arr = np.empty((self.M, 2), dtype=np.float32)
            check(self._L.ivhd_positions(self._h, arr.ctypes.data, 0), "ivhd_positions")
            return arr
        if out is None:
            out = torch.empty((self.M, 2), dtype=torch.float32, device=self.device)
        assert out.dtype == torch.float32 and out.is_contiguous() and out.numel() == 2 * self.M
        check(self._L.ivhd_positions(self._h, out.data_ptr(), int(out.is_cuda)), "ivhd_positions")
        return out

    def forces(self, host: bool = True):
        if host:
            arr = np.empty((self.M, 2), dtype=np.float32)
            check(self._L.ivhd_forces(self._h, arr.ctypes.data, 0), "ivhd_forces")
            return arr
        out = torch.empty((self.M, 2), dtype=torch.float32, device=self.device)
        check(self._L.ivhd_forces(self._h, out.data_ptr(), 1), "ivhd_forces")
        return out

    def warm_start(self, xy) -> bool:
        """ivhd_warm_start: starts from the placement xy (M x 2, e.g. the warm-start
        network's output) when its stress is finite and below that of the current
        positions, else keeps them (plain IVHD is the fallback).  Zeroes the
        optimiser state either way.  Returns whether the placement was taken."""
        taken = ctypes.c_int32()
        if isinstance(xy, np.ndarray):
            arr = np.ascontiguousarray(xy, dtype=np.float32)
            check(self._L.ivhd_warm_start(self._h, arr.ctypes.data, 0, ctypes.byref(taken)),
                  "ivhd_warm_start")
            return bool(taken.value)
        t = xy.to(dtype=torch.float32).contiguous()
        check(self._L.ivhd_warm_start(self._h, t.data_ptr(), int(t.is_cuda), ctypes.byref(taken)),
              "ivhd_warm_start")
        return bool(taken.value)

    def stress(self) -> float:
        v = ctypes.c_double()
        check(self._L.ivhd_stress(self._h, ctypes.byref(v)), "ivhd_stress")
        return v.value

    def random_neighbors(self) -> np.ndarray:
        arr = np.empty((self.M, self.r), dtype=np.int32)
        check(self._L.ivhd_random_neighbors(self._h, arr.ctypes.data, 0), "ivhd_random_neighbors")
        return arr

    def info(self) -> dict:
        inf = Info()
        check(self._L.ivhd_info(self._h, ctypes.byref(inf)), "ivhd_info")
        return {name: getattr(inf, name) for name, _ in Info._fields_}

    def set_metric(self, metric: str):
        """'l2' (the method) or 'l1' (the late-stage variant)."""
        check(self._L.ivhd_set_metric(self._h, METRICS[metric]), "ivhd_set_metric")

    def resample_random_neighbors(self, epoch: int):
        check(self._L.ivhd_resample_random_neighbors(self._h, epoch & 0xFFFFFFFFFFFFFFFF),
              "ivhd_resample_random_neighbors")

    def restrict_nn(self, helper=None):
        """Reverse-neighbour restriction with a helper kNN graph; None restores the graph."""
        if helper is None:
            check(self._L.ivhd_restrict_nn(self._h, None, 0, 0), "ivhd_restrict_nn")
            return
        if isinstance(helper, np.ndarray):
            h = np.ascontiguousarray(helper, dtype=np.int32)
            check(self._L.ivhd_restrict_nn(self._h, h.ctypes.data, h.shape[1], 0),
                  "ivhd_restrict_nn")
        else:
            h = helper.to(dtype=torch.int32).contiguous()
            check(self._L.ivhd_restrict_nn(self._h, h.data_ptr(), h.shape[1], int(h.is_cuda)),
                  "ivhd_restrict_nn")

    @classmethod
    def batch(cls, graphs, r, seeds, c: float = 0.01, **kw):
        """One context for several independent embeddings.

        graphs: list of int32 [M_e, k_e] local kNN rows; r, seeds: per-embedding
        lists (or scalars).  Positions come back concatenated in list order."""
        n = len(graphs)
        rs = list(r) if np.ndim(r) else [int(r)] * n
        sd = list(seeds) if np.ndim(seeds) else [int(seeds) + e for e in range(n)]
        if all(isinstance(g, torch.Tensor) and g.is_cuda for g in graphs):
            flat = torch.cat([g.to(torch.int32).reshape(-1) for g in graphs])
        else:
            flat = np.concatenate([np.ascontiguousarray(
                g.cpu().numpy() if isinstance(g, torch.Tensor) else g, dtype=np.int32).ravel()
                for g in graphs])
        meta = {"M": [g.shape[0] for g in graphs], "k": [g.shape[1] for g in graphs], "r": rs,
                "seed": sd}
        return cls(flat, r=max(rs), c=c, batch=meta, **kw)

    def autotune(self, trial_steps: int = 20) -> dict:
        bb = ctypes.c_int32()
        bh = ctypes.c_int32()
        bv = ctypes.c_int32()
        us = ctypes.c_float()
        check(self._L.ivhd_autotune(self._h, int(trial_steps), ctypes.byref(bb), ctypes.byref(bh),
                                    ctypes.byref(bv), ctypes.byref(us)), "ivhd_autotune")
        return {"block": bb.value, "hub_threshold": bh.value, "vertices_per_warp": bv.value,
                "us_per_step": us.value}

    def adaptive_state(self) -> dict:
        b = ctypes.c_float()
        acc = ctypes.c_int64()
        rej = ctypes.c_int64()
        check(self._L.ivhd_adaptive_state(self._h, ctypes.byref(b), ctypes.byref(acc),
                                          ctypes.byref(rej)), "ivhd_adaptive_state")
        return {"b": b.value, "accepted": acc.value, "rejected": rej.value}

    def get_state(self) -> bytes:
        n = ctypes.c_size_t()
        check(self._L.ivhd_state_size(self._h, ctypes.byref(n)), "ivhd_state_size")
        buf = ctypes.create_string_buffer(n.value)
        check(self._L.ivhd_get_state(self._h, buf, n.value), "ivhd_get_state")
        return buf.raw

    def set_state(self, state: bytes):
        buf = ctypes.create_string_buffer(state, len(state))
        check(self._L.ivhd_set_state(self._h, buf, len(state)), "ivhd_set_state")


KNN_METHODS = {"auto": 0, "cuda_cores": 1, "tensor_cores": 2}


def knn_build(X: torch.Tensor, k: int, stream=None, method: str = "auto",
              return_stats: bool = False):
    """Exact kNN graph of the rows of X (float32 or uint8 CUDA tensor) -> int32 [M, k].

    method: "auto" (tensor cores when they apply), "cuda_cores" or "tensor_cores";
    the graph is the same for every method.  return_stats adds a dict with the
    method that ran, the rows recomputed after a failed certificate, and the
    largest observed approximation error against the bound."""
    L = _lib.load()
    if not X.is_cuda:
        raise ValueError("knn_build expects a CUDA tensor")
    X = X.contiguous()
    if X.dtype == torch.float32:
        dt = 0
    elif X.dtype == torch.uint8:
        dt = 1
    else:
        raise ValueError("X must be float32 or uint8")
    M, N = int(X.shape[0]), int(X.shape[1])
    out = torch.empty((M, k), dtype=torch.int32, device=X.device)
    st = _lib.KnnStats()
    check(L.ivhd_knn_build_ex(X.data_ptr(), dt, M, N, int(k), out.data_ptr(), KNN_METHODS[method],
                              ctypes.byref(st), _stream_ptr(stream)), "ivhd_knn_build_ex")
    if return_stats:
        names = {v: n for n, v in KNN_METHODS.items()}
        return out, {"method": names[st.method], "fallback_rows": st.fallback_rows,
                     "max_rel_err": st.max_rel_err, "eps_coef": st.eps_coef}
    return out


def knn_query(Q: torch.Tensor, X: torch.Tensor, k: int, stream=None, method: str = "auto",
              return_stats: bool = False):
    """The k rows of the base set X nearest to each row of Q (ivhd_knn_query) -> int32 [Mq, k].

    Same dtypes, distances, tie rule and methods as knn_build; nothing is excluded."""
    L = _lib.load()
    if not (Q.is_cuda and X.is_cuda) or Q.dtype != X.dtype or Q.shape[1] != X.shape[1]:
        raise ValueError("knn_query expects CUDA tensors of one dtype and width")
    dts = {torch.float32: 0, torch.uint8: 1}
    if X.dtype not in dts:
        raise ValueError("X must be float32 or uint8")
    Q, X = Q.contiguous(), X.contiguous()
    Mq, M, N = int(Q.shape[0]), int(X.shape[0]), int(X.shape[1])
    out = torch.empty((Mq, k), dtype=torch.int32, device=X.device)
    st = _lib.KnnStats()
    check(L.ivhd_knn_query(Q.data_ptr(), Mq, X.data_ptr(), M, dts[X.dtype], N, int(k),
                           out.data_ptr(), KNN_METHODS[method], ctypes.byref(st),
                           _stream_ptr(stream)), "ivhd_knn_query")
    if return_stats:
        names = {v: n for n, v in KNN_METHODS.items()}
        return out, {"method": names[st.method], "fallback_rows": st.fallback_rows,
                     "max_rel_err": st.max_rel_err, "eps_coef": st.eps_coef}
    return out


class KnnIndex:
    """A base set held for repeated kNN queries (ivhd_knn_index_*): the rows of X
    (float32 or uint8 CUDA tensor) are copied and prepared once."""

    _DTYPES = {torch.float32: 0, torch.uint8: 1}

    def __init__(self, X: torch.Tensor, stream=None):
        self._L = _lib.load()
        if not X.is_cuda or X.dtype not in self._DTYPES:
            raise ValueError("KnnIndex expects a float32 or uint8 CUDA tensor")
        X = X.contiguous()
        self.dtype, self.M, self.N = X.dtype, int(X.shape[0]), int(X.shape[1])
        self.device = X.device
        h = ctypes.c_void_p()
        check(self._L.ivhd_knn_index_create(X.data_ptr(), self._DTYPES[X.dtype], self.M, self.N,
                                            _stream_ptr(stream), ctypes.byref(h)),
              "ivhd_knn_index_create")
        self._h = h

    def query(self, Q: torch.Tensor, k: int, method: str = "auto", return_stats: bool = False):
        """The k base rows nearest to each row of Q -> int32 [Mq, k] (as knn_query)."""
        if not Q.is_cuda or Q.dtype != self.dtype or Q.shape[1] != self.N:
            raise ValueError("Q must be a CUDA tensor of the index's dtype and width")
        Q = Q.contiguous()
        out = torch.empty((int(Q.shape[0]), k), dtype=torch.int32, device=Q.device)
        st = _lib.KnnStats()
        check(self._L.ivhd_knn_index_query(self._h, Q.data_ptr(), int(Q.shape[0]), int(k),
                                           out.data_ptr(), KNN_METHODS[method],
                                           ctypes.byref(st)), "ivhd_knn_index_query")
        if return_stats:
            names = {v: n for n, v in KNN_METHODS.items()}
            return out, {"method": names[st.method], "fallback_rows": st.fallback_rows,
                         "max_rel_err": st.max_rel_err, "eps_coef": st.eps_coef}
        return out

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._L.ivhd_knn_index_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def place_nn(Y: torch.Tensor, ids: torch.Tensor, stream=None) -> torch.Tensor:
    """New points at the mean embedding of their base neighbours (ivhd_place_nn) -> [n, 2]."""
    L = _lib.load()
    Y = Y.to(torch.float32).contiguous()
    ids = ids.to(device=Y.device, dtype=torch.int32).contiguous()
    n, k = int(ids.shape[0]), int(ids.shape[1])
    out = torch.empty((n, 2), dtype=torch.float32, device=Y.device)
    check(L.ivhd_place_nn(Y.data_ptr(), int(Y.shape[0]), ids.data_ptr(), n, k, out.data_ptr(),
                          _stream_ptr(stream)), "ivhd_place_nn")
    return out


def eval_qnx(Y: torch.Tensor, knn: torch.Tensor, rows: torch.Tensor, return_lowd: bool = False,
             stream=None):
    """Q_NX(k) on the sampled rows (Sec. 4.1); optionally the embedded neighbours found."""
    L = _lib.load()
    Y = Y.to(dtype=torch.float32).contiguous()
    knn = _dev_i32(knn, Y.device)
    rows = rows.to(device=Y.device, dtype=torch.int64).contiguous()
    k = int(knn.shape[1])
    low = torch.empty((rows.numel(), k), dtype=torch.int32, device=Y.device) if return_lowd else None
    q = ctypes.c_double()
    check(L.ivhd_eval_qnx(Y.data_ptr(), int(Y.shape[0]), knn.data_ptr(), k, rows.data_ptr(),
                          rows.numel(), low.data_ptr() if low is not None else None,
                          ctypes.byref(q), _stream_ptr(stream)), "ivhd_eval_qnx")
    return (q.value, low) if return_lowd else q.value


def eval_cf(Y: torch.Tensor, labels, nn: int, rows: torch.Tensor, stream=None) -> float:
    """Neighbour hit cf_nn (Sec. 4.1, Eq. 4.4) on the sampled rows."""
    L = _lib.load()
    Y = Y.to(dtype=torch.float32).contiguous()
    lab = _dev_i32(labels, Y.device)
    rows = rows.to(device=Y.device, dtype=torch.int64).contiguous()
    v = ctypes.c_double()
    check(L.ivhd_eval_cf(Y.data_ptr(), int(Y.shape[0]), lab.data_ptr(), int(nn), rows.data_ptr(),
                         rows.numel(), ctypes.byref(v), _stream_ptr(stream)), "ivhd_eval_cf")
    return v.value


def probe_gather(n_positions: int, n_gathers: int = 16_777_216, repeats: int = 20,
                 stream=None) -> float:
    """Random float2 gathers per second the GPU sustains from n_positions elements."""
    L = _lib.load()
    v = ctypes.c_double()
    check(L.ivhd_probe_gather(int(n_positions), int(n_gathers), int(repeats), ctypes.byref(v),
                              _stream_ptr(stream)), "ivhd_probe_gather")
    return v.value


def probe_launch(grid: int, block: int = 128, n_launches: int = 2000, stream=None) -> float:
    """Device microseconds per launch of a graph of chained programmatic
    dependent launches of an empty kernel of ``grid`` x ``block`` threads."""
    L = _lib.load()
    v = ctypes.c_double()
    check(L.ivhd_probe_launch(int(grid), int(block), int(n_launches), ctypes.byref(v),
                              _stream_ptr(stream)), "ivhd_probe_launch")
    return v.value


# Every callback pair ever registered stays referenced: blocks keep the free
# routine of the allocator that made them after the setting changes.
_ALLOCATORS: list = []
_FINALIZING = [False]


def _stop_user_frees():
    # blocks still held at interpreter exit are left to the process teardown
    _FINALIZING[0] = True


atexit.register(_stop_user_frees)


def set_allocator(alloc=None, free=None) -> None:
    """ivhd_set_allocator: take the library's device memory from ``alloc``.

    ``alloc(nbytes, stream) -> int`` returns a device address (0 or an
    exception = out of memory) usable on the ``cudaStream_t`` value
    ``stream``; ``free(ptr, nbytes, stream)`` gives it back.  Both None
    restores the library's own stream-ordered pool.
    """
    L = _lib.load()
    if (alloc is None) != (free is None):
        raise ValueError("set_allocator needs both alloc and free, or neither")
    if alloc is None:
        check(L.ivhd_set_allocator(ctypes.cast(None, _lib.ALLOC_FN),
                                   ctypes.cast(None, _lib.FREE_FN), None), "ivhd_set_allocator")
        return

    def _alloc(nbytes, stream, _user):
        try:
            return int(alloc(int(nbytes), int(stream or 0))) or None
        except Exception:
            return None

    def _free(ptr, nbytes, stream, _user):
        if _FINALIZING[0]:
            return
        try:
            free(int(ptr), int(nbytes), int(stream or 0))
        except Exception:
            pass

    cbs = (_lib.ALLOC_FN(_alloc), _lib.FREE_FN(_free))
    _ALLOCATORS.append(cbs)
    check(L.ivhd_set_allocator(cbs[0], cbs[1], None), "ivhd_set_allocator")


def check_violations(reset: bool = False) -> int:
    """Out-of-range indices / rows the step kernels met and skipped (checked
    builds, IVHD_CHECKED=1); -1 with the normal library."""
    L = _lib.load()
    v = ctypes.c_int64()
    check(L.ivhd_check_violations(ctypes.byref(v), int(bool(reset))), "ivhd_check_violations")
    return int(v.value)


def use_torch_allocator(device=None) -> None:
    """Route the library's device allocations through PyTorch's caching allocator."""
    dev = torch.cuda.current_device() if device is None else torch.device(device).index

    def alloc(nbytes, stream):
        return torch.cuda.caching_allocator_alloc(nbytes, dev, stream)

    def free(ptr, _nbytes, _stream):
        torch.cuda.caching_allocator_delete(ptr)

    set_allocator(alloc, free)


def gemm_bf16_tn(A: torch.Tensor, B: torch.Tensor, stream=None,
                 out: torch.Tensor | None = None) -> torch.Tensor:
    """C = A @ B.T on the tensor cores: A [M, K], B [N, K] BF16 CUDA tensors -> FP32 [M, N]."""
    L = _lib.load()
    A = A.to(torch.bfloat16).contiguous()
    B = B.to(torch.bfloat16).contiguous()
    M, K = A.shape
    N = B.shape[0]
    C = out if out is not None else torch.empty((M, N), dtype=torch.float32, device=A.device)
    assert C.dtype == torch.float32 and C.is_contiguous() and tuple(C.shape) == (M, N)
    check(L.ivhd_gemm_bf16_tn(A.data_ptr(), B.data_ptr(), C.data_ptr(), M, N, K,
                              _stream_ptr(stream)), "ivhd_gemm_bf16_tn")
    return C


_X_DTYPES = {torch.bfloat16: 0, torch.uint8: 1, torch.float32: 2}


class MLP:
    """The learned warm start (ivhd_mlp_*): n_in -> hidden -> hidden -> 2 with GELU."""

    def __init__(self, n_in: int = 784, hidden: int = 512, max_batch: int = 4096, stream=None):
        self._L = _lib.load()
        self.n_in, self.hidden, self.max_batch = n_in, hidden, max_batch
        h = ctypes.c_void_p()
        check(self._L.ivhd_mlp_create(n_in, hidden, max_batch, _stream_ptr(stream),
                                      ctypes.byref(h)), "ivhd_mlp_create")
        self._h = h
        self.n_params = int(self._L.ivhd_mlp_num_params(h))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._L.ivhd_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, flat):
        if isinstance(flat, np.ndarray):
            a = np.ascontiguousarray(flat, dtype=np.float32)
            assert a.size == self.n_params
            check(self._L.ivhd_mlp_set_params(self._h, a.ctypes.data, 0), "ivhd_mlp_set_params")
        else:
            t = flat.to(torch.float32).contiguous()
            check(self._L.ivhd_mlp_set_params(self._h, t.data_ptr(), int(t.is_cuda)),
                  "ivhd_mlp_set_params")

    def init_params(self, seed: int, out_scale: float = 0.1):
        """He-uniform weights (U(-sqrt(6/fan_in), +sqrt(6/fan_in))), zero biases;
        the output layer's weights scaled by out_scale.  Seeded numpy PCG64."""
        rng = np.random.Generator(np.random.PCG64(seed))
        parts = []
        for fo, fi, sc in ((self.hidden, self.n_in, 1.0), (self.hidden, self.hidden, 1.0),
                           (2, self.hidden, out_scale)):
            lim = np.sqrt(6.0 / fi)
            parts += [rng.uniform(-lim, lim, size=fo * fi) * sc, np.zeros(fo)]
        self.set_params(np.concatenate(parts).astype(np.float32))

    def get_params(self) -> np.ndarray:
        a = np.empty(self.n_params, dtype=np.float32)
        check(self._L.ivhd_mlp_get_params(self._h, a.ctypes.data, 0), "ivhd_mlp_get_params")
        return a

    @staticmethod
    def _x(x: torch.Tensor):
        assert x.is_cuda and x.is_contiguous()
        return x.data_ptr(), _X_DTYPES[x.dtype]

    def loss_grad(self, x: torch.Tensor, t: torch.Tensor, x_scale: float = 1.0):
        ptr, dt = self._x(x)
        g = torch.empty(self.n_params, dtype=torch.float32, device=x.device)
        loss = ctypes.c_double()
        tt = t.to(torch.float32).contiguous()
        check(self._L.ivhd_mlp_loss_grad(self._h, ptr, dt, x_scale, tt.data_ptr(), x.shape[0],
                                         ctypes.byref(loss), g.data_ptr()), "ivhd_mlp_loss_grad")
        return loss.value, g

    def train_step(self, x: torch.Tensor, t: torch.Tensor, lr: float = 1e-3, x_scale: float = 1.0,
                   want_loss: bool = False):
        ptr, dt = self._x(x)
        tt = t if (t.dtype == torch.float32 and t.is_contiguous()) else t.to(torch.float32).contiguous()
        loss = ctypes.c_double() if want_loss else None
        check(self._L.ivhd_mlp_train_step(self._h, ptr, dt, x_scale, tt.data_ptr(), x.shape[0], lr,
                                          ctypes.byref(loss) if loss is not None else None),
              "ivhd_mlp_train_step")
        return loss.value if loss is not None else None

    def forward(self, x: torch.Tensor, x_scale: float = 1.0) -> torch.Tensor:
        ptr, dt = self._x(x)
        y = torch.empty((x.shape[0], 2), dtype=torch.float32, device=x.device)
        check(self._L.ivhd_mlp_forward(self._h, ptr, dt, x_scale, x.shape[0], y.data_ptr()),
              "ivhd_mlp_forward")
        return y

    def launches(self) -> int:
        return int(self._L.ivhd_mlp_launches(self._h))

    _ACT = {"x": (0, "bf16", "in"), "z1": (1, "f32", "h"), "h1": (2, "bf16", "h"),
            "z2": (3, "f32", "h"), "h2": (4, "bf16", "h"), "y": (5, "f32", 2),
            "dy": (6, "f32", 2), "dz2": (7, "bf16", "h"), "dz1": (8, "bf16", "h")}

    def activations(self, which: str) -> np.ndarray:
        """One intermediate array of the last batch (ivhd_mlp_activations), as float32."""
        code, kind, width = self._ACT[which]
        cols = self.n_in if width == "in" else (self.hidden if width == "h" else 2)
        buf = np.empty((self.max_batch, cols), dtype=np.uint16 if kind == "bf16" else np.float32)
        rows = ctypes.c_int64()
        check(self._L.ivhd_mlp_activations(self._h, code, buf.ctypes.data, ctypes.byref(rows)),
              "ivhd_mlp_activations")
        out = buf[:rows.value]
        if kind == "bf16":
            out = (out.astype(np.uint32) << 16).view(np.float32)
        return np.ascontiguousarray(out)
