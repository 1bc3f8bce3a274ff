"""Host-only checks of the C ABI: the library loads, exports every declared
symbol, and rejects bad arguments before touching the GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2303_05455_gb300 import _lib, build_lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ivhd.h")


@pytest.fixture(scope="module")
def L():
    build_lib.build()
    return _lib.load()


_LAYOUT_CACHE = {}


def c_layout(expr: str) -> int:
    """Evaluates a sizeof/offsetof expression against include/ivhd.h with the host C compiler."""
    import subprocess
    import tempfile

    if expr not in _LAYOUT_CACHE:
        with tempfile.TemporaryDirectory() as d:
            src = os.path.join(d, "t.c")
            exe = os.path.join(d, "t")
            with open(src, "w") as f:
                f.write(f'#include <stddef.h>\n#include <stdio.h>\n#include "{HEADER}"\n'
                        f'int main(void) {{ printf("%zu", (size_t)({expr})); return 0; }}\n')
            subprocess.run(["gcc", "-std=c11", "-o", exe, src], check=True)
            _LAYOUT_CACHE[expr] = int(subprocess.run([exe], capture_output=True, text=True,
                                                     check=True).stdout)
    return _LAYOUT_CACHE[expr]


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ivhd_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_binding_symbols():
    assert set(declared_symbols()) == set(_lib.SYMBOLS)


def test_every_declared_symbol_is_exported(L):
    for name in declared_symbols():
        assert hasattr(L, name), name


def test_params_struct_layout_and_defaults(L):
    p = _lib.Params()
    L.ivhd_default_params(ctypes.byref(p))
    assert ctypes.sizeof(_lib.Params) == c_layout("sizeof(ivhd_params)")
    for name, _ in _lib.Params._fields_:
        assert getattr(_lib.Params, name).offset == c_layout(f"offsetof(ivhd_params, {name})"), name
    assert ctypes.sizeof(_lib.Info) == c_layout("sizeof(ivhd_info_t)")
    assert (p.opt, p.init_uniform, p.dedup_mutual, p.hub_threshold) == (0, 1, 0, 0)
    assert p.a == pytest.approx(0.9) and p.b == pytest.approx(0.01)
    assert p.rho == pytest.approx(0.95) and p.eps == pytest.approx(1e-6)
    assert L.ivhd_version() == (0 << 16) | (3 << 8)
    assert p.adaptive == 0 and p.tau == pytest.approx(0.5)
    assert p.gamma1 == pytest.approx(1.1) and p.gamma2 == pytest.approx(0.5)
    for s in (0, -1, -2, -3, -4, -5, -6, -7, 42):
        assert isinstance(L.ivhd_status_string(s), bytes)


def _create(L, knn, M, k, r, c, p=None, on_dev=0):
    h = ctypes.c_void_p()
    pp = ctypes.byref(p) if p is not None else None
    data = knn.ctypes.data if knn is not None else None
    st = L.ivhd_create(data, M, k, r, c, pp, on_dev, ctypes.byref(h))
    return st, h


@pytest.mark.parametrize("M,k,r,c", [
    (1, 1, 1, 0.1),      # M < 2
    (10, 0, 1, 0.1),     # k = 0
    (10, 10, 1, 0.1),    # k > M - 1
    (10, 2, -1, 0.1),    # r < 0
    (10, 2, 1, 0.0),     # c <= 0
    (10, 2, 1, -1.0),
    (10, 2, 1, float("nan")),
    (10, 2, 1, float("inf")),
    (2 ** 31, 2, 1, 0.1),  # M too large
    (400_000_000, 2, 1, 0.1),  # symmetric layout beyond 2^31 slots
])
def test_create_rejects_bad_sizes(L, M, k, r, c):
    knn = np.zeros((2, 2), np.int32)
    st, h = _create(L, knn, M, k, r, c)
    assert st == -1 and not h.value


@pytest.mark.parametrize("field,value", [
    ("opt", 3), ("opt", -1), ("a", -0.1), ("a", 1.5), ("a", float("nan")), ("b", 0.0),
    ("b", float("inf")), ("rho", 1.0), ("rho", 0.0), ("eps", 0.0), ("hub_threshold", -1),
    ("hub_threshold", 70000), ("pos_format", 3), ("pos_format", -1), ("adaptive", 2),
    ("block_size", 64), ("block_size", 1024), ("resident", 4), ("resident", -2),
    ("vertices_per_warp", 3), ("vertices_per_warp", 16), ("vertices_per_warp", -1),
])
def test_create_rejects_bad_params(L, field, value):
    p = _lib.Params()
    L.ivhd_default_params(ctypes.byref(p))
    setattr(p, field, value)
    knn = np.array([[1], [0], [0]], np.int32)
    st, h = _create(L, knn, 3, 1, 1, 0.1, p)
    assert st == -1 and not h.value


def test_null_pointers_rejected(L):
    h = ctypes.c_void_p()
    assert L.ivhd_create(None, 3, 1, 1, 0.1, None, 0, ctypes.byref(h)) == -1
    knn = np.array([[1], [0], [0]], np.int32)
    assert L.ivhd_create(knn.ctypes.data, 3, 1, 1, 0.1, None, 0, None) == -1
    assert L.ivhd_step(None, 1) == -1
    assert L.ivhd_positions(None, None, 0) == -1
    assert L.ivhd_forces(None, None, 0) == -1
    assert L.ivhd_stress(None, None) == -1
    assert L.ivhd_random_neighbors(None, None, 0) == -1
    assert L.ivhd_set_positions(None, None, 0) == -1
    assert L.ivhd_info(None, None) == -1
    n = ctypes.c_size_t()
    assert L.ivhd_state_size(None, ctypes.byref(n)) == -1
    assert L.ivhd_get_state(None, None, 0) == -1
    assert L.ivhd_set_state(None, None, 0) == -1
    L.ivhd_destroy(None)  # no-op


def test_knn_build_and_eval_reject_bad_args(L):
    out = ctypes.c_double()
    assert L.ivhd_knn_build(None, 0, 10, 4, 2, None, None) == -1
    dummy = ctypes.c_void_p(16)  # never dereferenced: validation fails first
    assert L.ivhd_knn_build(dummy, 0, 1, 4, 2, dummy, None) == -1     # M < 2
    assert L.ivhd_knn_build(dummy, 0, 10, 0, 2, dummy, None) == -1    # N < 1
    assert L.ivhd_knn_build(dummy, 0, 10, 4, 10, dummy, None) == -1   # k > M-1
    assert L.ivhd_knn_build(dummy, 0, 1000, 4, 65, dummy, None) == -1  # k > 64
    assert L.ivhd_knn_build(dummy, 2, 10, 4, 2, dummy, None) == -1    # dtype
    assert L.ivhd_eval_qnx(dummy, 10, dummy, 0, dummy, 5, None, ctypes.byref(out), None) == -1
    assert L.ivhd_eval_qnx(dummy, 10, dummy, 3, dummy, 0, None, ctypes.byref(out), None) == -1
    assert L.ivhd_eval_cf(dummy, 10, dummy, 129, dummy, 5, ctypes.byref(out), None) == -1
    assert L.ivhd_probe_gather(0, 1 << 20, 1, ctypes.byref(out), None) == -1
    assert L.ivhd_probe_gather(1000, 100, 1, ctypes.byref(out), None) == -1
    assert L.ivhd_probe_gather(1000, 1 << 20, 0, ctypes.byref(out), None) == -1
    assert L.ivhd_probe_gather(1000, 1 << 20, 1, None, None) == -1
    us = ctypes.c_double()
    assert L.ivhd_probe_launch(0, 128, 10, ctypes.byref(us), None) == -1         # grid < 1
    assert L.ivhd_probe_launch((1 << 20) + 1, 128, 10, ctypes.byref(us), None) == -1
    assert L.ivhd_probe_launch(152, 100, 10, ctypes.byref(us), None) == -1       # not 32 k
    assert L.ivhd_probe_launch(152, 2048, 10, ctypes.byref(us), None) == -1      # > 1024
    assert L.ivhd_probe_launch(152, 128, 0, ctypes.byref(us), None) == -1        # n < 1
    assert L.ivhd_probe_launch(152, 128, 100001, ctypes.byref(us), None) == -1
    assert L.ivhd_probe_launch(152, 128, 10, None, None) == -1


@pytest.mark.parametrize("opt,field,value", [
    (2, "adaptive", 1),                      # adaptive b needs momentum or Nesterov
    (0, "tau", 0.0), (0, "gamma1", 1.0), (0, "gamma2", 1.0), (0, "gamma2", 0.0),
])
def test_create_rejects_bad_adaptive_params(L, opt, field, value):
    p = _lib.Params()
    L.ivhd_default_params(ctypes.byref(p))
    p.opt = opt
    p.adaptive = 1
    setattr(p, field, value)
    knn = np.array([[1], [0], [0]], np.int32)
    st, h = _create(L, knn, 3, 1, 1, 0.1, p)
    assert st == -1 and not h.value


def test_knn_index_rejects_bad_args(L):
    h = ctypes.c_void_p()
    assert L.ivhd_knn_index_create(None, 0, 10, 4, None, ctypes.byref(h)) == -1
    X = np.zeros((10, 4), np.float32)
    assert L.ivhd_knn_index_create(X.ctypes.data, 2, 10, 4, None, ctypes.byref(h)) == -1
    assert L.ivhd_knn_index_create(X.ctypes.data, 0, 0, 4, None, ctypes.byref(h)) == -1
    assert L.ivhd_knn_index_query(None, X.ctypes.data, 1, 1, X.ctypes.data, 0, None) == -1
    L.ivhd_knn_index_destroy(None)


def test_persistent_grid_needs_fp32_gathers_without_adaptive_b(L):
    knn = np.array([[1], [0], [0]], np.int32)
    for field, value in (("pos_format", 1), ("adaptive", 1)):
        p = _lib.Params()
        L.ivhd_default_params(ctypes.byref(p))
        p.resident = 3
        setattr(p, field, value)
        st, h = _create(L, knn, 3, 1, 1, 0.1, p)
        assert st == -1 and not h.value
    assert L.ivhd_probe_grid_barrier_timeout(0, None) == -1


def test_new_entry_points_reject_null(L):
    assert L.ivhd_warm_start(None, None, 0, None) == -1
    taken = ctypes.c_int32(7)
    assert L.ivhd_warm_start(None, ctypes.c_void_p(16), 0, ctypes.byref(taken)) == -1
    assert L.ivhd_mlp_activations(None, 0, None, None) == -1
    assert L.ivhd_set_metric(None, 0) == -1
    assert L.ivhd_resample_random_neighbors(None, 1) == -1
    assert L.ivhd_restrict_nn(None, None, 0, 0) == -1
    assert L.ivhd_adaptive_state(None, None, None, None) == -1
    assert L.ivhd_autotune(None, 5, None, None, None, None) == -1
    h = ctypes.c_void_p()
    M = np.array([10, 1], np.int64)           # an embedding with a single vertex
    k = np.array([2, 1], np.int32)
    r = np.array([1, 1], np.int32)
    sd = np.array([0, 0], np.uint64)
    knn = np.zeros(21, np.int32)
    assert L.ivhd_create_batch(knn.ctypes.data, M.ctypes.data, k.ctypes.data, r.ctypes.data,
                               sd.ctypes.data, 2, 0.1, None, 0, ctypes.byref(h)) == -1
    assert L.ivhd_create_batch(knn.ctypes.data, M.ctypes.data, k.ctypes.data, r.ctypes.data,
                               sd.ctypes.data, 0, 0.1, None, 0, ctypes.byref(h)) == -1


def test_set_allocator_pairs_and_reset(L):
    """Host logic of ivhd_set_allocator: alloc and free come in pairs, both
    NULL restores the built-in pool; no callback runs without an allocation."""
    calls = []
    alloc = _lib.ALLOC_FN(lambda n, s, u: calls.append(n))
    free = _lib.FREE_FN(lambda p, n, s, u: calls.append(p))
    null_alloc = ctypes.cast(None, _lib.ALLOC_FN)
    null_free = ctypes.cast(None, _lib.FREE_FN)
    assert L.ivhd_set_allocator(alloc, null_free, None) == -1
    assert L.ivhd_set_allocator(null_alloc, free, None) == -1
    assert L.ivhd_set_allocator(alloc, free, None) == 0
    assert L.ivhd_set_allocator(null_alloc, null_free, None) == 0
    assert calls == []
    with pytest.raises(ValueError):
        from paper_2303_05455_gb300 import ivhd
        ivhd.set_allocator(lambda n, s: 0)


@pytest.mark.skipif(os.environ.get("IVHD_CHECKED", "") not in ("", "0"),
                    reason="the checked library counts violations")
def test_normal_build_counts_no_violations_and_refuses_corruption(L):
    v = ctypes.c_int64(7)
    assert L.ivhd_check_violations(ctypes.byref(v), 0) == 0 and v.value == -1
    assert L.ivhd_check_violations(None, 0) == -1
    assert L.ivhd_test_corrupt_layout(None, 0, 0) == -1


def test_binding_rejects_host_tensors_before_any_cuda_call():
    import torch
    from paper_2303_05455_gb300 import ivhd
    X = torch.zeros((10, 4))
    with pytest.raises(ValueError):
        ivhd.KnnIndex(X)
    with pytest.raises(ValueError):
        ivhd.knn_query(X, X, 2)
    with pytest.raises(ValueError):
        ivhd.knn_build(X, 2)
