"""ctypes loader for ``libivhd.so`` (the C ABI declared in ``include/ivhd.h``).

Only argument marshalling lives here.  The library must have been built
(``__graft_entry__.build()`` or ``python -m paper_2303_05455_gb300.build_lib``);
there is no fallback implementation, so a missing library is an error.
"""
from __future__ import annotations

import ctypes
import os

from . import build_lib

STATUS = {
    0: "IVHD_OK", -1: "IVHD_ERR_ARG", -2: "IVHD_ERR_INDEX", -3: "IVHD_ERR_OOM",
    -4: "IVHD_ERR_CUDA", -5: "IVHD_ERR_NONFINITE", -6: "IVHD_ERR_TIMEOUT", -7: "IVHD_ERR_STATE",
}

# exported symbols declared in include/ivhd.h
SYMBOLS = (
    "ivhd_default_params", "ivhd_create", "ivhd_set_positions", "ivhd_step", "ivhd_positions",
    "ivhd_forces", "ivhd_stress", "ivhd_random_neighbors", "ivhd_info", "ivhd_state_size",
    "ivhd_get_state", "ivhd_set_state", "ivhd_destroy", "ivhd_status_string", "ivhd_version",
    "ivhd_knn_build", "ivhd_knn_build_ex", "ivhd_eval_qnx", "ivhd_eval_cf", "ivhd_eval_qnx_static",
    "ivhd_probe_gather", "ivhd_probe_launch", "ivhd_set_metric", "ivhd_resample_random_neighbors",
    "ivhd_restrict_nn", "ivhd_adaptive_state", "ivhd_create_batch", "ivhd_autotune",
    "ivhd_gemm_bf16_tn", "ivhd_mlp_create", "ivhd_mlp_destroy", "ivhd_mlp_num_params",
    "ivhd_mlp_set_params", "ivhd_mlp_get_params", "ivhd_mlp_loss_grad", "ivhd_mlp_train_step",
    "ivhd_mlp_forward", "ivhd_mlp_launches", "ivhd_probe_wait_timeout", "ivhd_test_fail_alloc",
    "ivhd_test_live_allocs", "ivhd_set_allocator", "ivhd_knn_query", "ivhd_place_nn",
    "ivhd_check_violations", "ivhd_test_corrupt_layout", "ivhd_probe_grid_barrier_timeout",
    "ivhd_knn_index_create", "ivhd_knn_index_query", "ivhd_knn_index_destroy",
    "ivhd_mlp_activations", "ivhd_warm_start",
)

# callback types of ivhd_set_allocator
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                           ctypes.c_void_p)


class IvhdError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {STATUS.get(status, status)}")


class Params(ctypes.Structure):
    _fields_ = [
        ("opt", ctypes.c_int32), ("a", ctypes.c_float), ("b", ctypes.c_float),
        ("rho", ctypes.c_float), ("eps", ctypes.c_float), ("seed", ctypes.c_uint64),
        ("dedup_mutual", ctypes.c_int32), ("init_uniform", ctypes.c_int32),
        ("hub_threshold", ctypes.c_int32), ("pos_format", ctypes.c_int32),
        ("adaptive", ctypes.c_int32), ("tau", ctypes.c_float), ("gamma1", ctypes.c_float),
        ("gamma2", ctypes.c_float), ("block_size", ctypes.c_int32),
        ("resident", ctypes.c_int32), ("vertices_per_warp", ctypes.c_int32),
        ("order", ctypes.c_int32), ("stream", ctypes.c_void_p),
    ]


class Info(ctypes.Structure):
    _fields_ = [
        ("M", ctypes.c_int64), ("k", ctypes.c_int32), ("r", ctypes.c_int32),
        ("n_terms", ctypes.c_int64), ("nnz_sym", ctypes.c_int64),
        ("layout_slots", ctypes.c_int64), ("n_hub", ctypes.c_int64),
        ("max_degree", ctypes.c_int32), ("empty_rn", ctypes.c_int32),
        ("steps_done", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
        ("setup_launches", ctypes.c_int64), ("aux_launches", ctypes.c_int64),
        ("launch_form", ctypes.c_int32),
        ("step_blocks", ctypes.c_int32),
        ("step_threads", ctypes.c_int32),
    ]


class KnnStats(ctypes.Structure):
    _fields_ = [
        ("method", ctypes.c_int32), ("fallback_rows", ctypes.c_int64),
        ("max_rel_err", ctypes.c_float), ("eps_coef", ctypes.c_float),
    ]


_lib = None


def lib_path() -> str:
    return build_lib.LIB


def load(build_if_missing: bool = False):
    """Loads libivhd.so (libivhd_checked.so when IVHD_CHECKED is set); raises if
    it is absent (no CPU fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    checked = os.environ.get("IVHD_CHECKED", "") not in ("", "0")
    path = build_lib.LIB_CHECKED if checked else build_lib.LIB
    if not os.path.exists(path):
        if build_if_missing:
            build_lib.build(checked=checked)
        else:
            raise RuntimeError(f"libivhd.so is not built ({path}); run __graft_entry__.build()")
    L = ctypes.CDLL(path)
    P, i32, i64, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
    L.ivhd_default_params.argtypes = [ctypes.POINTER(Params)]
    L.ivhd_default_params.restype = None
    L.ivhd_create.argtypes = [P, i64, i32, i32, ctypes.c_float, ctypes.POINTER(Params), i32,
                              ctypes.POINTER(P)]
    L.ivhd_create.restype = i32
    L.ivhd_set_positions.argtypes = [P, P, i32]
    L.ivhd_warm_start.argtypes = [P, P, i32, ctypes.POINTER(ctypes.c_int32)]
    L.ivhd_warm_start.restype = i32
    L.ivhd_step.argtypes = [P, i64]
    L.ivhd_positions.argtypes = [P, P, i32]
    L.ivhd_forces.argtypes = [P, P, i32]
    L.ivhd_stress.argtypes = [P, ctypes.POINTER(ctypes.c_double)]
    L.ivhd_random_neighbors.argtypes = [P, P, i32]
    L.ivhd_info.argtypes = [P, ctypes.POINTER(Info)]
    L.ivhd_state_size.argtypes = [P, ctypes.POINTER(ctypes.c_size_t)]
    L.ivhd_get_state.argtypes = [P, P, ctypes.c_size_t]
    L.ivhd_set_state.argtypes = [P, P, ctypes.c_size_t]
    for name in ("ivhd_set_positions", "ivhd_step", "ivhd_positions", "ivhd_forces",
                 "ivhd_stress", "ivhd_random_neighbors", "ivhd_info", "ivhd_state_size",
                 "ivhd_get_state", "ivhd_set_state"):
        getattr(L, name).restype = i32
    L.ivhd_destroy.argtypes = [P]
    L.ivhd_destroy.restype = None
    L.ivhd_status_string.argtypes = [i32]
    L.ivhd_status_string.restype = ctypes.c_char_p
    L.ivhd_version.argtypes = []
    L.ivhd_version.restype = i32
    L.ivhd_knn_build.argtypes = [P, i32, i64, i32, i32, P, P]
    L.ivhd_knn_build.restype = i32
    L.ivhd_knn_build_ex.argtypes = [P, i32, i64, i32, i32, P, i32, P, P]
    L.ivhd_knn_build_ex.restype = i32
    L.ivhd_check_violations.argtypes = [ctypes.POINTER(ctypes.c_int64), i32]
    L.ivhd_check_violations.restype = i32
    L.ivhd_test_corrupt_layout.argtypes = [P, i64, ctypes.c_uint32]
    L.ivhd_test_corrupt_layout.restype = i32
    L.ivhd_knn_query.argtypes = [P, i64, P, i64, i32, i32, i32, P, i32, P, P]
    L.ivhd_knn_query.restype = i32
    L.ivhd_knn_index_create.argtypes = [P, i32, i64, i32, P, ctypes.POINTER(P)]
    L.ivhd_knn_index_create.restype = i32
    L.ivhd_knn_index_query.argtypes = [P, P, i64, i32, P, i32, P]
    L.ivhd_knn_index_query.restype = i32
    L.ivhd_knn_index_destroy.argtypes = [P]
    L.ivhd_knn_index_destroy.restype = None
    L.ivhd_place_nn.argtypes = [P, i64, P, i64, i32, P, P]
    L.ivhd_place_nn.restype = i32
    L.ivhd_probe_wait_timeout.argtypes = [i32, P]
    L.ivhd_probe_wait_timeout.restype = i32
    L.ivhd_probe_grid_barrier_timeout.argtypes = [i32, P]
    L.ivhd_probe_grid_barrier_timeout.restype = i32
    L.ivhd_test_fail_alloc.argtypes = [i64]
    L.ivhd_test_fail_alloc.restype = None
    L.ivhd_test_live_allocs.argtypes = []
    L.ivhd_test_live_allocs.restype = i64
    L.ivhd_set_allocator.argtypes = [ALLOC_FN, FREE_FN, P]
    L.ivhd_set_allocator.restype = i32
    L.ivhd_eval_qnx.argtypes = [P, i64, P, i32, P, i64, P, ctypes.POINTER(ctypes.c_double), P]
    L.ivhd_eval_qnx.restype = i32
    L.ivhd_eval_cf.argtypes = [P, i64, P, i32, P, i64, ctypes.POINTER(ctypes.c_double), P]
    L.ivhd_eval_cf.restype = i32
    L.ivhd_eval_qnx_static.argtypes = [P, i64, P, i32, P, i64, P,
                                       ctypes.POINTER(ctypes.c_double), P]
    L.ivhd_eval_qnx_static.restype = i32
    L.ivhd_probe_gather.argtypes = [i64, i64, i32, ctypes.POINTER(ctypes.c_double), P]
    L.ivhd_probe_gather.restype = i32
    L.ivhd_probe_launch.argtypes = [i32, i32, i32, ctypes.POINTER(ctypes.c_double), P]
    L.ivhd_probe_launch.restype = i32
    L.ivhd_set_metric.argtypes = [P, i32]
    L.ivhd_set_metric.restype = i32
    L.ivhd_resample_random_neighbors.argtypes = [P, u64]
    L.ivhd_resample_random_neighbors.restype = i32
    L.ivhd_restrict_nn.argtypes = [P, P, i32, i32]
    L.ivhd_restrict_nn.restype = i32
    L.ivhd_adaptive_state.argtypes = [P, ctypes.POINTER(ctypes.c_float),
                                      ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
    L.ivhd_adaptive_state.restype = i32
    L.ivhd_create_batch.argtypes = [P, P, P, P, P, i32, ctypes.c_float, ctypes.POINTER(Params),
                                    i32, ctypes.POINTER(P)]
    L.ivhd_create_batch.restype = i32
    L.ivhd_autotune.argtypes = [P, i32, ctypes.POINTER(ctypes.c_int32),
                                ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                ctypes.POINTER(ctypes.c_float)]
    L.ivhd_autotune.restype = i32
    L.ivhd_gemm_bf16_tn.argtypes = [P, P, P, i64, i64, i64, P]
    L.ivhd_gemm_bf16_tn.restype = i32
    L.ivhd_mlp_create.argtypes = [i32, i32, i32, P, ctypes.POINTER(P)]
    L.ivhd_mlp_create.restype = i32
    L.ivhd_mlp_destroy.argtypes = [P]
    L.ivhd_mlp_destroy.restype = None
    L.ivhd_mlp_num_params.argtypes = [P]
    L.ivhd_mlp_num_params.restype = i64
    L.ivhd_mlp_set_params.argtypes = [P, P, i32]
    L.ivhd_mlp_set_params.restype = i32
    L.ivhd_mlp_get_params.argtypes = [P, P, i32]
    L.ivhd_mlp_get_params.restype = i32
    L.ivhd_mlp_loss_grad.argtypes = [P, P, i32, ctypes.c_float, P, i32,
                                     ctypes.POINTER(ctypes.c_double), P]
    L.ivhd_mlp_loss_grad.restype = i32
    L.ivhd_mlp_train_step.argtypes = [P, P, i32, ctypes.c_float, P, i32, ctypes.c_float,
                                      ctypes.POINTER(ctypes.c_double)]
    L.ivhd_mlp_train_step.restype = i32
    L.ivhd_mlp_forward.argtypes = [P, P, i32, ctypes.c_float, i64, P]
    L.ivhd_mlp_forward.restype = i32
    L.ivhd_mlp_launches.argtypes = [P]
    L.ivhd_mlp_launches.restype = i64
    L.ivhd_mlp_activations.argtypes = [P, i32, P, ctypes.POINTER(ctypes.c_int64)]
    L.ivhd_mlp_activations.restype = i32
    _lib = L
    return L


def check(status: int, what: str):
    if status != 0:
        raise IvhdError(status, what)
