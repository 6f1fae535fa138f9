"""ctypes binding of ``libgbcg.so`` (the C ABI in ``include/gbcg.h``).

Argument marshalling only: every step of a product or a solve runs in the
library's CUDA kernels.  Loading fails loudly when the library has not been
built; there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgbcg.so")

GBCG_CSR, GBCG_SYM_CSR_UPPER, GBCG_CSC = 0, 1, 2
GBCG_FP64, GBCG_FP32_IR, GBCG_FP32_RU = 0, 1, 2
GBCG_HOST, GBCG_DEVICE = 0, 1
GBCG_STANDARD, GBCG_PIPELINED = 0, 1
STATUS_NAMES = ["OK", "INVALID", "NOT_SPD", "MAXIT", "NONFINITE", "TIMEOUT", "CUDA", "NOMEM"]

# Every entry point declared in include/gbcg.h.
EXPORTS = ["gbcg_create", "gbcg_destroy", "gbcg_spmv", "gbcg_spmv_f32", "gbcg_solve", "gbcg_solve_async", "gbcg_stats",
           "gbcg_status_string", "gbcg_last_error", "gbcg_selftest_wait_timeout", "gbcg_solve_csr_static",
           "gbcg_batch_create", "gbcg_batch_destroy", "gbcg_batch_autotune", "gbcg_batch_set_tuning",
           "gbcg_batch_solve", "gbcg_batch_instance_times", "gbcg_batch_stats",
           "gbcg_batch_selftest_group_timeout", "gbcg_update_values", "gbcg_grad_values", "gbcg_element_grad",
           "gbcg_assemble", "gbcg_ablation_spmv", "gbcg_ablation_solve", "gbcg_measure_fp64_fma_rate"]
STATIC_MAX_N = 680000


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("max_outer", ctypes.c_int32), ("inner_tol", ctypes.c_double),
                ("wait_timeout_ms", ctypes.c_int32), ("max_restarts", ctypes.c_int32), ("variant", ctypes.c_int32),
                ("pad_", ctypes.c_int32)]


# gbcg_device_info, the device-resident result of gbcg_solve_async (32 bytes)
DEVICE_INFO_BYTES = 32


class Info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("outer", ctypes.c_int32), ("status", ctypes.c_int32),
                ("pad_", ctypes.c_int32), ("rel_res_recursive", ctypes.c_double),
                ("rel_res_true", ctypes.c_double), ("ms", ctypes.c_double), ("kernel_ms", ctypes.c_double),
                ("kernel_launches", ctypes.c_int32), ("launches", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz_input", ctypes.c_int64), ("nnz_full", ctypes.c_int64),
                ("stored_slots", ctypes.c_int64), ("plan_slots", ctypes.c_int64), ("long_rows", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("spmv_bytes_fp64", ctypes.c_int64),
                ("spmv_bytes_fp32", ctypes.c_int64), ("ext_slots", ctypes.c_int64), ("format", ctypes.c_int32),
                ("grid_ctas", ctypes.c_int32), ("layout", ctypes.c_int32), ("tiles", ctypes.c_int32),
                ("index_bytes", ctypes.c_int32), ("pad_", ctypes.c_int32)]


class BatchInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("outer", ctypes.c_int32), ("status", ctypes.c_int32),
                ("pad_", ctypes.c_int32), ("rel_res_true", ctypes.c_double)]


class BatchOpts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("max_outer", ctypes.c_int32), ("inner_tol", ctypes.c_double),
                ("fixed_order", ctypes.c_int32), ("max_group", ctypes.c_int32), ("force_group", ctypes.c_int32),
                ("wait_timeout_ms", ctypes.c_int32)]


class BatchReport(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double), ("kernel_ms", ctypes.c_double), ("span_ms", ctypes.c_double),
                ("busy_fraction", ctypes.c_double), ("products", ctypes.c_int64), ("iterations", ctypes.c_int64),
                ("max_iterations", ctypes.c_int32), ("launches", ctypes.c_int32), ("graph", ctypes.c_int32),
                ("threads", ctypes.c_int32), ("cluster", ctypes.c_int32), ("clusters", ctypes.c_int32),
                ("groups", ctypes.c_int32), ("max_group", ctypes.c_int32)]


class BatchTuning(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int32), ("cluster", ctypes.c_int32), ("rows_per_warp", ctypes.c_int32 * 8),
                ("clusters", ctypes.c_int32), ("from_cache", ctypes.c_int32), ("candidates", ctypes.c_int32),
                ("pad_", ctypes.c_int32), ("probe_ms", ctypes.c_double)]


class BatchStats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
                ("iter_bytes_fp32", ctypes.c_int64), ("iter_bytes_fp64", ctypes.c_int64), ("count", ctypes.c_int32),
                ("nrhs", ctypes.c_int32), ("threads", ctypes.c_int32 * 2), ("cluster", ctypes.c_int32 * 2),
                ("rows_per_warp", (ctypes.c_int32 * 8) * 2)]


class GbcgError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{where}: GBCG_{name}: {msg}")
        self.status = status


_lib = None


def load(path: str = LIB_PATH):
    """Load libgbcg.so; raises if it is missing (build it with ``build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: the CUDA library must be built (paper_1010_4639_gb300.build())")
    lib = ctypes.CDLL(path)
    vp, i32, i64, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    lib.gbcg_create.argtypes = [ctypes.POINTER(vp), i32, i64, i64, vp, vp, vp, i32, i32, vp]
    lib.gbcg_destroy.argtypes = [vp]
    lib.gbcg_spmv.argtypes = [vp, vp, vp, vp]
    lib.gbcg_spmv_f32.argtypes = [vp, vp, vp, vp]
    lib.gbcg_solve.argtypes = [vp, vp, vp, d, i32, ctypes.POINTER(Opts), ctypes.POINTER(Info), vp]
    lib.gbcg_solve_async.argtypes = [vp, vp, vp, d, i32, ctypes.POINTER(Opts), vp, vp]
    lib.gbcg_stats.argtypes = [vp, ctypes.POINTER(Stats)]
    lib.gbcg_status_string.argtypes = [ctypes.c_int]
    lib.gbcg_status_string.restype = ctypes.c_char_p
    lib.gbcg_last_error.argtypes = []
    lib.gbcg_last_error.restype = ctypes.c_char_p
    lib.gbcg_selftest_wait_timeout.argtypes = [i32, i32, vp]
    lib.gbcg_solve_csr_static.argtypes = [i64, i64, vp, vp, vp, vp, vp, d, i32, ctypes.POINTER(Info), vp]
    lib.gbcg_batch_create.argtypes = [ctypes.POINTER(vp), i32, vp, vp, vp, vp, i32, i32, i32, vp]
    lib.gbcg_batch_destroy.argtypes = [vp]
    lib.gbcg_batch_autotune.argtypes = [vp, i32, ctypes.POINTER(BatchTuning), vp]
    lib.gbcg_batch_set_tuning.argtypes = [vp, i32, ctypes.POINTER(BatchTuning)]
    lib.gbcg_batch_solve.argtypes = [vp, vp, vp, d, i32, ctypes.POINTER(BatchOpts), vp,
                                     ctypes.POINTER(BatchReport), vp]
    lib.gbcg_batch_instance_times.argtypes = [vp, vp, vp, vp]
    lib.gbcg_batch_stats.argtypes = [vp, ctypes.POINTER(BatchStats)]
    lib.gbcg_batch_selftest_group_timeout.argtypes = [vp, i32, vp]
    lib.gbcg_update_values.argtypes = [vp, vp, i32, vp]
    lib.gbcg_grad_values.argtypes = [i32, i64, i64, vp, vp, i32, vp, vp, vp, vp]
    lib.gbcg_element_grad.argtypes = [i64, i32, vp, vp, vp, vp, vp]
    lib.gbcg_assemble.argtypes = [i64, vp, vp, vp, vp, vp, vp]
    lib.gbcg_ablation_spmv.argtypes = [i32, i64, vp, vp, vp, vp, vp, vp]
    lib.gbcg_ablation_solve.argtypes = [i32, i64, vp, vp, vp, vp, vp, d, i32, ctypes.POINTER(Info), vp]
    lib.gbcg_measure_fp64_fma_rate.argtypes = [ctypes.POINTER(d), vp]
    for name in ("gbcg_create", "gbcg_destroy", "gbcg_spmv", "gbcg_spmv_f32", "gbcg_solve", "gbcg_stats",
                 "gbcg_selftest_wait_timeout", "gbcg_solve_csr_static", "gbcg_batch_create", "gbcg_batch_destroy",
                 "gbcg_batch_autotune", "gbcg_batch_set_tuning", "gbcg_batch_solve", "gbcg_batch_instance_times",
                 "gbcg_batch_stats", "gbcg_batch_selftest_group_timeout", "gbcg_update_values",
                 "gbcg_grad_values", "gbcg_element_grad", "gbcg_assemble", "gbcg_ablation_spmv",
                 "gbcg_ablation_solve", "gbcg_measure_fp64_fma_rate"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def last_error() -> str:
    return load().gbcg_last_error().decode()


def check(rc: int, where: str):
    if rc != 0:
        raise GbcgError(rc, where, last_error())
