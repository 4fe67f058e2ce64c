"""ctypes declarations of the C ABI in include/hps.h.

Argument marshalling only: every step of the solver runs in libhps_gb300.so.
Importing this module fails loudly when the library has not been built.
"""

from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_int, c_int64, c_void_p

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhps_gb300.so")

HPS_OK, HPS_ERR_INVALID, HPS_ERR_OOM, HPS_ERR_SINGULAR, HPS_ERR_CUDA, HPS_ERR_TIMEOUT = 0, -1, -2, -3, -4, -5
HPS_PENDING = 1
HPS_DTN, HPS_ITI = 0, 1
HPS_F64, HPS_C128 = 0, 1

EXPORTED = [
    "hps_nodes", "hps_sizes", "hps_build", "hps_solve", "hps_solve_batched", "hps_solve_multi", "hps_free",
    "hps_error_string", "hps_last_error_detail", "hps_device_bytes", "hps_last_launch_count",
    "hps_kernel_stats", "hps_set_profiling", "hps_solve_noalloc", "hps_refine", "hps_trace_count",
    "hps_trace_get", "hps_plan_bytes", "hps_solve_adjoint", "hps_coeff_gradient", "hps_gemm", "hps_getrf",
    "hps_debug_fail_alloc", "hps_debug_alloc_count", "hps_debug_wait_timeout",
    "hps_tune_set", "hps_tune_get",
    # request server (include/hps_serve.h)
    "hps_server_create", "hps_server_destroy", "hps_server_submit_build", "hps_server_submit_solve",
    "hps_server_wait", "hps_server_poll", "hps_server_get_stats", "hps_server_operator",
]

EVAL_FN = ctypes.CFUNCTYPE(c_int, c_void_p, c_int64, POINTER(c_double), POINTER(c_double))

KCLASSES = ["gemm", "lu_panel", "laswp_trsm", "trsm_diag", "assemble", "gather", "down", "other", "gemm_tc",
            "split"]


class hps_tree(ctypes.Structure):
    _fields_ = [("dim", c_int), ("lo", c_double * 3), ("hi", c_double * 3),
                ("uniform_depth", c_int), ("n_leaves", c_int64),
                ("morton", c_void_p), ("level", c_void_p)]


class hps_coeffs(ctypes.Structure):
    _fields_ = [("kind", c_int), ("dtype", c_int), ("eta", c_double), ("a", c_void_p),
                ("b", c_void_p * 3), ("c", c_void_p)]


class hps_options(ctypes.Structure):
    _fields_ = [("version", c_int), ("want_root_map", c_int), ("profile", c_int),
                ("lazy_root", c_int), ("graph_solve", c_int), ("iti_leaf", c_int), ("fp64_gemm", c_int),
                ("recompute_budget_mb", c_int)]


class hps_kernel_stat(ctypes.Structure):
    _fields_ = [("launches", c_int64), ("flops", c_double), ("ms", c_double), ("exec_flops", c_double)]


class hps_trace_rec(ctypes.Structure):
    _fields_ = [("kclass", c_int), ("m", c_int), ("n", c_int), ("k", c_int), ("batch", c_int64),
                ("flops", c_double), ("ms", c_double)]


class hps_server_options(ctypes.Structure):
    _fields_ = [("version", c_int), ("n_slots", c_int), ("n_streams", c_int), ("max_batch", c_int),
                ("hbm_budget", c_int64), ("lazy_root", c_int), ("n_builders", c_int), ("max_group", c_int),
                ("reserved", c_int * 5)]


class hps_ticket_info(ctypes.Structure):
    _fields_ = [("status", c_int), ("kind", c_int), ("slot", c_int), ("batch", c_int),
                ("t_submit_ms", c_double), ("t_start_ms", c_double), ("t_done_ms", c_double)]


class hps_server_stats(ctypes.Structure):
    _fields_ = [("solves", c_int64), ("builds", c_int64), ("batches", c_int64), ("max_batch_seen", c_int64),
                ("multi_batches", c_int64), ("max_group_seen", c_int64), ("resident_bytes", c_int64),
                ("hbm_budget", c_int64)]


_lib = None


def lib() -> ctypes.CDLL:
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build the CUDA extension first "
            "(python -m paper_2503_17535_gb300.build or __graft_entry__.build())")
    L = ctypes.CDLL(LIB_PATH)
    L.hps_nodes.argtypes = [POINTER(hps_tree), c_int, c_int, c_void_p, c_void_p]
    L.hps_nodes.restype = c_int
    L.hps_sizes.argtypes = [POINTER(hps_tree), c_int, c_int, POINTER(c_int64), POINTER(c_int64),
                            POINTER(c_int64)]
    L.hps_sizes.restype = c_int
    L.hps_build.argtypes = [POINTER(hps_tree), c_int, c_int, POINTER(hps_coeffs), c_void_p,
                            POINTER(hps_options), c_void_p, POINTER(c_void_p)]
    L.hps_build.restype = c_int
    L.hps_solve.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]
    L.hps_solve.restype = c_int
    L.hps_solve_batched.argtypes = [c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_void_p]
    L.hps_solve_batched.restype = c_int
    L.hps_solve_multi.argtypes = [c_int, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]
    L.hps_solve_multi.restype = c_int
    L.hps_free.argtypes = [c_void_p]
    L.hps_free.restype = None
    L.hps_error_string.argtypes = [c_int]
    L.hps_error_string.restype = c_char_p
    L.hps_last_error_detail.argtypes = [c_void_p, POINTER(c_int64)]
    L.hps_last_error_detail.restype = c_int
    L.hps_device_bytes.argtypes = [c_void_p]
    L.hps_device_bytes.restype = c_int64
    L.hps_last_launch_count.argtypes = [c_void_p]
    L.hps_last_launch_count.restype = c_int64
    L.hps_kernel_stats.argtypes = [c_void_p, c_int, POINTER(hps_kernel_stat)]
    L.hps_kernel_stats.restype = c_int
    L.hps_set_profiling.argtypes = [c_void_p, c_int]
    L.hps_set_profiling.restype = c_int
    L.hps_trace_count.argtypes = [c_void_p, POINTER(c_int64)]
    L.hps_trace_count.restype = c_int
    L.hps_trace_get.argtypes = [c_void_p, c_int64, POINTER(hps_trace_rec)]
    L.hps_trace_get.restype = c_int
    L.hps_plan_bytes.argtypes = [POINTER(hps_tree), c_int, c_int, c_int, POINTER(c_int64)]
    L.hps_plan_bytes.restype = c_int
    L.hps_solve_adjoint.argtypes = [c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_void_p]
    L.hps_solve_adjoint.restype = c_int
    L.hps_coeff_gradient.argtypes = [c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]
    L.hps_coeff_gradient.restype = c_int
    L.hps_gemm.argtypes = [c_int, c_int, c_int, c_int, c_int, c_int, c_double, c_void_p, c_int, c_int64,
                           c_void_p, c_int, c_int64, c_double, c_void_p, c_int, c_int64, c_void_p]
    L.hps_gemm.restype = c_int
    L.hps_getrf.argtypes = [c_int, c_int, c_int, c_int, c_void_p, c_int, c_int64, c_void_p, c_void_p, c_void_p]
    L.hps_getrf.restype = c_int
    L.hps_debug_fail_alloc.argtypes = [c_int64]
    L.hps_debug_fail_alloc.restype = None
    L.hps_debug_alloc_count.argtypes = []
    L.hps_debug_alloc_count.restype = c_int64
    L.hps_debug_wait_timeout.argtypes = [c_int, c_int, c_int64, c_void_p]
    L.hps_debug_wait_timeout.restype = c_int
    L.hps_tune_set.argtypes = [c_int, c_int]
    L.hps_tune_set.restype = c_int
    L.hps_tune_get.argtypes = [c_int, POINTER(c_int)]
    L.hps_tune_get.restype = c_int
    L.hps_server_create.argtypes = [POINTER(hps_server_options), POINTER(c_void_p)]
    L.hps_server_create.restype = c_int
    L.hps_server_destroy.argtypes = [c_void_p]
    L.hps_server_destroy.restype = None
    L.hps_server_submit_build.argtypes = [c_void_p, c_int, POINTER(hps_tree), c_int, c_int,
                                          POINTER(hps_coeffs), c_void_p, POINTER(hps_options),
                                          POINTER(c_int64)]
    L.hps_server_submit_build.restype = c_int
    L.hps_server_submit_solve.argtypes = [c_void_p, c_int, c_void_p, c_void_p, c_void_p, POINTER(c_int64)]
    L.hps_server_submit_solve.restype = c_int
    L.hps_server_wait.argtypes = [c_void_p, c_int64, POINTER(hps_ticket_info)]
    L.hps_server_wait.restype = c_int
    L.hps_server_poll.argtypes = [c_void_p, c_int64, POINTER(hps_ticket_info)]
    L.hps_server_poll.restype = c_int
    L.hps_server_get_stats.argtypes = [c_void_p, POINTER(hps_server_stats)]
    L.hps_server_get_stats.restype = c_int
    L.hps_server_operator.argtypes = [c_void_p, c_int, POINTER(c_void_p)]
    L.hps_server_operator.restype = c_int
    L.hps_solve_noalloc.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p]
    L.hps_solve_noalloc.restype = c_int
    L.hps_refine.argtypes = [POINTER(c_double), POINTER(c_double), c_int, c_double, c_int, c_int, c_int,
                             POINTER(EVAL_FN), POINTER(c_void_p), c_int64, POINTER(c_int64), c_void_p,
                             c_void_p, c_void_p]
    L.hps_refine.restype = c_int
    _lib = L
    return L
