"""ctypes mirror of include/rsm.h and the loader of librsm.so.

Argument marshalling only: every computation runs in the CUDA library.  The
loader fails loudly when the library is missing; there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librsm.so")

RSM_OK = 0
RSM_ERR_INVALID_ARG = 1
RSM_ERR_NO_MEMORY = 2
RSM_ERR_UNDERDETERMINED = 3
RSM_ERR_ROWS_UNDERDETERMINED = 4
RSM_ERR_TIMEOUT = 5
RSM_ERR_CANCELLED = 6
RSM_ERR_CUDA = 7
RSM_ERR_NOT_IMPLEMENTED = 8
RSM_PENDING = 9
RSM_ERR_QUEUE_FULL = 10

RSM_F64, RSM_F32 = 0, 1
RSM_PREC_F64, RSM_PREC_F32X2, RSM_PREC_F32 = 0, 1, 2
RSM_COLS_RANDOM, RSM_COLS_ADJACENT, RSM_ROWS_RANDOM = 0, 1, 2
RSM_FAULT_ADMISSION, RSM_FAULT_ALLOC, RSM_FAULT_STALL, RSM_FAULT_DEVICE_WAIT = 0x1, 0x2, 0x4, 0x8


class rsm_config(C.Structure):
    _fields_ = [
        ("device", C.c_int32),
        ("max_slots", C.c_int32),
        ("hbm_budget_bytes", C.c_size_t),
        ("wait_timeout_ns", C.c_uint64),
        ("stream", C.c_void_p),
        ("fault_inject", C.c_uint32),
        ("reserved", C.c_uint32),
    ]


class rsm_problem(C.Structure):
    _fields_ = [
        ("m", C.c_int64),
        ("n", C.c_int64),
        ("r", C.c_int32),
        ("l", C.c_int32),
        ("n_minor", C.c_int32),
        ("variant", C.c_int32),
        ("trials", C.c_int64),
        ("seed", C.c_uint64),
        ("problem_id", C.c_uint32),
        ("y_dtype", C.c_int32),
        ("gram_prec", C.c_int32),
        ("solve_prec", C.c_int32),
        ("Y", C.c_void_p),
        ("ldy", C.c_int64),
        ("W", C.c_void_p),
        ("ldw", C.c_int64),
        ("U", C.c_void_p),
        ("ldu", C.c_int64),
        ("V", C.c_void_p),
        ("ldv", C.c_int64),
        ("debug_cols", C.c_void_p),
        ("debug_row_counts", C.c_void_p),
        ("debug_Z", C.c_void_p),
        ("debug_M", C.c_void_p),
        ("epsilon", C.c_double),
        ("coverage", C.c_int32),
        ("norm", C.c_int32),
        ("irls_iters", C.c_int32),
        ("reserved", C.c_int32),
        ("irls_delta_v", C.c_double),
        ("irls_delta_u", C.c_double),
        ("debug_visited", C.c_void_p),
    ]


class rsm_result(C.Structure):
    _fields_ = [
        ("status", C.c_int32),
        ("n_eig", C.c_int32),
        ("accepted_trials", C.c_int64),
        ("rows_underdetermined", C.c_int64),
        ("rows_selected", C.c_int64),
        ("kernel_launches", C.c_int64),
        ("eig_factor_bits", C.c_int32),
        ("eig_iterations", C.c_int32),
        ("eig_M", C.c_double * 32),
        ("eig_residual", C.c_double),
        ("e_known_rms", C.c_double),
        ("stage_ms", C.c_float * 12),
        ("queue_ms", C.c_double),
        ("run_ms", C.c_double),
        ("coverage", C.c_double),
        ("trials", C.c_int64),
    ]


class rsm_trial_plan(C.Structure):
    _fields_ = [
        ("p_visit", C.c_double),
        ("trials", C.c_double),
        ("p_visit_theorem3", C.c_double),
        ("trials_theorem3", C.c_double),
    ]


class rsm_tune(C.Structure):
    _fields_ = [
        ("schedule", C.c_int32),
        ("slab_mib", C.c_int32),
        ("variant", C.c_int32),
        ("candidates", C.c_int32),
        ("gram_ms", C.c_double),
        ("default_ms", C.c_double),
    ]


STAGES = ["setup", "pack_mask", "sample_cols", "select_gram", "minor_scatter", "eig_M", "solve_U", "residual", "total"]


# every symbol include/rsm.h declares, with (restype, argtypes)
SIGNATURES = {
    "rsm_version": (C.c_char_p, []),
    "rsm_struct_size": (C.c_size_t, [C.c_int32]),
    "rsm_status_string": (C.c_char_p, [C.c_int32]),
    "rsm_last_error": (C.c_char_p, []),
    "rsm_create": (C.c_int32, [C.POINTER(rsm_config), C.POINTER(C.c_void_p)]),
    "rsm_destroy": (None, [C.c_void_p]),
    "rsm_footprint_bytes": (C.c_size_t, [C.POINTER(rsm_problem)]),
    "rsm_decompose": (C.c_int32, [C.c_void_p, C.POINTER(rsm_problem), C.POINTER(rsm_result)]),
    "rsm_decompose_batch": (C.c_int32, [C.c_void_p, C.POINTER(rsm_problem), C.c_int32, C.POINTER(rsm_result)]),
    "rsm_submit": (C.c_int32, [C.c_void_p, C.POINTER(rsm_problem), C.POINTER(C.c_uint64)]),
    "rsm_submit_on": (C.c_int32, [C.c_void_p, C.POINTER(rsm_problem), C.c_void_p, C.POINTER(C.c_uint64)]),
    "rsm_poll": (C.c_int32, [C.c_void_p, C.c_uint64, C.POINTER(rsm_result)]),
    "rsm_wait": (C.c_int32, [C.c_void_p, C.c_uint64, C.c_uint64, C.POINTER(rsm_result)]),
    "rsm_cancel": (C.c_int32, [C.c_void_p, C.c_uint64]),
    "rsm_release": (C.c_int32, [C.c_void_p, C.c_uint64]),
    "rsm_pack_mask": (C.c_int32, [C.c_void_p, C.c_int64, C.c_int64, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p]),
    "rsm_sample_columns": (C.c_int32, [C.c_int64, C.c_int32, C.c_int64, C.c_int64, C.c_uint64, C.c_uint32, C.c_int32,
                                       C.c_void_p, C.c_void_p]),
    "rsm_select_rows": (C.c_int32, [C.c_void_p, C.c_int64, C.c_int64, C.c_void_p, C.c_int32, C.c_int64, C.c_void_p,
                                    C.c_void_p, C.c_void_p, C.c_void_p]),
    "rsm_eig_smallest": (C.c_int32, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_int64,
                                     C.POINTER(rsm_result)]),
    "rsm_plan_trials": (C.c_int32, [C.c_int64, C.c_int64, C.c_double, C.c_int32, C.c_int32, C.c_int32, C.c_double,
                                    C.POINTER(rsm_trial_plan)]),
    "rsm_check_fp64_math": (C.c_int32, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    "rsm_probe_gather": (C.c_int32, [C.c_void_p, C.c_int64, C.c_int64, C.c_int32, C.c_int32, C.c_void_p,
                                     C.c_void_p]),
    "rsm_autotune": (C.c_int32, [C.c_void_p, C.POINTER(rsm_problem), C.c_int32, C.POINTER(rsm_tune)]),
    "rsm_autotune_lookup": (C.c_int32, [C.c_void_p, C.POINTER(rsm_problem), C.POINTER(rsm_tune)]),
    "rsm_autotune_clear": (C.c_int32, [C.c_void_p]),
    "rsm_autotune_save": (C.c_int32, [C.c_void_p, C.c_char_p]),
    "rsm_autotune_load": (C.c_int32, [C.c_void_p, C.c_char_p]),
    "rsm_residual_noalloc": (C.c_int32, [C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_int64, C.c_void_p,
                                         C.c_int64, C.c_void_p, C.c_int64, C.c_int64, C.c_int64, C.c_int32,
                                         C.c_void_p, C.c_void_p]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load librsm.so and bind every entry point; raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is not built: run `python -m paper_1411_0814_gb300.build` "
                           "(or __graft_entry__.build()); there is no CPU fallback")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    for which, cls in enumerate((rsm_config, rsm_problem, rsm_result)):
        if lib.rsm_struct_size(which) != C.sizeof(cls):
            raise RuntimeError(f"ABI mismatch for {cls.__name__}: C {lib.rsm_struct_size(which)} vs "
                               f"ctypes {C.sizeof(cls)}")
    _lib = lib
    return lib
