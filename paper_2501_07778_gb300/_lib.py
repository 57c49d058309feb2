"""ctypes declarations of the C ABI in include/qtt.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libqtt.so")

QTT_OK = 0
QTT_EINVAL = -1
QTT_ENOMEM = -2
QTT_ECUDA = -3
QTT_ENOCONV = -4
QTT_ETIMEOUT = -5
QTT_ERANKCAP = -6
QTT_F64, QTT_F32, QTT_MIXED = 0, 1, 2
QTT_ORDER_Z_BLOCK, QTT_ORDER_CANONICAL = 0, 1
QTT_MAX_CORES = 40

ERR_NAMES = {0: "QTT_OK", -1: "QTT_EINVAL", -2: "QTT_ENOMEM", -3: "QTT_ECUDA", -4: "QTT_ENOCONV",
             -5: "QTT_ETIMEOUT", -6: "QTT_ERANKCAP"}


class QttProblem(C.Structure):
    _fields_ = [("L", C.c_int), ("q", C.c_int), ("patch_xy", C.POINTER(C.c_int)),
                ("E", C.c_double), ("nu", C.c_double), ("bc", C.POINTER(C.c_int)),
                ("n_body", C.c_int), ("body_terms", C.POINTER(C.c_int)), ("body_coef", C.POINTER(C.c_double)),
                ("n_trac", C.c_int), ("trac_where", C.POINTER(C.c_int)), ("trac_val", C.POINTER(C.c_double)),
                ("gamma", C.c_double), ("tol", C.c_double), ("n_dir", C.c_int), ("dir_terms", C.POINTER(C.c_int)),
                ("dir_coef", C.POINTER(C.c_double))]


class QttSolveOpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_rank", C.c_int), ("kick_rank", C.c_int), ("max_sweeps", C.c_int),
                ("local_direct_max", C.c_int), ("local_restart", C.c_int), ("local_max_cycles", C.c_int),
                ("precision", C.c_int), ("refine_max", C.c_int), ("inner_tol", C.c_double), ("verbose", C.c_int),
                ("tensor_cores", C.c_int)]


class QttSolveInfo(C.Structure):
    _fields_ = [("status", C.c_int), ("sweeps", C.c_int), ("local_solves", C.c_int), ("local_iters", C.c_int),
                ("max_rank", C.c_int), ("refinements", C.c_int), ("max_local_res", C.c_double),
                ("rel_residual", C.c_double), ("erank", C.c_double), ("checks", C.c_int),
                ("check_ms", C.c_double), ("refine_ms", C.c_double)]


P = C.c_void_p
PP = C.POINTER(C.c_void_p)
IP = C.POINTER(C.c_int)

SIGNATURES = {
    "qtt_tensor_create": (C.c_int, [C.c_int, IP, IP, IP, C.c_int, PP, PP]),
    "qtt_tensor_info": (C.c_int, [P, IP, IP, IP, IP, IP]),
    "qtt_tensor_get_cores": (C.c_int, [P, PP]),
    "qtt_tensor_core_ptr": (C.c_int, [P, C.c_int, PP]),
    "qtt_tensor_copy": (C.c_int, [P, C.c_int, PP, P]),
    "qtt_free": (None, [P]),
    "qtt_last_error": (C.c_char_p, []),
    "qtt_assemble_stiffness": (C.c_int, [C.POINTER(QttProblem), PP, PP, P]),
    "qtt_matvec": (C.c_int, [P, P, C.c_double, C.c_int, PP, P]),
    "qtt_round": (C.c_int, [P, C.c_double, C.c_int, P]),
    "qtt_axpby": (C.c_int, [C.c_double, P, C.c_double, P, PP, P]),
    "qtt_norm": (C.c_int, [P, C.POINTER(C.c_double), P]),
    "qtt_to_full": (C.c_int, [P, P, C.c_size_t, C.c_int, P]),
    "qtt_to_full_noalloc": (C.c_int, [P, P, C.c_size_t, P]),
    "qtt_solve": (C.c_int, [P, P, P, P, C.POINTER(QttSolveOpts), PP, C.POINTER(QttSolveInfo), P]),
    "qtt_residual": (C.c_int, [P, P, P, C.POINTER(C.c_double), P]),
    "qtt_residual_fe": (C.c_int, [P, P, P, C.POINTER(C.c_double), P]),
    "qtt_residual_fe_tt": (C.c_int, [P, P, P, C.c_double, C.c_int, PP, C.POINTER(C.c_double), P]),
    "qtt_fe_apply": (C.c_int, [P, P, P, C.c_size_t, P]),
    "qtt_round_residual": (C.c_int, [P, P, P, C.c_int, C.c_ulonglong, C.POINTER(C.c_double), PP, P]),
    "qtt_solve_batched": (C.c_int, [C.c_int, PP, PP, PP, C.POINTER(QttSolveOpts), C.c_int, PP,
                                    C.POINTER(QttSolveInfo), P]),
    "qtt_ws_forward": (C.c_int, [C.c_int] * 4 + [P] * 10 + [P]),
    "qtt_ws_backward": (C.c_int, [C.c_int] * 4 + [P] * 13 + [P]),
    "qtt_ws_basis_gram": (C.c_int, [C.c_int, C.c_int, PP, C.POINTER(C.c_double), P]),
    "qtt_ws_tt_loss": (C.c_int, [C.c_int, C.c_int, IP, C.c_int, P, C.c_int, PP, C.POINTER(C.c_double),
                                 C.POINTER(C.c_double), P, P, P]),
    "qtt_ws_adam": (C.c_int, [C.c_int, P, P, P, P, C.c_float, C.c_float, C.c_float, C.c_float, C.c_int, P]),
    "qtt_ws_to_tensor": (C.c_int, [P, C.c_int, IP, C.c_int, C.c_double, PP, P]),
    "qtt_gemm_tf32x3": (C.c_int, [C.c_int, C.c_int, C.c_int, P, C.c_int, P, C.c_int, P, C.c_int, P]),
    "qtt_autotune_table": (C.c_int, [C.c_int, IP, IP, IP, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "qtt_kernel_launches": (C.c_ulonglong, []),
    "qtt_device_allocations": (C.c_ulonglong, []),
    "qtt_measure_fma_peak": (C.c_int, [C.c_int, C.POINTER(C.c_double), P]),
    "qtt_profile_enable": (C.c_int, [C.c_int]),
    "qtt_profile_read": (C.c_int, [C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double),
                                   C.POINTER(C.c_longlong)]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libqtt.so; raises if it is missing (there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing: run __graft_entry__.build() first")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    return list(SIGNATURES)
