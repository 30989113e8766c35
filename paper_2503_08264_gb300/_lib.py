"""ctypes declarations of the libqem C ABI (include/qem.h).

Argument marshalling only: every computation of the E-step and M-step runs in
the library's CUDA kernels.  Loading fails loudly when the library has not
been built; there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libqem.so")

QEM_MAX_LEVELS = 4
QEM_GAMMA_TRIES = 8

QEM_OK, QEM_ERR_INVALID_ARG, QEM_ERR_UNSUPPORTED, QEM_ERR_OOM, QEM_ERR_CUDA, QEM_ERR_NUMERIC, QEM_ERR_TIMEOUT = range(7)
QEM_PREC_FP32, QEM_PREC_BF16, QEM_PREC_BF16X3, QEM_PREC_TF32 = 0, 1, 2, 3
QEM_TILE_AUTO, QEM_TUNE_FORCE = -1, 1
QEM_MLP_DIM, QEM_MLP_HIDDEN, QEM_MLP_PARAMS = 18, 128, 26020


class LevelDesc(C.Structure):
    _fields_ = [("n", C.c_int64), ("dim", C.c_int), ("prior", C.c_int),
                ("prior_a", C.c_double), ("prior_b", C.c_double),
                ("lik", C.c_int), ("lik_var", C.c_double), ("n_obs", C.c_int), ("qfam", C.c_int),
                ("parent", C.c_void_p), ("x", C.c_void_p), ("y", C.c_void_p), ("chain", C.c_int),
                ("qcond", C.c_int)]


class ModelDesc(C.Structure):
    _fields_ = [("n_levels", C.c_int), ("levels", LevelDesc * QEM_MAX_LEVELS)]


class PlanOpts(C.Structure):
    _fields_ = [("K", C.c_int), ("precision", C.c_int), ("tile", C.c_int), ("stream", C.c_void_p),
                ("var_floor", C.c_double), ("timeout_s", C.c_double)]


# name -> (restype, argtypes); mirrors include/qem.h one to one
SIGNATURES = {
    "qem_status_string": (C.c_char_p, [C.c_int]),
    "qem_plan": (C.c_int, [C.POINTER(ModelDesc), C.POINTER(PlanOpts), C.POINTER(C.c_void_p)]),
    "qem_plan_destroy": (C.c_int, [C.c_void_p]),
    "qem_workspace_size": (C.c_int, [C.c_void_p, C.POINTER(C.c_size_t)]),
    "qem_layout": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                             C.POINTER(C.c_int64)]),
    "qem_sizes": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                            C.POINTER(C.c_int64)]),
    "qem_estep": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint64, C.c_uint64, C.c_void_p,
                            C.c_void_p]),
    "qem_estep_split_root": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint64, C.c_uint64, C.c_void_p,
                                       C.c_void_p, C.c_void_p]),
    "qem_set_perm": (C.c_int, [C.c_void_p, C.c_void_p]),
    "qem_set_elem_base": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    "qem_test_expire_wait": (C.c_int, [C.c_void_p, C.c_int]),
    "qem_estep_shard_forward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint64, C.c_uint64, C.c_void_p]),
    "qem_estep_shard_finish": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "qem_log_pmp_fresh": (C.c_int, [C.c_void_p, C.c_void_p, C.c_uint64, C.c_uint64, C.c_void_p]),
    "qem_predictive": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "qem_moments_rescale": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "qem_mstep": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_double,
                            C.c_int64]),
    "qem_mean_params": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "qem_log_pmp": (C.c_int, [C.c_void_p, C.c_void_p]),
    "qem_weights": (C.c_int, [C.c_void_p, C.c_void_p]),
    "qem_samples": (C.c_int, [C.c_void_p, C.c_void_p]),
    "qem_run": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_double, C.c_double, C.c_uint64, C.c_void_p,
                          C.c_void_p, C.c_void_p, C.c_void_p]),
    "qem_profile_enable": (C.c_int, [C.c_void_p, C.c_int]),
    "qem_profile_read": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
    "qem_profile_name": (C.c_char_p, [C.c_int]),
    "qem_diag_tc_gemm": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p]),
    "qem_run_kernels": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "qem_tune": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "qem_tune_get": (C.c_int, [C.c_void_p, C.POINTER(C.c_int)]),
    "qem_tune_set": (C.c_int, [C.c_void_p, C.POINTER(C.c_int)]),
    "qem_adjoint_pairs": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "qem_mlp_features": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int, C.c_int, C.c_void_p, C.c_void_p]),
    "qem_mlp_forward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    "qem_mlp_workspace_size": (C.c_int, [C.c_int64, C.POINTER(C.c_size_t)]),
    "qem_mlp_backward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p,
                                   C.c_void_p, C.c_void_p]),
    "qem_mlp_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_double,
                               C.c_double, C.c_double, C.c_double, C.c_void_p]),
    "qem_mlp_to_q": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    "qem_estep_single_noalloc": (C.c_int, [C.POINTER(LevelDesc), C.c_int, C.c_void_p, C.c_void_p, C.c_uint64,
                                           C.c_uint64, C.c_void_p, C.c_void_p, C.c_void_p]),
}

QEM_K_NAMES = ["sample_local", "parent_params", "finalize", "forward", "plate_sum", "root", "adjoint", "moments",
               "mstep", "operands", "adjoint_small"]

_lib = None


class QemError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = load().qem_status_string(code).decode() if _lib is not None else str(code)
        super().__init__(f"{where}: {msg}")


def load() -> C.CDLL:
    """Load libqem.so (built in-tree by build.py); raise if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libqem.so is not built ({LIB_PATH}); run paper_2503_08264_gb300/build.py")
        lib = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def check(code: int, where: str) -> None:
    if code != QEM_OK:
        raise QemError(code, where)
