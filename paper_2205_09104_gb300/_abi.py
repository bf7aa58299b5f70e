"""ctypes mirror of include/coarse.h (structs, enums, function prototypes)."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
lib_path = os.path.join(HERE, "_build", "libcoarse.so")

PREC_FP64, PREC_FP32, PREC_BF16 = 0, 1, 2
COARSE_ASSUME_GAMMA5 = 0x1
COARSE_ZERO_GUESS = 0x1
COARSE_REBUILD_POLY = 0x2
COARSE_RESET_RECYCLE = 0x4
COARSE_TIME_APPLY = 0x8
COARSE_POLY_BF16 = 0x10
COARSE_ODD_EVEN = 0x20
COARSE_RECYCLE_FULL_CYCLE = 0x40
COARSE_PIPELINED = 0x80

STATUS = {0: "OK", -1: "INVALID_ARG", -2: "OOM", -3: "CUDA", -4: "NOT_CONVERGED", -5: "BREAKDOWN",
          -6: "NONFINITE", -7: "TIMEOUT", -8: "NOT_GAMMA5"}

# every symbol the header declares
EXPORTS = ["coarse_op_create", "coarse_op_update", "coarse_op_destroy", "coarse_apply", "coarse_apply_adjoint",
           "coarse_residual", "coarse_solve", "coarse_solve_adjoint", "coarse_solve_batched", "coarse_block_grad",
           "coarse_op_poly", "coarse_last_error", "coarse_version", "coarse_residual_noalloc",
           "coarse_autotune_report", "coarse_schur_apply", "coarse_recycle_check",
           "coarse_recycle_get", "coarse_autotune_set", "coarse_measure_fp64_fma", "coarse_recycle_set"]


class CoarseError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class OpDesc(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int32 * 4), ("nv", ctypes.c_int32), ("mu", ctypes.c_double),
                ("flags", ctypes.c_uint32), ("max_nrhs", ctypes.c_int32), ("precisions", ctypes.c_uint32)]


class SolveParams(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int32), ("max_restarts", ctypes.c_int32), ("tol", ctypes.c_double),
                ("poly_degree", ctypes.c_int32), ("defl_k", ctypes.c_int32), ("recycle_updates", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("inner_tol", ctypes.c_double), ("max_ir", ctypes.c_int32),
                ("flags", ctypes.c_uint32), ("seed", ctypes.c_uint64), ("poly_start", ctypes.c_void_p)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iterations", ctypes.c_int32), ("matvecs", ctypes.c_int32),
                ("cycles", ctypes.c_int32), ("ir_steps", ctypes.c_int32), ("recycle_updates", ctypes.c_int32),
                ("rel_residual", ctypes.c_double), ("setup_ms", ctypes.c_double), ("solve_ms", ctypes.c_double),
                ("apply_ms", ctypes.c_double), ("apply_count", ctypes.c_int32), ("kernel_launches", ctypes.c_int32),
                ("apply_bytes", ctypes.c_double), ("apply_ms_prec", ctypes.c_double * 3),
                ("apply_bytes_prec", ctypes.c_double * 3), ("apply_count_prec", ctypes.c_int32 * 3),
                ("breakdowns", ctypes.c_int32)]

    def as_dict(self):
        out = {}
        for f, _ in self._fields_:
            v = getattr(self, f)
            out[f] = list(v) if isinstance(v, ctypes.Array) else v
        return out


_lib = None


def lib() -> ctypes.CDLL:
    """The loaded CUDA library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(lib_path):
        raise ImportError(f"CUDA library {lib_path} is missing: run paper_2205_09104_gb300.build() "
                          "(there is no CPU fallback)")
    L = ctypes.CDLL(lib_path)
    vp, i32, u32, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32, ctypes.c_double
    P = ctypes.POINTER
    L.coarse_op_create.argtypes = [P(OpDesc), vp, vp, vp, P(vp)]
    L.coarse_op_update.argtypes = [vp, vp, vp, vp]
    L.coarse_op_destroy.argtypes = [vp]
    L.coarse_op_destroy.restype = None
    L.coarse_apply.argtypes = [vp, vp, vp, i32, i32, vp]
    L.coarse_apply_adjoint.argtypes = [vp, vp, vp, i32, i32, vp]
    L.coarse_residual.argtypes = [vp, vp, vp, vp, P(dbl), vp]
    L.coarse_schur_apply.argtypes = [vp, vp, vp, i32, vp]
    L.coarse_residual_noalloc.argtypes = [vp, vp, vp, vp, P(dbl), vp]
    L.coarse_solve.argtypes = [vp, vp, vp, i32, P(SolveParams), P(SolveInfo), vp]
    L.coarse_solve_adjoint.argtypes = [vp, vp, vp, i32, P(SolveParams), P(SolveInfo), vp]
    L.coarse_solve_batched.argtypes = [P(vp), i32, P(vp), P(vp), P(i32), P(SolveParams), P(SolveInfo), vp]
    L.coarse_block_grad.argtypes = [vp, vp, vp, vp, vp, i32, vp]
    L.coarse_op_poly.argtypes = [vp, i32, P(dbl), i32, P(i32)]
    L.coarse_recycle_check.argtypes = [vp, i32, i32, i32, P(dbl), vp]
    L.coarse_recycle_get.argtypes = [vp, i32, i32, i32, vp, vp, i32, P(i32), vp]
    L.coarse_recycle_set.argtypes = [vp, i32, i32, i32, vp, vp, i32, i32, vp]
    L.coarse_autotune_report.argtypes = [ctypes.c_char_p, ctypes.c_longlong]
    L.coarse_autotune_set.argtypes = [ctypes.c_char_p, i32, i32, i32]
    L.coarse_measure_fp64_fma.argtypes = [i32, P(dbl), vp]
    L.coarse_last_error.restype = ctypes.c_char_p
    L.coarse_version.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("coarse_op_destroy", "coarse_last_error", "coarse_version"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def check(rc: int, allow_not_converged: bool = False):
    if rc == 0 or (allow_not_converged and rc == -4):
        return rc
    raise CoarseError(rc, lib().coarse_last_error().decode())
