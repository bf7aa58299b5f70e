"""GB300 coarsest-level solver for aggregation-based multigrid (arXiv:2205.09104).

Thin Python binding of the C ABI declared in ``include/coarse.h``: the
functions below carry the C names and only marshal arguments (tensor data
pointers, the current CUDA stream, ctypes structs).  Every step of the
apply and of the solver runs in the compiled CUDA library
``_build/libcoarse.so``; importing the binding without that library (or
calling it without a CUDA device) raises, there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

from . import _abi
from ._abi import (COARSE_ASSUME_GAMMA5, COARSE_ODD_EVEN, COARSE_POLY_BF16, COARSE_REBUILD_POLY,
                   COARSE_PIPELINED, COARSE_RECYCLE_FULL_CYCLE, COARSE_RESET_RECYCLE, COARSE_TIME_APPLY, COARSE_ZERO_GUESS, PREC_BF16,
                   PREC_FP32, PREC_FP64, CoarseError, SolveInfo, SolveParams, lib, lib_path)
from .op import (CoarseOp, CoarseSolve, autotune_report, autotune_set, measure_fp64_fma, solve_batched,
                 solve_params)

__all__ = ["CoarseOp", "CoarseSolve", "autotune_report", "autotune_set", "measure_fp64_fma", "solve_batched", "solve_params", "SolveParams", "SolveInfo", "CoarseError", "lib", "lib_path",
           "PREC_FP64", "PREC_FP32", "PREC_BF16", "COARSE_ZERO_GUESS", "COARSE_REBUILD_POLY",
           "COARSE_RESET_RECYCLE", "COARSE_ASSUME_GAMMA5", "COARSE_TIME_APPLY", "COARSE_POLY_BF16", "COARSE_ODD_EVEN",
           "COARSE_RECYCLE_FULL_CYCLE", "COARSE_PIPELINED", "build"]


def build(force: bool = False) -> str:
    """Compile the CUDA library for sm_103a in-tree (nvcc) and return its path."""
    from .build import build as _b
    return _b(force=force)
