"""Tensor-level convenience over the C ABI (argument marshalling only) and the autograd Function."""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _abi
from ._abi import OpDesc, SolveInfo, SolveParams, check, lib

_PREC_DT = {_abi.PREC_FP64: torch.complex128, _abi.PREC_FP32: torch.complex64, _abi.PREC_BF16: torch.complex64}


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t: torch.Tensor):
    return ctypes.c_void_p(t.data_ptr())


def solve_params(m=30, max_restarts=200, tol=1e-10, poly_degree=0, defl_k=0, recycle_updates=10,
                 precision=_abi.PREC_FP64, inner_tol=1e-5, max_ir=30, flags=_abi.COARSE_ZERO_GUESS, seed=1234,
                 poly_start: torch.Tensor | None = None) -> SolveParams:
    p = SolveParams()
    p.m, p.max_restarts, p.tol = m, max_restarts, tol
    p.poly_degree, p.defl_k, p.recycle_updates = poly_degree, defl_k, recycle_updates
    p.precision, p.inner_tol, p.max_ir, p.flags, p.seed = precision, inner_tol, max_ir, flags, seed
    p.poly_start = poly_start.data_ptr() if poly_start is not None else None
    p._keep = poly_start  # keep the start vector alive as long as the params
    return p


class CoarseOp:
    """Owns a ``coarse_op`` handle built from Galerkin blocks on the current CUDA device.

    self_blocks: complex128 [V, n, n]; hop_blocks: complex128 [V, 8, n, n] (or [V, 4, n, n]
    with ``assume_gamma5``), both CUDA tensors in the canonical layout of include/coarse.h.
    """

    def __init__(self, self_blocks: torch.Tensor, hop_blocks: torch.Tensor, dims, nv: int, mu: float = 0.0,
                 precisions=(_abi.PREC_FP32, _abi.PREC_BF16), max_nrhs: int = 1, assume_gamma5: bool = False,
                 stream=None):
        for t in (self_blocks, hop_blocks):
            if not (t.is_cuda and t.dtype == torch.complex128 and t.is_contiguous()):
                raise ValueError("blocks must be contiguous complex128 CUDA tensors")
        self.dims = tuple(int(v) for v in dims)
        self.nv = int(nv)
        self.n = 2 * self.nv
        self.V = int(np.prod(self.dims))
        self.mu = float(mu)
        self.max_nrhs = max_nrhs
        d = OpDesc()
        d.dims[:] = self.dims
        d.nv, d.mu, d.max_nrhs = self.nv, self.mu, max_nrhs
        d.flags = _abi.COARSE_ASSUME_GAMMA5 if assume_gamma5 else 0
        d.precisions = sum(1 << p for p in precisions) | 1
        h = ctypes.c_void_p()
        check(lib().coarse_op_create(ctypes.byref(d), _ptr(self_blocks), _ptr(hop_blocks), _stream(stream),
                                     ctypes.byref(h)))
        self.handle = h
        self.device = self_blocks.device

    # -- helpers
    def _vec(self, x: torch.Tensor, dtype) -> tuple[torch.Tensor, int]:
        if not x.is_cuda or x.dtype != dtype:
            raise ValueError(f"expected a CUDA tensor of dtype {dtype}")
        x = x.contiguous()
        N = self.V * self.n
        if x.numel() % N:
            raise ValueError(f"vector size {x.numel()} is not a multiple of V*n = {N}")
        return x, x.numel() // N

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().coarse_op_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def update(self, self_blocks, hop_blocks, stream=None):
        check(lib().coarse_op_update(self.handle, _ptr(self_blocks), _ptr(hop_blocks), _stream(stream)))

    # -- ABI calls
    def apply(self, x: torch.Tensor, precision: int = _abi.PREC_FP64, adjoint: bool = False, stream=None,
              out: torch.Tensor = None):
        """y = D_c x (or D_c^H x); x is (N,) or (nrhs, N) on this operator's device.  With BF16 and
        nrhs > 1 the columns go through the tensor-core multi-right-hand-side kernel."""
        x, nrhs = self._vec(x, _PREC_DT[precision])
        if out is None:
            y = torch.empty_like(x)
        else:
            if out.shape != x.shape or out.dtype != x.dtype or not out.is_contiguous() or out.device != x.device:
                raise ValueError("out must be a contiguous tensor of the shape, dtype and device of x")
            y = out
        fn = lib().coarse_apply_adjoint if adjoint else lib().coarse_apply
        check(fn(self.handle, _ptr(x), _ptr(y), nrhs, precision, _stream(stream)))
        return y

    def schur(self, x: torch.Tensor, precision: int = _abi.PREC_FP64, stream=None) -> torch.Tensor:
        """y = S x, S = 1 - D_ee^{-1} D_eo D_oo^{-1} D_oe on the even sites (x: V/2 * n entries)."""
        dt = _PREC_DT[precision]
        if not x.is_cuda or x.dtype != dt or x.numel() != self.V * self.n // 2:
            raise ValueError(f"expected a CUDA tensor of {self.V * self.n // 2} entries of dtype {dt}")
        x = x.contiguous()
        y = torch.empty_like(x)
        check(lib().coarse_schur_apply(self.handle, _ptr(x), _ptr(y), precision, _stream(stream)))
        return y

    def residual(self, b: torch.Tensor, x: torch.Tensor, stream=None):
        b, _ = self._vec(b, torch.complex128)
        x, _ = self._vec(x, torch.complex128)
        r = torch.empty_like(b)
        norms = (ctypes.c_double * 2)()
        check(lib().coarse_residual(self.handle, _ptr(b), _ptr(x), _ptr(r), norms, _stream(stream)))
        return r, norms[0], norms[1]

    def solve(self, b: torch.Tensor, x: torch.Tensor | None = None, params: SolveParams | None = None,
              adjoint: bool = False, stream=None, allow_not_converged: bool = False):
        b, nrhs = self._vec(b, torch.complex128)
        p = params if params is not None else solve_params()
        if x is None:
            x = torch.zeros_like(b)
        infos = (SolveInfo * nrhs)()
        fn = lib().coarse_solve_adjoint if adjoint else lib().coarse_solve
        rc = fn(self.handle, _ptr(b), _ptr(x), nrhs, ctypes.byref(p), infos, _stream(stream))
        check(rc, allow_not_converged)
        return x, [i.as_dict() for i in infos]

    def block_grad(self, lam: torch.Tensor, x: torch.Tensor, hop_dirs: int = 8, stream=None):
        """Block gradients -lambda_x x_y^H: g_self [V, n, n] and g_hop [V, hop_dirs, n, n]
        (hop_dirs = 4: with respect to the forward blocks of a gamma5-compressed input)."""
        lam, _ = self._vec(lam, torch.complex128)
        x, _ = self._vec(x, torch.complex128)
        gs = torch.empty((self.V, self.n, self.n), dtype=torch.complex128, device=lam.device)
        gh = torch.empty((self.V, hop_dirs, self.n, self.n), dtype=torch.complex128, device=lam.device)
        check(lib().coarse_block_grad(self.handle, _ptr(lam), _ptr(x), _ptr(gs), _ptr(gh), hop_dirs, _stream(stream)))
        return gs, gh

    def recycle_check(self, precision: int, odd_even: bool = False, adjoint: bool = False, stream=None) -> dict:
        """Defects of the held GCRO-DR recycle space: ||A u_i - c_i|| / ||c_i|| (max over i),
        max |C^H C - I|, the columns held and the updates made."""
        out = (ctypes.c_double * 4)()
        check(lib().coarse_recycle_check(self.handle, precision, int(odd_even), int(adjoint), out, _stream(stream)))
        return {"au_minus_c": out[0], "chc_minus_i": out[1], "k": int(out[2]), "updates": int(out[3])}

    def recycle_get(self, precision: int, odd_even: bool = False, adjoint: bool = False, cap: int = 64,
                    stream=None):
        """The held recycle space (U_k, C_k) as two [k, N] tensors (None if none is held)."""
        dt = _PREC_DT[precision]
        N = self.V * self.n // (2 if odd_even else 1)
        u = torch.empty((cap, N), dtype=dt, device=self.device)
        c = torch.empty_like(u)
        k = ctypes.c_int()
        check(lib().coarse_recycle_get(self.handle, precision, int(odd_even), int(adjoint), _ptr(u), _ptr(c), cap,
                                       ctypes.byref(k), _stream(stream)))
        if k.value == 0:
            return None
        return u[: k.value], c[: k.value]

    def recycle_set(self, precision: int, u: torch.Tensor | None, c: torch.Tensor | None, updates: int,
                    odd_even: bool = False, adjoint: bool = False, stream=None):
        """Install a recycle space ([k, N] tensors of the inner precision; None drops it)."""
        k = 0 if u is None else int(u.shape[0])
        if k:
            dt = _PREC_DT[precision]
            for t in (u, c):
                if not (t.is_cuda and t.dtype == dt and t.is_contiguous() and t.shape == u.shape):
                    raise ValueError(f"u and c must be contiguous CUDA tensors of dtype {dt} and one shape")
        check(lib().coarse_recycle_set(self.handle, precision, int(odd_even), int(adjoint),
                                       _ptr(u) if k else None, _ptr(c) if k else None, k, updates, _stream(stream)))

    def poly(self, precision: int):
        buf = (ctypes.c_double * 64)()
        d = ctypes.c_int()
        check(lib().coarse_op_poly(self.handle, precision, buf, 32, ctypes.byref(d)))
        a = np.array(buf[: 2 * d.value])
        return a[0::2] + 1j * a[1::2]


def solve_batched(ops, bs, xs, params: SolveParams, stream=None, allow_not_converged=False):
    """coarse_solve_batched over lists of CoarseOp, right-hand sides and solutions."""
    n = len(ops)
    H = (ctypes.c_void_p * n)(*[o.handle.value for o in ops])
    B = (ctypes.c_void_p * n)(*[b.data_ptr() for b in bs])
    X = (ctypes.c_void_p * n)(*[x.data_ptr() for x in xs])
    nr = [b.numel() // (o.V * o.n) for o, b in zip(ops, bs)]
    R = (ctypes.c_int * n)(*nr)
    infos = (SolveInfo * sum(nr))()
    rc = lib().coarse_solve_batched(H, n, B, X, R, ctypes.byref(params), infos, _stream(stream))
    check(rc, allow_not_converged)
    return [i.as_dict() for i in infos]


class CoarseSolve(torch.autograd.Function):
    """x = D_c^{-1} b with a hand-written backward: lambda = D_c^{-H} grad_x (adjoint solve through
    sigma3 D_c(-mu) sigma3), dL/db = lambda, and block gradients -lambda_x x_y^H.  Nothing of the
    Krylov process is stored; the backward recomputes through a fresh adjoint solve."""

    @staticmethod
    def forward(ctx, b, self_blocks, hop_blocks, op: CoarseOp, params: SolveParams):
        x, info = op.solve(b.detach(), params=params)
        ctx.op, ctx.params = op, params
        ctx.hop_dirs = hop_blocks.shape[1]   # 4: gamma5-compressed input (forward hops only)
        ctx.save_for_backward(x)
        return x

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        lam, _ = ctx.op.solve(gx.contiguous(), params=ctx.params, adjoint=True)
        gs = gh = None
        if ctx.needs_input_grad[1] or ctx.needs_input_grad[2]:
            gs, gh = ctx.op.block_grad(lam, x, hop_dirs=ctx.hop_dirs)
        return lam, gs, gh, None, None


def autotune_report() -> str:
    """Decisions of the library's launch autotuner (one line per kernel family and shape)."""
    buf = ctypes.create_string_buffer(1 << 16)
    check(lib().coarse_autotune_report(buf, len(buf)))
    return buf.value.decode()


def autotune_set(key: str, a: int, b: int = 0, c: int = 0) -> None:
    """Fix the launch configuration of one kernel family and shape (coarse_autotune_set)."""
    check(lib().coarse_autotune_set(key.encode(), a, b, c))


def measure_fp64_fma(iters: int = 20000, stream=None) -> float:
    """FP64 FMA throughput of the current device in TFLOP/s (coarse_measure_fp64_fma)."""
    out = ctypes.c_double()
    check(lib().coarse_measure_fp64_fma(iters, ctypes.byref(out), _stream(stream)))
    return out.value
