"""Arnoldi steps per solve of the FP64 oracle on the benchmark workload (writes a JSON next to this file).

Workload: Wilson-clover coarse 8^4 (fine 16^4, c_sw = 1, m0 = -0.42), nv = 16;
GCRO-DR(50, k = 16, u = 10) with the Leja-ordered degree-4 GMRES polynomial
(Sec. 3.3-3.4) to a true relative residual of 1e-10, right-hand sides solved
one after another with the recycle space kept.  Only oracle/ and the shared
seeded generator are used.  The count scales the timed oracle samples of the
benchmark's CPU baseline to whole solves.

Run: python -m oracle.bench_iterations [nrhs]
"""
import json
import os
import sys
import time

import numpy as np

from oracle import coarse, krylov
from synthetic import draws
from synthetic.coarse_op import build_coarse_operator

KEY = (2, 0)


def main(nrhs: int = 4):
    op = build_coarse_operator(KEY, (16, 16, 16, 16), 16, -0.42, 1.0, device="cpu")
    s, h = op.self_blocks.numpy(), op.hop_blocks.numpy()
    N = s.shape[0] * s.shape[1]
    A = lambda v: coarse.apply(s, h, op.dims, v)
    theta, _ = krylov.poly_setup(A, draws.poly_start(KEY, N), 4)
    M = lambda v: krylov.poly_apply(A, theta, v)
    rec = krylov.Recycle()
    its, res, secs = [], [], []
    for i in range(nrhs):
        b = draws.rhs((*KEY, 100), 1, N, i)[0]
        t0 = time.perf_counter()
        x, info, rec = krylov.gcrodr(A, b, m=50, k=16, tol=1e-10, precond=M, recycle=rec, u_limit=10)
        secs.append(time.perf_counter() - t0)
        its.append(info.iterations)
        res.append(info.rel_residual)
        print(f"rhs {i}: {info.iterations} Arnoldi steps, {info.cycles} cycles, residual {info.rel_residual:.2e}, "
              f"{secs[-1]:.1f} s", flush=True)
    out = {"iterations_per_solve": float(np.mean(its[1:] if len(its) > 1 else its)), "iterations": its,
           "rel_residuals": res, "seconds": secs, "theta": [[t.real, t.imag] for t in theta],
           "workload": "wilson-clover coarse 8^4, nv=16, m0=-0.42; GCRO-DR(50,16,u=10) + Leja poly d=4; tol 1e-10",
           "note": "mean over right-hand sides 2..n (recycle space built by the first)"}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "bench_workload_iterations.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 4)
