"""Arnoldi steps per solve of the FP64 oracle on a benchmark workload (writes a JSON next to this file).

Workloads (Sec. 3.3-3.4 solver, right-hand sides solved one after another with the recycle
space kept, true relative residual 1e-10):
  wilson8  Wilson-clover coarse 8^4 (fine 16^4, c_sw = 1, m0 = -0.42), nv = 16;
           GCRO-DR(50, k = 16, u = 10) with the Leja-ordered degree-4 GMRES polynomial.
  tm16     twisted mass coarse 16^4 (fine 32^4, c_sw = 1, m0 = -0.42, mu = 3e-3), nv = 24;
           GCRO-DR(50, k = 32, u = 10) with the degree-8 polynomial.
Only oracle/ and the shared seeded generator are used.  The count scales the timed oracle
samples of the benchmark's CPU baseline to whole solves.

Run: python -m oracle.bench_iterations <workload> [nrhs]
"""
import json
import os
import sys
import time

import numpy as np

from oracle import coarse, krylov
from synthetic import draws
from synthetic.coarse_op import build_coarse_operator

WORKLOADS = {
    # name: (key, fine dims, nv, m0, mu, poly degree, k, description)
    "wilson8": ((2, 0), (16, 16, 16, 16), 16, -0.42, 0.0, 4, 16,
                "wilson-clover coarse 8^4, nv=16, m0=-0.42; GCRO-DR(50,16,u=10) + Leja poly d=4; tol 1e-10"),
    "tm16": ((3, 0), (32, 32, 32, 32), 24, -0.42, 3e-3, 8, 32,
             "twisted mass coarse 16^4, nv=24, m0=-0.42, mu=3e-3; GCRO-DR(50,32,u=10) + Leja poly d=8; tol 1e-10"),
}


def path(name: str) -> str:
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), f"bench_iterations_{name}.json")


def main(name: str, nrhs: int = 4):
    key, fine, nv, m0, mu, d, k, desc = WORKLOADS[name]
    t0 = time.perf_counter()
    op = build_coarse_operator(key, fine, nv, m0, 1.0, device="cpu")
    s, h = op.self_blocks.numpy(), op.hop_blocks.numpy()
    del op
    print(f"operator built in {time.perf_counter() - t0:.0f} s", flush=True)
    N = s.shape[0] * s.shape[1]
    cdims = tuple(L // 2 for L in fine)
    A = lambda v: coarse.apply(s, h, cdims, v, mu)
    theta, _ = krylov.poly_setup(A, draws.poly_start(key, N), d)
    M = lambda v: krylov.poly_apply(A, theta, v)
    rec = krylov.Recycle()
    its, res, secs = [], [], []
    for i in range(nrhs):
        b = draws.rhs((*key, 100), 1, N, i)[0]
        t0 = time.perf_counter()
        x, info, rec = krylov.gcrodr(A, b, m=50, k=k, tol=1e-10, precond=M, recycle=rec, u_limit=10)
        secs.append(time.perf_counter() - t0)
        its.append(info.iterations)
        res.append(info.rel_residual)
        print(f"rhs {i}: {info.iterations} Arnoldi steps, {info.cycles} cycles, residual {info.rel_residual:.2e}, "
              f"{secs[-1]:.1f} s", flush=True)
    out = {"iterations_per_solve": float(np.mean(its[1:] if len(its) > 1 else its)), "iterations": its,
           "rel_residuals": res, "seconds": secs, "theta": [[t.real, t.imag] for t in theta],
           "workload": desc, "note": "mean over right-hand sides 2..n (recycle space built by the first)"}
    with open(path(name), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main(sys.argv[1], int(sys.argv[2]) if len(sys.argv) > 2 else 4)
