#!/usr/bin/env python
"""Benchmark: coarsest-level solves/s at relative residual 1e-10 on the Wilson-clover
8^4 coarse lattice (n = 32 dof per site, 131072 unknowns), with the D_c apply's
achieved HBM bandwidth against the measured peak.

One step = one right-hand side solved to a true FP64 relative residual of
1e-10 with GMRES(50) + Leja-ordered degree-4 polynomial + GCRO-DR k = 16
(u = 10) in the inner precision, inside FP64 iterative refinement.  The
polynomial and the recycle space are built during the warm-up solves and
reused, as for repeated coarsest-level solves with one operator.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FINE_DIMS = (16, 16, 16, 16)
NV = 16
M0 = -0.42
CSW = 1.0
KEY = (2, 0)
PARAMS = dict(m=50, poly_degree=4, defl_k=16, recycle_updates=10, tol=1e-10, max_restarts=100, max_ir=20)
WORKLOAD = ("wilson-clover coarse 8^4 (fine 16^4, 2^4 aggregates), nv=16 -> n=32, 131072 unknowns, "
            "m0=-0.42, c_sw=1.0; GMRES(50) + Leja poly d=4 + GCRO-DR k=16 u=10; {prec} inner + FP64 "
            "refinement to 1e-10")
ORACLE_ITERS = os.path.join(ROOT, "oracle", "bench_workload_iterations.json")


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_init():
    from paper_2205_09104_gb300.replicas import dist_env
    return dist_env()


def run_gb300(args):
    import torch

    import paper_2205_09104_gb300 as cg
    from paper_2205_09104_gb300 import replicas
    from synthetic import draws
    from synthetic.coarse_op import build_coarse_operator

    world, rank, local = dist_init()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    prec = cg.PREC_BF16 if args.prec == "bf16" else cg.PREC_FP32
    poly_bf16 = prec == cg.PREC_FP32 and args.poly == "bf16"
    extra = (cg.COARSE_POLY_BF16 if poly_bf16 else 0) | (cg.COARSE_ODD_EVEN if args.oddeven == "on" else 0)
    # replicas: each rank solves its own right-hand sides with its own copy of the operator
    op = build_coarse_operator(KEY, FINE_DIMS, NV, M0, CSW, device=dev)
    cop = cg.CoarseOp(op.self_blocks, op.hop_blocks, op.dims, op.nv,
                      precisions=(prec, cg.PREC_BF16) if poly_bf16 else (prec,))
    host_blocks = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        host_blocks = (op.self_blocks.cpu().numpy(), op.hop_blocks.cpu().numpy(), op.dims)
    del op
    torch.cuda.empty_cache()
    n, V = 2 * NV, cop.V
    N = V * n
    total = args.warmup + 2 * args.steps
    B = torch.from_numpy(draws.rhs(replicas.rhs_key(KEY, rank), total, N)).to(dev)
    S = torch.from_numpy(draws.rhs((*KEY, 50 + rank), 4, N)).to(dev)  # setup right-hand sides
    X = torch.zeros_like(B)
    # FP32 inner solves to 2e-6: two refinement steps reach 1e-10 ((2e-6)^2 with margin)
    inner_tol = args.inner_tol if args.inner_tol > 0 else (2e-6 if prec == cg.PREC_FP32 else 1e-2)
    p = cg.solve_params(precision=prec, inner_tol=inner_tol, flags=cg.COARSE_ZERO_GUESS | extra, **PARAMS)
    pt = cg.solve_params(precision=prec, inner_tol=inner_tol,
                         flags=cg.COARSE_ZERO_GUESS | cg.COARSE_TIME_APPLY | extra, **PARAMS)
    # setup: the polynomial and the first u recycle-space updates (after u updates U_k, C_k
    # stay frozen for all later solves with this operator, Sec. 4.1.1); reported separately
    t_setup = time.perf_counter()
    setup_solves = 0
    for i in range(40):
        _, inf = cop.solve(S[i % S.shape[0]], X[0], params=p)
        setup_solves += 1
        if inf[0]["recycle_updates"] >= PARAMS["recycle_updates"]:
            break
        if i >= 3 and inf[0]["recycle_updates"] == 0:
            break  # the solves converge inside their first cycle: no recycle space forms
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t_setup
    for i in range(args.warmup):
        cop.solve(B[i], X[i], params=p)
    torch.cuda.synchronize()
    barrier = (lambda: __import__("torch.distributed").distributed.barrier()) if world > 1 else (lambda: None)
    infos = []
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("timed")
        e0.record(stream)
        for i in range(args.steps):
            _, inf = cop.solve(B[args.warmup + i], X[args.warmup + i], params=p)
            infos.append(inf[0])
        e1.record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        barrier()
    ms = replicas.max_over_ranks(e0.elapsed_time(e1), dev)
    value = replicas.job_rate(args.steps, world, ms)
    # the stencil's roofline: a second timed pass over the same solves with a CUDA-event pair
    # around every stencil launch (COARSE_TIME_APPLY; these solves launch eagerly, not through
    # the step graphs, so the pass itself is a little slower)
    tinfos = []
    for i in range(min(args.steps, 20)):
        _, inf = cop.solve(B[args.warmup + i], X[args.warmup + i], params=pt)
        tinfos.append(inf[0])
    torch.cuda.synchronize()
    worst_res = max(i["rel_residual"] for i in infos)
    # end to end: pinned host b -> device, solve, device x -> pinned host, every step
    hb = B[args.warmup + args.steps:].cpu().pin_memory()
    hx = torch.empty_like(hb).pin_memory()
    db = torch.empty(N, dtype=torch.complex128, device=dev)
    dx = torch.empty_like(db)
    barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    for i in range(args.steps):
        db.copy_(hb[i], non_blocking=True)
        cop.solve(db, dx, params=p)
        hx[i].copy_(dx, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms_e2e = replicas.max_over_ranks(e0.elapsed_time(e1), dev)
    # roofline of the stencil apply (the dominant kernel): algorithmic bytes of every timed launch
    # (5 n^2 V block bytes of its precision + 2 N vector bytes) over their summed device time
    apply_ms = sum(i["apply_ms"] for i in tinfos)
    apply_cnt = sum(i["apply_count"] for i in tinfos)
    apply_bytes = sum(i["apply_bytes"] for i in tinfos)
    avg = apply_ms / max(apply_cnt, 1)
    bytes_per_apply = apply_bytes / max(apply_cnt, 1)
    achieved = apply_bytes / (apply_ms * 1e-3) / 1e9
    peak, src = peaks()
    iters = statistics.mean(i["iterations"] for i in infos)
    line = {
        "metric": "coarsest-level solves/s at rel. residual 1e-10",
        "value": round(value, 3),
        "unit": "solves/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms / args.steps, 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32" if prec == cg.PREC_FP32 else "bf16",
        "data": "synthetic",
        "config": {"workload": WORKLOAD.format(prec=args.prec.upper()), "l2": "inputs larger than L2 "
                   "(FP64 blocks 335 MB read every refinement step; FP32 blocks 168 MB)",
                   "polynomial_chain_blocks": "bf16" if poly_bf16 else args.prec,
                   "inner_system": ("odd-even reduced, block-Jacobi preconditioned S = 1 - D_ee^-1 D_eo D_oo^-1 D_oe"
                                    if args.oddeven == "on" else "full coarse operator"),
                   "parallelism": f"replicas x{world}"},
        "e2e": {"value": round(replicas.job_rate(args.steps, world, ms_e2e), 3), "unit": "solves/s",
                "h2d_bytes_per_step": N * 16, "d2h_bytes_per_step": N * 16},
        "gpu_launches": int(sum(i["kernel_launches"] for i in infos)),
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": None,
                     "kernel": (("%s<32,float2> x2 (operator S) + %s<32,cbf16> x2 (polynomial chain); "
                                 "one launch = one S apply = two half passes" % (eo_layout(cg, 1), eo_layout(cg, 2)))
                                if args.oddeven == "on" and poly_bf16 else
                                "%s<32,%s> x2 per S apply" % (eo_layout(cg, prec),
                                                               "cbf16" if prec == cg.PREC_BF16 else "float2")
                                if args.oddeven == "on" else
                                "k_apply*<32,float2> (operator) + k_apply*<32,cbf16> (polynomial chain)" if poly_bf16 else
                                f"k_apply*<32,{'cbf16' if prec == cg.PREC_BF16 else 'float2'}>"),
                     "bytes_per_launch": round(bytes_per_apply), "avg_launch_us": round(avg * 1e3, 2),
                     "launches_timed": apply_cnt, "peak_source": src,
                     "measured_over": "second timed pass of the same solves with an event pair per stencil launch"},
        "solver": {"iterations_per_solve": iters, "matvecs_per_solve": statistics.mean(i["matvecs"] for i in infos),
                   "ir_steps": statistics.mean(i["ir_steps"] for i in infos), "worst_rel_residual": worst_res,
                   "recycle_updates": infos[-1]["recycle_updates"],
                   "setup": {"solves": setup_solves, "seconds": round(t_setup, 3),
                             "what": "polynomial + recycle-space updates until u=10 is reached (or none forms)"}},
        "clocks": clk.summary(),
        "autotune": cg.autotune_report().strip().split("\n"),
    }
    if args.fp64_baseline_steps > 0:
        # plain FP64 GPU GMRES(50) on the same right-hand sides: the reference point of the speedup
        p64 = cg.solve_params(precision=cg.PREC_FP64, m=PARAMS["m"], tol=PARAMS["tol"], max_restarts=2000,
                              max_ir=5, flags=cg.COARSE_ZERO_GUESS)
        nb = args.fp64_baseline_steps
        cop.solve(B[0], X[0], params=p64)
        torch.cuda.synchronize()
        e0.record(stream)
        its64 = []
        for i in range(nb):
            _, inf = cop.solve(B[args.warmup + i], X[args.warmup + i], params=p64)
            its64.append(inf[0]["iterations"])
        e1.record(stream)
        torch.cuda.synchronize()
        v64 = nb / (e0.elapsed_time(e1) / 1e3)
        line["fp64_gmres_baseline"] = {"value": round(v64, 4), "unit": "solves/s", "steps": nb,
                                       "iterations_per_solve": statistics.mean(its64),
                                       "speedup": round(value / world / v64, 2)}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(host_blocks, iters)
    if rank == 0:
        print(json.dumps(line), flush=True)
    cop.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def oracle_workload():
    """Blocks of the bench operator on the host (built with the shared generator on the CPU)."""
    from synthetic.coarse_op import build_coarse_operator
    op = build_coarse_operator(KEY, FINE_DIMS, NV, M0, CSW, device="cpu")
    return op


def oracle_sample(s, h, dims, budget_s: float, steps: int):
    """Time the oracle's FP64 GCRO-DR (GMRES(50), degree-4 polynomial, k=16) for its first
    `steps` Arnoldi steps on one right-hand side; returns seconds per Arnoldi step."""
    from oracle import coarse as oc
    from oracle import krylov
    from synthetic import draws
    N = s.shape[0] * s.shape[1]
    A = lambda v: oc.apply(s, h, dims, v)
    v0 = draws.poly_start(KEY, N)
    theta, _ = krylov.poly_setup(A, v0, PARAMS["poly_degree"])
    M = lambda v: krylov.poly_apply(A, theta, v)
    b = draws.rhs((*KEY, 999), 1, N)[0]
    t0 = time.perf_counter()
    krylov.gmres(A, b, m=steps, tol=1e-300, max_restarts=1, precond=M)
    return (time.perf_counter() - t0) / steps


def oracle_iterations():
    try:
        with open(ORACLE_ITERS) as f:
            return json.load(f)["iterations_per_solve"], "oracle run to 1e-10 (stored)"
    except Exception:
        return None, None


def cpu_baseline(host_blocks, gpu_iters):
    s, h, dims = host_blocks
    steps = 8
    per_step = oracle_sample(s, h, dims, 0, steps)
    iters, src = oracle_iterations()
    if iters is None:
        iters, src = gpu_iters, "Arnoldi steps per solve of this run"
    return {"value": round(1.0 / (per_step * iters), 6), "unit": "solves/s", "cores": 1, "kind": "oracle",
            "sample": f"oracle FP64 pp-GMRES, {steps} Arnoldi steps (d=4: {4 * steps} applies + MGS) on one "
                      f"right-hand side; seconds per step x {iters:.0f} steps per solve ({src}); NumPy einsum, "
                      f"single thread"}


# layouts of the odd-even half apply, by the autotuner's candidate number
EO_LAYOUTS = {0: "k_eo_half[CTA of 4 warps]", 1: "k_eo_half_w[warp per site]", 2: "k_eo_half[CTA of 2 warps]",
              3: "k_eo_half[CTA of 2 warps, unrolled]", 4: "k_eo_half[CTA of 2 warps, prefetch]",
              5: "k_eo_half[CTA of 2 warps, unrolled, prefetch]", 6: "k_eo_ring[streamed]"}


def eo_layout(cg, prec):
    """Name of the half-apply layout the autotuner chose for block precision `prec` (n = 32)."""
    for line in cg.autotune_report().splitlines():
        if line.startswith(f"eo/p{prec}/n32/") and "->" in line:
            return EO_LAYOUTS.get(int(line.split("->")[1].split()[0]), "k_eo_half")
    return "k_eo_half"


def run_reference(args):
    world, rank, local = dist_init()
    if rank != 0:
        return
    op = oracle_workload()
    s, h = op.self_blocks.numpy(), op.hop_blocks.numpy()
    iters, src = oracle_iterations()
    if iters is None:
        iters, src = 200.0, "assumed 200 Arnoldi steps per solve"
    steps = 4
    for _ in range(args.warmup):
        oracle_sample(s, h, op.dims, 10, steps)
    t = []
    for _ in range(args.steps):
        t.append(oracle_sample(s, h, op.dims, 10, steps))
    per = statistics.mean(t)
    value = 1.0 / (per * iters)
    line = {"impl": "reference", "metric": "coarsest-level solves/s at rel. residual 1e-10", "value": round(value, 6),
            "unit": "solves/s", "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(per * iters * 1e3, 1), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD.format(prec="FP64 oracle")},
            "cpu_baseline": {"value": round(value, 6), "unit": "solves/s", "cores": 1, "kind": "oracle",
                             "sample": f"each step: {steps} Arnoldi steps of the FP64 oracle pp-GMRES; seconds per "
                                       f"step x {iters:.0f} steps per solve ({src})"},
            "e2e": {"value": round(value, 6), "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


APPLY_CASES = {
    # name: (fine dims, nv, m0, mu, description)
    "wilson8": ((16, 16, 16, 16), 16, -0.42, 0.0, "wilson-clover coarse 8^4, n=32"),
    "tm16": ((32, 32, 32, 32), 24, -0.42, 3e-3, "twisted mass coarse 16^4, n=48, mu=3e-3"),
    "tm12": ((24, 24, 24, 24), 24, -0.42, 3e-3, "twisted mass coarse 12^4, n=48, mu=3e-3 (profiling size)"),
}


def run_apply_only(args):
    """Stencil apply alone: achieved algorithmic GB/s with an L2 flush (256 MB write) between launches."""
    import torch

    import paper_2205_09104_gb300 as cg
    from synthetic.coarse_op import build_coarse_operator
    fine, nv, m0, mu, desc = APPLY_CASES[args.apply_only]
    prec = {"fp64": cg.PREC_FP64, "fp32": cg.PREC_FP32, "bf16": cg.PREC_BF16}[args.prec]
    dev = torch.device("cuda", 0)
    op = build_coarse_operator((3, 0), fine, nv, m0, CSW, device=dev)
    cop = cg.CoarseOp(op.self_blocks, op.hop_blocks, op.dims, op.nv, mu=mu,
                      precisions=(prec,) if prec else ())
    del op
    torch.cuda.empty_cache()
    n, V = 2 * nv, cop.V
    N = n * V
    dt = torch.complex128 if prec == cg.PREC_FP64 else torch.complex64
    g = torch.Generator(device="cpu").manual_seed(5)
    x = torch.randn(N, dtype=dt, generator=g).to(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        cop.apply(x, precision=prec)
    torch.cuda.synchronize()
    ts = []
    for _ in range(args.steps):
        if not args.no_flush:
            flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        y = cop.apply(x, precision=prec)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    esize = {cg.PREC_FP64: 16, cg.PREC_FP32: 8, cg.PREC_BF16: 4}[prec]
    vsize = 16 if prec == cg.PREC_FP64 else 8
    nbytes = 5 * n * n * V * esize + 2 * N * vsize
    flops = 9 * n * n * 8 * V
    med = statistics.median(ts)
    peak, src = peaks()
    print(json.dumps({"mode": "apply", "case": args.apply_only, "workload": desc, "precision": args.prec,
                      "l2_flush": not args.no_flush, "median_us": round(med * 1e3, 2), "min_us": round(min(ts) * 1e3, 2),
                      "bytes_per_launch": nbytes, "achieved_gbs": round(nbytes / (med * 1e-3) / 1e9, 1),
                      "peak_gbs": peak, "frac": round(nbytes / (med * 1e-3) / 1e9 / peak, 4), "peak_source": src,
                      "gflops": round(flops / (med * 1e-3) / 1e9, 1), "launches": len(ts),
                      "autotune": cg.autotune_report().strip().split("\n")}), flush=True)
    cop.close()


def run_schur_only(args):
    """Odd-even reduced operator S = 1 - D_ee^-1 D_eo D_oo^-1 D_oe alone (two half passes): achieved
    algorithmic GB/s with an L2 flush (256 MB write) between launches."""
    import torch

    import paper_2205_09104_gb300 as cg
    from synthetic.coarse_op import build_coarse_operator
    fine, nv, m0, mu, desc = APPLY_CASES[args.schur_only]
    prec = {"fp64": cg.PREC_FP64, "fp32": cg.PREC_FP32, "bf16": cg.PREC_BF16}[args.prec]
    dev = torch.device("cuda", 0)
    op = build_coarse_operator((3, 0), fine, nv, m0, CSW, device=dev)
    cop = cg.CoarseOp(op.self_blocks, op.hop_blocks, op.dims, op.nv, mu=mu, precisions=(prec,) if prec else ())
    del op
    torch.cuda.empty_cache()
    n, V = 2 * nv, cop.V
    N = n * V
    dt = torch.complex128 if prec == cg.PREC_FP64 else torch.complex64
    g = torch.Generator(device="cpu").manual_seed(5)
    x = torch.randn(N // 2, dtype=dt, generator=g).to(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        cop.schur(x, precision=prec)
    torch.cuda.synchronize()
    ts = []
    for _ in range(args.steps):
        if not args.no_flush:
            flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        cop.schur(x, precision=prec)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    esize = {cg.PREC_FP64: 16, cg.PREC_FP32: 8, cg.PREC_BF16: 4}[prec]
    vsize = 16 if prec == cg.PREC_FP64 else 8
    nbytes = 9 * n * n * V * esize + 2.5 * N * vsize
    med = statistics.median(ts)
    peak, src = peaks()
    print(json.dumps({"mode": "schur", "case": args.schur_only, "workload": desc, "precision": args.prec,
                      "l2_flush": not args.no_flush, "median_us": round(med * 1e3, 2), "min_us": round(min(ts) * 1e3, 2),
                      "bytes_per_launch": int(nbytes), "achieved_gbs": round(nbytes / (med * 1e-3) / 1e9, 1),
                      "peak_gbs": peak, "frac": round(nbytes / (med * 1e-3) / 1e9 / peak, 4), "peak_source": src,
                      "launches": len(ts), "autotune": cg.autotune_report().splitlines()}), flush=True)
    cop.close()


def run_mrhs(args):
    """Multi-right-hand-side BF16 apply on tensor cores vs one single-column BF16 apply per column:
    coarse 4^4 / 6^4 / 8^4 (V = 256, 1296, 4096), n = 16 / 32 / 48, 1-12 columns; L2 flushed
    (256 MB write) before every timed launch."""
    import torch

    import paper_2205_09104_gb300 as cg
    from synthetic.coarse_op import build_coarse_operator
    dev = torch.device("cuda", 0)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    peak, src = peaks()
    g = torch.Generator(device="cpu").manual_seed(6)

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        ts = []
        for _ in range(args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    cases = [(L, nv, (1, 2, 4, 8, 12)) for L in (4, 6, 8) for nv in (8, 16, 24)]
    if args.mrhs_case:
        L, nv, nr = (int(v) for v in args.mrhs_case.split(","))
        cases = [(L, nv, (nr,))]
    for L, nv, counts in cases:
        op = build_coarse_operator((6, L, nv), (2 * L,) * 4, nv, -0.42, CSW, device=dev)
        cop = cg.CoarseOp(op.self_blocks, op.hop_blocks, op.dims, op.nv, precisions=(cg.PREC_BF16,),
                          max_nrhs=12)
        del op
        torch.cuda.empty_cache()
        n, V = 2 * nv, cop.V
        N = n * V
        for nrhs in counts:
            X = torch.randn(nrhs, N, dtype=torch.complex64, generator=g).to(dev)
            Y = torch.empty_like(X)
            t_m = timed(lambda: cop.apply(X, precision=cg.PREC_BF16, out=Y))
            t_c = timed(lambda: [cop.apply(X[c], precision=cg.PREC_BF16, out=Y[c]) for c in range(nrhs)])
            nbytes = 5 * n * n * 4 * V + 2 * nrhs * N * 8
            flops = 9 * n * n * 8 * V * nrhs
            print(json.dumps({"mode": "mrhs", "coarse": f"{L}^4", "V": V, "n": n, "nrhs": nrhs,
                              "us_mrhs": round(t_m * 1e3, 2), "us_per_column_path": round(t_c * 1e3, 2),
                              "speedup": round(t_c / t_m, 2),
                              "achieved_gbs": round(nbytes / (t_m * 1e-3) / 1e9, 1),
                              "frac": round(nbytes / (t_m * 1e-3) / 1e9 / peak, 4), "peak_source": src,
                              "tflops": round(flops / (t_m * 1e-3) / 1e12, 2)}), flush=True)
        cop.close()
    print(json.dumps({"mode": "mrhs-autotune", "decisions": cg.autotune_report().strip().split("\n")}), flush=True)


def run_batched(args):
    """Uneven batch of coarse solves (coarse 4^4 / 6^4 / 8^4, nv 8 / 16 / 24, 1-12 right-hand sides
    each, m0 in [-0.44, -0.38]): the lockstep engine vs the single-operator path on the same inputs."""
    import torch

    import paper_2205_09104_gb300 as cg
    from synthetic import draws
    from synthetic.coarse_op import build_coarse_operator
    dev = torch.device("cuda", 0)
    prec = cg.PREC_BF16 if args.prec == "bf16" else cg.PREC_FP32
    recipe = draws.batch_recipe((4, 0), args.batched)
    t = time.perf_counter()
    ops, bs, xs = [], [], []
    for i, (L, nv, m0, nr) in enumerate(recipe):
        op = build_coarse_operator((4, 1 + i), (2 * L,) * 4, nv, m0, CSW, device=dev)
        ops.append(cg.CoarseOp(op.self_blocks, op.hop_blocks, op.dims, op.nv, precisions=(prec, cg.PREC_BF16),
                               max_nrhs=12))
        N = op.volume * op.n
        bs.append(torch.from_numpy(draws.rhs((4, 1 + i, 7), nr, N)).to(dev))
        xs.append(torch.zeros_like(bs[-1]))
        del op
    t_gen = time.perf_counter() - t
    inner_tol = 1e-5 if prec == cg.PREC_FP32 else 1e-2
    chain = cg.COARSE_POLY_BF16 if (prec == cg.PREC_FP32 and args.poly == "bf16") else 0
    p = cg.solve_params(precision=prec, inner_tol=inner_tol, flags=cg.COARSE_ZERO_GUESS | chain, **PARAMS)
    t = time.perf_counter()
    cg.solve_batched(ops, bs, xs, p)          # setup (polynomials, recycle spaces) + first batch
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t
    for _ in range(args.warmup):
        cg.solve_batched(ops, bs, xs, p)
    torch.cuda.synchronize()
    nrhs = sum(b.shape[0] for b in bs)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        e0.record()
        infos = []
        for _ in range(args.steps):
            infos = cg.solve_batched(ops, bs, xs, p)
        e1.record()
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    worst = max(i["rel_residual"] for i in infos)
    # the same columns through the single-operator path, one operator after another
    e0.record()
    for o, b, x in zip(ops, bs, xs):
        o.solve(b, x, params=p)
    e1.record()
    torch.cuda.synchronize()
    ms_seq = e0.elapsed_time(e1)
    print(json.dumps({"mode": "batched", "operators": len(ops), "right_hand_sides": nrhs,
                      "precision": args.prec, "polynomial_chain_blocks": "bf16" if chain else args.prec,
                      "ms_per_batch": round(ms, 2),
                      "rhs_solves_per_s": round(nrhs / (ms / 1e3), 1), "operator_batches_per_s": round(1e3 / ms, 3),
                      "sequential_ms": round(ms_seq, 2), "speedup_vs_sequential": round(ms_seq / ms, 2),
                      "worst_rel_residual": worst, "kernel_launches_per_batch": infos[0]["kernel_launches"],
                      "generate_s": round(t_gen, 1), "setup_s": round(t_setup, 2), "clocks": clk.summary()}),
          flush=True)
    for o in ops:
        o.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--prec", default="fp32", choices=["fp32", "bf16", "fp64"])
    ap.add_argument("--inner-tol", type=float, default=0.0,
                    help="relative tolerance of the inner solves (0: 2e-6 for FP32, 1e-2 for BF16)")
    ap.add_argument("--oddeven", default="on", choices=["on", "off"],
                    help="inner solves on the odd-even reduced system (COARSE_ODD_EVEN)")
    ap.add_argument("--poly", default="bf16", choices=["bf16", "same"],
                    help="blocks of the polynomial-chain applies for FP32 inner solves (COARSE_POLY_BF16)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--apply-only", choices=sorted(APPLY_CASES), default=None,
                    help="time the stencil apply alone on one of the named lattices")
    ap.add_argument("--schur-only", choices=sorted(APPLY_CASES), default=None,
                    help="time the odd-even reduced operator alone on one of the named lattices")
    ap.add_argument("--no-flush", action="store_true")
    ap.add_argument("--fp64-baseline-steps", type=int, default=2,
                    help="plain FP64 GMRES(50) solves timed for the speedup (0 = skip)")
    ap.add_argument("--mrhs", action="store_true",
                    help="time the multi-right-hand-side tensor-core apply against the per-column path")
    ap.add_argument("--mrhs-case", default="",
                    help="one multi-right-hand-side case 'L,nv,nrhs' (coarse L^4, n = 2 nv)")
    ap.add_argument("--batched", type=int, default=0,
                    help="time the lockstep batched engine on this many uneven operators")
    args = ap.parse_args()
    if args.batched:
        run_batched(args)
        return
    if args.mrhs:
        run_mrhs(args)
        return
    if args.schur_only:
        run_schur_only(args)
        return
    if args.apply_only:
        run_apply_only(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gb300(args)


if __name__ == "__main__":
    main()
