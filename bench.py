#!/usr/bin/env python
"""Benchmark: coarsest-level solves/s at relative residual 1e-10, and the D_c apply's achieved
HBM bandwidth against the measured peak.

Default workload: twisted mass, coarse 16^4 lattice (fine 32^4, 2^4 aggregates), nv = 24 ->
n = 48 dof per site, 3,145,728 unknowns, m0 = -0.42, c_sw = 1, mu = 3e-3.  One step = one
right-hand side solved to a true FP64 relative residual of 1e-10 with GMRES(50) + the
Leja-ordered degree-8 GMRES polynomial (Sec. 3.3) + GCRO-DR with k = 32 recycled harmonic Ritz
vectors (Sec. 3.4, u = 10 updates), FP32 inner solves on the odd-even reduced, block-Jacobi
preconditioned system (Sec. 2, Sec. 3.2; polynomial chain on BF16 blocks) inside FP64
iterative refinement.  The polynomial and the recycle space are built during setup solves and
reused, as for repeated coarsest-level solves with one operator.

--workload wilson8 runs the Wilson-clover coarse 8^4 workload (n = 32, d = 4, k = 16) instead;
--sweep prints one line per point of the mu sweep (1e-3, 3e-3, 1e-2) of the twisted-mass
workload and of the m0 sweep (-0.40, -0.42, -0.44) of the Wilson-clover one, each with and
without deflation (iterations, solves/s, recycle updates).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
       [--workload tm16|wilson8] [--sweep] [--apply-only CASE] [--schur-only CASE] [--mrhs]
       [--batched K]
"""
from __future__ import annotations

import argparse
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

CSW = 1.0
WORKLOADS = {
    "tm16": dict(key=(3, 0), fine=(32, 32, 32, 32), nv=24, m0=-0.42, mu=3e-3, d=8, k=32,
                 desc="twisted mass coarse 16^4 (fine 32^4, 2^4 aggregates), nv=24 -> n=48, 3145728 unknowns, "
                      "m0={m0}, c_sw=1.0, mu={mu:g}; GMRES(50) + Leja poly d=8 + GCRO-DR k={k} u=10; {prec} inner "
                      "+ FP64 refinement to 1e-10"),
    "wilson8": dict(key=(2, 0), fine=(16, 16, 16, 16), nv=16, m0=-0.42, mu=0.0, d=4, k=16,
                    desc="wilson-clover coarse 8^4 (fine 16^4, 2^4 aggregates), nv=16 -> n=32, 131072 unknowns, "
                         "m0={m0}, c_sw=1.0; GMRES(50) + Leja poly d=4 + GCRO-DR k={k} u=10; {prec} inner + FP64 "
                         "refinement to 1e-10"),
}
SOLVER = dict(m=50, recycle_updates=10, tol=1e-10, max_restarts=100, max_ir=20)
METRIC = "coarsest-level solves/s at rel. residual 1e-10"
PROFILES = os.path.join(ROOT, "profiles")


def oracle_iterations_path(name):
    return os.path.join(ROOT, "oracle", f"bench_iterations_{name}.json")


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def profiled_traffic(workload):
    """DRAM bytes per S apply by half-apply layout and block precision, from the ncu summary of
    the odd-even half apply on this workload (profiles/k_eo_half_<workload>.md, lines
    'traffic_per_S_apply layout=<v>: fp32=<B> bf16=<B>'): {(layout, "fp32"|"bf16"): bytes}, or {}
    when no summary is committed."""
    path = os.path.join(PROFILES, f"k_eo_half_{workload}.md")
    out = {}
    try:
        with open(path) as f:
            for line in f:
                m = re.match(r"\s*traffic_per_S_apply\s+layout=(\d+):\s*(.*)", line)
                if m:
                    for kv in m.group(2).split():
                        k, v = kv.split("=")
                        out[(int(m.group(1)), k)] = float(v)
    except OSError:
        pass
    return out, (os.path.relpath(path, ROOT) if out else None)


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


def build_operator(wl, device):
    """Seeded synthetic Galerkin blocks of the workload (on `device`) and the seconds it took."""
    import torch

    from synthetic.coarse_op import build_coarse_operator
    t = time.perf_counter()
    op = build_coarse_operator(wl["key"], wl["fine"], wl["nv"], wl["m0"], CSW, device=device)
    if str(device).startswith("cuda"):
        torch.cuda.synchronize()
    return op, time.perf_counter() - t


PIPELINED = {"on": False}


def solver_params(cg, wl, k, extra=0, time_apply=False):
    flags = cg.COARSE_ZERO_GUESS | cg.COARSE_POLY_BF16 | cg.COARSE_ODD_EVEN | extra
    if PIPELINED["on"]:
        flags |= cg.COARSE_PIPELINED
    if time_apply:
        flags |= cg.COARSE_TIME_APPLY
    # FP32 inner solves to 2e-6: two refinement steps reach 1e-10 ((2e-6)^2 with margin)
    return cg.solve_params(precision=cg.PREC_FP32, inner_tol=2e-6, poly_degree=wl["d"], defl_k=k, flags=flags,
                           **SOLVER)


def setup_solves(cg, cop, wl, k, S, X):
    """Polynomial, autotuner decisions and recycle space (Sec. 3.4: the first from a full GMRES(m)
    cycle, then updates until u are made, after which U_k, C_k stay frozen); returns
    (solves, seconds, recycle updates)."""
    import torch
    t = time.perf_counter()
    n, rec = 0, 0
    if k > 0:
        _, inf = cop.solve(S[0], X, params=solver_params(cg, wl, k, cg.COARSE_RECYCLE_FULL_CYCLE))
        n, rec = 1, inf[0]["recycle_updates"]
    while n < 12:
        _, inf = cop.solve(S[n % S.shape[0]], X, params=solver_params(cg, wl, k))
        n += 1
        rec = inf[0]["recycle_updates"]
        if k == 0 or rec >= SOLVER["recycle_updates"]:
            break
    torch.cuda.synchronize()
    return n, time.perf_counter() - t, rec


# layouts of the odd-even half apply, by the autotuner's candidate number
EO_LAYOUTS = {0: "k_eo_half[CTA of 4 warps]", 1: "k_eo_half_w[warp per site]", 2: "k_eo_half[CTA of 2 warps]",
              3: "k_eo_half[CTA of 2 warps, unrolled]", 4: "k_eo_half[CTA of 2 warps, prefetch]",
              5: "k_eo_half[CTA of 2 warps, unrolled, prefetch]", 6: "k_eo_ring[streamed]"}


def eo_choice(cg, prec, n):
    """Half-apply layout number the autotuner chose for block precision `prec`, or None."""
    for line in cg.autotune_report().splitlines():
        if line.startswith(f"eo/p{prec}/n{n}/") and "->" in line:
            return int(line.split("->")[1].split()[0])
    return None


def eo_layout(cg, prec, n):
    """Name of the half-apply layout the autotuner chose for block precision `prec`."""
    return EO_LAYOUTS.get(eo_choice(cg, prec, n), "k_eo_half")


def roofline_entries(cg, tinfos, n, peak, src, workload):
    """Per block precision of the S applies timed with events: algorithmic bytes per S apply
    (9 n^2 V block entries + 2.5 V n vector entries) over the average event time of one S apply."""
    traffic, tsrc = profiled_traffic(workload)
    out = []
    for q, name, role in ((cg.PREC_FP32, "fp32", "operator S"), (cg.PREC_BF16, "bf16", "polynomial chain S")):
        ms = sum(i["apply_ms_prec"][q] for i in tinfos)
        by = sum(i["apply_bytes_prec"][q] for i in tinfos)
        cnt = sum(i["apply_count_prec"][q] for i in tinfos)
        if cnt == 0:
            continue
        achieved = by / (ms * 1e-3) / 1e9
        bt = "float2" if q == cg.PREC_FP32 else "cbf16"
        out.append({"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                    "frac": round(achieved / peak, 4), "traffic": traffic.get((eo_choice(cg, q, n), name)),
                    "traffic_source": tsrc if (eo_choice(cg, q, n), name) in traffic else None,
                    "kernel": f"{eo_layout(cg, q, n)}<{n},{bt}> x2 ({role}); one launch = one S apply = two "
                              "half passes",
                    "bytes_per_launch": round(by / cnt), "avg_launch_us": round(ms / cnt * 1e3, 2),
                    "launches_timed": cnt, "time_share_ms": round(ms, 3), "peak_source": src,
                    "measured_over": "second pass of the timed solves with a CUDA-event pair around every S apply"})
    out.sort(key=lambda e: -e["time_share_ms"])
    return out


def host_memory_available():
    try:
        return os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
    except (ValueError, OSError):
        return 0


def oracle_iters(name):
    try:
        with open(oracle_iterations_path(name)) as f:
            d = json.load(f)
        return d["iterations_per_solve"], "oracle run to 1e-10 (stored)"
    except Exception:
        return None, None


def oracle_apply_seconds(host, budget_s, max_samples=8, warm=1):
    """Median seconds of the FP64 oracle's D_c apply (NumPy, einsum over sites) on the workload."""
    from oracle import coarse as oc
    s, h, dims, mu, v = host
    for _ in range(warm):
        oc.apply(s, h, dims, v, mu)
    ts = []
    t_end = time.perf_counter() + budget_s
    while len(ts) < max_samples:
        t0 = time.perf_counter()
        oc.apply(s, h, dims, v, mu)
        ts.append(time.perf_counter() - t0)
        if time.perf_counter() > t_end:
            break
    return statistics.median(ts), len(ts)


def oracle_apply_throughput(host, threads, per_thread=2):
    """Applications per second of the FP64 oracle's D_c when `threads` independent applications run
    at once on the host cores (the oracle as it stands, one application per thread; NumPy's einsum
    releases the interpreter lock), i.e. the throughput of as many independent oracle solves."""
    import concurrent.futures as cf

    from oracle import coarse as oc
    s, h, dims, mu, v = host

    def work(_):
        for _ in range(per_thread):
            oc.apply(s, h, dims, v, mu)
    with cf.ThreadPoolExecutor(threads) as ex:
        list(ex.map(work, range(threads)))      # warm-up round
        t0 = time.perf_counter()
        list(ex.map(work, range(threads)))
        dt = time.perf_counter() - t0
    return threads * per_thread / dt


def threads_used():
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS"):
        if os.environ.get(var):
            return int(os.environ[var])
    return 1   # numpy einsum runs on one thread


def cpu_baseline(wl, name, host, gpu_iters, budget_s):
    t_apply, cnt = oracle_apply_seconds(host, budget_s)
    iters, src = oracle_iters(name)
    if iters is None:
        iters, src = gpu_iters, "Arnoldi steps per solve of this run's GPU solver"
    per_solve = t_apply * wl["d"] * iters
    out = {"value": round(1.0 / per_solve, 6), "unit": "solves/s", "cores": threads_used(), "kind": "oracle",
           "sample": f"{cnt} applications of the FP64 oracle's D_c (NumPy) on this workload, median "
                     f"{t_apply:.3f} s; x {wl['d']} applies per preconditioned Arnoldi step x {iters:.1f} steps "
                     f"per solve ({src}); the oracle's Gram-Schmidt and small dense work are not counted, so "
                     f"this overstates its solves/s"}
    ncores = os.cpu_count() or 1
    # each thread holds a few vector-sized temporaries (about 3 N complex128)
    per_thread_bytes = 3 * host[4].size * 16
    threads = max(1, min(ncores, int(host_memory_available() * 0.5 // max(per_thread_bytes, 1))))
    if threads > 1:
        rate = oracle_apply_throughput(host, threads)
        out["all_cores"] = {"value": round(rate / (wl["d"] * iters), 6), "unit": "solves/s", "cores": threads,
                            "kind": "oracle",
                            "sample": f"{threads} independent oracle applications at once, 2 per thread after a "
                                      f"warm-up round: {rate:.2f} applications/s, projected per solve as above "
                                      "(throughput of that many independent single-threaded oracle solves)"}
    return out


def run_gb300(args):
    import torch

    import paper_2205_09104_gb300 as cg
    from paper_2205_09104_gb300 import replicas
    from synthetic import draws

    world, rank, local = dist_init()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    name = args.workload
    wl = dict(WORKLOADS[name])
    k = wl["k"]
    # replicas: each rank solves its own right-hand sides with its own copy of the operator
    op, gen_s = build_operator(wl, dev)
    n, V = op.n, op.volume
    N = V * n
    host = None
    want_cpu = rank == 0 and world == 1 and not args.no_cpu_baseline
    block_bytes = (op.self_blocks.numel() + op.hop_blocks.numel()) * 16
    if want_cpu and host_memory_available() > 3 * block_bytes:
        host = (op.self_blocks.cpu().numpy(), op.hop_blocks.cpu().numpy(), op.dims, wl["mu"],
                draws.rhs((*wl["key"], 999), 1, N)[0])
    cop = cg.CoarseOp(op.self_blocks, op.hop_blocks, op.dims, op.nv, mu=wl["mu"],
                      precisions=(cg.PREC_FP32, cg.PREC_BF16))
    del op
    torch.cuda.empty_cache()
    total = args.warmup + 2 * args.steps
    B = torch.from_numpy(draws.rhs(replicas.rhs_key(wl["key"], rank), total, N)).to(dev)
    S = torch.from_numpy(draws.rhs((*wl["key"], 50 + rank), 4, N)).to(dev)  # setup right-hand sides
    X = torch.zeros_like(B)
    p = solver_params(cg, wl, k)
    setup_n, setup_s, rec = setup_solves(cg, cop, wl, k, S, X[0])
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
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        barrier()
    ms = replicas.max_over_ranks(e0.elapsed_time(e1), dev)
    value = replicas.job_rate(args.steps, world, ms)
    # the stencil's roofline: a second pass over the same solves with a CUDA-event pair around
    # every S apply (COARSE_TIME_APPLY; these solves launch eagerly, not through the step graphs)
    pt = solver_params(cg, wl, k, time_apply=True)
    tinfos = []
    for i in range(min(args.steps, 10)):
        _, inf = cop.solve(B[args.warmup + i], X[args.warmup + i], params=pt)
        tinfos.append(inf[0])
    torch.cuda.synchronize()
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
    peak, src = peaks()
    roofs = roofline_entries(cg, tinfos, n, peak, src, name)
    iters = statistics.mean(i["iterations"] for i in infos)
    props = torch.cuda.get_device_properties(dev)
    l2_mb = getattr(props, "L2_cache_size", 0) / 2 ** 20
    esz = {"fp32": 8, "bf16": 4}
    s_bytes = {q: 9 * n * n * V * e for q, e in esz.items()}
    line = {
        "metric": METRIC,
        "value": round(value, 3),
        "unit": "solves/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms / args.steps, 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": wl["desc"].format(m0=wl["m0"], mu=wl["mu"], k=k, prec="FP32"),
                   "l2": f"inputs larger than L2 ({l2_mb:.0f} MB, cudaDeviceProp): every S apply reads "
                         f"{s_bytes['fp32'] / 1e9:.2f} GB of FP32 or {s_bytes['bf16'] / 1e9:.2f} GB of BF16 block "
                         "entries, every refinement step the FP64 blocks",
                   "polynomial_chain_blocks": "bf16",
                   "inner_system": "odd-even reduced, block-Jacobi preconditioned S = 1 - D_ee^-1 D_eo D_oo^-1 D_oe",
                   "arnoldi": "latency-1 pipelined (Sec. 3.5)" if PIPELINED["on"] else "classical, CGS2",
                   "parallelism": f"replicas x{world}"},
        "e2e": {"value": round(replicas.job_rate(args.steps, world, ms_e2e), 3), "unit": "solves/s",
                "h2d_bytes_per_step": N * 16, "d2h_bytes_per_step": N * 16},
        "gpu_launches": int(sum(i["kernel_launches"] for i in infos)),
        "roofline": roofs[0] if roofs else None,
        "roofline_kernels": roofs,
        "solver": {"iterations_per_solve": iters, "breakdowns": sum(i["breakdowns"] for i in infos),
                   "matvecs_per_solve": statistics.mean(i["matvecs"] for i in infos),
                   "ir_steps": statistics.mean(i["ir_steps"] for i in infos),
                   "worst_rel_residual": max(i["rel_residual"] for i in infos),
                   "recycle_updates": infos[-1]["recycle_updates"], "recycle_k": k,
                   "setup": {"solves": setup_n, "seconds": round(setup_s, 3), "recycle_updates": rec,
                             "what": "polynomial, autotuner decisions, first recycle space from a full GMRES(50) "
                                     "cycle, then updates until u=10"},
                   "generate_s": round(gen_s, 1)},
        "clocks": clk.summary(),
        "autotune": cg.autotune_report().strip().split("\n"),
    }
    # the FP64 stencil of the refinement residual: bound by the FP64 FMA rate, measured here
    fp64_peak = cg.measure_fp64_fma()
    y64 = torch.empty(N, dtype=torch.complex128, device=dev)
    r_ms = []
    for i in range(6):
        e0.record(stream)
        cop.apply(B[i % B.shape[0]], precision=cg.PREC_FP64, out=y64)
        e1.record(stream)
        torch.cuda.synchronize()
        r_ms.append(e0.elapsed_time(e1))
    t64 = statistics.median(r_ms[1:])
    tf64 = 72.0 * n * n * V / (t64 * 1e-3) / 1e12
    line["roofline_fp64_residual"] = {"bound": "alu", "achieved": round(tf64, 3), "peak": round(fp64_peak, 3),
                                      "unit": "TFLOP/s", "frac": round(tf64 / fp64_peak, 4),
                                      "kernel": f"k_apply<{n},double2> (r = b - D_c x, one per refinement step)",
                                      "flops_per_launch": 72 * n * n * V, "avg_launch_us": round(t64 * 1e3, 1),
                                      "peak_source": "coarse_measure_fp64_fma: FP64 FMA-loop kernel on this GPU"}
    chk = cop.recycle_check(cg.PREC_FP32, odd_even=True)
    line["solver"]["recycle_space"] = {"k": chk["k"], "max_rel_AU_minus_C": chk["au_minus_c"],
                                       "max_CHC_minus_I": chk["chc_minus_i"]}
    if args.fp64_baseline_steps > 0:
        line["fp64_gmres_baseline"] = fp64_baseline(cg, cop, B, X, args, value / world, stream)
    if host is not None:
        line["cpu_baseline"] = cpu_baseline(wl, name, host, iters, args.cpu_budget)
    elif want_cpu:
        line["cpu_baseline"] = {"value": None, "unit": "solves/s", "cores": 0, "kind": "oracle",
                                "sample": "not run: the host has too little free memory for the FP64 blocks"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    cop.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def fp64_baseline(cg, cop, B, X, args, value_per_gpu, stream):
    """Plain FP64 GPU GMRES(50) on the same right-hand sides and the same 1e-10: the reference point
    of the speedup (no polynomial, no deflation, no odd-even reduction, no mixed precision)."""
    import torch
    p64 = cg.solve_params(precision=cg.PREC_FP64, m=SOLVER["m"], tol=SOLVER["tol"], max_restarts=4000, max_ir=5,
                          flags=cg.COARSE_ZERO_GUESS)
    nb = args.fp64_baseline_steps
    cop.solve(B[0], X[0], params=p64)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    its, worst = [], 0.0
    with ClockSampler(torch.cuda.current_device()) as clk:
        e0.record(stream)
        for i in range(nb):
            _, inf = cop.solve(B[args.warmup + i], X[args.warmup + i], params=p64)
            its.append(inf[0]["iterations"])
            worst = max(worst, inf[0]["rel_residual"])
        e1.record(stream)
        torch.cuda.synchronize()
    v64 = nb / (e0.elapsed_time(e1) / 1e3)
    return {"value": round(v64, 4), "unit": "solves/s", "steps": nb, "iterations_per_solve": statistics.mean(its),
            "worst_rel_residual": worst, "speedup": round(value_per_gpu / v64, 2), "clocks": clk.summary()}


SWEEP = {"tm16": ("mu", (1e-3, 3e-3, 1e-2)), "wilson8": ("m0", (-0.40, -0.42, -0.44))}


def run_sweep(args):
    """One JSON line per point: the twisted-mass workload over mu and the Wilson-clover workload
    over m0 (toward ill-conditioning), each with deflation (k of the workload) and without (k = 0):
    Arnoldi steps, refinement steps, recycle updates and solves/s (Sec. 4.1.3's comparison of
    deflation across masses, on the synthetic operators), plus plain FP64 GMRES(50) iterations."""
    import torch

    import paper_2205_09104_gb300 as cg
    from synthetic import draws
    dev = torch.device("cuda", 0)
    names = [args.workload] if args.sweep_workload == "one" else ["tm16", "wilson8"]
    for name in names:
        base = dict(WORKLOADS[name])
        par, values = SWEEP[name]
        op = None
        for val in values:
            wl = dict(base, **{par: val})
            if op is None or par == "m0":
                op = None
                torch.cuda.empty_cache()
                op, gen_s = build_operator(wl, dev)
            N = op.volume * op.n
            B = torch.from_numpy(draws.rhs((*wl["key"], 70), args.warmup + args.steps, N)).to(dev)
            S = torch.from_numpy(draws.rhs((*wl["key"], 71), 4, N)).to(dev)
            X = torch.zeros_like(B)
            its64 = None
            for k in (wl["k"], 0):
                cop = cg.CoarseOp(op.self_blocks, op.hop_blocks, op.dims, op.nv, mu=wl["mu"],
                                  precisions=(cg.PREC_FP32, cg.PREC_BF16))
                setup_n, setup_s, rec = setup_solves(cg, cop, wl, k, S, X[0])
                p = solver_params(cg, wl, k)
                for i in range(args.warmup):
                    cop.solve(B[i], X[i], params=p)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                infos = []
                e0.record()
                for i in range(args.steps):
                    _, inf = cop.solve(B[args.warmup + i], X[args.warmup + i], params=p)
                    infos.append(inf[0])
                e1.record()
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1)
                if its64 is None and args.fp64_baseline_steps > 0:
                    p64 = cg.solve_params(precision=cg.PREC_FP64, m=SOLVER["m"], tol=SOLVER["tol"],
                                          max_restarts=4000, max_ir=5, flags=cg.COARSE_ZERO_GUESS)
                    t = time.perf_counter()
                    _, inf = cop.solve(B[0], X[0], params=p64)
                    its64 = {"iterations": inf[0]["iterations"], "seconds": round(time.perf_counter() - t, 3)}
                print(json.dumps({"mode": "sweep", "workload": name, par: val, "k": k,
                                  "config": wl["desc"].format(m0=wl["m0"], mu=wl["mu"], k=k, prec="FP32"),
                                  "solves_per_s": round(args.steps / (ms / 1e3), 3),
                                  "ms_per_solve": round(ms / args.steps, 3),
                                  "iterations_per_solve": statistics.mean(i["iterations"] for i in infos),
                                  "ir_steps": statistics.mean(i["ir_steps"] for i in infos),
                                  "matvecs_per_solve": statistics.mean(i["matvecs"] for i in infos),
                                  "worst_rel_residual": max(i["rel_residual"] for i in infos),
                                  "recycle_updates": infos[-1]["recycle_updates"],
                                  "setup": {"solves": setup_n, "seconds": round(setup_s, 2)},
                                  "fp64_gmres_one_solve": its64}), flush=True)
                cop.close()
            del B, S, X
        op = None
        torch.cuda.empty_cache()


def run_reference(args):
    """The oracle as it stands on the host cores, on this workload: each step times one application
    of the FP64 oracle's D_c (the dominant cost of its solver) and the solve time is projected as
    applies per solve x that time; rank 0 only."""
    world, rank, local = dist_init()
    if rank != 0:
        return
    import torch
    from synthetic import draws
    name = args.workload
    wl = WORKLOADS[name]
    device = torch.device("cuda", local) if torch.cuda.is_available() else "cpu"
    op, gen_s = build_operator(wl, device)
    N = op.volume * op.n
    host = (op.self_blocks.cpu().numpy(), op.hop_blocks.cpu().numpy(), op.dims, wl["mu"],
            draws.rhs((*wl["key"], 999), 1, N)[0])
    del op
    if str(device).startswith("cuda"):
        torch.cuda.empty_cache()
    iters, src = oracle_iters(name)
    if iters is None:
        iters, src = 50.0, "assumed 50 Arnoldi steps per solve"
    from oracle import coarse as oc
    s, h, dims, mu, v = host
    for _ in range(args.warmup):
        oc.apply(s, h, dims, v, mu)
    t = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oc.apply(s, h, dims, v, mu)
        t.append(time.perf_counter() - t0)
    per_apply = statistics.median(t)
    per_solve = per_apply * wl["d"] * iters
    value = 1.0 / per_solve
    sample = (f"each step: one application of the FP64 oracle's D_c (NumPy) on this workload (median "
              f"{per_apply:.3f} s); a solve is projected as {wl['d']} applies per preconditioned Arnoldi step x "
              f"{iters:.1f} steps per solve ({src}), Gram-Schmidt and small dense work not counted")
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": "solves/s", "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(per_solve * 1e3, 1),
            "measured_ms_per_sample": round(per_apply * 1e3, 1), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl["desc"].format(m0=wl["m0"], mu=wl["mu"], k=wl["k"], prec="FP64 oracle")},
            "cpu_baseline": {"value": round(value, 6), "unit": "solves/s", "cores": threads_used(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 6), "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


APPLY_CASES = {
    # name: (fine dims, nv, m0, mu, description)
    "wilson8": ((16, 16, 16, 16), 16, -0.42, 0.0, "wilson-clover coarse 8^4, n=32"),
    "tm16": ((32, 32, 32, 32), 24, -0.42, 3e-3, "twisted mass coarse 16^4, n=48, mu=3e-3"),
    "tm12": ((24, 24, 24, 24), 24, -0.42, 3e-3, "twisted mass coarse 12^4, n=48, mu=3e-3 (profiling size)"),
    "tm8": ((16, 16, 16, 16), 24, -0.42, 3e-3, "twisted mass coarse 8^4, n=48, mu=3e-3 (profiling size)"),
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
    coarse 4^4 / 6^4 / 8^4 (V = 256, 1296, 4096), n = 16 / 32 / 48, 1-16 columns; L2 flushed
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

    cases = [(L, nv, (1, 2, 4, 8, 12, 16)) for L in (4, 6, 8) for nv in (8, 16, 24)]
    if args.mrhs_case:
        L, nv, nr = (int(v) for v in args.mrhs_case.split(","))
        cases = [(L, nv, (nr,))]
    for L, nv, counts in cases:
        op = build_coarse_operator((6, L, nv), (2 * L,) * 4, nv, -0.42, CSW, device=dev)
        cop = cg.CoarseOp(op.self_blocks, op.hop_blocks, op.dims, op.nv, precisions=(cg.PREC_BF16,),
                          max_nrhs=16)
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
    eo = cg.COARSE_ODD_EVEN if args.batched_oddeven == "on" else 0
    p = cg.solve_params(precision=prec, inner_tol=inner_tol, flags=cg.COARSE_ZERO_GUESS | chain | eo, poly_degree=4,
                        defl_k=16, **SOLVER)
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
    # plain FP64 GPU GMRES(50) on the same right-hand sides of every `fp64_stride`-th operator (a
    # sample of the same mix of sizes): the reference point of the batched mixed-precision speedup
    p64 = cg.solve_params(precision=cg.PREC_FP64, m=SOLVER["m"], tol=SOLVER["tol"], max_restarts=4000, max_ir=5,
                          flags=cg.COARSE_ZERO_GUESS)
    sample = list(range(0, len(ops), max(1, args.fp64_stride)))
    n64 = sum(bs[i].shape[0] for i in sample)
    ops[sample[0]].solve(bs[sample[0]][:1].contiguous(), xs[sample[0]][:1].contiguous(), params=p64)
    torch.cuda.synchronize()
    worst64 = 0.0
    with ClockSampler(0) as clk64:
        e0.record()
        for i in sample:
            _, inf = ops[i].solve(bs[i], xs[i], params=p64)
            worst64 = max(worst64, max(q["rel_residual"] for q in inf))
        e1.record()
        torch.cuda.synchronize()
    ms64 = e0.elapsed_time(e1)
    rate64 = n64 / (ms64 / 1e3)
    rate = nrhs / (ms / 1e3)
    print(json.dumps({"mode": "batched", "operators": len(ops), "right_hand_sides": nrhs,
                      "precision": args.prec, "polynomial_chain_blocks": "bf16" if chain else args.prec,
                      "inner_system": "odd-even reduced, block-Jacobi preconditioned" if eo else "full operator",
                      "ms_per_batch": round(ms, 2),
                      "rhs_solves_per_s": round(nrhs / (ms / 1e3), 1), "operator_batches_per_s": round(1e3 / ms, 3),
                      "sequential_ms": round(ms_seq, 2), "speedup_vs_sequential": round(ms_seq / ms, 2),
                      "worst_rel_residual": worst, "kernel_launches_per_batch": infos[0]["kernel_launches"],
                      "per_solve": {f: {"mean": round(statistics.mean(i[f] for i in infos), 2),
                                        "max": max(i[f] for i in infos)}
                                    for f in ("iterations", "cycles", "ir_steps", "recycle_updates")},
                      "generate_s": round(t_gen, 1), "setup_s": round(t_setup, 2), "clocks": clk.summary(),
                      "fp64_gmres_baseline": {"rhs_solves_per_s": round(rate64, 2), "right_hand_sides": n64,
                                              "operators": len(sample), "ms": round(ms64, 1),
                                              "worst_rel_residual": worst64, "speedup": round(rate / rate64, 2),
                                              "sample": f"every {max(1, args.fp64_stride)}-th operator, all its "
                                                        "right-hand sides, solved one after another",
                                              "clocks": clk64.summary()}}),
          flush=True)
    for o in ops:
        o.close()


def run_autograd(args):
    """Differentiation workload: L = Re <c, D_c^{-1} b> on the Wilson-clover coarse 8^4, n = 32
    operator (m0 = -0.42); one step = the forward solve and the backward pass (adjoint solve through
    sigma3 D_c(-mu) sigma3 and the block gradients), FP32 inner solves with FP64 refinement."""
    import torch

    import paper_2205_09104_gb300 as cg
    from synthetic import draws
    dev = torch.device("cuda", 0)
    wl = dict(WORKLOADS["wilson8"], key=(5, 0))
    op, gen_s = build_operator(wl, dev)
    n, V = op.n, op.volume
    N = n * V
    S = op.self_blocks.clone().requires_grad_()
    H = op.hop_blocks.clone().requires_grad_()
    cop = cg.CoarseOp(S.detach(), H.detach(), op.dims, op.nv, precisions=(cg.PREC_FP32, cg.PREC_BF16))
    p = solver_params(cg, wl, wl["k"])
    c, b, _ = draws.grad_draws((5, 1), N, V, n, 1)
    bt = torch.from_numpy(b).to(dev).requires_grad_()
    ct = torch.from_numpy(c).to(dev)

    def step():
        S.grad = H.grad = bt.grad = None
        x = cg.CoarseSolve.apply(bt, S, H, cop, p)
        loss = (ct.conj() * x).sum().real
        loss.backward()
        return loss
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        e0.record()
        for _ in range(args.steps):
            step()
        e1.record()
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    print(json.dumps({"mode": "autograd", "workload": "wilson-clover coarse 8^4, nv=16 -> n=32, m0=-0.42; "
                      "L = Re<c, D_c^-1 b>, forward + backward (adjoint solve + block gradients)",
                      "steps_per_s": round(1e3 / ms, 2), "ms_per_step": round(ms, 3),
                      "gradient_bytes_per_step": int((S.numel() + H.numel()) * 16),
                      "clocks": clk.summary()}), flush=True)
    cop.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="tm16", choices=sorted(WORKLOADS))
    ap.add_argument("--prec", default="fp32", choices=["fp32", "bf16", "fp64"],
                    help="block precision of --apply-only / --schur-only / --batched")
    ap.add_argument("--poly", default="bf16", choices=["bf16", "same"],
                    help="blocks of the polynomial-chain applies of --batched FP32 inner solves")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0,
                    help="seconds of oracle applies timed for the CPU baseline")
    ap.add_argument("--sweep", action="store_true",
                    help="mu sweep of the twisted-mass and m0 sweep of the Wilson-clover workload, k > 0 and k = 0")
    ap.add_argument("--sweep-workload", default="both", choices=["both", "one"],
                    help="with --sweep: both workloads, or only --workload")
    ap.add_argument("--apply-only", choices=sorted(APPLY_CASES), default=None,
                    help="time the stencil apply alone on one of the named lattices")
    ap.add_argument("--schur-only", choices=sorted(APPLY_CASES), default=None,
                    help="time the odd-even reduced operator alone on one of the named lattices")
    ap.add_argument("--no-flush", action="store_true")
    ap.add_argument("--fp64-baseline-steps", type=int, default=5,
                    help="plain FP64 GMRES(50) solves timed for the speedup (0 = skip)")
    ap.add_argument("--mrhs", action="store_true",
                    help="time the multi-right-hand-side tensor-core apply against the per-column path")
    ap.add_argument("--mrhs-case", default="",
                    help="one multi-right-hand-side case 'L,nv,nrhs' (coarse L^4, n = 2 nv)")
    ap.add_argument("--pipelined", action="store_true",
                    help="latency-1 pipelined Arnoldi (COARSE_PIPELINED) in the solves of the default line")
    ap.add_argument("--autograd", action="store_true",
                    help="time forward + backward of the differentiable solve (Wilson-clover 8^4, n = 32)")
    ap.add_argument("--batched", type=int, default=0,
                    help="time the lockstep batched engine on this many uneven operators")
    ap.add_argument("--batched-oddeven", default="on", choices=["on", "off"],
                    help="with --batched: inner solves on the odd-even reduced system (COARSE_ODD_EVEN)")
    ap.add_argument("--fp64-stride", type=int, default=4,
                    help="with --batched: plain FP64 GMRES on every n-th operator for the speedup")
    args = ap.parse_args()
    PIPELINED["on"] = args.pipelined
    if args.autograd:
        run_autograd(args)
        return
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
    if args.sweep:
        run_sweep(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gb300(args)


if __name__ == "__main__":
    main()
