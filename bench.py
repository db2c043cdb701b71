#!/usr/bin/env python
"""Benchmark of the hierarchical subspace iteration on one GB300.

Metric: wall seconds for hsim_solve to the p lowest eigenpairs of a synthetic
mesh at a relative M^{-1}-norm residual (eq. conv2) of tol, with the level-0
matrices and the hierarchy resident on the device when the timed region
starts (the Galerkin products, every factorisation, solve, Gram, Ritz and
update are inside it).  Default workload: bumpy torus R = 1, r = 0.3 on a
1000 x 1000 grid (10^6 vertices, 2 x 10^6 triangles), p = 500, tol = 1e-5,
three levels.

One JSON line on stdout (rank 0).  Extra keys:
  e2e           the same solve through the C ABI from pinned host buffers:
                S values + M diagonal copied in, eigenpairs copied out
  roofline      dominant kernel of the solve: algorithmic work / CUDA-event time
  cpu_baseline  the FP64 CPU oracle on a bounded sample (see oracle/baseline.py)
  clocks        nvidia-smi samples taken during the timed region
  info          iteration counts, shifts and per-phase times of the last solve

--impl reference times the CPU oracle instead (bounded sample per step).
Under torchrun with N > 1 every rank solves its own replica (the solve does
not shard); the reported time is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "s to 500 lowest eigenpairs, 1M-vert mesh, resid<=1e-5; mixed vs FP64 GPU"


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# FP64 rate: no FP64 figure is measured by the pool; GB300's nominal FP64
# rate is 1.25 TFLOP/s (152 SMs).  A probe on this machine measured 1.19.
FP64_PEAK_TFLOPS = 1.25
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


class ClockSampler:
    def __init__(self):
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,"
                 "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self, gpu_index=0):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9 or parts[0] != str(gpu_index):
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax = float(parts[2])
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": smax, "samples": len(sm),
                "reasons": sorted(reasons)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(value, world, device):
    """The largest value over the ranks: every rank times its own replica of
    the solve, and the slowest one sets the job's time."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# Iterations per level (finest first) that the mixed GPU solve takes on each
# benchmark workload (its info["iters"]); the reference arm's CPU model charges
# the oracle the same number of subspace iterations.
GPU_ITERS = {"bumpy_torus_1000": [8, 13, 0]}


def run_reference(args, world, rank):
    """CPU oracle, bounded sample per step; rank 0 only.  Each sample runs in
    a fresh subprocess (the oracle's solve workers are forked from it)."""
    if rank != 0:
        return
    iters = GPU_ITERS.get(args.workload)
    samples = []
    for i in range(args.warmup + args.steps):
        r = cpu_baseline(args.workload, {"iters": iters})
        if "error" in r:
            raise RuntimeError(r["error"])
        if i >= args.warmup:
            samples.append(r)
    v = sum(s["value"] for s in samples) / len(samples)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1000.0,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload},
            "cpu_baseline": {"kind": "oracle", "cores": samples[-1]["cores"], "sample": samples[-1]["sample"],
                             "value": v, "unit": "s", "model": samples[-1].get("model")},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="hsim", choices=["hsim", "reference"])
    ap.add_argument("--workload", default="bumpy_torus_1000")
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--fp64-steps", type=int, default=1,
                    help="timed FP64 solves for the mixed-vs-FP64 comparison (0 = skip)")
    ap.add_argument("--tol", type=float, default=None)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--max-iters", type=int, default=100)
    ap.add_argument("--leaf-size", type=int, default=0, help="nested-dissection leaf size (0: library default)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--kernel", default=None, choices=["gram", "gram_tc", "update", "update_tc", "spmm", "ritz", "ritz_tc",
                                                       "factor_tc", "hierarchy"],
                    help="time one step-level kernel on random data instead of the solve (profiling)")
    ap.add_argument("--mesh-nu", type=int, default=0,
                    help="--kernel spmm: an nu x nu bumpy torus instead of the workload's mesh")
    ap.add_argument("--rows", type=int, default=200000)
    ap.add_argument("--digits", type=int, default=6, choices=[5, 6], help="--kernel gram_tc: digits per value")
    ap.add_argument("--cols", type=int, default=750)
    ap.add_argument("--batch", type=int, default=0,
                    help="time the batched solve of this many seeded meshes (5k-80k vertices, p = 50) "
                         "against sequential solves instead of the 10^6-vertex workload")
    ap.add_argument("--streams", type=int, default=0, help="worker streams of the batched solve (0 = 8)")
    ap.add_argument("--sweep", default=None, choices=["levels", "sigma", "alpha"],
                    help="solve --workload for a range of one parameter (the paper's level, support and shift "
                         "tables) and print iteration counts and times, instead of the benchmark")
    ap.add_argument("--compare-sim", action="store_true",
                    help="time plain SIM (Alg. 1 from the initialisation heuristic) against HSIM on --workload "
                         "(FP64, both with the shift HSIM takes on the finest level) instead of the benchmark")
    args = ap.parse_args()
    if args.kernel:
        run_kernel(args)
        return
    if args.batch:
        run_batch(args)
        return
    if args.compare_sim:
        run_compare_sim(args)
        return
    if args.sweep:
        run_sweep(args)
        return
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return

    import numpy as np
    import torch

    import paper_2111_09039_gb300 as hs
    import synth

    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    w, mesh, start = synth.make_workload(args.workload)
    p = w.p
    tol = args.tol if args.tol is not None else (1e-5 if w.tol < 1e-5 else w.tol)
    prec = hs.HSIM_FP64 if args.precision == "fp64" else hs.HSIM_MIXED
    ctx = hs.Context(local)
    leaf = {"leaf_size": args.leaf_size} if args.leaf_size > 0 else {}
    t0 = time.perf_counter()
    if mesh.V is not None:
        hier = hs.Hierarchy(ctx, mesh.F, V=mesh.V, p=p, levels=w.levels, start_vertex=start, precision=prec, **leaf)
        S, Md = hs.assemble(ctx, hier, V=torch.as_tensor(mesh.V, device=dev))
    else:
        hier = hs.Hierarchy(ctx, mesh.F, L2=mesh.L2, p=p, levels=w.levels, start_vertex=start, precision=prec, **leaf)
        S, Md = hs.assemble(ctx, hier, L2=torch.as_tensor(mesh.L2, device=dev))
    torch.cuda.synchronize()
    hier_s = time.perf_counter() - t0
    opts = hs.default_options(levels=w.levels, start_vertex=start, precision=prec, max_iters=args.max_iters)
    stream = ctx.stream

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    info = None
    for _ in range(args.warmup):
        lam, Phi, info = hs.solve(ctx, hier, S, Md, p, tol, options=opts)
    barrier()
    clocks = ClockSampler()
    clocks.start()
    launches0 = hs.kernel_launches()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    infos = []
    ev0.record(stream)
    for _ in range(args.steps):
        lam, Phi, info = hs.solve(ctx, hier, S, Md, p, tol, options=opts)
        infos.append(info)
    ev1.record(stream)
    barrier()
    clk = clocks.stop(local)
    launches = (hs.kernel_launches() - launches0) / args.steps
    ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, world, dev)

    # end to end through the C ABI from pinned host buffers, right after the
    # timed solves (before the long FP64 comparison) so that both run in the
    # same state of the GPU
    S_h = S.cpu().pin_memory()
    Md_h = Md.cpu().pin_memory()
    lam_h = torch.empty(p, dtype=torch.float64).pin_memory()
    vec_h = torch.empty((p, hier.n), dtype=torch.float64).pin_memory()
    S_d = torch.empty_like(S)
    Md_d = torch.empty_like(Md)
    e2e_ms = []
    seg = {"h2d": [], "solve": [], "d2h": []}
    # one untimed step first (first use of the pinned buffers and of the
    # output allocations), then the mean of the timed steps; host clock
    # marks after the input copy and after the solve split each step into
    # its segments (the marks synchronise the stream, which the copies and
    # the solve's own convergence tests do anyway)
    for step in range(max(0, args.e2e_steps) + (1 if args.e2e_steps > 0 else 0)):
        barrier()
        t1 = time.perf_counter()
        with torch.cuda.stream(stream):
            S_d.copy_(S_h, non_blocking=True)
            Md_d.copy_(Md_h, non_blocking=True)
        stream.synchronize()
        t2 = time.perf_counter()
        lam_d, Phi_d, _ = hs.solve(ctx, hier, S_d, Md_d, p, tol, options=opts)
        stream.synchronize()
        t3 = time.perf_counter()
        with torch.cuda.stream(stream):
            lam_h.copy_(lam_d, non_blocking=True)
            vec_h.copy_(Phi_d.t(), non_blocking=True)
        stream.synchronize()
        t4 = time.perf_counter()
        if step > 0:
            e2e_ms.append((t4 - t1) * 1000.0)
            seg["h2d"].append(t2 - t1)
            seg["solve"].append(t3 - t2)
            seg["d2h"].append(t4 - t3)
    e2e_mean = max_over_ranks(sum(e2e_ms) / len(e2e_ms), world, dev) if e2e_ms else None
    e2e_seg = {k: sum(v) / len(v) for k, v in seg.items()} if e2e_ms else None
    h2d = S.numel() * 8 + Md.numel() * 8
    d2h = p * 8 + p * hier.n * 8

    # the FP64 GPU form of the same solve, for the mixed-vs-FP64 comparison
    fp64 = None
    if args.precision == "mixed" and args.fp64_steps > 0:
        o64 = hs.default_options(levels=w.levels, start_vertex=start, precision=hs.HSIM_FP64,
                                 max_iters=args.max_iters)
        hs.solve(ctx, hier, S, Md, p, tol, options=o64)  # warm-up
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.fp64_steps):
            lam64, Phi64, info64 = hs.solve(ctx, hier, S, Md, p, tol, options=o64)
        e1.record(stream)
        barrier()
        ms64 = e0.elapsed_time(e1) / args.fp64_steps
        dl = (lam - lam64).abs() / torch.clamp(lam64.abs(), min=float(lam64[1]))
        fp64 = {"value": ms64 / 1000.0, "unit": "s", "steps": args.fp64_steps,
                "speedup_mixed_vs_fp64": ms64 / ms, "max_rel_eigenvalue_diff": float(dl.max().item()),
                "max_residual_check": check_residual(hier, S, Md, lam64, Phi64, ctx), "info": info64}

    # residual check of the timed result, in FP64 on the device
    res = check_residual(hier, S, Md, lam, Phi, ctx)

    if rank != 0:
        return
    peaks, peak_src = load_peaks()
    roof = roofline(info, infos, hier, p, peaks, peak_src, args.precision, tol)
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline(args.workload, info)
    line = {
        "metric": METRIC, "value": ms / 1000.0, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "bf16+f32+f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "vertices": hier.n, "triangles": hier.m, "p": p, "tol": tol,
                   "levels": hier.sizes, "precision": args.precision, "parallelism": "replicas" if world > 1 else "1 gpu",
                   "l2": "working set > L2 (n x q float64 blocks of 6 GB)"},
        "hier_build_s": hier_s, "hier_plus_solve_s": hier_s + ms / 1000.0, "max_residual_check": res,
        "e2e": ({"value": e2e_mean / 1000.0, "unit": "s", "h2d_bytes_per_step": h2d,
                 "d2h_bytes_per_step": d2h, "steps": len(e2e_ms), "warmup": 1,
                 "segments_s": e2e_seg} if e2e_ms else None),
        "gpu_launches": int(round(launches)),
        "fp64_gpu": fp64,
        "roofline": roof, "cpu_baseline": cpu, "clocks": clk, "info": info,
    }
    print(json.dumps(line), flush=True)


def run_kernel(args):
    """One step-level kernel on seeded random data (rows x cols FP64 blocks):
    two untimed calls, then `steps` timed calls with CUDA events."""
    import torch

    import paper_2111_09039_gb300 as hs
    ctx = hs.Context(0)
    if args.kernel == "hierarchy":
        run_hierarchy(args, hs, ctx)
        return
    g = torch.Generator(device="cuda:0").manual_seed(0)
    n, q = args.rows, args.cols
    A = torch.randn((n, q), dtype=torch.float64, device="cuda:0", generator=g)
    B = torch.randn((n, q), dtype=torch.float64, device="cuda:0", generator=g)
    P = torch.randn((q, q), dtype=torch.float64, device="cuda:0", generator=g)
    if args.kernel == "spmm":
        import synth
        if args.mesh_nu > 0:
            mesh = synth.bumpy_torus(args.mesh_nu, args.mesh_nu, 3)
            hier = hs.Hierarchy(ctx, mesh.F, V=mesh.V, p=min(50, mesh.n // 40), levels=2, start_vertex=0)
        else:
            w, mesh, start = synth.make_workload("bumpy_torus_1000" if n >= 10**6 else "bumpy_torus_100")
            hier = hs.Hierarchy(ctx, mesh.F, V=mesh.V, p=w.p, levels=w.levels, start_vertex=start)
        S, Md = hs.assemble(ctx, hier, V=torch.as_tensor(mesh.V, device="cuda:0"))
        rp, cl = hier.pattern()
        A = torch.randn((mesh.n, q), dtype=torch.float64, device="cuda:0", generator=g)
        fn = lambda: hs.spmm(ctx, rp, cl, S, A)
        flops, nbytes = 2.0 * S.numel() * q, 16.0 * mesh.n * q + 12.0 * S.numel()
    elif args.kernel == "factor_tc":
        # FP32 factorisation (blocked, tensor-core Schur updates on large
        # fronts) and inverted-form solve of S - mu M, mu = -5, level 0 of a
        # --mesh-nu x --mesh-nu bumpy torus, --cols right-hand sides
        import synth
        nu = args.mesh_nu if args.mesh_nu > 0 else 320
        mesh = synth.bumpy_torus(nu, nu, 5)
        hier = hs.Hierarchy(ctx, mesh.F, V=mesh.V, p=50, levels=2, start_vertex=11, precision=hs.HSIM_MIXED)
        S, Md = hs.assemble(ctx, hier, V=torch.as_tensor(mesh.V, device="cuda:0"))
        n = mesh.n
        X0 = torch.randn((n, q), dtype=torch.float64, device="cuda:0", generator=g)
        fn = lambda: hs.shifted_solve(ctx, hier, 0, S, Md, -5.0, X0, f32=True)
        flops, nbytes = 0.0, 8.0 * n * q
    elif args.kernel in ("gram", "gram_tc"):
        fn = (lambda: hs.gram(ctx, A, B)) if args.kernel == "gram" else (lambda: hs.gram_tc(ctx, A, B, args.digits))
        flops, nbytes = 2.0 * n * q * q, 16.0 * n * q
    elif args.kernel in ("ritz", "ritz_tc"):
        # q x q symmetric S_bar and SPD M_bar with random eigenvectors
        Sb = P + P.t()
        C = torch.randn((q, q), dtype=torch.float64, device="cuda:0", generator=g)
        Mb = torch.eye(q, dtype=torch.float64, device="cuda:0") + (C @ C.t()) / (10.0 * q)
        tc = args.kernel == "ritz_tc"
        fn = lambda: hs.ritz(ctx, Sb, Mb, tc=tc)
        flops, nbytes = 0.0, 16.0 * q * q
    else:
        f = hs.gemm_update if args.kernel == "update" else hs.gemm_update_tc
        fn = lambda: f(ctx, A, P)
        flops, nbytes = 2.0 * n * q * q, 16.0 * n * q
    for _ in range(2):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(ctx.stream)
    for _ in range(max(1, args.steps)):
        fn()
    e1.record(ctx.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(1, args.steps)
    extra = {}
    if args.kernel in ("ritz", "ritz_tc"):
        extra["sweeps"] = fn()[2]
    print(json.dumps({"kernel": args.kernel, "rows": n, "cols": q, "ms": ms, **extra,
                      "fp64_equivalent_tflops": flops / (ms * 1e-3) / 1e12,
                      "algorithmic_gbs": nbytes / (ms * 1e-3) / 1e9}), flush=True)


def run_hierarchy(args, hs, ctx):
    """Wall time of hsim_build_hierarchy on --workload: the farthest-point
    order and prolongations on the GPU (the default) and on the host, one
    untimed GPU build first, `steps` timed builds each."""
    import time

    import torch

    import synth
    w, mesh, start = synth.make_workload(args.workload)
    kw = dict(V=mesh.V) if mesh.V is not None else dict(L2=mesh.L2)

    def build(dev):
        torch.cuda.synchronize()
        t = time.perf_counter()
        h = hs.Hierarchy(ctx, mesh.F, p=w.p, levels=w.levels, start_vertex=start, hier_device=dev, **kw)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t
        h.close()
        return dt

    build(1)
    out = {"kernel": "hierarchy", "workload": args.workload, "vertices": mesh.n}
    for dev, key in ((1, "gpu_s"), (0, "host_s")):
        out[key] = min(build(dev) for _ in range(max(1, args.steps)))
    print(json.dumps(out), flush=True)


def run_sweep(args):
    """One JSON line per value of the swept parameter (T in 2..5, sigma in
    3..11, alpha in 0.05..1/3, as in the paper's level, support and shift
    tables): hierarchy build time (host wall clock), solve time (CUDA events,
    after one untimed solve) and iterations per level."""
    import torch

    import paper_2111_09039_gb300 as hs
    import synth
    w, mesh, start = synth.make_workload(args.workload)
    tol = args.tol if args.tol is not None else w.tol
    prec = hs.HSIM_FP64 if args.precision == "fp64" else hs.HSIM_MIXED
    values = {"levels": [2, 3, 4, 5], "sigma": [3.0, 5.0, 7.0, 9.0, 11.0],
              "alpha": [0.05, 0.1, 0.2, 1.0 / 3.0]}[args.sweep]
    ctx = hs.Context(0)
    V = torch.as_tensor(mesh.V, device="cuda:0")
    for v in values:
        kw = {"levels": w.levels, "sigma": 7.0, "alpha": 0.1}
        kw[args.sweep] = v
        t0 = time.perf_counter()
        hier = hs.Hierarchy(ctx, mesh.F, V=mesh.V, p=w.p, start_vertex=start, precision=prec, levels=kw["levels"],
                            sigma=kw["sigma"])
        S, Md = hs.assemble(ctx, hier, V=V)
        torch.cuda.synchronize()
        t_h = time.perf_counter() - t0
        solve = lambda: hs.solve(ctx, hier, S, Md, w.p, tol, precision=prec, alpha=kw["alpha"],
                                 max_iters=args.max_iters)
        solve()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(ctx.stream)
        lam, _, info = solve()
        e1.record(ctx.stream)
        torch.cuda.synchronize()
        print(json.dumps({"mode": "sweep", "parameter": args.sweep, "value": v, "workload": args.workload,
                          "p": w.p, "tol": tol, "precision": args.precision, "levels": info["sizes"],
                          "iters": info["iters"], "hier_s": t_h, "solve_s": e0.elapsed_time(e1) / 1000.0,
                          "max_residual": info["max_residual"]}), flush=True)


def run_compare_sim(args):
    """HSIM against plain SIM (the paper's SIM column of Table vsAll) on one
    workload, FP64: HSIM first, then plain SIM with the shift HSIM used on the
    finest level, so that only the starting subspace differs.  Device time of
    each solve (CUDA events, after one untimed solve of each)."""
    import torch

    import paper_2111_09039_gb300 as hs
    import synth
    w, mesh, start = synth.make_workload(args.workload)
    tol = args.tol if args.tol is not None else 1e-2
    ctx = hs.Context(0)
    V = torch.as_tensor(mesh.V, device="cuda:0")
    hier = hs.Hierarchy(ctx, mesh.F, V=mesh.V, p=w.p, levels=w.levels, start_vertex=start)
    S, Md = hs.assemble(ctx, hier, V=V)
    flat = hs.Hierarchy(ctx, mesh.F, V=mesh.V, p=w.p, start_vertex=start, plain_sim=1)
    S1, Md1 = hs.assemble(ctx, flat, V=V)

    def timed(fn):
        fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(ctx.stream)
        out = fn()
        e1.record(ctx.stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1000.0, out

    t_h, (lam_h, _, info_h) = timed(lambda: hs.solve(ctx, hier, S, Md, w.p, tol, max_iters=args.max_iters))
    mu = info_h["shift"][0]
    t_s, (lam_s, _, info_s) = timed(lambda: hs.solve(ctx, flat, S1, Md1, w.p, tol, sim_shift=mu, seed=1,
                                                     max_iters=args.max_iters))
    dl = float(((lam_h - lam_s).abs() / lam_h.abs().clamp_min(float(lam_h[1]))).max())
    print(json.dumps({"mode": "compare_sim", "workload": args.workload, "vertices": mesh.n, "p": w.p, "tol": tol,
                      "hsim_s": t_h, "hsim_iters": info_h["iters"], "sim_s": t_s, "sim_iters": info_s["iters"][0],
                      "speedup_hsim_vs_sim": t_s / t_h, "shift": mu, "max_rel_eigenvalue_diff": dl,
                      "dtype": "f64", "data": "synthetic"}), flush=True)


def batch_shard(sizes, world):
    """Independent meshes onto ranks: largest first onto the least loaded rank
    (the lower rank on ties); one ascending index list per rank.  The meshes
    share nothing, so the ranks exchange only their times."""
    load = [0] * world
    out = [[] for _ in range(world)]
    for i in sorted(range(len(sizes)), key=lambda i: (-sizes[i], i)):
        r = min(range(world), key=lambda r: (load[r], r))
        out[r].append(i)
        load[r] += sizes[i]
    return [sorted(o) for o in out]


def run_batch(args):
    """Batched solve of `args.batch` seeded meshes (displaced geodesic
    icospheres and bumpy tori, 5k-80k vertices, p = 50, T = 2, tol 1e-5, mixed
    precision) against the same solves one after the other.  Both are timed on
    the host around the calls, with the device synchronised on both sides
    (the batched call spans several streams); inputs resident, workspaces
    allocated by the warm-up.  Under torchrun the meshes are split over the
    ranks (batch_shard) and the times are the maxima over ranks."""
    import torch

    import paper_2111_09039_gb300 as hs
    import synth
    from synth import workloads

    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    ctx = hs.Context(local)
    everything = synth.batch(count=args.batch)
    mine = batch_shard([m.n for m, _ in everything], world)[rank]
    items = [everything[i] for i in mine]
    p, T, tol = workloads.BATCH_P, workloads.BATCH_LEVELS, args.tol or workloads.BATCH_TOL
    t0 = time.perf_counter()
    hiers = [hs.Hierarchy(ctx, m.F, V=m.V, p=p, levels=T, start_vertex=st, precision=hs.HSIM_MIXED)
             for m, st in items]
    hier_s = time.perf_counter() - t0
    S, M = [], []
    for (m, _), h in zip(items, hiers):
        s_, md = hs.assemble(ctx, h, V=torch.as_tensor(m.V, device=dev))
        S.append(s_)
        M.append(md)
    opts = hs.default_options(precision=hs.HSIM_MIXED, levels=T, max_iters=args.max_iters)
    for _ in range(max(1, args.warmup)):
        hs.solve_batched(ctx, hiers, S, M, p, tol, options=opts, streams=args.streams)
    torch.cuda.synchronize()

    def timed(fn):
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        t = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        return max_over_ranks(time.perf_counter() - t, world, dev), out

    seq, bat = [], []
    l0 = hs.kernel_launches()
    for _ in range(args.steps):
        dt, out_b = timed(lambda: hs.solve_batched(ctx, hiers, S, M, p, tol, options=opts, streams=args.streams))
        bat.append(dt)
    launches = (hs.kernel_launches() - l0) / max(1, args.steps)
    for _ in range(args.steps):
        def one_by_one():
            return [hs.solve(ctx, h, S[i], M[i], p, tol, options=opts) for i, h in enumerate(hiers)]
        dt, out_s = timed(one_by_one)
        seq.append(dt)
    res = max([check_residual(h, S[i], M[i], out_b[i][0], out_b[i][1], ctx) for i, h in enumerate(hiers)] + [0.0])
    dl = max([float(((out_b[i][0] - out_s[i][0]).abs() / out_s[i][0].abs().clamp_min(out_s[i][0][1])).max())
              for i in range(len(hiers))] + [0.0])
    res, dl = max_over_ranks(res, world, dev), max_over_ranks(dl, world, dev)
    vb, vs = min(bat), min(seq)
    if rank != 0:
        return
    line = {"metric": f"s for {len(everything)} independent meshes ({min(m.n for m, _ in everything)}-"
                      f"{max(m.n for m, _ in everything)} vertices), {p} lowest eigenpairs each, resid<={tol:g}",
            "value": vb, "unit": "s", "n_gpus": world, "steps": args.steps, "warmup": max(1, args.warmup),
            "scaling": "strong", "meshes_per_rank": [len(x) for x in batch_shard([m.n for m, _ in everything], world)],
            "higher_is_better": False, "mode": "batched", "streams": args.streams or 8,
            "sequential_s": vs, "speedup_batched_vs_sequential": vs / vb,
            "vertices_total": int(sum(m.n for m, _ in everything)), "max_residual_check": res,
            "max_rel_eigenvalue_diff_batched_vs_sequential": dl, "hier_build_s": hier_s,
            "gpu_launches": int(round(launches)), "dtype": "bf16+f32+f64", "data": "synthetic",
            "config": {"workload": f"batch of {len(everything)} (seed 4)", "p": p, "levels": T, "tol": tol,
                       "precision": "mixed", "parallelism": f"meshes split over {world} rank(s)"},
            "timing": "host clock around the call, device synchronised on both sides"}
    print(json.dumps(line), flush=True)


def check_residual(hier, S, Md, lam, Phi, ctx):
    """max_i ||S phi_i - lam_i M phi_i||_{M^-1} / ||S phi_i||_{M^-1}, FP64, with
    torch's sparse CSR product (independent of the library's kernels)."""
    import torch
    rp, cl = hier.pattern()
    A = torch.sparse_csr_tensor(rp.long(), cl.long(), S, size=(hier.n, hier.n))
    SP = (A @ Phi.contiguous())
    MP = Md[:, None] * Phi
    R = SP - MP * lam[None, :]
    w = (1.0 / Md)[:, None]
    nr = torch.sqrt((R * R * w).sum(0))
    ns = torch.sqrt((SP * SP * w).sum(0))
    nm = torch.sqrt((MP * MP * w).sum(0))
    above = lam[lam > 1e-8 * lam[-1]]
    lref = above[0] if above.numel() else lam[-1]
    return float((nr / torch.maximum(ns, lref * nm)).max().item())


# the library's Grams take five digits per value from this tolerance up (six below)
GRAM_FIVE_DIGIT_TOL = 1e-6


def roofline(info, infos, hier, p, peaks, peak_src, precision, tol):
    """Achieved rate against the peak for the kernels of the solve; the
    top-level entry is the kernel of the dominant phase."""
    q = info["q"]
    sizes = info["sizes"]
    iters = info["iters"]
    steps = len(infos)
    avg = lambda key: sum(i[key] for i in infos) / steps
    phases = {k: avg("ms_" + k) for k in
              ("galerkin", "coarse", "prolong", "factor", "solve", "spmm", "gram", "ritz", "update", "residual")}
    dom = max(phases, key=phases.get)
    sim_levels = range(len(sizes) - 1)
    n_products = sum(iters[t] for t in sim_levels)
    kernels = {}
    # Ritz eigensolver: Householder tridiagonalisation (4/3 q^3 FP64 flops) and
    # back transformation of the q eigenvectors (2 q^3), per call
    calls = avg("ritz_calls")
    ms_ritz = phases["ritz"]
    rflops = (4.0 / 3.0 + 2.0) * q ** 3 * calls
    jac = rflops / (ms_ritz * 1e-3) / 1e12 if ms_ritz > 0 else 0.0
    kernels["ritz"] = {"kernel": "k_tridiag + k_tri_* (Householder tridiagonalisation, bisection, inverse "
                                 "iteration, back transformation; FP64)", "bound": "alu",
                       "achieved": jac, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": jac / FP64_PEAK_TFLOPS,
                       "peak_source": "GB300 nominal FP64 (1.25 TFLOP/s; a DFMA probe measured 1.19)",
                       "traffic": None, "flops_per_call": (4.0 / 3.0 + 2.0) * q ** 3, "calls_per_step": calls,
                       "note": "time includes the LDL^T of M_bar and the triangular transforms of the "
                       "Rayleigh-Ritz step; the tridiagonalisation takes one grid barrier per column"}
    # supernodal triangular solves: 4 nnz(L) flops per right-hand side
    sflops = avg("solve_flops")
    ms_solve = phases["solve"]
    fp_peak = FP32_PEAK_TFLOPS if precision != "fp64" else FP64_PEAK_TFLOPS
    sach = sflops / (ms_solve * 1e-3) / 1e12 if ms_solve > 0 else 0.0
    kernels["solve"] = {"kernel": "k_solve_* (supernodal LDL^T forward/backward solves, %s)" %
                        ("FP32" if precision != "fp64" else "FP64"), "bound": "alu", "achieved": sach,
                        "peak": fp_peak, "unit": "TFLOP/s", "frac": sach / fp_peak,
                        "peak_source": "FP32: 152 SMs x 128 lanes x 2 flop x 2.07 GHz = 80.5 TFLOP/s"
                        if precision != "fp64" else "GB300 nominal FP64 (1.25 TFLOP/s)",
                        "traffic": None, "note": "phase time includes the residual and SpMM of the "
                        "correction-form iteration"}
    gram_flops = sum(iters[t] * 2.0 * sizes[t] * q * (q + 1) for t in sim_levels)
    upd_flops = sum(iters[t] * 2.0 * sizes[t] * q * q for t in sim_levels)
    if precision == "fp64":
        ms_gram = phases["gram"]
        ach = gram_flops / (ms_gram * 1e-3) / 1e12 if ms_gram > 0 else 0.0
        kernels["gram"] = {"kernel": "k_gram (FP64 DFMA, Psi^T S Psi and Psi^T M Psi)", "bound": "alu",
                           "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                           "frac": ach / FP64_PEAK_TFLOPS,
                           "peak_source": "GB300 nominal FP64 (1.25 TFLOP/s; a DFMA probe measured 1.19)",
                           "traffic": None, "launches_per_step": 2 * n_products,
                           "update_gemm_tflops": upd_flops / (phases["update"] * 1e-3) / 1e12
                           if phases["update"] > 0 else 0.0}
        kernels["update"] = kernels["gram"]
    else:
        # tensor-core products: digit-pair products (d digits: pairs s + t < d,
        # d (d + 1) / 2 of them) of 2 n q(q+1)/2 BF16 flops for each symmetric
        # Gram (two per iteration; 5 digits at tol >= 1e-6, else 6) and 21 of
        # 2 n q^2 for the update, timed without the digit split
        gd = 5 if tol >= GRAM_FIVE_DIGIT_TOL else 6
        gram_pairs, upd_pairs = gd * (gd + 1) // 2, 21
        tc_flops = gram_pairs * gram_flops + upd_pairs * upd_flops
        ms_tc = avg("ms_tc_product")
        peak = peaks.get("bf16_tflops_sustained", 1743.3)
        ach = tc_flops / (ms_tc * 1e-3) / 1e12 if ms_tc > 0 else 0.0
        kernels["gram"] = {"kernel": "k_ozaki_tc (FP64-accurate products on tcgen05 BF16 tensor cores)",
                           "bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                           "frac": ach / peak, "peak_source": f"{peak_src} bf16_tflops_sustained",
                           "traffic": None, "launches_per_step": 3 * n_products,
                           "fp64_equivalent_tflops": (gram_flops + upd_flops) / (ms_tc * 1e-3) / 1e12
                           if ms_tc > 0 else 0.0, "ms_per_step": ms_tc}
        kernels["update"] = kernels["gram"]
    # the top-level entry is the single kernel with the most GPU time: the
    # FP64-accurate product kernel (mixed) or the FP64 Gram (FP64 path); the
    # solve and Ritz phases are spread over several kernels (ncu launch lists)
    top = dict(kernels["gram"])
    if precision != "fp64":
        # achieved = the method's work (FP64 products of the two Grams and the
        # update) / the kernel's time; the BF16 pipe occupancy of the 21
        # digit-pair products is reported beside it
        ms_tc = top["ms_per_step"]
        fp64_eq = top["fp64_equivalent_tflops"]
        top["bf16_pipe"] = {"achieved": top["achieved"], "frac": top["frac"], "unit": "TFLOP/s",
                            "note": f"{gram_pairs} (Grams) and {upd_pairs} (update) BF16 digit-pair products "
                                    "per FP64 product (emulation work)"}
        top["achieved"] = fp64_eq
        top["frac"] = fp64_eq / top["peak"]
        top["work"] = ("method FLOPs: FP64 products of the Grams Psi^T [S Psi | M Psi] (n q (q+1) each, lower "
                       "triangles) and the update Psi Phi_bar (2 n q^2) of every subspace iteration")
        top["traffic"] = None
        tr = tc_traffic(sizes, iters, q, gd)
        if tr is not None:
            top["traffic"] = tr["per_launch"]
            top["traffic_note"] = tr["note"]
            top["algorithmic_bytes_per_launch"] = tr["algorithmic_per_launch"]
    top["dominant_phase"] = dom
    top["phase_ms"] = phases
    top["kernels"] = {k: {kk: v[kk] for kk in ("kernel", "bound", "achieved", "peak", "unit", "frac")}
                      for k, v in kernels.items() if k != "update"}
    return top


# DRAM bytes (read + write) per operand row of one k_ozaki_tc launch, from
# one ncu capture of each product shape at 200,000 rows, q = 750
# (profiles/ozaki_tc_traffic_n200k_q750.md): update (6 digits) 1.852 GB read +
# 1.170 GB written; Gram with the solve's 5 digits 3.090 GB read + 3 MB written
# for the full square product of the capture (the solve's Grams compute the
# lower triangle: an upper bound).
TC_TRAFFIC_PER_ROW = {"gram": (3090402816 + 3154688) / 200000, "update": (1852248576 + 1170459392) / 200000}


def tc_traffic(sizes, iters, q, gram_digits=6):
    """Per-launch DRAM traffic of k_ozaki_tc over one solve, scaled from the
    200,000-row captures by the rows each launch processes (traffic grows in
    proportion to the rows), against the algorithmic bytes (the BF16 digit
    slices read once: d slices x 2 bytes per operand value, d = gram_digits
    for the Grams and 6 for the update; the update's FP64 output, 8 bytes per
    value)."""
    if TC_TRAFFIC_PER_ROW["gram"] is None or TC_TRAFFIC_PER_ROW["update"] is None:
        return None
    qp = (q + 31) // 32 * 32
    tot, alg, launches = 0.0, 0.0, 0
    for t in range(len(sizes) - 1):
        n = sizes[t]
        # two Grams (Psi against S Psi, Psi against M Psi) and one update per iteration
        tot += iters[t] * (2 * TC_TRAFFIC_PER_ROW["gram"] * n + TC_TRAFFIC_PER_ROW["update"] * n)
        # Gram: both operands' slices (2 x 2 d bytes per value); update: Psi's
        # six slices plus the FP64 output Phi
        alg += iters[t] * (2 * 4.0 * gram_digits * n * qp + (12.0 * n * qp + 8.0 * n * q))
        launches += 3 * iters[t]
    return {"per_launch": tot / launches, "algorithmic_per_launch": alg / launches,
            "note": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one 5-digit Gram (full square, an "
                    "upper bound for the solve's lower-triangle Grams) and one 6-digit update launch at "
                    "200,000 x 750, scaled by rows to every launch of the solve and averaged per launch"}


def cpu_baseline(workload, info):
    """FP64 oracle on a bounded sample, in a fresh process (no CUDA state; its
    solve workers are spawned from it)."""
    cmd = [sys.executable, "-c",
           "import json,sys; sys.path.insert(0, %r); from oracle import baseline; "
           "print(json.dumps(baseline.sample(%r, iters=%s)))" % (ROOT, workload, json.dumps(info["iters"]))]
    try:
        out = subprocess.run(cmd, capture_output=True, text=True, timeout=1200)
        return json.loads(out.stdout.strip().splitlines()[-1])
    except Exception as e:  # the baseline is a report, not the measurement
        return {"kind": "oracle", "error": str(e)[:200]}


if __name__ == "__main__":
    main()
