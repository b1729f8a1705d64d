#!/usr/bin/env python
"""Benchmark: unknowns solved to tolerance per second for the 3D Monge-Ampere
FAS multigrid solver (FMG initialisation + V(2,2) cycles, 8-colour nonlinear
Gauss-Seidel) on one GB300 per rank.

Default workload: Example 4 of the paper (u = exp(|x|^2/2) on [0,1]^3) on a
257^3 grid (16,581,375 unknowns), stopping at a relative max-norm residual of
1e-10 evaluated in FP64.  A step is one complete solve: copy f and g into the
resident hierarchy, FMG, cycles to tolerance.  value = the mixed-precision
solve (FP32 correction cycles under an FP64 residual and update); the plain
FP64 solve of the same workload is reported beside it ("fp64").  Inputs are resident in HBM when the
timed region starts; the hierarchy's working set (4 x 136 MB of level-0
fields) exceeds the 129 MB L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--n 257] [--problem exp] [--tol 1e-10]

--impl reference times the FP64 CPU oracle (oracle/) on the host cores.  Under
torchrun (N > 1) each rank solves its own copy of the workload (replicas, no
collective in the data path) and rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# FP64 operations of one FP64-smoother point update: gather 15 adds + 1 (-8 v0),
# 4x-scaled diagonal 3, shifted determinant 12, h^6 rhs 1, subtraction 1,
# FP64 Newton correction 1, centre update 1; the FP32 first pass and the
# integer FP64<->FP32 moves are not counted.
SMOOTH_FP64_OPS_PER_POINT = 35
FP64_NOMINAL_GOPS = 629.0   # 2 FP64 ops/clk/SM x 152 SMs x 2.07 GHz (nominal 1.25 TFLOP/s, FMA = 2 flops)
# Algorithmic HBM bytes of one FP32 correction-smoother point update: base
# Hessian 6 x 4 B, rhs 4 B, e read 4 B and written 4 B (each e value read
# once per sweep for the stencils, counted at its own update).
CORR_SMOOTH_BYTES_PER_POINT = 36
# HBM roofline denominator: the copy bandwidth measured on this GPU model
# (hbm_gbs of MEASURED_PEAKS.json at the repository root, written by the
# measurement of the pool's peaks); 6800 GB/s, an earlier GB300 measurement,
# when that file is absent.
HBM_PEAK_FALLBACK_GBS = 6800.0


def hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs, copy bandwidth)"
    except (OSError, KeyError, ValueError, TypeError):
        return HBM_PEAK_FALLBACK_GBS, "fallback (6.8 TB/s, an earlier GB300 copy measurement)"


# FP32 correction V-cycles per outer iteration of the single mixed solves
# (129^3 and up): with 2 the FP64 residual checks the stopping rule every two
# cycles, which ends a solve nearer the cycle that reaches the tolerance and
# spends fewer cycles detecting a round-off floor; the library default, 3,
# suits small grids and batches, where an outer iteration's fixed cost weighs
# more.
MIXED_INNER = 2
# DRAM bytes (read + write) per launch of the colour-pair correction smoother
# (MA_CORR_PAIRS = 5) at 257^3, from one ncu capture of the current kernel
# with a warm L2 (--cache-control none): 167.0-168.9 MB read + 43.0-43.4 MB
# written.  Other variants: no current capture (null).
CORR_SMOOTH_TRAFFIC_257 = {5: 211.2e6}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=257)
    ap.add_argument("--problem", default="exp")
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--cpu-threads", type=int, default=0,
                    help="host threads of the oracle (cpu_baseline and --impl reference); 0 = all cores")
    args = ap.parse_args()
    if args.cpu_threads > 0:
        # read by the oracle's OpenMP runtime when the library is first loaded
        os.environ["OMP_NUM_THREADS"] = str(args.cpu_threads)
    return args


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def oracle_solve(pr, tol):
    """One complete oracle solve of the benchmark workload, timed: FMG with
    tricubic interpolation (Algorithm 2, as the GPU solve), then FAS V(2,2)
    cycles (Algorithm 1) until the relative max-norm residual is <= tol
    (full weighting, 3^3 coarsest grid, ascending 8-colour Gauss-Seidel), on
    the host cores (OpenMP within a colour; OMP_NUM_THREADS sets how many)."""
    from oracle import oracle as O
    u = pr.initial()
    t0 = time.perf_counter()
    info = O.solve(u, pr.f, pr.h, tol=tol, max_cycles=30, params=O.Params(fmg_interp=O.FMG_CUBIC))
    secs = time.perf_counter() - t0
    return {"s": secs, "cycles": info.cycles, "residual": float(info.res_hist[-1]), "cores": O.max_threads()}


def oracle_baseline(pr, tol):
    """cpu_baseline: one measured oracle solve of the same workload (about
    20 s on 16 Grace cores at 257^3)."""
    r = oracle_solve(pr, tol)
    return {"value": pr.unknowns / r["s"], "unit": "unknowns/s", "cores": r["cores"], "kind": "oracle",
            "sample": (f"one complete oracle solve of the {pr.n}^3 workload, measured: tricubic FMG + "
                       f"{r['cycles']} V(2,2) cycles to relative residual {r['residual']:.2e} "
                       f"(tol {tol:g}) in {r['s']:.1f} s on {r['cores']} host threads"),
            "solve_s": r["s"], "cycles": r["cycles"], "residual": r["residual"]}


def workload_config(args, world: int = 1) -> dict:
    """The benchmark's workload description, shared by both arms."""
    return {"workload": f"Example 4 exp(|x|^2/2) {args.n}^3, FMG (tricubic) + FAS V(2,2), 8-colour nonlinear GS, "
                        f"tol {args.tol:g} relative max-norm residual (FP64)",
            "n": args.n, "tol": args.tol,
            "precision": f"mixed: FP32 correction V-cycles x{MIXED_INNER} per FP64 fine residual and update",
            "restrict": "full weighting", "fmg_interpolation": "tricubic",
            "fmg_levels": "mixed outer iterations (FP64 residual, 2 FP32 correction cycles, FP64 update)",
            "parallelism": f"replicas x{world}",
            "l2": "working set larger than L2 (no flush needed)"}


# Wall-clock budget of the reference arm's timed solves: each step is one
# complete oracle solve (about 20 s at 257^3 on 16 cores), so the arm times as
# many of the requested steps as fit, at least one, and reports that count.
REFERENCE_BUDGET_S = 150.0


def run_reference(args):
    """The oracle arm: every timed step is one complete, measured oracle solve
    of the benchmark workload on the host cores.  Warm-up is one solve of the
    same problem on a 33^3 grid (loads the library, faults in its code).
    Steps beyond the time budget are not run; `steps` is the number timed and
    `steps_requested` the number asked for."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_1411_7018_gb300 import problems
    pr = problems.make(args.problem, args.n)
    warm = min(args.warmup, 1)
    for _ in range(warm):
        oracle_solve(problems.make(args.problem, 33), args.tol)
    runs = []
    t0 = time.perf_counter()
    while len(runs) < max(1, args.steps):
        runs.append(oracle_solve(pr, args.tol))
        if time.perf_counter() - t0 + runs[-1]["s"] > REFERENCE_BUDGET_S:
            break
    wall = time.perf_counter() - t0
    ms = 1e3 * statistics.mean(r["s"] for r in runs)
    value = pr.unknowns / (ms / 1e3)
    last = runs[-1]
    sample = (f"{len(runs)} complete oracle solve(s) of the {pr.n}^3 workload, each measured: tricubic FMG + "
              f"{last['cycles']} V(2,2) cycles to relative residual {last['residual']:.2e} (tol {args.tol:g}), "
              f"{ms / 1e3:.1f} s per solve on {last['cores']} host threads")
    line = {"impl": "reference", "metric": "unknowns solved to tolerance per second", "value": value,
            "unit": "unknowns/s", "n_gpus": args.gpus, "steps": len(runs), "warmup": warm,
            "steps_requested": args.steps, "warmup_requested": args.warmup,
            "steps_note": (f"each step is one complete solve (~{ms / 1e3:.0f} s); the steps that fit a "
                           f"{REFERENCE_BUDGET_S:.0f} s budget were timed"),
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": workload_config(args),
            "cpu_baseline": {"value": value, "unit": "unknowns/s", "cores": last["cores"], "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "unknowns/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "cycles_per_solve": last["cycles"], "residual": last["residual"],
            "solve_s": [r["s"] for r in runs], "wall_s": wall}
    print(json.dumps(line), flush=True)


def _timed_solve(H, torch, stream, **kw):
    """One solve of a resident hierarchy timed with CUDA events on its stream."""
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    r = H.solve(**kw)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), r


def bench_paper_mode(args, M, problems, dev):
    """Section 4's configuration (one FMG pass with tricubic interpolation,
    h0 = 1/2 with one sweep, stop at a 1e-6 discrete-L2 reduction against the
    initial residual) on Example 4 at 129^3 and 257^3: iterations, time and
    max-norm error beside Table 3's (the paper's N = 128 row; N = 256 is beyond
    the table)."""
    import torch
    stream = torch.cuda.current_stream(dev)
    out = {"config": "paper: tricubic FMG, 3^3 one sweep, 1e-6 L2 reduction vs initial residual, FW, 8 colours",
           "table3_n128": {"error": 6.2e-06, "iter": 1, "cpu_s_matlab_laptop": 136.9}}
    for n in (129, 257):
        f, g, length = problems.make_on_device("exp", n, device=dev)
        u_ex = g.clone()
        pr = problems.make("exp", n)
        u_ex.copy_(torch.from_numpy(pr.u))
        for prec, key in ((M.MA_FP64, "fp64"), (M.MA_MIXED, "mixed")):
            H = M.Hierarchy(M.paper_desc(n, length=length, precision=prec), device=dev)
            times = []
            for _ in range(3):
                H.set_rhs_bc(f, g)
                ms, r = _timed_solve(H, torch, stream, tol=1e-6, norm=M.MA_NORM_L2, relative=M.MA_REL_INITIAL,
                                     max_cycles=30)
                times.append(ms)
            u = torch.empty_like(f)
            H.get_solution(u)
            H.close()
            out[f"{key}_{n}"] = {"ms": min(times), "iter": r.cycles + 1, "relres": r.res,
                                 "error": (u - u_ex).abs().max().item(),
                                 "unknowns_per_s": (n - 2) ** 3 / (min(times) / 1e3)}
        del f, g, u_ex
        torch.cuda.empty_cache()
    return out


def bench_fp32_mode(args, M, problems, dev):
    """The full-FP32 mode on Example 4 at 129^3 and 257^3: time, the FP32
    residual floor it stops at, and its error against the exact solution and
    against the FP64 discrete solution (the round-off floor per N)."""
    import torch
    stream = torch.cuda.current_stream(dev)
    out = {"mode": "FP32 FAS cycles on the solution, stop at the FP32 residual floor (2 stagnant cycles)"}
    for n in (129, 257):
        f, g, length = problems.make_on_device("exp", n, device=dev)
        u_ex = torch.from_numpy(problems.make("exp", n).u).to(dev)
        res = {}
        for prec, key in ((M.MA_FP64, "fp64"), (M.MA_FP32, "fp32")):
            H = M.Hierarchy(M.make_desc(n, length=length, precision=prec), device=dev)
            ts = []
            for _ in range(3):
                H.set_rhs_bc(f, g)
                ms, r = _timed_solve(H, torch, stream, tol=1e-10 if prec == M.MA_FP64 else 1e-12, max_cycles=40,
                                     raise_on_error=False)
                ts.append(ms)
            u = torch.empty_like(f)
            H.get_solution(u)
            H.close()
            res[key] = (u, r, min(ts))
        u32, r32, ms32 = res["fp32"]
        umax = u_ex.abs().max().item()
        out[str(n)] = {"ms": ms32, "unknowns_per_s": (n - 2) ** 3 / (ms32 / 1e3), "cycles": r32.cycles,
                       "residual_floor": r32.res, "error_vs_exact": (u32 - u_ex).abs().max().item(),
                       "fp64_error_vs_exact": (res["fp64"][0] - u_ex).abs().max().item(),
                       "rel_diff_vs_fp64_solution": (u32 - res["fp64"][0]).abs().max().item() / umax,
                       "fp64_ms": res["fp64"][2]}
        del f, g, u_ex, res, u32
        torch.cuda.empty_cache()
    return out


def bench_2d(args, M, problems, dev):
    """The 2D version (Section 4.1): Example 1 at N = 8192 in Section 4's
    configuration (red-black smoother, bicubic FMG), against Table 1's row
    (error 1.0e-9, one iteration; 67.1 s in MATLAB on a laptop, context only)."""
    import torch
    from paper_1411_7018_gb300 import problems2d as P2
    stream = torch.cuda.current_stream(dev)
    n = 8193
    u_ex, f, g = P2.make2d_on_device("ex1", n, device=dev)
    H = M.Hierarchy2D(M.paper_desc2d(n), device=dev)
    times = []
    for _ in range(3):
        H.set_rhs_bc(f, g)
        ms, r = _timed_solve(H, torch, stream, tol=1e-6, norm=M.MA_NORM_L2, relative=M.MA_REL_INITIAL,
                             max_cycles=30)
        times.append(ms)
    u = torch.empty_like(f)
    H.get_solution(u)
    err = (u - u_ex).abs().max().item()
    H.close()
    return {"workload": "Example 1 (2D) N = 8192, paper configuration, red-black", "ms": min(times),
            "unknowns_per_s": (n - 2) ** 2 / (min(times) / 1e3), "iter": r.cycles + 1, "error": err,
            "table1": {"error": 1.0e-9, "iter": 1, "cpu_s_matlab_laptop": 67.1}}


def bench_precision(args, M, problems, dev):
    """The precision workload at full size: 257^3 and 513^3, the three seeded
    exact solutions (Example 4, |x|^2/2, random cosine), mixed precision and
    plain FP64 to the same tolerance; per case the solve time, unknowns/s,
    cycles, final residual, max-norm error against the exact solution, and
    the mixed-vs-FP64 difference relative to max|u| (the FP64 GPU path is the
    FP64 solution the oracle pins at smaller sizes)."""
    import torch
    stream = torch.cuda.current_stream(dev)
    out = {"tol": args.tol, "timing": "one solve after one warm-up solve, CUDA events on the solve stream"}
    for n in (257, 513):
        for name in ("exp", "quadratic", "cosine"):
            f, g, length, u_ex = problems.make_on_device(name, n, device=dev, exact=True)
            unknowns = (n - 2) ** 3
            row, sols = {}, {}
            for prec, key in ((M.MA_MIXED, "mixed"), (M.MA_FP64, "fp64")):
                H = M.Hierarchy(M.make_desc(n, length=length, precision=prec, inner_cycles=MIXED_INNER),
                                device=dev)
                for _ in range(2):
                    H.set_rhs_bc(f, g)
                    ms, r = _timed_solve(H, torch, stream, tol=args.tol, max_cycles=60, raise_on_error=False)
                u = torch.empty_like(f)
                H.get_solution(u)
                H.close()
                sols[key] = u
                row[key] = {"ms": ms, "unknowns_per_s": unknowns / (ms / 1e3), "cycles": r.cycles,
                            "residual": r.res, "status": r.status, "floor_reached": r.floor_reached,
                            "max_err_vs_exact": float((u - u_ex).abs().max())}
            row["mixed_vs_fp64_speed"] = row["fp64"]["ms"] / row["mixed"]["ms"]
            row["max_rel_diff_mixed_vs_fp64"] = float((sols["mixed"] - sols["fp64"]).abs().max() / u_ex.abs().max())
            out[f"{name}_{n}"] = row
            del f, g, u_ex, sols
            torch.cuda.empty_cache()
    return out


def bench_batching(args, M, problems, dev):
    """64 instances, sizes drawn by seed from {33, 65, 129}^3, each |x|^2/2
    plus seeded cosine modes with amplitude drawn from [0.005, 0.02]; mixed
    precision; solved together as a shared per-level batch (ma_batch_run: one
    launch per kernel and level depth over all instances, an outer iteration
    of all of them as one CUDA graph), with ma_batch_solve (each hierarchy's
    own cycle graphs on its own stream, overlapping), and one at a time."""
    import numpy as np
    import torch
    rng = np.random.default_rng(2024)
    sizes = rng.choice([33, 65, 129], size=64)
    hs, keep = [], []
    for b, n in enumerate(sizes):
        f, g, _ = problems.make_on_device("cosine", int(n), seed=1000 + b, eps=(0.005, 0.02), device=dev)
        H = M.Hierarchy(M.make_desc(int(n), precision=M.MA_MIXED), stream=torch.cuda.Stream(device=dev),
                        device=dev)
        torch.cuda.synchronize()
        H.set_rhs_bc(f, g)
        hs.append(H)
        keep.append((f, g))
    opts = M.ma_solve_opts(args.tol, M.MA_NORM_MAX, 1, 60, M.MA_INIT_FMG)
    handles = [H.handle for H in hs]
    M.ma_batch_solve(handles, opts)            # warm-up: graph capture
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = M.ma_batch_solve(handles, opts, raise_on_error=False)
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    t0 = time.perf_counter()
    for H in hs:
        M.ma_solve(H.handle, opts, raise_on_error=False)
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    B = M.Batch(hs, device=dev)   # default grouping: 2 concurrently replayed groups
    B.solve(tol=args.tol, max_cycles=60, raise_on_error=False)   # warm-up: graph capture
    torch.cuda.synchronize()
    l0 = M.ma_kernel_launch_count()
    t0 = time.perf_counter()
    res_l = B.solve(tol=args.tol, max_cycles=60, raise_on_error=False)
    torch.cuda.synchronize()
    t_levels = time.perf_counter() - t0
    launches_levels = M.ma_kernel_launch_count() - l0
    B.close()
    unknowns = int(sum((int(n) - 2) ** 3 for n in sizes))
    for H in hs:
        H.close()
    # the persistent alternative to the shared batch's launch chains: per
    # phase, a launch edge in a CUDA graph against a grid barrier in one
    # cooperative kernel (ma_probe_phase_chain), at a small and a large phase
    chain = {}
    for n_el in (1 << 16, 1 << 21):
        a = torch.zeros(n_el, dtype=torch.float32, device=dev)
        b = torch.zeros_like(a)
        sync = torch.zeros(4, dtype=torch.int32, device=dev)
        chain[str(n_el)] = M.ma_probe_phase_chain(a, b, sync, phases=64, blocks_per_sm=4)
        del a, b, sync
    return {"instances": 64, "sizes": {str(k): int((sizes == k).sum()) for k in (33, 65, 129)},
            "unknowns": unknowns, "tol": args.tol, "precision": "mixed",
            "ms": t_levels * 1e3, "unknowns_per_s": unknowns / t_levels,
            "mode": "shared per-level launches (ma_batch_run)", "kernel_launches": launches_levels,
            "converged": int(sum(1 for r in res_l if r.status == 0)),
            "concurrent_graphs_ms": t_batch * 1e3, "concurrent_graphs_unknowns_per_s": unknowns / t_batch,
            "concurrent_graphs_converged": int(sum(1 for r in res if r.status == 0)),
            "sequential_ms": t_seq * 1e3, "sequential_unknowns_per_s": unknowns / t_seq,
            "speedup_vs_sequential": t_seq / t_levels,
            "persistent_phase_chain_us_per_phase": chain}


def bench_serving(args, M, problems, dev):
    """Poisson arrivals (seeded, 200 req/s offered) of solves with sizes drawn
    from {65, 129, 257}^3, |x|^2/2 plus seeded cosine modes, tol 1e-8
    relative: continuous batching of mixed-precision solves versus FP64 solves
    served one at a time, on the same request stream.  Latency = completion -
    arrival (queueing included); the first requests that build the resident
    hierarchies and capture their graphs are not counted."""
    import numpy as np
    import torch
    from paper_1411_7018_gb300 import serve
    sizes = (65, 129, 257)
    keys = 2
    inputs = {}
    for n in sizes:
        for k in range(keys):
            inputs[(n, k)] = problems.make_on_device("cosine", n, seed=500 + 10 * n + k, eps=(0.005, 0.02),
                                                     device=dev)
    torch.cuda.synchronize()
    out = {"offered_req_s": 200.0, "sizes": list(sizes), "tol": 1e-8,
           "note": "the *_60 runs offer 60 req/s to both arms with the same requests (the latency comparison); "
                   "200 req/s of this size mix exceeds one GPU's capacity, so latency there is mostly queueing"}
    # the 60 req/s pair is the latency comparison (both arms serve the same
    # requests); at 200 req/s the FP64 arm is far beyond its capacity, so it
    # serves a shorter prefix of the stream and its latency is queueing
    runs = (("mixed_continuous_60", M.MA_MIXED, max(100, args.serve_requests // 2), 32, 60.0),
            ("fp64_one_at_a_time_60", M.MA_FP64, max(100, args.serve_requests // 2), 1, 60.0),
            ("mixed_continuous", M.MA_MIXED, args.serve_requests, 32, 200.0),
            ("fp64_one_at_a_time", M.MA_FP64, max(50, args.serve_requests // 8), 1, 200.0))
    for label, precision, count, max_active, rate in runs:
        be = serve.LibmaBackend(precision, inputs, device=dev)
        srv = serve.Server(be, hbm_budget=48 << 30, max_active=max_active)
        warm = [serve.Request(rid=-1 - i, n=n, arrival=0.0, key=(n, 0), tol=1e-8)
                for i, n in enumerate(sizes * 2)]
        srv.run(warm)
        reqs = serve.poisson_stream(count, rate, sizes, keys, seed=77, tol=1e-8)
        t0 = time.perf_counter()
        done = srv.run(reqs)
        wall = time.perf_counter() - t0
        srv.close()
        summ = serve.summarize(done, wall)
        summ["max_active"] = max_active
        summ["offered_req_s"] = rate
        out[label] = summ
    out["unknowns_per_s_mixed_vs_fp64"] = (out["mixed_continuous"]["unknowns_per_s"]
                                          / out["fp64_one_at_a_time"]["unknowns_per_s"])
    out["latency_60_req_s"] = {k: {q: out[f"{k}_60"][q] for q in ("requests", "p50_ms", "p99_ms", "unknowns_per_s")}
                               for k in ("mixed_continuous", "fp64_one_at_a_time")}
    return out


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1411_7018_gb300 import libma as M
    from paper_1411_7018_gb300 import problems, replicas

    rank, local, world = replicas.rank_info()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    # autotune the correction smoother and residual variants for every grid size
    # the workloads use (before any hierarchy records its graphs)
    tune_sizes = set(M.level_sizes(args.n)) | set(M.level_sizes(129)) | set(M.level_sizes(257)) | {513}
    tuning = M.autotune(sorted(tune_sizes), reps=5, device=dev)

    pr = problems.make(args.problem, args.n)
    f_dev = torch.from_numpy(pr.f).to(dev)
    g_dev = torch.from_numpy(pr.initial()).to(dev)
    hier = {"mixed": M.Hierarchy(M.make_desc(pr.n, length=pr.length, precision=M.MA_MIXED,
                                             inner_cycles=MIXED_INNER), device=dev),
            "fp64": M.Hierarchy(M.make_desc(pr.n, length=pr.length, precision=M.MA_FP64), device=dev)}

    def step(H):
        H.set_rhs_bc(f_dev, g_dev)
        r = H.solve(tol=args.tol, max_cycles=60)
        return r

    def timed(H, steps):
        """CUDA-event time per solve on the solve stream (max over ranks)."""
        for _ in range(args.warmup):
            step(H)
        torch.cuda.synchronize()
        replicas.barrier()
        l0 = M.ma_kernel_launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        cyc = []
        for _ in range(steps):
            r = step(H)
            cyc.append(r.cycles)
        e1.record(stream)
        torch.cuda.synchronize()
        launches = M.ma_kernel_launch_count() - l0
        ms = replicas.max_over_ranks(e0.elapsed_time(e1) / steps, device=dev)
        replicas.barrier()
        return ms, statistics.mean(cyc), r, launches

    sampler = ClockSampler(local)
    sampler.start()
    ms_mixed, cyc_mixed, res_mixed, launches = timed(hier["mixed"], args.steps)
    clocks = sampler.stop()
    ms_fp64, cyc_fp64, res_fp64, _ = timed(hier["fp64"], max(1, args.steps // 2))
    value = replicas.whole_job_rate(pr.unknowns, ms_mixed / 1e3, world)
    sols = {}
    for k, H in hier.items():
        u = torch.empty_like(f_dev)
        H.get_solution(u)
        sols[k] = u.cpu().numpy()
    torch.cuda.synchronize()
    err = {k: float(np.max(np.abs(v - pr.u))) for k, v in sols.items()}
    diff = float(np.max(np.abs(sols["mixed"] - sols["fp64"])) / np.max(np.abs(pr.u)))

    # live kernel timings on the solve stream, same grid: the FP32 correction
    # smoother (one colour phase) and the FP64 smoother
    n, h = pr.n, pr.h
    u64 = torch.from_numpy(sols["mixed"]).to(dev)
    hi = u64.float()
    lo = (u64 - hi.double()).float()
    e = torch.zeros_like(hi)
    rhs = (1e-8 * f_dev).float()
    rhs[0], rhs[-1] = 0, 0
    _keep, scr, nb = M.correction_scratch(n, device=dev)
    M.ma_smooth_correction(e, hi, lo, rhs, n, h, 1, scr, nb)
    sweeps = 4
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    M.ma_smooth_correction(e, hi, lo, rhs, n, h, sweeps, scr, nb)
    e1.record(stream)
    torch.cuda.synchronize()
    # the call also runs the base-Hessian and layout kernels; time them alone and subtract
    b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    b0.record(stream)
    M.ma_smooth_correction(e, hi, lo, rhs, n, h, 0, scr, nb)
    b1.record(stream)
    torch.cuda.synchronize()
    stream_sweeps_ms = e0.elapsed_time(e1) - b0.elapsed_time(b1)

    def graph_ms(nsw, reps=5):
        """Median time of one replay of a CUDA graph holding the call with nsw
        sweeps: the form in which the solve runs its sweeps."""
        cap = torch.cuda.Stream(device=dev)
        with torch.cuda.stream(cap):
            M.ma_smooth_correction(e, hi, lo, rhs, n, h, nsw, scr, nb)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=cap):
            M.ma_smooth_correction(e, hi, lo, rhs, n, h, nsw, scr, nb)
        torch.cuda.synchronize()
        cs = torch.cuda.current_stream()
        ts = []
        for r in range(reps + 1):
            g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            g0.record(cs)
            g.replay()
            g1.record(cs)
            torch.cuda.synchronize()
            if r:
                ts.append(g0.elapsed_time(g1))
        del g
        return sorted(ts)[len(ts) // 2]

    graph_sweeps = 8
    graph_sweeps_ms = graph_ms(graph_sweeps) - graph_ms(0)
    # the variant in force at this size: by colour (8 launches per sweep, an
    # eighth of the points each), colour pairs (4 launches, a quarter each) or
    # by k parity (2 launches, half the points)
    corr_choice = M.ma_get_corr_tuning(n)[0]
    corr_launches = {M.MA_CORR_BY_COLOUR: 8, M.MA_CORR_PAIRS: 4}.get(corr_choice, 2)
    corr_kernel = {8: "k_smooth_corr (FP32 correction smoother, one colour phase)",
                   4: "k_smooth_corr_pair (FP32 correction smoother, colours c and c^7 in one launch)"}.get(
        corr_launches, f"k_smooth_corr_plane (FP32 correction smoother, {M.CORR_NAMES[corr_choice]}, one k-parity "
                       f"phase: four colours)")
    # the roofline kernel's launch time as the solve runs it (graph replays);
    # the stream-launched figure is reported beside it
    corr_launch_ms = graph_sweeps_ms / (corr_launches * graph_sweeps)
    corr_launch_ms_stream = stream_sweeps_ms / (corr_launches * sweeps)
    corr_gbs = CORR_SMOOTH_BYTES_PER_POINT * ((n - 2) ** 3 / corr_launches) / (corr_launch_ms / 1e3) / 1e9
    pts_launch = (n - 2) ** 3 / 8.0
    u_tmp = u64.clone()
    M.ma_smooth(u_tmp, f_dev, n, h, 1)
    e0.record(stream)
    M.ma_smooth(u_tmp, f_dev, n, h, sweeps)
    e1.record(stream)
    torch.cuda.synchronize()
    f64_launch_ms = e0.elapsed_time(e1) / (8 * sweeps)
    f64_gops = SMOOTH_FP64_OPS_PER_POINT * pts_launch / (f64_launch_ms / 1e3) / 1e9
    # the FP64 peak, measured on this GPU: independent DFMA chains on every SM
    fp64_peak_gops = max(M.ma_probe_fp64_rate() for _ in range(3)) / 1e9
    del u_tmp, hi, lo, e, rhs, _keep

    # V-cycles per second on the resident 257^3 hierarchies: an FP64 FAS
    # V-cycle, and an FP32 correction V-cycle (an outer iteration of the
    # mixed solve is inner_cycles of them plus the FP64 residual and update)
    vc = {}
    for key in ("fp64", "mixed"):
        H = hier[key]
        H.set_rhs_bc(f_dev, g_dev)
        H.solve(tol=args.tol, max_cycles=60)
        H.vcycle(1)
        e0.record(stream)
        H.vcycle(3)
        e1.record(stream)
        torch.cuda.synchronize()
        per = e0.elapsed_time(e1) / 3.0
        inner = MIXED_INNER if key == "mixed" else 1
        vc[key] = {"ms_per_cycle": per / inner, "vcycles_per_s": 1e3 * inner / per}

    # end to end through the C ABI with host buffers (pinned), mixed precision.
    # Two resident hierarchies, each on its own stream, take the steps in
    # turn.  While the main thread solves step k on one of them (ma_solve
    # blocks), a second host thread reads step k-1's solution out of the other
    # and uploads step k+1's f and g into it (ma_get_solution_host, then
    # ma_set_rhs_bc_host, in that order on that hierarchy's stream), so the
    # host-link copies run beside the solve.  One solve runs at a time.  Every
    # step's copies lie inside the timed region: it opens before step 0's
    # upload and closes after the last step's download.
    from concurrent.futures import ThreadPoolExecutor
    e2e_h = [M.Hierarchy(M.make_desc(pr.n, length=pr.length, precision=M.MA_MIXED, inner_cycles=MIXED_INNER),
                         stream=torch.cuda.Stream(device=dev), device=dev) for _ in range(2)]
    f_host = torch.from_numpy(pr.f).pin_memory()
    g_host = torch.from_numpy(pr.initial()).pin_memory()
    u_host = [torch.empty_like(f_host).pin_memory() for _ in range(2)]
    e2e_steps = max(2, min(args.steps, 10))
    e2e_res = []

    def e2e_run(steps):
        with ThreadPoolExecutor(max_workers=1) as io:
            e2e_h[0].set_rhs_bc_host(f_host, g_host)
            pending = None
            for k in range(steps):
                H, other = e2e_h[k % 2], e2e_h[(k + 1) % 2]
                if pending is not None:
                    pending.result()          # step k's inputs are in H

                def io_job(k=k, other=other):
                    if k >= 1:
                        other.get_solution_host(u_host[(k - 1) % 2])   # step k-1's result
                    if k + 1 < steps:
                        other.set_rhs_bc_host(f_host, g_host)          # step k+1's inputs

                pending = io.submit(io_job)
                e2e_res.append(H.solve(tol=args.tol, max_cycles=60))
            pending.result()
            e2e_h[(steps - 1) % 2].get_solution_host(u_host[(steps - 1) % 2])

    e2e_run(2)   # warm-up: graph capture on both hierarchies, first use of the pinned buffers
    torch.cuda.synchronize()
    e2e_res.clear()
    t0 = time.perf_counter()
    e2e_run(e2e_steps)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e_ok = all(r.status == 0 and r.cycles == e2e_res[0].cycles for r in e2e_res)
    u_check = torch.empty_like(f_dev)
    e2e_h[(e2e_steps - 1) % 2].get_solution(u_check)
    torch.cuda.synchronize()
    e2e_same = bool(torch.equal(u_check.cpu(), u_host[(e2e_steps - 1) % 2]))
    for H in e2e_h:
        H.close()
    del e2e_h, u_check

    for H in hier.values():
        H.close()
    del hier
    torch.cuda.empty_cache()
    extras = {}
    if world == 1:
        for name, fn in (("precision", bench_precision), ("batching", bench_batching), ("serving", bench_serving),
                         ("paper_mode", bench_paper_mode), ("two_d", bench_2d), ("fp32_mode", bench_fp32_mode)):
            try:
                extras[name] = fn(args, M, problems, dev)
            except Exception as exc:   # reported, not fatal: the headline line still prints
                extras[name] = {"error": f"{type(exc).__name__}: {exc}"}
            torch.cuda.empty_cache()
    cpu = oracle_baseline(pr, args.tol) if (rank == 0 and world == 1) else None
    peak_gbs, peak_src = hbm_peak()
    if rank == 0:
        line = {
            "metric": "unknowns solved to tolerance per second",
            "value": value, "unit": "unknowns/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_mixed, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": workload_config(args, world),
            "cycles_per_solve": cyc_mixed, "residual": res_mixed.res,
            "fp64": {"value": world * pr.unknowns / (ms_fp64 / 1e3), "unit": "unknowns/s",
                     "ms_per_step": ms_fp64, "cycles_per_solve": cyc_fp64, "residual": res_fp64.res},
            "mixed_vs_fp64": ms_fp64 / ms_mixed,
            "accuracy": {"max_err_vs_exact_mixed": err["mixed"], "max_err_vs_exact_fp64": err["fp64"],
                         "max_rel_diff_mixed_vs_fp64": diff},
            "roofline": {"bound": "hbm", "kernel": corr_kernel,
                         "achieved": corr_gbs, "peak": peak_gbs, "unit": "GB/s",
                         "frac": corr_gbs / peak_gbs,
                         "traffic": CORR_SMOOTH_TRAFFIC_257.get(corr_choice) if n == 257 else None,
                         "traffic_note": (f"ncu dram bytes per launch, warm L2; algorithmic 36 B x (n-2)^3/"
                                          f"{corr_launches} = {36 * (n - 2) ** 3 / corr_launches / 1e6:.0f} MB"),
                         "launch_ms": corr_launch_ms,
                         "launch_timing": f"CUDA events around replays of a CUDA graph of {graph_sweeps} sweeps "
                                          f"(the form the solve runs), median of 5, minus the same graph with none",
                         "launch_ms_stream_launched": corr_launch_ms_stream,
                         "bytes_per_point": CORR_SMOOTH_BYTES_PER_POINT,
                         "peak_source": peak_src},
            "roofline_fp64_smoother": {"bound": "alu", "kernel": "k_smooth_colour (FP64 smoother, one colour phase)",
                                       "achieved": f64_gops, "peak": fp64_peak_gops, "unit": "GFP64op/s",
                                       "frac": f64_gops / fp64_peak_gops, "launch_ms": f64_launch_ms,
                                       "ops_per_point": SMOOTH_FP64_OPS_PER_POINT,
                                       "peak_source": "measured: ma_probe_fp64_rate (DFMA chains on every SM, "
                                                      "CUDA events), best of 3",
                                       "nominal_peak": FP64_NOMINAL_GOPS},
            "cpu_baseline": {k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample")} if cpu else None,
            "e2e": {"value": world * pr.unknowns / e2e_s, "unit": "unknowns/s",
                    "h2d_bytes_per_step": 2 * 8 * pr.n ** 3, "d2h_bytes_per_step": 8 * pr.n ** 3,
                    "steps": e2e_steps, "ms_per_step": 1e3 * e2e_s, "converged_all": e2e_ok,
                    "solution_read_matches_device": e2e_same,
                    "mode": "ma_set_rhs_bc_host / ma_solve / ma_get_solution_host on pinned buffers; "
                            "2 resident hierarchies in turn, a host thread moving step k-1's solution out "
                            "and step k+1's inputs in while step k solves; one solve at a time"},
            "clocks": clocks,
            "gpu_launches": launches,
            "vcycles": {"fp64_fas_vcycle": vc["fp64"],
                        "fp32_correction_vcycle_with_fp64_update_share": vc["mixed"]},
            "tuning": {str(k): {"smoother": v["smoother"], "residual": v["residual"],
                                "us_per_sweep": v["us_per_sweep"]} for k, v in tuning.items()},
            **extras,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
