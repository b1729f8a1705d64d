"""Run one piece of the solver on a benchmark-shaped grid, for profiler captures.

    python -m paper_1411_7018_gb300.profile_case --case smooth --n 257 --reps 2

Cases: ``smooth`` (FP64 smoother sweeps, 8 colour launches each), ``residual``
(the FP64 residual kernel), ``residual_f2`` (the mixed solve's fine residual:
exact integer differences, two-float determinant), ``smooth_corr`` (FP32 correction-smoother sweeps of
the mixed path on a small correction, in the variant the tuning table picks for
n or the one --smoother names), ``residual_corr`` (the correction residual
rhs - N(e) of the mixed path on that correction, in the variant the tuning
table picks for n or the one --residual names), ``vcycle`` (whole V-cycles of
a resident hierarchy), ``solve`` (one FMG + V-cycle solve to 1e-10), ``solve2d`` (the 2D paper-configuration solve of
Example 1 on an n x n grid), ``smooth2d`` (2D red-black sweeps on that grid),
``batch`` (the batching workload: 64 mixed-precision instances of sizes drawn
by seed from {33, 65, 129}^3, solved once as a shared per-level batch),
``batch_graphs`` (the same instances solved with ma_batch_solve: each
hierarchy's own graphs on its own stream);
``--precision mixed`` runs the hierarchy cases in mixed precision.  The grid holds
Example 4 (u = exp(|x|^2/2)) with a small seeded perturbation; fields of a
257^3 grid are 136 MB each, larger than L2.  Prints nothing but a one-line
summary; it measures nothing itself.
"""
from __future__ import annotations

import argparse

import numpy as np
import torch

from . import libma as M
from . import problems


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", choices=["smooth", "residual", "residual_f2", "smooth_corr", "residual_corr", "vcycle",
                                       "solve", "solve2d", "smooth2d", "batch", "batch_graphs"], default="smooth")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="fp64")
    ap.add_argument("--n", type=int, default=257)
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--problem", default="exp")
    ap.add_argument("--inner", type=int, default=0,
                    help="FP32 correction cycles per outer iteration of a mixed hierarchy (0: library default)")
    variants = {name: c for c, name in M.CORR_NAMES.items()}
    ap.add_argument("--smoother", choices=["by_colour", "colour_pairs", "plane16", "plane32", "plane64"], default=None,
                    help="correction-smoother variant for grid size n (default: the tuning table's)")
    ap.add_argument("--residual", choices=["column", "plane16", "plane32", "plane64"], default=None,
                    help="correction-residual variant for grid size n (default: the tuning table's)")
    a = ap.parse_args()
    if a.smoother or a.residual:
        M.ma_set_corr_tuning(a.n, variants[a.smoother] if a.smoother else -1,
                             variants[a.residual] if a.residual else -1)
    if a.case == "smooth2d":
        from . import problems2d
        u_ex, f2, g2 = problems2d.make2d_on_device("ex1", a.n)
        u2 = u_ex.clone()
        t2 = torch.empty_like(u2)
        for _ in range(a.reps):
            M.ma2d_smooth(u2, f2, a.n, 1.0 / (a.n - 1), 1, M.MA2D_REDBLACK, t2)
        torch.cuda.synchronize()
        print(f"profile_case {a.case} n={a.n} reps={a.reps} done")
        return
    if a.case in ("batch", "batch_graphs"):
        rng = np.random.default_rng(2024)
        sizes = rng.choice([33, 65, 129], size=64)
        hs, keep = [], []
        for b, n in enumerate(sizes):
            f, g, _ = problems.make_on_device("cosine", int(n), seed=1000 + b, eps=(0.005, 0.02))
            H = M.Hierarchy(M.make_desc(int(n), precision=M.MA_MIXED), stream=torch.cuda.Stream())
            torch.cuda.synchronize()
            H.set_rhs_bc(f, g)
            hs.append(H)
            keep.append((f, g))
        if a.case == "batch":
            B = M.Batch(hs)
            for _ in range(a.reps):
                B.solve(tol=1e-10, max_cycles=60, raise_on_error=False)
            B.close()
        else:   # each hierarchy's own cycle graphs on its own stream, overlapping
            opts = M.ma_solve_opts(1e-10, M.MA_NORM_MAX, 1, 60, M.MA_INIT_FMG)
            for _ in range(a.reps):
                M.ma_batch_solve([H.handle for H in hs], opts, raise_on_error=False)
        for H in hs:
            H.close()
        torch.cuda.synchronize()
        print(f"profile_case {a.case} reps={a.reps} done")
        return
    if a.case == "solve2d":
        from . import problems2d
        u_ex, f2, g2 = problems2d.make2d_on_device("ex1", a.n)
        H = M.Hierarchy2D(M.paper_desc2d(a.n))
        for _ in range(a.reps):
            H.set_rhs_bc(f2, g2)
            H.solve(tol=1e-6, norm=M.MA_NORM_L2, relative=M.MA_REL_INITIAL, max_cycles=30)
        H.close()
        torch.cuda.synchronize()
        print(f"profile_case {a.case} n={a.n} reps={a.reps} done")
        return
    pr = problems.make(a.problem, a.n)
    rng = np.random.default_rng(0)
    u0 = pr.u.copy()
    u0[1:-1, 1:-1, 1:-1] += 1e-6 * rng.standard_normal((a.n - 2,) * 3)
    u = torch.from_numpy(u0).cuda()
    f = torch.from_numpy(pr.f).cuda()
    if a.case == "smooth":
        for _ in range(a.reps):
            M.ma_smooth(u, f, a.n, pr.h, 1)
    elif a.case == "residual":
        r = torch.empty_like(u)
        for _ in range(a.reps):
            M.ma_residual(u, f, r, a.n, pr.h)
    elif a.case == "residual_f2":
        r = torch.empty_like(u)
        for _ in range(a.reps):
            M.ma_residual_f2(u, f, r, a.n, pr.h)
    elif a.case == "residual_corr":
        hi = u.float()
        lo = (u - hi.double()).float()
        e = (1e-7 * (u - torch.from_numpy(pr.u).cuda())).float()
        res = torch.zeros_like(hi)
        _keep, scr, nb = M.correction_scratch(a.n)
        rhs = (1e-6 * f).float()
        rhs[0], rhs[-1] = 0, 0
        for _ in range(a.reps):
            M.ma_residual_correction(e, hi, lo, rhs, res, a.n, pr.h, scr, nb)
    elif a.case == "smooth_corr":
        hi = u.float()
        lo = (u - hi.double()).float()
        e = torch.zeros_like(hi)
        _keep, scr, nb = M.correction_scratch(a.n)
        rhs = (1e-6 * f).float()
        rhs[0], rhs[-1] = 0, 0
        for _ in range(a.reps):
            M.ma_smooth_correction(e, hi, lo, rhs, a.n, pr.h, 2, scr, nb)
    else:
        prec = M.MA_MIXED if a.precision == "mixed" else M.MA_FP64
        kw = {"inner_cycles": a.inner} if a.inner > 0 else {}
        H = M.Hierarchy(M.make_desc(a.n, length=pr.length, precision=prec, **kw))
        H.set_rhs_bc(f, u)
        if a.case == "vcycle":
            H.vcycle(a.reps)
        else:
            H.solve(tol=1e-10, raise_on_error=False)
        H.close()
    torch.cuda.synchronize()
    print(f"profile_case {a.case} n={a.n} reps={a.reps} done")


if __name__ == "__main__":
    main()
