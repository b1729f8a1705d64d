"""The shared per-level batch (ma_create_batch / ma_batch_run): uneven
hierarchies whose outer iterations run as one launch per kernel and level
depth over all of them.  Each hierarchy executes the per-point operations of
its own solve, so every result -- solution, cycle count, residual, root
events -- must be bitwise the one ma_solve gives for it alone, also when the
hierarchies stop at different cycles (the finished ones are masked) and
whatever the fused-tail bound."""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1411_7018_gb300 import libma as M
from paper_1411_7018_gb300 import problems as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    M.load()


def _problems(spec):
    out = []
    for b, (name, n) in enumerate(spec):
        if name == "cosine":
            out.append(P.make("cosine", n, seed=20 + b, eps=(0.005, 0.02)))
        else:
            out.append(P.make(name, n))
    return out


def _solo(pr, desc_kw, tol, solve_kw):
    H = M.Hierarchy(M.make_desc(pr.n, length=pr.length, precision=M.MA_MIXED, **desc_kw))
    H.set_rhs_bc(torch.from_numpy(pr.f).cuda(), torch.from_numpy(pr.initial()).cuda())
    r = H.solve(tol=tol, max_cycles=40, raise_on_error=False, **solve_kw)
    u = torch.empty(pr.f.shape, dtype=torch.float64, device="cuda")
    H.get_solution(u)
    torch.cuda.synchronize()
    H.close()
    return u.cpu().numpy(), r


def _batched(prs, desc_kw, tol, solve_kw):
    hs, keep = [], []
    for pr in prs:
        H = M.Hierarchy(M.make_desc(pr.n, length=pr.length, precision=M.MA_MIXED, **desc_kw),
                        stream=torch.cuda.Stream())
        f, g = torch.from_numpy(pr.f).cuda(), torch.from_numpy(pr.initial()).cuda()
        torch.cuda.synchronize()
        H.set_rhs_bc(f, g)
        hs.append(H)
        keep += [f, g]
    B = M.Batch(hs)
    c0 = M.ma_kernel_launch_count()
    res = B.solve(tol=tol, max_cycles=40, raise_on_error=False, **solve_kw)
    launches = M.ma_kernel_launch_count() - c0
    sols = []
    for pr, H in zip(prs, hs):
        u = torch.empty(pr.f.shape, dtype=torch.float64, device="cuda")
        H.get_solution(u)
        torch.cuda.synchronize()
        sols.append(u.cpu().numpy())
    B.close()
    for H in hs:
        H.close()
    return sols, res, launches


def _check_same(prs, desc_kw, tol, solve_kw=None):
    solve_kw = solve_kw or {}
    sols, res, launches = _batched(prs, desc_kw, tol, solve_kw)
    cycles = set()
    for pr, u, r in zip(prs, sols, res):
        ref, rr = _solo(pr, desc_kw, tol, solve_kw)
        assert (r.cycles, r.status, r.floor_reached) == (rr.cycles, rr.status, rr.floor_reached)
        assert r.res == rr.res and r.res0 == rr.res0
        assert r.nonconvex_root_events == rr.nonconvex_root_events
        assert np.array_equal(u, ref)
        cycles.add(r.cycles)
    return cycles, launches


def test_uneven_batch_is_bitwise_the_solo_solves():
    spec = [("cosine", 33), ("cosine", 65), ("exp", 33), ("cosine", 129), ("quadratic", 65), ("cosine", 33),
            ("exp", 65), ("sine", 33)]
    cycles, _ = _check_same(_problems(spec), {}, 1e-10)
    # the hierarchies stop at different cycles, so the masking is exercised
    assert len(cycles) > 1


def test_batch_bitwise_with_the_batched_start():
    """The start (norms of f, FMG, first outer iteration) as batched launches
    too: FMG step j on one level size across the hierarchies."""
    spec = [("cosine", 33), ("exp", 65), ("quadratic", 17), ("exp", 129)]
    try:
        M.ma_set_batch_start(True)
        _check_same(_problems(spec), {}, 1e-10)
    finally:
        M.ma_set_batch_start(False)


@pytest.mark.parametrize("groups", [1, 3])
def test_batch_bitwise_for_any_grouping(groups):
    spec = [("cosine", 33), ("exp", 65), ("cosine", 17), ("quadratic", 33), ("exp", 33)]
    try:
        M.ma_set_batch_groups(groups)
        _check_same(_problems(spec), {}, 1e-10)
    finally:
        M.ma_set_batch_groups(2)


@pytest.mark.parametrize("tail", [0, 5, 17])
def test_batch_bitwise_for_every_tail_bound(tail):
    spec = [("cosine", 33), ("exp", 65), ("cosine", 17), ("quadratic", 33)]
    try:
        M.ma_set_corr_tail(tail)
        _check_same(_problems(spec), {}, 1e-10)
    finally:
        M.ma_set_corr_tail(True)


def test_batch_bitwise_with_other_cycle_settings():
    """V(1,3), half weighting with injected approximation, 5^3 coarsest grid
    with four sweeps, two inner cycles.  With half weighting the 33^3 solve
    diverges (many rhs <= 0 root events) while 9^3 and 17^3 converge: the
    batch must reproduce both, root-event counts included."""
    kw = dict(nu1=1, nu2=3, restrict_kind=M.MA_HALF_WEIGHTING, approx_restrict=M.MA_APPROX_INJECTION,
              coarsest_n=5, coarse_sweeps=4, inner_cycles=2)
    spec = [("exp", 17), ("cosine", 33), ("exp", 9)]
    _check_same(_problems(spec), kw, 1e-9)


@pytest.mark.parametrize("relative", [M.MA_REL_RHS, M.MA_REL_INITIAL])
def test_batch_bitwise_in_the_paper_configuration(relative):
    """Tricubic FMG, 3^3 coarsest grid with one sweep, the L2 stopping rule,
    with the batched start: against ||f|| the start runs batched (FMG steps
    aligned by level size), against the initial residual each hierarchy
    starts on its own."""
    kw = dict(coarsest_n=3, coarse_sweeps=1, fmg_interp=M.MA_FMG_CUBIC)
    spec = [("exp", 33), ("ex6", 65), ("sine", 17), ("cosine", 33)]
    try:
        M.ma_set_batch_start(True)
        _check_same(_problems(spec), kw, 1e-8, dict(norm=M.MA_NORM_L2, relative=relative))
    finally:
        M.ma_set_batch_start(False)


def test_batch_rejects_mismatched_hierarchies():
    a = M.Hierarchy(M.make_desc(33, precision=M.MA_MIXED))
    b = M.Hierarchy(M.make_desc(33, precision=M.MA_MIXED, nu1=1))
    c = M.Hierarchy(M.make_desc(33, precision=M.MA_FP64))
    d = M.Hierarchy(M.make_desc(33, precision=M.MA_MIXED, coarsest_n=5))
    try:
        for hs in ([a.handle, b.handle], [a.handle, c.handle], [a.handle, a.handle], [a.handle, d.handle], []):
            with pytest.raises(M.MAError):
                M.ma_batch_footprint(hs)
    finally:
        for H in (a, b, c, d):
            H.close()


def test_batch_with_single_level_and_deep_hierarchies():
    """A 3^3 hierarchy (one unknown: its whole cycle is the coarsest solve in
    the fused tail) and a 5^3 one batched with deeper ones."""
    spec = [("exp", 3), ("cosine", 5), ("exp", 9), ("cosine", 33)]
    for start in (False, True):
        try:
            M.ma_set_batch_start(start)
            _check_same(_problems(spec), {}, 1e-10)
        finally:
            M.ma_set_batch_start(False)
