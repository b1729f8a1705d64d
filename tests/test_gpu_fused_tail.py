"""The fused tail of the FP64 V-cycle (Algorithm 1): the levels with n <= 9
(or 17, or 5) run as one single-block launch with the arithmetic of the
separate kernels,
so every solve that runs FP64 cycles -- FP64 solves, the paper's FMG
configuration, FMG below the finest level of the mixed-precision solve --
gives the same bits and cycle count with the tail fused or level by level,
in fewer kernel launches.
"""
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


TAILS = (17, 9, 5, 0)   # largest fused level; 0: level by level


def _runs(desc_fn, name, n, solve_kw, vcycles=0):
    """Runs the same solve for each tail size of TAILS; returns
    [(u, cycles, res, launches)] in that order."""
    pr = P.make(name, n)
    outs = []
    try:
        for max_n in TAILS:
            M.ma_set_vcycle_tail(max_n)
            H = M.Hierarchy(desc_fn(pr))
            H.set_rhs_bc(dev(pr.f), dev(pr.initial()))
            torch.cuda.synchronize()
            c0 = M.ma_kernel_launch_count()
            if vcycles:
                H.vcycle(vcycles)
                cycles, res = vcycles, 0.0
            else:
                r = H.solve(raise_on_error=False, **solve_kw)
                cycles, res = r.cycles, r.res
            u = torch.empty_like(dev(pr.f))
            H.get_solution(u)
            launches = M.ma_kernel_launch_count() - c0
            outs.append((host(u), cycles, res, launches))
            H.close()
    finally:
        M.ma_set_vcycle_tail(True)
    return outs


def _same_bits(outs):
    u0, c0, r0, _ = outs[-1]
    for u, c, r, _ in outs[:-1]:
        assert c == c0 and r == r0
        assert np.array_equal(u, u0)


def _fewer_launches(outs, coarsest):
    """A tail spanning two or more levels replaces their launches by one."""
    separate = outs[-1][3]
    for max_n, (_, _, _, launches) in zip(TAILS[:-1], outs[:-1]):
        assert launches < separate if max_n > coarsest else launches == separate


@pytest.mark.parametrize("name,n,coarsest", [("exp", 65, 3), ("cosine", 17, 3), ("exp", 33, 5), ("sine", 129, 3),
                                             ("exp", 9, 3), ("cosine", 33, 17)])
def test_fp64_fused_tail_is_bitwise_the_level_by_level_solve(name, n, coarsest):
    outs = _runs(lambda pr: M.make_desc(n, length=pr.length, coarsest_n=coarsest), name, n,
                 dict(tol=1e-12, max_cycles=40))
    _same_bits(outs)
    _fewer_launches(outs, coarsest)


@pytest.mark.parametrize("name,n", [("exp", 33), ("ex6", 33), ("sine", 65)])
def test_fp64_fused_tail_bitwise_in_the_paper_configuration(name, n):
    """Tricubic FMG, 3^3 coarsest grid with one sweep, the relative-L2 stop of
    Section 4: FMG runs a V-cycle from every level, all through the tail on
    the levels up to 17^3."""
    outs = _runs(lambda pr: M.paper_desc(n, length=pr.length), name, n,
                 dict(tol=1e-6, norm=M.MA_NORM_L2, relative=M.MA_REL_INITIAL, max_cycles=30))
    _same_bits(outs)
    _fewer_launches(outs, 3)


@pytest.mark.parametrize("precision", [M.MA_MIXED, M.MA_FP32])
def test_fused_fp64_tail_bitwise_under_the_other_precisions(precision):
    """Neither the mixed solve (its FMG levels run FP32 correction cycles)
    nor the FP32 mode runs an FP64 V-cycle: the switch must not change
    anything there."""
    outs = _runs(lambda pr: M.make_desc(65, length=pr.length, precision=precision), "exp", 65,
                 dict(tol=1e-10 if precision == M.MA_MIXED else 1e-5, max_cycles=40))
    _same_bits(outs)


def test_fp64_fused_tail_bitwise_for_plain_vcycles_with_half_weighting():
    """ma_vcycle from the Dirichlet data, half weighting with injected
    approximation, V(1,3), a fixed count of coarsest sweeps."""
    outs = _runs(lambda pr: M.make_desc(33, length=pr.length, nu1=1, nu2=3, restrict_kind=M.MA_HALF_WEIGHTING,
                                        approx_restrict=M.MA_APPROX_INJECTION, coarse_sweeps=4),
                 "exp", 33, {}, vcycles=3)
    _same_bits(outs)
    _fewer_launches(outs, 3)


def test_tail_sizes_outside_the_level_sizes_are_refused():
    for bad in (2, 4, 7, 33, -1):
        with pytest.raises(M.MAError):
            M.ma_set_vcycle_tail(bad)
        with pytest.raises(M.MAError):
            M.ma_set_corr_tail(bad)
    assert M.ma_set_vcycle_tail(True) is None and M.ma_set_corr_tail(True) is None
