"""GPU parity of the mixed-precision path (FP32 correction cycles under an FP64
residual and update) against the FP64 CPU oracle.

The correction operator N(e) = det(D^2_h(u + e)) - det(D^2_h u) has a plain
definition, so its oracle is two FP64 oracle evaluations of the discrete
Monge-Ampere operator; a correction sweep is one oracle Gauss-Seidel sweep on
w = u + e with right-hand side det(D^2_h u) + rhs.  FP32 bounds: the
correction kernels carry ~1e-5 relative error in the base Hessian (hi/lo
split) and FP32 rounding of e, so they are compared relative to the size of
the quantity they compute.  Whole solves meet the same FP64 tolerance as the
FP64 path and are compared with the oracle at the FP64 bound (1e-10 relative).
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
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


def split(u):
    hi = u.astype(np.float32)
    lo = (u - hi.astype(np.float64)).astype(np.float32)
    return hi, lo


def smooth_correction_field(n, amp, seed):
    x, y, z = P.grid_coords(n)
    rng = np.random.default_rng(seed)
    a = rng.uniform(0.5, 1.5, 3)
    e = amp * np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z) * (1 + a[0] * x + a[1] * y * z)
    e += 0.1 * amp * rng.standard_normal(e.shape)
    e[0], e[-1], e[:, 0], e[:, -1], e[:, :, 0], e[:, :, -1] = 0, 0, 0, 0, 0, 0
    return e.astype(np.float32)


@pytest.mark.parametrize("name,n,amp", [("exp", 33, 1e-4), ("cosine", 65, 1e-5), ("exp", 129, 1e-6)])
def test_correction_residual_matches_oracle_definition(name, n, amp):
    pr = P.make(name, n, seed=3)
    u = pr.u
    e = smooth_correction_field(n, amp, n)
    rng = np.random.default_rng(1)
    rhs = (1e-3 * rng.standard_normal(u.shape)).astype(np.float32)
    N_ref = O.discrete_ma(np.ascontiguousarray(u + e.astype(np.float64)), pr.h) - O.discrete_ma(u, pr.h)
    ref = rhs.astype(np.float64) - N_ref
    ref[0], ref[-1], ref[:, 0], ref[:, -1], ref[:, :, 0], ref[:, :, -1] = 0, 0, 0, 0, 0, 0
    hi, lo = split(u)
    res = torch.empty(u.shape, dtype=torch.float32, device="cuda")
    _keep, scr, nb = M.correction_scratch(n)
    M.ma_residual_correction(dev(e), dev(hi), dev(lo), dev(rhs), res, n, pr.h, scr, nb)
    got = host(res).astype(np.float64)
    inner = (slice(1, -1),) * 3
    scale = np.max(np.abs(N_ref[inner])) + np.max(np.abs(rhs))
    assert np.max(np.abs(got - ref)) <= 2e-4 * scale


@pytest.mark.parametrize("pairs", [False, True])
@pytest.mark.parametrize("name,n,amp", [("exp", 33, 1e-4), ("cosine", 65, 1e-5), ("exp", 129, 1e-6),
                                        ("exp", 45, 1e-5)])
def test_correction_sweep_matches_oracle_sweep(name, n, amp, pairs):
    """One correction sweep against the oracle's Gauss-Seidel sweep on
    w = u + e with right-hand side det(D^2_h u) + rhs, in the regime the
    inner cycles run in (|rhs| ~ 1e-5 |f|, corrections of that order).  The
    kernel's base Hessian comes from the FP32 hi/lo split (~1e-5 relative),
    and e is FP32.  pairs: the colour-pair sweep (colours c and c^7 in one
    launch) against the oracle's sweep in the colour order 0, 7, 1, 6, 2, 5,
    3, 4; otherwise the by-colour sweep against ascending colours."""
    pr = P.make(name, n, seed=4)
    u = pr.u
    e = smooth_correction_field(n, amp, n + 1)
    rng = np.random.default_rng(2)
    rhs = (1e-5 * rng.standard_normal(u.shape) * np.max(pr.f)).astype(np.float32)
    rhs[0], rhs[-1] = 0, 0
    w = np.ascontiguousarray(u + e.astype(np.float64))
    ftot = O.discrete_ma(u, pr.h) + rhs.astype(np.float64)
    O.gs_sweep(w, ftot, pr.h, O.COLOUR8_PAIRS if pairs else O.COLOUR8)
    e_ref = w - u
    hi, lo = split(u)
    ed = dev(e)
    _keep, scr, nb = M.correction_scratch(n)
    try:
        M.ma_set_corr_tuning(n, M.MA_CORR_PAIRS if pairs else M.MA_CORR_BY_COLOUR, -1)
        M.ma_smooth_correction(ed, dev(hi), dev(lo), dev(rhs), n, pr.h, 1, scr, nb)
        got = host(ed).astype(np.float64)
    finally:
        M.ma_set_corr_tuning(n, -1, -1)
    change = np.max(np.abs(e_ref - e.astype(np.float64)))
    assert change > 0
    assert np.max(np.abs(got - e_ref)) <= 1e-3 * change + 1e-6 * np.max(np.abs(e_ref))


@pytest.mark.parametrize("name,n", [("exp", 33), ("cosine", 129), ("exp", 257), ("exp", 37), ("cosine", 71),
                                    ("exp", 135)])   # ragged last tiles for every tile size
def test_plane_sweeps_equal_colour_sweeps_bitwise(name, n):
    """Pairs of sweeps run by k parity (two launches per sweep, plane tiles
    of 16, 32 or 64 points that recompute a halo, a second e buffer) give the
    same bits as sweeps run colour by colour in place: all are the
    sequential 8-colour sweep.  At 129^3 and 257^3 every tile size has
    several tiles per plane edge."""
    pr = P.make(name, n, seed=6)
    u = pr.u
    e = smooth_correction_field(n, 1e-5, n + 2)
    rng = np.random.default_rng(3)
    rhs = (1e-5 * rng.standard_normal(u.shape) * np.max(pr.f)).astype(np.float32)
    hi, lo = (dev(a) for a in split(u))
    rhs_d = dev(rhs)
    _keep, scr, nb = M.correction_scratch(n)
    try:
        M.ma_set_corr_tuning(n, M.MA_CORR_BY_COLOUR, -1)
        refs = {}
        for sweeps in (2, 3):
            b = dev(e)
            for _ in range(sweeps):
                M.ma_smooth_correction(b, hi, lo, rhs_d, n, pr.h, 1, scr, nb)
            refs[sweeps] = b
        for choice in (M.MA_CORR_PLANE16, M.MA_CORR_PLANE32, M.MA_CORR_PLANE64):
            M.ma_set_corr_tuning(n, choice, -1)
            for sweeps in (2, 3):
                a = dev(e)
                M.ma_smooth_correction(a, hi, lo, rhs_d, n, pr.h, sweeps, scr, nb)
                torch.cuda.synchronize()
                assert not torch.equal(a, dev(e))
                d = (a - refs[sweeps]).abs().max().item()
                assert torch.equal(a, refs[sweeps]), f"{M.CORR_NAMES[choice]}, {sweeps} sweeps: max diff {d}"
    finally:
        M.ma_set_corr_tuning(n, -1, -1)


@pytest.mark.parametrize("n", [71, 129, 65])
def test_colour_pair_sweep_equals_its_colour_sequence_on_slow_points(n):
    """The colour-pair sweep (colours c and c^7 in one launch) is the
    sequential sweep in the order 0, 7, 1, 6, 2, 5, 3, 4: the same bits as
    the by-colour launches run in that order, here where the FP32 fast path
    fails.  A rough correction (K of the size of B) leaves G = B + K
    indefinite at many points, and a right-hand side of -2 f at scattered
    points makes det(B) + r <= 0 (the nonconvex branch); e and the count of
    nonconvex points agree bit for bit."""
    pr = P.make("exp", n, seed=2)
    rng = np.random.default_rng(n)
    e = np.zeros(pr.u.shape, dtype=np.float32)
    e[1:-1, 1:-1, 1:-1] = (0.5 * pr.h ** 2 * rng.standard_normal((n - 2,) * 3)).astype(np.float32)
    rhs = (1e-3 * rng.standard_normal(pr.u.shape) * pr.f).astype(np.float32)
    pick = rng.random(pr.u.shape) < 0.02
    rhs[pick] = (-2.0 * pr.f[pick]).astype(np.float32)
    rhs[0], rhs[-1], rhs[:, 0], rhs[:, -1], rhs[:, :, 0], rhs[:, :, -1] = 0, 0, 0, 0, 0, 0
    hi, lo = (dev(a) for a in split(pr.u))
    rhs_d = dev(rhs)
    _keep, scr, nb = M.correction_scratch(n)
    try:
        M.ma_set_corr_tuning(n, M.MA_CORR_PAIRS, -1)
        ed = dev(e)
        ev = torch.zeros(1, dtype=torch.int64, device="cuda")
        M.ma_smooth_correction(ed, hi, lo, rhs_d, n, pr.h, 2, scr, nb, events=ev)
        got = (host(ed), int(ev.item()))
    finally:
        M.ma_set_corr_tuning(n, -1, -1)
    ref = dev(e)
    ev = torch.zeros(1, dtype=torch.int64, device="cuda")
    for _ in range(2):
        for c in (0, 7, 1, 6, 2, 5, 3, 4):
            M.ma_smooth_correction_colour(ref, hi, lo, rhs_d, n, pr.h, c, scr, nb, events=ev)
    assert got[1] > 0 and got[1] == int(ev.item())
    assert np.array_equal(got[0], host(ref), equal_nan=True)
    assert not np.array_equal(got[0], e)


@pytest.mark.parametrize("n", [129, 71, 33, 257, 9])
@pytest.mark.parametrize("choice", [1, 2, 3, 4])
def test_residual_tiles_agree(choice, n):
    """The three residual tile sizes and the column kernel compute the same
    values (the same arithmetic per point), with a zero shell; sizes whose
    interior is not a multiple of the 30-point column span or the tiles."""
    pr = P.make("cosine", n, seed=7)
    e = smooth_correction_field(n, 1e-5, 11)
    rng = np.random.default_rng(4)
    rhs = (1e-5 * rng.standard_normal(pr.u.shape)).astype(np.float32)
    hi, lo = (dev(a) for a in split(pr.u))
    _keep, scr, nb = M.correction_scratch(n)
    outs = []
    try:
        for c in (M.MA_CORR_PLANE64, choice):
            M.ma_set_corr_tuning(n, -1, c)
            res = torch.full(pr.u.shape, 7.0, dtype=torch.float32, device="cuda")
            M.ma_residual_correction(dev(e), hi, lo, dev(rhs), res, n, pr.h, scr, nb)
            outs.append(host(res))
    finally:
        M.ma_set_corr_tuning(n, -1, -1)
    assert np.array_equal(outs[0], outs[1])
    sh = outs[1]
    assert np.all(sh[0] == 0) and np.all(sh[-1] == 0) and np.all(sh[:, 0] == 0) and np.all(sh[:, :, -1] == 0)


def test_autotune_records_a_choice_per_size():
    table = M.autotune([17, 33, 65], reps=2)
    try:
        for n in (17, 33, 65):
            t = table[n]
            sm, rs = M.ma_get_corr_tuning(n)
            assert M.CORR_NAMES[sm] == t["smoother"] and M.CORR_NAMES[rs] == t["residual"]
            assert t["us_per_sweep"][t["smoother"]] == min(t["us_per_sweep"].values())
            assert all(v > 0 for v in t["us_per_sweep"].values())
    finally:
        for n in (17, 33, 65):
            M.ma_set_corr_tuning(n, -1, -1)


@pytest.mark.parametrize("name,n", [("exp", 33), ("cosine", 65), ("exp", 129), ("quadratic", 65), ("sine", 65)])
def test_mixed_solve_matches_fp64_oracle(name, n):
    pr = P.make(name, n, seed=5)
    H = M.Hierarchy(M.make_desc(n, length=pr.length, precision=M.MA_MIXED))
    H.set_rhs_bc(dev(pr.f), dev(pr.initial()))
    res = H.solve(tol=1e-10, max_cycles=40)
    u = torch.empty_like(dev(pr.f))
    H.get_solution(u)
    got = host(u)
    H.close()
    ref = pr.initial()
    O.solve(ref, pr.f, pr.h, tol=1e-10, params=O.Params())
    assert res.res <= 1e-10
    assert np.max(np.abs(got - ref)) <= 1e-10 * np.max(np.abs(ref))
    e_gpu, e_ref = np.max(np.abs(got - pr.u)), np.max(np.abs(ref - pr.u))
    assert abs(e_gpu - e_ref) <= 1e-3 * e_ref + 1e-12 * np.max(np.abs(ref))


def test_mixed_and_fp64_agree_at_257():
    pr = P.make("exp", 257)
    outs = {}
    for prec in (M.MA_FP64, M.MA_MIXED):
        H = M.Hierarchy(M.make_desc(257, precision=prec))
        H.set_rhs_bc(dev(pr.f), dev(pr.initial()))
        r = H.solve(tol=1e-10, max_cycles=40)
        assert r.res <= 1e-10
        u = torch.empty_like(dev(pr.f))
        H.get_solution(u)
        outs[prec] = host(u)
        H.close()
    assert np.max(np.abs(outs[M.MA_FP64] - outs[M.MA_MIXED])) <= 1e-10 * np.max(np.abs(pr.u))
    r = O.residual(outs[M.MA_MIXED], pr.f, pr.h)
    assert np.max(np.abs(r)) <= 1.5e-10 * np.max(np.abs(pr.f[1:-1, 1:-1, 1:-1]))


@pytest.mark.parametrize("precision", [M.MA_MIXED, M.MA_FP32])
@pytest.mark.parametrize("name,n,coarsest", [("exp", 65, 3), ("cosine", 17, 3), ("exp", 33, 5), ("sine", 129, 3)])
def test_fused_tail_cycle_is_bitwise_the_level_by_level_cycle(name, n, coarsest, precision):
    """The levels with n <= 17 (9, 5) run as one single-block launch; the
    solve gives the same bits and cycle count as the level-by-level launches."""
    pr = P.make(name, n)
    outs = []
    try:
        for max_n in (17, 9, 5, 0):
            M.ma_set_corr_tail(max_n)
            H = M.Hierarchy(M.make_desc(n, length=pr.length, precision=precision, coarsest_n=coarsest))
            H.set_rhs_bc(dev(pr.f), dev(pr.initial()))
            r = H.solve(tol=1e-10 if precision == M.MA_MIXED else 1e-12, max_cycles=40, raise_on_error=False)
            u = torch.empty_like(dev(pr.f))
            H.get_solution(u)
            outs.append((host(u), r.cycles, r.res))
            H.close()
    finally:
        M.ma_set_corr_tail(True)
    for u, cycles, res in outs[:-1]:
        assert cycles == outs[-1][1] and res == outs[-1][2]
        assert np.array_equal(u, outs[-1][0])
