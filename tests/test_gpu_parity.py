"""GPU parity: every step of the FP64 V-cycle and the whole solve, through the
C ABI, against the FP64 CPU oracle on the same seeded inputs.

Tolerances.  Kernels whose arithmetic is a fixed sum (transfers, norms) must
agree to a few ulps.  Kernels that form second differences (residual, coarse
right-hand side) lose log10(|u| / (h^2 |D^2 u|)) digits to cancellation in
either implementation, so they are compared against an explicit bound
C eps |u| / h^2 times the cofactor size.  The smoother and whole cycles agree to
1e-12 relative; solves to 1e-10 relative in max norm (FP64 parity target).
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_1411_7018_gb300 import libma as M
from paper_1411_7018_gb300 import problems as P

pytestmark = pytest.mark.gpu
EPS = np.finfo(np.float64).eps


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


def perturbed(name, n, amp, seed=0):
    pr = P.make(name, n, seed=seed)
    rng = np.random.default_rng(seed)
    u = pr.u.copy()
    u[1:-1, 1:-1, 1:-1] += amp * rng.standard_normal((n - 2,) * 3)
    return pr, np.ascontiguousarray(u)


# ---------------------------------------------------------------------------
# single steps
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name,n,amp", [("exp", 17, 1e-4), ("exp", 33, 1e-5), ("cosine", 65, 1e-6),
                                        ("exp", 129, 1e-7), ("sine", 33, 1e-4),
                                        ("exp", 23, 1e-4), ("cosine", 71, 1e-6)])   # ragged: n - 1 not 2^k
def test_smooth_one_sweep_matches_oracle(name, n, amp):
    pr, u0 = perturbed(name, n, amp)
    ref = u0.copy()
    O.gs_sweep(ref, pr.f, pr.h)
    u = dev(u0)
    M.ma_smooth(u, dev(pr.f), n, pr.h, 1)
    got = host(u)
    assert np.array_equal(got[0], u0[0]) and np.array_equal(got[:, :, -1], u0[:, :, -1])
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_smooth_far_from_convex_and_nonpositive_rhs():
    """Zero interior (Hessian far from positive definite near the shell) and a
    right-hand side with negative entries: exercises the FP64 fallback roots
    and the literal smallest-real-root rule."""
    n = 17
    pr = P.make("exp", n)
    u0 = pr.initial()
    f = pr.f.copy()
    rng = np.random.default_rng(3)
    mask = rng.random(f.shape) < 0.1
    f[mask] = -f[mask]
    ref = u0.copy()
    ev_ref = O.gs_sweep(ref, f, pr.h)
    u = dev(u0)
    ev = torch.zeros(1, dtype=torch.int64, device="cuda")
    M.ma_smooth(u, dev(f), n, pr.h, 1, ev)
    got = host(u)
    assert int(ev.item()) == ev_ref > 0
    assert np.max(np.abs(got - ref)) <= 1e-9 * np.max(np.abs(ref))


def test_smooth_quadratic_is_a_fixed_point_bitwise():
    pr = P.make("quadratic", 65)
    u = dev(pr.u)
    M.ma_smooth(u, dev(pr.f), 65, pr.h, 2)
    assert np.array_equal(host(u), pr.u)


def test_smooth_single_unknown_grid():
    rng = np.random.default_rng(11)
    g = rng.uniform(0, 1, (3, 3, 3))
    f = np.full((3, 3, 3), 1.7)
    ref = g.copy()
    O.gs_sweep(ref, f, 0.5)
    u = dev(g)
    M.ma_smooth(u, dev(f), 3, 0.5, 1)
    assert abs(host(u)[1, 1, 1] - ref[1, 1, 1]) <= 1e-13


def _residual_bound(u, h, name):
    """C eps |u| / h^2 times the largest cofactor of the Hessian."""
    hmax = {"exp": np.exp(1.5) * 4.0, "cosine": 1.2, "sine": 2.0, "quadratic": 1.0}[name]
    return 64.0 * EPS * np.max(np.abs(u)) / h ** 2 * hmax ** 2


@pytest.mark.parametrize("name,n", [("exp", 17), ("exp", 65), ("cosine", 129), ("sine", 33), ("exp", 23),
                                    ("cosine", 71)])
def test_residual_matches_oracle(name, n):
    pr, u0 = perturbed(name, n, 1e-6)
    ref = O.residual(u0, pr.f, pr.h)
    r = torch.full_like(dev(u0), 7.0)
    M.ma_residual(dev(u0), dev(pr.f), r, n, pr.h)
    got = host(r)
    shell = np.ones_like(got, bool)
    shell[1:-1, 1:-1, 1:-1] = False
    assert np.all(got[shell] == 0.0)
    assert np.max(np.abs(got - ref)) <= _residual_bound(u0, pr.h, name)


@pytest.mark.parametrize("name,n", [("exp", 17), ("exp", 65), ("cosine", 129), ("sine", 33), ("exp", 23),
                                    ("cosine", 71)])
def test_residual_f2_matches_oracle(name, n):
    """The residual of the mixed solve's fine grid (exact integer second
    differences, two-float determinant, FP64 where a stencil crosses a
    binade) against the oracle's FP64 residual, with the FP64 kernel's bound
    (the oracle's own rounding is the larger error), and 0 on the shell."""
    pr, u0 = perturbed(name, n, 1e-6)
    ref = O.residual(u0, pr.f, pr.h)
    r = torch.full_like(dev(u0), 7.0)
    M.ma_residual_f2(dev(u0), dev(pr.f), r, n, pr.h)
    got = host(r)
    shell = np.ones_like(got, bool)
    shell[1:-1, 1:-1, 1:-1] = False
    assert np.all(got[shell] == 0.0)
    assert np.max(np.abs(got - ref)) <= _residual_bound(u0, pr.h, name)


def _exact_residual(u, f, h, k, j, i):
    """f - det(D^2_h u) at one point in exact rational arithmetic on the FP64
    input values (the discrete operator of Eq. MA_discrete written out)."""
    from fractions import Fraction as Fr
    v = lambda dk, dj, di: Fr(float(u[k + dk, j + dj, i + di]))
    c = v(0, 0, 0)
    h2 = Fr(float(h)) ** 2
    xx = (v(0, 0, 1) + v(0, 0, -1) - 2 * c) / h2
    yy = (v(0, 1, 0) + v(0, -1, 0) - 2 * c) / h2
    zz = (v(1, 0, 0) + v(-1, 0, 0) - 2 * c) / h2
    xy = ((v(0, 1, 1) + v(0, -1, -1)) - (v(0, 1, -1) + v(0, -1, 1))) / (4 * h2)
    xz = ((v(1, 0, 1) + v(-1, 0, -1)) - (v(1, 0, -1) + v(-1, 0, 1))) / (4 * h2)
    yz = ((v(1, 1, 0) + v(-1, -1, 0)) - (v(1, -1, 0) + v(-1, 1, 0))) / (4 * h2)
    det = xx * (yy * zz - yz * yz) - xy * (xy * zz - xz * yz) + xz * (xy * yz - yy * xz)
    return Fr(float(f[k, j, i])) - det


@pytest.mark.parametrize("name,n", [("exp", 129), ("cosine", 65)])
def test_residual_f2_against_exact_rational_arithmetic(name, n):
    """At 60 sampled points the two-float residual is within 1e-12 max|f| of
    the residual computed in exact rational arithmetic from the same FP64
    values (brute force), which the FP64 kernel, whose gather rounds the
    sums of neighbours, misses by orders of magnitude more at 129^3."""
    pr, u0 = perturbed(name, n, 1e-6)
    r2 = torch.empty_like(dev(u0))
    r64 = torch.empty_like(dev(u0))
    M.ma_residual_f2(dev(u0), dev(pr.f), r2, n, pr.h)
    M.ma_residual(dev(u0), dev(pr.f), r64, n, pr.h)
    g2, g64 = host(r2), host(r64)
    rng = np.random.default_rng(n)
    pts = rng.integers(1, n - 1, size=(60, 3))
    fmax = np.max(np.abs(pr.f[1:-1, 1:-1, 1:-1]))
    e2 = max(abs(float(_exact_residual(u0, pr.f, pr.h, *p) - __import__("fractions").Fraction(float(g2[tuple(p)]))))
             for p in pts)
    e64 = max(abs(float(_exact_residual(u0, pr.f, pr.h, *p) - __import__("fractions").Fraction(float(g64[tuple(p)]))))
              for p in pts)
    assert e2 <= 1e-12 * fmax, (e2, e64)
    if name == "exp":
        assert e2 < e64


def test_residual_of_quadratic_is_exactly_zero():
    pr = P.make("quadratic", 129)
    r = torch.empty_like(dev(pr.u))
    M.ma_residual(dev(pr.u), dev(pr.f), r, 129, pr.h)
    assert np.all(host(r) == 0.0)
    M.ma_residual_f2(dev(pr.u), dev(pr.f), r, 129, pr.h)
    assert np.all(host(r) == 0.0)


@pytest.mark.parametrize("nf", [9, 33, 129, 23, 71])
@pytest.mark.parametrize("kind", [M.MA_HALF_WEIGHTING, M.MA_FULL_WEIGHTING])
def test_restrictions_match_oracle(nf, kind):
    rng = np.random.default_rng(nf + kind)
    v = rng.standard_normal((nf, nf, nf))
    nc = (nf + 1) // 2
    rc = torch.full((nc, nc, nc), 9.0, dtype=torch.float64, device="cuda")
    M.ma_restrict_residual(dev(v), nf, rc, kind)
    np.testing.assert_allclose(host(rc), O.restrict_residual(v, kind), rtol=0, atol=8 * EPS * np.abs(v).max())
    uc = torch.full_like(rc, 9.0)
    M.ma_restrict_solution(dev(v), nf, uc, M.MA_APPROX_WEIGHTED, kind)
    np.testing.assert_allclose(host(uc), O.restrict_solution(v, kind), rtol=0, atol=8 * EPS * np.abs(v).max())
    M.ma_restrict_solution(dev(v), nf, uc, M.MA_APPROX_INJECTION, kind)
    assert np.array_equal(host(uc), O.inject(v))


@pytest.mark.parametrize("nc", [5, 17, 65, 13, 37])
def test_prolong_interpolate_coarse_rhs_match_oracle(nc):
    nf = 2 * nc - 1
    rng = np.random.default_rng(nc)
    uc = rng.standard_normal((nc, nc, nc))
    wc = rng.standard_normal((nc, nc, nc))
    wc[0], wc[-1] = uc[0], uc[-1]
    uf0 = rng.standard_normal((nf, nf, nf))
    ref = uf0.copy()
    O.prolong_add(uc, wc, ref)
    uf = dev(uf0)
    M.ma_prolong_add(dev(uc), dev(wc), nc, uf)
    np.testing.assert_allclose(host(uf), ref, rtol=0, atol=16 * EPS * 8)
    ref2 = uf0.copy()
    O.interpolate(uc, ref2)
    uf = dev(uf0)
    M.ma_interpolate(dev(uc), nc, uf)
    np.testing.assert_allclose(host(uf), ref2, rtol=0, atol=16 * EPS * 8)
    # tau right-hand side on a convex coarse field
    pr, w = perturbed("cosine", nc, 1e-5)
    H = pr.h
    r = 1e-3 * rng.standard_normal((nc, nc, nc))
    b = torch.empty_like(dev(w))
    M.ma_coarse_rhs(dev(w), dev(r), b, nc, H)
    np.testing.assert_allclose(host(b), O.coarse_rhs(w, r, H), rtol=0, atol=_residual_bound(w, H, "cosine"))


@pytest.mark.parametrize("nc", [5, 13, 65])
def test_prolongation_on_a_buffer_not_aligned_to_pairs_gives_the_same_bits(nc):
    """The prolongation moves each fine row's two points as one aligned
    2-element access where the fine array allows it and as scalars otherwise:
    a fine array that starts one element (8 bytes) past a 16-byte boundary
    takes the scalar path and must give the same bits, in both modes."""
    nf = 2 * nc - 1
    rng = np.random.default_rng(100 + nc)
    uc = dev(rng.standard_normal((nc, nc, nc)))
    wc = dev(rng.standard_normal((nc, nc, nc)))
    uf0 = rng.standard_normal((nf, nf, nf))
    m = nf ** 3
    for mode in ("add", "interpolate"):
        aligned = dev(uf0).reshape(-1).clone()
        store = torch.zeros(m + 2, dtype=torch.float64, device="cuda")
        shifted = store[1:1 + m]
        shifted.copy_(aligned)
        assert shifted.data_ptr() % 16 == 8 and aligned.data_ptr() % 16 == 0
        if mode == "add":
            M.ma_prolong_add(uc, wc, nc, aligned)
            M.ma_prolong_add(uc, wc, nc, shifted)
        else:
            M.ma_interpolate(uc, nc, aligned)
            M.ma_interpolate(uc, nc, shifted)
        torch.cuda.synchronize()
        assert torch.equal(aligned, shifted), mode
        assert store[0].item() == 0.0 and store[-1].item() == 0.0   # nothing written outside


@pytest.mark.parametrize("n,sweeps", [(5, 0), (9, 0), (5, 1), (3, 1), (17, 3)])
def test_coarsest_solve_matches_oracle(n, sweeps):
    pr = P.make("exp", n)
    u0 = pr.initial()
    ref = u0.copy()
    if sweeps:
        for _ in range(sweeps):
            O.gs_sweep(ref, pr.f, pr.h)
    else:
        for _ in range(100):
            prev = ref.copy()
            O.gs_sweep(ref, pr.f, pr.h)
            if np.max(np.abs(ref - prev)) <= 1e-14 * np.max(np.abs(ref)):
                break
    u = dev(u0)
    M.ma_coarsest_solve(u, dev(pr.f), n, pr.h, sweeps)
    assert np.max(np.abs(host(u) - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("n", [5, 33, 129])
def test_norms_match_oracle(n):
    rng = np.random.default_rng(n)
    v = rng.standard_normal((n, n, n))
    h = 1.0 / (n - 1)
    nb = M.ma_norm_scratch_bytes(n)
    scratch = torch.empty(nb, dtype=torch.uint8, device="cuda")
    mx, l2 = M.ma_norm(dev(v), n, h, scratch, nb)
    assert mx == O.norm(v, h, O.NORM_MAX)
    assert abs(l2 - O.norm(v, h, O.NORM_L2)) <= 1e-13 * l2


# ---------------------------------------------------------------------------
# whole cycles and solves
# ---------------------------------------------------------------------------

def _params(kind=M.MA_FULL_WEIGHTING, approx=M.MA_APPROX_WEIGHTED, coarsest=3, csweeps=0):
    # the settings of M.make_desc's defaults (tricubic FMG start)
    return O.Params(nu1=2, nu2=2, coarsest_n=coarsest, restrict_kind=kind, coarse_sweeps=csweeps,
                    approx_restrict=approx, fmg_interp=O.FMG_CUBIC)


@pytest.mark.parametrize("name,n,kind,approx", [
    ("exp", 33, M.MA_FULL_WEIGHTING, M.MA_APPROX_WEIGHTED),
    ("cosine", 65, M.MA_FULL_WEIGHTING, M.MA_APPROX_INJECTION),
    ("exp", 17, M.MA_HALF_WEIGHTING, M.MA_APPROX_INJECTION),
])
def test_vcycle_matches_oracle(name, n, kind, approx):
    pr, u0 = perturbed(name, n, 1e-4)
    H = M.Hierarchy(M.make_desc(n, restrict_kind=kind, approx_restrict=approx))
    H.set_rhs_bc(dev(pr.f), dev(u0))
    H.vcycle(2)
    u = torch.empty_like(dev(u0))
    H.get_solution(u)
    got = host(u)
    H.close()
    ref = u0.copy()
    O.vcycle(ref, pr.f, pr.h, 2, _params(kind, approx))
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("name,n,coarsest", [("exp", 33, 5), ("quadratic", 33, 3), ("cosine", 65, 3),
                                             ("exp", 129, 3), ("sine", 65, 5)])
def test_solve_matches_oracle(name, n, coarsest):
    """Whole FP64 solves (FMG + V(2,2) to 1e-10) against the oracle, with the
    coarsest grid at 3^3 (Section 4's h0 = 1/2) or at 5^3 swept to
    convergence."""
    pr = P.make(name, n, seed=7)
    length = pr.length
    H = M.Hierarchy(M.make_desc(n, length=length, coarsest_n=coarsest))
    H.set_rhs_bc(dev(pr.f), dev(pr.initial()))
    res = H.solve(tol=1e-10)
    u = torch.empty_like(dev(pr.f))
    H.get_solution(u)
    got = host(u)
    H.close()
    ref = pr.initial()
    info = O.solve(ref, pr.f, pr.h, tol=1e-10, params=_params(coarsest=coarsest))
    assert res.res <= 1e-10 and res.nonconvex_root_events == 0
    assert abs(res.cycles - info.cycles) <= 1
    assert np.max(np.abs(got - ref)) <= 1e-10 * np.max(np.abs(ref))
    # same discretisation error against the exact solution
    e_gpu, e_ref = np.max(np.abs(got - pr.u)), np.max(np.abs(ref - pr.u))
    assert abs(e_gpu - e_ref) <= 1e-3 * e_ref + 1e-13


def test_paper_coarsest_settings_solve():
    """Section 4 settings: coarsest 3^3 grid, one sweep there, lexicographic
    replaced by 8 colours; the solve still reaches the tolerance."""
    pr = P.make("exp", 33)
    H = M.Hierarchy(M.make_desc(33, coarsest_n=3, coarse_sweeps=1))
    H.set_rhs_bc(dev(pr.f), dev(pr.initial()))
    res = H.solve(tol=1e-10, max_cycles=60)
    u = torch.empty_like(dev(pr.f))
    H.get_solution(u)
    got = host(u)
    H.close()
    ref = pr.initial()
    O.solve(ref, pr.f, pr.h, tol=1e-10, max_cycles=60, params=_params(coarsest=3, csweeps=1))
    assert res.res <= 1e-10
    assert np.max(np.abs(got - ref)) <= 1e-10 * np.max(np.abs(ref))


def test_solve_is_deterministic():
    pr = P.make("cosine", 65, seed=2)
    outs = []
    for _ in range(2):
        H = M.Hierarchy(M.make_desc(65))
        H.set_rhs_bc(dev(pr.f), dev(pr.initial()))
        H.solve(tol=1e-10)
        u = torch.empty_like(dev(pr.f))
        H.get_solution(u)
        outs.append(host(u))
        H.close()
    assert np.array_equal(outs[0], outs[1])


def test_full_size_257_solution_checked_by_oracle_residual():
    """257^3 (the full benchmark grid): the oracle's residual of the GPU
    solution meets the tolerance, the error against the exact solution is a
    quarter of the 129^3 one (O(h^2)), and sampled discrete Hessians are
    positive definite (Theorem 2.2)."""
    errs = {}
    for n in (129, 257):
        pr = P.make("exp", n)
        H = M.Hierarchy(M.make_desc(n))
        H.set_rhs_bc(dev(pr.f), dev(pr.initial()))
        res = H.solve(tol=1e-10)
        u = torch.empty_like(dev(pr.f))
        H.get_solution(u)
        got = host(u)
        H.close()
        errs[n] = np.max(np.abs(got - pr.u))
        if n == 257:
            r = O.residual(got, pr.f, pr.h)
            assert np.max(np.abs(r)) <= 1.5e-10 * np.max(np.abs(pr.f[1:-1, 1:-1, 1:-1]))
            rng = np.random.default_rng(0)
            for _ in range(200):
                k, j, i = rng.integers(1, n - 1, 3)
                blk = np.ascontiguousarray(got[k - 1:k + 2, j - 1:j + 2, i - 1:i + 2])
                Hs = O.discrete_hessian(blk, pr.h)[:, 1, 1, 1]
                Mx = np.array([[Hs[0], Hs[3], Hs[4]], [Hs[3], Hs[1], Hs[5]], [Hs[4], Hs[5], Hs[2]]])
                assert np.linalg.eigvalsh(Mx).min() > 0
    order = np.log2(errs[129] / errs[257])
    assert 1.9 <= order <= 2.1


def test_invalid_arguments_rejected():
    pr = P.make("exp", 17)
    f = pr.f.copy()
    f[5, 5, 5] = -1.0
    H = M.Hierarchy(M.make_desc(17))
    with pytest.raises(M.MAError) as ei:
        H.set_rhs_bc(dev(f), dev(pr.initial()))
    assert ei.value.status == M.MA_ERR_INVALID_ARG
    H.close()
    d = M.make_desc(17)
    nb = M.ma_hierarchy_footprint(d)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    with pytest.raises(M.MAError):
        M.ma_create_hierarchy(d, ws.data_ptr(), nb - 256)
    with pytest.raises(M.MAError):
        M.ma_create_hierarchy(d, ws.data_ptr() + 8, nb)


def test_not_converged_status():
    pr = P.make("exp", 33)
    H = M.Hierarchy(M.make_desc(33))
    H.set_rhs_bc(dev(pr.f), dev(pr.initial()))
    r = H.solve(tol=1e-14, max_cycles=2, raise_on_error=False)
    assert r.status == M.MA_ERR_NOT_CONVERGED and r.cycles == 2
    H.close()


@pytest.mark.parametrize("precision", [M.MA_FP64, M.MA_MIXED, M.MA_FP32])
@pytest.mark.parametrize("n", [3, 5])
def test_single_level_hierarchy_solves(n, precision):
    """n = coarsest_n: the hierarchy is its coarsest grid, FMG is the coarsest
    solve and every cycle is one.  FP64 and mixed reach the oracle's discrete
    solution; FP32 reaches it to FP32 round-off."""
    pr = P.make("exp", n)
    H = M.Hierarchy(M.make_desc(n, coarsest_n=n, precision=precision))
    H.set_rhs_bc(dev(pr.f), dev(pr.initial()))
    r = H.solve(tol=1e-11 if precision != M.MA_FP32 else 1e-5, max_cycles=40, raise_on_error=False)
    u = torch.empty_like(dev(pr.f))
    H.get_solution(u)
    got = host(u)
    H.close()
    assert r.status == M.MA_OK or (r.status == M.MA_ERR_NOT_CONVERGED and r.floor_reached)
    ref = pr.initial()
    O.solve(ref, pr.f, pr.h, tol=1e-13, max_cycles=60, params=O.Params(coarsest_n=n))
    bound = 1e-10 if precision != M.MA_FP32 else 1e-6
    assert np.max(np.abs(got - ref)) <= bound * np.max(np.abs(ref))
