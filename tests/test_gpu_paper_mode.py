"""GPU parity of the paper-fidelity FMG (Algorithm 2 with tricubic
interpolation, h0 = 1/2 with one sweep, Section 4's relative-L2 stopping
rule) and of the singular Examples 6 and 7, against the FP64 CPU oracle run
in the same configuration (8-colour ordering, full weighting on both sides).
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


@pytest.mark.parametrize("nc", [3, 4, 5, 17, 65])
def test_cubic_interpolation_matches_oracle(nc):
    nf = 2 * nc - 1
    rng = np.random.default_rng(nc)
    uc = rng.standard_normal((nc, nc, nc))
    uf0 = rng.standard_normal((nf, nf, nf))
    ref = uf0.copy()
    O.interpolate_cubic(uc, ref)
    uf = dev(uf0)
    nb = M.ma_interpolate_cubic_scratch_bytes(nc)
    scr = torch.empty(nb // 8 + 1, dtype=torch.float64, device="cuda")
    M.ma_interpolate_cubic(dev(uc), nc, uf, scr, nb)
    got = host(uf)
    # the GPU sums the three one-axis passes in another order than the
    # oracle's triple sum: a few ulp of the O(1) values
    np.testing.assert_allclose(got, ref, rtol=0, atol=64 * EPS * 4)
    assert np.array_equal(got[0], uf0[0]) and np.array_equal(got[:, :, -1], uf0[:, :, -1])


def _oracle_paper(name, n):
    pr = P.make(name, n)
    u = pr.initial()
    prm = O.paper_params(O.COLOUR8)          # FW, 8 colours: the GPU's configuration
    info = O.solve(u, pr.f, pr.h, tol=1e-6, norm_kind=O.NORM_L2, max_cycles=30, params=prm, ref=O.REF_INITIAL)
    return pr, u, info


@pytest.mark.parametrize("name,n", [("exp", 33), ("sine", 33), ("ex6", 33), ("ex7", 33), ("exp", 65)])
def test_paper_mode_solve_matches_oracle(name, n):
    """One FMG pass with cubic interpolation meets Section 4's 1e-6 L2
    reduction (Iter = 1) on GPU and oracle alike, and the iterates agree."""
    pr, ref, info = _oracle_paper(name, n)
    H = M.Hierarchy(M.paper_desc(n, length=pr.length))
    H.set_rhs_bc(dev(pr.f), dev(pr.initial()))
    r = H.solve(tol=1e-6, norm=M.MA_NORM_L2, relative=M.MA_REL_INITIAL, max_cycles=30)
    u = torch.empty_like(dev(pr.f))
    H.get_solution(u)
    got = host(u)
    H.close()
    assert r.cycles == info.cycles
    assert r.res <= 1e-6
    assert np.max(np.abs(got - ref)) <= 1e-9 * np.max(np.abs(ref))
    e_gpu, e_ref = np.max(np.abs(got - pr.u)), np.max(np.abs(ref - pr.u))
    assert abs(e_gpu - e_ref) <= 1e-6 * e_ref


@pytest.mark.parametrize("precision", [M.MA_FP64, M.MA_MIXED])
def test_example6_solves_to_tolerance(precision):
    """Example 6 (singular at the corner x = 0) solved to a 1e-10 relative
    max-norm residual matches the oracle's discrete solution, in FP64 and in
    mixed precision."""
    n = 33
    pr = P.make("ex6", n)
    H = M.Hierarchy(M.make_desc(n, precision=precision))
    H.set_rhs_bc(dev(pr.f), dev(pr.initial()))
    r = H.solve(tol=1e-10, max_cycles=60)
    u = torch.empty_like(dev(pr.f))
    H.get_solution(u)
    got = host(u)
    H.close()
    ref = pr.initial()
    O.solve(ref, pr.f, pr.h, tol=1e-10, max_cycles=60)
    assert r.res <= 1e-10 and r.nonconvex_root_events == 0
    assert np.max(np.abs(got - ref)) <= 1e-10 * np.max(np.abs(ref))


def test_example7_fp64_meets_the_paper_criterion_and_ends_cleanly():
    """Example 7 (unbounded gradient at the corner (1,1,1)): Section 4's
    criterion (1e-6 discrete-L2 reduction against the initial residual) is
    met after the FMG pass, with the oracle's error.  A 1e-10 max-norm target
    is out of reach on this grid for the oracle as well (coarse right-hand
    sides <= 0 near the corner, a limit cycle of the max-norm residual): the
    solve must then stop with a finite iterate and a not-converged status."""
    n = 33
    pr, ref, info = _oracle_paper("ex7", n)
    H = M.Hierarchy(M.paper_desc(n))
    H.set_rhs_bc(dev(pr.f), dev(pr.initial()))
    r = H.solve(tol=1e-6, norm=M.MA_NORM_L2, relative=M.MA_REL_INITIAL, max_cycles=30)
    u = torch.empty_like(dev(pr.f))
    H.get_solution(u)
    got = host(u)
    assert r.res <= 1e-6 and r.cycles == info.cycles
    e_gpu, e_ref = np.max(np.abs(got - pr.u)), np.max(np.abs(ref - pr.u))
    assert abs(e_gpu - e_ref) <= 1e-3 * e_ref
    H.set_rhs_bc(dev(pr.f), dev(pr.initial()))
    r2 = H.solve(tol=1e-10, max_cycles=20, raise_on_error=False)
    H.get_solution(u)
    H.close()
    assert r2.status == M.MA_ERR_NOT_CONVERGED
    assert np.all(np.isfinite(host(u)))


def test_example7_mixed_precision():
    """Mixed precision on Example 7: where the max-norm iteration converges
    (17^3) the discrete solution matches the oracle's to 1e-10; at 33^3 (the
    non-converging regime above) the paper criterion is met with a finite
    iterate whose error stays within 3x of Table 7's printed 4.3e-3 -- in that
    regime every extra cycle moves the iterate, in FP64 as in mixed."""
    pr = P.make("ex7", 17)
    H = M.Hierarchy(M.make_desc(17, precision=M.MA_MIXED))
    H.set_rhs_bc(dev(pr.f), dev(pr.initial()))
    r = H.solve(tol=1e-10, max_cycles=60)
    u = torch.empty_like(dev(pr.f))
    H.get_solution(u)
    got = host(u)
    H.close()
    ref = pr.initial()
    O.solve(ref, pr.f, pr.h, tol=1e-10, max_cycles=60)
    assert r.res <= 1e-10
    assert np.max(np.abs(got - ref)) <= 1e-10 * np.max(np.abs(ref))
    pr = P.make("ex7", 33)
    H = M.Hierarchy(M.paper_desc(33, precision=M.MA_MIXED))
    H.set_rhs_bc(dev(pr.f), dev(pr.initial()))
    r = H.solve(tol=1e-6, norm=M.MA_NORM_L2, relative=M.MA_REL_INITIAL, max_cycles=30)
    u = torch.empty_like(dev(pr.f))
    H.get_solution(u)
    got = host(u)
    H.close()
    assert r.res <= 1e-6 and np.all(np.isfinite(got))
    assert np.max(np.abs(got - pr.u)) <= 3 * 4.3e-3
