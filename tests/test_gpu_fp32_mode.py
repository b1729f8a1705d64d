"""The full-FP32 mode (MA_FP32): FP32 FAS cycles on the solution itself,
stopping on the FP32 residual.  Its accuracy is limited by FP32 round-off of
the second differences, so the tests state the floor per grid size and check
the solution against the FP64 oracle's discrete solution within it."""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_1411_7018_gb300 import libma as M
from paper_1411_7018_gb300 import problems as P

pytestmark = pytest.mark.gpu
EPS32 = 2.0 ** -23


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    M.load()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("interp", [M.MA_FMG_CUBIC, M.MA_FMG_TRILINEAR])
@pytest.mark.parametrize("name,n", [("exp", 17), ("exp", 33), ("exp", 65), ("cosine", 65)])
def test_fp32_mode_floor_and_parity(name, n, interp):
    """The FP32 residual stalls at its round-off floor, stated as
    4 eps_32 max|u| N^2 relative to max|f| (second differences carry
    ~eps_32 |u| N^2 each; measured 0.04-0.5 of the bound), and the
    solution then agrees with the FP64 discrete solution to 1e-6 relative
    (measured <= 1.3e-7 up to 129^3) with the same error against the exact
    solution to 10 %; from the tricubic FMG start (through the FP64 level
    arrays) and from the trilinear one (FP32 throughout)."""
    pr = P.make(name, n)
    H = M.Hierarchy(M.make_desc(n, precision=M.MA_FP32, fmg_interp=interp))
    H.set_rhs_bc(dev(pr.f), dev(pr.initial()))
    r = H.solve(tol=1e-12, max_cycles=40, raise_on_error=False)
    u = torch.empty_like(dev(pr.f))
    H.get_solution(u)
    torch.cuda.synchronize()
    got = u.cpu().numpy()
    H.close()
    N = n - 1
    umax = np.max(np.abs(pr.u))
    assert r.status == M.MA_ERR_NOT_CONVERGED and r.floor_reached
    assert r.res <= 4 * EPS32 * umax * N * N
    ref = pr.initial()
    O.solve(ref, pr.f, pr.h, tol=1e-11, max_cycles=60)
    assert np.max(np.abs(got - ref)) <= 1e-6 * umax
    e32, e64 = np.max(np.abs(got - pr.u)), np.max(np.abs(ref - pr.u))
    assert abs(e32 - e64) <= 0.1 * e64


def test_fp32_mode_reaches_a_tolerance_above_its_floor():
    n = 33
    pr = P.make("exp", n)
    H = M.Hierarchy(M.make_desc(n, precision=M.MA_FP32))
    H.set_rhs_bc(dev(pr.f), dev(pr.initial()))
    r = H.solve(tol=1e-3, max_cycles=40)
    H.close()
    assert r.status == M.MA_OK and r.res <= 1e-3
