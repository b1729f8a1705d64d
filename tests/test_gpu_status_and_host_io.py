"""Error status of a non-finite iterate, and the host-buffer entry points of
the C ABI (ma_set_rhs_bc_host / ma_get_solution_host) against the device ones.

The non-finite case is made on the host: a NaN written into one interior
point of the initial iterate (ma_set_solution, then a solve that keeps the
iterate, MA_INIT_KEEP).  No kernel faults; the residual norms carry the NaN
back and the solve must stop with MA_ERR_NONFINITE instead of reporting a
finite residual."""
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


@pytest.mark.parametrize("precision", [M.MA_FP64, M.MA_MIXED, M.MA_FP32])
@pytest.mark.parametrize("where", ["one point", "every point"])
def test_nan_in_the_initial_iterate_ends_the_solve_as_nonfinite(precision, where):
    pr = P.make("exp", 33)
    H = M.Hierarchy(M.make_desc(33, precision=precision))
    H.set_rhs_bc(dev(pr.f), dev(pr.initial()))
    u0 = pr.u.copy()
    if where == "one point":
        u0[16, 9, 20] = np.nan
    else:
        u0[1:-1, 1:-1, 1:-1] = np.nan
    H.set_solution(dev(u0))
    r = H.solve(tol=1e-10, max_cycles=5, init=M.MA_INIT_KEEP, raise_on_error=False)
    assert r.status == M.MA_ERR_NONFINITE, r
    with pytest.raises(M.MAError) as ei:
        H.set_solution(dev(u0))
        H.solve(tol=1e-10, max_cycles=5, init=M.MA_INIT_KEEP)
    assert ei.value.status == M.MA_ERR_NONFINITE
    # the hierarchy stays usable: new data and a normal solve
    H.set_rhs_bc(dev(pr.f), dev(pr.initial()))
    r = H.solve(tol=1e-10 if precision != M.MA_FP32 else 1e-4, max_cycles=40, raise_on_error=False)
    assert r.status == M.MA_OK or (r.status == M.MA_ERR_NOT_CONVERGED and r.floor_reached)
    H.close()


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("precision", [M.MA_FP64, M.MA_MIXED])
def test_host_buffer_calls_equal_the_device_calls(precision, pinned):
    """f and g copied in from host memory and u copied out to host memory
    give bit for bit the solve of the device-pointer calls; a bad f in a host
    buffer is rejected the same way."""
    pr = P.make("cosine", 65, seed=5)
    H = M.Hierarchy(M.make_desc(65, precision=precision))
    H.set_rhs_bc(dev(pr.f), dev(pr.initial()))
    r_dev = H.solve(tol=1e-10, max_cycles=40)
    u_dev = torch.empty((65,) * 3, dtype=torch.float64, device="cuda")
    H.get_solution(u_dev)
    torch.cuda.synchronize()
    ref = u_dev.cpu().numpy()

    f_h, g_h = torch.from_numpy(pr.f.copy()), torch.from_numpy(pr.initial())
    u_h = torch.full((65,) * 3, np.nan, dtype=torch.float64)
    if pinned:
        f_h, g_h, u_h = f_h.pin_memory(), g_h.pin_memory(), u_h.pin_memory()
    H.set_rhs_bc_host(f_h, g_h)
    r_host = H.solve(tol=1e-10, max_cycles=40)
    H.get_solution_host(u_h)
    assert (r_host.cycles, r_host.res) == (r_dev.cycles, r_dev.res)
    assert np.array_equal(u_h.numpy(), ref)
    # numpy arrays work as well
    u_np = np.empty((65,) * 3)
    H.get_solution_host(u_np)
    assert np.array_equal(u_np, ref)
    bad = pr.f.copy()
    bad[3, 4, 5] = 0.0
    with pytest.raises(M.MAError) as ei:
        H.set_rhs_bc_host(bad, pr.initial())
    assert ei.value.status == M.MA_ERR_INVALID_ARG
    H.close()
