"""The device probes behind the design: the FP64 rate and the phase-chain
probe (launch edges in a CUDA graph against grid barriers in one cooperative
kernel).  The phase-chain check also confirms that the barriers order the
phases: from a uniform start every element follows the same chain of phases,
so a phase that read stale data would leave elements that differ."""
from __future__ import annotations

import pytest
import torch

from paper_1411_7018_gb300 import libma as M

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [1000, 1 << 16, (1 << 20) + 77])
def test_phase_chain_probe_orders_its_phases_and_reports_times(n):
    a = torch.full((n,), 0.5, dtype=torch.float32, device="cuda")
    b = torch.zeros_like(a)
    sync = torch.zeros(3, dtype=torch.int32, device="cuda")
    r = M.ma_probe_phase_chain(a, b, sync, phases=16, blocks_per_sm=4)
    torch.cuda.synchronize()
    assert all(v > 0 for v in r.values()), r
    # 3 forms x 7 runs x 16 phases = 336 phases, even: a holds the result
    assert torch.isfinite(a).all()
    assert bool((a == a[0]).all()) and bool((b == b[0]).all())
    # the value after 336 phases of x -> 1.0001 x + 1 from 0.5, in FP64: FP32
    # rounding over the chain stays well inside 1e-4 relative
    x = 0.5
    for _ in range(336):
        x = x * 1.0001 + 1.0
    assert abs(float(a[0]) - x) <= 1e-4 * x
    assert int(sync[2].item()) == 0


def test_phase_chain_probe_rejects_bad_arguments():
    a = torch.zeros(64, dtype=torch.float32, device="cuda")
    b = torch.zeros_like(a)
    sync = torch.zeros(3, dtype=torch.int32, device="cuda")
    with pytest.raises(M.MAError):
        M.ma_probe_phase_chain(a, b, sync, phases=1, blocks_per_sm=1)
    with pytest.raises(M.MAError):
        M.ma_probe_phase_chain(a, b, sync, phases=8, blocks_per_sm=10_000)


def test_fp64_rate_probe_is_positive_and_below_the_fp32_scale():
    r = M.ma_probe_fp64_rate()
    assert 1e10 < r < 1e14
