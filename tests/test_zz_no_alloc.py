"""ma_norm_static: the norms of ma_norm for callers that cannot allocate
device memory (all of it owned by another allocator, or no implicit
cudaMalloc synchronisation allowed), with its scratch in a fixed array inside
the library.  Checked against ma_norm on two calls in a row; kept in a file
that pytest collects last."""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1411_7018_gb300 import libma as M

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    M.load()


def _norm_with_caller_scratch(v, n, h):
    nb = M.ma_norm_scratch_bytes(n)
    scratch = torch.empty(nb, dtype=torch.uint8, device="cuda")
    return M.ma_norm(v, n, h, scratch, nb)


@pytest.mark.parametrize("n", [33, 257, M.MA_NORM_STATIC_MAX_N])
def test_static_scratch_norm_matches_ma_norm_twice(n):
    h = 1.0 / (n - 1)
    rng = np.random.default_rng(n)
    for call in range(2):   # the second call must not depend on the first's leftovers
        v = torch.from_numpy(rng.standard_normal((n, n, n)) * (1.0 + 10.0 * call)).cuda()
        mx_ref, l2_ref = _norm_with_caller_scratch(v, n, h)
        mx, l2 = M.ma_norm_static(v, n, h)
        assert mx == mx_ref
        assert abs(l2 - l2_ref) <= 1e-13 * l2_ref


def test_static_scratch_norm_rejects_grids_beyond_its_limit():
    n = M.MA_NORM_STATIC_MAX_N + 2
    with pytest.raises(M.MAError) as ei:
        M.ma_norm_static(torch.zeros(1, dtype=torch.float64, device="cuda"), n, 1.0 / (n - 1))
    assert ei.value.status == M.MA_ERR_INVALID_ARG
    assert str(M.MA_NORM_STATIC_MAX_N) in M.ma_last_error_string()
