"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point include/*.h declares; host-only calls behave (no compute)."""
from __future__ import annotations

import ctypes as C
import os
import re
import shutil

import pytest

from paper_1411_7018_gb300 import libma as M

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

pytestmark = pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                                reason="nvcc not available")


def declared_symbols():
    names = set()
    inc = os.path.join(ROOT, "include")
    for fn in os.listdir(inc):
        if fn.endswith(".h"):
            txt = open(os.path.join(inc, fn)).read()
            names.update(re.findall(r"^\s*(?:ma_status|const char \*)\s*(ma_\w+)\s*\(", txt, re.M))
    return names


def test_library_exports_every_declared_symbol():
    lib = M.load()
    names = declared_symbols()
    assert len(names) >= 20
    for name in sorted(names):
        assert hasattr(lib, name), name
    assert set(M.EXPORTED) >= names


def test_footprint_is_host_only_and_counts_levels():
    d = M.make_desc(33)
    nb = M.ma_hierarchy_footprint(d)
    # four n^3 double fields per level (33, 17, 9, 5) plus reduction scratch
    fields = 4 * 8 * sum(m ** 3 for m in (33, 17, 9, 5))
    assert fields <= nb <= fields + 256 * 64 + 2 * 8 * 16 * 9 * 2 * 33
    d2 = M.make_desc(257)
    assert M.ma_hierarchy_footprint(d2) > 4 * 8 * 257 ** 3


@pytest.mark.parametrize("kw", [dict(n=32), dict(n=33, coarsest_n=4), dict(n=33, nu1=0, nu2=0),
                                dict(n=33, restrict_kind=7), dict(n=33, precision=3), dict(n=33, length=0.0),
                                dict(n=35)])
def test_bad_descriptors_rejected(kw):
    length = kw.pop("length", 1.0)
    d = M.make_desc(length=length, **kw)
    with pytest.raises(M.MAError) as ei:
        M.ma_hierarchy_footprint(d)
    assert ei.value.status == M.MA_ERR_INVALID_ARG
    assert M.ma_last_error_string()


def test_step_calls_reject_bad_arguments_before_any_launch():
    lib = M.load()
    assert lib.ma_smooth(None, None, 33, 0.1, 1, None, None) == M.MA_ERR_INVALID_ARG
    assert lib.ma_residual(C.c_void_p(256), C.c_void_p(256), C.c_void_p(256), 32, 0.1, None) == M.MA_ERR_INVALID_ARG
    assert lib.ma_coarsest_solve(C.c_void_p(256), C.c_void_p(256), 33, 0.1, 0, None, None) == M.MA_ERR_INVALID_ARG
    assert M.ma_norm_scratch_bytes(33) > 0


def test_host_only_settings_validate_their_arguments():
    """The process-wide switches of the fused tails, the batches and the
    correction tuning table check their values without touching a GPU."""
    for fn, bad in ((M.ma_set_corr_tail, (2, 4, 7, 33, -1)), (M.ma_set_vcycle_tail, (2, 6, 65, -3)),
                    (M.ma_set_batch_groups, (0, 17, -1))):
        for v in bad:
            with pytest.raises(M.MAError) as ei:
                fn(v)
            assert ei.value.status == M.MA_ERR_INVALID_ARG
    # the C entry point of the start switch takes 0 or 1 only (the binding maps a bool)
    assert M.load().ma_set_batch_start(2) == M.MA_ERR_INVALID_ARG
    M.ma_set_batch_start(False)
    for v in (0, 3, 5, 9, 17, True):
        M.ma_set_corr_tail(v)
        M.ma_set_vcycle_tail(v)
    M.ma_set_corr_tail(True)
    M.ma_set_vcycle_tail(True)
    for g in (1, 16, 2):
        M.ma_set_batch_groups(g)
    with pytest.raises(M.MAError):
        M.ma_set_corr_tuning(34, 1, 1)          # n must be odd
    with pytest.raises(M.MAError):
        M.ma_set_corr_tuning(33, 6, 1)          # no smoother variant 6
    with pytest.raises(M.MAError):
        M.ma_set_corr_tuning(33, M.MA_CORR_COLUMN, 1)      # the column form is a residual only
    with pytest.raises(M.MAError):
        M.ma_set_corr_tuning(33, 1, M.MA_CORR_PAIRS)      # the paired form is a smoother only
    with pytest.raises(M.MAError):
        M.ma_set_corr_tuning(33, 1, M.MA_CORR_BY_COLOUR)   # the residual has no by-colour form
    M.ma_set_corr_tuning(33, M.MA_CORR_PLANE32, M.MA_CORR_COLUMN)
    assert M.ma_get_corr_tuning(33) == (M.MA_CORR_PLANE32, M.MA_CORR_COLUMN)
    M.ma_set_corr_tuning(33, M.MA_CORR_PAIRS, M.MA_CORR_PLANE16)
    assert M.ma_get_corr_tuning(33) == (M.MA_CORR_PAIRS, M.MA_CORR_PLANE16)
    for colour in (-1, 8):   # rejected on the host, before any device work
        with pytest.raises(M.MAError):
            M.ma_smooth_correction_colour(256, 256, 256, 256, 33, 0.1, colour, 256, 1 << 24, stream=0)
    M.ma_set_corr_tuning(33, -1, -1)


def test_batch_footprint_rejects_an_empty_batch():
    with pytest.raises(M.MAError) as ei:
        M.ma_batch_footprint([])
    assert ei.value.status == M.MA_ERR_INVALID_ARG


def test_static_norm_limit_in_the_binding_matches_the_header():
    """The Python binding's copy of MA_NORM_STATIC_MAX_N is the value the C
    header defines, so the no-allocation norm's tests probe the real limit."""
    txt = open(os.path.join(ROOT, "include", "ma.h")).read()
    m = re.search(r"^#define\s+MA_NORM_STATIC_MAX_N\s+(\d+)\s*$", txt, re.M)
    assert m is not None
    assert int(m.group(1)) == M.MA_NORM_STATIC_MAX_N
