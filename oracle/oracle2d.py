"""ctypes binding to the 2D C oracle (oracle/ma2d_oracle.c).

TEST INFRASTRUCTURE ONLY (tests, the smoke check, the benchmark's CPU
baseline).  Arrays are numpy float64, C-contiguous, shape (n, n) indexed
[j, i], boundary included; h = len / N.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np

from . import build as _build

REDBLACK, LEXICOGRAPHIC, COLOUR4 = 0, 1, 2
HALF_WEIGHTING, FULL_WEIGHTING = 0, 1
NORM_MAX, NORM_L2 = 0, 1
APPROX_INJECTION, APPROX_WEIGHTED = 0, 1
FMG_BILINEAR, FMG_CUBIC = 0, 1
REF_RHS, REF_INITIAL = 0, 1

_lib = None
_dp = C.POINTER(C.c_double)


class _Params2(C.Structure):
    _fields_ = [(k, C.c_int) for k in ("nu1", "nu2", "coarsest_n", "restrict_kind", "coarse_sweeps", "ordering",
                                      "approx_restrict", "fmg_interp")]


@dataclass
class Params2D:
    nu1: int = 2
    nu2: int = 2
    coarsest_n: int = 3
    restrict_kind: int = FULL_WEIGHTING
    coarse_sweeps: int = 0
    ordering: int = REDBLACK
    approx_restrict: int = APPROX_WEIGHTED
    fmg_interp: int = FMG_BILINEAR

    def c(self):
        return _Params2(self.nu1, self.nu2, self.coarsest_n, self.restrict_kind, self.coarse_sweeps, self.ordering,
                        self.approx_restrict, self.fmg_interp)


def paper_params2d(ordering: int = REDBLACK, restrict_kind: int = HALF_WEIGHTING) -> Params2D:
    """Section 4's settings in 2D: V(2,2), h0 = 1/2 with one sweep, bicubic FMG."""
    return Params2D(coarsest_n=3, coarse_sweeps=1, ordering=ordering, restrict_kind=restrict_kind,
                    fmg_interp=FMG_CUBIC)


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(str(_build.build()))
        L.o2_point_update.restype = C.c_double
        L.o2_point_update.argtypes = [C.c_double] * 5
        L.o2_gs_sweep.restype = C.c_long
        L.o2_gs_sweep.argtypes = [_dp, _dp, C.c_int, C.c_double, C.c_int]
        L.o2_residual.restype = None
        L.o2_residual.argtypes = [_dp, _dp, _dp, C.c_int, C.c_double]
        L.o2_norm.restype = C.c_double
        L.o2_norm.argtypes = [_dp, C.c_int, C.c_double, C.c_int]
        L.o2_restrict_residual.restype = None
        L.o2_restrict_residual.argtypes = [_dp, C.c_int, _dp, C.c_int, C.c_int]
        L.o2_inject.restype = None
        L.o2_inject.argtypes = [_dp, C.c_int, _dp, C.c_int]
        L.o2_restrict_solution.restype = None
        L.o2_restrict_solution.argtypes = [_dp, C.c_int, _dp, C.c_int, C.c_int, C.c_int]
        L.o2_prolong_add.restype = None
        L.o2_prolong_add.argtypes = [_dp, _dp, C.c_int, _dp, C.c_int]
        L.o2_interpolate.restype = None
        L.o2_interpolate.argtypes = [_dp, C.c_int, _dp, C.c_int, C.c_int]
        L.o2_coarse_rhs.restype = None
        L.o2_coarse_rhs.argtypes = [_dp, _dp, _dp, C.c_int, C.c_double]
        L.o2_solve.restype = C.c_int
        L.o2_solve.argtypes = [_dp, _dp, C.c_int, C.c_double, C.POINTER(_Params2), C.c_double, C.c_int, C.c_int,
                               C.c_int, C.c_int, _dp, C.POINTER(C.c_long)]
        L.o2_discrete_ma.restype = None
        L.o2_discrete_ma.argtypes = [_dp, C.c_int, C.c_double, _dp]
        _lib = L
    return _lib


def _p(a):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_dp)


def point_update(a, b, r, h, rhs) -> float:
    return lib().o2_point_update(a, b, r, h, rhs)


def gs_sweep(u, rhs, h, ordering=REDBLACK) -> int:
    return lib().o2_gs_sweep(_p(u), _p(rhs), u.shape[0], h, ordering)


def residual(u, rhs, h):
    r = np.empty_like(u)
    lib().o2_residual(_p(u), _p(rhs), _p(r), u.shape[0], h)
    return r


def norm(v, h, kind=NORM_MAX) -> float:
    return lib().o2_norm(_p(v), v.shape[0], h, kind)


def _coarse(vf):
    nc = (vf.shape[0] + 1) // 2
    return np.zeros((nc, nc))


def restrict_residual(rf, kind=FULL_WEIGHTING):
    rc = _coarse(rf)
    lib().o2_restrict_residual(_p(rf), rf.shape[0], _p(rc), rc.shape[0], kind)
    return rc


def restrict_solution(uf, approx=APPROX_WEIGHTED, kind=FULL_WEIGHTING):
    uc = _coarse(uf)
    lib().o2_restrict_solution(_p(uf), uf.shape[0], _p(uc), uc.shape[0], approx, kind)
    return uc


def inject(vf):
    vc = _coarse(vf)
    lib().o2_inject(_p(vf), vf.shape[0], _p(vc), vc.shape[0])
    return vc


def prolong_add(uc, wc, uf) -> None:
    lib().o2_prolong_add(_p(uc), _p(wc), uc.shape[0], _p(uf), uf.shape[0])


def interpolate(uc, uf, cubic: bool = False) -> None:
    lib().o2_interpolate(_p(uc), uc.shape[0], _p(uf), uf.shape[0], 1 if cubic else 0)


def coarse_rhs(wc, rc, H):
    bc = np.empty_like(wc)
    lib().o2_coarse_rhs(_p(wc), _p(rc), _p(bc), wc.shape[0], H)
    return bc


def discrete_ma(u, h):
    out = np.empty_like(u)
    lib().o2_discrete_ma(_p(u), u.shape[0], h, _p(out))
    return out


@dataclass
class SolveInfo2D:
    cycles: int
    res_hist: np.ndarray
    events: int


def solve(u, f, h, tol=1e-10, norm_kind=NORM_MAX, max_cycles=50, init_fmg=True, params=None, ref=REF_RHS):
    p = (params or Params2D()).c()
    hist = np.full(max_cycles + 1, np.nan)
    ev = C.c_long(0)
    c = lib().o2_solve(_p(u), _p(f), u.shape[0], h, C.byref(p), tol, norm_kind, max_cycles, 1 if init_fmg else 0,
                       ref, _p(hist), C.byref(ev))
    if c < 0:
        raise ValueError("grid size does not coarsen to the coarsest grid")
    return SolveInfo2D(cycles=c, res_hist=hist[: c + 1], events=ev.value)
