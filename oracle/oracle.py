"""ctypes binding to the C oracle (oracle/ma_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the
benchmark's CPU-baseline leg are the only callers.  Arrays are numpy float64,
C-contiguous, shape (n, n, n) indexed [k, j, i] with the boundary shell
included; n = N + 1 points per side and h = len / N (Section 2).
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np

from . import build as _build

COLOUR8, LEXICOGRAPHIC, COLOUR8_REVERSED, COLOUR8_PAIRS = 0, 1, 2, 3
HALF_WEIGHTING, FULL_WEIGHTING = 0, 1
NORM_MAX, NORM_L2 = 0, 1
APPROX_INJECTION, APPROX_WEIGHTED = 0, 1
FMG_TRILINEAR, FMG_CUBIC = 0, 1
REF_RHS, REF_INITIAL = 0, 1

_lib = None
_dp = C.POINTER(C.c_double)


class _Params(C.Structure):
    _fields_ = [("nu1", C.c_int), ("nu2", C.c_int), ("coarsest_n", C.c_int),
                ("restrict_kind", C.c_int), ("coarse_sweeps", C.c_int), ("ordering", C.c_int),
                ("approx_restrict", C.c_int), ("fmg_interp", C.c_int)]


@dataclass
class Params:
    """FAS parameters: V(nu1, nu2), coarsest grid size, residual restriction
    kind, coarsest sweeps (0 = sweep to convergence), smoother ordering, the
    approximation restriction (injection or the residual's weighting) and the
    FMG interpolation (trilinear or tricubic)."""
    nu1: int = 2
    nu2: int = 2
    coarsest_n: int = 3
    restrict_kind: int = FULL_WEIGHTING
    coarse_sweeps: int = 0
    ordering: int = COLOUR8
    approx_restrict: int = APPROX_WEIGHTED
    fmg_interp: int = FMG_TRILINEAR

    def c(self) -> _Params:
        return _Params(self.nu1, self.nu2, self.coarsest_n, self.restrict_kind,
                       self.coarse_sweeps, self.ordering, self.approx_restrict, self.fmg_interp)


def paper_params(ordering: int = LEXICOGRAPHIC) -> "Params":
    """The settings of Section 4: V(2,2), h0 = 1/2 (3^3 coarsest grid) with one
    Gauss-Seidel sweep, tricubic FMG interpolation (lexicographic ordering by
    default, as the paper's smoother)."""
    return Params(nu1=2, nu2=2, coarsest_n=3, coarse_sweeps=1, ordering=ordering, fmg_interp=FMG_CUBIC)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(str(path))
        L.orc_gs_sweep.restype = C.c_long
        L.orc_gs_sweep.argtypes = [_dp, _dp, C.c_int, C.c_double, C.c_int]
        L.orc_residual.restype = None
        L.orc_residual.argtypes = [_dp, _dp, _dp, C.c_int, C.c_double]
        L.orc_norm.restype = C.c_double
        L.orc_norm.argtypes = [_dp, C.c_int, C.c_double, C.c_int]
        for name in ("orc_restrict_residual", "orc_restrict_solution"):
            getattr(L, name).restype = None
            getattr(L, name).argtypes = [_dp, C.c_int, _dp, C.c_int, C.c_int]
        L.orc_inject.restype = None
        L.orc_inject.argtypes = [_dp, C.c_int, _dp, C.c_int]
        L.orc_prolong_add.restype = None
        L.orc_prolong_add.argtypes = [_dp, _dp, C.c_int, _dp, C.c_int]
        for name in ("orc_interpolate", "orc_interpolate_cubic"):
            getattr(L, name).restype = None
            getattr(L, name).argtypes = [_dp, C.c_int, _dp, C.c_int]
        L.orc_coarse_rhs.restype = None
        L.orc_coarse_rhs.argtypes = [_dp, _dp, _dp, C.c_int, C.c_double]
        L.orc_vcycle.restype = C.c_long
        L.orc_vcycle.argtypes = [_dp, _dp, C.c_int, C.c_double, C.POINTER(_Params), C.c_int]
        L.orc_fmg.restype = C.c_long
        L.orc_fmg.argtypes = [_dp, _dp, C.c_int, C.c_double, C.POINTER(_Params)]
        L.orc_solve.restype = C.c_int
        L.orc_solve.argtypes = [_dp, _dp, C.c_int, C.c_double, C.POINTER(_Params), C.c_double,
                                C.c_int, C.c_int, C.c_int, C.c_int, _dp, C.POINTER(C.c_long)]
        L.orc_smallest_root.restype = C.c_double
        L.orc_smallest_root.argtypes = [_dp, C.c_double]
        L.orc_point_update.restype = C.c_double
        L.orc_point_update.argtypes = [_dp, C.c_double, C.c_double, C.c_double]
        L.orc_sym3_eigenvalues.restype = None
        L.orc_sym3_eigenvalues.argtypes = [_dp, _dp]
        L.orc_discrete_ma.restype = None
        L.orc_discrete_ma.argtypes = [_dp, _dp, C.c_int, C.c_double]
        L.orc_discrete_hessian.restype = None
        L.orc_discrete_hessian.argtypes = [_dp, _dp, C.c_int, C.c_double]
        L.orc_max_threads.restype = C.c_int
        L.orc_max_threads.argtypes = []
        _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_dp)


def _grid(a: np.ndarray) -> int:
    assert a.ndim == 3 and a.shape[0] == a.shape[1] == a.shape[2]
    return a.shape[0]


def max_threads() -> int:
    return lib().orc_max_threads()


def gs_sweep(u: np.ndarray, rhs: np.ndarray, h: float, ordering: int = COLOUR8) -> int:
    """One nonlinear Gauss-Seidel sweep in place on u (Section 2, Eq. realroots).
    Returns the count of point updates with rhs <= 0."""
    return lib().orc_gs_sweep(_p(u), _p(rhs), _grid(u), h, ordering)


def residual(u: np.ndarray, rhs: np.ndarray, h: float) -> np.ndarray:
    """rhs - det(D^2_h u) on the interior, 0 on the shell (Algorithm 1, step 3)."""
    r = np.empty_like(u)
    lib().orc_residual(_p(u), _p(rhs), _p(r), _grid(u), h)
    return r


def norm(v: np.ndarray, h: float, kind: int = NORM_MAX) -> float:
    """Max norm or discrete L2 norm sqrt(h^3 sum v^2) over the interior."""
    return lib().orc_norm(_p(v), _grid(v), h, kind)


def _coarse_like(vf: np.ndarray) -> np.ndarray:
    nf = _grid(vf)
    assert (nf - 1) % 2 == 0
    nc = (nf + 1) // 2
    return np.zeros((nc, nc, nc))


def restrict_residual(rf: np.ndarray, kind: int = HALF_WEIGHTING) -> np.ndarray:
    rc = _coarse_like(rf)
    lib().orc_restrict_residual(_p(rf), _grid(rf), _p(rc), _grid(rc), kind)
    return rc


def restrict_solution(uf: np.ndarray, kind: int = HALF_WEIGHTING) -> np.ndarray:
    uc = _coarse_like(uf)
    lib().orc_restrict_solution(_p(uf), _grid(uf), _p(uc), _grid(uc), kind)
    return uc


def inject(vf: np.ndarray) -> np.ndarray:
    vc = _coarse_like(vf)
    lib().orc_inject(_p(vf), _grid(vf), _p(vc), _grid(vc))
    return vc


def prolong_add(uc: np.ndarray, wc: np.ndarray, uf: np.ndarray) -> None:
    """uf += trilinear(uc - wc) on the fine interior, in place."""
    lib().orc_prolong_add(_p(uc), _p(wc), _grid(uc), _p(uf), _grid(uf))


def interpolate(uc: np.ndarray, uf: np.ndarray) -> None:
    """Fine interior of uf := trilinear interpolation of uc, in place."""
    lib().orc_interpolate(_p(uc), _grid(uc), _p(uf), _grid(uf))


def interpolate_cubic(uc: np.ndarray, uf: np.ndarray) -> None:
    """Fine interior of uf := tricubic interpolation of uc (Algorithm 2 step 4), in place."""
    lib().orc_interpolate_cubic(_p(uc), _grid(uc), _p(uf), _grid(uf))


def coarse_rhs(wc: np.ndarray, rc: np.ndarray, H: float) -> np.ndarray:
    bc = np.empty_like(wc)
    lib().orc_coarse_rhs(_p(wc), _p(rc), _p(bc), _grid(wc), H)
    return bc


def vcycle(u: np.ndarray, f: np.ndarray, h: float, ncycles: int = 1, params: Params | None = None) -> int:
    """ncycles FAS V-cycles (Algorithm 1) in place on u; returns nonconvex events."""
    p = (params or Params()).c()
    ev = lib().orc_vcycle(_p(u), _p(f), _grid(u), h, C.byref(p), ncycles)
    if ev < 0:
        raise ValueError("grid size does not coarsen to the coarsest grid")
    return ev


def fmg(u: np.ndarray, f: np.ndarray, h: float, params: Params | None = None) -> int:
    """One FMG-FAS pass (Algorithm 2) in place on u (its shell supplies g)."""
    p = (params or Params()).c()
    ev = lib().orc_fmg(_p(u), _p(f), _grid(u), h, C.byref(p))
    if ev < 0:
        raise ValueError("grid size does not coarsen to the coarsest grid")
    return ev


@dataclass
class SolveInfo:
    cycles: int
    res_hist: np.ndarray
    events: int


def solve(u: np.ndarray, f: np.ndarray, h: float, tol: float = 1e-10, norm_kind: int = NORM_MAX,
          max_cycles: int = 50, init_fmg: bool = True, params: Params | None = None,
          ref: int = REF_RHS) -> SolveInfo:
    """FMG init then V-cycles until ||f - S_h u|| / ref <= tol, in place on u;
    ref = ||f|| (REF_RHS) or the residual norm of the initial iterate
    (REF_INITIAL, the relative residual of Section 4)."""
    p = (params or Params()).c()
    hist = np.full(max_cycles + 1, np.nan)
    ev = C.c_long(0)
    c = lib().orc_solve(_p(u), _p(f), _grid(u), h, C.byref(p), tol, norm_kind, max_cycles,
                        1 if init_fmg else 0, ref, _p(hist), C.byref(ev))
    if c < 0:
        raise ValueError("grid size does not coarsen to the coarsest grid")
    return SolveInfo(cycles=c, res_hist=hist[: c + 1], events=ev.value)


def smallest_root(H: np.ndarray, rhs: float) -> float:
    """Smallest real root z of det(H - z I) = rhs (Eq. realroots, shifted form)."""
    Hm = np.ascontiguousarray(H, dtype=np.float64).reshape(9)
    return lib().orc_smallest_root(_p(Hm), rhs)


def point_update(q6, v0: float, h: float, rhs: float) -> float:
    """New centre value: smallest real root of P3(.; u) given (a, b, c, r, s, t)."""
    q = np.ascontiguousarray(q6, dtype=np.float64)
    return lib().orc_point_update(_p(q), v0, h, rhs)


def sym3_eigenvalues(H: np.ndarray) -> np.ndarray:
    Hm = np.ascontiguousarray(H, dtype=np.float64).reshape(9)
    lam = np.zeros(3)
    lib().orc_sym3_eigenvalues(_p(Hm), _p(lam))
    return lam


def discrete_ma(u: np.ndarray, h: float) -> np.ndarray:
    out = np.empty_like(u)
    lib().orc_discrete_ma(_p(u), _p(out), _grid(u), h)
    return out


def discrete_hessian(u: np.ndarray, h: float) -> np.ndarray:
    """(6, n, n, n): xx, yy, zz, xy, xz, yz on the interior, zero on the shell."""
    n = _grid(u)
    out = np.empty((6, n, n, n))
    lib().orc_discrete_hessian(_p(u), _p(out), n, h)
    return out
