"""Python binding of libma (include/ma.h): ctypes argument marshalling only.

Every function here has the name of the C entry point it calls and does no
arithmetic of its own; a non-zero ma_status raises MAError carrying
ma_last_error_string().  Device buffers are torch CUDA tensors (float64,
contiguous) or raw device addresses; streams are torch.cuda.Stream objects or
None for the current stream.  There is no CPU fallback: if libma.so cannot be
built or loaded, every call raises.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

from . import build as _build

MA_OK, MA_ERR_INVALID_ARG, MA_ERR_OOM, MA_ERR_CUDA, MA_ERR_NOT_CONVERGED, MA_ERR_NONFINITE = range(6)
MA_HALF_WEIGHTING, MA_FULL_WEIGHTING = 0, 1
MA_APPROX_INJECTION, MA_APPROX_WEIGHTED = 0, 1
MA_FP64, MA_MIXED, MA_FP32 = 0, 1, 2
MA_NORM_MAX, MA_NORM_L2 = 0, 1
MA_INIT_FMG, MA_INIT_ZERO, MA_INIT_KEEP = 0, 1, 2
MA_FMG_TRILINEAR, MA_FMG_CUBIC = 0, 1
MA_REL_NONE, MA_REL_RHS, MA_REL_INITIAL = 0, 1, 2
MA_CORR_BY_COLOUR, MA_CORR_PLANE16, MA_CORR_PLANE32, MA_CORR_PLANE64, MA_CORR_COLUMN, MA_CORR_PAIRS = 0, 1, 2, 3, 4, 5
CORR_NAMES = {MA_CORR_BY_COLOUR: "by_colour", MA_CORR_PLANE16: "plane16", MA_CORR_PLANE32: "plane32",
              MA_CORR_PLANE64: "plane64", MA_CORR_COLUMN: "column", MA_CORR_PAIRS: "colour_pairs"}

STATUS_NAMES = {0: "MA_OK", 1: "MA_ERR_INVALID_ARG", 2: "MA_ERR_OOM", 3: "MA_ERR_CUDA",
                4: "MA_ERR_NOT_CONVERGED", 5: "MA_ERR_NONFINITE"}


class MAError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class ma_hier_desc(C.Structure):
    _fields_ = [("n", C.c_int), ("x0", C.c_double * 3), ("len", C.c_double), ("nu1", C.c_int),
                ("nu2", C.c_int), ("coarsest_n", C.c_int), ("restrict_kind", C.c_int),
                ("approx_restrict", C.c_int), ("precision", C.c_int), ("coarse_sweeps", C.c_int),
                ("inner_cycles", C.c_int), ("fmg_interp", C.c_int)]


class ma_solve_opts(C.Structure):
    _fields_ = [("tol", C.c_double), ("norm", C.c_int), ("relative", C.c_int), ("max_cycles", C.c_int),
                ("init", C.c_int)]


class ma_solve_result(C.Structure):
    _fields_ = [("cycles", C.c_int), ("res0", C.c_double), ("res", C.c_double), ("status", C.c_int),
                ("floor_reached", C.c_int), ("nonconvex_root_events", C.c_longlong)]


_vp = C.c_void_p
_SIGS = {
    "ma_hierarchy_footprint": [C.POINTER(ma_hier_desc), C.POINTER(C.c_size_t)],
    "ma_create_hierarchy": [C.POINTER(ma_hier_desc), _vp, C.c_size_t, _vp, C.POINTER(_vp)],
    "ma_set_rhs_bc": [_vp, _vp, _vp],
    "ma_set_rhs_bc_host": [_vp, _vp, _vp],
    "ma_vcycle": [_vp, C.c_int],
    "ma_solve": [_vp, C.POINTER(ma_solve_opts), C.POINTER(ma_solve_result)],
    "ma_solve_begin": [_vp, C.POINTER(ma_solve_opts)],
    "ma_solve_advance": [_vp, C.POINTER(C.c_int)],
    "ma_solve_get_result": [_vp, C.POINTER(ma_solve_result)],
    "ma_batch_solve": [C.POINTER(_vp), C.c_int, C.POINTER(ma_solve_opts), C.POINTER(ma_solve_result)],
    "ma_batch_footprint": [C.POINTER(_vp), C.c_int, C.POINTER(C.c_size_t)],
    "ma_create_batch": [C.POINTER(_vp), C.c_int, _vp, C.c_size_t, _vp, C.POINTER(_vp)],
    "ma_batch_run": [_vp, C.POINTER(ma_solve_opts), C.POINTER(ma_solve_result)],
    "ma_destroy_batch": [_vp],
    "ma_set_batch_groups": [C.c_int],
    "ma_set_batch_start": [C.c_int],
    "ma_residual_norm": [_vp, C.c_int, C.POINTER(C.c_double)],
    "ma_get_solution": [_vp, _vp],
    "ma_get_solution_host": [_vp, _vp],
    "ma_set_solution": [_vp, _vp],
    "ma_hierarchy_info": [_vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_size_t)],
    "ma_destroy_hierarchy": [_vp],
    "ma_smooth": [_vp, _vp, C.c_int, C.c_double, C.c_int, _vp, _vp],
    "ma_residual": [_vp, _vp, _vp, C.c_int, C.c_double, _vp],
    "ma_residual_f2": [_vp, _vp, _vp, C.c_int, C.c_double, _vp],
    "ma_restrict_residual": [_vp, C.c_int, _vp, C.c_int, _vp],
    "ma_restrict_solution": [_vp, C.c_int, _vp, C.c_int, C.c_int, _vp],
    "ma_coarse_rhs": [_vp, _vp, _vp, C.c_int, C.c_double, _vp],
    "ma_prolong_add": [_vp, _vp, C.c_int, _vp, _vp],
    "ma_interpolate": [_vp, C.c_int, _vp, _vp],
    "ma_coarsest_solve": [_vp, _vp, C.c_int, C.c_double, C.c_int, _vp, _vp],
    "ma_norm_scratch_bytes": [C.c_int, C.POINTER(C.c_size_t)],
    "ma_norm": [_vp, C.c_int, C.c_double, _vp, C.c_size_t, C.POINTER(C.c_double), _vp],
    "ma_kernel_launch_count": [C.POINTER(C.c_ulonglong)],
    "ma_probe_fp64_rate": [C.POINTER(C.c_double), _vp],
    "ma_probe_phase_chain": [_vp, _vp, C.c_size_t, C.c_int, C.c_int, _vp, C.POINTER(C.c_double), _vp],
    "ma_correction_scratch_bytes": [C.c_int, C.POINTER(C.c_size_t)],
    "ma_smooth_correction": [_vp, _vp, _vp, _vp, C.c_int, C.c_double, C.c_int, _vp, C.c_size_t, _vp, _vp],
    "ma_smooth_correction_colour": [_vp, _vp, _vp, _vp, C.c_int, C.c_double, C.c_int, _vp, C.c_size_t, _vp, _vp],
    "ma_residual_correction": [_vp, _vp, _vp, _vp, _vp, C.c_int, C.c_double, _vp, C.c_size_t, _vp],
    "ma_norm_static": [_vp, C.c_int, C.c_double, C.POINTER(C.c_double), _vp],
    "ma_set_corr_tuning": [C.c_int, C.c_int, C.c_int],
    "ma_set_corr_tail": [C.c_int],
    "ma_set_vcycle_tail": [C.c_int],
    "ma2d_hierarchy_footprint": [C.c_void_p, C.POINTER(C.c_size_t)],
    "ma2d_create_hierarchy": [C.c_void_p, _vp, C.c_size_t, _vp, C.POINTER(_vp)],
    "ma2d_set_rhs_bc": [_vp, _vp, _vp],
    "ma2d_vcycle": [_vp, C.c_int],
    "ma2d_solve": [_vp, C.POINTER(ma_solve_opts), C.POINTER(ma_solve_result)],
    "ma2d_get_solution": [_vp, _vp],
    "ma2d_destroy_hierarchy": [_vp],
    "ma2d_smooth": [_vp, _vp, C.c_int, C.c_double, C.c_int, C.c_int, _vp, _vp, _vp],
    "ma2d_residual": [_vp, _vp, _vp, C.c_int, C.c_double, _vp],
    "ma2d_restrict_residual": [_vp, C.c_int, _vp, C.c_int, _vp],
    "ma2d_prolong_add": [_vp, _vp, C.c_int, _vp, _vp],
    "ma2d_interpolate": [_vp, C.c_int, _vp, C.c_int, _vp],
    "ma_interpolate_cubic_scratch_bytes": [C.c_int, C.POINTER(C.c_size_t)],
    "ma_interpolate_cubic": [_vp, C.c_int, _vp, _vp, C.c_size_t, _vp],
    "ma_get_corr_tuning": [C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)],
    "ma_tune_corr": [_vp, _vp, _vp, _vp, C.c_int, C.c_double, C.c_int, _vp, C.c_size_t, C.POINTER(C.c_double),
                     C.POINTER(C.c_double), _vp],
}
# Declared in include/ma.h; the test suite checks that the library exports them.
EXPORTED = sorted(list(_SIGS) + ["ma_last_error_string"])

_lib = None


def load():
    """Build (if stale) and load libma.so; raises if that is impossible."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(str(path))
        for name, args in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = C.c_int
        L.ma_last_error_string.argtypes = []
        L.ma_last_error_string.restype = C.c_char_p
        _lib = L
    return _lib


def _check(st: int) -> int:
    if st != MA_OK:
        msg = load().ma_last_error_string().decode(errors="replace")
        raise MAError(st, msg)
    return st


def _ptr(x) -> int | None:
    """Device address of a torch tensor (or an int address, or None)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if not x.is_cuda or not x.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return x.data_ptr()


def _host_ptr(x) -> int:
    """Host address of a contiguous CPU float64 array (numpy array or torch
    tensor, pinned or pageable)."""
    if hasattr(x, "is_cuda"):
        if x.is_cuda or not x.is_contiguous() or x.element_size() != 8:
            raise ValueError("expected a contiguous CPU float64 tensor")
        return x.data_ptr()
    if not (x.flags["C_CONTIGUOUS"] and x.dtype.itemsize == 8):
        raise ValueError("expected a C-contiguous float64 array")
    return x.ctypes.data


def _stream(s) -> int | None:
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


# ---- hierarchy ------------------------------------------------------------

def ma_hierarchy_footprint(desc: ma_hier_desc) -> int:
    b = C.c_size_t(0)
    _check(load().ma_hierarchy_footprint(C.byref(desc), C.byref(b)))
    return b.value


def ma_create_hierarchy(desc: ma_hier_desc, workspace, nbytes: int, stream=None) -> int:
    h = _vp()
    _check(load().ma_create_hierarchy(C.byref(desc), _ptr(workspace), nbytes, _stream(stream), C.byref(h)))
    return h.value


def ma_set_rhs_bc(hier: int, f, g) -> None:
    _check(load().ma_set_rhs_bc(hier, _ptr(f), _ptr(g)))


def ma_set_rhs_bc_host(hier: int, f, g) -> None:
    """f and g in host memory (numpy arrays or CPU tensors, n^3 float64)."""
    _check(load().ma_set_rhs_bc_host(hier, _host_ptr(f), _host_ptr(g)))


def ma_vcycle(hier: int, ncycles: int = 1) -> None:
    _check(load().ma_vcycle(hier, ncycles))


def ma_solve(hier: int, opts: ma_solve_opts, raise_on_error: bool = True) -> ma_solve_result:
    res = ma_solve_result()
    st = load().ma_solve(hier, C.byref(opts), C.byref(res))
    if raise_on_error:
        _check(st)
    return res


def ma_solve_begin(hier: int, opts: ma_solve_opts) -> None:
    _check(load().ma_solve_begin(hier, C.byref(opts)))


def ma_solve_advance(hier: int) -> bool:
    done = C.c_int(0)
    _check(load().ma_solve_advance(hier, C.byref(done)))
    return bool(done.value)


def ma_solve_get_result(hier: int, raise_on_error: bool = True) -> ma_solve_result:
    res = ma_solve_result()
    st = load().ma_solve_get_result(hier, C.byref(res))
    if raise_on_error:
        _check(st)
    return res


def ma_batch_solve(hiers, opts: ma_solve_opts, raise_on_error: bool = True):
    n = len(hiers)
    arr = (_vp * n)(*hiers)
    res = (ma_solve_result * n)()
    st = load().ma_batch_solve(arr, n, C.byref(opts), res)
    if raise_on_error:
        _check(st)
    return list(res)


def ma_batch_footprint(hiers) -> int:
    n = len(hiers)
    arr = (_vp * n)(*hiers)
    b = C.c_size_t(0)
    _check(load().ma_batch_footprint(arr, n, C.byref(b)))
    return b.value


def ma_create_batch(hiers, workspace, nbytes: int, stream=None) -> int:
    n = len(hiers)
    arr = (_vp * n)(*hiers)
    out = _vp()
    _check(load().ma_create_batch(arr, n, _ptr(workspace), nbytes, _stream(stream), C.byref(out)))
    return out.value


def ma_batch_run(batch: int, count: int, opts: ma_solve_opts, raise_on_error: bool = True):
    res = (ma_solve_result * count)()
    st = load().ma_batch_run(batch, C.byref(opts), res)
    if raise_on_error:
        _check(st)
    return list(res)


def ma_destroy_batch(batch: int) -> None:
    _check(load().ma_destroy_batch(batch))


def ma_set_batch_groups(groups: int) -> None:
    _check(load().ma_set_batch_groups(int(groups)))


def ma_set_batch_start(batched: bool) -> None:
    _check(load().ma_set_batch_start(1 if batched else 0))


def ma_residual_norm(hier: int, norm: int = MA_NORM_MAX) -> float:
    out = C.c_double(0.0)
    _check(load().ma_residual_norm(hier, norm, C.byref(out)))
    return out.value


def ma_get_solution(hier: int, u) -> None:
    _check(load().ma_get_solution(hier, _ptr(u)))


def ma_get_solution_host(hier: int, u) -> None:
    """u in host memory (numpy array or CPU tensor, n^3 float64); blocks."""
    _check(load().ma_get_solution_host(hier, _host_ptr(u)))


def ma_set_solution(hier: int, u) -> None:
    _check(load().ma_set_solution(hier, _ptr(u)))


def ma_hierarchy_info(hier: int):
    n, L, b = C.c_int(0), C.c_int(0), C.c_size_t(0)
    _check(load().ma_hierarchy_info(hier, C.byref(n), C.byref(L), C.byref(b)))
    return n.value, L.value, b.value


def ma_destroy_hierarchy(hier: int) -> None:
    _check(load().ma_destroy_hierarchy(hier))


def ma_kernel_launch_count() -> int:
    out = C.c_ulonglong(0)
    _check(load().ma_kernel_launch_count(C.byref(out)))
    return out.value


def ma_probe_fp64_rate(stream=None) -> float:
    """Measured FP64 DFMA operations per second of the current device."""
    out = C.c_double(0.0)
    _check(load().ma_probe_fp64_rate(C.byref(out), _stream(stream)))
    return out.value


def ma_probe_phase_chain(a, b, sync, phases: int, blocks_per_sm: int, stream=None) -> dict:
    """Per-phase cost (us) of a chain of dependent phases: a CUDA graph of
    launches (one element per thread, and a grid-stride grid of blocks_per_sm
    blocks per SM) and one cooperative kernel with grid barriers.  a, b: float32
    device tensors of n elements; sync: 3 int32 on the device."""
    if a.element_size() != 4 or b.element_size() != 4 or b.numel() != a.numel():
        raise ValueError("a, b: float32 device tensors of one size")
    if sync.element_size() != 4 or sync.numel() < 3:
        raise ValueError("sync: at least 3 int32 on the device")
    out = (C.c_double * 3)()
    _check(load().ma_probe_phase_chain(_ptr(a), _ptr(b), a.numel(), phases, blocks_per_sm, _ptr(sync), out,
                                       _stream(stream)))
    return {"graph_one_element_per_thread_us": out[0], "graph_grid_stride_us": out[1],
            "cooperative_barriers_us": out[2]}


def ma_last_error_string() -> str:
    return load().ma_last_error_string().decode(errors="replace")


# ---- single steps ---------------------------------------------------------

def ma_smooth(u, rhs, n: int, h: float, nsweeps: int = 1, events=None, stream=None) -> None:
    _check(load().ma_smooth(_ptr(u), _ptr(rhs), n, h, nsweeps, _ptr(events), _stream(stream)))


def ma_residual(u, rhs, r, n: int, h: float, stream=None) -> None:
    _check(load().ma_residual(_ptr(u), _ptr(rhs), _ptr(r), n, h, _stream(stream)))


def ma_residual_f2(u, rhs, r, n: int, h: float, stream=None) -> None:
    _check(load().ma_residual_f2(_ptr(u), _ptr(rhs), _ptr(r), n, h, _stream(stream)))


def ma_restrict_residual(rf, nf: int, rc, kind: int, stream=None) -> None:
    _check(load().ma_restrict_residual(_ptr(rf), nf, _ptr(rc), kind, _stream(stream)))


def ma_restrict_solution(uf, nf: int, uc, approx: int, kind: int, stream=None) -> None:
    _check(load().ma_restrict_solution(_ptr(uf), nf, _ptr(uc), approx, kind, _stream(stream)))


def ma_coarse_rhs(wc, rc, bc, nc: int, H: float, stream=None) -> None:
    _check(load().ma_coarse_rhs(_ptr(wc), _ptr(rc), _ptr(bc), nc, H, _stream(stream)))


def ma_prolong_add(uc, wc, nc: int, uf, stream=None) -> None:
    _check(load().ma_prolong_add(_ptr(uc), _ptr(wc), nc, _ptr(uf), _stream(stream)))


def ma_interpolate(uc, nc: int, uf, stream=None) -> None:
    _check(load().ma_interpolate(_ptr(uc), nc, _ptr(uf), _stream(stream)))


def ma_interpolate_cubic_scratch_bytes(nc: int) -> int:
    b = C.c_size_t(0)
    _check(load().ma_interpolate_cubic_scratch_bytes(nc, C.byref(b)))
    return b.value


def ma_interpolate_cubic(uc, nc: int, uf, scratch, scratch_bytes: int, stream=None) -> None:
    _check(load().ma_interpolate_cubic(_ptr(uc), nc, _ptr(uf), _ptr(scratch), scratch_bytes, _stream(stream)))


def ma_coarsest_solve(u, rhs, n: int, h: float, sweeps: int = 0, events=None, stream=None) -> None:
    _check(load().ma_coarsest_solve(_ptr(u), _ptr(rhs), n, h, sweeps, _ptr(events), _stream(stream)))


def ma_correction_scratch_bytes(n: int) -> int:
    b = C.c_size_t(0)
    _check(load().ma_correction_scratch_bytes(n, C.byref(b)))
    return b.value


def ma_smooth_correction(e, u_hi, u_lo, rhs, n: int, h: float, nsweeps: int, scratch, scratch_bytes: int,
                         events=None, stream=None) -> None:
    _check(load().ma_smooth_correction(_ptr(e), _ptr(u_hi), _ptr(u_lo), _ptr(rhs), n, h, nsweeps, _ptr(scratch),
                                       scratch_bytes, _ptr(events), _stream(stream)))


def ma_smooth_correction_colour(e, u_hi, u_lo, rhs, n: int, h: float, colour: int, scratch, scratch_bytes: int,
                                events=None, stream=None) -> None:
    _check(load().ma_smooth_correction_colour(_ptr(e), _ptr(u_hi), _ptr(u_lo), _ptr(rhs), n, h, colour,
                                              _ptr(scratch), scratch_bytes, _ptr(events), _stream(stream)))


def ma_residual_correction(e, u_hi, u_lo, rhs, res, n: int, h: float, scratch, scratch_bytes: int,
                           stream=None) -> None:
    _check(load().ma_residual_correction(_ptr(e), _ptr(u_hi), _ptr(u_lo), _ptr(rhs), _ptr(res), n, h,
                                         _ptr(scratch), scratch_bytes, _stream(stream)))


def correction_scratch(n: int, device=None):
    """A 256-byte-aligned uint8 CUDA buffer for the correction step calls: (tensor, address, bytes)."""
    import torch
    nb = ma_correction_scratch_bytes(n)
    t = torch.empty(nb + 256, dtype=torch.uint8, device=device or torch.device("cuda"))
    addr = (t.data_ptr() + 255) // 256 * 256
    return t, addr, nb


def ma_set_corr_tuning(n: int, smooth_choice: int, residual_choice: int) -> None:
    _check(load().ma_set_corr_tuning(n, smooth_choice, residual_choice))


def ma_set_corr_tail(max_n) -> None:
    """True / 1: the default; False / 0: level by level; 3, 5, 9, 17: the largest fused level."""
    _check(load().ma_set_corr_tail(int(max_n)))


def ma_set_vcycle_tail(max_n) -> None:
    """True / 1: the default; False / 0: level by level; 3, 5, 9, 17: the largest fused level."""
    _check(load().ma_set_vcycle_tail(int(max_n)))


def ma_get_corr_tuning(n: int):
    a, b = C.c_int(0), C.c_int(0)
    _check(load().ma_get_corr_tuning(n, C.byref(a), C.byref(b)))
    return a.value, b.value


def ma_tune_corr(e, u_hi, u_lo, rhs, n: int, h: float, reps: int, scratch, scratch_bytes: int, stream=None):
    """Runs the autotuner on one grid; returns (us_smooth[6], us_residual[5]) and records the fastest."""
    us = (C.c_double * 6)()
    ur = (C.c_double * 5)()
    _check(load().ma_tune_corr(_ptr(e), _ptr(u_hi), _ptr(u_lo), _ptr(rhs), n, h, reps, _ptr(scratch), scratch_bytes,
                               us, ur, _stream(stream)))
    return list(us), list(ur)


def autotune(sizes, reps: int = 5, device=None) -> dict:
    """Autotunes the correction smoother and residual for each grid size in
    `sizes` on Example 4 data (the base Hessian of u = exp(|x|^2/2), a small
    smooth correction and right-hand side) and records the fastest variants
    for this process.  Returns {n: {"smoother": name, "residual": name,
    "us_per_sweep": {...}, "us_residual": {...}}}."""
    import numpy as np
    import torch
    from . import problems
    dev = device or torch.device("cuda")
    out = {}
    for n in sorted(set(int(v) for v in sizes)):
        if n < 5:
            continue
        pr = problems.make("exp", n)
        u = torch.from_numpy(pr.u).to(dev)
        hi = u.float()
        lo = (u - hi.double()).float()
        x = torch.linspace(0.0, 1.0, n, device=dev, dtype=torch.float64)
        s = torch.sin(np.pi * x)
        e = (1e-6 * s[:, None, None] * s[None, :, None] * s[None, None, :]).float().contiguous()
        rhs = (1e-6 * torch.from_numpy(pr.f).to(dev)).float()
        rhs[0], rhs[-1] = 0, 0
        keep, scr, nb = correction_scratch(n, device=dev)
        us, ur = ma_tune_corr(e, hi, lo, rhs, n, pr.h, reps, scr, nb)
        torch.cuda.synchronize(dev)
        sm, rs = ma_get_corr_tuning(n)
        out[n] = {"smoother": CORR_NAMES[sm], "residual": CORR_NAMES[rs],
                  "us_per_sweep": {CORR_NAMES[c]: round(us[c], 2) for c in (0, 1, 2, 3, 5)},
                  "us_residual": {CORR_NAMES[c]: round(ur[c], 2) for c in range(1, 5)}}
        del keep, u, hi, lo, e, rhs
    return out


def level_sizes(n: int, coarsest_n: int = 3):
    """Grid sizes of the levels of a hierarchy on n points per side."""
    out = [n]
    while out[-1] > coarsest_n:
        out.append((out[-1] + 1) // 2)
    return out


def ma_norm_scratch_bytes(n: int) -> int:
    b = C.c_size_t(0)
    _check(load().ma_norm_scratch_bytes(n, C.byref(b)))
    return b.value


def ma_norm(v, n: int, h: float, scratch, scratch_bytes: int, stream=None):
    out = (C.c_double * 2)()
    _check(load().ma_norm(_ptr(v), n, h, _ptr(scratch), scratch_bytes, out, _stream(stream)))
    return out[0], out[1]


MA_NORM_STATIC_MAX_N = 513


def ma_norm_static(v, n: int, h: float, stream=None):
    """ma_norm without caller scratch: for callers that cannot allocate device
    memory (all of it owned by another allocator, or no implicit cudaMalloc
    synchronisation allowed).  n <= MA_NORM_STATIC_MAX_N; calls that overlap
    on the GPU race on the library's one fixed scratch array."""
    out = (C.c_double * 2)()
    _check(load().ma_norm_static(_ptr(v), n, h, out, _stream(stream)))
    return out[0], out[1]


# ---- convenience: a hierarchy whose workspace is a torch tensor --------------

@dataclass
class SolveResult:
    cycles: int
    res0: float
    res: float
    status: int
    floor_reached: bool
    nonconvex_root_events: int


def make_desc(n: int, length: float = 1.0, x0=(0.0, 0.0, 0.0), nu1: int = 2, nu2: int = 2,
              coarsest_n: int = 3, restrict_kind: int = MA_FULL_WEIGHTING,
              approx_restrict: int = MA_APPROX_WEIGHTED, precision: int = MA_FP64,
              coarse_sweeps: int = 0, inner_cycles: int = 0, fmg_interp: int = MA_FMG_CUBIC) -> ma_hier_desc:
    """A hierarchy description.  The FMG start interpolates with tricubic
    Lagrange polynomials (Algorithm 2 step 4) by default: its second
    differences carry O(h^2) error where trilinear ones carry O(1), so the
    first residual after FMG is ~1000x smaller (Example 4 at 257^3: 5e-9
    against 5e-6 after one outer iteration of the mixed solve).
    inner_cycles (mixed and FP32 modes; 0 = 3): FP32 correction V-cycles per
    FP64 residual.  3 suits small grids and batches; single solves from
    129^3 up run faster with 2, which checks the stopping rule every two
    cycles."""
    d = ma_hier_desc()
    d.n = n
    d.x0[0], d.x0[1], d.x0[2] = x0
    d.len = length
    d.nu1, d.nu2 = nu1, nu2
    d.coarsest_n = coarsest_n
    d.restrict_kind = restrict_kind
    d.approx_restrict = approx_restrict
    d.precision = precision
    d.coarse_sweeps = coarse_sweeps
    d.inner_cycles = inner_cycles
    d.fmg_interp = fmg_interp
    return d


def paper_desc(n: int, length: float = 1.0, precision: int = MA_FP64) -> ma_hier_desc:
    """The settings of Section 4 on the GPU: V(2,2), h0 = 1/2 (3^3) with one
    sweep, tricubic FMG interpolation; full-weighting restriction (the
    8-colour smoother diverges with half weighting from 33^3 up)."""
    return make_desc(n, length=length, coarsest_n=3, coarse_sweeps=1, precision=precision, fmg_interp=MA_FMG_CUBIC)


class Hierarchy:
    """Owns a torch uint8 workspace tensor and the hierarchy built in it."""

    def __init__(self, desc: ma_hier_desc, stream=None, device=None):
        import torch
        self.desc = desc
        self.nbytes = ma_hierarchy_footprint(desc)
        self.workspace = torch.empty(self.nbytes + 256, dtype=torch.uint8,
                                     device=device or torch.device("cuda"))
        base = self.workspace.data_ptr()
        aligned = (base + 255) // 256 * 256
        self.stream = stream
        self.handle = ma_create_hierarchy(desc, aligned, self.nbytes, stream)

    def set_rhs_bc(self, f, g):
        ma_set_rhs_bc(self.handle, f, g)

    def set_rhs_bc_host(self, f, g):
        ma_set_rhs_bc_host(self.handle, f, g)

    def vcycle(self, ncycles: int = 1):
        ma_vcycle(self.handle, ncycles)

    def solve(self, tol: float = 1e-10, norm: int = MA_NORM_MAX, relative=True,
              max_cycles: int = 50, init: int = MA_INIT_FMG, raise_on_error: bool = True) -> SolveResult:
        """relative: True / MA_REL_RHS (||f||), False / MA_REL_NONE, or MA_REL_INITIAL."""
        rel = int(relative) if not isinstance(relative, bool) else (MA_REL_RHS if relative else MA_REL_NONE)
        o = ma_solve_opts(tol, norm, rel, max_cycles, init)
        r = ma_solve(self.handle, o, raise_on_error)
        return SolveResult(r.cycles, r.res0, r.res, r.status, bool(r.floor_reached), r.nonconvex_root_events)

    def residual_norm(self, norm: int = MA_NORM_MAX) -> float:
        return ma_residual_norm(self.handle, norm)

    def get_solution(self, u):
        ma_get_solution(self.handle, u)

    def get_solution_host(self, u):
        ma_get_solution_host(self.handle, u)

    def set_solution(self, u):
        ma_set_solution(self.handle, u)

    def close(self):
        if self.handle:
            ma_destroy_hierarchy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Shared per-level batch over Hierarchy objects (ma_create_batch): owns
    its torch workspace; the hierarchies must stay open while it lives."""

    def __init__(self, hierarchies, stream=None, device=None):
        import torch
        self.hierarchies = list(hierarchies)
        handles = [h.handle for h in self.hierarchies]
        self.nbytes = ma_batch_footprint(handles)
        self.workspace = torch.empty(self.nbytes + 256, dtype=torch.uint8, device=device or torch.device("cuda"))
        aligned = (self.workspace.data_ptr() + 255) // 256 * 256
        self.handle = ma_create_batch(handles, aligned, self.nbytes, stream)

    def solve(self, tol: float = 1e-10, norm: int = MA_NORM_MAX, relative=True, max_cycles: int = 50,
              init: int = MA_INIT_FMG, raise_on_error: bool = True):
        rel = int(relative) if not isinstance(relative, bool) else (MA_REL_RHS if relative else MA_REL_NONE)
        o = ma_solve_opts(tol, norm, rel, max_cycles, init)
        rs = ma_batch_run(self.handle, len(self.hierarchies), o, raise_on_error)
        return [SolveResult(r.cycles, r.res0, r.res, r.status, bool(r.floor_reached), r.nonconvex_root_events)
                for r in rs]

    def close(self):
        if self.handle:
            ma_destroy_batch(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- the 2D version of the method (include/ma2d.h) ------------------------------

MA2D_REDBLACK, MA2D_COLOUR4 = 0, 2


class ma2d_desc(C.Structure):
    _fields_ = [("n", C.c_int), ("len", C.c_double), ("nu1", C.c_int), ("nu2", C.c_int), ("coarsest_n", C.c_int),
                ("restrict_kind", C.c_int), ("approx_restrict", C.c_int), ("coarse_sweeps", C.c_int),
                ("ordering", C.c_int), ("fmg_interp", C.c_int)]


def make_desc2d(n: int, length: float = 1.0, nu1: int = 2, nu2: int = 2, coarsest_n: int = 3,
                restrict_kind: int = MA_FULL_WEIGHTING, approx_restrict: int = MA_APPROX_WEIGHTED,
                coarse_sweeps: int = 0, ordering: int = MA2D_REDBLACK, fmg_interp: int = MA_FMG_TRILINEAR):
    return ma2d_desc(n, length, nu1, nu2, coarsest_n, restrict_kind, approx_restrict, coarse_sweeps, ordering,
                     fmg_interp)


def paper_desc2d(n: int, ordering: int = MA2D_REDBLACK):
    """Section 4's settings in 2D: V(2,2), h0 = 1/2 with one sweep, bicubic FMG,
    full weighting (the weighting the errors of Table 1 match)."""
    return make_desc2d(n, coarsest_n=3, coarse_sweeps=1, ordering=ordering, fmg_interp=MA_FMG_CUBIC)


class Hierarchy2D:
    """A 2D hierarchy in a torch-owned device workspace, on one stream."""

    def __init__(self, desc, stream=None, device=None):
        import torch
        self.desc = desc
        self.device = device or torch.device("cuda")
        b = C.c_size_t(0)
        _check(load().ma2d_hierarchy_footprint(C.byref(desc), C.byref(b)))
        self.nbytes = b.value
        self.ws = torch.empty(self.nbytes + 256, dtype=torch.uint8, device=self.device)
        addr = (self.ws.data_ptr() + 255) // 256 * 256
        self.stream = stream
        h = _vp()
        _check(load().ma2d_create_hierarchy(C.byref(desc), addr, self.nbytes, _stream(stream), C.byref(h)))
        self.handle = h.value

    def set_rhs_bc(self, f, g):
        _check(load().ma2d_set_rhs_bc(self.handle, _ptr(f), _ptr(g)))

    def vcycle(self, n: int = 1):
        _check(load().ma2d_vcycle(self.handle, n))

    def solve(self, tol: float = 1e-10, norm: int = MA_NORM_MAX, relative=True, max_cycles: int = 50,
              init: int = MA_INIT_FMG, raise_on_error: bool = True):
        rel = int(relative) if not isinstance(relative, bool) else (MA_REL_RHS if relative else MA_REL_NONE)
        o = ma_solve_opts(tol, norm, rel, max_cycles, init)
        r = ma_solve_result()
        st = load().ma2d_solve(self.handle, C.byref(o), C.byref(r))
        if raise_on_error:
            _check(st)
        return SolveResult(r.cycles, r.res0, r.res, r.status, bool(r.floor_reached), r.nonconvex_root_events)

    def get_solution(self, out):
        _check(load().ma2d_get_solution(self.handle, _ptr(out)))

    def close(self):
        if self.handle:
            _check(load().ma2d_destroy_hierarchy(self.handle))
            self.handle = None


def ma2d_smooth(u, rhs, n: int, h: float, nsweeps: int, ordering: int = MA2D_REDBLACK, scratch=None, events=None,
                stream=None):
    _check(load().ma2d_smooth(_ptr(u), _ptr(rhs), n, h, nsweeps, ordering, _ptr(scratch), _ptr(events),
                              _stream(stream)))


def ma2d_residual(u, rhs, r, n: int, h: float, stream=None):
    _check(load().ma2d_residual(_ptr(u), _ptr(rhs), _ptr(r), n, h, _stream(stream)))


def ma2d_restrict_residual(rf, nf: int, rc, kind: int = MA_FULL_WEIGHTING, stream=None):
    _check(load().ma2d_restrict_residual(_ptr(rf), nf, _ptr(rc), kind, _stream(stream)))


def ma2d_prolong_add(uc, wc, nc: int, uf, stream=None):
    _check(load().ma2d_prolong_add(_ptr(uc), _ptr(wc), nc, _ptr(uf), _stream(stream)))


def ma2d_interpolate(uc, nc: int, uf, cubic: bool = False, stream=None):
    _check(load().ma2d_interpolate(_ptr(uc), nc, _ptr(uf), 1 if cubic else 0, _stream(stream)))
