"""GPU parity of the mixed-precision path (FP32 correction cycles under an FP64
residual and update) against the FP64 CPU oracle.

The correction operator N(e) = det(D^2_h(u + e)) - det(D^2_h u) has a plain
definition, so its oracle is two FP64 oracle evaluations of the discrete
Monge-Ampere operator; a correction sweep is one oracle Gauss-Seidel sweep on
w = u + e with right-hand side det(D^2_h u) + rhs.  FP32 bounds: the
correction kernels carry ~1e-5 relative error in the base Hessian (hi/lo
split) and FP32 rounding of e, so they are compared relative to the size of
the quantity they compute.  Whole solves meet the same FP64 tolerance as the
FP64 path and are compared with the oracle at the FP64 bound (1e-10 relative).
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
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


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def split(u):
    hi = u.astype(np.float32)
    lo = (u - hi.astype(np.float64)).astype(np.float32)
    return hi, lo


def smooth_correction_field(n, amp, seed):
    x, y, z = P.grid_coords(n)
    rng = np.random.default_rng(seed)
    a = rng.uniform(0.5, 1.5, 3)
    e = amp * np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z) * (1 + a[0] * x + a[1] * y * z)
    e += 0.1 * amp * rng.standard_normal(e.shape)
    e[0], e[-1], e[:, 0], e[:, -1], e[:, :, 0], e[:, :, -1] = 0, 0, 0, 0, 0, 0
    return e.astype(np.float32)


@pytest.mark.parametrize("name,n,amp", [("exp", 33, 1e-4), ("cosine", 65, 1e-5), ("exp", 129, 1e-6)])
def test_correction_residual_matches_oracle_definition(name, n, amp):
    pr = P.make(name, n, seed=3)
    u = pr.u
    e = smooth_correction_field(n, amp, n)
    rng = np.random.default_rng(1)
    rhs = (1e-3 * rng.standard_normal(u.shape)).astype(np.float32)
    N_ref = O.discrete_ma(np.ascontiguousarray(u + e.astype(np.float64)), pr.h) - O.discrete_ma(u, pr.h)
    ref = rhs.astype(np.float64) - N_ref
    ref[0], ref[-1], ref[:, 0], ref[:, -1], ref[:, :, 0], ref[:, :, -1] = 0, 0, 0, 0, 0, 0
    hi, lo = split(u)
    res = torch.empty(u.shape, dtype=torch.float32, device="cuda")
    _keep, scr, nb = M.correction_scratch(n)
    M.ma_residual_correction(dev(e), dev(hi), dev(lo), dev(rhs), res, n, pr.h, scr, nb)
    got = host(res).astype(np.float64)
    inner = (slice(1, -1),) * 3
    scale = np.max(np.abs(N_ref[inner])) + np.max(np.abs(rhs))
    assert np.max(np.abs(got - ref)) <= 2e-4 * scale


@pytest.mark.parametrize("pairs", [False, True])
@pytest.mark.parametrize("name,n,amp", [("exp", 33, 1e-4), ("cosine", 65, 1e-5), ("exp", 129, 1e-6),
                                        ("exp", 45, 1e-5)])
def test_correction_sweep_matches_oracle_sweep(name, n, amp, pairs):
    """One correction sweep against the oracle's Gauss-Seidel sweep on
    w = u + e with right-hand side det(D^2_h u) + rhs, in the regime the
    inner cycles run in (|rhs| ~ 1e-5 |f|, corrections of that order).  The
    kernel's base Hessian comes from the FP32 hi/lo split (~1e-5 relative),
    and e is FP32.  pairs: the colour-pair sweep (colours c and c^7 in one
    launch) against the oracle's sweep in the colour order 0, 7, 1, 6, 2, 5,
    3, 4; otherwise the by-colour sweep against ascending colours."""
    pr = P.make(name, n, seed=4)
    u = pr.u
    e = smooth_correction_field(n, amp, n + 1)
    rng = np.random.default_rng(2)
    rhs = (1e-5 * rng.standard_normal(u.shape) * np.max(pr.f)).astype(np.float32)
    rhs[0], rhs[-1] = 0, 0
    w = np.ascontiguousarray(u + e.astype(np.float64))
    ftot = O.discrete_ma(u, pr.h) + rhs.astype(np.float64)
    O.gs_sweep(w, ftot, pr.h, O.COLOUR8_PAIRS if pairs else O.COLOUR8)
    e_ref = w - u
    hi, lo = split(u)
    ed = dev(e)
    _keep, scr, nb = M.correction_scratch(n)
    try:
        M.ma_set_corr_tuning(n, M.MA_CORR_PAIRS if pairs else M.MA_CORR_BY_COLOUR, -1)
        M.ma_smooth_correction(ed, dev(hi), dev(lo), dev(rhs), n, pr.h, 1, scr, nb)
        got = host(ed).astype(np.float64)
    finally:
        M.ma_set_corr_tuning(n, -1, -1)
    change = np.max(np.abs(e_ref - e.astype(np.float64)))
    assert change > 0
    assert np.max(np.abs(got - e_ref)) <= 1e-3 * change + 1e-6 * np.max(np.abs(e_ref))


# ---- large corrections: a bound derived from the FP32 rounding model ----------
#
# The kernel and the oracle solve the same point equation
#     det(B + K - z I) - det(B) = r,   e_new = e_old + h^2 z / 2,
# with B = D^2_h u, K = D^2_h e; the oracle in FP64 on w = u + e, the kernel
# in FP32 with B from the FP32 hi/lo split of u.  The inputs e are the same
# FP32 values on both sides.  To first order the kernel's root differs from
# the oracle's by
#   dz = [ tr((cof G_z - cof B) dB) + tr(cof(G_z) dK) + dF ] / M(G_z),
# G_z = B + K - z I at the root, M = tr cof G_z = -dF/dz, where
#   dB, dK: FP32 rounding of the second differences, at most
#           4 u (sum of |first differences| / h^2 + |entry|) per entry
#           (u = 2^-24; the split's hi differences, the lo part, two sums and
#           the 1/h^2 scaling each round once);
#   dF:     FP32 evaluation of F = c - M z + T z^2 - z^3 with
#           c = tr(cof(B)K) + tr(B cof K) + det K - r: at most 16 u times the
#           sum of the magnitudes of its terms, plus 1e-7 |z| for the
#           Newton stop (a step <= 1e-4 |z| leaves ~(1e-4)^2 |z|).
# e_new adds one FP32 rounding, u |e_new|.  Within a sweep a point reads the
# new values of the colours before it, so their errors enter its K: with
# weights |cof_qq| / (2|M|) per face neighbour and |cof_pq| / (4|M|) per edge
# neighbour (the linearised update).  The bound D is propagated colour by
# colour in the sweep's order, with G_z taken at the moment of the update
# (the oracle's new values on the colours already swept, the old ones
# elsewhere), and the test allows 2 D for the first-order approximation.

_U32 = 2.0 ** -24
_SYM = np.array([1.0, 1.0, 1.0, 2.0, 2.0, 2.0])   # off-diagonal entries count twice
_FACES = [((0, 0, 1), 0), ((0, 0, -1), 0), ((0, 1, 0), 1), ((0, -1, 0), 1), ((1, 0, 0), 2), ((-1, 0, 0), 2)]
_EDGES = ([((0, s, t), 3) for s in (1, -1) for t in (1, -1)] + [((s, 0, t), 4) for s in (1, -1) for t in (1, -1)]
          + [((s, t, 0), 5) for s in (1, -1) for t in (1, -1)])


def _cof6(A):
    xx, yy, zz, xy, xz, yz = A
    return np.stack([yy * zz - yz * yz, xx * zz - xz * xz, xx * yy - xy * xy,
                     xz * yz - xy * zz, xy * yz - xz * yy, xy * xz - xx * yz])


def _shift(a, off):
    """a at interior point + off (zero on the shell)."""
    dk, dj, di = off
    n = a.shape[0]
    out = np.zeros_like(a)
    out[1:-1, 1:-1, 1:-1] = a[1 + dk:n - 1 + dk, 1 + dj:n - 1 + dj, 1 + di:n - 1 + di]
    return out


def _diff_sums(v, h):
    """Per Hessian entry, the sum of |v(neighbour) - v(centre)| that enters it,
    scaled as the entry (1/h^2 faces, 1/(4 h^2) edges)."""
    out = np.zeros((6,) + v.shape)
    for off, q in _FACES:
        out[q] += np.abs(_shift(v, off) - v) / h ** 2
    for off, q in _EDGES:
        out[q] += np.abs(_shift(v, off) - v) / (4 * h ** 2)
    out[:, 0], out[:, -1], out[:, :, 0], out[:, :, -1], out[:, :, :, 0], out[:, :, :, -1] = 0, 0, 0, 0, 0, 0
    return out


def correction_sweep_bound(u, e, e_ref, rhs, h, order):
    """Per-point bound D on |kernel - oracle| after one correction sweep in
    the colour order `order` (see the derivation above)."""
    n = u.shape[0]
    k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    colour = (i & 1) | ((j & 1) << 1) | ((k & 1) << 2)
    interior = np.zeros((n,) * 3, bool)
    interior[1:-1, 1:-1, 1:-1] = True
    e64 = e.astype(np.float64)
    B = O.discrete_hessian(np.ascontiguousarray(u), h)
    cB = _cof6(B)
    dB = 4 * _U32 * (_diff_sums(u, h) + np.abs(B))
    z = 2 * (e_ref - e64) / h ** 2
    D = np.zeros((n,) * 3)
    done = np.zeros((n,) * 3, bool)
    for c in order:
        m = (colour == c) & interior
        before = np.where(done, e_ref, e64)
        at = np.where(done | m, e_ref, e64)
        Y = O.discrete_hessian(np.ascontiguousarray(at), h)
        K0 = O.discrete_hessian(np.ascontiguousarray(before), h)
        cG = _cof6(B + Y)
        aM = np.where(m, np.abs(cG[0] + cG[1] + cG[2]), 1.0)
        dK = 4 * _U32 * (_diff_sums(at, h) + np.abs(Y))
        zB = (_SYM[:, None, None, None] * np.abs(cG - cB) * dB).sum(0) / aM
        zK = (_SYM[:, None, None, None] * np.abs(cG) * dK).sum(0) / aM
        bm, km, gm = np.abs(B).max(0), np.abs(K0).max(0), np.abs(B + K0).max(0)
        terms = (18 * (bm * bm * km + bm * km * km + km ** 3) + np.abs(rhs)
                 + 3 * gm * gm * np.abs(z) + 3 * gm * z * z + np.abs(z) ** 3)
        zF = 16 * _U32 * terms / aM + 1e-7 * np.abs(z)
        own = h * h / 2 * (zB + zK + zF) + _U32 * np.abs(e_ref)
        prop = np.zeros((n,) * 3)
        for off, q in _FACES:
            prop += np.abs(cG[q]) / (2 * aM) * _shift(D, off)
        for off, q in _EDGES:
            prop += np.abs(cG[q]) / (4 * aM) * _shift(D, off)
        D = np.where(m, own + prop, D)
        done |= m
    return D


@pytest.mark.parametrize("pairs", [False, True])
@pytest.mark.parametrize("name,n,kamp,nonconvex", [("exp", 33, 1.5, False), ("exp", 45, 1.5, False),
                                                   ("cosine", 65, 0.5, False), ("exp", 71, 1.0, False),
                                                   ("exp", 33, 0.5, True), ("cosine", 65, 0.5, True)])
def test_correction_sweep_large_corrections_match_oracle_within_derived_bound(name, n, kamp, nonconvex, pairs):
    """One correction sweep far from convergence, against the oracle's
    Gauss-Seidel sweep on w = u + e (right-hand side det(D^2_h u) + rhs),
    element by element within the bound derived above: a rough e whose
    K = D^2_h e is as large as B (G = B + K indefinite at many points, so the
    FP64 fallback runs), rhs = 1e-2 f, and with `nonconvex` 2 % of scattered
    points at rhs = -2 f, where det(B) + rhs <= 0 takes the smallest-real-
    root branch; the count of those updates equals the oracle's.  Sizes with
    several blocks per colour box and ragged last blocks (45, 71)."""
    pr = P.make(name, n, seed=4)
    u, h = pr.u, pr.h
    rng = np.random.default_rng(n)
    Bd = O.discrete_hessian(u, h)
    scale = np.median(np.abs(Bd[:3, 1:-1, 1:-1, 1:-1]))
    e = np.zeros(u.shape, dtype=np.float32)
    e[1:-1, 1:-1, 1:-1] = (kamp * h * h * scale / 4 * rng.standard_normal((n - 2,) * 3)).astype(np.float32)
    rhs = (1e-2 * rng.standard_normal(u.shape) * pr.f).astype(np.float32)
    if nonconvex:
        pick = rng.random(u.shape) < 0.02
        rhs[pick] = (-2.0 * pr.f[pick]).astype(np.float32)
    rhs[0], rhs[-1], rhs[:, 0], rhs[:, -1], rhs[:, :, 0], rhs[:, :, -1] = 0, 0, 0, 0, 0, 0
    K = O.discrete_hessian(e.astype(np.float64), h)
    assert np.abs(K).max() >= 0.3 * np.abs(Bd).max()
    order = (0, 7, 1, 6, 2, 5, 3, 4) if pairs else tuple(range(8))
    w = np.ascontiguousarray(u + e.astype(np.float64))
    ftot = O.discrete_ma(u, h) + rhs.astype(np.float64)
    ev_ref = O.gs_sweep(w, ftot, h, O.COLOUR8_PAIRS if pairs else O.COLOUR8)
    e_ref = w - u
    hi, lo = split(u)
    ed = dev(e)
    ev = torch.zeros(1, dtype=torch.int64, device="cuda")
    _keep, scr, nb = M.correction_scratch(n)
    try:
        M.ma_set_corr_tuning(n, M.MA_CORR_PAIRS if pairs else M.MA_CORR_BY_COLOUR, -1)
        M.ma_smooth_correction(ed, dev(hi), dev(lo), dev(rhs), n, h, 1, scr, nb, events=ev)
        got = host(ed).astype(np.float64)
    finally:
        M.ma_set_corr_tuning(n, -1, -1)
    assert int(ev.item()) == ev_ref and (ev_ref > 0) == nonconvex
    D = correction_sweep_bound(u, e, e_ref, rhs, h, order)
    err = np.abs(got - e_ref)
    change = np.max(np.abs(e_ref - e.astype(np.float64)))
    worst = np.unravel_index(np.argmax(err - 2 * D), err.shape)
    assert np.all(err <= 2 * D), (f"max err {err.max():.3e} (change {change:.3e}); at {worst}: "
                                  f"err {err[worst]:.3e} > 2 D = {2 * D[worst]:.3e}")
    # the bound is tight enough to mean something: far below the sweep's change
    assert 2 * D.max() <= 2e-3 * change


@pytest.mark.parametrize("name,n", [("exp", 33), ("cosine", 129), ("exp", 257), ("exp", 37), ("cosine", 71),
                                    ("exp", 135)])   # ragged last tiles for every tile size
def test_plane_sweeps_equal_colour_sweeps_bitwise(name, n):
    """Pairs of sweeps run by k parity (two launches per sweep, plane tiles
    of 16, 32 or 64 points that recompute a halo, a second e buffer) give the
    same bits as sweeps run colour by colour in place: all are the
    sequential 8-colour sweep.  At 129^3 and 257^3 every tile size has
    several tiles per plane edge."""
    pr = P.make(name, n, seed=6)
    u = pr.u
    e = smooth_correction_field(n, 1e-5, n + 2)
    rng = np.random.default_rng(3)
    rhs = (1e-5 * rng.standard_normal(u.shape) * np.max(pr.f)).astype(np.float32)
    hi, lo = (dev(a) for a in split(u))
    rhs_d = dev(rhs)
    _keep, scr, nb = M.correction_scratch(n)
    try:
        M.ma_set_corr_tuning(n, M.MA_CORR_BY_COLOUR, -1)
        refs = {}
        for sweeps in (2, 3):
            b = dev(e)
            for _ in range(sweeps):
                M.ma_smooth_correction(b, hi, lo, rhs_d, n, pr.h, 1, scr, nb)
            refs[sweeps] = b
        for choice in (M.MA_CORR_PLANE16, M.MA_CORR_PLANE32, M.MA_CORR_PLANE64):
            M.ma_set_corr_tuning(n, choice, -1)
            for sweeps in (2, 3):
                a = dev(e)
                M.ma_smooth_correction(a, hi, lo, rhs_d, n, pr.h, sweeps, scr, nb)
                torch.cuda.synchronize()
                assert not torch.equal(a, dev(e))
                d = (a - refs[sweeps]).abs().max().item()
                assert torch.equal(a, refs[sweeps]), f"{M.CORR_NAMES[choice]}, {sweeps} sweeps: max diff {d}"
    finally:
        M.ma_set_corr_tuning(n, -1, -1)


@pytest.mark.parametrize("n", [71, 129, 65])
def test_colour_pair_sweep_equals_its_colour_sequence_on_slow_points(n):
    """The colour-pair sweep (colours c and c^7 in one launch) is the
    sequential sweep in the order 0, 7, 1, 6, 2, 5, 3, 4: the same bits as
    the by-colour launches run in that order, here where the FP32 fast path
    fails.  A rough correction (K of the size of B) leaves G = B + K
    indefinite at many points, and a right-hand side of -2 f at scattered
    points makes det(B) + r <= 0 (the nonconvex branch); e and the count of
    nonconvex points agree bit for bit."""
    pr = P.make("exp", n, seed=2)
    rng = np.random.default_rng(n)
    e = np.zeros(pr.u.shape, dtype=np.float32)
    e[1:-1, 1:-1, 1:-1] = (0.5 * pr.h ** 2 * rng.standard_normal((n - 2,) * 3)).astype(np.float32)
    rhs = (1e-3 * rng.standard_normal(pr.u.shape) * pr.f).astype(np.float32)
    pick = rng.random(pr.u.shape) < 0.02
    rhs[pick] = (-2.0 * pr.f[pick]).astype(np.float32)
    rhs[0], rhs[-1], rhs[:, 0], rhs[:, -1], rhs[:, :, 0], rhs[:, :, -1] = 0, 0, 0, 0, 0, 0
    hi, lo = (dev(a) for a in split(pr.u))
    rhs_d = dev(rhs)
    _keep, scr, nb = M.correction_scratch(n)
    try:
        M.ma_set_corr_tuning(n, M.MA_CORR_PAIRS, -1)
        ed = dev(e)
        ev = torch.zeros(1, dtype=torch.int64, device="cuda")
        M.ma_smooth_correction(ed, hi, lo, rhs_d, n, pr.h, 2, scr, nb, events=ev)
        got = (host(ed), int(ev.item()))
    finally:
        M.ma_set_corr_tuning(n, -1, -1)
    ref = dev(e)
    ev = torch.zeros(1, dtype=torch.int64, device="cuda")
    for _ in range(2):
        for c in (0, 7, 1, 6, 2, 5, 3, 4):
            M.ma_smooth_correction_colour(ref, hi, lo, rhs_d, n, pr.h, c, scr, nb, events=ev)
    assert got[1] > 0 and got[1] == int(ev.item())
    assert np.array_equal(got[0], host(ref), equal_nan=True)
    assert not np.array_equal(got[0], e)


@pytest.mark.parametrize("n", [129, 257])
def test_colour_pair_sweep_on_an_unaligned_correction_grid_gives_the_same_bits(n):
    """At 129^3 and up the colour-pair kernel is compiled for the grid size and
    reads the neighbour pairs its colour aligns as 8-byte loads; an e that is
    not 8-byte aligned goes to the generic kernel (4-byte loads, the size at
    run time).  Both run the same arithmetic: e and the count of nonconvex
    points must agree bit for bit."""
    pr = P.make("exp", n, seed=3)
    rng = np.random.default_rng(7 * n)
    e = np.zeros(pr.u.shape, dtype=np.float32)
    e[1:-1, 1:-1, 1:-1] = (0.5 * pr.h ** 2 * rng.standard_normal((n - 2,) * 3)).astype(np.float32)
    rhs = (1e-3 * rng.standard_normal(pr.u.shape) * pr.f).astype(np.float32)
    pick = rng.random(pr.u.shape) < 0.02
    rhs[pick] = (-2.0 * pr.f[pick]).astype(np.float32)
    rhs[0], rhs[-1], rhs[:, 0], rhs[:, -1], rhs[:, :, 0], rhs[:, :, -1] = 0, 0, 0, 0, 0, 0
    hi, lo = (dev(a) for a in split(pr.u))
    rhs_d = dev(rhs)
    _keep, scr, nb = M.correction_scratch(n)
    m = n ** 3
    outs = []
    try:
        M.ma_set_corr_tuning(n, M.MA_CORR_PAIRS, -1)
        for offset in (0, 1):
            store = torch.zeros(m + 2, dtype=torch.float32, device="cuda")
            ed = store[offset:offset + m].view(n, n, n)
            ed.copy_(dev(e))
            assert (ed.data_ptr() % 8 == 0) == (offset == 0)
            ev = torch.zeros(1, dtype=torch.int64, device="cuda")
            M.ma_smooth_correction(ed, hi, lo, rhs_d, n, pr.h, 2, scr, nb, events=ev)
            outs.append((host(ed), int(ev.item())))
    finally:
        M.ma_set_corr_tuning(n, -1, -1)
    assert outs[0][1] == outs[1][1] and outs[0][1] > 0
    assert np.array_equal(outs[0][0], outs[1][0], equal_nan=True)
    assert not np.array_equal(outs[0][0], e)


@pytest.mark.parametrize("n", [129, 71, 33, 257, 9])
@pytest.mark.parametrize("choice", [1, 2, 3, 4])
def test_residual_tiles_agree(choice, n):
    """The three residual tile sizes and the column kernel compute the same
    values (the same arithmetic per point), with a zero shell; sizes whose
    interior is not a multiple of the 30-point column span or the tiles."""
    pr = P.make("cosine", n, seed=7)
    e = smooth_correction_field(n, 1e-5, 11)
    rng = np.random.default_rng(4)
    rhs = (1e-5 * rng.standard_normal(pr.u.shape)).astype(np.float32)
    hi, lo = (dev(a) for a in split(pr.u))
    _keep, scr, nb = M.correction_scratch(n)
    outs = []
    try:
        for c in (M.MA_CORR_PLANE64, choice):
            M.ma_set_corr_tuning(n, -1, c)
            res = torch.full(pr.u.shape, 7.0, dtype=torch.float32, device="cuda")
            M.ma_residual_correction(dev(e), hi, lo, dev(rhs), res, n, pr.h, scr, nb)
            outs.append(host(res))
    finally:
        M.ma_set_corr_tuning(n, -1, -1)
    assert np.array_equal(outs[0], outs[1])
    sh = outs[1]
    assert np.all(sh[0] == 0) and np.all(sh[-1] == 0) and np.all(sh[:, 0] == 0) and np.all(sh[:, :, -1] == 0)


def test_autotune_records_a_choice_per_size():
    table = M.autotune([17, 33, 65], reps=2)
    try:
        for n in (17, 33, 65):
            t = table[n]
            sm, rs = M.ma_get_corr_tuning(n)
            assert M.CORR_NAMES[sm] == t["smoother"] and M.CORR_NAMES[rs] == t["residual"]
            assert t["us_per_sweep"][t["smoother"]] == min(t["us_per_sweep"].values())
            assert all(v > 0 for v in t["us_per_sweep"].values())
    finally:
        for n in (17, 33, 65):
            M.ma_set_corr_tuning(n, -1, -1)


@pytest.mark.parametrize("name,n", [("exp", 33), ("cosine", 65), ("exp", 129), ("quadratic", 65), ("sine", 65)])
def test_mixed_solve_matches_fp64_oracle(name, n):
    pr = P.make(name, n, seed=5)
    H = M.Hierarchy(M.make_desc(n, length=pr.length, precision=M.MA_MIXED))
    H.set_rhs_bc(dev(pr.f), dev(pr.initial()))
    res = H.solve(tol=1e-10, max_cycles=40)
    u = torch.empty_like(dev(pr.f))
    H.get_solution(u)
    got = host(u)
    H.close()
    ref = pr.initial()
    O.solve(ref, pr.f, pr.h, tol=1e-10, params=O.Params())
    assert res.res <= 1e-10
    assert np.max(np.abs(got - ref)) <= 1e-10 * np.max(np.abs(ref))
    e_gpu, e_ref = np.max(np.abs(got - pr.u)), np.max(np.abs(ref - pr.u))
    assert abs(e_gpu - e_ref) <= 1e-3 * e_ref + 1e-12 * np.max(np.abs(ref))


def test_mixed_and_fp64_agree_at_257():
    pr = P.make("exp", 257)
    outs = {}
    for prec in (M.MA_FP64, M.MA_MIXED):
        H = M.Hierarchy(M.make_desc(257, precision=prec))
        H.set_rhs_bc(dev(pr.f), dev(pr.initial()))
        r = H.solve(tol=1e-10, max_cycles=40)
        assert r.res <= 1e-10
        u = torch.empty_like(dev(pr.f))
        H.get_solution(u)
        outs[prec] = host(u)
        H.close()
    assert np.max(np.abs(outs[M.MA_FP64] - outs[M.MA_MIXED])) <= 1e-10 * np.max(np.abs(pr.u))
    r = O.residual(outs[M.MA_MIXED], pr.f, pr.h)
    assert np.max(np.abs(r)) <= 1.5e-10 * np.max(np.abs(pr.f[1:-1, 1:-1, 1:-1]))


@pytest.mark.parametrize("choice", [M.MA_CORR_BY_COLOUR, M.MA_CORR_PLANE16])
def test_fused_tail_follows_each_levels_tuned_sweep_order(choice):
    """The fused correction tail sweeps each of its levels in the order that
    level's own sweep uses (colour pairs by default, ascending for the
    by-colour and plane variants).  With the tail levels tuned to an
    ascending variant, the tail must still give the bits, cycle count and
    residual of the level-by-level cycle, and those must differ from the
    colour-pair default (the order matters)."""
    n = 33
    pr = P.make("exp", n)
    runs = {}
    try:
        for tuned in (False, True):
            for sz in (5, 9, 17):
                M.ma_set_corr_tuning(sz, choice if tuned else -1, -1)
            outs = []
            for max_n in (17, 9, 0):
                M.ma_set_corr_tail(max_n)
                H = M.Hierarchy(M.make_desc(n, length=pr.length, precision=M.MA_MIXED))
                H.set_rhs_bc(dev(pr.f), dev(pr.initial()))
                r = H.solve(tol=1e-10, max_cycles=40, raise_on_error=False)
                u = torch.empty_like(dev(pr.f))
                H.get_solution(u)
                outs.append((host(u), r.cycles, r.res))
                H.close()
            runs[tuned] = outs
    finally:
        M.ma_set_corr_tail(True)
        for sz in (5, 9, 17):
            M.ma_set_corr_tuning(sz, -1, -1)
    for outs in runs.values():
        for u, cycles, res in outs[:-1]:
            assert cycles == outs[-1][1] and res == outs[-1][2]
            assert np.array_equal(u, outs[-1][0])
    assert not np.array_equal(runs[True][-1][0], runs[False][-1][0])


@pytest.mark.parametrize("precision", [M.MA_MIXED, M.MA_FP32])
@pytest.mark.parametrize("name,n,coarsest", [("exp", 65, 3), ("cosine", 17, 3), ("exp", 33, 5), ("sine", 129, 3)])
def test_fused_tail_cycle_is_bitwise_the_level_by_level_cycle(name, n, coarsest, precision):
    """The levels with n <= 17 (9, 5) run as one single-block launch; the
    solve gives the same bits and cycle count as the level-by-level launches."""
    pr = P.make(name, n)
    outs = []
    try:
        for max_n in (17, 9, 5, 0):
            M.ma_set_corr_tail(max_n)
            H = M.Hierarchy(M.make_desc(n, length=pr.length, precision=precision, coarsest_n=coarsest))
            H.set_rhs_bc(dev(pr.f), dev(pr.initial()))
            r = H.solve(tol=1e-10 if precision == M.MA_MIXED else 1e-12, max_cycles=40, raise_on_error=False)
            u = torch.empty_like(dev(pr.f))
            H.get_solution(u)
            outs.append((host(u), r.cycles, r.res))
            H.close()
    finally:
        M.ma_set_corr_tail(True)
    for u, cycles, res in outs[:-1]:
        assert cycles == outs[-1][1] and res == outs[-1][2]
        assert np.array_equal(u, outs[-1][0])
