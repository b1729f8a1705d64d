"""Seeded synthetic Monge-Ampere problems (exact solution u and f = det D^2 u).

This module holds only problem definitions: closed-form solutions and their
analytic right-hand sides, sampled on the grid.  It contains none of the
solver's arithmetic and serves both the CUDA path (benchmark, smoke check) and
the oracle-based tests.

Grids follow Section 2 of the paper: n = N + 1 points per side, h = len / N,
point (i, j, k) at x0 + (i h, j h, k h); arrays are float64 of shape
(n, n, n) indexed [k, j, i].

Examples (Section 4):
  * ``exp``        Example 4: u = exp(|x|^2/2), f = (1 + |x|^2) exp(3|x|^2/2).
  * ``quadratic``  u = |x|^2/2, f = 1 (the centred scheme is exact for it).
  * ``sine``       Example 5 on (0, pi)^3: u = -sum sin x_a + |x|^2/2,
                   f = prod (sin x_a + 1).
  * ``ex6``        Example 6: u = |x|^{3/2} / 3, f = |x|^{-3/2} / 16 (singular at
                   the corner x = 0, a boundary point).
  * ``ex7``        Example 7: u = -sqrt(3 - |x|^2), f = 3 (3 - |x|^2)^{-5/2}
                   (unbounded gradient at the corner x = (1, 1, 1)).
  * ``cosine``     |x|^2/2 plus eight seeded cosine modes (a synthetic
                   perturbation used for the GPU workloads; not in the paper):
                   u = |x|^2/2 + sum_m e_m / (4 pi^2 |k_m|^2) cos(2 pi k_m.x + phi_m)
                   with k_m uniform in {1,2,3}^3, phi_m uniform in [0, 2 pi) and
                   amplitude e_m.  Then D^2 u = I - sum_m e_m cos(theta_m) k^_m k^_m^T
                   (k^ = k/|k|) has smallest eigenvalue >= 1 - sum e_m > 0, so u
                   is convex, and f = det(D^2 u) is evaluated from that matrix.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Problem:
    name: str
    n: int
    x0: tuple = (0.0, 0.0, 0.0)
    length: float = 1.0
    u: np.ndarray = field(repr=False, default=None)   # exact solution on the grid
    f: np.ndarray = field(repr=False, default=None)   # right-hand side on the grid

    @property
    def h(self) -> float:
        return self.length / (self.n - 1)

    @property
    def unknowns(self) -> int:
        return (self.n - 2) ** 3

    def initial(self) -> np.ndarray:
        """Dirichlet data g = u on the shell, zero interior."""
        g = self.u.copy()
        g[1:-1, 1:-1, 1:-1] = 0.0
        return g


def grid_coords(n: int, x0=(0.0, 0.0, 0.0), length: float = 1.0):
    h = length / (n - 1)
    t = np.arange(n, dtype=np.float64) * h
    z, y, x = np.meshgrid(x0[2] + t, x0[1] + t, x0[0] + t, indexing="ij")
    return x, y, z


def cosine_modes(seed: int, eps: float | tuple = 0.02, modes: int = 8):
    """Seeded cosine-mode parameters: k (modes, 3) ints in {1,2,3}, phi, amplitudes."""
    rng = np.random.default_rng(seed)
    k = rng.integers(1, 4, size=(modes, 3))
    phi = rng.uniform(0.0, 2.0 * np.pi, size=modes)
    if isinstance(eps, tuple):
        amp = np.full(modes, rng.uniform(eps[0], eps[1]))
    else:
        amp = np.full(modes, float(eps))
    return k, phi, amp


def _cosine_fields(xp, x, y, z, k, phi, amp):
    """u = |x|^2/2 + sum_m amp_m / (4 pi^2 |k_m|^2) cos(theta_m) and
    f = det(I - sum_m amp_m cos(theta_m) k^_m k^_m^T), theta_m = 2 pi k_m.x + phi_m,
    with array module xp (numpy or torch)."""
    u = (x * x + y * y + z * z) / 2.0
    hxx = xp.ones_like(u); hyy = xp.ones_like(u); hzz = xp.ones_like(u)
    hxy = xp.zeros_like(u); hxz = xp.zeros_like(u); hyz = xp.zeros_like(u)
    for m in range(k.shape[0]):
        km = [float(v) for v in k[m]]
        kk = km[0] ** 2 + km[1] ** 2 + km[2] ** 2
        c = xp.cos(2.0 * np.pi * (km[0] * x + km[1] * y + km[2] * z) + float(phi[m]))
        u = u + (float(amp[m]) / (4.0 * np.pi ** 2 * kk)) * c
        w = (float(amp[m]) / kk) * c
        hxx = hxx - (km[0] * km[0]) * w
        hyy = hyy - (km[1] * km[1]) * w
        hzz = hzz - (km[2] * km[2]) * w
        hxy = hxy - (km[0] * km[1]) * w
        hxz = hxz - (km[0] * km[2]) * w
        hyz = hyz - (km[1] * km[2]) * w
    f = hxx * (hyy * hzz - hyz * hyz) - hxy * (hxy * hzz - hyz * hxz) + hxz * (hxy * hyz - hyy * hxz)
    return u, f


def make_on_device(name: str, n: int, seed: int = 0, eps=0.02, device="cuda", exact: bool = False):
    """(f, g, length) as float64 torch tensors on `device`, g = u on the shell
    and 0 inside: the same problems as make(), evaluated with torch (values
    agree with make() to rounding).  For workloads that are only solved, not
    compared with the CPU oracle.  exact=True appends the exact solution u
    on the whole grid."""
    import torch
    length = np.pi if name == "sine" else 1.0
    h = length / (n - 1)
    t = torch.arange(n, dtype=torch.float64, device=device) * h
    z, y, x = torch.meshgrid(t, t, t, indexing="ij")
    if name == "cosine":
        u, f = _cosine_fields(torch, x, y, z, *cosine_modes(seed, eps))
    elif name == "exp":
        s = x * x + y * y + z * z
        u, f = torch.exp(s / 2.0), (1.0 + s) * torch.exp(1.5 * s)
    elif name == "quadratic":
        u = (x * x + y * y + z * z) / 2.0
        f = torch.ones_like(u)
    elif name == "ex6":
        s = x * x + y * y + z * z
        u = s ** 0.75 / 3.0
        f = torch.where(s > 0, s.clamp_min(1e-300) ** -0.75 / 16.0, torch.full_like(s, float("inf")))
    elif name == "ex7":
        s = 3.0 - (x * x + y * y + z * z)
        u = -torch.sqrt(s)
        f = torch.where(s > 0, 3.0 * s.clamp_min(1e-300) ** -2.5, torch.full_like(s, float("inf")))
    else:
        raise ValueError(f"unknown problem {name!r}")
    g = u.clone()
    g[1:-1, 1:-1, 1:-1] = 0.0
    if exact:
        return f.contiguous(), g.contiguous(), length, u.contiguous()
    return f.contiguous(), g.contiguous(), length


def make(name: str, n: int, seed: int = 0, eps=0.02) -> Problem:
    if name == "exp":
        x, y, z = grid_coords(n)
        s = x * x + y * y + z * z
        u = np.exp(s / 2.0)
        f = (1.0 + s) * np.exp(1.5 * s)
        return Problem(name, n, u=u, f=f)
    if name == "quadratic":
        x, y, z = grid_coords(n)
        u = (x * x + y * y + z * z) / 2.0
        f = np.ones_like(u)
        return Problem(name, n, u=u, f=f)
    if name == "sine":
        L = np.pi
        x, y, z = grid_coords(n, length=L)
        u = -np.sin(x) - np.sin(y) - np.sin(z) + (x * x + y * y + z * z) / 2.0
        f = (np.sin(x) + 1.0) * (np.sin(y) + 1.0) * (np.sin(z) + 1.0)
        return Problem(name, n, length=L, u=u, f=f)
    if name == "cosine":
        x, y, z = grid_coords(n)
        u, f = _cosine_fields(np, x, y, z, *cosine_modes(seed, eps))
        return Problem(name, n, u=u, f=f)
    if name == "ex6":
        x, y, z = grid_coords(n)
        s = x * x + y * y + z * z
        u = s ** 0.75 / 3.0
        with np.errstate(divide="ignore"):
            f = np.where(s > 0, s ** -0.75 / 16.0, np.inf)   # f is only read on the interior
        return Problem(name, n, u=u, f=f)
    if name == "ex7":
        x, y, z = grid_coords(n)
        s = 3.0 - (x * x + y * y + z * z)
        u = -np.sqrt(s)
        with np.errstate(divide="ignore"):
            f = np.where(s > 0, 3.0 * s ** -2.5, np.inf)
        return Problem(name, n, u=u, f=f)
    raise ValueError(f"unknown problem {name!r}")
