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
        k, phi, amp = cosine_modes(seed, eps)
        u = (x * x + y * y + z * z) / 2.0
        Hm = np.zeros((3, 3) + x.shape)
        for a in range(3):
            Hm[a, a] = 1.0
        for m in range(k.shape[0]):
            km = k[m].astype(np.float64)
            kk = float(km @ km)
            theta = 2.0 * np.pi * (km[0] * x + km[1] * y + km[2] * z) + phi[m]
            c = np.cos(theta)
            u = u + amp[m] / (4.0 * np.pi ** 2 * kk) * c
            for a in range(3):
                for b in range(3):
                    Hm[a, b] = Hm[a, b] - amp[m] * c * km[a] * km[b] / kk
        f = (Hm[0, 0] * (Hm[1, 1] * Hm[2, 2] - Hm[1, 2] * Hm[2, 1])
             - Hm[0, 1] * (Hm[1, 0] * Hm[2, 2] - Hm[1, 2] * Hm[2, 0])
             + Hm[0, 2] * (Hm[1, 0] * Hm[2, 1] - Hm[1, 1] * Hm[2, 0]))
        return Problem(name, n, u=u, f=f)
    raise ValueError(f"unknown problem {name!r}")
