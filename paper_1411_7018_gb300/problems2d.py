"""Seeded synthetic problems of the 2D Monge-Ampere equation u_xx u_yy - u_xy^2 = f
(Eq. MA2D; the 2D examples of Section 4.1), sampled on the grid.

Holds only closed-form solutions and their right-hand sides (none of the
solver's arithmetic); serves the 2D CUDA path and the oracle-based tests.
Grids: n = N + 1 points per side on (0,1)^2, h = 1/N, arrays float64 of shape
(n, n) indexed [j, i].

  * ``ex1``  Example 1: u = exp(|x|^2/2), f = (1 + |x|^2) exp(|x|^2).
  * ``ex2``  Example 2: u = (2 sqrt(2)/3) |x|^{3/2}, f = 1/|x| (singular at the
             corner x = 0, a boundary point).
  * ``ex3``  Example 3: u = -sqrt(2 - |x|^2), f = 2/(2 - |x|^2)^2 (unbounded
             gradient at the corner (1, 1)).
  * ``quadratic``  u = |x|^2/2, f = 1 (the centred scheme is exact for it).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Problem2D:
    name: str
    n: int
    length: float = 1.0
    u: np.ndarray = field(repr=False, default=None)
    f: np.ndarray = field(repr=False, default=None)

    @property
    def h(self) -> float:
        return self.length / (self.n - 1)

    @property
    def unknowns(self) -> int:
        return (self.n - 2) ** 2

    def initial(self) -> np.ndarray:
        g = self.u.copy()
        g[1:-1, 1:-1] = 0.0
        return g


def grid2(n: int, length: float = 1.0):
    t = np.arange(n, dtype=np.float64) * (length / (n - 1))
    y, x = np.meshgrid(t, t, indexing="ij")
    return x, y


def make2d(name: str, n: int) -> Problem2D:
    x, y = grid2(n)
    s = x * x + y * y
    with np.errstate(divide="ignore", invalid="ignore"):
        if name == "ex1":
            u, f = np.exp(s / 2.0), (1.0 + s) * np.exp(s)
        elif name == "ex2":
            u = (2.0 * np.sqrt(2.0) / 3.0) * s ** 0.75
            f = np.where(s > 0, 1.0 / np.sqrt(s), np.inf)      # read on the interior only
        elif name == "ex3":
            u = -np.sqrt(2.0 - s)
            f = np.where(s < 2.0, 2.0 / (2.0 - s) ** 2, np.inf)
        elif name == "quadratic":
            u, f = s / 2.0, np.ones_like(s)
        else:
            raise ValueError(f"unknown 2D problem {name!r}")
    return Problem2D(name, n, u=u, f=f)


def make2d_on_device(name: str, n: int, device="cuda"):
    """(u_exact, f, g) as float64 torch tensors on `device` (g = u on the
    boundary, 0 inside): the problems of make2d evaluated with torch, for grids
    too large to build on the host."""
    import torch
    t = torch.arange(n, dtype=torch.float64, device=device) / (n - 1)
    y, x = torch.meshgrid(t, t, indexing="ij")
    s = x * x + y * y
    if name == "ex1":
        u, f = torch.exp(s / 2.0), (1.0 + s) * torch.exp(s)
    elif name == "ex2":
        u = (2.0 * 2.0 ** 0.5 / 3.0) * s ** 0.75
        f = torch.where(s > 0, 1.0 / torch.sqrt(s.clamp_min(1e-300)), torch.full_like(s, float("inf")))
    elif name == "ex3":
        u = -torch.sqrt(2.0 - s)
        f = torch.where(s < 2.0, 2.0 / (2.0 - s).clamp_min(1e-300) ** 2, torch.full_like(s, float("inf")))
    elif name == "quadratic":
        u, f = s / 2.0, torch.ones_like(s)
    else:
        raise ValueError(f"unknown 2D problem {name!r}")
    g = u.clone()
    g[1:-1, 1:-1] = 0.0
    return u.contiguous(), f.contiguous(), g.contiguous()
