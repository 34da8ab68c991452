"""Seeded input fields shaped like the paper's experiments.

Every array is a nodal field on the full uniform grid of the unit square or
cube, boundary nodes included, stored C-order as ``[z][y][x]`` (x fastest).
Nothing here knows about finite elements or the interior point method.

Experiment shapes (Section 5 of the paper):
  * 2D Poisson: y_d = sin(pi x1) sin(pi x2), control box [-2, 1.5].
  * 2D convection-diffusion: y_d = exp(-64((x1-1/2)^2 + (x2-1/2)^2)),
    wind (2 x2 (1 - x1^2), -2 x1 (1 - x2^2)), control box [-2, 1.5].
  * 3D Poisson: desired state only shown in a figure; we use
    x y z sin(pi x) sin(pi y) sin(pi z).
The 1025^2 sweep draws y_d as a sum of eight Gaussians (amplitude U[-1,1],
width U[0.05,0.2], centre U[0,1]^2) from numpy's PCG64 with a fixed seed.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np


def node_coords(dim: int, n: int):
    """Coordinates of an ``n``-per-direction node grid on [0,1]^dim, C-order (z, y, x)."""
    t = np.linspace(0.0, 1.0, n)
    if dim == 2:
        y, x = np.meshgrid(t, t, indexing="ij")
        return x, y
    if dim == 3:
        z, y, x = np.meshgrid(t, t, t, indexing="ij")
        return x, y, z
    raise ValueError("dim must be 2 or 3")


def yd_sin_product(n: int) -> np.ndarray:
    x, y = node_coords(2, n)
    return np.sin(np.pi * x) * np.sin(np.pi * y)


def yd_gaussian_sum(n: int, seed: int, k: int = 8, dim: int = 2) -> np.ndarray:
    """Sum of ``k`` Gaussians with amplitude U[-1,1], width U[0.05,0.2], centre U[0,1]^dim."""
    rng = np.random.Generator(np.random.PCG64(seed))
    amp = rng.uniform(-1.0, 1.0, k)
    wid = rng.uniform(0.05, 0.2, k)
    ctr = rng.uniform(0.0, 1.0, (k, dim))
    xs = node_coords(dim, n)
    out = np.zeros(xs[0].shape)
    for a, s, c in zip(amp, wid, ctr):
        r2 = sum((xs[d] - c[d]) ** 2 for d in range(dim))
        out += a * np.exp(-r2 / (2.0 * s * s))
    return out


def yd_cube_sin(n: int) -> np.ndarray:
    x, y, z = node_coords(3, n)
    return x * y * z * np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)


def yd_cd_bump(n: int) -> np.ndarray:
    x, y = node_coords(2, n)
    return np.exp(-64.0 * ((x - 0.5) ** 2 + (y - 0.5) ** 2))


def heat_moving_target(n: int, T: float) -> dict:
    """Inputs of an all-at-once heat-equation problem with n - 2 time levels on [0, T]:
    a desired state sin(pi x) sin(pi y) (1 + 2t) cos(2 pi t) at t_k = k T / (n - 2),
    k = 1 .. n - 2, and the initial state 0.5 sin(pi x) sin(2 pi y) (zero on the boundary).
    Returned per level (``yd``: (n - 2, n^2), ``y0``: n^2) and in the space-time layout of an
    n^3 array whose plane k is time level k (``yd3``: planes 1 .. n - 2; ``g3``: plane 0 =
    y0, the rest zero)."""
    nt = n - 2
    tau = T / nt
    x, y = node_coords(2, n)
    x, y = x.reshape(-1), y.reshape(-1)
    base = np.sin(np.pi * x) * np.sin(np.pi * y)
    yd = np.stack([base * (1.0 + 2.0 * (k + 1) * tau) * np.cos(2.0 * np.pi * (k + 1) * tau)
                   for k in range(nt)])
    y0 = 0.5 * np.sin(np.pi * x) * np.sin(2.0 * np.pi * y)
    edge = (x == 0.0) | (x == 1.0) | (y == 0.0) | (y == 1.0)
    yd3 = np.zeros((n, n * n))
    yd3[1:n - 1] = yd
    g3 = np.zeros((n, n * n))
    g3[0] = np.where(edge, 0.0, y0)
    return dict(yd=yd, y0=y0, yd3=yd3.reshape(-1), g3=g3.reshape(-1), nt=nt, tau=tau)


@dataclasses.dataclass
class Workload:
    """One optimal control problem instance (inputs only)."""
    name: str
    dim: int
    n: int                       # nodes per direction, boundary included
    kind: str                    # "poisson" or "cd"
    alpha: float
    beta: float
    ua: float
    ub: float
    ya: float = -math.inf
    yb: float = math.inf
    eps: float = 1.0             # diffusion coefficient (convection-diffusion only)
    sigma: float = 0.2           # barrier reduction factor
    yd: Optional[np.ndarray] = None
    f: Optional[np.ndarray] = None
    g: Optional[np.ndarray] = None
    seed: int = 0

    @property
    def unknowns(self) -> int:
        return (self.n - 2) ** self.dim


def workload_c1(n: int = 33, alpha: float = 1e-2, beta: float = 1e-3,
                ua: float = -2.0, ub: float = 2.0) -> Workload:
    """2D Poisson, y_d = sin(pi x) sin(pi y), no state bounds (33^2 by default)."""
    return Workload("poisson2d-sin", 2, n, "poisson", alpha, beta, ua, ub,
                    yd=yd_sin_product(n))


def poisson_2d_sweep() -> List[tuple]:
    """The (alpha, beta) grid of the 1025^2 experiment, in a fixed order with its seeds."""
    out = []
    seed = 0
    for a in (1e-2, 1e-4, 1e-6):
        for b in (1e-2, 1e-3, 1e-4):
            out.append((a, b, seed))
            seed += 1
    return out


def workload_c2(n: int = 1025, cell: int = 0) -> Workload:
    """2D Poisson, Gaussian-sum y_d, u in [-30,30], y <= 0.1; ``cell`` picks (alpha, beta, seed)."""
    a, b, seed = poisson_2d_sweep()[cell % 9]
    return Workload(f"poisson2d-gauss8-a{a:g}-b{b:g}", 2, n, "poisson", a, b, -30.0, 30.0,
                    yb=0.1, yd=yd_gaussian_sum(n, seed), seed=seed)


def workload_c3(n: int = 129, alpha: float = 1e-4, beta: float = 1e-3) -> Workload:
    """3D Poisson, y_d = xyz sin sin sin, u in [-50,50]."""
    return Workload("poisson3d-sin", 3, n, "poisson", alpha, beta, -50.0, 50.0,
                    yd=yd_cube_sin(n))


def workload_c4(n: int = 513, eps: float = 1.0 / 50.0, alpha: float = 1e-3,
                beta: float = 1e-3, sigma: float = 0.25) -> Workload:
    """2D convection-diffusion with the recirculating wind, u in [-2,1.5]."""
    return Workload("cd2d-bump", 2, n, "cd", alpha, beta, -2.0, 1.5, eps=eps,
                    sigma=sigma, yd=yd_cd_bump(n))


def serving_stream(num: int = 512, seed: int = 0, grids2d=(65, 129, 257, 513),
                   grids3d=(33, 65), cd_frac: float = 0.3,
                   with_fields: bool = True) -> List[dict]:
    """Seeded request mix: grid, PDE, log-uniform alpha/beta, Gaussian-sum y_d, symmetric box.

    Exponential inter-arrival gaps with unit mean are returned in ``gap``; the
    caller scales them to an offered load.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    grids = [(2, g) for g in grids2d] + [(3, g) for g in grids3d]
    reqs = []
    for i in range(num):
        dim, n = grids[int(rng.integers(len(grids)))]
        kind = "cd" if (dim == 2 and rng.uniform() < cd_frac) else "poisson"
        alpha = 10.0 ** rng.uniform(-6.0, -2.0)
        beta = 10.0 ** rng.uniform(-5.0, -2.0)
        half = rng.uniform(1.0, 50.0)
        gap = rng.exponential(1.0)
        yd_seed = int(rng.integers(1 << 31))
        r = dict(index=i, dim=dim, n=n, kind=kind, alpha=alpha, beta=beta,
                 ua=-half, ub=half, eps=1.0 / 50.0, gap=gap, yd_seed=yd_seed,
                 sigma=0.25 if kind == "cd" else 0.2)
        if with_fields:
            r["yd"] = yd_gaussian_sum(n, yd_seed, dim=dim)
        reqs.append(r)
    return reqs
