"""The discrete quadratic program (pb_fe_lin) of Section 2.

  min_{y, z}  1/2 (y - y_d)^T M (y - y_d) + alpha/2 z^T M~ z + beta 1^T Dbar z
  s.t.        L y - Mbar z = f,   z_a <= z <= z_b,   y_a <= y <= y_b,
with z = [w; v], u = w - v (split), M~ = [[M, -M], [-M, M]], Mbar = [M, -M],
Dbar = [D, D], z_a = [max(u_a, 0); -min(u_b, 0)], z_b = [max(u_b, 0); -min(u_a, 0)].

Unknowns are the interior nodes of the grid for y, u and p alike (the state
equation carries Dirichlet data y = g on the boundary); L and M are the
interior-interior blocks of the full-grid Galerkin matrices. Nodal data enter
through the full-grid matrices:
  c_y  = (M_full (y_d - g_lift))_I     (the vector written "M y_d"),
  f    = (M_full f)_I - (L_full g_lift)_I,
where g_lift is g on boundary nodes and zero inside.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np
import scipy.sparse as sp

from . import fem


@dataclasses.dataclass
class QP:
    dim: int
    n: int
    h: float
    idx: np.ndarray          # interior full-grid indices
    Lfull: sp.csr_matrix
    Mfull: sp.csr_matrix
    L: sp.csr_matrix         # interior block of L
    M: sp.csr_matrix         # interior block of M
    d: np.ndarray            # lumped mass D (interior)
    dM: np.ndarray           # diag(M) (interior)
    alpha: float
    beta: float
    ya: np.ndarray
    yb: np.ndarray
    za: np.ndarray           # length 2 nI
    zb: np.ndarray
    cy: np.ndarray           # "M y_d"
    fvec: np.ndarray
    yd_full: np.ndarray
    g_full: np.ndarray
    # partial observation: mass of the observed subdomain in the cost (None = M)
    Mc: Optional[sp.csr_matrix] = None
    Mcfull: Optional[sp.csr_matrix] = None

    @property
    def nI(self) -> int:
        return self.idx.size

    @property
    def Mcost(self) -> sp.csr_matrix:
        """Mass of the tracking term: M, or M_s for partial observation."""
        return self.M if self.Mc is None else self.Mc

    def full(self, x_int: np.ndarray, boundary: Optional[np.ndarray] = None) -> np.ndarray:
        """Embed an interior vector in the full grid (boundary = ``boundary`` or zero)."""
        out = np.zeros(self.n ** self.dim) if boundary is None else boundary.copy()
        out[self.idx] = x_int
        return out

    def objective(self, y: np.ndarray, w: np.ndarray, v: np.ndarray) -> float:
        """Q(y, z): 1/2 ||y_h - y_d,h||^2_{L2} + alpha/2 u^T M u + beta 1^T Dbar z (full-grid state)."""
        e = self.full(y, self.g_full) - self.yd_full
        u = w - v
        Mt = self.Mfull if self.Mcfull is None else self.Mcfull
        return float(0.5 * e @ (Mt @ e) + 0.5 * self.alpha * u @ (self.M @ u)
                     + self.beta * self.d @ (w + v))


def _as_interior(val, n_int: int, idx: np.ndarray) -> np.ndarray:
    """Scalar -> constant array; full-grid nodal array -> its interior entries."""
    a = np.asarray(val, dtype=np.float64)
    if a.ndim == 0:
        return np.full(n_int, float(a))
    return a.reshape(-1)[idx].copy()


def split_bounds(ua: np.ndarray, ub: np.ndarray):
    """z_a, z_b of the splitting u = w - v (Section 2)."""
    za = np.concatenate([np.maximum(ua, 0.0), -np.minimum(ub, 0.0)])
    zb = np.concatenate([np.maximum(ub, 0.0), -np.minimum(ua, 0.0)])
    return za, zb


def build(dim: int, n: int, alpha: float, beta: float, ua, ub, ya=-math.inf, yb=math.inf,
          yd=None, f=None, g=None, kind: str = "poisson", eps: float = 1.0,
          supg: bool = True, lump: bool = False, observe=None) -> QP:
    """Assemble the QP for a Q1 grid with ``n`` nodes per direction on the unit square/cube.

    ``lump=True`` replaces every mass matrix by the lumped D (row sums), the
    setting of the eigenvalue theorem of Section 4.2 and of the pointwise
    optimality relation u = P_[ua,ub](sign(p) max(|p| - beta, 0)/alpha).
    ``observe``: partial observation (the subsection on partial observations): the
    tracking term integrates over the elements whose centre satisfies
    ``observe(centres)``, so the cost mass M_s differs from the coupling mass M."""
    if kind == "poisson":
        Lfull, Mfull = fem.poisson_matrices(dim, n)
    elif kind == "cd":
        if dim != 2:
            raise ValueError("convection-diffusion is two-dimensional")
        Lfull, Mfull, _ = fem.convdiff_matrices(n, eps, supg=supg)
    else:
        raise ValueError(kind)
    if lump:
        Mfull = sp.diags(np.asarray(Mfull.sum(axis=1)).ravel()).tocsr()
    idx = fem.interior(dim, n)
    nn = n ** dim
    L = Lfull[idx][:, idx].tocsr()
    M = Mfull[idx][:, idx].tocsr()
    d = fem.lumped(Mfull, idx)
    dM = M.diagonal().copy()
    nI = idx.size
    ua_i = _as_interior(ua, nI, idx)
    ub_i = _as_interior(ub, nI, idx)
    ya_i = _as_interior(ya, nI, idx)
    yb_i = _as_interior(yb, nI, idx)
    if np.any(ua_i >= 0.0) or np.any(ub_i <= 0.0):
        raise ValueError("control bounds must satisfy u_a < 0 < u_b")
    if np.any(ya_i >= yb_i):
        raise ValueError("empty state box")
    za, zb = split_bounds(ua_i, ub_i)
    yd_full = np.zeros(nn) if yd is None else np.asarray(yd, np.float64).reshape(-1).copy()
    f_full = np.zeros(nn) if f is None else np.asarray(f, np.float64).reshape(-1).copy()
    g_full = np.zeros(nn) if g is None else np.asarray(g, np.float64).reshape(-1).copy()
    g_lift = g_full.copy()
    g_lift[idx] = 0.0
    g_full = g_lift
    Mcfull = None if observe is None else fem.mass_subdomain(dim, n, observe)
    Mc = None if Mcfull is None else Mcfull[idx][:, idx].tocsr()
    cy = ((Mfull if Mcfull is None else Mcfull) @ (yd_full - g_lift))[idx]
    fvec = (Mfull @ f_full)[idx] - (Lfull @ g_lift)[idx]
    return QP(dim, n, 1.0 / (n - 1), idx, Lfull, Mfull, L, M, d, dM, float(alpha), float(beta),
              ya_i, yb_i, za, zb, cy, fvec, yd_full, g_full, Mc, Mcfull)


def from_workload(wl, **kw) -> QP:
    """Build the QP of a :class:`workloads.Workload`."""
    return build(wl.dim, wl.n, wl.alpha, wl.beta, wl.ua, wl.ub, wl.ya, wl.yb, yd=wl.yd,
                 f=wl.f, g=wl.g, kind=wl.kind, eps=wl.eps, **kw)
