"""All-at-once heat-equation control problem (Section 3.4, time-dependent problems).

Test infrastructure: only tests may import this module.

  min  1/2 ||y - y_d||^2_{L2(Omega x (0,T))} + alpha/2 ||u||^2 + beta ||u||_{L1}
  s.t. y_t - Delta y = u + f on Omega x (0,T), y = 0 on the boundary, y(0) = y_0,
       u_a <= u <= u_b,

with Q1 elements in space and backward Euler in time (nt steps of size tau = T/nt).
With the rectangle rule in time the discrete problem has exactly the structure of the
stationary QP (pb_fe_lin) with
  M  -> tau blkdiag(M, ..., M)          (cost, control and coupling mass),
  L  -> calL = [[M + tau K], [-M, M + tau K], ..., [-M, M + tau K]]   (block bidiagonal),
  D  -> tau blkdiag(D, ..., D),
  f  -> [M y_0 + tau M f^1; tau M f^2; ...; tau M f^nt],
so the oracle's interior point method and brute-force solver apply unchanged.
Unknowns: interior nodes of every time level t_1..t_nt (t_0 carries y_0).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.sparse as sp

from . import fem
from .qp import QP, split_bounds


@dataclasses.dataclass
class HeatQP(QP):
    nt: int = 1
    tau: float = 1.0
    n_space: int = 0           # interior nodes per time level

    def full(self, x_int: np.ndarray, boundary=None) -> np.ndarray:
        """Space-time vector -> (nt, n^dim) nodal array with zero boundary."""
        out = np.zeros((self.nt, self.n ** self.dim))
        sidx = fem.interior(self.dim, self.n)
        out[:, sidx] = np.asarray(x_int).reshape(self.nt, self.n_space)
        return out

    def objective(self, y: np.ndarray, w: np.ndarray, v: np.ndarray) -> float:
        """Rectangle rule in time: sum_k tau (1/2 |y^k - y_d^k|_M^2) + alpha/2 u^T M u + beta d^T |z|."""
        e = self.full(y) - self.yd_full
        u = w - v
        track = sum(0.5 * self.tau * e[k] @ (self.Mfull @ e[k]) for k in range(self.nt))
        return float(track + 0.5 * self.alpha * u @ (self.M @ u) + self.beta * self.d @ (w + v))


def build_heat(n: int, nt: int, T: float, alpha: float, beta: float, ua, ub,
               yd=None, y0=None, f=None, dim: int = 2) -> HeatQP:
    """Assemble the all-at-once QP. ``yd``, ``f``: (nt, n^dim) nodal arrays for t_1..t_nt
    (or None = 0); ``y0``: nodal initial state (boundary entries ignored)."""
    Kfull, Mfull = fem.poisson_matrices(dim, n)
    sidx = fem.interior(dim, n)
    K = Kfull[sidx][:, sidx].tocsr()
    Ms = Mfull[sidx][:, sidx].tocsr()
    ns = sidx.size
    tau = T / nt
    eye = sp.identity(nt, format="csr")
    sub = sp.diags([np.ones(nt - 1)], [-1], shape=(nt, nt), format="csr")
    calL = (sp.kron(eye, Ms + tau * K) - sp.kron(sub, Ms)).tocsr()
    calM = (tau * sp.kron(eye, Ms)).tocsr()
    d = tau * np.tile(fem.lumped(Mfull, sidx), nt)
    dM = calM.diagonal().copy()
    nn = n ** dim
    yd_full = np.zeros((nt, nn)) if yd is None else np.asarray(yd, np.float64).reshape(nt, nn).copy()
    f_full = np.zeros((nt, nn)) if f is None else np.asarray(f, np.float64).reshape(nt, nn).copy()
    y0_full = np.zeros(nn) if y0 is None else np.asarray(y0, np.float64).reshape(-1).copy()
    bmask = fem.boundary_mask(dim, n)
    y0_full[bmask] = 0.0
    cy = np.concatenate([tau * (Mfull @ yd_full[k])[sidx] for k in range(nt)])
    fvec = np.concatenate([tau * (Mfull @ f_full[k])[sidx] for k in range(nt)])
    fvec[:ns] += (Mfull @ y0_full)[sidx]
    N = nt * ns
    ua_i = np.full(N, float(ua)) if np.ndim(ua) == 0 else np.asarray(ua, np.float64).reshape(-1)
    ub_i = np.full(N, float(ub)) if np.ndim(ub) == 0 else np.asarray(ub, np.float64).reshape(-1)
    if np.any(ua_i >= 0.0) or np.any(ub_i <= 0.0):
        raise ValueError("control bounds must satisfy u_a < 0 < u_b")
    za, zb = split_bounds(ua_i, ub_i)
    inf = np.full(N, math.inf)
    return HeatQP(dim, n, 1.0 / (n - 1), np.arange(N), Kfull, Mfull, calL, calM, d, dM,
                  float(alpha), float(beta), -inf, inf.copy(), za, zb, cy, fvec, yd_full,
                  np.zeros(nn), nt=nt, tau=tau, n_space=ns)


def schur_formula(qp: HeatQP, th_y, th_w, th_v):
    """Schur complement of the time-dependent Newton matrix (rectangle rule, M_c = M):
      calL (tau calM + Theta_y)^{-1} calL^T + tau calM / alpha
        - alpha^{-2} (Theta_w^{-1} + Theta_v^{-1} + (alpha tau calM)^{-1})^{-1},
    the stationary (Schur) formula with M -> tau calM (dense). ``qp.M`` already holds
    tau calM."""
    M = qp.M.toarray()
    L = qp.L.toarray()
    a = qp.alpha
    inner = np.diag(1.0 / th_w) + np.diag(1.0 / th_v) + np.linalg.inv(M) / a
    return L @ np.linalg.solve(M + np.diag(th_y), L.T) + M / a - np.linalg.inv(inner) / (a * a)


def mhat(qp: HeatQP, th_y, th_w, th_v):
    """Diagonal M_hat of the time-dependent Schur approximation (D_M -> tau D_M)."""
    dM = qp.dM
    a = qp.alpha
    inner = 1.0 / th_w + 1.0 / th_v + 1.0 / (a * dM)
    return np.sqrt(dM / a - 1.0 / (a * a * inner)) * np.sqrt(dM + th_y)


def schur_approx(qp: HeatQP, th_y, th_w, th_v):
    """(calL + M_hat)(tau calM + Theta_y)^{-1}(calL + M_hat)^T (dense)."""
    M = qp.M.toarray()
    LM = qp.L.toarray() + np.diag(mhat(qp, th_y, th_w, th_v))
    return LM @ np.linalg.solve(M + np.diag(th_y), LM.T)
