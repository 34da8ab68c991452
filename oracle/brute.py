"""Direct solution of the discrete problem (pb_fe)+(boxvector) without state bounds.

Plain definition, no interior point machinery: eliminate the state through the
state equation L y = M u + f, y(u) = G u + y0 with G = L^{-1} M, y0 = L^{-1} f,
and minimise the strictly convex reduced objective
  J(u) = 1/2 y(u)^T M_c y(u) - y(u)^T c_y + alpha/2 u^T M u + beta ||D u||_1
(M_c the tracking mass: M, or the observed subdomain's mass under partial observation)
over the box u_a <= u <= u_b by cyclic coordinate descent with exact
one-dimensional minimisation (soft threshold, then clip). The result is
certified by the subgradient optimality conditions.
Dense linear algebra: tiny grids only (a few hundred unknowns at most).
"""
from __future__ import annotations

import numpy as np

from .qp import QP


def reduced_qp(qp: QP):
    """Hessian H, linear term q of the smooth part of J, and (G, y0)."""
    L = qp.L.toarray()
    M = qp.M.toarray()
    Mc = qp.Mcost.toarray()
    G = np.linalg.solve(L, M)
    y0 = np.linalg.solve(L, qp.fvec)
    H = G.T @ Mc @ G + qp.alpha * M
    q = G.T @ (Mc @ y0 - qp.cy)
    return H, q, G, y0


def solve(qp: QP, ua: np.ndarray, ub: np.ndarray, tol: float = 1e-15,
          max_sweeps: int = 200000):
    """Coordinate descent on J; returns (y, u, p, sweeps)."""
    if np.any(np.isfinite(qp.ya)) or np.any(np.isfinite(qp.yb)):
        raise ValueError("brute force handles control bounds only")
    H, q, G, y0 = reduced_qp(qp)
    n = qp.nI
    u = np.zeros(n)
    g = H @ u + q
    bd = qp.beta * qp.d
    hd = np.diag(H).copy()
    for sweep in range(max_sweeps):
        change = 0.0
        for i in range(n):
            t = u[i] - g[i] / hd[i]
            thr = bd[i] / hd[i]
            t = np.sign(t) * max(abs(t) - thr, 0.0)
            t = min(max(t, ua[i]), ub[i])
            du = t - u[i]
            if du != 0.0:
                g += H[:, i] * du
                u[i] = t
                change = max(change, abs(du))
        if change <= tol * max(1.0, np.abs(u).max()):
            break
    y = G @ u + y0
    Lt = qp.L.toarray().T
    p = -np.linalg.solve(Lt, qp.Mcost @ y - qp.cy)
    return y, u, p, sweep + 1


def certificate(qp: QP, u: np.ndarray, p: np.ndarray, ua, ub, atol: float):
    """Largest violation of the optimality conditions of J at u, with gradient
    g = alpha M u - M p of the smooth part (p the adjoint of y(u)):
      ua < u_i < ub, u_i != 0:  g_i + beta d_i sign(u_i) = 0
      u_i = 0:                  |g_i| <= beta d_i
      u_i = ub_i:               g_i + beta d_i <= 0
      u_i = ua_i:               g_i - beta d_i >= 0
    """
    g = qp.alpha * (qp.M @ u) - qp.M @ p
    bd = qp.beta * qp.d
    viol = np.zeros_like(u)
    at_ub = np.abs(u - ub) <= atol
    at_ua = np.abs(u - ua) <= atol
    zero = (np.abs(u) <= atol) & ~at_ub & ~at_ua
    free = ~(at_ub | at_ua | zero)
    viol[free] = np.abs(g[free] + bd[free] * np.sign(u[free]))
    viol[zero] = np.maximum(np.abs(g[zero]) - bd[zero], 0.0)
    viol[at_ub] = np.maximum(g[at_ub] + bd[at_ub], 0.0)
    viol[at_ua] = np.maximum(-(g[at_ua] - bd[at_ua]), 0.0)
    return float(viol.max()), dict(free=int(free.sum()), zero=int(zero.sum()),
                                   upper=int(at_ub.sum()), lower=int(at_ua.sum()))
