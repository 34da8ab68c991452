"""Algorithm A.1 (Appendix): infeasible primal-dual path-following IPM for (pb_fe_lin).

Each iteration, in the paper's order:
  1. mu <- sigma mu.
  2. Theta_y, Theta_z (after NewtonSystem) and the right-hand side of
     (NewtonSystem), formed with the reduced mu.
  3. Solve (NewtonSystem) for (dy, dz, dp) -- here with a sparse direct LU
     (plus iterative refinement), i.e. the exact Newton direction that the
     preconditioned Krylov solvers of Section 4 approximate.
  4. Multiplier steps (zupdate1)-(zupdate4).
  5. Step lengths: the largest steps in (0, 1] keeping y, z strictly inside
     their bounds (alpha_P) and the multipliers positive (alpha_D), then
     scaled by alpha_0.
  6. y, z move with alpha_P; p and the multipliers with alpha_D.
  7. Feasibilities (prdu) and complementarity (gap).

Readings where the paper is silent or garbled:
  * mu^0 = 1 and a central-path start: y^0 = 0 (or the box centre / a unit
    offset if 0 is not strictly inside), z^0 = (z_a + z_b)/2 (z_a + 1 when z_b
    is infinite), p^0 = 0, lambda^0 = mu^0 / distance-to-bound.
  * The last block of (gap) uses lambda_{z,b} (the printed lambda_{z,a} is a typo).
  * Absent (infinite) bounds carry no barrier term, multiplier or Theta entry.
  * Step lengths are capped at 1 before the alpha_0 factor.
  * kkt_rel = max( ||xi_p|| / (1 + ||f|| + ||M y_d||),
                   ||xi_d|| / (1 + ||M y_d|| + beta ||D 1||),
                   (sum of complementarity products / number of bounds) / (1 + |Q|) ),
    2-norms of the discrete vectors.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .qp import QP


@dataclasses.dataclass
class State:
    y: np.ndarray
    w: np.ndarray
    v: np.ndarray
    p: np.ndarray
    lya: np.ndarray
    lyb: np.ndarray
    lwa: np.ndarray
    lwb: np.ndarray
    lva: np.ndarray
    lvb: np.ndarray
    mu: float

    def copy(self) -> "State":
        return State(*(a.copy() for a in dataclasses.astuple(self)[:-1]), self.mu)


def _start_point(lo: np.ndarray, hi: np.ndarray) -> np.ndarray:
    """Zero if strictly inside, else the box centre, else one unit inside the finite bound."""
    inside = (lo < 0.0) & (0.0 < hi)
    both = np.isfinite(lo) & np.isfinite(hi)
    with np.errstate(invalid="ignore"):
        mid = 0.5 * (lo + hi)
    return np.where(inside, 0.0, np.where(both, mid,
                                          np.where(np.isfinite(lo), lo + 1.0, hi - 1.0)))


def _z_start(za: np.ndarray, zb: np.ndarray) -> np.ndarray:
    return np.where(np.isfinite(zb), 0.5 * (za + zb), za + 1.0)


def _barrier_mult(mu, x, lo, hi):
    """lambda_a = mu/(x - lo), lambda_b = mu/(hi - x); zero where the bound is absent."""
    la = np.where(np.isfinite(lo), mu / np.where(np.isfinite(lo), x - lo, 1.0), 0.0)
    lb = np.where(np.isfinite(hi), mu / np.where(np.isfinite(hi), hi - x, 1.0), 0.0)
    return la, lb


def initial_state(qp: QP, mu0: float = 1.0) -> State:
    n = qp.nI
    y = _start_point(qp.ya, qp.yb)
    z = _z_start(qp.za, qp.zb)
    w, v = z[:n].copy(), z[n:].copy()
    lya, lyb = _barrier_mult(mu0, y, qp.ya, qp.yb)
    lza, lzb = _barrier_mult(mu0, z, qp.za, qp.zb)
    return State(y, w, v, np.zeros(n), lya, lyb, lza[:n].copy(), lzb[:n].copy(),
                 lza[n:].copy(), lzb[n:].copy(), float(mu0))


def _inv_dist(x, lo, hi):
    """(1/(x - lo), 1/(hi - x)) with zeros for absent bounds."""
    ia = np.where(np.isfinite(lo), 1.0 / np.where(np.isfinite(lo), x - lo, 1.0), 0.0)
    ib = np.where(np.isfinite(hi), 1.0 / np.where(np.isfinite(hi), hi - x, 1.0), 0.0)
    return ia, ib


def thetas(qp: QP, s: State):
    """Theta_y = (Y - Y_a)^{-1} Lambda_{y,a} + (Y_b - Y)^{-1} Lambda_{y,b}; Theta_w, Theta_v likewise."""
    n = qp.nI
    iya, iyb = _inv_dist(s.y, qp.ya, qp.yb)
    iwa, iwb = _inv_dist(s.w, qp.za[:n], qp.zb[:n])
    iva, ivb = _inv_dist(s.v, qp.za[n:], qp.zb[n:])
    th_y = iya * s.lya + iyb * s.lyb
    th_w = iwa * s.lwa + iwb * s.lwb
    th_v = iva * s.lva + ivb * s.lvb
    return th_y, th_w, th_v


def gradients(qp: QP, s: State):
    """The three blocks of the optimality system without barrier terms:
    g_y = M y - M y_d + L^T p,
    g_z = alpha M~ z + beta Dbar^T 1 - Mbar^T p   (split into w, v rows),
    g_p = L y - Mbar z - f."""
    Mu = qp.M @ (s.w - s.v)
    Mp = qp.M @ s.p
    g_y = qp.Mcost @ s.y - qp.cy + qp.L.T @ s.p
    g_w = qp.alpha * Mu + qp.beta * qp.d - Mp
    g_v = -qp.alpha * Mu + qp.beta * qp.d + Mp
    g_p = qp.L @ s.y - Mu - qp.fvec
    return g_y, g_w, g_v, g_p


def newton_matrix(qp: QP, th_y, th_w, th_v) -> sp.csc_matrix:
    """The reduced Newton matrix (NewtonSystem) in the variables (dy, dw, dv, dp)."""
    a = qp.alpha
    M, L = qp.M, qp.L
    D = sp.diags
    return sp.bmat([
        [qp.Mcost + D(th_y), None, None, L.T],
        [None, a * M + D(th_w), -a * M, -M],
        [None, -a * M, a * M + D(th_v), M],
        [L, -M, M, None],
    ]).tocsc()


def newton_rhs(qp: QP, s: State, mu: float):
    """Right-hand side of (NewtonSystem) at barrier parameter ``mu``."""
    n = qp.nI
    g_y, g_w, g_v, g_p = gradients(qp, s)
    iya, iyb = _inv_dist(s.y, qp.ya, qp.yb)
    iwa, iwb = _inv_dist(s.w, qp.za[:n], qp.zb[:n])
    iva, ivb = _inv_dist(s.v, qp.za[n:], qp.zb[n:])
    r_y = -(g_y - mu * iya + mu * iyb)
    r_w = -(g_w - mu * iwa + mu * iwb)
    r_v = -(g_v - mu * iva + mu * ivb)
    r_p = -g_p
    return np.concatenate([r_y, r_w, r_v, r_p])


def solve_direct(A: sp.csc_matrix, b: np.ndarray, refine: int = 2) -> np.ndarray:
    """Sparse LU solve of A x = b with ``refine`` steps of iterative refinement.

    The matrix is first equilibrated symmetrically, S A S with S = diag(1/sqrt(max_j |a_ij|)),
    then factorised with a symmetric-mode minimum-degree ordering and a small diagonal
    pivot threshold; this keeps the fill near its structural minimum although Theta spans
    many orders of magnitude. Refinement runs on the unscaled system."""
    rmax = np.asarray(abs(A).max(axis=1).todense()).ravel()
    sc = 1.0 / np.sqrt(np.maximum(rmax, 1e-300))
    S = sp.diags(sc)
    As = (S @ A @ S).tocsc()
    try:
        lu = spla.splu(As, permc_spec="MMD_AT_PLUS_A", diag_pivot_thresh=0.01,
                       options=dict(SymmetricMode=True))
    except RuntimeError:
        # a zero pivot under relaxed pivoting: fall back to partial pivoting
        lu = spla.splu(As, permc_spec="MMD_AT_PLUS_A")
    x = sc * lu.solve(sc * b)
    for _ in range(refine):
        x = x + sc * lu.solve(sc * (b - A @ x))
    return x


def multiplier_steps(qp: QP, s: State, dy, dw, dv, mu):
    """(zupdate1)-(zupdate4); zero for absent bounds."""
    n = qp.nI
    iya, iyb = _inv_dist(s.y, qp.ya, qp.yb)
    iwa, iwb = _inv_dist(s.w, qp.za[:n], qp.zb[:n])
    iva, ivb = _inv_dist(s.v, qp.za[n:], qp.zb[n:])

    def pair(ia, ib, la, lb, dx, lo, hi):
        dla = np.where(np.isfinite(lo), -ia * la * dx - la + mu * ia, 0.0)
        dlb = np.where(np.isfinite(hi), ib * lb * dx - lb + mu * ib, 0.0)
        return dla, dlb

    dlya, dlyb = pair(iya, iyb, s.lya, s.lyb, dy, qp.ya, qp.yb)
    dlwa, dlwb = pair(iwa, iwb, s.lwa, s.lwb, dw, qp.za[:n], qp.zb[:n])
    dlva, dlvb = pair(iva, ivb, s.lva, s.lvb, dv, qp.za[n:], qp.zb[n:])
    return dlya, dlyb, dlwa, dlwb, dlva, dlvb


def max_step(x, dx, lo, hi) -> float:
    """Largest a in (0, 1] with lo <= x + a dx <= hi (componentwise ratio test)."""
    a = 1.0
    m = (dx < 0.0) & np.isfinite(lo)
    if np.any(m):
        a = min(a, float(np.min((x[m] - lo[m]) / (-dx[m]))))
    m = (dx > 0.0) & np.isfinite(hi)
    if np.any(m):
        a = min(a, float(np.min((hi[m] - x[m]) / dx[m])))
    return a


def residuals(qp: QP, s: State):
    """xi_p, xi_d (prdu) and xi_c (gap) at the state's mu, present bounds only."""
    n = qp.nI
    g_y, g_w, g_v, g_p = gradients(qp, s)
    xi_p = g_p
    xi_d = np.concatenate([g_y - s.lya + s.lyb, g_w - s.lwa + s.lwb, g_v - s.lva + s.lvb])
    prods = []
    for x, lo, hi, la, lb in ((s.y, qp.ya, qp.yb, s.lya, s.lyb),
                              (s.w, qp.za[:n], qp.zb[:n], s.lwa, s.lwb),
                              (s.v, qp.za[n:], qp.zb[n:], s.lva, s.lvb)):
        ma = np.isfinite(lo)
        mb = np.isfinite(hi)
        prods.append((x[ma] - lo[ma]) * la[ma])
        prods.append((hi[mb] - x[mb]) * lb[mb])
    prods = np.concatenate(prods)
    xi_c = prods - s.mu
    return xi_p, xi_d, xi_c, prods


def kkt_rel(qp: QP, s: State, xi_p, xi_d, prods) -> float:
    """Relative KKT residual (reading of the paper's stopping measures; see module doc)."""
    nf = np.linalg.norm(qp.fvec)
    nyd = np.linalg.norm(qp.cy)
    nd = np.linalg.norm(qp.d)
    rp = np.linalg.norm(xi_p) / (1.0 + nf + nyd)
    rd = np.linalg.norm(xi_d) / (1.0 + nyd + qp.beta * nd)
    gap = (prods.sum() / prods.size) if prods.size else 0.0
    rc = gap / (1.0 + abs(qp.objective(s.y, s.w, s.v)))
    return float(max(rp, rd, rc))


@dataclasses.dataclass
class Result:
    state: State
    history: List[dict]
    converged: bool

    def y_full(self, qp: QP) -> np.ndarray:
        return qp.full(self.state.y, qp.g_full)

    def u(self) -> np.ndarray:
        return self.state.w - self.state.v


def _record(qp: QP, s: State, k: int, extra: dict) -> dict:
    xi_p, xi_d, xi_c, prods = residuals(qp, s)
    rec = dict(k=k, mu=s.mu, xi_p=float(np.linalg.norm(xi_p)),
               xi_d=float(np.linalg.norm(xi_d)), xi_c=float(np.linalg.norm(xi_c)),
               kkt_rel=kkt_rel(qp, s, xi_p, xi_d, prods))
    rec.update(extra)
    return rec


def solve(qp: QP, sigma: float = 0.2, alpha0: float = 0.995, mu0: float = 1.0,
          eps_p: float = 1e-6, eps_d: float = 1e-6, eps_c: float = 1e-6,
          stop: str = "paper", kkt_tol: float = 1e-6, max_iter: int = 200,
          n_iter: Optional[int] = None, refine: int = 2, mu_rule: str = "schedule",
          common_step: bool = False, newton_solve=None) -> Result:
    """Run Algorithm A.1.

    stop = "paper": ||xi_p|| <= eps_p and ||xi_d|| <= eps_d and ||xi_c|| <= eps_c;
    stop = "kkt":   kkt_rel <= kkt_tol;
    n_iter given:   exactly that many iterations (for trajectory comparisons).

    mu_rule = "schedule": mu^{k+1} = sigma mu^k as printed in Algorithm A.1 (default);
    mu_rule = "gap":      mu^{k+1} = sigma * (mean complementarity product of the current
                          iterate), the duality-measure form of the path-following scheme
                          the paper cites; it equals the schedule while full steps are taken.
    common_step = True:   both primal and dual variables move with min(alpha_P, alpha_D).
    newton_solve:         None = the sparse direct solve (direct tier); else a callable
                          (qp, A, b, Theta_y, Theta_w, Theta_v) -> dx, e.g. the iterative
                          tier's FGMRES + P_T (``oracle.iterative.newton_solver``).
    """
    n = qp.nI
    s = initial_state(qp, mu0)
    hist = [_record(qp, s, 0, {})]
    converged = False
    k = 0
    while True:
        h = hist[-1]
        if n_iter is not None:
            if k >= n_iter:
                converged = True
                break
        elif stop == "paper":
            if h["xi_p"] <= eps_p and h["xi_d"] <= eps_d and h["xi_c"] <= eps_c:
                converged = True
                break
        else:
            if h["kkt_rel"] <= kkt_tol:
                converged = True
                break
        if k >= max_iter:
            break
        if mu_rule == "gap":
            _, _, _, prods = residuals(qp, s)
            mu = sigma * float(prods.mean())
        else:
            mu = sigma * s.mu
        th_y, th_w, th_v = thetas(qp, s)
        A = newton_matrix(qp, th_y, th_w, th_v)
        b = newton_rhs(qp, s, mu)
        if newton_solve is None:
            dx = solve_direct(A, b, refine)
        else:
            dx = newton_solve(qp, A, b, th_y, th_w, th_v)
        dy, dw, dv, dp = dx[:n], dx[n:2 * n], dx[2 * n:3 * n], dx[3 * n:]
        dl = multiplier_steps(qp, s, dy, dw, dv, mu)
        aP = min(max_step(s.y, dy, qp.ya, qp.yb),
                 max_step(s.w, dw, qp.za[:n], qp.zb[:n]),
                 max_step(s.v, dv, qp.za[n:], qp.zb[n:]))
        lams = (s.lya, s.lyb, s.lwa, s.lwb, s.lva, s.lvb)
        bnds = (qp.ya, qp.yb, qp.za[:n], qp.zb[:n], qp.za[n:], qp.zb[n:])
        aD = 1.0
        for lam, dlam, bnd in zip(lams, dl, bnds):
            m = np.isfinite(bnd)
            if np.any(m):
                aD = min(aD, max_step(lam[m], dlam[m], np.zeros(m.sum()),
                                      np.full(m.sum(), np.inf)))
        aP *= alpha0
        aD *= alpha0
        if common_step:
            aP = aD = min(aP, aD)
        s.y = s.y + aP * dy
        s.w = s.w + aP * dw
        s.v = s.v + aP * dv
        s.p = s.p + aD * dp
        s.lya = s.lya + aD * dl[0]
        s.lyb = s.lyb + aD * dl[1]
        s.lwa = s.lwa + aD * dl[2]
        s.lwb = s.lwb + aD * dl[3]
        s.lva = s.lva + aD * dl[4]
        s.lvb = s.lvb + aD * dl[5]
        s.mu = mu
        k += 1
        hist.append(_record(qp, s, k, dict(alpha_P=aP, alpha_D=aD)))
    return Result(s, hist, converged)


def natural_residual(qp: QP, u: np.ndarray, p: np.ndarray, ua, ub) -> np.ndarray:
    """r = u - P_[ua,ub]( shrink(u - D^{-1}(alpha M u - M p), beta) ): zero exactly at the
    optimum of (pb_fe)+(boxvector) in u given the adjoint p (any positive diagonal scaling
    gives the same zero set; D is the natural one)."""
    g = qp.alpha * (qp.M @ u) - qp.M @ p
    t = u - g / qp.d
    sh = np.sign(t) * np.maximum(np.abs(t) - qp.beta, 0.0)
    return u - np.clip(sh, ua, ub)
