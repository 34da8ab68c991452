"""Preconditioner P_Pi for partial observations (subsection "Preconditioner for Partial
Observations"), dense, tiny grids only.

Test infrastructure: only tests may import this module.

With partial observation the (1,1) block M_s + Theta_y of (NewtonSystem) is singular
(M_s the mass of the observed subdomain, Theta_y = 0 without state bounds). The system in
the variables (y, z, p) is permuted to (p-row, z-row, y-row) order,
  Pi calA = [[L, -Mbar, 0], [0, alpha M~ + Theta_z, -Mbar^T], [M_s + Theta_y, 0, L^T]],
preconditioned by the block-triangular
  P~ = [[L, -Mbar, 0], [0, alpha M~ + Theta_z, 0], [M_s + Theta_y, 0, -S_Pi_hat]],
and P_Pi^{-1} = P~^{-1} Pi. Applying it to w = (w1, w2, w3) takes three solves:
  v2 = (alpha M~ + Theta_z)^{-1} w2,
  v1 = L^{-1} (Mbar v2 + w3),
  v3 = S_Pi_hat^{-1} ((M_s + Theta_y) v1 - w1).
The Schur complement of the permuted system is
  S_Pi = L^T + (M_s + Theta_y) L^{-1} Mbar (alpha M~ + Theta_z)^{-1} Mbar^T,
approximated by S_Pi_hat = (L^T + M_l) L^{-1} (L + M_r) with M_l = M_s + Theta_y and
M_r = Mbar (alpha M~ + Theta_z)^{-1} Mbar^T (exact here; the z-block may be replaced by its
diagonal-mass approximation).
"""
from __future__ import annotations

import numpy as np

from .blocks import dense, zblock
from .qp import QP


def parts(qp: QP, th_y, th_w, th_v, zapprox: bool = False):
    """(L, Mbar, Z = alpha M~ + Theta_z [or its D_M approximation], Ml = M_s + Theta_y)."""
    L = dense(qp.L)
    M = dense(qp.M)
    Mbar = np.hstack([M, -M])
    ex, ap = zblock(qp, th_w, th_v)
    Z = ap if zapprox else ex
    Ml = dense(qp.Mcost) + np.diag(th_y)
    return L, Mbar, Z, Ml


def schur_pi(qp: QP, th_y, th_w, th_v):
    """S_Pi = L^T + (M_s + Theta_y) L^{-1} Mbar (alpha M~ + Theta_z)^{-1} Mbar^T."""
    L, Mbar, Z, Ml = parts(qp, th_y, th_w, th_v)
    return L.T + Ml @ np.linalg.solve(L, Mbar @ np.linalg.solve(Z, Mbar.T))


def schur_pi_approx(qp: QP, th_y, th_w, th_v, zapprox: bool = False):
    """S_Pi_hat = (L^T + M_l) L^{-1} (L + M_r), M_l = M_s + Theta_y, M_r = Mbar Z^{-1} Mbar^T."""
    L, Mbar, Z, Ml = parts(qp, th_y, th_w, th_v, zapprox)
    Mr = Mbar @ np.linalg.solve(Z, Mbar.T)
    return (L.T + Ml) @ np.linalg.solve(L, L + Mr)


def apply(qp: QP, th_y, th_w, th_v, w, S=None, zapprox: bool = False):
    """v = P_Pi^{-1} w by the three solves (w = (w1, w2, w3) in the (y, z, p) order)."""
    n = qp.nI
    L, Mbar, Z, Ml = parts(qp, th_y, th_w, th_v, zapprox)
    S = schur_pi_approx(qp, th_y, th_w, th_v, zapprox) if S is None else S
    w1, w2, w3 = w[:n], w[n:3 * n], w[3 * n:]
    v2 = np.linalg.solve(Z, w2)
    v1 = np.linalg.solve(L, Mbar @ v2 + w3)
    v3 = np.linalg.solve(S, Ml @ v1 - w1)
    return np.concatenate([v1, v2, v3])


def matrix_inverse(qp: QP, th_y, th_w, th_v, S=None, zapprox: bool = False):
    """P_Pi^{-1} = P~^{-1} Pi as a dense matrix (from the permuted block-triangular P~)."""
    n = qp.nI
    L, Mbar, Z, Ml = parts(qp, th_y, th_w, th_v, zapprox)
    S = schur_pi_approx(qp, th_y, th_w, th_v, zapprox) if S is None else S
    Pt = np.block([[L, -Mbar, np.zeros((n, n))],
                   [np.zeros((2 * n, n)), Z, np.zeros((2 * n, n))],
                   [Ml, np.zeros((n, 2 * n)), -S]])
    Pi = np.zeros((4 * n, 4 * n))
    Pi[:n, 3 * n:] = np.eye(n)           # first block row of Pi calA: the p-row (L y ...)
    Pi[n:3 * n, n:3 * n] = np.eye(2 * n)
    Pi[3 * n:, :n] = np.eye(n)           # last: the y-row
    return np.linalg.solve(Pt, Pi)
