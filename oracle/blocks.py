"""Dense block matrices of Section 4 (tiny grids only) and Chebyshev semi-iteration.

Saddle-point form of (NewtonSystem): calA = [[A, B^T], [B, 0]] with
  A = blkdiag(M + Theta_y, alpha M~ + Theta_z),   B = [L, -M, M]   (z = [w; v];
  under partial observation the (1,1) block holds the observed mass M_s instead of M),
negative Schur complement S = B A^{-1} B^T, ideal preconditioners
P_1 = blkdiag(A, S), P_2 = [[A, 0], [B, -S]] and the practical
P_D = blkdiag(A_hat, S_hat), P_T = [[A_hat, 0], [B, -S_hat]] with
  A_hat = blkdiag(M + Theta_y, alpha D~_M + Theta_z)     (Section 4.1),
  S_hat = (L + M_hat)(M + Theta_y)^{-1}(L + M_hat)^T      (SchurApprox),
  M_hat = [D_M/alpha - alpha^{-2}(Theta_w^{-1} + Theta_v^{-1} + alpha^{-1} D_M^{-1})^{-1}]^{1/2}
          (D_M + Theta_y)^{1/2}.
Inside P_D/P_T the paper applies (M + Theta_y)^{-1} by 20 steps of Chebyshev
semi-iteration with the Jacobi splitting D_M + Theta_y; ``chebyshev`` below is
that iteration (three-term form of Golub and Varga), x_0 = 0.
"""
from __future__ import annotations

import numpy as np

from .qp import QP


def dense(a):
    return a.toarray() if hasattr(a, "toarray") else np.asarray(a)


def blocks(qp: QP, th_y, th_w, th_v):
    """(A, B) of the saddle-point form, dense."""
    M = dense(qp.M)
    L = dense(qp.L)
    a = qp.alpha
    n = qp.nI
    A = np.zeros((3 * n, 3 * n))
    A[:n, :n] = dense(qp.Mcost) + np.diag(th_y)
    A[n:2 * n, n:2 * n] = a * M + np.diag(th_w)
    A[n:2 * n, 2 * n:] = -a * M
    A[2 * n:, n:2 * n] = -a * M
    A[2 * n:, 2 * n:] = a * M + np.diag(th_v)
    B = np.hstack([L, -M, M])
    return A, B


def saddle(A, B):
    n = B.shape[0]
    return np.block([[A, B.T], [B, np.zeros((n, n))]])


def schur_exact(A, B):
    return B @ np.linalg.solve(A, B.T)


def schur_formula(qp: QP, th_y, th_w, th_v, M=None):
    """(Schur): L (M + Theta_y)^{-1} L^T + M/alpha - alpha^{-2}(Theta_w^{-1} + Theta_v^{-1} + M^{-1}/alpha)^{-1}."""
    M = dense(qp.M) if M is None else M
    L = dense(qp.L)
    a = qp.alpha
    Minv = np.linalg.inv(M)
    inner = np.diag(1.0 / th_w) + np.diag(1.0 / th_v) + Minv / a
    return L @ np.linalg.solve(M + np.diag(th_y), L.T) + M / a - np.linalg.inv(inner) / (a * a)


def mhat(dM, th_y, th_w, th_v, alpha):
    """M_hat of Section 4.2 evaluated as printed (diagonal entries)."""
    inner = 1.0 / th_w + 1.0 / th_v + 1.0 / (alpha * dM)
    return np.sqrt(dM / alpha - 1.0 / (alpha * alpha * inner)) * np.sqrt(dM + th_y)


def schur_approx(qp: QP, th_y, th_w, th_v, M=None, dM=None):
    """(SchurApprox) with the diagonal M_hat; M may be replaced by a lumped matrix."""
    M = dense(qp.M) if M is None else M
    dM = np.diag(M).copy() if dM is None else dM
    L = dense(qp.L)
    Mh = np.diag(mhat(dM, th_y, th_w, th_v, qp.alpha))
    LM = L + Mh
    return LM @ np.linalg.solve(M + np.diag(th_y), LM.T)


def zblock(qp: QP, th_w, th_v, M=None):
    """alpha M~ + Theta_z (exact) and alpha D~_M + Theta_z (its diagonal-mass approximation)."""
    M = dense(qp.M) if M is None else M
    a = qp.alpha
    DM = np.diag(np.diag(M))
    ex = np.block([[a * M + np.diag(th_w), -a * M], [-a * M, a * M + np.diag(th_v)]])
    ap = np.block([[a * DM + np.diag(th_w), -a * DM], [-a * DM, a * DM + np.diag(th_v)]])
    return ex, ap


def preconditioners(qp: QP, th_y, th_w, th_v):
    """Dense P_D and P_T (with M + Theta_y kept exact, as displayed in Section 4.2)."""
    A, B = blocks(qp, th_y, th_w, th_v)
    n = qp.nI
    _, zap = zblock(qp, th_w, th_v)
    Ah = A.copy()
    Ah[n:, n:] = zap
    Sh = schur_approx(qp, th_y, th_w, th_v)
    Z = np.zeros((n, 3 * n))
    PD = np.block([[Ah, Z.T], [Z, Sh]])
    PT = np.block([[Ah, Z.T], [B, -Sh]])
    return PD, PT


def chebyshev(A, jac, b, steps, lmin, lmax):
    """Chebyshev semi-iteration for A x = b with Jacobi splitting diag ``jac``, x_0 = 0,
    for the eigenvalue interval [lmin, lmax] of jac^{-1} A. Returns x after ``steps`` updates."""
    theta = 0.5 * (lmax + lmin)
    delta = 0.5 * (lmax - lmin)
    sig = theta / delta
    rho = 1.0 / sig
    x = np.zeros_like(b)
    r = b.copy()
    d = r / jac / theta
    for _ in range(steps):
        x = x + d
        r = r - A @ d
        rho_new = 1.0 / (2.0 * sig - rho)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * (r / jac)
        rho = rho_new
    return x


def chebyshev_error_factor(steps, lmin, lmax):
    """1 / T_k(theta/delta): the Chebyshev bound on ||e_k||_A / ||e_0||_A."""
    sig = (lmax + lmin) / (lmax - lmin)
    return 1.0 / np.cosh(steps * np.arccosh(sig))
