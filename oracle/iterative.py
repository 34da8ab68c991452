"""Iterative tier of the oracle: the Newton systems of Algorithm A.1 solved by FGMRES with P_T.

TEST INFRASTRUCTURE ONLY (see the package docstring).

For grids where the direct tier's sparse LU of the 4n x 4n Newton matrix is out of reach
(1025^2, 65^3 and up), each Newton system (NewtonSystem, Section 3) is solved by flexible
GMRES, right-preconditioned so that the monitored residual is the unpreconditioned one,
with the block-triangular preconditioner of Section 4:

    P_T = [[A_hat, 0], [B, -S_hat]],   A_hat = blkdiag(M + Theta_y, alpha D~_M + Theta_z),
    B = [L, -M, M],                    S_hat = (L + M_hat)(M + Theta_y)^{-1}(L + M_hat)^T,

with (M + Theta_y)^{-1} by 20 steps of Chebyshev semi-iteration (Section 4.1), the z-block
by pointwise 2x2 solves with D_M (Section 4.1), and (L + M_hat)^{-1} by geometric multigrid
V-cycles (a stand-in for the paper's AMG, Section 5) or, for convection-diffusion, by a
sparse LU of L + M_hat. The preconditioner only decides how fast FGMRES converges: every
Newton solve runs until the true residual ||b - A x|| of the assembled Newton matrix is
below ``tol`` ||b|| (1e-12 by default) or stops decreasing at the FP64 attainable accuracy,
so the direction equals the direct tier's up to that level. The multigrid here is its own plain construction (Galerkin coarse
operators P^T A P from bilinear / trilinear interpolation, damped Jacobi smoothing,
sparse LU on the coarsest grid) and shares nothing with the GPU library.
"""
from __future__ import annotations

import dataclasses
import math
import time
from typing import Callable, List, Optional

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import blocks, fem
from .qp import QP


# --------------------------------------------------------------------------------------
# geometric multigrid on the interior nodes of a 2^k + 1 grid
# --------------------------------------------------------------------------------------

def prolongation_1d(n: int) -> sp.csr_matrix:
    """Linear interpolation from the interior nodes of the (n+1)/2-node grid to the interior
    nodes of the n-node grid (boundary values zero): fine node 2j takes coarse node j, fine
    node 2j+1 the mean of coarse nodes j and j+1 (full-grid numbering)."""
    nc = (n + 1) // 2
    rows, cols, vals = [], [], []
    for i in range(1, n - 1):              # fine interior node (full-grid index)
        if i % 2 == 0:
            j = i // 2
            if 0 < j < nc - 1:
                rows.append(i - 1); cols.append(j - 1); vals.append(1.0)
        else:
            for j in (i // 2, i // 2 + 1):
                if 0 < j < nc - 1:
                    rows.append(i - 1); cols.append(j - 1); vals.append(0.5)
    return sp.csr_matrix((vals, (rows, cols)), shape=(n - 2, nc - 2))


def prolongation(dim: int, n: int) -> sp.csr_matrix:
    """Bilinear / trilinear interpolation between interior-node vectors (x fastest)."""
    p1 = prolongation_1d(n)
    P = p1
    for _ in range(dim - 1):
        P = sp.kron(p1, P)
    return P.tocsr()


@dataclasses.dataclass
class _Level:
    A: sp.csr_matrix
    dinv: np.ndarray
    P: Optional[sp.csr_matrix]      # prolongation from the next coarser level


class GMG:
    """V-cycles for A x = b with A = L + diag(m) on a 2^k + 1 grid; Galerkin hierarchy
    A_c = P^T A P down to ``coarsest`` nodes per direction, where a sparse LU solves exactly.
    Damped Jacobi with weight ``omega``, ``nu`` sweeps before and after the coarse-grid
    correction. For a symmetric A the cycle is a symmetric operator."""

    def __init__(self, A: sp.spmatrix, dim: int, n: int, coarsest: int = 9, nu: int = 2,
                 omega: Optional[float] = None):
        self.nu = nu
        self.omega = (0.8 if dim == 2 else 0.7) if omega is None else omega
        self.levels: List[_Level] = []
        A = A.tocsr()
        while n > coarsest:
            P = prolongation(dim, n)
            self.levels.append(_Level(A, 1.0 / A.diagonal(), P))
            A = (P.T @ A @ P).tocsr()
            n = (n + 1) // 2
        self.coarse = spla.splu(A.tocsc())

    def _cycle(self, k: int, b: np.ndarray) -> np.ndarray:
        if k == len(self.levels):
            return self.coarse.solve(b)
        lv = self.levels[k]
        x = self.omega * lv.dinv * b
        for _ in range(self.nu - 1):
            x = x + self.omega * lv.dinv * (b - lv.A @ x)
        r = b - lv.A @ x
        x = x + lv.P @ self._cycle(k + 1, lv.P.T @ r)
        for _ in range(self.nu):
            x = x + self.omega * lv.dinv * (b - lv.A @ x)
        return x

    def solve(self, b: np.ndarray, cycles: int = 1) -> np.ndarray:
        """``cycles`` V-cycles from x = 0."""
        if not self.levels:
            return self.coarse.solve(b)
        A0 = self.levels[0].A
        x = self._cycle(0, b)
        for _ in range(cycles - 1):
            x = x + self._cycle(0, b - A0 @ x)
        return x


# --------------------------------------------------------------------------------------
# the block-triangular preconditioner P_T
# --------------------------------------------------------------------------------------

class BlockTriangular:
    """z = P_T^{-1} r for r = (r_y, r_w, r_v, r_p) (Section 4):
        z_y = Chebyshev_20 (M + Theta_y)^{-1} r_y,
        (z_w, z_v) = (alpha D~_M + Theta_z)^{-1} (r_w, r_v)   (pointwise 2x2),
        z_p = S_hat^{-1} (L z_y - M z_w + M z_v - r_p),
        S_hat^{-1} t = (L + M_hat)^{-T} (M + Theta_y) (L + M_hat)^{-1} t."""

    def __init__(self, qp: QP, th_y, th_w, th_v, inner: str = "gmg", cheb_steps: int = 20,
                 vcycles: int = 2):
        n = qp.nI
        self.qp = qp
        self.n = n
        self.MT = (qp.Mcost + sp.diags(th_y)).tocsr()
        self.jac = qp.dM + th_y
        self.cheb_steps = cheb_steps
        self.lmin, self.lmax = fem.chebyshev_interval(qp.dim)
        a = qp.alpha
        dm = qp.dM
        # 2x2 blocks [[a d + th_w, -a d], [-a d, a d + th_v]] and their determinants
        self.z11 = a * dm + th_w
        self.z22 = a * dm + th_v
        self.z12 = -a * dm
        self.det = self.z11 * self.z22 - self.z12 * self.z12
        # M_hat of Section 4.2 in the cancellation-free form sqrt(d^2 s / (1 + a d s) (d + th_y)),
        # s = 1/th_w + 1/th_v, algebraically equal to the printed expression
        s_ = 1.0 / th_w + 1.0 / th_v
        mh = np.sqrt(dm * dm * s_ / (1.0 + a * dm * s_) * (dm + th_y))
        self.LM = (qp.L + sp.diags(mh)).tocsr()
        self.inner = inner
        self.vcycles = vcycles
        if inner == "gmg":
            self.gmg = GMG(self.LM, qp.dim, qp.n)
            self.gmg_t = self.gmg if _symmetric(self.LM) else GMG(self.LM.T.tocsr(), qp.dim, qp.n)
        elif inner == "lu":
            self.lu = spla.splu(self.LM.tocsc())
        else:
            raise ValueError(inner)

    def _lm_solve(self, t: np.ndarray, transpose: bool) -> np.ndarray:
        if self.inner == "lu":
            return self.lu.solve(t, trans="T" if transpose else "N")
        g = self.gmg_t if transpose else self.gmg
        return g.solve(t, self.vcycles)

    def __call__(self, r: np.ndarray) -> np.ndarray:
        n = self.n
        ry, rw, rv, rp = r[:n], r[n:2 * n], r[2 * n:3 * n], r[3 * n:]
        zy = blocks.chebyshev(self.MT, self.jac, ry, self.cheb_steps, self.lmin, self.lmax)
        zw = (self.z22 * rw - self.z12 * rv) / self.det
        zv = (self.z11 * rv - self.z12 * rw) / self.det
        qp = self.qp
        t = qp.L @ zy - qp.M @ zw + qp.M @ zv - rp
        s = self._lm_solve(t, False)
        s = self.MT @ s
        zp = self._lm_solve(s, True)
        return np.concatenate([zy, zw, zv, zp])


def _symmetric(A: sp.csr_matrix) -> bool:
    d = A - A.T
    return d.nnz == 0 or abs(d).max() <= 1e-14 * abs(A).max()


# --------------------------------------------------------------------------------------
# flexible GMRES
# --------------------------------------------------------------------------------------

@dataclasses.dataclass
class KrylovStats:
    iterations: int
    relres: float
    setup_s: float = 0.0    # preconditioner construction (multigrid hierarchy or LU)
    solve_s: float = 0.0    # the FGMRES iterations


def fgmres(A: sp.spmatrix, b: np.ndarray, prec: Callable[[np.ndarray], np.ndarray],
           tol: float = 1e-12, restart: int = 40, maxiter: int = 2000):
    """Right-preconditioned flexible GMRES (Saad): x = x_0 + Z_j y_j with Z the preconditioned
    Arnoldi vectors, y_j minimising ||beta e_1 - H_j y|| (Givens rotations), modified
    Gram-Schmidt applied twice. Each cycle ends when the Arnoldi estimate of the residual
    reaches tol ||b|| or after ``restart`` steps; the solve ends when the TRUE residual
    ||b - A x|| / ||b|| computed from A is at most ``tol``."""
    nb = float(np.linalg.norm(b))
    x = np.zeros_like(b)
    if nb == 0.0:
        return x, KrylovStats(0, 0.0)
    total = 0
    r = b.copy()
    beta = nb
    best = nb
    while True:
        V = [r / beta]
        Z = []
        H = np.zeros((restart + 1, restart))
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        j = 0
        while j < restart and total < maxiter:
            z = prec(V[j])
            Z.append(z)
            w = A @ z
            for _ in range(2):
                for i in range(j + 1):
                    hij = float(V[i] @ w)
                    H[i, j] += hij
                    w -= hij * V[i]
            hnext = float(np.linalg.norm(w))
            H[j + 1, j] = hnext
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = math.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / den
            sn[j] = H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            total += 1
            j += 1
            if abs(g[j]) <= 0.1 * tol * nb or hnext == 0.0:
                break
            V.append(w / hnext)
        y = np.linalg.solve(np.triu(H[:j, :j]), g[:j])
        for i in range(j):
            x += y[i] * Z[i]
        r = b - A @ x
        beta = float(np.linalg.norm(r))
        if beta <= tol * nb or total >= maxiter:
            return x, KrylovStats(total, beta / nb)
        if beta > 0.5 * best:
            # a whole cycle without halving the true residual: the attainable accuracy of
            # FP64 for this system is reached
            return x, KrylovStats(total, beta / nb)
        best = beta


def newton_solver(inner: str = "gmg", tol: float = 1e-12, restart: int = 40,
                  vcycles: int = 2, stats: Optional[list] = None, accept: float = 1e-10,
                  maxiter: int = 2000):
    """A Newton-system solver for ``oracle.ipm.solve``: FGMRES + P_T to true relative
    residual ``tol``, or until a restart cycle no longer halves it (the FP64 attainable
    accuracy, which for strongly scaled late barrier systems lies near 1e-12); a final
    true relative residual above ``accept`` raises (``maxiter`` caps the iterations, for
    timing samples). Appends a :class:`KrylovStats` per solve to ``stats`` if given."""

    def solve(qp: QP, A: sp.spmatrix, b: np.ndarray, th_y, th_w, th_v) -> np.ndarray:
        t0 = time.perf_counter()
        P = BlockTriangular(qp, th_y, th_w, th_v, inner=inner, vcycles=vcycles)
        t1 = time.perf_counter()
        x, st = fgmres(A.tocsr(), b, P, tol=tol, restart=restart, maxiter=maxiter)
        st.setup_s = t1 - t0
        st.solve_s = time.perf_counter() - t1
        if not st.relres <= accept:
            raise RuntimeError(f"FGMRES did not reach {accept:g}: {st.relres:.3e} "
                               f"after {st.iterations} iterations")
        if stats is not None:
            stats.append(st)
        return x

    return solve
