"""Pins of the all-at-once heat-equation oracle (time-dependent problems, backward Euler):
an exact discrete eigen-solution of the state equation, first-order convergence in time,
the brute-force optimum, a closed form (zero data), and a dense check of the Schur
complement formula against B A^{-1} B^T (the printed one lacks an inverse)."""
import math

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import blocks, brute, fem, heat
from oracle import ipm as oipm


def _grid(n):
    x = np.linspace(0.0, 1.0, n)
    X, Y = np.meshgrid(x, x, indexing="xy")
    return X.reshape(-1), Y.reshape(-1)


@pytest.mark.parametrize("n,nt", [(9, 3), (17, 5), (33, 8)])
def test_state_equation_is_backward_euler_on_a_q1_eigenvector(n, nt):
    """sin(pi x) sin(pi y) on the grid is an eigenvector of K v = lambda M v for Q1
    (tensor product of the 1D linear-element pair, lambda = 2 lambda_1 with
    lambda_1 = (6/h^2)(1 - cos(pi h))/(2 + cos(pi h))), so with u = f = 0 the discrete
    state must be (1 + tau lambda)^{-k} y_0 at step k, exactly."""
    T = 0.05
    X, Y = _grid(n)
    y0 = np.sin(math.pi * X) * np.sin(math.pi * Y)
    qp = heat.build_heat(n, nt, T, 1e-2, 1e-3, -1.0, 1.0, y0=y0)
    Ys = spla.spsolve(qp.L.tocsc(), qp.fvec).reshape(nt, -1)
    h = 1.0 / (n - 1)
    lam = 2.0 * (6.0 / h ** 2) * (1.0 - math.cos(math.pi * h)) / (2.0 + math.cos(math.pi * h))
    sidx = fem.interior(2, n)
    for k in range(nt):
        want = y0[sidx] * (1.0 + qp.tau * lam) ** (-(k + 1))
        assert np.max(np.abs(Ys[k] - want)) < 1e-12 * np.max(np.abs(y0))


def test_state_equation_converges_to_the_heat_kernel():
    """Backward Euler is first order in time: at fixed fine h the final-time error against
    exp(-2 pi^2 T) sin sin halves when tau halves."""
    n, T = 33, 0.05
    X, Y = _grid(n)
    y0 = np.sin(math.pi * X) * np.sin(math.pi * Y)
    sidx = fem.interior(2, n)
    errs = []
    for nt in (8, 16, 32):
        qp = heat.build_heat(n, nt, T, 1e-2, 1e-3, -1.0, 1.0, y0=y0)
        yT = spla.spsolve(qp.L.tocsc(), qp.fvec).reshape(nt, -1)[-1]
        exact = math.exp(-2.0 * math.pi ** 2 * T) * y0[sidx]
        errs.append(np.linalg.norm(yT - exact) / np.linalg.norm(exact))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 1.7 < r1 < 2.3 and 1.7 < r2 < 2.3


def test_interior_point_oracle_matches_brute_force():
    """The oracle's IPM on the space-time QP reaches the plain-definition optimum
    (coordinate descent on the reduced problem) on a tiny grid with several time steps."""
    n, nt, T = 5, 3, 0.3
    X, Y = _grid(n)
    yd = np.stack([2.0 * np.sin(2 * math.pi * X) * np.sin(math.pi * Y) * (k + 1) / nt
                   for k in range(nt)])
    qp = heat.build_heat(n, nt, T, 1e-2, 5e-3, -2.0, 1.5, yd=yd)
    N = qp.nI
    y_b, u_b, p_b, _ = brute.solve(qp, np.full(N, -2.0), np.full(N, 1.5))
    cert, counts = brute.certificate(qp, u_b, p_b, -2.0, 1.5, 1e-14)
    assert cert < 1e-14
    assert all(c > 0 for c in counts.values()), counts   # free, zero, upper and lower all occur
    r = oipm.solve(qp, n_iter=22)                          # mu = 0.2^22 ~ 4e-16
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
    assert rel(r.u(), u_b) < 1e-7
    assert rel(r.state.y, y_b) < 1e-8
    assert rel(r.state.p, p_b) < 1e-8


def test_zero_data_gives_zero_control():
    """y_d = 0, y_0 = 0, f = 0: the optimum is u = 0, y = 0 (beta > 0)."""
    qp = heat.build_heat(5, 2, 0.2, 1e-2, 1e-3, -1.0, 1.0)
    r = oipm.solve(qp, sigma=0.2, stop="kkt", kkt_tol=1e-10, max_iter=80, common_step=True)
    assert r.converged
    assert np.max(np.abs(r.u())) < 1e-8 and np.max(np.abs(r.state.y)) < 1e-8


def test_schur_complement_formula_and_the_printed_one():
    """Reading of the time-dependent Schur complement: the stationary (Schur) formula with
    M -> tau calM equals B A^{-1} B^T exactly; the printed expression, which lacks the
    inverse of (Theta_w^{-1} + Theta_v^{-1} + (alpha tau)^{-1} calM^{-1}), does not."""
    n, nt = 5, 3
    qp = heat.build_heat(n, nt, 0.3, 1e-2, 1e-3, -1.0, 1.0)
    rng = np.random.default_rng(5)
    th = [10.0 ** rng.uniform(-3, 3, qp.nI) for _ in range(3)]
    A, B = blocks.blocks(qp, *th)
    S = blocks.schur_exact(A, B)
    Sf = heat.schur_formula(qp, *th)
    assert np.linalg.norm(Sf - S) < 1e-10 * np.linalg.norm(S)
    calM = qp.M.toarray() / qp.tau
    a, tau = qp.alpha, qp.tau
    L = qp.L.toarray()
    Minv = np.linalg.inv(calM)
    printed = (L @ np.linalg.solve(tau * calM + np.diag(th[0]), L.T) + tau / a * calM
               - (1.0 / a ** 2) * calM @ Minv @ (np.diag(1.0 / th[1]) + np.diag(1.0 / th[2])
                                                 + Minv / (a * tau)) @ Minv @ calM)
    assert np.linalg.norm(printed - S) > 1e-3 * np.linalg.norm(S)


def test_schur_approximation_is_the_stationary_one_with_tau_mass():
    """M_hat of the time-dependent approximation equals the stationary M_hat evaluated with
    D_M -> tau D_M, and with exact mass the approximation's eigenvalues relative to S stay
    positive and bounded at late interior point iterates."""
    n, nt = 5, 3
    X, Y = _grid(n)
    yd = np.stack([np.sin(math.pi * X) * np.sin(math.pi * Y)] * nt)
    qp = heat.build_heat(n, nt, 0.3, 1e-2, 1e-3, -2.0, 1.5, yd=yd)
    r = oipm.solve(qp, sigma=0.2, n_iter=7, common_step=True)
    th = oipm.thetas(qp, r.state)
    assert np.allclose(heat.mhat(qp, *th), blocks.mhat(qp.dM, *th, qp.alpha), rtol=1e-14)
    A, B = blocks.blocks(qp, *th)
    S = blocks.schur_exact(A, B)
    Sh = heat.schur_approx(qp, *th)
    ev = np.linalg.eigvals(np.linalg.solve(Sh, S))
    assert np.all(ev.real > 0.1) and np.all(ev.real < 2.0)
