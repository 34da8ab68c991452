"""Pins of the partial-observation oracle and of the preconditioner P_Pi.

* the observation mass integrates the observed area and reduces to M on the whole domain;
* the IPM with a singular tracking block reaches the brute-force optimum;
* P_Pi applied by its three solves equals the inverse of the permuted block-triangular
  matrix times the permutation;
* with the exact Schur complement S_Pi the preconditioned matrix has minimal polynomial
  (x - 1)(x + 1): GMRES converges in two iterations;
* with the approximation S_Pi_hat the eigenvalues stay real in [-1, 1] at a late iterate.
"""
import numpy as np

import workloads as W
from oracle import brute, fem, partial
from oracle import ipm as oipm
from oracle import qp as Q


def omega1(c):
    """Observation domain 0.2 < x1 < 0.4, 0.4 < x2 < 0.9 (all x3), element centres."""
    return (c[:, 0] > 0.2) & (c[:, 0] < 0.4) & (c[:, 1] > 0.4) & (c[:, 1] < 0.9)


def _qp(n=11, alpha=1e-2, beta=3e-3, amp=10.0, dim=2):
    x, y = W.node_coords(dim, n)[:2]
    yd = amp * np.sin(4 * np.pi * (y - 0.4))
    return Q.build(dim, n, alpha, beta, -2.0, 1.5, yd=yd, observe=omega1)


def test_observation_mass():
    """1^T M_s 1 is the observed area (element-aligned at h = 0.1); the whole domain gives M."""
    for dim, n in ((2, 11), (3, 11)):
        Ms = fem.mass_subdomain(dim, n, omega1)
        assert abs(Ms.sum() - 0.2 * 0.5) < 1e-13
        _, M = fem.poisson_matrices(dim, n)
        Mall = fem.mass_subdomain(dim, n, lambda c: np.ones(len(c), bool))
        assert abs(Mall - M).max() < 1e-15
    qp = _qp()
    assert qp.Mcost.shape == qp.M.shape and np.linalg.matrix_rank(qp.Mcost.toarray()) < qp.nI


def test_ipm_matches_brute_force_with_partial_observation():
    qp = _qp()
    N = qp.nI
    y_b, u_b, p_b, _ = brute.solve(qp, np.full(N, -2.0), np.full(N, 1.5))
    cert, counts = brute.certificate(qp, u_b, p_b, -2.0, 1.5, 1e-14)
    assert cert < 1e-15
    assert all(c > 0 for c in counts.values()), counts
    r = oipm.solve(qp, n_iter=22)
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
    assert rel(r.u(), u_b) < 1e-7
    assert rel(r.state.y, y_b) < 1e-8
    assert rel(r.state.p, p_b) < 1e-9


def test_ipm_matches_brute_force_with_partial_observation_3d():
    """The paper's three-dimensional case: observation in 0.2 < x1 < 0.4, 0.4 < x2 < 0.9,
    all x3 (9^3 grid)."""
    n = 9
    x, y, z = W.node_coords(3, n)
    yd = 20.0 * np.sin(4 * np.pi * (y - 0.4)) * np.sin(np.pi * z)
    qp = Q.build(3, n, 1e-2, 3e-3, -2.0, 1.5, yd=yd, observe=omega1)
    N = qp.nI
    y_b, u_b, p_b, _ = brute.solve(qp, np.full(N, -2.0), np.full(N, 1.5))
    cert, counts = brute.certificate(qp, u_b, p_b, -2.0, 1.5, 1e-14)
    assert cert < 1e-15
    assert all(c > 0 for c in counts.values()), counts
    r = oipm.solve(qp, n_iter=22)
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
    assert rel(r.u(), u_b) < 1e-7
    assert rel(r.state.y, y_b) < 1e-8
    assert rel(r.state.p, p_b) < 1e-9


def _late_thetas(qp, k=7):
    r = oipm.solve(qp, n_iter=k)
    return oipm.thetas(qp, r.state)


def test_three_solve_recipe_equals_the_dense_inverse():
    qp = _qp(n=7)
    th = _late_thetas(qp)
    w = np.random.default_rng(2).standard_normal(4 * qp.nI)
    v = partial.apply(qp, *th, w)
    Pinv = partial.matrix_inverse(qp, *th)
    assert np.linalg.norm(v - Pinv @ w) < 1e-10 * np.linalg.norm(v)


def test_exact_schur_complement_gives_two_gmres_iterations():
    qp = _qp(n=7)
    th = _late_thetas(qp)
    A = oipm.newton_matrix(qp, *th).toarray()
    S = partial.schur_pi(qp, *th)
    T = partial.matrix_inverse(qp, *th, S=S) @ A
    I = np.eye(T.shape[0])
    assert np.linalg.norm((T - I) @ (T + I)) < 1e-10 * np.linalg.norm(T)


def test_approximate_schur_complement_spectrum():
    for alpha, beta in ((1e-2, 1e-3), (1e-4, 1e-3), (1e-3, 1e-2)):
        qp = _qp(n=9, alpha=alpha, beta=beta)
        th = _late_thetas(qp)
        A = oipm.newton_matrix(qp, *th).toarray()
        ev = np.linalg.eigvals(partial.matrix_inverse(qp, *th) @ A)
        assert np.max(np.abs(ev.imag)) < 1e-8
        assert ev.real.min() > -1.0 - 1e-8 and ev.real.max() < 1.0 + 1e-8
        assert np.min(np.abs(ev.real)) > 1e-3
