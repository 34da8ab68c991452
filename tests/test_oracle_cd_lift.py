"""Pins of the oracle's convection direction and Dirichlet lift against closed forms (no GPU).

Convection (Section 5.2, wind w = (2 x2 (1 - x1^2), -2 x1 (1 - x2^2))). Linear functions lie
in the Q1 space, so for the Galerkin convection matrix N_ij = int (w . grad phi_j) phi_i the
product with the nodal values of x1 is exactly int w1 phi_i. For an interior node (a, b) with
the tensor hat phi_i(x1, x2) = t(x1 - a) t(x2 - b), the one-dimensional moments of the hat are
int t = h, int x t = a h, int x^2 t = h (a^2 + h^2 / 6), hence
    (N x1)_i =  2 b (1 - a^2 - h^2/6) h^2,
    (N x2)_i = -2 a (1 - b^2 - h^2/6) h^2.
A flipped wind, swapped components or the transposed matrix change the sign or the pattern.

Dirichlet lift (Section 1, y = g on the boundary). A bilinear (trilinear) harmonic g = x1 x2
(x1 x2 x3) lies in the Q1 space, so the Galerkin state equation with u = f = 0 reproduces it
exactly at the interior nodes: L_II y_I = -(L g)_I must give y_I = g_I. A wrong sign of the
lift gives -g_I. For convection-diffusion, g = 1 solves the equation exactly (w . grad 1 = 0),
with and without SUPG (its residual vanishes).
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads as W
from oracle import fem
from oracle import qp as Q


@pytest.mark.parametrize("n", [9, 33, 65])
def test_convection_matrix_on_linear_functions(n):
    h = 1.0 / (n - 1)
    L, _, _ = fem.convdiff_matrices(n, eps=0.0, supg=False)     # L = N when eps = 0, no SUPG
    x1, x2 = (c.ravel() for c in W.node_coords(2, n))
    idx = fem.interior(2, n)
    a, b = x1[idx], x2[idx]
    want1 = 2.0 * b * (1.0 - a * a - h * h / 6.0) * h * h
    want2 = -2.0 * a * (1.0 - b * b - h * h / 6.0) * h * h
    got1 = (L @ x1)[idx]
    got2 = (L @ x2)[idx]
    scale = 2.0 * h * h
    assert np.abs(got1 - want1).max() < 1e-13 * scale
    assert np.abs(got2 - want2).max() < 1e-13 * scale
    # the closed forms themselves differ from the flipped / swapped / transposed variants
    assert np.abs(want1 + want1).max() > 0.1 * scale
    assert np.abs((L.T @ x1)[idx] - want1).max() > 0.1 * scale


@pytest.mark.parametrize("n", [9, 17, 33])
def test_dirichlet_lift_poisson_2d(n):
    x1, x2 = (c.ravel() for c in W.node_coords(2, n))
    g = x1 * x2
    qp = Q.build(2, n, 1e-2, 0.0, -1.0, 1.0, g=g)
    y = spla.spsolve(qp.L.tocsc(), qp.fvec)
    assert np.abs(y - g[qp.idx]).max() < 1e-12
    # the tracking data carry the lift too: c_y = (M (y_d - g_lift))_I
    assert np.abs(qp.cy - (qp.Mfull @ -qp.g_full)[qp.idx]).max() < 1e-15


@pytest.mark.parametrize("n", [5, 9])
def test_dirichlet_lift_poisson_3d(n):
    x1, x2, x3 = (c.ravel() for c in W.node_coords(3, n))
    g = x1 * x2 * x3
    qp = Q.build(3, n, 1e-2, 0.0, -1.0, 1.0, g=g)
    y = spla.spsolve(qp.L.tocsc(), qp.fvec)
    assert np.abs(y - g[qp.idx]).max() < 1e-12


@pytest.mark.parametrize("supg", [False, True])
def test_dirichlet_lift_convdiff_constant(supg):
    n = 33
    g = np.ones(n * n)
    qp = Q.build(2, n, 1e-2, 0.0, -1.0, 1.0, g=g, kind="cd", eps=1.0 / 50.0, supg=supg)
    y = spla.spsolve(qp.L.tocsc(), qp.fvec)
    assert np.abs(y - 1.0).max() < 1e-11


def test_dirichlet_lift_with_source():
    """Lift and source together: -Lap y = 2 with y = x1 x2 + x1 (1 - x1) on the boundary. The
    solution is the bilinear part plus a function of x1 alone; for the latter the tensor Q1
    system separates into the 1D P1 system (the stiffness in x2 annihilates constants), and
    1D P1 Galerkin solutions are exact at the nodes. So the nodal values are exact, and a
    wrong sign in the lift or in the source term leaves an O(1) error."""
    for n in (17, 33, 65):
        x1, x2 = (c.ravel() for c in W.node_coords(2, n))
        ex = x1 * x2 + x1 * (1.0 - x1)
        qp = Q.build(2, n, 1e-2, 0.0, -1.0, 1.0, f=np.full(n * n, 2.0), g=ex)
        y = spla.spsolve(qp.L.tocsc(), qp.fvec)
        assert np.abs(y - ex[qp.idx]).max() < 1e-11
