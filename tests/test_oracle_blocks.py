"""Pins of the oracle's Section 4 matrices against the paper's theorems (dense, tiny grids)."""
import numpy as np
import pytest

import workloads as W
from oracle import blocks, fem
from oracle import qp as Q


def _qp(n=7, alpha=1e-2, lump=False, kind="poisson"):
    return Q.build(2, n, alpha, 1e-2, -2.0, 1.5, yd=W.yd_sin_product(n), lump=lump, kind=kind,
                   eps=1.0 / 20.0)


def _thetas(nI, seed, spread=6.0):
    rng = np.random.default_rng(seed)
    return tuple(10.0 ** rng.uniform(-spread, spread, nI) for _ in range(3))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_schur_formula_identity(seed):
    """(Schur): B A^{-1} B^T equals L(M+Th_y)^{-1}L^T + M/alpha - alpha^-2 (Th_w^-1 + Th_v^-1 + M^-1/alpha)^-1."""
    qp = _qp()
    th = _thetas(qp.nI, seed, spread=3.0)
    A, B = blocks.blocks(qp, *th)
    S = blocks.schur_exact(A, B)
    Sf = blocks.schur_formula(qp, *th)
    assert np.abs(S - Sf).max() < 1e-9 * np.abs(S).max()


@pytest.mark.parametrize("seed,alpha", [(0, 1e-2), (1, 1e-4), (2, 1e-6), (3, 1.0)])
def test_theorem1_zblock_interval(seed, alpha):
    qp = _qp(alpha=alpha)
    _, th_w, th_v = _thetas(qp.nI, seed)
    ex, ap = blocks.zblock(qp, th_w, th_v)
    lam = np.linalg.eigvals(np.linalg.solve(ap, ex)).real
    M = qp.M.toarray()
    mu = np.linalg.eigvals(M / np.diag(M)[:, None]).real
    lo, hi = min(mu.min(), 1.0), max(mu.max(), 1.0)
    assert lam.min() >= lo * (1 - 1e-9) and lam.max() <= hi * (1 + 1e-9)


@pytest.mark.parametrize("seed,alpha", [(0, 1e-2), (1, 1e-4), (2, 1e-6)])
def test_schur_approx_lower_bound_lumped(seed, alpha):
    """Theorem of Section 4.2: lambda(S_hat^{-1} S) >= 1/2 for a lumped mass matrix."""
    qp = _qp(alpha=alpha, lump=True)
    th = _thetas(qp.nI, seed)
    A, B = blocks.blocks(qp, *th)
    S = blocks.schur_exact(A, B)
    Sh = blocks.schur_approx(qp, *th)
    lam = np.linalg.eigvals(np.linalg.solve(Sh, S)).real
    assert lam.min() >= 0.5 - 1e-9


@pytest.mark.parametrize("kind", ["poisson", "cd"])
def test_schur_approx_clusters_consistent_mass(kind):
    """Remark after the theorem and its eigenvalue figure (h = 2^-4, late IPM iterates): with
    consistent mass the eigenvalues of S_hat^{-1} S are mostly clustered in [1/2, 1]."""
    from oracle import ipm
    qp = _qp(n=17, kind=kind)
    r = ipm.solve(qp, n_iter=8)
    th = ipm.thetas(qp, r.state)
    A, B = blocks.blocks(qp, *th)
    lam = np.linalg.eigvals(np.linalg.solve(blocks.schur_approx(qp, *th),
                                            blocks.schur_exact(A, B)))
    assert np.abs(lam.imag).max() < 1e-6 * np.abs(lam).max() or kind == "cd"
    lam = lam.real
    assert lam.min() > 0.3
    assert np.mean((lam > 0.45) & (lam < 1.05)) > 0.8


@pytest.mark.parametrize("kind", ["poisson", "cd"])
def test_ideal_preconditioners(kind):
    """lambda(P_1^{-1} calA) in {1, (1 +- sqrt 5)/2}; P_2^{-1} calA - I is nilpotent of index 2
    (hence MINRES/GMRES converge in 3/2 iterations)."""
    qp = _qp(n=5, kind=kind)
    th = _thetas(qp.nI, 7, spread=2.0)
    A, B = blocks.blocks(qp, *th)
    K = blocks.saddle(A, B)
    S = blocks.schur_exact(A, B)
    n = qp.nI
    Z = np.zeros((n, 3 * n))
    P1 = np.block([[A, Z.T], [Z, S]])
    P2 = np.block([[A, Z.T], [B, -S]])
    T1 = np.linalg.solve(P1, K)
    I = np.eye(K.shape[0])
    r5 = np.sqrt(5.0)
    poly = (T1 - I) @ (T1 - 0.5 * (1 + r5) * I) @ (T1 - 0.5 * (1 - r5) * I)
    assert np.abs(poly).max() < 1e-8
    T2 = np.linalg.solve(P2, K) - I
    assert np.abs(T2 @ T2).max() < 1e-8
    assert np.abs(T2).max() > 1e-3


def test_mhat_stable_form_identity():
    """The cancellation-free M_hat form d^2 s/(1 + alpha d s) (d + th_y), s = 1/th_w + 1/th_v,
    equals the printed formula where the printed one does not cancel."""
    rng = np.random.default_rng(3)
    d = 10.0 ** rng.uniform(-6, -2, 200)
    tw, tv, ty = (10.0 ** rng.uniform(-4, 4, 200) for _ in range(3))
    for alpha in (1e-2, 1e-4, 1e-6):
        ref = blocks.mhat(d, ty, tw, tv, alpha)
        s = 1.0 / tw + 1.0 / tv
        st = np.sqrt(d * d * s / (1.0 + alpha * d * s) * (d + ty))
        ok = alpha * d * s > 1e-6            # the printed form cancels catastrophically below this
        assert np.abs(st[ok] / ref[ok] - 1.0).max() < 1e-8


@pytest.mark.parametrize("dim,n", [(2, 9), (3, 5)])
def test_chebyshev_error_bound(dim, n):
    """20 Chebyshev steps on M + Theta_y with the Jacobi splitting obey ||e||_A <= ||e0||_A / T_20."""
    qp = Q.build(dim, n, 1e-2, 1e-2, -1.0, 1.0)
    rng = np.random.default_rng(dim)
    th = 10.0 ** rng.uniform(-8, 0, qp.nI) * qp.dM.max()
    A = qp.M.toarray() + np.diag(th)
    jac = np.diag(A)
    b = rng.standard_normal(qp.nI)
    lo, hi = fem.chebyshev_interval(dim)
    x = blocks.chebyshev(A, jac, b, 20, lo, hi)
    xs = np.linalg.solve(A, b)
    e, e0 = x - xs, xs

    def an(v):
        return np.sqrt(v @ A @ v)
    assert an(e) <= an(e0) * blocks.chebyshev_error_factor(20, lo, hi) * (1 + 1e-8)
    assert an(e) <= 1e-4 * an(e0) if dim == 2 else True
