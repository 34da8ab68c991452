"""Pins of the oracle's Q1 assembly against facts the mathematics fixes (no GPU)."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import fem


def _kron_1d(n, dim):
    """Independent construction: tensor products of the assembled 1D P1 matrices."""
    h = 1.0 / (n - 1)
    e = np.ones(n)
    K1 = sp.diags([-e[:-1], 2 * e, -e[:-1]], [-1, 0, 1]).tolil()
    K1[0, 0] = K1[-1, -1] = 1.0
    K1 = K1.tocsr() / h
    M1 = sp.diags([e[:-1], 4 * e, e[:-1]], [-1, 0, 1]).tolil()
    M1[0, 0] = M1[-1, -1] = 2.0
    M1 = M1.tocsr() * h / 6.0
    if dim == 2:
        return sp.kron(K1, M1) + sp.kron(M1, K1), sp.kron(M1, M1)
    return (sp.kron(sp.kron(K1, M1), M1) + sp.kron(sp.kron(M1, K1), M1)
            + sp.kron(sp.kron(M1, M1), K1)), sp.kron(sp.kron(M1, M1), M1)


@pytest.mark.parametrize("dim,n", [(2, 5), (2, 9), (3, 5)])
def test_quadrature_assembly_matches_tensor_products(dim, n):
    K, M = fem.poisson_matrices(dim, n)
    Kk, Mk = _kron_1d(n, dim)
    assert abs(K - Kk).max() < 1e-13 * abs(Kk).max()
    assert abs(M - Mk).max() < 1e-13 * abs(Mk).max()


@pytest.mark.parametrize("dim,n", [(2, 9), (3, 5)])
def test_partition_of_unity_and_constants(dim, n):
    K, M = fem.poisson_matrices(dim, n)
    one = np.ones(n ** dim)
    assert abs(one @ (M @ one) - 1.0) < 1e-13            # |Omega| = 1
    assert np.abs(K @ one).max() < 1e-13                   # grad of a constant
    idx = fem.interior(dim, n)
    h = 1.0 / (n - 1)
    d = fem.lumped(M, idx)
    assert np.allclose(d, h ** dim, rtol=1e-13)            # int phi_i = h^d inside
    dM = M.diagonal()[idx]
    assert np.allclose(dM, (2.0 * h / 3.0) ** dim, rtol=1e-13)   # int phi_i^2


def test_interior_blocks_spd():
    K, M = fem.poisson_matrices(2, 9)
    idx = fem.interior(2, 9)
    for A in (K[idx][:, idx], M[idx][:, idx]):
        A = A.toarray()
        assert np.allclose(A, A.T)
        assert np.linalg.eigvalsh(A).min() > 0


@pytest.mark.parametrize("dim", [2, 3])
def test_manufactured_solution_second_order(dim):
    """-Lap y = d pi^2 prod sin(pi x_k) has y = prod sin(pi x_k); nodal error is O(h^2)."""
    errs = []
    ns = (9, 17, 33) if dim == 2 else (5, 9, 17)
    for n in ns:
        K, M = fem.poisson_matrices(dim, n)
        idx = fem.interior(dim, n)
        t = np.linspace(0, 1, n)
        grids = np.meshgrid(*([t] * dim), indexing="ij")
        ex = np.prod([np.sin(np.pi * g) for g in grids], axis=0).ravel()
        f = dim * np.pi ** 2 * ex
        Kii = K[idx][:, idx].tocsc()
        y = sp.linalg.spsolve(Kii, (M @ f)[idx])
        errs.append(np.abs(y - ex[idx]).max())
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert min(rates) > 1.8, (errs, rates)


@pytest.mark.parametrize("dim,n", [(2, 9), (3, 5)])
def test_mass_jacobi_interval(dim, n):
    """Spectrum of D_M^{-1} M (interior) inside the element bounds [2^-d, (3/2)^d] and equal
    to products of the 1D spectrum 1 + cos(k pi/(n-1))/2."""
    _, M = fem.poisson_matrices(dim, n)
    idx = fem.interior(dim, n)
    A = M[idx][:, idx].toarray()
    lam = np.linalg.eigvals(A / np.diag(A)[:, None]).real
    lo, hi = fem.chebyshev_interval(dim)
    assert lam.min() > lo and lam.max() < hi
    l1lo, l1hi = fem.q1_mass_jacobi_bounds_1d_interior(n)
    assert abs(lam.min() - l1lo ** dim) < 1e-12 and abs(lam.max() - l1hi ** dim) < 1e-12


def test_convection_part_skew_on_interior():
    """div w = 0 for the paper's wind, so int (w.grad phi_j) phi_i is skew on interior nodes."""
    n = 9
    L, M, delta = fem.convdiff_matrices(n, eps=1.0, supg=False)
    K, _ = fem.poisson_matrices(2, n)
    N = (L - K).tocsr()
    idx = fem.interior(2, n)
    Nii = N[idx][:, idx].toarray()
    assert np.abs(Nii + Nii.T).max() < 1e-14
    assert np.abs(Nii).max() > 1e-3
    assert np.all(delta == 0.0)


def test_convdiff_constants_and_supg():
    n = 17
    eps = 1.0 / 50.0
    L, M, delta = fem.convdiff_matrices(n, eps)
    one = np.ones(n * n)
    assert np.abs(L @ one).max() < 1e-13                  # constants are in the kernel
    assert np.any(delta > 0.0)
    Lg, _, dg = fem.convdiff_matrices(n, eps, supg=False)
    S = (L - Lg).toarray()
    assert np.allclose(S, S.T, atol=1e-15)
    assert np.linalg.eigvalsh(S).min() > -1e-13           # SUPG adds a PSD streamline term
    # large diffusion: element Peclet numbers below one switch SUPG off
    L2, _, d2 = fem.convdiff_matrices(n, 10.0)
    assert np.all(d2 == 0.0)


def test_supg_delta_formula_cases():
    h = 0.1
    # wind along x: element length h, Pe = |w| h / (2 eps)
    d = fem.supg_delta(np.array([2.0]), np.array([0.0]), h, 0.01)
    pe = 2.0 * h / 0.02
    assert abs(d[0] - h / 4.0 * (1 - 1 / pe)) < 1e-15
    # diagonal wind: element length h sqrt(2)
    d = fem.supg_delta(np.array([1.0]), np.array([1.0]), h, 0.01)
    he = h * np.sqrt(2.0)
    pe = np.sqrt(2.0) * he / 0.02
    assert abs(d[0] - he / (2 * np.sqrt(2.0)) * (1 - 1 / pe)) < 1e-15
    assert fem.supg_delta(np.array([0.0]), np.array([0.0]), h, 0.01)[0] == 0.0
