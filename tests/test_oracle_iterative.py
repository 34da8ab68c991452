"""The oracle's iterative tier (FGMRES + P_T Newton solves) against its direct tier (no GPU).

Both tiers run Algorithm A.1 with the same start and barrier schedule; the only difference
is how each Newton system is solved (sparse LU with refinement, or FGMRES to the FP64
attainable accuracy). The final iterates must agree to ~1e-11 relative: then the iterative
tier can stand in for the direct one at sizes where the LU is out of reach.
"""
import numpy as np
import pytest

import workloads as W
from oracle import fem, iterative, ipm
from oracle import qp as Q


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("make,inner,k", [
    (lambda: W.workload_c2(n=65, cell=1), "gmg", 10),
    (lambda: W.workload_c2(n=129, cell=3), "gmg", 6),
    (lambda: W.workload_c3(n=9), "gmg", 10),
    (lambda: W.workload_c3(n=17), "gmg", 5),
    (lambda: W.workload_c4(n=65), "lu", 10),
    (lambda: W.workload_c4(n=65), "gmg", 6),
])
def test_iterative_tier_matches_direct_tier(make, inner, k):
    wl = make()
    qp = Q.from_workload(wl)
    rd = ipm.solve(qp, sigma=wl.sigma, n_iter=k, common_step=True)
    stats = []
    ri = ipm.solve(qp, sigma=wl.sigma, n_iter=k, common_step=True,
                   newton_solve=iterative.newton_solver(inner, stats=stats))
    assert len(stats) == k and max(s.relres for s in stats) < 1e-10
    assert _rel(ri.u(), rd.u()) < 1e-11
    assert _rel(ri.state.y, rd.state.y) < 1e-11
    assert _rel(ri.state.p, rd.state.p) < 1e-11
    for a, b in zip(ri.history, rd.history):
        assert a["mu"] == b["mu"]


@pytest.mark.parametrize("dim,n", [(2, 9), (2, 17), (3, 9)])
def test_prolongation_is_exact_on_coarse_basis_functions(dim, n):
    """Interpolating a coarse unit vector gives the fine nodal values of that coarse Q1 hat
    function (a product of 1D hats of width 2h), and the Galerkin product P^T K P of the Q1
    stiffness equals the coarse grid's stiffness (nested Q1 spaces)."""
    nc = (n + 1) // 2
    H = 1.0 / (nc - 1)
    P = iterative.prolongation(dim, n)
    cf = [c.ravel()[fem.interior(dim, n)] for c in W.node_coords(dim, n)]
    cc = [c.ravel()[fem.interior(dim, nc)] for c in W.node_coords(dim, nc)]
    for j in (0, len(cc[0]) // 2, len(cc[0]) - 1):
        e = np.zeros(len(cc[0]))
        e[j] = 1.0
        hat = np.prod([np.maximum(0.0, 1.0 - np.abs(f - c[j]) / H) for f, c in zip(cf, cc)],
                      axis=0)
        assert np.abs(P @ e - hat).max() < 1e-15
    K, _ = fem.poisson_matrices(dim, n)
    Kc, _ = fem.poisson_matrices(dim, nc)
    i, ic = fem.interior(dim, n), fem.interior(dim, nc)
    G = (P.T @ K[i][:, i] @ P).toarray()
    assert np.abs(G - Kc[ic][:, ic].toarray()).max() < 1e-13


def test_fgmres_solves_a_nonsymmetric_system_exactly():
    """FGMRES with a variable (Jacobi-then-identity) preconditioner on a small nonsymmetric
    system reaches the requested true residual and the dense solution."""
    rng = np.random.default_rng(3)
    A = np.eye(60) * 4.0 + rng.standard_normal((60, 60)) * 0.3
    b = rng.standard_normal(60)
    calls = []

    def prec(r):
        calls.append(1)
        return r / np.diag(A) if len(calls) % 2 else r

    x, st = iterative.fgmres(A, b, prec, tol=1e-13, restart=7)
    assert st.relres <= 1e-13
    assert _rel(x, np.linalg.solve(A, b)) < 1e-12


@pytest.mark.parametrize("n,k", [(9, 8), (17, 6)])
def test_iterative_tier_matches_direct_tier_on_the_heat_equation(n, k):
    """The all-at-once heat problem (Section 3.4; calL block bidiagonal in time, so P_T's
    inner solves use the exact LU of calL + M_hat): both tiers give the same iterates."""
    from oracle import heat
    T = 0.5
    d = W.heat_moving_target(n, T)
    qp = heat.build_heat(n, n - 2, T, 1e-2, 1e-3, -2.0, 1.5, yd=d["yd"], y0=d["y0"])
    rd = ipm.solve(qp, sigma=0.25, n_iter=k)
    stats = []
    ri = ipm.solve(qp, sigma=0.25, n_iter=k,
                   newton_solve=iterative.newton_solver("lu", stats=stats))
    assert len(stats) == k and max(s.relres for s in stats) < 1e-10
    assert _rel(ri.u(), rd.u()) < 1e-11
    assert _rel(ri.state.y, rd.state.y) < 1e-11
    assert _rel(ri.state.p, rd.state.p) < 1e-11
    for a, b in zip(ri.history, rd.history):
        assert a["mu"] == b["mu"]
