"""GPU kernels in isolation vs the oracle, through the C ABI (element-wise parity).

Sizes span one tile (3, 5 nodes), several tiles with ragged tails (33, 65, 129 nodes:
31, 63, 127 interior points against 32 x 8 thread tiles) and 3D grids.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import workloads as W
from oracle import blocks, fem, ipm as oipm
from oracle import qp as Q
from paper_1806_05896_gb300 import ipm

from gpu_util import dev, embed, embed4, host, interior4, iterate_arrays, rel, torch_cuda

pytestmark = pytest.mark.gpu

CASES = [(2, 3), (2, 5), (2, 33), (2, 65), (2, 129), (3, 3), (3, 5), (3, 17), (3, 33)]


EPS_CD = 1.0 / 50.0


def _qp(dim, n, alpha=1e-2, beta=1e-3, ua=-2.0, ub=1.5, kind="poisson", **kw):
    return Q.build(dim, n, alpha, beta, ua, ub, kind=kind, eps=EPS_CD, **kw)


def _solver(qp, ua=-2.0, ub=1.5, kind="poisson", **kw):
    return ipm.Solver(qp.dim, qp.n, qp.alpha, qp.beta, ua, ub, kind=kind, eps=EPS_CD, **kw)


def _thetas(nI, rng, spread=4.0):
    return [10.0 ** rng.uniform(-spread, spread, nI) for _ in range(3)]


@pytest.mark.parametrize("dim,n,kind", [c + ("poisson",) for c in CASES] +
                         [(2, 5, "cd"), (2, 33, "cd"), (2, 65, "cd"), (2, 257, "cd")])
def test_newton_apply_matches_oracle(dim, n, kind):
    """Saddle operator of (NewtonSystem), with L and L^T for the convection-diffusion case."""
    torch = torch_cuda()
    qp = _qp(dim, n, kind=kind)
    rng = np.random.default_rng(n + dim)
    th = _thetas(qp.nI, rng)
    x = rng.standard_normal(4 * qp.nI)
    A = oipm.newton_matrix(qp, *th)
    ref = A @ x
    s = _solver(qp, kind=kind)
    out = torch.empty(4 * n ** dim, dtype=torch.float64, device="cuda")
    s.newton_apply(*[dev(embed(qp, t)) for t in th], dev(embed4(qp, x)), out)
    got = interior4(qp, host(out))
    # element-wise, relative to each row's magnitude |A| |x|
    absA = abs(A) @ np.abs(x)
    assert np.max(np.abs(got - ref) / absA) < 1e-14
    # boundary entries of the output are zero
    full = host(out).reshape(4, -1)
    bmask = fem.boundary_mask(dim, n)
    assert np.all(full[:, bmask] == 0.0)
    s.close()


@pytest.mark.parametrize("n", [5, 33, 65, 257, 1025])
def test_newton_apply_float_float_matches_oracle(n):
    """The float-float saddle operator of the mixed FGMRES path (2D Poisson): element-wise
    within 2e-13 of |A| |x|: each float-float operation rounds at about 2^-46 = 1.4e-14
    relative to its operands, and a row adds about a dozen terms (Theta spans eight orders
    of magnitude here)."""
    torch = torch_cuda()
    qp = _qp(2, n)
    rng = np.random.default_rng(n + 7)
    th = _thetas(qp.nI, rng)
    x = rng.standard_normal(4 * qp.nI)
    A = oipm.newton_matrix(qp, *th)
    ref = A @ x
    s = _solver(qp)
    out = torch.empty(4 * n * n, dtype=torch.float64, device="cuda")
    s.newton_apply(*[dev(embed(qp, t)) for t in th], dev(embed4(qp, x)), out, float_float=True)
    got = interior4(qp, host(out))
    absA = abs(A) @ np.abs(x)
    assert np.max(np.abs(got - ref) / absA) < 2e-13
    full = host(out).reshape(4, -1)
    assert np.all(full[:, fem.boundary_mask(2, n)] == 0.0)
    s.close()


@pytest.mark.parametrize("dim,n", [(2, 5), (2, 33), (2, 65), (3, 9), (3, 17)])
def test_chebyshev_matches_oracle(dim, n):
    torch = torch_cuda()
    qp = _qp(dim, n)
    rng = np.random.default_rng(7)
    thy = 10.0 ** rng.uniform(-8, 2, qp.nI) * qp.dM.max()
    b = rng.standard_normal(qp.nI)
    A = (qp.M + sp.diags(thy)).tocsr()
    lo, hi = fem.chebyshev_interval(dim)
    ref = blocks.chebyshev(A, qp.dM + thy, b, 20, lo, hi)
    s = _solver(qp)
    x = torch.empty(n ** dim, dtype=torch.float64, device="cuda")
    s.chebyshev(20, dev(embed(qp, thy)), dev(embed(qp, b)), x)
    got = host(x)[qp.idx]
    assert rel(got, ref) < 1e-12
    s.close()


@pytest.mark.parametrize("dim,n,mlog", [(2, 33, (-6, 3)), (2, 129, (-6, 3)), (2, 33, (-3, -3)),
                                        (2, 257, (-3, -3))])
def test_vcycle_convdiff_contracts_and_transposes(dim, n, mlog):
    """Multigrid on L + diag(m) with the SUPG operator and Galerkin coarse operators: three
    cycles reduce the error, and the cycle on L^T + diag(m) is the adjoint of the cycle on
    L + diag(m) (Jacobi smoothing with equal pre/post counts)."""
    torch = torch_cuda()
    qp = _qp(dim, n, kind="cd")
    rng = np.random.default_rng(5)
    m = qp.dM * 10.0 ** rng.uniform(mlog[0], mlog[1], qp.nI)
    A = (qp.L + sp.diags(m)).tocsc()
    b = rng.standard_normal(qp.nI)
    u = rng.standard_normal(qp.nI)
    xs = spla.spsolve(A, b)
    s = _solver(qp, kind="cd")
    out = torch.empty(n ** dim, dtype=torch.float64, device="cuda")
    vb = host(s.vcycle(False, dev(embed(qp, m)), dev(embed(qp, b)), out))[qp.idx]
    assert np.linalg.norm(vb - xs) < 0.1 * np.linalg.norm(xs)
    vtu = host(s.vcycle(True, dev(embed(qp, m)), dev(embed(qp, u)), out))[qp.idx]
    assert abs(u @ vb - vtu @ b) < 1e-11 * np.linalg.norm(u) * np.linalg.norm(vb)
    s.close()


@pytest.mark.parametrize("flags", [0, 1])
@pytest.mark.parametrize("dim,n", [(2, 33), (2, 129), (2, 257), (3, 17), (3, 33)])
def test_vcycle_contracts_and_is_symmetric(dim, n, flags):
    """Three V-cycles from zero approximate (L + diag m)^{-1} b (error factor well below one) and
    define a symmetric operator (<u, V b> = <V u, b>), as MINRES with P_D requires."""
    torch = torch_cuda()
    qp = _qp(dim, n)
    rng = np.random.default_rng(3)
    m = qp.dM * 10.0 ** rng.uniform(-6, 3, qp.nI)
    A = (qp.L + sp.diags(m)).tocsc()
    b = rng.standard_normal(qp.nI)
    u = rng.standard_normal(qp.nI)
    xs = spla.spsolve(A, b)
    s = _solver(qp)
    out = torch.empty(n ** dim, dtype=torch.float64, device="cuda")
    vb = host(s.vcycle(False, dev(embed(qp, m)), dev(embed(qp, b)), out, kernel_flags=flags))[qp.idx]
    e = vb - xs
    an = lambda v: np.sqrt(v @ (A @ v))
    assert an(e) < 0.05 * an(xs)
    vu = host(s.vcycle(False, dev(embed(qp, m)), dev(embed(qp, u)), out, kernel_flags=flags))[qp.idx]
    assert abs(u @ vb - vu @ b) < 1e-12 * np.linalg.norm(u) * np.linalg.norm(vb)
    vt = host(s.vcycle(True, dev(embed(qp, m)), dev(embed(qp, b)), out, kernel_flags=flags))[qp.idx]
    assert np.array_equal(vt, vb)  # L symmetric: the transposed cycle is the same operator
    # one cycle contracts less than three
    v1 = host(s.vcycle(False, dev(embed(qp, m)), dev(embed(qp, b)), out, vcycles=1,
                       kernel_flags=flags))[qp.idx]
    assert an(v1 - xs) > an(e)
    if flags == 0 and dim == 2:
        # the fused tiled kernels compute the same cycle as the per-sweep kernels
        ref = host(s.vcycle(False, dev(embed(qp, m)), dev(embed(qp, b)), out, kernel_flags=1))[qp.idx]
        assert rel(vb, ref) < 1e-12
    s.close()


@pytest.mark.parametrize("flags", [0, 1])
@pytest.mark.parametrize("dim,n", [(2, 33), (2, 129), (3, 9)])
def test_preconditioner_blocks(dim, n, flags):
    """P_T^{-1} r: y-block = Chebyshev(20), (w, v)-block = exact 2x2 solves with D_M, p-block close
    to S_hat^{-1}(B x_A - r_p); P_D^{-1} is symmetric."""
    torch = torch_cuda()
    qp = _qp(dim, n)
    rng = np.random.default_rng(11)
    th = _thetas(qp.nI, rng, 3.0)
    th = [t * qp.dM.max() for t in th]
    r = rng.standard_normal(4 * qp.nI)
    s = _solver(qp)
    z = torch.empty(4 * n ** dim, dtype=torch.float64, device="cuda")
    thd = [dev(embed(qp, t)) for t in th]
    s.precond_apply(True, *thd, dev(embed4(qp, r)), z, kernel_flags=flags)
    zi = interior4(qp, host(z))
    nI = qp.nI
    ry, rw, rv, rp = (r[k * nI:(k + 1) * nI] for k in range(4))
    lo, hi = fem.chebyshev_interval(dim)
    A = (qp.M + sp.diags(th[0])).tocsr()
    zy = blocks.chebyshev(A, qp.dM + th[0], ry, 20, lo, hi)
    assert rel(zi[:nI], zy) < 1e-12
    _, zap = blocks.zblock(qp, th[1], th[2])
    zwv = np.linalg.solve(zap, np.concatenate([rw, rv]))
    assert rel(zi[nI:3 * nI], zwv) < 1e-13
    t = qp.L @ zi[:nI] - qp.M @ (zi[nI:2 * nI] - zi[2 * nI:3 * nI]) - rp
    if qp.nI > 5000:  # dense Schur approximation too large: check the other blocks only
        s.close()
        return
    Sh = blocks.schur_approx(qp, *th)
    zp = np.linalg.solve(Sh, t)
    assert rel(zi[3 * nI:], zp) < 0.1
    # P_D symmetric: <u, P^{-1} r> = <P^{-1} u, r>
    u = rng.standard_normal(4 * nI)
    zr = torch.empty_like(z)
    zu = torch.empty_like(z)
    s.precond_apply(False, *thd, dev(embed4(qp, r)), zr, kernel_flags=flags)
    s.precond_apply(False, *thd, dev(embed4(qp, u)), zu, kernel_flags=flags)
    a = u @ interior4(qp, host(zr))
    b = interior4(qp, host(zu)) @ r
    assert abs(a - b) < 1e-11 * abs(a)
    s.close()


@pytest.mark.parametrize("dim,n,k", [(2, 33, 3), (2, 33, 9), (2, 65, 7), (3, 9, 6)])
@pytest.mark.parametrize("krylov,prec,tol,flags", [(ipm.KRYLOV_GMRES_PT, ipm.PREC_FP64, 1e-8, 0),
                                                   (ipm.KRYLOV_GMRES_PT, ipm.PREC_FP64, 1e-8, 3),
                                                   (ipm.KRYLOV_MINRES_PD, ipm.PREC_FP64, 1e-7, 0),
                                                   (ipm.KRYLOV_GMRES_PT, ipm.PREC_MIXED, 1e-8, 0),
                                                   (ipm.KRYLOV_GMRES_PT, ipm.PREC_MIXED, 1e-8, 3)])
def test_newton_step_matches_direct_solve(dim, n, k, krylov, prec, tol, flags):
    """The preconditioned Krylov Newton direction equals the oracle's direct solve of
    (NewtonSystem) at an oracle iterate (Krylov tolerance 1e-10 relative residual)."""
    torch = torch_cuda()
    yd = W.yd_sin_product(n) if dim == 2 else W.yd_cube_sin(n)
    qp = Q.build(dim, n, 1e-2, 1e-3, -2.0, 1.5, yd=yd)
    st = oipm.solve(qp, n_iter=k).state
    mu = 0.2 * st.mu
    A = oipm.newton_matrix(qp, *oipm.thetas(qp, st))
    ref = oipm.solve_direct(A, oipm.newton_rhs(qp, st, mu))
    s = _solver(qp)
    s.set_data(yd)
    dx = torch.empty(4 * n ** dim, dtype=torch.float64, device="cuda")
    it, rr = s.newton_step([dev(a) for a in iterate_arrays(qp, st)], mu, dx, krylov=krylov,
                           precision=prec, kernel_flags=flags)
    got = interior4(qp, host(dx))
    assert rr < 1.5e-10
    assert 0 < it < 100
    assert rel(got, ref) < tol
    s.close()
