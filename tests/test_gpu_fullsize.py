"""Full-size checks on the 1025^2 Poisson workload (the benchmarked configuration) and the
multigrid tile kernels at every level size they run on.

The oracle's IPM with direct Newton solves does not finish at 1025^2, so these tests check
what the oracle can compute at that size: the saddle operator element by element, the
Newton system each Krylov solve must satisfy (residual against the oracle's matrix and
right-hand side), the V-cycle's contraction against the oracle's operator, and properties
of the final iterate (state equation, bounds, mixed vs FP64 agreement).
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import workloads as W
from oracle import blocks, fem
from oracle import ipm as oipm
from oracle import qp as Q
from paper_1806_05896_gb300 import ipm

from gpu_util import dev, embed, embed4, host, interior4, iterate_arrays, rel, torch_cuda

pytestmark = pytest.mark.gpu

N_FULL = 1025


@pytest.fixture(scope="module")
def full():
    """The 1025^2 sweep workload (cell 0) with its oracle QP and a GPU solver."""
    torch_cuda()
    wl = W.workload_c2(n=N_FULL, cell=0)
    qp = Q.from_workload(wl)
    s = ipm.Solver(2, N_FULL, wl.alpha, wl.beta, wl.ua, wl.ub, wl.ya, wl.yb)
    s.set_data(wl.yd)
    yield wl, qp, s
    s.close()


@pytest.mark.parametrize("n", [129, 257, 513, 1025])
def test_mixed_vcycle_tile_kernels(n):
    """Mixed-precision V-cycles (FP32 tile kernels, float-float outer residual and iterate):
    the fused tiled kernels agree with the per-sweep kernels and the FP64 cycles to FP32
    accuracy, the float-float outer step with the FP64 one, and the cycles contract the
    error of (L + diag m) x = b for the oracle's operator."""
    torch = torch_cuda()
    qp = Q.build(2, n, 1e-2, 1e-3, -2.0, 1.5)
    rng = np.random.default_rng(n)
    m = qp.dM * 10.0 ** rng.uniform(-6, 3, qp.nI)
    b = rng.standard_normal(qp.nI)
    A = (qp.L + sp.diags(m)).tocsr()
    s = ipm.Solver(2, n, qp.alpha, qp.beta, -2.0, 1.5)
    out = torch.empty(n * n, dtype=torch.float64, device="cuda")
    md, bd = dev(embed(qp, m)), dev(embed(qp, b))
    v = host(s.vcycle(False, md, bd, out, precision=ipm.PREC_MIXED))[qp.idx]
    v_sweep = host(s.vcycle(False, md, bd, out, precision=ipm.PREC_MIXED, kernel_flags=1))[qp.idx]
    v_o64 = host(s.vcycle(False, md, bd, out, precision=ipm.PREC_MIXED, kernel_flags=16))[qp.idx]
    # one persistent cooperative launch for the levels from 129^2 down vs one launch per level
    v_lvl = host(s.vcycle(False, md, bd, out, precision=ipm.PREC_MIXED, kernel_flags=128))[qp.idx]
    v64 = host(s.vcycle(False, md, bd, out))[qp.idx]
    # every candidate tile shape of the autotuner computes the same cycle bit for bit
    v_fixed = host(s.vcycle(False, md, bd, out, precision=ipm.PREC_MIXED, kernel_flags=512))[qp.idx]
    assert np.array_equal(v, v_fixed)
    assert f"pre_restrict n={n} " in ipm.tuning_report()  # the first mixed cycle tuned this grid
    if n in (257, 1025):
        levels = [n >> k | 1 for k in range(0, 4) if (n >> k | 1) > 65]
        for shape in range(7):
            for lv in levels:
                ipm.tuning_set(0, lv, shape)
                ipm.tuning_set(1, lv, shape)
            vs = host(s.vcycle(False, md, bd, out, precision=ipm.PREC_MIXED))[qp.idx]
            assert np.array_equal(vs, v), shape
        for lv in levels:
            ipm.tuning_set(0, lv, -1)
            ipm.tuning_set(1, lv, -1)
    s.close()
    # the per-sweep FP32 kernels take the stiffness stencil as 8 x_c - (sum of 8), the fused
    # ones on differences (x_c - x_nb): both within FP32 reach of the FP64 cycles
    assert rel(v, v_sweep) < 1e-5
    assert rel(v, v_o64) < 2e-6  # float-float vs FP64 outer residual
    assert rel(v, v_lvl) < 2e-6
    assert rel(v, v64) < 1e-5
    assert np.linalg.norm(b - A @ v) < 0.05 * np.linalg.norm(b)
    if n <= 513:
        xs = spla.spsolve(A.tocsc(), b)
        an = lambda e: np.sqrt(e @ (A @ e))
        assert an(v - xs) < 0.05 * an(xs)


@pytest.mark.parametrize("n", [129, 257, 513, 1025])
def test_mixed_preconditioner_tile_kernels(n):
    """P_T^{-1} r in mixed precision (FP32 Chebyshev and V-cycle tile kernels): the y-block
    is the oracle's 20-step Chebyshev to FP32 accuracy, the (w, v)-block the FP64 path's
    to FP32 accuracy, and the fused kernels agree with the per-sweep ones to FP32 accuracy."""
    torch = torch_cuda()
    qp = Q.build(2, n, 1e-2, 1e-3, -2.0, 1.5)
    rng = np.random.default_rng(n + 1)
    th = [t * qp.dM.max() for t in (10.0 ** rng.uniform(-3, 3, qp.nI) for _ in range(3))]
    r = rng.standard_normal(4 * qp.nI)
    s = ipm.Solver(2, n, qp.alpha, qp.beta, -2.0, 1.5)
    z = torch.empty(4 * n * n, dtype=torch.float64, device="cuda")
    thd = [dev(embed(qp, t)) for t in th]
    rd = dev(embed4(qp, r))
    zi = interior4(qp, host(s.precond_apply(True, *thd, rd, z, precision=ipm.PREC_MIXED)))
    zs = interior4(qp, host(s.precond_apply(True, *thd, rd, z, precision=ipm.PREC_MIXED,
                                            kernel_flags=1)))
    z64 = interior4(qp, host(s.precond_apply(True, *thd, rd, z)))
    s.close()
    nI = qp.nI
    lo, hi = fem.chebyshev_interval(2)
    A = (qp.M + sp.diags(th[0])).tocsr()
    zy = blocks.chebyshev(A, qp.dM + th[0], r[:nI], 20, lo, hi)
    assert rel(zi[:nI], zy) < 1e-5
    # the (w, v)-block: pointwise 2x2 solves, in FP32 on the mixed path
    assert rel(zi[nI:3 * nI], z64[nI:3 * nI]) < 1e-6
    for a, b in ((zi, zs), (zi, z64)):
        for k in range(4):
            blk = slice(k * nI, (k + 1) * nI)
            assert rel(a[blk], b[blk]) < 1e-5


def test_newton_apply_full_size(full):
    """(NewtonSystem) operator at 1025^2, element-wise against the oracle's matrix."""
    torch = torch_cuda()
    wl, qp, s = full
    rng = np.random.default_rng(11)
    th = [10.0 ** rng.uniform(-4, 4, qp.nI) for _ in range(3)]
    x = rng.standard_normal(4 * qp.nI)
    A = oipm.newton_matrix(qp, *th)
    ref = A @ x
    out = torch.empty(4 * N_FULL ** 2, dtype=torch.float64, device="cuda")
    s.newton_apply(*[dev(embed(qp, t)) for t in th], dev(embed4(qp, x)), out)
    got = interior4(qp, host(out))
    absA = abs(A) @ np.abs(x)
    assert np.max(np.abs(got - ref) / absA) < 1e-14


@pytest.mark.parametrize("prec", [ipm.PREC_MIXED, ipm.PREC_FP64])
def test_newton_step_full_size_solves_oracle_system(full, prec):
    """The Krylov Newton direction at 1025^2 (FGMRES + P_T, the benchmarked solver) solves
    the oracle's Newton system: relative residual ||A dx - rhs|| / ||rhs|| with the
    oracle's matrix and right-hand side at the oracle's starting iterate. The mixed path's
    float-float Arnoldi basis needs the same iterations as an FP64 basis."""
    torch = torch_cuda()
    wl, qp, s = full
    st = oipm.initial_state(qp)
    mu = wl.sigma * st.mu
    A = oipm.newton_matrix(qp, *oipm.thetas(qp, st))
    rhs = oipm.newton_rhs(qp, st, mu)
    dx = torch.empty(4 * N_FULL ** 2, dtype=torch.float64, device="cuda")
    it, rr = s.newton_step([dev(a) for a in iterate_arrays(qp, st)], mu, dx,
                           krylov=ipm.KRYLOV_GMRES_PT, precision=prec, krylov_tol=1e-10,
                           max_krylov=200)
    got = interior4(qp, host(dx))
    res = np.linalg.norm(A @ got - rhs) / np.linalg.norm(rhs)
    assert rr < 1.5e-10 and res < 2e-10
    assert 0 < it < 100
    if prec == ipm.PREC_MIXED:
        # the float-float Arnoldi basis converges like an FP64 one (kernel_flags bit 5)
        it64, rr64 = s.newton_step([dev(a) for a in iterate_arrays(qp, st)], mu, dx,
                                   krylov=ipm.KRYLOV_GMRES_PT, precision=prec, krylov_tol=1e-10,
                                   max_krylov=200, kernel_flags=32)
        assert abs(it - it64) <= 1 and rr64 < 1.5e-10


def test_full_size_solve_properties(full):
    """The benchmarked solve (mixed precision, FGMRES + P_T, kkt_rel <= 1e-6) and the same
    number of FP64 IPM steps: the iterate satisfies the bounds strictly, the state
    equation to the KKT tolerance (oracle matrices), and both precisions agree."""
    wl, qp, s = full
    opts = dict(krylov=ipm.KRYLOV_GMRES_PT, stop=ipm.STOP_KKT, kkt_tol=1e-6, restart=50,
                max_krylov=200, common_step=1, max_ipm=60, sigma=wl.sigma)
    rep = s.solve(precision=ipm.PREC_MIXED, **opts)
    assert rep["kkt_rel"] <= 1e-6
    y = s.state().reshape(-1)[qp.idx]
    u = s.control().reshape(-1)[qp.idx]
    assert np.all(u > wl.ua) and np.all(u < wl.ub)
    assert np.all(y < wl.yb)
    scale = 1.0 + np.linalg.norm(qp.fvec) + np.linalg.norm(qp.cy)
    assert np.linalg.norm(qp.L @ y - qp.M @ u - qp.fvec) / scale <= 1e-6
    # same IPM steps in FP64 (tight Krylov tolerance on both sides)
    k = rep["ipm_iters"]
    fixed = dict(opts, stop=ipm.STOP_FIXED, fixed_iters=k, krylov_tol=1e-10)
    s.solve(precision=ipm.PREC_MIXED, **fixed)
    um, ym, pm = (s.control().reshape(-1), s.state().reshape(-1), s.adjoint().reshape(-1))
    s.solve(precision=ipm.PREC_FP64, **fixed)
    u64, y64, p64 = (s.control().reshape(-1), s.state().reshape(-1), s.adjoint().reshape(-1))
    assert rel(um, u64) < 1e-6 and rel(ym, y64) < 1e-6 and rel(pm, p64) < 1e-6
