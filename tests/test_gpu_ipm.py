"""Whole interior point solves on the GPU vs the oracle (Algorithm A.1 with direct Newton solves).

Both sides run the same number of IPM iterations (same mu^k) from the same start and are
compared at their final iterates. Bars: relative L2 error <= 1e-8 on u, y, p for the FP64 path
(alpha >= 1e-4) and <= 1e-6 for the mixed path.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import ipm as oipm
from oracle import qp as Q
from paper_1806_05896_gb300 import ipm

from gpu_util import dev, host, rel, torch_cuda

pytestmark = pytest.mark.gpu


def _run_pair(wl, k, common=False, **opts):
    qp = Q.from_workload(wl)
    ref = oipm.solve(qp, sigma=wl.sigma, n_iter=k, common_step=common)
    s = ipm.Solver(wl.dim, wl.n, wl.alpha, wl.beta, wl.ua, wl.ub, wl.ya, wl.yb, kind=wl.kind,
                   eps=wl.eps)
    s.set_data(wl.yd)
    rep = s.solve(stop=ipm.STOP_FIXED, fixed_iters=k, sigma=wl.sigma, common_step=int(common),
                  **opts)
    got = dict(y=s.state().reshape(-1), u=s.control().reshape(-1), p=s.adjoint().reshape(-1))
    want = dict(y=ref.y_full(qp), u=qp.full(ref.u()), p=qp.full(ref.state.p))
    hist = s.history()
    s.close()
    return got, want, rep, hist, ref


def _iters_to(wl, tol, common=False):
    qp = Q.from_workload(wl)
    r = oipm.solve(qp, sigma=wl.sigma, stop="kkt", kkt_tol=tol, max_iter=40, common_step=common)
    assert r.converged
    return len(r.history) - 1


@pytest.mark.parametrize("krylov,flags", [(ipm.KRYLOV_MINRES_PD, 0), (ipm.KRYLOV_GMRES_PT, 0),
                                          (ipm.KRYLOV_GMRES_PT, 3)])
def test_poisson_33_fp64(krylov, flags):
    """The 33^2 Poisson configuration (alpha 1e-2, beta 1e-3, u in [-2, 2]) driven to kkt_rel 1e-10."""
    wl = W.workload_c1()
    k = _iters_to(wl, 1e-10)
    got, want, rep, hist, ref = _run_pair(wl, k, krylov=krylov, kernel_flags=flags)
    for f in ("y", "u", "p"):
        assert rel(got[f], want[f]) < 1e-8, (f, rel(got[f], want[f]))
    assert rep["ipm_iters"] == k and rep["krylov_relres_max"] < 1.5e-10
    for a, b in zip(hist, ref.history):
        assert a["mu"] == b["mu"]
        assert abs(a["kkt_rel"] - b["kkt_rel"]) <= 1e-6 * b["kkt_rel"] + 1e-14
        if a["k"] > 0:
            assert abs(a["alpha_P"] - b["alpha_P"]) < 1e-8 and abs(a["alpha_D"] - b["alpha_D"]) < 1e-8


@pytest.mark.parametrize("cell,common", [(0, False), (1, False), (2, False), (0, True), (3, True),
                                         (5, True)])
def test_gaussian_state_bound_65(cell, common):
    """y <= 0.1, Gaussian-sum y_d, u in [-30, 30] (the 1025^2 sweep's recipe at 65^2), alpha >= 1e-4,
    with Algorithm A.1's separate step lengths and with the common-step variant."""
    wl = W.workload_c2(n=65, cell=cell)
    k = _iters_to(wl, 1e-10, common)
    # these paths have blocked steps where tiny differences in the Newton direction change
    # alpha_P / alpha_D; a Krylov tolerance tighter than the default 1e-10 keeps the two
    # trajectories together over the 15-35 iterations to kkt_rel 1e-10
    got, want, rep, _, _ = _run_pair(wl, k, common, krylov_tol=1e-13)
    for f in ("y", "u", "p"):
        assert rel(got[f], want[f]) < 1e-8, (f, rel(got[f], want[f]))
    assert got["y"].max() <= 0.1


def test_gaussian_state_bound_65_blocked_path():
    """alpha = 1e-4, beta = 1e-3 (cell 4): from IPM step 9 on, most steps are blocked
    (alpha ~ 0.01-0.5) and alpha_P depends discontinuously on the Newton direction, so two
    correct runs follow different paths afterwards. Same-step parity holds before the
    blocked phase; both runs reach kkt_rel 1e-6. (Driving this cell much further, repeated
    blocking by one component shrinks its bound distance by 1 - alpha_0 per step until it
    underflows, in the oracle as on the GPU: a limit of Algorithm A.1, not of the kernels.)"""
    wl = W.workload_c2(n=65, cell=4)
    got, want, _, hist, ref = _run_pair(wl, 8, True)
    for f in ("y", "u", "p"):
        assert rel(got[f], want[f]) < 1e-8, (f, rel(got[f], want[f]))
    s = ipm.Solver(wl.dim, wl.n, wl.alpha, wl.beta, wl.ua, wl.ub, wl.ya, wl.yb)
    s.set_data(wl.yd)
    rep = s.solve(stop=ipm.STOP_KKT, kkt_tol=1e-6, max_ipm=60, common_step=1)
    assert rep["status"] == ipm.OK and rep["kkt_rel"] <= 1e-6
    assert s.state().max() <= 0.1
    s.close()


@pytest.mark.parametrize("cell,n", [(1, 65), (4, 65), (6, 65), (1, 129)])
def test_mixed_precision_gaussian(cell, n):
    wl = W.workload_c2(n=n, cell=cell)
    k = _iters_to(wl, 1e-6, True)
    got, want, rep, _, _ = _run_pair(wl, k, True, precision=ipm.PREC_MIXED)
    for f in ("y", "u", "p"):
        assert rel(got[f], want[f]) < 1e-6, (f, rel(got[f], want[f]))


@pytest.mark.parametrize("make", [lambda: W.workload_c1(), lambda: W.workload_c2(n=65, cell=1),
                                  lambda: W.workload_c2(n=129, cell=3)])
def test_mixed_minres_with_refinement(make):
    """MINRES + P_D on the mixed-precision path (FP32 Chebyshev, z-block and V-cycles) inside
    FP64 iterative refinement: every Newton system reaches the FP64 tolerance on its true
    residual, and the solve matches the oracle at the same mu^k within the mixed bar."""
    wl = make()
    common = wl.ya != -math.inf or wl.yb != math.inf
    k = _iters_to(wl, 1e-6, common)
    got, want, rep, _, _ = _run_pair(wl, k, common, krylov=ipm.KRYLOV_MINRES_PD,
                                     precision=ipm.PREC_MIXED)
    for f in ("y", "u", "p"):
        assert rel(got[f], want[f]) < 1e-6, (f, rel(got[f], want[f]))
    assert rep["krylov_relres_max"] < 1.5e-10


def test_gap_mu_rule_matches_oracle():
    wl = W.workload_c2(n=33, cell=3)
    qp = Q.from_workload(wl)
    ref = oipm.solve(qp, sigma=wl.sigma, n_iter=12, mu_rule="gap", common_step=True)
    s = ipm.Solver(2, 33, wl.alpha, wl.beta, wl.ua, wl.ub, wl.ya, wl.yb)
    s.set_data(wl.yd)
    s.solve(stop=ipm.STOP_FIXED, fixed_iters=12, mu_rule=1, common_step=1)
    h = s.history()
    for a, b in zip(h, ref.history):
        assert abs(a["mu"] - b["mu"]) <= 1e-9 * b["mu"]
    assert rel(s.control().reshape(-1), qp.full(ref.u())) < 1e-8
    s.close()


@pytest.mark.parametrize("n", [5, 9, 17])
def test_poisson_3d(n):
    wl = W.workload_c3(n=n)
    k = _iters_to(wl, 1e-10)
    got, want, rep, _, _ = _run_pair(wl, k)
    for f in ("y", "u", "p"):
        assert rel(got[f], want[f]) < 1e-8, (f, rel(got[f], want[f]))


@pytest.mark.parametrize("n,krylov,prec,tol", [(33, ipm.KRYLOV_GMRES_PT, ipm.PREC_FP64, 1e-8),
                                                (65, ipm.KRYLOV_GMRES_PT, ipm.PREC_FP64, 1e-8),
                                                (33, ipm.KRYLOV_MINRES_PD, ipm.PREC_FP64, 1e-8),
                                                (65, ipm.KRYLOV_GMRES_PT, ipm.PREC_MIXED, 1e-6)])
def test_convection_diffusion_supg(n, krylov, prec, tol):
    """Section 5.2 problem (eps = 1/50, recirculating wind, SUPG, u in [-2, 1.5],
    sigma = 0.25) at small grids against the oracle's assembled SUPG matrices."""
    wl = W.workload_c4(n=n)
    k = _iters_to(wl, 1e-10 if prec == ipm.PREC_FP64 else 1e-6, True)
    got, want, rep, _, _ = _run_pair(wl, k, True, krylov=krylov, precision=prec, krylov_tol=1e-12)
    for f in ("y", "u", "p"):
        assert rel(got[f], want[f]) < tol, (f, rel(got[f], want[f]))
    assert rep["krylov_relres_max"] < 2e-12


def test_single_unknown_and_tiny_grids():
    for n in (3, 5):
        wl = W.workload_c1(n=n)
        got, want, rep, _, _ = _run_pair(wl, 12)
        for f in ("y", "u", "p"):
            assert rel(got[f], want[f]) < 1e-8


def test_nodal_bounds_and_dirichlet_data():
    """Nodal bound arrays, an active lower state bound and non-zero boundary data g."""
    n = 17
    x, y = W.node_coords(2, n)
    ua = -1.0 - x
    ub = 1.0 + y
    g = 0.1 * np.sin(np.pi * x)  # boundary values used
    yd = W.yd_sin_product(n)
    qp = Q.build(2, n, 1e-3, 1e-3, ua, ub, ya=-0.05, yb=math.inf, yd=-yd, g=g)
    ref = oipm.solve(qp, n_iter=14)
    s = ipm.Solver(2, n, 1e-3, 1e-3, ua, ub, -0.05, math.inf)
    s.set_data(-yd, None, g)
    s.solve(stop=ipm.STOP_FIXED, fixed_iters=14)
    assert rel(s.control().reshape(-1), qp.full(ref.u())) < 1e-8
    assert rel(s.state().reshape(-1), ref.y_full(qp)) < 1e-8
    assert np.allclose(s.state()[0, :], g[0, :])
    s.close()


def test_paper_stopping_rule_and_report():
    wl = W.workload_c1()
    qp = Q.from_workload(wl)
    ref = oipm.solve(qp, stop="paper")
    s = ipm.Solver(2, 33, wl.alpha, wl.beta, wl.ua, wl.ub)
    s.set_data(wl.yd)
    rep = s.solve()  # paper defaults
    assert rep["status"] == ipm.OK
    assert rep["ipm_iters"] == len(ref.history) - 1
    assert rep["xi_c"] <= 1e-6 and rep["xi_p"] <= 1e-6 and rep["xi_d"] <= 1e-6
    s.close()


def test_deterministic_and_device_io():
    torch = torch_cuda()
    wl = W.workload_c2(n=65, cell=4)
    s = ipm.Solver(2, 65, wl.alpha, wl.beta, wl.ua, wl.ub, wl.ya, wl.yb)
    s.set_data_device(dev(wl.yd))
    s.solve(stop=ipm.STOP_KKT, kkt_tol=1e-8, common_step=1)
    u1 = s.control()
    s.set_data(wl.yd)
    s.solve(stop=ipm.STOP_KKT, kkt_tol=1e-8, common_step=1)
    u2 = s.control()
    assert np.array_equal(u1, u2)
    out = torch.empty(65 * 65, dtype=torch.float64, device="cuda")
    s.get_device("control", out)
    assert np.array_equal(host(out).reshape(65, 65), u2)
    s.close()


def test_errors_are_reported():
    with pytest.raises(ipm.IpmError) as e:
        ipm.Solver(2, 30, 1e-2, 1e-3, -1.0, 1.0)
    assert e.value.code == ipm.EINVAL
    with pytest.raises(ipm.IpmError) as e:
        ipm.Solver(2, 17, 1e-2, 1e-3, 0.0, 1.0)
    assert e.value.code == ipm.EINVAL
    with pytest.raises(ipm.IpmError) as e:
        ipm.Solver(2, 17, 0.0, 1e-3, -1.0, 1.0)
    assert e.value.code == ipm.EINVAL
    s = ipm.Solver(2, 17, 1e-2, 1e-3, -1.0, 1.0)
    with pytest.raises(ipm.IpmError) as e:
        s.solve()
    assert e.value.code == ipm.ESTATE
    with pytest.raises(ipm.IpmError) as e:
        s.state()
    assert e.value.code == ipm.ESTATE
    s.set_data(W.yd_sin_product(17))
    rep = s.solve(max_ipm=2)
    assert rep["status"] == ipm.ENOTCONV and rep["ipm_iters"] == 2
    s.close()


def test_krylov_reports_true_residual_with_boundary_data():
    """Non-zero boundary values of y_d must not leak into Krylov vectors: the reported final
    residual is the true one and repeated solves are bitwise identical."""
    wl = W.workload_c2(n=65, cell=1)
    assert np.abs(wl.yd[0, :]).max() > 1e-3
    s = ipm.Solver(2, 65, wl.alpha, wl.beta, wl.ua, wl.ub, wl.ya, wl.yb)
    s.set_data(wl.yd)
    r1 = s.solve(stop=ipm.STOP_KKT, kkt_tol=1e-8, common_step=1)
    h1 = s.history()
    u1 = s.control()
    r2 = s.solve(stop=ipm.STOP_KKT, kkt_tol=1e-8, common_step=1)
    assert np.array_equal(u1, s.control())
    assert [h["krylov_iters"] for h in h1] == [h["krylov_iters"] for h in s.history()]
    assert r1["krylov_relres_max"] < 1e-9 and r2["krylov_relres_max"] < 1e-9
    s.close()
