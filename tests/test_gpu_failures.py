"""Failure handling through the C ABI (GPU): the failure is made on the host, no kernel faults.

* Non-finite data: a NaN in the desired state makes the Newton right-hand side non-finite;
  the solve returns IPM_EBREAKDOWN (Krylov breakdown or non-finite values), and the solver
  stays usable: new data and a new solve succeed on the same device context.
* Wall-clock limit: with ipm_options.time_limit_s tiny the solve returns IPM_ETIMEOUT with the
  last iterate retrievable (strictly inside the control box).
"""
import numpy as np
import pytest

import workloads as W
from paper_1806_05896_gb300 import ipm

from gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("krylov,precision", [(ipm.KRYLOV_GMRES_PT, ipm.PREC_FP64),
                                              (ipm.KRYLOV_GMRES_PT, ipm.PREC_MIXED),
                                              (ipm.KRYLOV_MINRES_PD, ipm.PREC_FP64)])
def test_nan_in_desired_state_is_a_breakdown(krylov, precision):
    torch_cuda()
    wl = W.workload_c2(n=65, cell=1)
    s = ipm.Solver(2, wl.n, wl.alpha, wl.beta, wl.ua, wl.ub, wl.ya, wl.yb)
    try:
        yd = wl.yd.copy().reshape(-1)
        yd[(wl.n // 2) * wl.n + wl.n // 3] = np.nan
        s.set_data(yd)
        with pytest.raises(ipm.IpmError) as e:
            s.solve(krylov=krylov, precision=precision, stop=ipm.STOP_KKT, kkt_tol=1e-6,
                    common_step=1)
        assert e.value.code == ipm.EBREAKDOWN
        # the context is intact: the same solver solves clean data
        s.set_data(wl.yd)
        rep = s.solve(krylov=krylov, precision=precision, stop=ipm.STOP_KKT, kkt_tol=1e-6,
                      common_step=1)
        assert rep["status"] == ipm.OK and rep["kkt_rel"] <= 1e-6
    finally:
        s.close()


def test_time_limit_returns_timeout_with_iterate():
    torch_cuda()
    wl = W.workload_c2(n=257, cell=1)
    s = ipm.Solver(2, wl.n, wl.alpha, wl.beta, wl.ua, wl.ub, wl.ya, wl.yb)
    try:
        s.set_data(wl.yd)
        full = s.solve(precision=ipm.PREC_FP64, stop=ipm.STOP_KKT, kkt_tol=1e-8, common_step=1)
        assert full["status"] == ipm.OK and full["ipm_iters"] >= 5
        # a limit of 1/4 of the full solve's wall time stops it early
        lim = 0.25 * full["seconds"]
        with pytest.raises(ipm.IpmError) as e:
            s.solve(precision=ipm.PREC_FP64, stop=ipm.STOP_KKT, kkt_tol=1e-8, common_step=1,
                    time_limit_s=lim)
        assert e.value.code == ipm.ETIMEOUT
        hist = s.history()
        k = int(hist[-1]["k"])
        assert 1 <= k < full["ipm_iters"]
        u = s.control()
        assert np.all(np.isfinite(u))
        assert u.max() < wl.ub and u.min() > wl.ua
        assert s.state().max() < wl.yb
        # a limit below any iteration's time: the start point is the iterate
        with pytest.raises(ipm.IpmError) as e:
            s.solve(precision=ipm.PREC_FP64, stop=ipm.STOP_KKT, kkt_tol=1e-8, time_limit_s=1e-9)
        assert e.value.code == ipm.ETIMEOUT
        assert len(s.history()) == 1
        assert np.all(s.control() == 0.0)
    finally:
        s.close()
