"""Partial observation on the GPU (the subsection on partial observations) against the oracle.

The tracking term integrates over the elements whose centre lies in
Omega_1 = {0.2 < x1 < 0.4, 0.4 < x2 < 0.9} (all x3), so the state row of (NewtonSystem)
carries the singular observation mass M_s; GMRES is preconditioned with P_Pi. Checked: the
saddle operator element-wise against the oracle's assembled matrix (cost mass M_s), and
whole solves at the same mu^k (FP64, rel-L2 <= 1e-8 on u, y, p), in 2D and 3D.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import ipm as oipm
from oracle import qp as Q
from paper_1806_05896_gb300 import ipm

from gpu_util import dev, embed, embed4, host, interior4, rel, torch_cuda

pytestmark = pytest.mark.gpu

LO, HI = (0.2, 0.4, -1.0), (0.4, 0.9, 2.0)


def omega1(c):
    return (c[:, 0] > 0.2) & (c[:, 0] < 0.4) & (c[:, 1] > 0.4) & (c[:, 1] < 0.9)


def _qp(dim, n, alpha=1e-2, beta=3e-3):
    coords = W.node_coords(dim, n)
    y = coords[1]
    yd = 10.0 * np.sin(4 * np.pi * (y - 0.4))
    if dim == 3:
        yd = 2.0 * yd * np.sin(np.pi * coords[2])
    return Q.build(dim, n, alpha, beta, -2.0, 1.5, yd=yd, observe=omega1), yd


@pytest.mark.parametrize("dim,n", [(2, 17), (2, 33), (3, 9)])
def test_partial_observation_operator(dim, n):
    torch = torch_cuda()
    qp, _ = _qp(dim, n)
    N = qp.nI
    rng = np.random.default_rng(n)
    th = [10.0 ** rng.uniform(-3, 3, N) * qp.dM[0] for _ in range(3)]
    x = rng.standard_normal(4 * N)
    A = oipm.newton_matrix(qp, *th)
    s = ipm.Solver(dim, n, qp.alpha, qp.beta, -2.0, 1.5)
    s.set_observation(LO[:dim], HI[:dim])
    out = torch.empty(4 * n ** dim, dtype=torch.float64, device="cuda")
    s.newton_apply(*[dev(embed(qp, t)) for t in th], dev(embed4(qp, x)), out)
    got = interior4(qp, host(out))
    s.close()
    want = A @ x
    scale = abs(A) @ abs(x)
    assert np.all(np.abs(got - want) <= 1e-13 * scale + 1e-300)


@pytest.mark.parametrize("dim,n", [(2, 17), (2, 33), (3, 9), (3, 17)])
def test_partial_observation_solve_matches_oracle(dim, n):
    torch_cuda()
    qp, yd = _qp(dim, n)
    ref = oipm.solve(qp, stop="kkt", kkt_tol=1e-10, max_iter=60)
    assert ref.converged
    k = len(ref.history) - 1
    s = ipm.Solver(dim, n, qp.alpha, qp.beta, -2.0, 1.5)
    s.set_observation(LO[:dim], HI[:dim])
    s.set_data(yd)
    rep = s.solve(stop=ipm.STOP_FIXED, fixed_iters=k, krylov=ipm.KRYLOV_GMRES_PT,
                  precision=ipm.PREC_FP64, krylov_tol=1e-12, max_krylov=400)
    got = dict(y=s.state().reshape(-1), u=s.control().reshape(-1), p=s.adjoint().reshape(-1))
    hist = s.history()
    s.close()
    want = dict(y=ref.y_full(qp), u=qp.full(ref.u()), p=qp.full(ref.state.p))
    for f in ("y", "u", "p"):
        assert rel(got[f], want[f]) < 1e-8, (f, rel(got[f], want[f]))
    assert rep["ipm_iters"] == k
    assert abs(hist[-1]["kkt_rel"] - ref.history[-1]["kkt_rel"]) <= 1e-3 * ref.history[-1]["kkt_rel"] + 1e-14


def test_partial_observation_arguments():
    torch_cuda()
    s = ipm.Solver(2, 17, 1e-2, 1e-3, -1.0, 1.0)
    with pytest.raises(ipm.IpmError):
        s.set_observation((0.41, 0.41), (0.42, 0.42))     # no element centre inside
    s.set_observation(LO[:2], HI[:2])
    s.set_data(np.zeros(17 * 17))
    with pytest.raises(ipm.IpmError):
        s.solve(precision=ipm.PREC_MIXED)                  # P_Pi runs in FP64
    s.set_observation()                                    # whole domain again
    s.set_data(np.zeros(17 * 17))
    rep = s.solve(stop=ipm.STOP_FIXED, fixed_iters=3)
    assert rep["ipm_iters"] == 3
    s.close()
