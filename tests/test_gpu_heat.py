"""The all-at-once heat equation on the GPU (Section 3.4) against the oracle (GPU).

The library stores the space-time problem with n - 2 backward-Euler steps on the planes
of an n^3 array (plane k = time level t_k, plane 0 the initial state). The oracle builds
the same QP (rectangle rule in time, block-bidiagonal calL) and runs Algorithm A.1 with
direct Newton solves. Checked: the saddle operator of (NewtonSystem) element-wise, and
whole solves at the same mu^k (FP64 <= 1e-8, mixed <= 1e-6 on u, y, p).
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import fem, heat
from oracle import ipm as oipm
from paper_1806_05896_gb300 import ipm

from gpu_util import dev, host, rel, torch_cuda

pytestmark = pytest.mark.gpu


def _data(n, T):
    """Desired state moving in time, a smooth initial state (n^3 nodal arrays and the
    oracle's (nt, n^2) arrays)."""
    nt = n - 2
    tau = T / nt
    x = np.linspace(0.0, 1.0, n)
    X, Y = np.meshgrid(x, x, indexing="xy")
    X, Y = X.reshape(-1), Y.reshape(-1)
    yd = np.stack([np.sin(math.pi * X) * np.sin(math.pi * Y) * (1.0 + 2.0 * (k + 1) * tau)
                   * np.cos(2.0 * math.pi * (k + 1) * tau) for k in range(nt)])
    y0 = 0.5 * np.sin(math.pi * X) * np.sin(2.0 * math.pi * Y)
    yd3 = np.zeros((n, n * n))
    yd3[1:n - 1] = yd
    g3 = np.zeros((n, n * n))
    g3[0] = y0
    g3[0][fem.boundary_mask(2, n)] = 0.0
    return yd, y0, yd3.reshape(-1), g3.reshape(-1)


def _embed(n, x_st):
    """Oracle space-time interior vector -> n^3 array (planes 1 .. n-2)."""
    nt = n - 2
    out = np.zeros((n, n * n))
    sidx = fem.interior(2, n)
    out[1:n - 1][:, sidx] = np.asarray(x_st).reshape(nt, -1)
    return out.reshape(-1)


@pytest.mark.parametrize("n", [9, 17])
def test_heat_newton_operator_matches_oracle(n):
    torch = torch_cuda()
    T = 0.5
    nt = n - 2
    qp = heat.build_heat(n, nt, T, 1e-2, 1e-3, -2.0, 1.5)
    N = qp.nI
    rng = np.random.default_rng(n)
    th = [10.0 ** rng.uniform(-3, 3, N) * qp.dM[0] for _ in range(3)]
    x = rng.standard_normal(4 * N)
    A = oipm.newton_matrix(qp, *th)
    want = A @ x
    s = ipm.Solver(2, n, qp.alpha, qp.beta, -2.0, 1.5, kind="heat", T=T)
    out = torch.empty(4 * n ** 3, dtype=torch.float64, device="cuda")
    xd = np.concatenate([_embed(n, x[b * N:(b + 1) * N]) for b in range(4)])
    s.newton_apply(*[dev(_embed(n, t)) for t in th], dev(xd), out)
    got = host(out)
    s.close()
    scale = abs(A) @ abs(x)
    for b in range(4):
        gb = got[b * n ** 3:(b + 1) * n ** 3].reshape(n, n * n)[1:n - 1][:, fem.interior(2, n)]
        wb = want[b * N:(b + 1) * N].reshape(nt, -1)
        sb = scale[b * N:(b + 1) * N].reshape(nt, -1)
        assert np.all(np.abs(gb - wb) <= 1e-13 * sb + 1e-300), b


# the oracle's direct space-time solve grows quickly (33^2 x 31 levels takes many minutes on
# the host): parity at 9^2 and 17^2 with 7 and 15 time levels
@pytest.mark.parametrize("n,prec,bar", [(9, ipm.PREC_FP64, 1e-8), (17, ipm.PREC_FP64, 1e-8),
                                        (9, ipm.PREC_MIXED, 1e-6), (17, ipm.PREC_MIXED, 1e-6)])
def test_heat_solve_matches_oracle(n, prec, bar):
    torch_cuda()
    T, alpha, beta, ua, ub, sigma = 0.5, 1e-2, 1e-3, -2.0, 1.5, 0.25
    yd, y0, yd3, g3 = _data(n, T)
    qp = heat.build_heat(n, n - 2, T, alpha, beta, ua, ub, yd=yd, y0=y0)
    ref = oipm.solve(qp, sigma=sigma, stop="kkt", kkt_tol=1e-10 if prec == ipm.PREC_FP64 else 1e-6,
                     max_iter=60)
    assert ref.converged
    k = len(ref.history) - 1
    s = ipm.Solver(2, n, alpha, beta, ua, ub, kind="heat", T=T)
    s.set_data(yd3, None, g3)
    rep = s.solve(stop=ipm.STOP_FIXED, fixed_iters=k, sigma=sigma, krylov=ipm.KRYLOV_GMRES_PT,
                  precision=prec, krylov_tol=1e-12 if prec == ipm.PREC_FP64 else 1e-10)
    got = dict(y=s.state().reshape(-1), u=s.control().reshape(-1), p=s.adjoint().reshape(-1))
    hist = s.history()
    s.close()
    want = dict(y=_embed(n, ref.state.y), u=_embed(n, ref.u()), p=_embed(n, ref.state.p))
    want["y"] = want["y"] + g3          # the state carries y_0 on level 0
    for f in ("y", "u", "p"):
        assert rel(got[f], want[f]) < bar, (f, rel(got[f], want[f]))
    assert rep["ipm_iters"] == k
    for a, b in zip(hist, ref.history):
        assert a["mu"] == pytest.approx(b["mu"], rel=1e-12)
    assert abs(hist[-1]["kkt_rel"] - ref.history[-1]["kkt_rel"]) <= 1e-3 * ref.history[-1]["kkt_rel"] + 1e-14


def test_heat_rejects_what_it_does_not_cover():
    torch_cuda()
    with pytest.raises(ipm.IpmError):
        ipm.Solver(2, 129, 1e-2, 1e-3, -1.0, 1.0, kind="heat", T=1.0)     # > 65 nodes
    with pytest.raises(ipm.IpmError):
        ipm.Solver(2, 9, 1e-2, 1e-3, -1.0, 1.0, yb=0.1, kind="heat", T=1.0)  # state bound
    s = ipm.Solver(2, 9, 1e-2, 1e-3, -1.0, 1.0, kind="heat", T=1.0)
    s.set_data(np.zeros(9 ** 3))
    with pytest.raises(ipm.IpmError):
        s.solve(krylov=ipm.KRYLOV_MINRES_PD)
    s.close()


# 33^2 with 31 time levels: expected values written by the oracle's iterative tier
# (tests/golden/make_heat_expected.py; the direct tier at this size takes many minutes)
@pytest.mark.parametrize("prec,bar", [(ipm.PREC_FP64, 1e-8), (ipm.PREC_MIXED, 1e-6)])
def test_heat_33_matches_oracle_iterative_tier(prec, bar):
    import os
    import workloads as W
    torch_cuda()
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "heat_33.npz")
    ref = dict(np.load(path))
    n, T, k = int(ref["n"]), float(ref["T"]), int(ref["k"])
    d = W.heat_moving_target(n, T)
    s = ipm.Solver(2, n, float(ref["alpha"]), float(ref["beta"]), float(ref["ua"]),
                   float(ref["ub"]), kind="heat", T=T)
    s.set_data(d["yd3"], None, d["g3"])
    rep = s.solve(stop=ipm.STOP_FIXED, fixed_iters=k, sigma=float(ref["sigma"]),
                  krylov=ipm.KRYLOV_GMRES_PT, precision=prec,
                  krylov_tol=1e-12 if prec == ipm.PREC_FP64 else 1e-10)
    got = dict(y=s.state().reshape(-1), u=s.control().reshape(-1), p=s.adjoint().reshape(-1))
    hist = s.history()
    s.close()
    assert rep["ipm_iters"] == k
    assert hist[-1]["mu"] == pytest.approx(float(ref["mu"]), rel=1e-12)
    for f in ("y", "u", "p"):
        assert rel(got[f], ref[f]) < bar, (f, rel(got[f], ref[f]))
    assert abs(hist[-1]["kkt_rel"] - float(ref["kkt_rel"])) <= 1e-2 * float(ref["kkt_rel"])
