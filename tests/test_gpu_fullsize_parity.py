"""Whole interior point solves at the benchmarked sizes against the oracle's iterative tier.

The expected values were written by ``tests/golden/make_fullsize_expected.py``, which runs
only the oracle (Algorithm A.1 with FGMRES + P_T Newton solves to the FP64 attainable
accuracy) to kkt_rel <= 1e-6 with the common step, and keeps the iterate's values on a coarse
grid of nodes covering the domain, on a dense patch, and the full vectors' 2-norms. The GPU
runs the same number of IPM steps (same mu^k) through the C ABI, FP64 and mixed precision.
Bars: relative L2 error <= 1e-8 (FP64, alpha >= 1e-4) and <= 1e-6 (mixed) on u, y and p over
the sampled nodes, and the same bars on the full vectors' norms.
"""
import os

import numpy as np
import pytest

import workloads as W
from paper_1806_05896_gb300 import ipm

from gpu_util import rel

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

CASES = {
    "poisson2d_1025_cell1": lambda: W.workload_c2(n=1025, cell=1),
    "poisson2d_1025_cell3": lambda: W.workload_c2(n=1025, cell=3),
    "cd2d_513": lambda: W.workload_c4(n=513),
    "poisson3d_65": lambda: W.workload_c3(n=65),
}


def _expected(name):
    path = os.path.join(GOLDEN, f"fullsize_{name}.npz")
    return dict(np.load(path))


def _solve(wl, k, precision):
    s = ipm.Solver(wl.dim, wl.n, wl.alpha, wl.beta, wl.ua, wl.ub, wl.ya, wl.yb, kind=wl.kind,
                   eps=wl.eps)
    try:
        s.set_data(wl.yd)
        rep = s.solve(stop=ipm.STOP_FIXED, fixed_iters=k, sigma=wl.sigma, common_step=1,
                      krylov=ipm.KRYLOV_GMRES_PT, precision=precision)
        out = dict(y=s.state().reshape(-1), u=s.control().reshape(-1),
                   p=s.adjoint().reshape(-1), hist=s.history())
    finally:
        s.close()
    return rep, out


@pytest.mark.parametrize("precision,bar", [(ipm.PREC_FP64, 1e-8), (ipm.PREC_MIXED, 1e-6)])
@pytest.mark.parametrize("name", sorted(CASES))
def test_full_size_solve_matches_oracle(name, precision, bar):
    ref = _expected(name)
    wl = CASES[name]()
    k = int(ref["k"])
    rep, got = _solve(wl, k, precision)
    assert rep["ipm_iters"] == k
    assert got["hist"][-1]["mu"] == pytest.approx(float(ref["mu"]), rel=1e-14)
    for f in ("y", "u", "p"):
        for part in ("grid", "patch"):
            idx = ref[f"{part}_idx"]
            e = rel(got[f][idx], ref[f"{f}_{part}"])
            assert e < bar, (f, part, e)
        nrm = float(ref[f"norm_{f}"])
        assert abs(np.linalg.norm(got[f]) - nrm) <= bar * nrm, f
    # the same stopping measure: both sides at kkt_rel <= 1e-6 after k steps
    assert got["hist"][-1]["kkt_rel"] <= 1e-6
    assert abs(got["hist"][-1]["kkt_rel"] - float(ref["kkt_rel"])) <= 1e-2 * float(ref["kkt_rel"])
