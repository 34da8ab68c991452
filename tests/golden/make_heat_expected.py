"""Write the oracle's expected values for the heat-equation parity test at 33^2 x 31 levels
(calls only ``oracle/``).

The all-at-once heat problem (Section 3.4, backward Euler, rectangle rule in time) on a
33^2 grid with 31 time levels on [0, 1/2], inputs from ``workloads.heat_moving_target``,
alpha = 1e-2, beta = 1e-3, u in [-2, 1.5], sigma = 0.25. The oracle runs Algorithm A.1 from
the central-path start with every Newton system solved by FGMRES + P_T (exact LU for
calL + M_hat, ``oracle.iterative``) to the FP64 attainable accuracy, until kkt_rel <= 1e-6,
and stores the final y, u, p in the space-time layout of an n^3 array (plane k = time level
k, plane 0 the initial state), with k, mu and kkt_rel. (The direct tier's 4N x 4N sparse LU
at this size takes many minutes; the iterative tier about one.)

Usage: python tests/golden/make_heat_expected.py
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W                      # noqa: E402
from oracle import fem, heat, ipm, iterative  # noqa: E402

N, T = 33, 0.5
ALPHA, BETA, UA, UB, SIGMA = 1e-2, 1e-3, -2.0, 1.5, 0.25
OUT = os.path.join(HERE, f"heat_{N}.npz")


def embed(n: int, x_st: np.ndarray) -> np.ndarray:
    """Space-time interior vector -> n^3 array (planes 1 .. n-2), zero elsewhere."""
    out = np.zeros((n, n * n))
    out[1:n - 1][:, fem.interior(2, n)] = np.asarray(x_st).reshape(n - 2, -1)
    return out.reshape(-1)


def main() -> str:
    data = W.heat_moving_target(N, T)
    qp = heat.build_heat(N, N - 2, T, ALPHA, BETA, UA, UB, yd=data["yd"], y0=data["y0"])
    stats = []
    t0 = time.time()
    r = ipm.solve(qp, sigma=SIGMA, stop="kkt", kkt_tol=1e-6, max_iter=60,
                  newton_solve=iterative.newton_solver("lu", stats=stats))
    if not r.converged:
        raise RuntimeError("the oracle did not reach kkt_rel 1e-6")
    y = embed(N, r.state.y) + data["g3"]     # the state carries y_0 on plane 0
    u = embed(N, r.u())
    p = embed(N, r.state.p)
    np.savez_compressed(OUT, n=N, T=T, alpha=ALPHA, beta=BETA, ua=UA, ub=UB, sigma=SIGMA,
                        k=len(r.history) - 1, mu=r.state.mu,
                        kkt_rel=r.history[-1]["kkt_rel"], y=y, u=u, p=p,
                        krylov_iters=np.array([s.iterations for s in stats]),
                        krylov_relres=np.array([s.relres for s in stats]))
    print(f"heat {N}^2 x {N - 2}: k={len(r.history) - 1} kkt_rel={r.history[-1]['kkt_rel']:.3e} "
          f"Krylov {sum(s.iterations for s in stats)}  {time.time() - t0:.0f} s -> {OUT}",
          flush=True)
    return OUT


if __name__ == "__main__":
    main()
