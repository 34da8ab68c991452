"""Write the oracle's expected values for the full-size parity tests (calls only ``oracle/``).

For each configuration below the iterative tier of the oracle (Algorithm A.1, every Newton
system solved by FGMRES + P_T to the FP64 attainable accuracy, ``oracle.iterative``) runs
from the central-path start until kkt_rel <= 1e-6 (the common-step variant used by the
benchmark), and the final iterate is sampled:

* ``grid``  -- the values of y, u, p on every ``stride``-th node in each direction
  (boundary included), a coarse copy that covers the whole domain;
* ``patch`` -- a dense block of consecutive nodes in the middle of the domain (2D) or three
  consecutive dense planes (3D), for the fine-scale structure;
* ``norm_*`` -- the 2-norms of the full nodal vectors;
* ``k``, ``mu``, ``kkt_rel`` -- iteration count, barrier parameter and the oracle's kkt_rel.

Inputs come from ``workloads`` (seeded generators, no method arithmetic). Usage:
    python tests/golden/make_fullsize_expected.py [name ...]
Takes tens of minutes on one CPU core (the 1025^2 cases dominate).
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
from oracle import ipm, iterative          # noqa: E402
from oracle import qp as Q                 # noqa: E402

# name -> (workload factory, inner solver of (L + M_hat), sampling stride, patch)
CASES = {
    "poisson2d_1025_cell1": (lambda: W.workload_c2(n=1025, cell=1), "gmg", 8, (448, 512)),
    "poisson2d_1025_cell3": (lambda: W.workload_c2(n=1025, cell=3), "gmg", 8, (448, 512)),
    "cd2d_513": (lambda: W.workload_c4(n=513), "lu", 4, (224, 288)),
    "poisson3d_65": (lambda: W.workload_c3(n=65), "gmg", 4, (31, 34)),
}


def sample_indices(dim: int, n: int, stride: int, patch):
    """Full-grid flat indices of the coarse sample grid and of the dense patch."""
    g = np.arange(0, n, stride)
    p = np.arange(patch[0], patch[1])
    if dim == 2:
        gy, gx = np.meshgrid(g, g, indexing="ij")
        py, px = np.meshgrid(p, p, indexing="ij")
        return (gy * n + gx).ravel(), (py * n + px).ravel()
    gz, gy, gx = np.meshgrid(g, g, g, indexing="ij")
    full = np.arange(n)
    pz, py, px = np.meshgrid(p, full, full, indexing="ij")   # planes z in [patch)
    return (gz * n * n + gy * n + gx).ravel(), (pz * n * n + py * n + px).ravel()


def run(name: str) -> str:
    make, inner, stride, patch = CASES[name]
    wl = make()
    qp = Q.from_workload(wl)
    stats = []
    t0 = time.time()
    r = ipm.solve(qp, sigma=wl.sigma, stop="kkt", kkt_tol=1e-6, max_iter=40, common_step=True,
                  newton_solve=iterative.newton_solver(inner, stats=stats))
    if not r.converged:
        raise RuntimeError(f"{name}: the oracle did not reach kkt_rel 1e-6")
    y = r.y_full(qp)
    u = qp.full(r.u())
    p = qp.full(r.state.p)
    gi, pi = sample_indices(wl.dim, wl.n, stride, patch)
    out = os.path.join(HERE, f"fullsize_{name}.npz")
    np.savez_compressed(
        out, k=len(r.history) - 1, mu=r.state.mu, kkt_rel=r.history[-1]["kkt_rel"],
        sigma=wl.sigma, grid_idx=gi, patch_idx=pi,
        y_grid=y[gi], u_grid=u[gi], p_grid=p[gi], y_patch=y[pi], u_patch=u[pi], p_patch=p[pi],
        norm_y=np.linalg.norm(y), norm_u=np.linalg.norm(u), norm_p=np.linalg.norm(p),
        krylov_iters=np.array([s.iterations for s in stats]),
        krylov_relres=np.array([s.relres for s in stats]))
    print(f"{name}: k={len(r.history) - 1} kkt_rel={r.history[-1]['kkt_rel']:.3e} "
          f"Krylov {sum(s.iterations for s in stats)} worst relres "
          f"{max(s.relres for s in stats):.1e}  {time.time() - t0:.0f} s -> {out}", flush=True)
    return out


if __name__ == "__main__":
    for nm in (sys.argv[1:] or list(CASES)):
        run(nm)
