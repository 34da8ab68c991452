"""The stored full-size expected values against what the problem fixes (CPU).

The GPU parity tests at the benchmarked sizes compare with values that the oracle's
iterative tier wrote once (``tests/golden/make_fullsize_expected.py``). These checks pin the
stored files themselves, independently of both the oracle and the GPU path:

* the sample indices are the documented coarse grid and dense patch;
* the barrier parameter is mu^k = sigma^k (mu^0 = 1, Algorithm A.1 with a fixed sigma);
* every Newton system was solved to the stated accuracy, one record per IPM step;
* y, u, p vanish on the boundary (zero Dirichlet data, interior unknowns), the control lies
  strictly inside its box and the state below its bound (interior-point iterates);
* the full vectors' norms bound the norms of any subset of their entries;
* on the dense patch (a block in 2D, three planes in 3D), the discrete state equation
  L y - M u = f (Section 2) holds at
  every node whose stencil lies inside the patch, within the primal residual that the stored
  kkt_rel allows: |(f - L y + M u)_i| <= ||xi_p||_2 <= kkt_rel (1 + ||f|| + ||M y_d||).
  That bound is rigorous but loose (the stored iterates meet it with a factor 1e-9 to
  spare). Still, it fails when the control sample is another field (p), another problem's
  control, or carries the wrong sign or a factor 2 (Poisson, by 5x to 40x), and when the
  convection-diffusion patch is transposed (its wind is not symmetric in x1 <-> x2). A
  one-node shift of a smooth field, or a transposed Poisson patch (the Q1 Laplacian and mass
  are symmetric in x1 <-> x2), is beyond what it can see.
"""
import os
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))

import make_fullsize_expected as G  # noqa: E402
from oracle import fem  # noqa: E402
from oracle import qp as Q  # noqa: E402

CASES = sorted(G.CASES)


def _load(name):
    path = os.path.join(HERE, "golden", f"fullsize_{name}.npz")
    return np.load(path, allow_pickle=False)


@pytest.mark.parametrize("name", CASES)
def test_stored_values_have_the_documented_shape_and_schedule(name):
    make, _inner, stride, patch = G.CASES[name]
    wl = make()
    d = _load(name)
    gi, pi = G.sample_indices(wl.dim, wl.n, stride, patch)
    assert np.array_equal(d["grid_idx"], gi)
    assert np.array_equal(d["patch_idx"], pi)
    for f in ("y", "u", "p"):
        assert d[f + "_grid"].shape == gi.shape and d[f + "_patch"].shape == pi.shape
        assert np.all(np.isfinite(d[f + "_grid"])) and np.all(np.isfinite(d[f + "_patch"]))
    k = int(d["k"])
    assert k >= 1
    assert float(d["sigma"]) == wl.sigma
    assert float(d["mu"]) == pytest.approx(wl.sigma ** k, rel=1e-12)
    assert float(d["kkt_rel"]) <= 1e-6
    # one Newton solve per IPM step, each to the iterative tier's acceptance level
    assert d["krylov_iters"].shape == (k,) and d["krylov_relres"].shape == (k,)
    assert np.all(d["krylov_iters"] >= 1)
    assert np.all(d["krylov_relres"] <= 1e-10)


@pytest.mark.parametrize("name", CASES)
def test_stored_values_respect_boundary_box_and_norms(name):
    make, _inner, stride, patch = G.CASES[name]
    wl = make()
    d = _load(name)
    n, dim = wl.n, wl.dim
    inner = np.zeros(n ** dim, dtype=bool)
    inner[fem.interior(dim, n)] = True
    for part in ("grid", "patch"):
        idx = d[part + "_idx"]
        on_b = ~inner[idx]
        for f in ("y", "u", "p"):
            assert np.all(d[f + "_" + part][on_b] == 0.0), (part, f)
        u = d["u_" + part][~on_b]
        y = d["y_" + part][~on_b]
        assert np.all(u > wl.ua) and np.all(u < wl.ub)
        if np.isfinite(wl.yb):
            assert np.all(y < wl.yb)
        if np.isfinite(wl.ya):
            assert np.all(y > wl.ya)
    # entries shared by the coarse grid and the patch carry the same values
    common, ig, ip = np.intersect1d(d["grid_idx"], d["patch_idx"], return_indices=True)
    for f in ("y", "u", "p"):
        assert np.array_equal(d[f + "_grid"][ig], d[f + "_patch"][ip])
    # a vector's norm bounds the norm of any subset of its entries
    for f in ("y", "u", "p"):
        nf = float(d["norm_" + f])
        assert nf > 0.0
        assert np.linalg.norm(d[f + "_grid"]) <= nf * (1 + 1e-14)
        assert np.linalg.norm(d[f + "_patch"]) <= nf * (1 + 1e-14)


@pytest.mark.parametrize("name", CASES)
def test_stored_patch_satisfies_the_state_equation(name):
    make, _inner, _stride, patch = G.CASES[name]
    wl = make()
    d = _load(name)
    qp = Q.from_workload(wl)
    n = wl.n
    nn = n ** wl.dim
    pidx = d["patch_idx"]
    y = np.zeros(nn)
    u = np.zeros(nn)
    y[pidx] = d["y_patch"]
    u[pidx] = d["u_patch"]
    known = np.zeros(nn, dtype=bool)
    known[pidx] = True
    inner = np.zeros(nn, dtype=bool)
    inner[qp.idx] = True
    # rows of interior nodes whose whole stencil (full-grid columns) is inside the patch
    A = qp.Lfull.tocsr()
    B = qp.Mfull.tocsr()
    rows = []
    for r in pidx:
        if not inner[r]:
            continue
        cols = np.union1d(A.indices[A.indptr[r]:A.indptr[r + 1]],
                          B.indices[B.indptr[r]:B.indptr[r + 1]])
        if known[cols].all():
            rows.append(r)
    rows = np.array(rows)
    # the patch's interior: (width - 2)^2 nodes in 2D, one full plane's interior in 3D
    want = (patch[1] - patch[0] - 2) ** 2 if wl.dim == 2 else \
        (patch[1] - patch[0] - 2) * (n - 2) ** 2
    assert rows.size == want
    f_full = np.zeros(nn)
    f_full[qp.idx] = qp.fvec
    resid = f_full[rows] - (A[rows] @ y - B[rows] @ u)
    bound = float(d["kkt_rel"]) * (1.0 + np.linalg.norm(qp.fvec) + np.linalg.norm(qp.cy))
    scale = abs(A[rows]) @ abs(y) + abs(B[rows]) @ abs(u)
    assert np.max(np.abs(resid)) <= bound * (1 + 1e-9) + 1e-14 * np.max(scale)
    # and the check is not vacuous: the state equation's terms are far above the bound
    assert np.max(scale) > 10.0 * bound
