"""Pins of the oracle's Algorithm A.1 against independent facts (no GPU).

* brute force: the QP (pb_fe)+(boxvector) solved by coordinate descent;
* beta = 0 with an inactive box: one linear KKT solve;
* lumped mass: the pointwise relation u = P_[ua,ub](sign(p) max(|p| - beta, 0)/alpha);
* the barrier schedule mu^k = sigma^k mu^0 (mu^9 = 5.12e-7 for sigma = 0.2, as in Section 5.1);
* linear constraints: xi_p^{k+1} = (1 - alpha_P) xi_p^k (the x0.005 ratio of the
  convergence-history figure when alpha_P = alpha_0 = 0.995);
* the sparsity table of Section 5.1 (33^2 grid, box [-2, 1.5], y_d = sin sin);
* KKT certificate with state bounds (convexity makes KKT sufficient).
"""
import math
import os

import numpy as np
import pytest

import workloads as W
from oracle import brute, ipm, linear_kkt
from oracle import qp as Q


def _yd_mixed(n, amp):
    x, y = W.node_coords(2, n)
    return amp * np.sin(2 * np.pi * x) * np.sin(np.pi * y)


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("n,amp,alpha,beta", [(9, 0.2, 1e-3, 1e-3), (9, 0.3, 1e-3, 1e-3),
                                              (7, 0.3, 1e-3, 1e-3), (9, 0.05, 1e-4, 1e-4)])
def test_ipm_matches_brute_force(n, amp, alpha, beta):
    ua, ub = -2.0, 1.5
    qp = Q.build(2, n, alpha, beta, ua, ub, yd=_yd_mixed(n, amp))
    y_bf, u_bf, p_bf, _ = brute.solve(qp, np.full(qp.nI, ua), np.full(qp.nI, ub))
    cert, counts = brute.certificate(qp, u_bf, p_bf, ua, ub, 1e-14)
    assert cert < 1e-15
    assert all(c > 0 for c in counts.values()), counts   # free, zero, upper and lower all occur
    r = ipm.solve(qp, n_iter=22)                          # mu = 0.2^22 ~ 4e-16
    assert _rel(r.u(), u_bf) < 1e-7
    assert _rel(r.state.y, y_bf) < 1e-8
    assert _rel(r.state.p, p_bf) < 1e-9


@pytest.mark.parametrize("mu_rule,common", [("gap", False), ("schedule", True), ("gap", True)])
def test_ipm_variants_reach_the_same_optimum(mu_rule, common):
    """The step-length / barrier-update variants change the path, not the unique optimum."""
    ua, ub = -2.0, 1.5
    qp = Q.build(2, 9, 1e-3, 1e-3, ua, ub, yd=_yd_mixed(9, 0.3))
    _, u_bf, _, _ = brute.solve(qp, np.full(qp.nI, ua), np.full(qp.nI, ub))
    r = ipm.solve(qp, stop="kkt", kkt_tol=1e-14, max_iter=60, mu_rule=mu_rule, common_step=common)
    assert r.converged
    assert _rel(r.u(), u_bf) < 1e-7
    if common:
        assert all(h["alpha_P"] == h["alpha_D"] for h in r.history[1:])


def test_beta_zero_matches_linear_kkt():
    qp = Q.build(2, 9, 1e-2, 0.0, -50.0, 50.0, yd=W.yd_sin_product(9))
    y, u, p = linear_kkt.solve(qp)
    assert np.abs(u).max() < 10.0                          # box inactive
    r = ipm.solve(qp, n_iter=20)
    assert _rel(r.u(), u) < 1e-11
    assert _rel(r.state.y, y) < 1e-11
    assert _rel(r.state.p, p) < 1e-11


def test_lumped_pointwise_relation():
    qp = Q.build(2, 9, 1e-2, 1e-2, -2.0, 1.5, yd=_yd_mixed(9, 1.0), lump=True)
    r = ipm.solve(qp, n_iter=20)
    p, u = r.state.p, r.u()
    pred = np.clip(np.sign(p) * np.maximum(np.abs(p) - qp.beta, 0.0) / qp.alpha, -2.0, 1.5)
    assert np.abs(u - pred).max() < 1e-8
    assert np.mean(np.abs(u) < 1e-6) > 0.2                 # a sparse part exists


def test_barrier_schedule_and_primal_contraction():
    # asymmetric box: z^0 = (z_a+z_b)/2 gives u^0 != 0, hence xi_p^0 != 0
    qp = Q.build(2, 17, 1e-2, 1e-2, -2.0, 1.5, yd=W.yd_sin_product(17))
    sigma, k = SCHEDULE["sigma"], int(SCHEDULE["iterations"])
    r = ipm.solve(qp, sigma=sigma, n_iter=k)
    mus = [h["mu"] for h in r.history]
    assert np.allclose(mus, [sigma ** j for j in range(k + 1)], rtol=1e-14)
    # printed to one significant digit: 0.2^9 = 5.12e-7
    assert abs(mus[k] - SCHEDULE["mu_final"]) < 0.05 * SCHEDULE["mu_final"]
    assert r.history[0]["xi_p"] > 1e-4
    for a, b in zip(r.history[:-1], r.history[1:]):
        pred = (1.0 - b["alpha_P"]) * a["xi_p"]
        assert abs(b["xi_p"] - pred) <= 1e-9 * a["xi_p"] + 1e-15
    # the first steps are not blocked by the bounds: ratio 1 - alpha_0
    assert abs(r.history[1]["xi_p"] / r.history[0]["xi_p"] - SCHEDULE["primal_ratio"]) < 1e-9


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _golden_rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


# Section 5.1 sparsity table at h = 2^-5: (alpha, beta) -> (sparsity %, ||u||_1), the cells
# reproduced under the readings taken here
SPARSITY_TABLE = {(float(a), float(b)): (float(sp_), float(l1))
                  for a, b, sp_, l1, ok in _golden_rows("sparsity_table_h2-5.txt") if ok == "1"}
SCHEDULE = {k: float(v) for k, v in _golden_rows("barrier_schedule.txt")}


@pytest.mark.parametrize("ab", sorted(SPARSITY_TABLE))
def test_sparsity_table(ab):
    """Sparsity = share of the 33^2 nodal control values below 1e-2 (boundary nodes carry u = 0),
    at the paper's stopping rule. The (1e-2, 1e-2) cell (paper: 15%) is not reproduced: the
    certified optimum of that cell has 40% (test below). ||u||_1 is compared within a factor
    1.6 where the control is not all-zero (for all-zero controls ||u||_1 only measures the
    distance of the last iterate from the bounds)."""
    alpha, beta = ab
    n = 33
    qp = Q.build(2, n, alpha, beta, -2.0, 1.5, yd=W.yd_sin_product(n))
    r = ipm.solve(qp, sigma=0.2, stop="paper")
    assert r.converged
    u = r.u()
    zeros = np.sum(np.abs(u) < 1e-2) + (n * n - qp.nI)
    sparsity = 100.0 * zeros / (n * n)
    want_s, want_l1 = SPARSITY_TABLE[ab]
    assert abs(sparsity - want_s) <= 3.0, sparsity
    if beta < 1e-1:
        l1 = np.abs(u).sum()
        assert want_l1 / 1.6 < l1 < want_l1 * 1.6, l1


def test_sparsity_cell_1e2_1e2_by_brute_force():
    """The sparsity-table cell alpha = beta = 1e-2 at h = 2^-5 (Section 5.1; printed 15%, 7e2)
    solved by the plain definition: coordinate descent on the reduced problem, certified by
    the subgradient conditions. The IPM oracle run to mu ~ 4e-16 agrees with it, ||u||_1
    rounds to the printed 7e2, and the optimum is far sparser than 15% (about 40% of all
    nodes, about 32% of the interior nodes): no feasible reading of the statistic gives 15%
    for this unique optimum, so the printed cell is taken as a misprint."""
    n = 33
    ua, ub = -2.0, 1.5
    qp = Q.build(2, n, 1e-2, 1e-2, ua, ub, yd=W.yd_sin_product(n))
    y_bf, u_bf, p_bf, _ = brute.solve(qp, np.full(qp.nI, ua), np.full(qp.nI, ub), tol=1e-14)
    cert, counts = brute.certificate(qp, u_bf, p_bf, ua, ub, 1e-12)
    assert cert < 1e-14
    assert all(counts[k] > 0 for k in ("free", "zero", "upper")), counts
    r = ipm.solve(qp, n_iter=22)
    assert _rel(r.u(), u_bf) < 1e-7
    assert _rel(r.state.p, p_bf) < 1e-8
    l1 = np.abs(u_bf).sum()
    assert 650.0 <= l1 < 750.0                                      # "7e2"
    interior = 100.0 * np.sum(np.abs(u_bf) < 1e-2) / qp.nI
    every = 100.0 * (np.sum(np.abs(u_bf) < 1e-2) + n * n - qp.nI) / (n * n)
    assert interior > 25.0 and every > 30.0                         # not 15%


def test_state_bounds_kkt_certificate():
    """With y <= y_b active, the final iterate satisfies the QP's KKT system with
    nonnegative multipliers, which certifies optimality for this convex problem."""
    n = 17
    qp = Q.build(2, n, 1e-3, 1e-3, -20.0, 20.0, ya=-0.1, yb=0.3, yd=W.yd_sin_product(n))
    r = ipm.solve(qp, n_iter=24)
    s = r.state
    assert s.y.max() <= 0.3 and s.y.min() >= -0.1
    assert np.sum(0.3 - s.y < 1e-8) > 0                     # the upper state bound binds
    for lam in (s.lya, s.lyb, s.lwa, s.lwb, s.lva, s.lvb):
        assert lam.min() >= 0.0
    xi_p, xi_d, xi_c, prods = ipm.residuals(qp, s)
    scale = np.linalg.norm(qp.cy)
    assert np.linalg.norm(xi_p) < 1e-12 * max(scale, 1.0)
    assert np.linalg.norm(xi_d) < 1e-10 * scale
    assert prods.max() < 1e-12


def test_kkt_rel_stopping_and_natural_residual():
    wl = W.workload_c1()
    qp = Q.from_workload(wl)
    r = ipm.solve(qp, stop="kkt", kkt_tol=1e-10)
    assert r.converged and r.history[-1]["kkt_rel"] <= 1e-10
    res = ipm.natural_residual(qp, r.u(), r.state.p, wl.ua, wl.ub)
    # components held at zero by the L1 term sit at w, v ~ mu / lambda with lambda ~ h^2 beta:
    # the averaged-product criterion leaves a natural residual of order mu / (h^d beta)
    bound = 10.0 * r.state.mu / (qp.h ** 2 * qp.beta)
    assert np.abs(res).max() < bound
    # xi norms are monotone in mu on this problem; first iterate is on the central path
    assert r.history[0]["xi_c"] == 0.0


def test_invalid_bounds_rejected():
    with pytest.raises(ValueError):
        Q.build(2, 9, 1e-2, 1e-2, 0.0, 1.0)
    with pytest.raises(ValueError):
        Q.build(2, 9, 1e-2, 1e-2, -1.0, 1.0, ya=0.5, yb=0.5)
