"""Serving loop: results are the same alone and in a concurrent mix; budget admission works."""
import math

import numpy as np
import pytest

import workloads as W
from paper_1806_05896_gb300 import ipm

from gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


def _mix():
    reqs = []
    for i, (dim, n, kind) in enumerate([(2, 33, "poisson"), (2, 65, "poisson"), (2, 33, "cd"),
                                        (2, 65, "cd"), (3, 9, "poisson"), (3, 17, "poisson"),
                                        (2, 129, "poisson"), (2, 65, "poisson"),
                                        (2, 257, "poisson"), (2, 257, "cd")]):
        rng = np.random.default_rng(100 + i)
        half = float(rng.uniform(1, 50))
        reqs.append(dict(dim=dim, n=n, kind=kind, eps=1.0 / 50.0,
                         alpha=float(10 ** rng.uniform(-6, -2)), beta=float(10 ** rng.uniform(-5, -2)),
                         ua=-half, ub=half, yd=W.yd_gaussian_sum(n, 100 + i, dim=dim)))
    return reqs


OPTS = dict(precision=ipm.PREC_MIXED, stop=ipm.STOP_KKT, kkt_tol=1e-6, common_step=1, max_ipm=60,
            restart=30)


def _alone(r):
    s = ipm.Solver(r["dim"], r["n"], r["alpha"], r["beta"], r["ua"], r["ub"], kind=r["kind"],
                   eps=r["eps"])
    s.set_data(r["yd"])
    rep = s.solve(**OPTS)
    u = s.control().reshape(-1)
    s.close()
    return rep, u


def test_server_results_equal_alone_and_in_mix():
    torch_cuda()
    reqs = _mix()
    alone = [_alone(r) for r in reqs]
    sv = ipm.Server(workers=4, budget_bytes=16 << 30)
    tickets = [sv.submit(r["dim"], r["n"], r["alpha"], r["beta"], r["ua"], r["ub"], r["yd"],
                         kind=r["kind"], eps=r["eps"], **OPTS) for r in reqs]
    # the same requests again, now against pooled (reset) solvers
    tickets2 = [sv.submit(r["dim"], r["n"], r["alpha"], r["beta"], r["ua"], r["ub"], r["yd"],
                          kind=r["kind"], eps=r["eps"], **OPTS) for r in reqs]
    for (rep_a, u_a), t, t2 in zip(alone, tickets, tickets2):
        rep, u, lat, q = sv.wait(t)
        rep2, u2, _, _ = sv.wait(t2)
        assert rep["status"] == ipm.OK and rep["kkt_rel"] <= 1e-6
        assert np.array_equal(u, u_a)
        assert np.array_equal(u2, u_a)
        assert rep["ipm_iters"] == rep_a["ipm_iters"]
        assert lat >= q >= 0.0
    st = sv.stats()
    assert st["completed"] == 2 * len(reqs)
    sv.close()


def test_server_respects_memory_budget():
    torch_cuda()
    reqs = _mix()[:4]
    one = ipm.Solver(2, 65, 1e-2, 1e-3, -1.0, 1.0)
    one.set_data(W.yd_sin_product(65))
    one.solve(**OPTS)  # the Krylov basis is allocated by the first solve
    budget = 3 * one.device_bytes()
    one.close()
    sv = ipm.Server(workers=3, budget_bytes=budget)
    tickets = [sv.submit(r["dim"], r["n"], r["alpha"], r["beta"], r["ua"], r["ub"], r["yd"],
                         kind=r["kind"], eps=r["eps"], **OPTS) for r in reqs]
    for t in tickets:
        rep, u, lat, q = sv.wait(t)
        assert rep["status"] == ipm.OK
    assert sv.stats()["bytes_in_use"] <= budget
    with pytest.raises(ipm.IpmError) as e:
        big = np.zeros(1025 * 1025)
        sv.submit(2, 1025, 1e-2, 1e-3, -1.0, 1.0, big, **OPTS)
    assert e.value.code == ipm.ENOMEM
    sv.close()


def test_server_many_workers_fresh_solvers_each_request():
    """16 workers, every request on a grid key of its own (convection-diffusion with its own
    eps), so solvers are created, zeroed and grown while the other workers' kernels run: each
    result equals the request solved alone, bit for bit."""
    torch_cuda()
    reqs = []
    for i in range(32):
        rng = np.random.default_rng(500 + i)
        n = (33, 65, 129)[i % 3]
        half = float(rng.uniform(1, 50))
        reqs.append(dict(dim=2, n=n, kind="cd" if i % 4 else "poisson", eps=1.0 / (20.0 + i),
                         alpha=float(10 ** rng.uniform(-6, -2)),
                         beta=float(10 ** rng.uniform(-5, -2)), ua=-half, ub=half,
                         yd=W.yd_gaussian_sum(n, 500 + i, dim=2)))
    alone = [_alone(r) for r in reqs]
    sv = ipm.Server(workers=16, budget_bytes=32 << 30)
    tickets = [sv.submit(r["dim"], r["n"], r["alpha"], r["beta"], r["ua"], r["ub"], r["yd"],
                         kind=r["kind"], eps=r["eps"], **OPTS) for r in reqs]
    for (rep_a, u_a), t in zip(alone, tickets):
        rep, u, _, _ = sv.wait(t)
        assert rep["status"] == rep_a["status"]
        assert rep["ipm_iters"] == rep_a["ipm_iters"]
        assert np.array_equal(u, u_a)
    sv.close()
