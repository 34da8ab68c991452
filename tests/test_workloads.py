"""The seeded input generators are deterministic and shaped like the paper's experiments."""
import numpy as np

import workloads as W


def test_gaussian_sum_seeded():
    a = W.yd_gaussian_sum(65, 3)
    b = W.yd_gaussian_sum(65, 3)
    c = W.yd_gaussian_sum(65, 4)
    assert a.shape == (65, 65) and np.array_equal(a, b) and not np.array_equal(a, c)
    assert np.abs(a).max() <= 8.0


def test_sweep_and_configs():
    sw = W.poisson_2d_sweep()
    assert len(sw) == 9 and sw[0] == (1e-2, 1e-2, 0)
    wl = W.workload_c2(n=33, cell=4)
    assert wl.yb == 0.1 and wl.ua == -30 and (wl.alpha, wl.beta) == (1e-4, 1e-3)
    assert W.workload_c3(n=9).yd.shape == (9, 9, 9)
    assert W.workload_c4(n=17).kind == "cd"


def test_serving_stream_mix():
    reqs = W.serving_stream(200, seed=0, with_fields=False)
    assert len(reqs) == 200
    assert all(r["kind"] == "poisson" for r in reqs if r["dim"] == 3)
    cd = sum(r["kind"] == "cd" for r in reqs if r["dim"] == 2)
    assert 0.15 < cd / sum(r["dim"] == 2 for r in reqs) < 0.45
    assert all(1e-6 <= r["alpha"] <= 1e-2 and 1e-5 <= r["beta"] <= 1e-2 for r in reqs)
    assert W.serving_stream(5, seed=0, with_fields=False)[3]["alpha"] == reqs[3]["alpha"]
