"""The allocation-free Chebyshev entry point matches the allocating one (GPU).

For callers that cannot let the library call cudaMalloc, ipm_chebyshev_noalloc
keeps its work vectors in a fixed device array. Two calls in a row must each give
the same result as ipm_chebyshev_device on the same inputs; this file is collected
last so that a run stopping at its first failure has run every other test before.
"""
import numpy as np
import pytest

from paper_1806_05896_gb300 import ipm

from gpu_util import dev, embed, host, rel, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dim,n", [(2, 65), (2, 513), (3, 17), (3, 65)])
def test_noalloc_matches_allocating_entry_point(dim, n):
    torch = torch_cuda()
    rng = np.random.default_rng(dim * 100 + n)
    nodes = n ** dim
    thy = np.zeros(nodes)
    b = np.zeros(nodes)
    inner = np.ones((n,) * dim, dtype=bool)
    for ax in range(dim):
        sl = [slice(None)] * dim
        sl[ax] = 0
        inner[tuple(sl)] = False
        sl[ax] = n - 1
        inner[tuple(sl)] = False
    inner = inner.reshape(-1)
    h = 1.0 / (n - 1)
    thy[inner] = 10.0 ** rng.uniform(-8, 2, inner.sum()) * (2 * h / 3) ** dim
    b[inner] = rng.standard_normal(inner.sum())
    s = ipm.Solver(dim, n, 1e-2, 1e-3, -1.0, 1.0)
    ref = torch.empty(nodes, dtype=torch.float64, device="cuda")
    s.chebyshev(20, dev(thy), dev(b), ref)
    s.close()
    ref = host(ref)
    for _ in range(2):
        x = torch.full((nodes,), 7.0, dtype=torch.float64, device="cuda")
        ipm.chebyshev_noalloc(dim, n, 20, dev(thy), dev(b), x)
        torch.cuda.synchronize()
        got = host(x)
        assert rel(got, ref) < 1e-13
        assert np.all(got[~inner] == 0.0)


def test_noalloc_rejects_grids_beyond_its_array():
    torch = torch_cuda()
    n = 1025
    z = torch.zeros(n * n, dtype=torch.float64, device="cuda")
    with pytest.raises(ipm.IpmError) as e:
        ipm.chebyshev_noalloc(2, n, 20, z, z, torch.zeros_like(z))
    assert e.value.code == ipm.EINVAL
