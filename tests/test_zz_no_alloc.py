"""The allocation-free Chebyshev entry point (GPU).

Some callers cannot let a library call cudaMalloc: applications that hand out all device
memory from their own pool, or service loops where an allocation would stall other work.
ipm_chebyshev_noalloc keeps its work vectors in a fixed device array instead. Two calls in
a row must each give the oracle's Chebyshev semi-iteration (Section 4.1) and the same result
as the allocating ipm_chebyshev_device on the same inputs, and a call after the first one
must not change the device's free memory. This file is collected last so that a run
stopping at its first failure has run every other test before.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import blocks, fem
from oracle import qp as Q
from paper_1806_05896_gb300 import ipm

from gpu_util import dev, embed, host, rel, torch_cuda

pytestmark = pytest.mark.gpu


def _inputs(dim, n):
    rng = np.random.default_rng(dim * 100 + n)
    nodes = n ** dim
    inner = np.zeros(nodes, dtype=bool)
    inner[fem.interior(dim, n)] = True
    h = 1.0 / (n - 1)
    thy = np.zeros(nodes)
    b = np.zeros(nodes)
    thy[inner] = 10.0 ** rng.uniform(-8, 2, inner.sum()) * (2 * h / 3) ** dim
    b[inner] = rng.standard_normal(inner.sum())
    return thy, b, inner


def _oracle(dim, n, steps, thy, b):
    qp = Q.build(dim, n, 1e-2, 1e-3, -1.0, 1.0)
    th = thy[qp.idx]
    A = (qp.M + sp.diags(th)).tocsr()
    lmin, lmax = fem.chebyshev_interval(dim)
    return embed(qp, blocks.chebyshev(A, qp.dM + th, b[qp.idx], steps, lmin, lmax))


@pytest.mark.parametrize("dim,n,steps", [(2, 65, 20), (2, 513, 20), (3, 17, 20), (3, 65, 20),
                                         (2, 33, 1), (2, 33, 2), (3, 9, 1), (3, 9, 2)])
def test_noalloc_matches_oracle_and_allocating_entry_point(dim, n, steps):
    torch = torch_cuda()
    nodes = n ** dim
    thy, b, inner = _inputs(dim, n)
    want = _oracle(dim, n, steps, thy, b)
    s = ipm.Solver(dim, n, 1e-2, 1e-3, -1.0, 1.0)
    ref = torch.empty(nodes, dtype=torch.float64, device="cuda")
    d_thy, d_b = dev(thy), dev(b)
    s.chebyshev(steps, d_thy, d_b, ref)
    s.close()
    ref = host(ref)
    assert rel(ref, want) < 1e-12
    xs = [torch.full((nodes,), 7.0, dtype=torch.float64, device="cuda") for _ in range(2)]
    torch.cuda.synchronize()
    for i, x in enumerate(xs):
        if i == 1:
            free_before = torch.cuda.mem_get_info()[0]
        ipm.chebyshev_noalloc(dim, n, steps, d_thy, d_b, x)
        torch.cuda.synchronize()
        if i == 1:
            assert torch.cuda.mem_get_info()[0] == free_before   # nothing allocated
        got = host(x)
        assert rel(got, want) < 1e-12
        assert rel(got, ref) < 1e-13
        assert np.all(got[~inner] == 0.0)


def test_noalloc_rejects_grids_beyond_its_array():
    torch = torch_cuda()
    n = 1025
    z = torch.zeros(n * n, dtype=torch.float64, device="cuda")
    with pytest.raises(ipm.IpmError) as e:
        ipm.chebyshev_noalloc(2, n, 20, z, z, torch.zeros_like(z))
    assert e.value.code == ipm.EINVAL
