"""Helpers shared by the GPU tests: device copies, embedding, error measures."""
import numpy as np


def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        import pytest
        pytest.skip("no CUDA device")
    return torch


def dev(a):
    torch = torch_cuda()
    return torch.as_tensor(np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1))).cuda()


def host(t):
    return t.detach().cpu().numpy()


def embed(qp, x_int):
    """Interior vector -> full-grid nodal array (zero boundary)."""
    out = np.zeros(qp.n ** qp.dim)
    out[qp.idx] = x_int
    return out


def embed4(qp, x4):
    n = qp.nI
    return np.concatenate([embed(qp, x4[b * n:(b + 1) * n]) for b in range(4)])


def interior4(qp, full4):
    m = qp.n ** qp.dim
    return np.concatenate([full4[b * m:(b + 1) * m][qp.idx] for b in range(4)])


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def iterate_arrays(qp, state):
    """The 10 nodal arrays (y, w, v, p, six multipliers) of an oracle iterate."""
    return [embed(qp, a) for a in (state.y, state.w, state.v, state.p, state.lya, state.lyb,
                                   state.lwa, state.lwb, state.lva, state.lvb)]
