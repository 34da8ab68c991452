"""Q1 finite-element matrices on the uniform grid of the unit square / cube.

Section 2 of the paper: L is the Galerkin discretisation of the elliptic
operator (stiffness matrix for Poisson; convection-diffusion with SUPG
upwinding in Section 5.2), M the Gram (mass) matrix of the Q1 basis, and D the
lumped mass matrix diag(int phi_i) used for the nodal-quadrature L1 term.
D_M = diag(M) is the Jacobi diagonal of the mass matrix used in Section 4.1.

Assembly follows the definition: a loop over elements computing
  K_e[a,b] = int_e grad phi_b . grad phi_a,   M_e[a,b] = int_e phi_b phi_a
by tensor Gauss quadrature (exact for these polynomial integrands), summed
into full-grid sparse matrices. Rows/columns are full-grid node indices in
C-order (x fastest); ``interior`` gives the indices of the unknowns (all
nodes off the Dirichlet boundary).

Convection-diffusion (Section 5.2): L = eps*K + N + S with
  N_e[a,b] = int_e (w . grad phi_b) phi_a,
  S_e[a,b] = delta_e int_e (w . grad phi_b)(w . grad phi_a),
delta_e = h_e/(2|w_e|) (1 - 1/Pe_e) when the element Peclet number
Pe_e = |w_e| h_e / (2 eps) exceeds one, else zero; w_e is the wind at the
element centre and h_e the element length along w_e. The paper only says
"SUPG as implemented in IFISS"; this textbook form is our reading.
"""
from __future__ import annotations

import itertools
import math

import numpy as np
import scipy.sparse as sp


def gauss01(npts: int):
    """Gauss-Legendre points and weights on [0, 1]."""
    t, w = np.polynomial.legendre.leggauss(npts)
    return 0.5 * (t + 1.0), 0.5 * w


def local_nodes(dim: int):
    """Local node offsets of a Q1 element, local index = sum offset_k 2^k (x first)."""
    return [tuple((l >> k) & 1 for k in range(dim)) for l in range(2 ** dim)]


def shape_1d(t):
    """1D linear shape functions and derivatives on [0,1] at points t."""
    return (np.stack([1.0 - t, t]), np.stack([-np.ones_like(t), np.ones_like(t)]))


def q1_basis(dim: int, pts_1d):
    """Values and reference gradients of the 2^dim bilinear/trilinear basis at tensor points.

    Returns (phi[a, q], dphi[a, k, q], weights[q], coords[k, q]) on the unit reference cell.
    """
    t, w = pts_1d
    N, dN = shape_1d(t)
    nq1 = len(t)
    qidx = list(itertools.product(range(nq1), repeat=dim))  # (qx, qy[, qz])
    nq = len(qidx)
    phi = np.zeros((2 ** dim, nq))
    dphi = np.zeros((2 ** dim, dim, nq))
    wq = np.zeros(nq)
    xq = np.zeros((dim, nq))
    for qi, q in enumerate(qidx):
        wq[qi] = np.prod([w[q[k]] for k in range(dim)])
        for k in range(dim):
            xq[k, qi] = t[q[k]]
        for a, off in enumerate(local_nodes(dim)):
            phi[a, qi] = np.prod([N[off[k], q[k]] for k in range(dim)])
            for k in range(dim):
                dphi[a, k, qi] = np.prod([(dN if kk == k else N)[off[kk], q[kk]]
                                          for kk in range(dim)])
    return phi, dphi, wq, xq


def element_connectivity(dim: int, n: int) -> np.ndarray:
    """Global node indices (n_elem, 2^dim) of every element, elements in C-order."""
    ne = n - 1
    if dim == 2:
        ey, ex = np.meshgrid(np.arange(ne), np.arange(ne), indexing="ij")
        base = (ey * n + ex).ravel()
        offs = [oy * n + ox for (ox, oy) in local_nodes(2)]
    else:
        ez, ey, ex = np.meshgrid(np.arange(ne), np.arange(ne), np.arange(ne), indexing="ij")
        base = (ez * n * n + ey * n + ex).ravel()
        offs = [oz * n * n + oy * n + ox for (ox, oy, oz) in local_nodes(3)]
    return base[:, None] + np.array(offs)[None, :]


def element_origins(dim: int, n: int) -> np.ndarray:
    """Lower-left(-front) corner coordinates (n_elem, dim) of every element."""
    h = 1.0 / (n - 1)
    ne = n - 1
    if dim == 2:
        ey, ex = np.meshgrid(np.arange(ne), np.arange(ne), indexing="ij")
        return np.stack([ex.ravel() * h, ey.ravel() * h], axis=1)
    ez, ey, ex = np.meshgrid(np.arange(ne), np.arange(ne), np.arange(ne), indexing="ij")
    return np.stack([ex.ravel() * h, ey.ravel() * h, ez.ravel() * h], axis=1)


def _scatter(conn: np.ndarray, local: np.ndarray, nn: int) -> sp.csr_matrix:
    """Sum element matrices local[e, a, b] into an (nn x nn) sparse matrix."""
    nl = conn.shape[1]
    rows = np.repeat(conn, nl, axis=1).ravel()
    cols = np.tile(conn, (1, nl)).ravel()
    return sp.coo_matrix((local.reshape(-1), (rows, cols)), shape=(nn, nn)).tocsr()


def poisson_matrices(dim: int, n: int):
    """Full-grid Q1 stiffness K and mass M (element quadrature, 2 Gauss points per direction)."""
    h = 1.0 / (n - 1)
    phi, dphi, wq, _ = q1_basis(dim, gauss01(2))
    # K_e = int grad phi_b . grad phi_a dx = h^(dim-2) * sum_q w_q dphi_ref . dphi_ref
    Ke = np.einsum("q,akq,bkq->ab", wq, dphi, dphi) * h ** (dim - 2)
    Me = np.einsum("q,aq,bq->ab", wq, phi, phi) * h ** dim
    conn = element_connectivity(dim, n)
    ne = conn.shape[0]
    nn = n ** dim
    K = _scatter(conn, np.broadcast_to(Ke, (ne,) + Ke.shape), nn)
    M = _scatter(conn, np.broadcast_to(Me, (ne,) + Me.shape), nn)
    return K, M


def mass_subdomain(dim: int, n: int, inside) -> sp.csr_matrix:
    """Full-grid Q1 mass over the elements whose centre satisfies ``inside(centres)``
    (centres: (n_elem, dim) array -> boolean mask), the observation mass of the
    partial-observation problem."""
    h = 1.0 / (n - 1)
    phi, _, wq, _ = q1_basis(dim, gauss01(2))
    Me = np.einsum("q,aq,bq->ab", wq, phi, phi) * h ** dim
    conn = element_connectivity(dim, n)
    mask = np.asarray(inside(element_origins(dim, n) + 0.5 * h), dtype=bool)
    local = np.broadcast_to(Me, (conn.shape[0],) + Me.shape) * mask[:, None, None]
    return _scatter(conn, local, n ** dim)


def paper_wind(x, y):
    """Recirculating wind of Section 5.2: w = (2 x2 (1 - x1^2), -2 x1 (1 - x2^2))."""
    return 2.0 * y * (1.0 - x * x), -2.0 * x * (1.0 - y * y)


def supg_delta(wx, wy, h, eps):
    """Element SUPG parameter from the centre wind (textbook Brooks-Hughes form)."""
    wn = np.hypot(wx, wy)
    safe = np.where(wn > 0.0, wn, 1.0)
    wmax = np.maximum(np.abs(wx), np.abs(wy))
    # length of the square element along the unit flow direction (c, s): h / max(|c|, |s|)
    he = np.where(wn > 0.0, h * wn / np.where(wmax > 0.0, wmax, 1.0), h)
    pe = wn * he / (2.0 * eps)
    delta = np.where(pe > 1.0, he / (2.0 * safe) * (1.0 - 1.0 / np.where(pe > 1.0, pe, 1.0)), 0.0)
    return delta


def convdiff_matrices(n: int, eps: float, wind=paper_wind, supg: bool = True):
    """Full-grid L = eps*K + N (+ S_SUPG) and M for the 2D convection-diffusion problem.

    Quadrature: 3 Gauss points per direction, exact for the polynomial wind of
    the paper. Returns (L, M, delta_per_element).
    """
    h = 1.0 / (n - 1)
    phi, dphi, wq, xq = q1_basis(2, gauss01(3))
    K, M = poisson_matrices(2, n)
    org = element_origins(2, n)
    # physical quadrature points per element: (ne, nq)
    px = org[:, 0:1] + h * xq[0][None, :]
    py = org[:, 1:2] + h * xq[1][None, :]
    wx, wy = wind(px, py)
    # w . grad phi_b at quadrature points: grad = dphi_ref / h
    wgrad = (wx[:, None, :] * dphi[None, :, 0, :] + wy[:, None, :] * dphi[None, :, 1, :]) / h
    area = h * h
    Ne = np.einsum("q,ebq,aq->eab", wq, wgrad, phi) * area
    cwx, cwy = wind(org[:, 0] + 0.5 * h, org[:, 1] + 0.5 * h)
    delta = supg_delta(cwx, cwy, h, eps) if supg else np.zeros(org.shape[0])
    Se = np.einsum("q,ebq,eaq->eab", wq, wgrad, wgrad) * area * delta[:, None, None]
    conn = element_connectivity(2, n)
    NS = _scatter(conn, Ne + Se, n * n)
    L = (eps * K + NS).tocsr()
    return L, M, delta


def interior(dim: int, n: int) -> np.ndarray:
    """Full-grid indices of the interior nodes (the unknowns), x fastest."""
    r = np.arange(1, n - 1)
    if dim == 2:
        j, i = np.meshgrid(r, r, indexing="ij")
        return (j * n + i).ravel()
    k, j, i = np.meshgrid(r, r, r, indexing="ij")
    return (k * n * n + j * n + i).ravel()


def boundary_mask(dim: int, n: int) -> np.ndarray:
    m = np.ones(n ** dim, dtype=bool)
    m[interior(dim, n)] = False
    return m


def lumped(Mfull: sp.spmatrix, idx: np.ndarray) -> np.ndarray:
    """D = diag(int phi_i) = row sums of the full mass matrix (partition of unity), interior rows."""
    return np.asarray(Mfull.sum(axis=1)).ravel()[idx]


def mesh_h(n: int) -> float:
    return 1.0 / (n - 1)


def chebyshev_interval(dim: int):
    """Extreme eigenvalues of D_M^{-1} M for one Q1 element (Wathen 1987): [2^-dim, (3/2)^dim]."""
    return 0.5 ** dim, 1.5 ** dim


def q1_mass_jacobi_bounds_1d_interior(n: int):
    """Exact spectrum ends of D^{-1}M for the interior 1D P1 mass matrix: 1 + cos(k pi/(n-1))/2."""
    m = n - 2
    k = np.arange(1, m + 1)
    lam = 1.0 + 0.5 * np.cos(k * math.pi / (n - 1))
    return lam.min(), lam.max()
