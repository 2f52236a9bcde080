"""Q1 finite elements on uniform meshes of the unit square / cube (oracle side).

TEST INFRASTRUCTURE: only tests, the smoke check and the CPU baseline use this.

The heat equation of Sec. 2 (eq. heat) in weak form, read with the sign that
eq. rkheat uses: (u_t, v) + (kappa grad u, grad v) = (f, v).  Its
semidiscretisation with continuous Q1 elements gives M u' + K u = F with

    M_ab = int phi_a phi_b,     K_ab = int kappa grad phi_a . grad phi_b.

Element matrices are the closed-form integrals (tensor products of the 1D
linear-element mass and stiffness integrals, see element_matrices), assembled
cell by cell (one scatter per local (a, b) pair, all cells at once).  ``kappa`` is
piecewise constant per cell.  Nodes are numbered x fastest over the full
(N+1)^dim grid; cells likewise over N^dim.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp


def local_corners(dim: int) -> np.ndarray:
    """Local corner offsets, local index a = sum_d bit_d * 2^d (x fastest)."""
    return np.array([[(a >> d) & 1 for d in range(dim)] for a in range(2**dim)], dtype=np.int64)


def element_matrices(dim: int, h: float) -> tuple[np.ndarray, np.ndarray]:
    """(M_e, K_e) for one cell [0, h]^dim with kappa = 1.

    Q1 shape functions are products of the 1D hats, so the element integrals are
    tensor products of the 1D linear-element integrals

        m = int phi_a phi_b = h [[1/3, 1/6], [1/6, 1/3]],   k = int phi_a' phi_b' = (1/h) [[1, -1], [-1, 1]]:

    M_e[a, b] = prod_d m[a_d, b_d] and K_e[a, b] = sum_d k[a_d, b_d] prod_{e != d} m[a_e, b_e] (local
    index a = sum_d a_d 2^d, x fastest).  Written out this way every stiffness row sums to zero in
    floating point as it does exactly (the gradient of a constant vanishes) when h is a power of two.
    """
    m1 = h * np.array([[1.0 / 3.0, 1.0 / 6.0], [1.0 / 6.0, 1.0 / 3.0]])
    k1 = (1.0 / h) * np.array([[1.0, -1.0], [-1.0, 1.0]])
    corners = local_corners(dim)
    nloc = 2**dim
    Me = np.zeros((nloc, nloc))
    Ke = np.zeros((nloc, nloc))
    for a in range(nloc):
        for b in range(nloc):
            ca, cb = corners[a], corners[b]
            Me[a, b] = np.prod([m1[ca[d], cb[d]] for d in range(dim)])
            Ke[a, b] = sum(k1[ca[d], cb[d]] * np.prod([m1[ca[e], cb[e]] for e in range(dim) if e != d])
                           for d in range(dim))
    return Me, Ke


def cell_node_ids(dim: int, N: int) -> np.ndarray:
    """(ncells, 2^dim) global node ids of each cell's corners."""
    nn = N + 1
    cidx = np.arange(N**dim)
    cc = [(cidx // N**d) % N for d in range(dim)]  # per-axis cell coordinates
    corners = local_corners(dim)
    ids = np.zeros((N**dim, 2**dim), dtype=np.int64)
    for a in range(2**dim):
        gid = np.zeros(N**dim, dtype=np.int64)
        for d in range(dim):
            gid += (cc[d] + corners[a, d]) * nn**d
        ids[:, a] = gid
    return ids


def assemble(dim: int, N: int, kappa=None, dtype=np.float64) -> tuple[sp.csr_matrix, sp.csr_matrix]:
    """Full-grid (M, K) in CSR, assembled cell by cell.  kappa: per cell or None (= 1)."""
    h = 1.0 / N
    Me, Ke = element_matrices(dim, h)
    ids = cell_node_ids(dim, N)
    ncell = ids.shape[0]
    kap = np.ones(ncell, dtype=dtype) if kappa is None else np.asarray(kappa).astype(dtype)
    nloc = 2**dim
    rows = np.repeat(ids, nloc, axis=1).reshape(-1)
    cols = np.tile(ids, (1, nloc)).reshape(-1)
    mvals = np.broadcast_to(Me.reshape(-1), (ncell, nloc * nloc)).reshape(-1).astype(dtype)
    kvals = (kap[:, None] * Ke.reshape(1, -1)).reshape(-1)
    nn = (N + 1) ** dim
    M = sp.coo_matrix((mvals, (rows, cols)), shape=(nn, nn)).tocsr()
    K = sp.coo_matrix((kvals, (rows, cols)), shape=(nn, nn)).tocsr()
    M.sum_duplicates()
    K.sum_duplicates()
    return M, K


def interior_index(dim: int, N: int) -> np.ndarray:
    """Global ids of interior nodes (homogeneous Dirichlet eliminates the rest)."""
    idx = np.arange(N + 1)
    inner = (idx > 0) & (idx < N)
    m = np.ones([N + 1] * dim, dtype=bool)
    for d in range(dim):
        shape = [1] * dim
        shape[dim - 1 - d] = N + 1
        m &= inner.reshape(shape)
    return np.nonzero(m.reshape(-1))[0]


class Discretisation:
    """Interior-node M and K for one mesh and diffusivity field."""

    def __init__(self, dim: int, N: int, kappa=None):
        self.dim, self.N = dim, N
        self.kappa = None if kappa is None else np.asarray(kappa, dtype=np.float64)
        Mf, Kf = assemble(dim, N, self.kappa)
        self.M_full, self.K_full = Mf, Kf
        self.interior = interior_index(dim, N)
        self.nfull = (N + 1) ** dim
        ii = self.interior
        self.M = Mf[ii][:, ii].tocsr()
        self.K = Kf[ii][:, ii].tocsr()
        self.n = len(ii)

    def to_interior(self, v_full: np.ndarray, s: int = 1) -> np.ndarray:
        """Full node-major vector -> (s, n_interior) stage-major array (or (n,) if s == 1)."""
        v = np.asarray(v_full).reshape(self.nfull, s)[self.interior]
        return v[:, 0].copy() if s == 1 else v.T.copy()

    def to_full(self, v_int: np.ndarray, s: int = 1) -> np.ndarray:
        """Inverse of to_interior: zeros on the boundary, node-major interleaved."""
        out = np.zeros((self.nfull, s), dtype=np.result_type(v_int, np.float64))
        if s == 1:
            out[self.interior, 0] = v_int
        else:
            out[self.interior] = np.asarray(v_int).T
        return out.reshape(-1)

    def l2_norm(self, e_int: np.ndarray) -> float:
        """FE L2 norm of a nodal (interior) difference: sqrt(e^T M e)."""
        return float(np.sqrt(e_int @ (self.M @ e_int)))


def load_by_quadrature(dim: int, N: int, f, order: int = 5) -> np.ndarray:
    """Full-grid load vector F_j = int f phi_j with Gauss-Legendre(order)^dim per cell."""
    h = 1.0 / N
    xg, wg = np.polynomial.legendre.leggauss(order)
    xg = 0.5 * (xg + 1.0)
    wg = 0.5 * wg
    corners = local_corners(dim)
    ids = cell_node_ids(dim, N)
    ncell = ids.shape[0]
    cidx = np.arange(ncell)
    origin = np.stack([((cidx // N**d) % N) * h for d in range(dim)], axis=1)
    F = np.zeros((N + 1) ** dim)
    for q in itertools.product(range(order), repeat=dim):
        xi = np.array([xg[qi] for qi in q])
        wq = np.prod([wg[qi] for qi in q]) * h**dim
        pts = origin + h * xi[None, :]
        fv = f(*[pts[:, d] for d in range(dim)])
        for a in range(2**dim):
            phi = np.prod(np.where(corners[a] == 1, xi, 1.0 - xi))
            np.add.at(F, ids[:, a], wq * phi * fv)
    return F
