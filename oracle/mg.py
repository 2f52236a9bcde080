"""Sparse-matrix restatement of the geometric-multigrid V-cycle (oracle side).

TEST INFRASTRUCTURE: only tests, the smoke check and the CPU baseline use this.

Sec. 3.1 leaves the inversion of each diagonal block, which for the
stage-derivative (AI) form is B = M + dt a_ii K, to a standard multigrid method.
This module writes that method out with explicit sparse matrices so that the
GPU V-cycle can be compared with it application by application:

* levels l = 0 (finest, N cells per axis) .. L-1 (N / 2^(L-1) cells), nested by
  uniform refinement;
* P_l: bilinear / trilinear interpolation from the interior nodes of level l+1
  to those of level l (tensor product of the 1D rule: even fine nodes copy the
  coarse node, odd ones average their two coarse neighbours);
* restriction R = P^T and Galerkin coarse operators M_{l+1} = P^T M_l P,
  K_{l+1} = P^T K_l P, so B_{l+1} = M_{l+1} + sigma K_{l+1} for sigma = dt a_ii;
* smoother: weighted Jacobi x <- x + omega D^{-1} (b - B x), D = diag(B);
* coarsest level: sparse LU (exact solve);
* V(nu1, nu2) cycle with zero initial guess, nu1 pre- and nu2 post-sweeps;
* MonolithicVCycle: the same cycle on the whole stage system with a stage-coupled
  point-block Jacobi relaxation (Sec. 3, 'Monolithic multigrid').
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .fem import interior_index


def interp_1d(Nc: int) -> sp.csr_matrix:
    """Full-grid 1D linear interpolation, (2 Nc + 1) x (Nc + 1)."""
    Nf = 2 * Nc
    rows, cols, vals = [], [], []
    for i in range(Nf + 1):
        if i % 2 == 0:
            rows.append(i), cols.append(i // 2), vals.append(1.0)
        else:
            rows += [i, i]
            cols += [(i - 1) // 2, (i + 1) // 2]
            vals += [0.5, 0.5]
    return sp.csr_matrix((vals, (rows, cols)), shape=(Nf + 1, Nc + 1))


def prolongation(dim: int, Nc: int) -> sp.csr_matrix:
    """Interior-to-interior interpolation from Nc to 2 Nc cells per axis (x fastest)."""
    P1 = interp_1d(Nc)
    P = P1
    for _ in range(dim - 1):
        P = sp.kron(P1, P)  # slower axes on the left
    P = P.tocsr()
    fi = interior_index(dim, 2 * Nc)
    ci = interior_index(dim, Nc)
    return P[fi][:, ci].tocsr()


class Hierarchy:
    """Galerkin hierarchy of M and K on ``levels`` nested grids."""

    def __init__(self, disc, levels: int):
        N = disc.N
        if levels < 1 or N % (2 ** (levels - 1)) != 0 or N // 2 ** (levels - 1) < 2:
            raise ValueError("mesh size not divisible for the requested number of levels")
        self.dim, self.levels = disc.dim, levels
        self.M = [disc.M]
        self.K = [disc.K]
        self.P = []
        for lev in range(levels - 1):
            Nc = N // 2 ** (lev + 1)
            P = prolongation(disc.dim, Nc)
            self.P.append(P)
            self.M.append((P.T @ self.M[-1] @ P).tocsr())
            self.K.append((P.T @ self.K[-1] @ P).tocsr())

    def operator(self, lev: int, sigma: float) -> sp.csr_matrix:
        return (self.M[lev] + sigma * self.K[lev]).tocsr()


class VCycle:
    """One V(nu1, nu2) cycle with weighted Jacobi for B = M + sigma K."""

    def __init__(self, hier: Hierarchy, sigma: float, nu1: int = 2, nu2: int = 2, omega: float = 2.0 / 3.0):
        self.h, self.sigma, self.nu1, self.nu2, self.omega = hier, float(sigma), nu1, nu2, omega
        self.B = [hier.operator(l, sigma) for l in range(hier.levels)]
        self.Dinv = [1.0 / B.diagonal() for B in self.B]
        self.coarse = spla.splu(self.B[-1].tocsc())

    def smooth(self, lev: int, x: np.ndarray, b: np.ndarray, sweeps: int) -> np.ndarray:
        for _ in range(sweeps):
            x = x + self.omega * self.Dinv[lev] * (b - self.B[lev] @ x)
        return x

    def cycle(self, b: np.ndarray, lev: int = 0) -> np.ndarray:
        if lev == self.h.levels - 1:
            return self.coarse.solve(b)
        x = np.zeros_like(b)
        x = self.smooth(lev, x, b, self.nu1)
        r = b - self.B[lev] @ x
        P = self.h.P[lev]
        e = self.cycle(P.T @ r, lev + 1)
        x = x + P @ e
        return self.smooth(lev, x, b, self.nu2)

    __call__ = cycle


class ExactBlock:
    """Exact block solve (sparse LU) of B = M + sigma K."""

    def __init__(self, M, K, sigma: float):
        self.lu = spla.splu((M + sigma * K).tocsc())

    def __call__(self, b: np.ndarray) -> np.ndarray:
        return self.lu.solve(b)


class MonolithicVCycle:
    """Monolithic multigrid for the whole stage system (Sec. 3, 'Monolithic multigrid').

    One V(nu1, nu2) cycle on S_l = I (x) M_l + dt A (x) K_l over the Galerkin hierarchy.  The
    relaxation is additive Schwarz over vertex patches with all s stages of a patch coupled; for Q1
    a vertex patch holds one node, so a sweep is point-block Jacobi

        x <- x + omega D^{-1} (b - S_l x),   D = blockdiag_p (M_l[p, p] I_s + dt K_l[p, p] A).

    Transfers act stage by stage (I (x) P, I (x) P^T) and the coarsest level is solved exactly.
    Vectors are stage-major arrays of shape (s, n), the oracle's convention.
    """

    def __init__(self, hier: Hierarchy, A: np.ndarray, dt: float, nu1: int = 2, nu2: int = 2,
                 omega: float = 2.0 / 3.0):
        from .rk import kronecker_operator

        self.h, self.A, self.dt = hier, np.asarray(A, dtype=np.float64), float(dt)
        self.nu1, self.nu2, self.omega = nu1, nu2, omega
        self.s = self.A.shape[0]
        self.S = [kronecker_operator(hier.M[l], hier.K[l], self.A, self.dt).tocsr() for l in range(hier.levels)]
        eye = np.eye(self.s)
        self.Dinv = []
        for l in range(hier.levels):
            m, k = hier.M[l].diagonal(), hier.K[l].diagonal()
            blocks = m[:, None, None] * eye[None] + self.dt * k[:, None, None] * self.A[None]
            self.Dinv.append(np.linalg.inv(blocks))  # (n, s, s)
        self.coarse = spla.splu(self.S[-1].tocsc())

    def _apply_S(self, lev: int, x: np.ndarray) -> np.ndarray:
        return (self.S[lev] @ x.reshape(-1)).reshape(x.shape)

    def relax(self, lev: int, x: np.ndarray, b: np.ndarray, sweeps: int) -> np.ndarray:
        for _ in range(sweeps):
            r = b - self._apply_S(lev, x)
            x = x + self.omega * np.einsum("pij,jp->ip", self.Dinv[lev], r)
        return x

    def cycle(self, b: np.ndarray, lev: int = 0) -> np.ndarray:
        b = np.asarray(b, dtype=np.float64).reshape(self.s, -1)
        if lev == self.h.levels - 1:
            return self.coarse.solve(b.reshape(-1)).reshape(b.shape)
        x = self.relax(lev, np.zeros_like(b), b, self.nu1)
        r = b - self._apply_S(lev, x)
        P = self.h.P[lev]
        e = self.cycle((P.T @ r.T).T, lev + 1)
        x = x + (P @ e.T).T
        return self.relax(lev, x, b, self.nu2)

    def __call__(self, v: np.ndarray) -> np.ndarray:
        """Preconditioner interface of oracle.krylov.fgmres: flat stage-major vectors."""
        return self.cycle(np.asarray(v).reshape(self.s, -1)).reshape(-1)
