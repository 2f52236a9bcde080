"""FGMRES with block stage preconditioners (oracle side).

TEST INFRASTRUCTURE: only tests, the smoke check and the CPU baseline use this.

The paper solves each step's linear system with FGMRES (Sec. 4.1: relative
residual tolerance, restart 50) preconditioned by the block preconditioners of
Sec. 3.1.  For the stage-derivative (AI) form of Sec. 3, eq. block_struct_AI the
additive splitting A = L + D + U of the Butcher matrix gives

* P_D = I (x) M + dt D (x) K        (block Jacobi, the AI form of eq. pcbjac),
* P_L = I (x) M + dt (L + D) (x) K  (block Gauss-Seidel, the AI form of eq. pcbgs),
* P_U = I (x) M + dt (U + D) (x) K  (the upper-triangular variant named in Sec. 3.1),
* P_LD = I (x) M + dt (L D) (x) K with A = L D U (the Rana-type preconditioner, eq. pcranald):
  ``BlockPreconditioner("lower", rana_ld(A), ...)``.

(The paper writes them for the IA form; the AI ones are the same preconditioners
up to a block scaling by D^{-1} or (L+D)^{-1}.)  Applying P_L^{-1} is a forward
substitution over stages; each diagonal block M + dt a_ii K is inverted
exactly or approximated (e.g. by one multigrid V-cycle).

FGMRES here is the textbook right-preconditioned flexible GMRES: Arnoldi with
classical Gram-Schmidt applied twice (CGS2), Givens rotations on the Hessenberg
matrix, and the stopping test ||r_j||_2 <= rtol ||r_0||_2 on the residual
estimate.  Vectors are stage-major (s, n) arrays flattened.
"""
from __future__ import annotations

import numpy as np


class BlockPreconditioner:
    """P_D / P_L / P_U for the system I (x) M + dt Amat (x) K.

    ``block_solves[i]`` approximates (M + dt Amat_ii K)^{-1}.
    """

    def __init__(self, kind: str, Amat: np.ndarray, K, dt: float, block_solves):
        if kind not in ("diag", "lower", "upper"):
            raise ValueError(kind)
        self.kind, self.A, self.K, self.dt, self.solves = kind, np.asarray(Amat), K, float(dt), block_solves
        self.s = self.A.shape[0]

    def __call__(self, v: np.ndarray) -> np.ndarray:
        s = self.s
        v = v.reshape(s, -1)
        z = np.zeros_like(v)
        if self.kind == "diag":
            for i in range(s):
                z[i] = self.solves[i](v[i])
            return z.reshape(-1)
        order = range(s) if self.kind == "lower" else range(s - 1, -1, -1)
        done = []
        for i in order:
            rhs = v[i].copy()
            for j in done:
                rhs -= self.dt * self.A[i, j] * (self.K @ z[j])
            z[i] = self.solves[i](rhs)
            done.append(i)
        return z.reshape(-1)


class IABlockPreconditioner:
    """Block preconditioners for the IA form (Sec. 3, eq. block_struct_IA), as the paper prints them
    (Sec. 3.1, eq. pcbjac / pcbgs / pcranald):

        P = (T^{-1} (x) M) + dt (I (x) K),   T = D (block Jacobi), L + D (block Gauss-Seidel) or L D (Rana),

    i.e. block (i, j) = (T^{-1})_ij M for j < i and diagonal blocks (1/T_ii) M + dt K.  ``block_solves[i]``
    approximates (M + dt T_ii K)^{-1}; the diagonal block inverse is T_ii times it.
    """

    def __init__(self, T: np.ndarray, M, dt: float, block_solves, diagonal_only: bool = False):
        T = np.asarray(T, dtype=np.float64)
        self.s = T.shape[0]
        self.T = np.diag(np.diag(T)) if diagonal_only else np.tril(T)
        self.Tinv = np.linalg.inv(self.T)
        self.M, self.dt, self.solves = M, float(dt), block_solves

    def __call__(self, v: np.ndarray) -> np.ndarray:
        s = self.s
        v = v.reshape(s, -1)
        z = np.zeros_like(v)
        for i in range(s):
            rhs = v[i].copy()
            for j in range(i):
                if self.Tinv[i, j] != 0.0:
                    rhs -= self.Tinv[i, j] * (self.M @ z[j])
            z[i] = self.T[i, i] * self.solves[i](rhs)
        return z.reshape(-1)


def ia_operator(M, K, A: np.ndarray, dt: float):
    """A^{-1} (x) M + dt I (x) K (Sec. 3, eq. block_struct_IA)."""
    import scipy.sparse as sp

    s = A.shape[0]
    return (sp.kron(sp.csr_matrix(np.linalg.inv(A)), M) + dt * sp.kron(sp.identity(s), K)).tocsr()


def ldu(A: np.ndarray):
    """A = L D U without pivoting (L unit lower, D diagonal, U unit upper), by Gaussian elimination."""
    A = np.asarray(A, dtype=np.float64)
    s = A.shape[0]
    L = np.eye(s)
    W = A.copy()
    for k in range(s):
        for i in range(k + 1, s):
            L[i, k] = W[i, k] / W[k, k]
            W[i, :] -= L[i, k] * W[k, :]
    D = np.diag(np.diag(W))
    U = np.linalg.solve(D, W)
    return L, D, U


def rana_ld(A: np.ndarray) -> np.ndarray:
    """The triangular approximation A_LD = L D of the Rana-type preconditioner (Sec. 3.1, eq. pcranald)."""
    L, D, _ = ldu(A)
    return L @ D


def fgmres(apply_A, b: np.ndarray, precond, rtol: float = 1e-10, restart: int = 50, maxit: int = 500, x0=None,
           info: dict | None = None):
    """Right-preconditioned flexible GMRES(restart).

    Returns (x, its, rel_res_estimate, history) where its counts preconditioner
    applications (Arnoldi steps) over all restart cycles.  If ``info`` is a dict
    it receives ``orth_loss`` = max |V^T V - I| over the restart cycles.
    """
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64).reshape(-1)
    r = b - apply_A(x) if x0 is not None else b.copy()
    r0 = np.linalg.norm(r)
    hist = [1.0]
    if r0 == 0.0:
        return x, 0, 0.0, hist
    its = 0
    rel = 1.0
    while its < maxit:
        beta = np.linalg.norm(r)
        m = restart
        V = np.zeros((m + 1, b.size))
        Z = np.zeros((m, b.size))
        H = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        j_done = 0
        for j in range(m):
            Z[j] = precond(V[j])
            w = apply_A(Z[j])
            h = V[: j + 1] @ w
            w = w - V[: j + 1].T @ h
            h2 = V[: j + 1] @ w
            w = w - V[: j + 1].T @ h2
            h = h + h2
            hn = np.linalg.norm(w)
            H[: j + 1, j] = h
            H[j + 1, j] = hn
            if hn > 0.0:
                V[j + 1] = w / hn
            for i in range(j):  # apply earlier rotations
                a, c = H[i, j], H[i + 1, j]
                H[i, j] = cs[i] * a + sn[i] * c
                H[i + 1, j] = -sn[i] * a + cs[i] * c
            a, c = H[j, j], H[j + 1, j]
            rho = np.hypot(a, c)
            cs[j], sn[j] = (1.0, 0.0) if rho == 0.0 else (a / rho, c / rho)
            H[j, j] = rho
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            j_done = j + 1
            rel = abs(g[j + 1]) / r0
            hist.append(rel)
            if rel <= rtol or hn == 0.0 or its >= maxit:
                break
        if info is not None:
            Vk = V[: j_done + 1] if hn > 0.0 else V[:j_done]
            loss = np.abs(Vk @ Vk.T - np.eye(Vk.shape[0])).max()
            info["orth_loss"] = max(info.get("orth_loss", 0.0), loss)
        y = np.linalg.solve(np.triu(H[:j_done, :j_done]), g[:j_done])
        x = x + Z[:j_done].T @ y
        if rel <= rtol or its >= maxit:
            break
        r = b - apply_A(x)
    return x, its, rel, hist
