"""The stage-coupled RK solve by sparse direct factorisation (oracle side).

TEST INFRASTRUCTURE: only tests, the smoke check and the CPU baseline use this.

One step of an s-stage RK method (Sec. 2, eq. stageeq and the update above it)
applied to M u' + K u = F(t) (Sec. 2, eq. rkheat, in the generalised mass-matrix
form the paper keeps) gives the stages k_i from

    M k_i + K (u_n + dt sum_j a_ij k_j) = F(t_n + c_i dt),   i = 1..s,

i.e. the Kronecker system of Sec. 3, eq. block_struct_AI,

    (I (x) M + dt A (x) K) k = r,    r_i = F(t_n + c_i dt) - K u_n,

followed by u_{n+1} = u_n + dt sum_i b_i k_i.  (The paper's eq. rkheat writes
the update without dt; the RK definition in Sec. 2 has it, and that reading is
used.)  Homogeneous Dirichlet conditions: the DAE-type conditions of Sec. 2.1
give sum_j a_ij k_j = 0 on the boundary, hence k = 0 there for invertible A, so
boundary unknowns are eliminated.  ``step_dirichlet`` handles nonzero data g.

Stage vectors are stage-major arrays of shape (s, n) over interior nodes.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def kronecker_operator(M: sp.spmatrix, K: sp.spmatrix, A: np.ndarray, dt: float) -> sp.csc_matrix:
    """I (x) M + dt A (x) K as one sparse matrix (stage-major blocks)."""
    s = A.shape[0]
    return (sp.kron(sp.identity(s), M) + dt * sp.kron(sp.csr_matrix(A), K)).tocsc()


class KroneckerSolver:
    """Factor I (x) M + dt A (x) K once with SuperLU and reuse it every step."""

    def __init__(self, M, K, A, dt):
        self.M, self.K, self.A, self.dt = M, K, np.asarray(A, dtype=np.float64), float(dt)
        self.s, self.n = self.A.shape[0], M.shape[0]
        self.S = kronecker_operator(M, K, self.A, self.dt)
        self.lu = spla.splu(self.S)

    def solve(self, r: np.ndarray, trans: bool = False) -> np.ndarray:
        """k = S^{-1} r (or S^{-T} r); r of shape (s, n)."""
        x = self.lu.solve(np.asarray(r).reshape(-1), trans="T" if trans else "N")
        return x.reshape(self.s, self.n)

    def apply(self, k: np.ndarray, trans: bool = False) -> np.ndarray:
        S = self.S.T if trans else self.S
        return (S @ np.asarray(k).reshape(-1)).reshape(self.s, self.n)


class EigenSolver:
    """Direct solve of the same system through the eigen-decomposition A = V diag(lam) V^{-1}.

    With k = (V (x) I) w the system splits into s independent complex solves
    (M + dt lam_i K) w_i = [(V^{-1} (x) I) r]_i, each by sparse LU.  Used where the
    Kronecker LU is too large; it is still a direct method.
    """

    def __init__(self, M, K, A, dt):
        self.A = np.asarray(A, dtype=np.float64)
        self.s, self.n = self.A.shape[0], M.shape[0]
        lam, V = np.linalg.eig(self.A)
        self.V, self.Vinv = V.astype(complex), np.linalg.inv(V).astype(complex)
        Mc, Kc = M.astype(complex), K.astype(complex)
        # M, K are real, so M + dt conj(lam) K is the complex conjugate of M + dt lam K: the second member
        # of a conjugate pair is solved with the first one's factor, x = conj(B^{-1} conj(r))
        self.lus, self.conj_of = [], []
        for i in range(self.s):
            j = next((j for j in range(i) if self.conj_of[j] < 0 and abs(lam[j].imag) > 0
                      and abs(lam[i] - np.conj(lam[j])) <= 1e-12 * abs(lam[j])), -1)
            self.conj_of.append(j)
            self.lus.append(None if j >= 0 else spla.splu((Mc + dt * lam[i] * Kc).tocsc()))

    def _block_solve(self, i, r):
        j = self.conj_of[i]
        return np.conj(self.lus[j].solve(np.conj(r))) if j >= 0 else self.lus[i].solve(r)

    def solve(self, r: np.ndarray, trans: bool = False) -> np.ndarray:
        """k = S^{-1} r, or S^{-T} r: S^T = I (x) M + dt A^T (x) K = (V^{-T} (x) I) D (V^T (x) I) with the
        same block-diagonal D (its blocks M + dt lam_i K are complex symmetric), so the factors are reused."""
        r = np.asarray(r, dtype=complex).reshape(self.s, self.n)
        left, right = (self.Vinv.T, self.V.T) if trans else (self.V, self.Vinv)
        rt = right @ r
        w = np.stack([self._block_solve(i, rt[i]) for i in range(self.s)])
        return np.real(left @ w)


def step(solver, K, b: np.ndarray, dt: float, u_n: np.ndarray, F_stages: np.ndarray):
    """One RK step.  F_stages: (s, n) loads at t_n + c_i dt.  Returns (u_{n+1}, k)."""
    r = F_stages - (K @ u_n)[None, :]
    k = solver.solve(r)
    u_next = u_n + dt * (np.asarray(b) @ k)
    return u_next, k


def run(disc, tab, dt: float, steps: int, u0_int: np.ndarray, load_fn, t0: float = 0.0, solver=None):
    """Integrate ``steps`` steps from u0 (interior).  load_fn(t) -> (n,) interior load.

    Returns (u_N, list of per-step stage arrays).
    """
    solver = solver or KroneckerSolver(disc.M, disc.K, tab.A, dt)
    u = np.array(u0_int, dtype=np.float64)
    stages = []
    t = t0
    for _ in range(steps):
        F = np.stack([load_fn(t + ci * dt) for ci in tab.c])
        u, k = step(solver, disc.K, tab.b, dt, u, F)
        stages.append(k)
        t += dt
    return u, stages


def step_dirichlet(M_full, K_full, interior, boundary, A, b, dt, u_full, F_full, g_full):
    """One RK step with DAE-type Dirichlet conditions (Sec. 2.1) on the full node set.

    On the boundary the stage values u_n + dt sum_j a_ij k_j must equal g(t_n + c_i dt), so
    k_B = A^{-1} (g_B - u_n,B) / dt (node by node).  The interior rows of the stage equations
    M k_i + K (u_n + dt sum_j a_ij k_j) = F_i then determine k_I with k_B known.
    F_full, g_full: (s, nfull) loads and boundary data at the stage times.  Returns (u_{n+1}, k) full.
    """
    A = np.asarray(A, dtype=np.float64)
    s = A.shape[0]
    I, B = interior, boundary
    kB = np.linalg.solve(A, (g_full[:, B] - u_full[None, B])) / dt  # (s, nB)
    M_II, K_II = M_full[I][:, I].tocsr(), K_full[I][:, I].tocsr()
    M_IB, K_IB = M_full[I][:, B].tocsr(), K_full[I][:, B].tocsr()
    r = np.empty((s, len(I)))
    for i in range(s):
        coupling = M_IB @ kB[i] + dt * sum(A[i, j] * (K_IB @ kB[j]) for j in range(s))
        r[i] = F_full[i, I] - (K_full[I] @ u_full) - coupling
    kI = KroneckerSolver(M_II, K_II, A, dt).solve(r)
    k = np.zeros((s, u_full.size))
    k[:, I] = kI
    k[:, B] = kB
    return u_full + dt * (np.asarray(b) @ k), k
