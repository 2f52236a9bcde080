"""Discrete adjoint of the RK time loop and its kappa gradient (oracle side).

TEST INFRASTRUCTURE: only tests, the smoke check and the CPU baseline use this.

The paper has no adjoint; this is the exact derivative of the discrete loop of
``oracle.rk`` (Sec. 2 eq. stageeq / rkheat, Sec. 3 eq. block_struct_AI):

    S k_n = F_n - (1 (x) K) u_n,   S = I (x) M + dt A (x) K(theta),
    u_{n+1} = u_n + dt (b^T (x) I) k_n,
    J = 1/2 (u_N - u*)^T M (u_N - u*),  kappa_c = exp(theta_c).

Reverse sweep, with lam_N = M (u_N - u*):

    S^T mu_n = dt (b (x) lam_{n+1}),      S^T = I (x) M + dt A^T (x) K,
    lam_n = lam_{n+1} - K sum_i mu_{n,i},
    dJ/dtheta_c += -kappa_c sum_i mu_{n,i}|_c^T K_e U_{n,i}|_c,
    U_{n,i} = u_n + dt sum_j a_ij k_{n,j},

where K_e is the unit-diffusivity element matrix and |_c gathers a cell's
corner values.  A complex-step derivative Im J(theta + i eps d) / eps pins it.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .fem import assemble, cell_node_ids, element_matrices, interior_index
from .rk import EigenSolver, kronecker_operator


def objective(M, u_N, u_target) -> float:
    e = u_N - u_target
    return 0.5 * float(e @ (M @ e))


class _KroneckerLU:
    """S = I (x) M + dt A (x) K factored whole; solve(r, trans) gives S^{-1} r or S^{-T} r."""

    def __init__(self, M, K, A, dt):
        self.lu = spla.splu(kronecker_operator(M, K, A, dt).tocsc())

    def solve(self, r, trans=False):
        return self.lu.solve(np.asarray(r).reshape(-1), trans="T" if trans else "N")


def direct_solver(M, K, tab, dt, direct: str):
    """The direct stage solver: the Kronecker LU, or the eigen-decoupled solve (s complex sparse LUs of
    M + dt lam_i K; exact up to rounding, for sizes where the Kronecker LU is too large)."""
    if direct == "kronecker":
        return _KroneckerLU(M, K, tab.A, dt)
    if direct == "eigen":
        return EigenSolver(M, K, tab.A, dt)
    raise ValueError(direct)


def forward(M, K, tab, dt, steps, u0, loads, solver=None):
    """loads: (steps, s, n) interior loads.  Returns (u list, k list)."""
    lu = solver or _KroneckerLU(M, K, tab.A, dt)
    us, ks = [np.array(u0)], []
    for n in range(steps):
        r = loads[n] - (K @ us[-1])[None, :]
        k = np.asarray(lu.solve(r)).reshape(tab.s, -1)
        ks.append(k)
        us.append(us[-1] + dt * (tab.b @ k))
    return us, ks


def cell_gradient_term(dim, N, kappa, mu_full, U_full):
    """-kappa_c sum_i mu_i|_c^T K_e U_i|_c per cell; mu_full, U_full: (s, nfull)."""
    ids = cell_node_ids(dim, N)
    _, Ke = element_matrices(dim, 1.0 / N)
    g = np.zeros(ids.shape[0])
    for i in range(mu_full.shape[0]):
        mc = mu_full[i][ids]  # (ncells, 2^dim)
        Uc = U_full[i][ids]
        g -= np.einsum("ca,ab,cb->c", mc, Ke, Uc)
    return kappa * g


def gradient(dim, N, kappa, tab, dt, steps, u0, loads, u_target, direct="kronecker"):
    """(J, dJ/dtheta) by the reverse sweep above, everything on interior nodes.  ``direct`` picks the
    direct stage solver ("kronecker" or "eigen", see direct_solver); both solve S and S^T exactly."""
    M, K = assemble(dim, N, kappa)
    ii = interior_index(dim, N)
    M, K = M[ii][:, ii].tocsr(), K[ii][:, ii].tocsr()
    lu = direct_solver(M, K, tab, dt, direct)
    us, ks = forward(M, K, tab, dt, steps, u0, loads, lu)
    J = objective(M, us[-1], u_target)
    nfull = (N + 1) ** dim
    lam = M @ (us[-1] - u_target)
    g = np.zeros(N**dim)
    for n in range(steps - 1, -1, -1):
        mu = np.asarray(lu.solve(dt * np.kron(tab.b, lam), trans=True)).reshape(tab.s, -1)
        U = us[n][None, :] + dt * (tab.A @ ks[n])
        mu_f = np.zeros((tab.s, nfull))
        U_f = np.zeros((tab.s, nfull))
        mu_f[:, ii] = mu
        U_f[:, ii] = U
        g += cell_gradient_term(dim, N, kappa, mu_f, U_f)
        lam = lam - K @ mu.sum(axis=0)
    return J, g, lam


def objective_complex(dim, N, theta_c, tab, dt, steps, u0, loads, u_target):
    """J evaluated in complex arithmetic (no conjugation), for the complex step."""
    kap = np.exp(theta_c)
    M, K = assemble(dim, N, kap, dtype=complex)
    ii = interior_index(dim, N)
    M, K = M[ii][:, ii].tocsr(), K[ii][:, ii].tocsr()
    S = (sp.kron(sp.identity(tab.s), M) + dt * sp.kron(sp.csr_matrix(tab.A), K)).tocsc()
    lu = spla.splu(S)
    u = np.array(u0, dtype=complex)
    for n in range(steps):
        r = loads[n] - (K @ u)[None, :]
        k = lu.solve(r.reshape(-1)).reshape(tab.s, -1)
        u = u + dt * (tab.b @ k)
    e = u - u_target
    return 0.5 * (e @ (M @ e))


def complex_step_derivative(dim, N, theta, direction, tab, dt, steps, u0, loads, u_target, eps=1e-30):
    Jc = objective_complex(dim, N, theta + 1j * eps * direction, tab, dt, steps, u0, loads, u_target)
    return float(np.imag(Jc) / eps)
