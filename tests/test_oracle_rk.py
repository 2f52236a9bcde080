"""Pins for the oracle's RK step (Sec. 2 eq. stageeq / rkheat, Sec. 3 eq. block_struct_AI)."""
import numpy as np
import pytest

import workloads as W
from oracle import fem, rk
from oracle import manufactured as mf
from oracle import tableaux as T


def small_problem(N=6, seed=0, dim=2):
    kap = W.lognormal_kappa(dim, N, 0.5, seed)
    return fem.Discretisation(dim, N, kap)


@pytest.mark.parametrize("tab", [T.radau_iia(3), T.gauss_legendre(2), T.alexander(), T.lobatto_iiic2()])
def test_stage_equations_hold(tab):
    """Each stage satisfies M k_i + K (u_n + dt sum_j a_ij k_j) = F_i (eq. rkheat) to roundoff."""
    d = small_problem()
    rng = np.random.default_rng(1)
    u = rng.standard_normal(d.n)
    F = rng.standard_normal((tab.s, d.n))
    dt = 0.05
    solver = rk.KroneckerSolver(d.M, d.K, tab.A, dt)
    _, k = rk.step(solver, d.K, tab.b, dt, u, F)
    for i in range(tab.s):
        res = d.M @ k[i] + d.K @ (u + dt * sum(tab.A[i, j] * k[j] for j in range(tab.s))) - F[i]
        assert np.abs(res).max() < 1e-12 * (1 + np.abs(F).max())


def test_eigen_solver_agrees_with_kronecker_lu():
    d = small_problem(N=8)
    tab = T.radau_iia(3)
    rng = np.random.default_rng(2)
    r = rng.standard_normal((3, d.n))
    k1 = rk.KroneckerSolver(d.M, d.K, tab.A, 0.1).solve(r)
    k2 = rk.EigenSolver(d.M, d.K, tab.A, 0.1).solve(r)
    assert np.abs(k1 - k2).max() < 1e-11 * np.abs(k1).max()


@pytest.mark.parametrize("tab", [T.radau_iia(3), T.gauss_legendre(4), T.radau_iia(2)])
def test_eigen_solver_transposed_solve(tab):
    """S^T k = r from the reused block factors: the residual against the assembled transpose."""
    d = small_problem(N=9)
    rng = np.random.default_rng(7)
    r = rng.standard_normal((tab.s, d.n))
    k = rk.EigenSolver(d.M, d.K, tab.A, 0.07).solve(r, trans=True)
    St = rk.kronecker_operator(d.M, d.K, tab.A, 0.07).T
    assert np.linalg.norm(St @ k.reshape(-1) - r.reshape(-1)) < 1e-12 * np.linalg.norm(r)
    kn = rk.EigenSolver(d.M, d.K, tab.A, 0.07).solve(r)
    assert np.linalg.norm(kn - k) > 1e-3 * np.linalg.norm(k)  # A is not symmetric: the two differ


def test_dense_brute_force():
    """Tiny grid: the sparse LU solve equals a dense solve of the same block system."""
    d = small_problem(N=4)
    tab = T.radau_iia(2)
    dt = 0.3
    Md, Kd = d.M.toarray(), d.K.toarray()
    n = d.n
    big = np.zeros((2 * n, 2 * n))
    for i in range(2):
        for j in range(2):
            big[i * n:(i + 1) * n, j * n:(j + 1) * n] = (i == j) * Md + dt * tab.A[i, j] * Kd
    r = np.random.default_rng(3).standard_normal(2 * n)
    k = rk.KroneckerSolver(d.M, d.K, tab.A, dt).solve(r.reshape(2, n)).reshape(-1)
    assert np.abs(k - np.linalg.solve(big, r)).max() < 1e-13


def test_backward_euler_reduction():
    """RadauIIA(1): (M + dt K) u_{n+1} = M u_n + dt F(t_{n+1}) (textbook backward Euler)."""
    d = small_problem(N=7)
    tab = T.radau_iia(1)
    rng = np.random.default_rng(4)
    u, F = rng.standard_normal(d.n), rng.standard_normal(d.n)
    dt = 0.2
    u1, _ = rk.step(rk.KroneckerSolver(d.M, d.K, tab.A, dt), d.K, tab.b, dt, u, F[None, :])
    res = (d.M + dt * d.K) @ u1 - d.M @ u - dt * F
    assert np.abs(res).max() < 1e-14 * 10


@pytest.mark.parametrize("dim,N,tab", [(2, 32, T.radau_iia(2)), (2, 16, T.gauss_legendre(2)), (3, 6, T.radau_iia(3))])
def test_eigenmode_matches_scalar_recursion(dim, N, tab):
    """Full system from u0 = S with the manufactured load stays a(t_n) S, a from the scalar RK recursion."""
    d = fem.Discretisation(dim, N)
    S = d.to_interior(W.sine_initial(dim, N))
    Fs = d.to_interior(W.sine_load_space(dim, N))
    dt = 1 / 32
    steps = 10
    uN, _ = rk.run(d, tab, dt, steps, S, lambda t: W.sine_load_time(dim, t) * Fs)
    a = mf.scalar_rk_amplitudes(dim, N, tab.A, tab.b, tab.c, dt, steps)
    assert np.abs(uN - a[-1] * S).max() < 1e-13


@pytest.mark.parametrize("tab,q", [(T.radau_iia(2), 2), (T.radau_iia(3), 3), (T.gauss_legendre(2), 2), (T.alexander(), 1)])
def test_polynomial_exactness(tab, q):
    """u(t) = sum_k t^k U_k with F = M u' + K u: exact for degree <= q (stage order), not for q+1."""
    d = small_problem(N=5, seed=2)
    rng = np.random.default_rng(5)
    dt, steps = 0.1, 3
    for deg, exact in ((q, True), (q + 1, False)):
        U = rng.standard_normal((deg + 1, d.n))
        u_of = lambda t: sum(t**k * U[k] for k in range(deg + 1))  # noqa: E731
        du_of = lambda t: sum(k * t ** (k - 1) * U[k] for k in range(1, deg + 1))  # noqa: E731
        load = lambda t: d.M @ du_of(t) + d.K @ u_of(t)  # noqa: E731
        uN, _ = rk.run(d, tab, dt, steps, u_of(0.0), load)
        err = np.abs(uN - u_of(dt * steps)).max() / np.abs(u_of(dt * steps)).max()
        if exact:
            assert err < 1e-12
        else:
            assert err > 1e-9


@pytest.mark.parametrize("tab,p", [(T.radau_iia(1), 1), (T.radau_iia(2), 3), (T.radau_iia(3), 5),
                                   (T.gauss_legendre(1), 2), (T.gauss_legendre(2), 4), (T.alexander(), 3)])
def test_convergence_order_eigenmode(tab, p):
    """Observed order against the exact semidiscrete amplitude: 2s-1 (RadauIIA), 2s (GL)."""
    dim, N, Tend = 2, 8, 1.0
    errs, dts = [], []
    for k in range(3, 8):
        dt = Tend / 2**k
        a = mf.scalar_rk_amplitudes(dim, N, tab.A, tab.b, tab.c, dt, 2**k)
        errs.append(abs(a[-1] - mf.exact_amplitude(dim, N, Tend)))
        dts.append(dt)
    errs, dts = np.array(errs), np.array(dts)
    use = errs > 1e-13
    slope = np.polyfit(np.log(dts[use][-3:]), np.log(errs[use][-3:]), 1)[0]
    assert abs(slope - p) < 0.25, slope


def _full_problem(dim, N, seed=0):
    kap = W.lognormal_kappa(dim, N, 0.5, seed)
    Mf, Kf = fem.assemble(dim, N, kap)
    I = fem.interior_index(dim, N)
    B = np.setdiff1d(np.arange(Mf.shape[0]), I)
    return Mf, Kf, I, B


@pytest.mark.parametrize("tab,q", [(T.radau_iia(2), 2), (T.radau_iia(3), 3), (T.gauss_legendre(2), 2),
                                   (T.alexander(), 1)])
def test_dae_dirichlet_keeps_stage_order(tab, q):
    """Sec. 2.1: DAE-type boundary conditions retain the stage order.  u(t) = sum_k t^k U_k with
    nonzero boundary values, g = u on the boundary, F = M u' + K u: exact for degree <= q, not q + 1."""
    Mf, Kf, I, B = _full_problem(2, 5, seed=3)
    rng = np.random.default_rng(6)
    dt, steps = 0.1, 3
    for deg, exact in ((q, True), (q + 1, False)):
        U = rng.standard_normal((deg + 1, Mf.shape[0]))
        u_of = lambda t: sum(t**k * U[k] for k in range(deg + 1))  # noqa: E731
        du_of = lambda t: sum(k * t ** (k - 1) * U[k] for k in range(1, deg + 1))  # noqa: E731
        u = u_of(0.0)
        for n in range(steps):
            ts = [(n + c) * dt for c in tab.c]
            F = np.stack([Mf @ du_of(t) + Kf @ u_of(t) for t in ts])
            g = np.stack([u_of(t) for t in ts])
            u, _ = rk.step_dirichlet(Mf, Kf, I, B, tab.A, tab.b, dt, u, F, g)
        err = np.abs(u - u_of(steps * dt)).max() / np.abs(u_of(steps * dt)).max()
        assert (err < 1e-12) if exact else (err > 1e-9), (deg, err)


def test_dae_dirichlet_stiffly_accurate_boundary_and_homogeneous_limit():
    """RadauIIA is stiffly accurate: u_{n+1} = g(t_{n+1}) on the boundary (Sec. 2.1); with g = 0 the
    step equals the homogeneous one."""
    tab = T.radau_iia(3)
    Mf, Kf, I, B = _full_problem(2, 6, seed=4)
    rng = np.random.default_rng(7)
    dt = 0.05
    u = rng.standard_normal(Mf.shape[0])
    F = rng.standard_normal((3, Mf.shape[0]))
    g = rng.standard_normal((3, Mf.shape[0]))
    u1, k = rk.step_dirichlet(Mf, Kf, I, B, tab.A, tab.b, dt, u, F, g)
    assert np.abs(u1[B] - g[-1, B]).max() < 1e-13
    u[B] = 0.0
    u1, k = rk.step_dirichlet(Mf, Kf, I, B, tab.A, tab.b, dt, u, F, np.zeros_like(g))
    M, K = Mf[I][:, I].tocsr(), Kf[I][:, I].tocsr()
    u1h, kh = rk.step(rk.KroneckerSolver(M, K, tab.A, dt), K, tab.b, dt, u[I], F[:, I])
    assert np.abs(u1[I] - u1h).max() < 1e-13 and np.abs(u1[B]).max() == 0.0


def test_dae_dirichlet_incompatible_data_relaxes():
    """The setting of Sec. 2.1's example in 2D: u0 = 0 inside, g = 1 on the boundary, f = 0.  With
    DAE-type conditions the discrete solution relaxes to the constant 1 (which Q1 represents exactly)."""
    tab = T.lobatto_iiic2()
    N = 10
    Mf, Kf = fem.assemble(2, N)
    I = fem.interior_index(2, N)
    B = np.setdiff1d(np.arange(Mf.shape[0]), I)
    u = np.zeros(Mf.shape[0])
    u[B] = 1.0
    g = np.ones((2, Mf.shape[0]))
    F = np.zeros((2, Mf.shape[0]))
    errs = []
    for n in range(40):
        u, _ = rk.step_dirichlet(Mf, Kf, I, B, tab.A, tab.b, 0.05, u, F, g)
        errs.append(np.abs(u - 1.0).max())
    assert errs[-1] < 1e-3 and all(b <= a + 1e-15 for a, b in zip(errs, errs[1:]))
