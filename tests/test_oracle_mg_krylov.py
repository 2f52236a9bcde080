"""Pins for the oracle's multigrid restatement and FGMRES with block preconditioners (Sec. 3.1)."""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import fem, krylov, mg, rk
from oracle import tableaux as T


def test_interpolation_exact_for_bilinear():
    Nc = 4
    P1 = mg.interp_1d(Nc)
    P = sp.kron(P1, P1).tocsr()
    xc = W.node_coords(2, Nc)
    xf = W.node_coords(2, 2 * Nc)
    f = lambda x, y: (0.3 + 1.7 * x) * (2.0 - 0.4 * y)  # noqa: E731
    assert np.abs(P @ f(*xc) - f(*xf)).max() < 1e-14


@pytest.mark.parametrize("dim,Nc", [(2, 4), (3, 2)])
def test_galerkin_equals_coarse_assembly(dim, Nc):
    """P^T K_h P = K_2h, P^T M_h P = M_2h for kappa constant on coarse cells."""
    kc = W.lognormal_kappa(dim, Nc, 0.5, 7)
    # refine kappa: each fine cell takes its coarse parent's value
    Nf = 2 * Nc
    idx = np.arange(Nf**dim)
    parent = sum(((idx // Nf**d) % Nf // 2) * Nc**d for d in range(dim))
    kf = kc[parent]
    fine = fem.Discretisation(dim, Nf, kf)
    coarse = fem.Discretisation(dim, Nc, kc)
    P = mg.prolongation(dim, Nc)
    assert abs(P.T @ fine.K @ P - coarse.K).max() < 1e-13
    assert abs(P.T @ fine.M @ P - coarse.M).max() < 1e-16


def vcycle_setup(N=32, levels=4, sigma=0.05):
    d = fem.Discretisation(2, N, W.lognormal_kappa(2, N, 0.5, 0))
    return d, mg.VCycle(mg.Hierarchy(d, levels), sigma)


def test_vcycle_symmetric_and_convergent():
    d, V = vcycle_setup()
    rng = np.random.default_rng(0)
    u, v = rng.standard_normal(d.n), rng.standard_normal(d.n)
    assert abs(u @ V(v) - v @ V(u)) < 1e-12 * abs(u @ V(v))
    # error propagation I - V B contracts: estimate its spectral radius by power iteration
    B = V.B[0]
    e = rng.standard_normal(d.n)
    for _ in range(15):
        e = e - V(B @ e)
        nrm = np.linalg.norm(e)
        e /= nrm
    assert nrm < 0.4  # V(2,2), omega = 2/3 on the 9-point Q1 operator: about 0.27 here


def test_one_level_is_exact():
    d = fem.Discretisation(2, 8, W.lognormal_kappa(2, 8, 0.5, 1))
    V = mg.VCycle(mg.Hierarchy(d, 1), 0.3)
    b = np.random.default_rng(1).standard_normal(d.n)
    assert np.abs(V.B[0] @ V(b) - b).max() < 1e-13


def test_fgmres_dense_identity_preconditioner():
    rng = np.random.default_rng(2)
    n = 40
    A = np.eye(n) * 4 + rng.standard_normal((n, n)) * 0.3
    b = rng.standard_normal(n)
    x, its, rel, _ = krylov.fgmres(lambda v: A @ v, b, lambda v: v, rtol=1e-12, restart=50)
    assert its <= n and rel <= 1e-12
    assert np.abs(x - np.linalg.solve(A, b)).max() < 1e-10
    # exact preconditioner: one step
    Ainv = np.linalg.inv(A)
    x, its, rel, _ = krylov.fgmres(lambda v: A @ v, b, lambda v: Ainv @ v, rtol=1e-12)
    assert its == 1 and np.abs(x - np.linalg.solve(A, b)).max() < 1e-12


def test_fgmres_basis_orthonormal():
    """CGS2 keeps the Arnoldi basis orthonormal to working precision on a hard spectrum."""
    rng = np.random.default_rng(8)
    n = 80
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = Q @ np.diag(np.logspace(0, 8, n)) @ Q.T + 1e-3 * rng.standard_normal((n, n))
    b = rng.standard_normal(n)
    info = {}
    krylov.fgmres(lambda v: A @ v, b, lambda v: v, rtol=1e-14, restart=60, maxit=60, info=info)
    assert info["orth_loss"] < 1e-13


def test_fgmres_restart():
    rng = np.random.default_rng(3)
    n = 60
    A = np.diag(np.linspace(1, 30, n)) + rng.standard_normal((n, n)) * 0.1
    b = rng.standard_normal(n)
    x, its, rel, _ = krylov.fgmres(lambda v: A @ v, b, lambda v: v, rtol=1e-10, restart=7, maxit=2000)
    assert rel <= 1e-10 and its > 7
    assert np.linalg.norm(A @ x - b) <= 1.01e-10 * np.linalg.norm(b)


def kron_setup(tab, N=8, dt=0.1):
    d = fem.Discretisation(2, N, W.lognormal_kappa(2, N, 0.5, 4))
    S = rk.kronecker_operator(d.M, d.K, tab.A, dt)
    return d, S


@pytest.mark.parametrize("kind,tab", [("lower", T.alexander()), ("upper", None), ("diag", None)])
def test_block_preconditioner_exact_on_matching_structure(kind, tab):
    """P_L with exact blocks equals the system for lower-triangular A, P_U for upper, P_D for diagonal:
    FGMRES then needs exactly one iteration."""
    if kind == "upper":
        base = T.alexander()
        tab = T.Tableau("upper", base.A.T.copy(), base.b, base.c, 1, 1)
    if kind == "diag":
        tab = T.Tableau("diag", np.diag([0.3, 0.7, 1.1]), np.ones(3) / 3, np.zeros(3), 1, 1)
    dt = 0.1
    d, S = kron_setup(tab, dt=dt)
    solves = [mg.ExactBlock(d.M, d.K, dt * tab.A[i, i]) for i in range(tab.s)]
    P = krylov.BlockPreconditioner(kind, tab.A, d.K, dt, solves)
    b = np.random.default_rng(5).standard_normal(S.shape[0])
    x, its, rel, _ = krylov.fgmres(lambda v: S @ v, b, P, rtol=1e-12)
    assert its == 1
    assert np.abs(S @ x - b).max() < 1e-12 * np.abs(b).max()


def test_block_gs_beats_block_jacobi():
    """Sec. 3.1 / 4.1: P_L needs no more iterations than P_D; both grow with s (exact blocks)."""
    its = {}
    for s in (2, 3):
        tab = T.radau_iia(s)
        dt = 0.05
        d, S = kron_setup(tab, N=16, dt=dt)
        solves = [mg.ExactBlock(d.M, d.K, dt * tab.A[i, i]) for i in range(s)]
        b = np.random.default_rng(6).standard_normal(S.shape[0])
        for kind in ("diag", "lower"):
            P = krylov.BlockPreconditioner(kind, tab.A, d.K, dt, solves)
            its[(kind, s)] = krylov.fgmres(lambda v: S @ v, b, P, rtol=1e-10)[1]
    assert its[("lower", 3)] <= its[("diag", 3)]
    assert its[("diag", 3)] >= its[("diag", 2)]


def test_fgmres_vcycle_matches_direct():
    tab = T.radau_iia(3)
    dt = 1 / 64
    d = fem.Discretisation(2, 32, W.lognormal_kappa(2, 32, 0.5, 0))
    S = rk.kronecker_operator(d.M, d.K, tab.A, dt)
    h = mg.Hierarchy(d, 4)
    solves = [mg.VCycle(h, dt * tab.A[i, i]) for i in range(3)]
    b = np.random.default_rng(7).standard_normal(S.shape[0])
    xd = rk.KroneckerSolver(d.M, d.K, tab.A, dt).solve(b.reshape(3, -1)).reshape(-1)
    for kind in ("diag", "lower", "upper"):
        P = krylov.BlockPreconditioner(kind, tab.A, d.K, dt, solves)
        x, its, rel, _ = krylov.fgmres(lambda v: S @ v, b, P, rtol=1e-12)
        assert rel <= 1e-12
        assert np.linalg.norm(x - xd) <= 1e-9 * np.linalg.norm(xd)


@pytest.mark.parametrize("s", [2, 3, 4])
def test_ldu_factorisation(s):
    A = T.radau_iia(s).A
    L, D, U = krylov.ldu(A)
    assert np.allclose(L @ D @ U, A, atol=1e-15)
    assert np.allclose(np.diag(L), 1) and np.allclose(np.diag(U), 1)
    assert np.allclose(np.triu(L, 1), 0) and np.allclose(np.tril(U, -1), 0)
    # for a lower-triangular (DIRK) tableau, L D = A: the Rana preconditioner is P_L
    assert np.allclose(krylov.rana_ld(T.alexander().A), T.alexander().A, atol=1e-15)


def test_rana_ld_iterations_vs_block_gauss_seidel():
    """Sec. 3.1 / 4.1: with exact blocks P_LD needs fewer iterations than P_L, and its count grows more
    slowly with s (the paper reports it flat for the IA form; in the AI form used here it grows, but
    less than P_L's)."""
    its = {}
    for s in (2, 3, 4):
        tab = T.radau_iia(s)
        dt = 0.05
        d, S = kron_setup(tab, N=16, dt=dt)
        b = np.random.default_rng(9).standard_normal(S.shape[0])
        for name, Am in (("lower", tab.A), ("rana", krylov.rana_ld(tab.A))):
            solves = [mg.ExactBlock(d.M, d.K, dt * Am[i, i]) for i in range(s)]
            P = krylov.BlockPreconditioner("lower", Am, d.K, dt, solves)
            its[(name, s)] = krylov.fgmres(lambda v: S @ v, b, P, rtol=1e-10)[1]
    for s in (2, 3, 4):
        assert its[("rana", s)] < its[("lower", s)]
    assert its[("rana", 4)] - its[("rana", 2)] < its[("lower", 4)] - its[("lower", 2)]


def test_ia_system_gives_the_same_stages():
    """w = (A (x) I) k solves (A^{-1} (x) M + dt I (x) K) w = r (Sec. 2.2, eq. stageeqw, linear case)."""
    tab = T.radau_iia(3)
    dt = 0.07
    d, S = kron_setup(tab, N=8, dt=dt)
    r = np.random.default_rng(10).standard_normal(S.shape[0])
    k = np.linalg.solve(S.toarray(), r)
    Sia = krylov.ia_operator(d.M, d.K, tab.A, dt)
    w = np.kron(tab.A, np.eye(d.n)) @ k
    assert np.abs(Sia @ w - r).max() < 1e-12 * np.abs(r).max()


@pytest.mark.parametrize("kind", ["diag", "lower"])
def test_ia_preconditioner_exact_on_matching_structure(kind):
    """IA P_L with exact blocks is the IA system itself for a lower-triangular A; P_D for a diagonal A."""
    tab = T.alexander() if kind == "lower" else T.Tableau("diag", np.diag([0.3, 0.7, 1.1]), np.ones(3) / 3,
                                                           np.array([0.3, 0.7, 1.1]), 1, 1)
    dt = 0.1
    d, _ = kron_setup(tab, dt=dt)
    Sia = krylov.ia_operator(d.M, d.K, tab.A, dt)
    solves = [mg.ExactBlock(d.M, d.K, dt * tab.A[i, i]) for i in range(tab.s)]
    P = krylov.IABlockPreconditioner(tab.A, d.M, dt, solves, diagonal_only=(kind == "diag"))
    b = np.random.default_rng(11).standard_normal(Sia.shape[0])
    x, its, rel, _ = krylov.fgmres(lambda v: Sia @ v, b, P, rtol=1e-12)
    assert its == 1 and np.abs(Sia @ x - b).max() < 1e-11 * np.abs(b).max()


def test_ia_rana_ld_iterations_flat_in_s():
    """Sec. 3.1 / 4.1 (IA form, exact blocks): P_LD iteration counts barely move with s, P_L's grow."""
    its = {}
    for s in (2, 3, 4):
        tab = T.radau_iia(s)
        dt = 0.05
        d, _ = kron_setup(tab, N=16, dt=dt)
        Sia = krylov.ia_operator(d.M, d.K, tab.A, dt)
        b = np.random.default_rng(12).standard_normal(Sia.shape[0])
        for name, Tm in (("lower", tab.A), ("rana", krylov.rana_ld(tab.A))):
            solves = [mg.ExactBlock(d.M, d.K, dt * Tm[i, i]) for i in range(s)]
            P = krylov.IABlockPreconditioner(Tm, d.M, dt, solves)
            its[(name, s)] = krylov.fgmres(lambda v: Sia @ v, b, P, rtol=1e-10)[1]
    print(its)
    assert its[("rana", 4)] - its[("rana", 2)] < its[("lower", 4)] - its[("lower", 2)]
    for s in (2, 3, 4):
        assert its[("rana", s)] <= its[("lower", s)]


# ----------------------------------------------------------------------------
# monolithic multigrid (Sec. 3, 'Monolithic multigrid')
# ----------------------------------------------------------------------------
def _mmg_setup(N=24, levels=3, seed=40):
    d = fem.Discretisation(2, N, W.lognormal_kappa(2, N, 0.5, seed))
    return d, mg.Hierarchy(d, levels)


def test_mmg_single_stage_is_the_block_vcycle():
    """s = 1: the stage-coupled relaxation is plain weighted Jacobi on M + dt a K, so one monolithic
    cycle equals the single-block V-cycle (itself pinned above)."""
    d, h = _mmg_setup()
    dt, a = 0.05, 0.7
    b = np.random.default_rng(41).standard_normal(d.n)
    x_m = mg.MonolithicVCycle(h, np.array([[a]]), dt)(b)
    x_v = mg.VCycle(h, dt * a)(b)
    assert np.abs(x_m - x_v).max() <= 1e-13 * np.abs(x_v).max()


def test_mmg_decouples_for_diagonal_A():
    """Diagonal A: the system and its point blocks are block diagonal over stages, so the cycle is
    the stack of single-block V-cycles with sigma_i = dt a_ii."""
    d, h = _mmg_setup(seed=42)
    dt, A = 0.03, np.diag([0.2, 0.55, 1.0])
    b = np.random.default_rng(43).standard_normal((3, d.n))
    x = mg.MonolithicVCycle(h, A, dt).cycle(b)
    for i in range(3):
        xi = mg.VCycle(h, dt * A[i, i])(b[i])
        assert np.abs(x[i] - xi).max() <= 1e-13 * np.abs(xi).max()


def test_mmg_one_level_is_exact():
    d, h = _mmg_setup(N=12, levels=1)
    tab, dt = T.radau_iia(3), 0.1
    r = np.random.default_rng(44).standard_normal((3, d.n))
    x = mg.MonolithicVCycle(h, tab.A, dt).cycle(r)
    k = rk.KroneckerSolver(d.M, d.K, tab.A, dt).solve(r)
    assert np.abs(x - k).max() <= 1e-12 * np.abs(k).max()


def test_mmg_relaxation_is_point_block_jacobi():
    """One sweep from zero: x = omega D^{-1} b with D_p = M[p,p] I + dt K[p,p] A solved node by node
    (checked against a dense solve of each 3 x 3 block)."""
    d, h = _mmg_setup(N=8, levels=2)
    tab, dt = T.radau_iia(3), 0.2
    b = np.random.default_rng(45).standard_normal((3, d.n))
    x = mg.MonolithicVCycle(h, tab.A, dt).relax(0, np.zeros_like(b), b, 1)
    m, k = d.M.diagonal(), d.K.diagonal()
    for p in range(d.n):
        Dp = m[p] * np.eye(3) + dt * k[p] * tab.A
        assert np.allclose(x[:, p], (2.0 / 3.0) * np.linalg.solve(Dp, b[:, p]), rtol=1e-13, atol=0)


def test_mmg_iterations_nearly_independent_of_s():
    """The paper reports stage-independent iteration counts for monolithic multigrid; FGMRES with one
    cycle per iteration on RadauIIA(1..4): counts within two of each other and at most 12."""
    d, h = _mmg_setup(N=32, levels=3, seed=46)
    dt = 1 / 32
    its = []
    for s in (1, 2, 3, 4):
        tab = T.radau_iia(s)
        S = rk.kronecker_operator(d.M, d.K, tab.A, dt)
        r = np.random.default_rng(47).standard_normal(s * d.n)
        _, it, res, _ = krylov.fgmres(lambda v: S @ v, r, mg.MonolithicVCycle(h, tab.A, dt), rtol=1e-10)
        assert res <= 1e-10
        its.append(it)
    assert max(its) - min(its) <= 2, its
    assert max(its) <= 12, its
