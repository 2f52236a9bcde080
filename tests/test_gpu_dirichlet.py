"""GPU parity for DAE-type non-homogeneous Dirichlet conditions (Sec. 2.1) against the oracle.

Inputs are full-node vectors: u_n with its boundary values, g at the stage times on the boundary,
and loads F_i of the interior test functions (boundary entries are ignored by both sides).
"""
import numpy as np
import pytest

import workloads as W
from oracle import fem, rk
from oracle import tableaux as OT

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("CUDA GPU required", allow_module_level=True)

from paper_2403_08084_gb300 import IRKError, Solver  # noqa: E402
from paper_2403_08084_gb300 import tableaux as PT  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def full_problem(dim, N, seed):
    kap = W.lognormal_kappa(dim, N, 0.5, seed) if dim == 2 else None
    Mf, Kf = fem.assemble(dim, N, kap)
    I = fem.interior_index(dim, N)
    B = np.setdiff1d(np.arange(Mf.shape[0]), I)
    return kap, Mf, Kf, I, B


def stage_major(v, s):
    """(s, n) stage-major -> node-major flat [p * s + i]."""
    return np.ascontiguousarray(np.asarray(v).T.reshape(-1))


def pair(name):
    if name == "radau3":
        return OT.radau_iia(3), PT.radau_iia(3)
    if name == "radau2":
        return OT.radau_iia(2), PT.radau_iia(2)
    if name == "gauss2":
        return OT.gauss_legendre(2), PT.gauss_legendre(2)
    if name == "alexander":
        return OT.alexander(), PT.alexander()
    raise KeyError(name)


CASES = [
    # dim, N, levels, tableau, precond, vcycle, splitting, solver
    (2, 40, 3, "radau3", "lower", "fp64", "ai", "fgmres"),
    (2, 40, 3, "radau3", "diag", "fp32", "ai", "fgmres"),
    (2, 48, 2, "gauss2", "rana_ld", "bf16", "ai", "fgmres"),
    (2, 40, 3, "radau3", "lower", "fp64", "ia", "fgmres"),
    (2, 40, 3, "alexander", "lower", "fp64", "ai", "dirk_cg"),
    (3, 12, 2, "radau3", "lower", "fp32", "ai", "fgmres"),
    (3, 12, 2, "radau2", "lower", "fp64", "ia", "fgmres"),
]


@pytest.mark.parametrize("dim,N,levels,tname,precond,vcycle,splitting,solver", CASES)
def test_dirichlet_step_matches_oracle(dim, N, levels, tname, precond, vcycle, splitting, solver):
    """Random u_n (boundary values included), random g and F: u_{n+1} and k on all nodes."""
    kap, Mf, Kf, I, B = full_problem(dim, N, seed=70)
    ot, tab = pair(tname)
    s = ot.s
    dt = 1 / 32
    rng = np.random.default_rng(71)
    nf = Mf.shape[0]
    u = rng.standard_normal(nf)
    g = rng.standard_normal((s, nf))
    F = rng.standard_normal((s, nf)) / N**dim
    u1_ref, k_ref = rk.step_dirichlet(Mf, Kf, I, B, ot.A, ot.b, dt, u, F, g)
    with Solver(N, tab, dt, dim=dim, kappa=kap, levels=levels, precond=precond, vcycle=vcycle, rtol=1e-13,
                maxit=400, splitting=splitting, solver=solver) as sv:
        u1 = np.empty(nf)
        k = np.empty(nf * s)
        st = sv.step_dirichlet(u, stage_major(g, s), u1, f_stages=stage_major(F, s), stages_out=k)
        assert st["converged"]
    assert rel(u1, u1_ref) < 1e-10
    assert rel(k.reshape(nf, s).T, k_ref) < 1e-9
    # boundary stages are exact: k_B = A^{-1} (g - u_n) / dt
    assert np.abs(k.reshape(nf, s)[B] - k_ref[:, B].T).max() <= 1e-12 * np.abs(k_ref[:, B]).max()


@pytest.mark.parametrize("tname,q", [("radau2", 2), ("radau3", 3), ("gauss2", 2)])
def test_dirichlet_stage_order_exactness(tname, q):
    """Sec. 2.1: polynomial-in-time solutions of degree <= q with nonzero boundary values are
    reproduced exactly by the GPU path (the oracle's pin, now through the CUDA kernels)."""
    kap, Mf, Kf, I, B = full_problem(2, 16, seed=72)
    ot, tab = pair(tname)
    s = ot.s
    rng = np.random.default_rng(73)
    nf = Mf.shape[0]
    U = rng.standard_normal((q + 1, nf))
    u_of = lambda t: sum(t**j * U[j] for j in range(q + 1))  # noqa: E731
    du_of = lambda t: sum(j * t ** (j - 1) * U[j] for j in range(1, q + 1))  # noqa: E731
    dt, steps = 0.1, 3
    with Solver(16, tab, dt, kappa=kap, levels=2, precond="lower", vcycle="fp64", rtol=1e-14, maxit=400) as sv:
        u = u_of(0.0).copy()
        for n in range(steps):
            ts = [(n + c) * dt for c in ot.c]
            F = np.stack([Mf @ du_of(t) + Kf @ u_of(t) for t in ts])
            g = np.stack([u_of(t) for t in ts])
            sv.step_dirichlet(u, stage_major(g, s), u, f_stages=stage_major(F, s))
    ex = u_of(steps * dt)
    assert np.abs(u - ex).max() < 1e-10 * np.abs(ex).max()


def test_dirichlet_stiffly_accurate_boundary_and_homogeneous_limit():
    kap, Mf, Kf, I, B = full_problem(2, 32, seed=74)
    ot, tab = pair("radau3")
    rng = np.random.default_rng(75)
    nf = Mf.shape[0]
    dt = 0.05
    u = rng.standard_normal(nf)
    g = rng.standard_normal((3, nf))
    F = rng.standard_normal((3, nf)) / 32**2
    with Solver(32, tab, dt, kappa=kap, levels=3, precond="lower", rtol=1e-13) as sv:
        u1 = np.empty(nf)
        sv.step_dirichlet(u, stage_major(g, 3), u1, f_stages=stage_major(F, 3))
        # RadauIIA: b^T A^{-1} = e_s^T, so u_{n+1} = g(t_{n+1}) on the boundary
        assert np.abs(u1[B] - g[-1, B]).max() < 1e-13
        # g = 0 and zero boundary values: the homogeneous step
        u[B] = 0.0
        ud = np.empty(nf)
        sv.step_dirichlet(u, np.zeros(nf * 3), ud, f_stages=stage_major(F, 3))
        uh = np.empty(nf)
        sv.step(u, uh, f_stages=stage_major(F, 3))
    assert np.abs(ud[B]).max() == 0.0
    assert rel(ud, uh) < 1e-13


def test_dirichlet_relaxes_to_boundary_value():
    """Sec. 2.1's setting in 2D: u0 = 0 inside, g = 1, f = 0; LobattoIIIC(2) relaxes monotonically to 1."""
    o = OT.lobatto_iiic2()
    tab = PT.ButcherTableau("LobattoIIIC2", o.A.copy(), o.b.copy(), o.c.copy())
    N = 32
    I = fem.interior_index(2, N)
    nf = (N + 1) ** 2
    u = np.ones(nf)
    u[I] = 0.0
    errs = []
    with Solver(N, tab, 0.02, levels=3, precond="lower", rtol=1e-12) as sv:
        for _ in range(30):
            sv.step_dirichlet(u, np.ones(nf * 2), u)
            errs.append(np.abs(u - 1.0).max())
    assert errs[-1] < 0.05 and all(b <= a + 1e-14 for a, b in zip(errs, errs[1:]))


def test_dirichlet_needs_invertible_A():
    """LobattoIIIA(2) has a zero first row: the boundary stages are not determined by g."""
    tab = PT.ButcherTableau("LobattoIIIA2", np.array([[0.0, 0.0], [0.5, 0.5]]), np.array([0.5, 0.5]),
                            np.array([0.0, 1.0]))
    with Solver(8, tab, 0.1, levels=2, precond="diag") as sv:
        nf = 81
        with pytest.raises(IRKError):
            sv.step_dirichlet(np.zeros(nf), np.zeros(nf * 2), np.zeros(nf))
