"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle.

Inputs come from the shared seeded generators in ``workloads``; expected values
come from ``oracle`` only.  Sizes span several thread blocks with ragged tails
(node counts per axis that are not multiples of the 32 x 8 block).
"""
import numpy as np
import pytest

import workloads as W
from oracle import fem, krylov, mg, rk
from oracle import tableaux as OT

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("CUDA GPU required", allow_module_level=True)

from paper_2403_08084_gb300 import IRKError, Solver  # noqa: E402
from parity import check_vcycle  # noqa: E402
from paper_2403_08084_gb300 import tableaux as PT  # noqa: E402


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def product_tableau(name, s):
    return PT.by_name(name, s)


def oracle_tableau(name, s):
    return OT.by_name(name, s)


# ----------------------------------------------------------------------------
# stage operator (I (x) M + dt A (x) K)
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("N,s", [(8, 1), (37 * 2, 3), (50, 2), (96, 4)])
@pytest.mark.parametrize("transpose", [False, True])
def test_stage_operator(N, s, transpose):
    kap = W.lognormal_kappa(2, N, 0.5, seed=3)
    d = fem.Discretisation(2, N, kap)
    ot = oracle_tableau("RadauIIA", s)
    dt = 0.01
    x_full = W.random_nodal(2, N, seed=4, s=s)
    S = rk.kronecker_operator(d.M, d.K, ot.A.T if transpose else ot.A, dt)
    y_ref = d.to_full((S @ d.to_interior(x_full, s).reshape(-1)).reshape(s, -1), s)
    levels = 1 if N <= 64 else 2
    with Solver(N, product_tableau("RadauIIA", s), dt, kappa=kap, levels=levels) as sv:
        y = torch.empty(sv.n_nodes * s, dtype=torch.float64, device="cuda")
        sv.apply_operator(dev(x_full), y, transpose=transpose)
        y = host(y)
    assert rel(y, y_ref) < 1e-14
    assert np.all(y.reshape(-1, s)[W.boundary_mask(2, N)] == 0.0)


# ----------------------------------------------------------------------------
# one application of the block preconditioner with V-cycle blocks
# ----------------------------------------------------------------------------
def oracle_preconditioner(d, ot, dt, levels, kind, transpose, nu=(2, 2), omega=2 / 3):
    h = mg.Hierarchy(d, levels)
    nu1, nu2 = (nu[1], nu[0]) if transpose else nu
    solves = [mg.VCycle(h, dt * ot.A[i, i], nu1, nu2, omega) for i in range(ot.s)]
    Amat = ot.A.T if transpose else ot.A
    k = kind
    if transpose and kind != "diag":
        k = "upper" if kind == "lower" else "lower"
    return krylov.BlockPreconditioner(k, Amat, d.K, dt, solves)


@pytest.mark.parametrize("kind", ["diag", "lower", "upper"])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
def test_preconditioner(kind, prec):
    N, levels, s, dt = 96, 3, 3, 1 / 64
    kap = W.lognormal_kappa(2, N, 0.5, seed=5)
    d = fem.Discretisation(2, N, kap)
    ot = oracle_tableau("RadauIIA", s)
    v_full = W.random_nodal(2, N, seed=6, s=s)
    for transpose in (False, True):
        P = oracle_preconditioner(d, ot, dt, levels, kind, transpose)
        z_ref = d.to_full(P(d.to_interior(v_full, s).reshape(-1)).reshape(s, -1), s)
        with Solver(N, product_tableau("RadauIIA", s), dt, kappa=kap, levels=levels, precond=kind,
                    vcycle=prec) as sv:
            z = torch.empty(sv.n_nodes * s, dtype=torch.float64, device="cuda")
            sv.apply_preconditioner(dev(v_full), z, transpose=transpose)
            z = host(z)
        check_vcycle(z, z_ref, prec, f"preconditioner-2d {kind} transpose={transpose}")


@pytest.mark.parametrize("levels", [1, 2, 4])
def test_vcycle_levels_single_stage(levels):
    """s = 1 (backward Euler): the preconditioner is one V-cycle (levels = 1: the exact solve)."""
    N, dt = 64, 0.02
    kap = W.lognormal_kappa(2, N, 0.5, seed=7)
    d = fem.Discretisation(2, N, kap)
    ot = oracle_tableau("RadauIIA", 1)
    v_full = W.random_nodal(2, N, seed=8)
    P = oracle_preconditioner(d, ot, dt, levels, "diag", False)
    z_ref = d.to_full(P(d.to_interior(v_full, 1)), 1)
    with Solver(N, product_tableau("RadauIIA", 1), dt, kappa=kap, levels=levels) as sv:
        z = torch.empty(sv.n_nodes, dtype=torch.float64, device="cuda")
        sv.apply_preconditioner(dev(v_full), z)
        z = host(z)
    check_vcycle(z, z_ref, "fp64", f"single-stage levels={levels}")


# ----------------------------------------------------------------------------
# the stage solve and the RK step
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("kind", ["diag", "lower", "upper"])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
@pytest.mark.parametrize("orth", ["cgs2", "dgks", "cgs"])
def test_solve_matches_direct_and_iteration_count(kind, prec, orth):
    N, levels, s, dt = 64, 3, 3, 1 / 64
    kap = W.lognormal_kappa(2, N, 0.5, seed=9)
    d = fem.Discretisation(2, N, kap)
    ot = oracle_tableau("RadauIIA", s)
    r_full = W.random_nodal(2, N, seed=10, s=s)
    r_int = d.to_interior(r_full, s)
    k_ref = rk.KroneckerSolver(d.M, d.K, ot.A, dt).solve(r_int)
    with Solver(N, product_tableau("RadauIIA", s), dt, kappa=kap, levels=levels, precond=kind, vcycle=prec,
                rtol=1e-12, orth=orth) as sv:
        k = torch.empty(sv.n_nodes * s, dtype=torch.float64, device="cuda")
        st = sv.solve(dev(r_full), k)
        k = host(k)
    assert st["converged"] and st["rel_resid"] <= 1e-12
    assert rel(d.to_interior(k, s), k_ref) < 1e-10
    if prec == "fp64":
        S = rk.kronecker_operator(d.M, d.K, ot.A, dt)
        P = oracle_preconditioner(d, ot, dt, levels, kind, False)
        _, its, _, _ = krylov.fgmres(lambda v: S @ v, r_int.reshape(-1), P, rtol=1e-12)
        # one-pass Gram-Schmidt may need a few more iterations at this tight tolerance
        assert abs(st["fgmres_its"] - its) <= (1 if orth != "cgs" else 3), (st["fgmres_its"], its)


def manufactured_run(N, name, s, dt, steps, levels, kind, prec, kappa=None, rtol=1e-12):
    """GPU run of the sine-forced heat problem; returns final u (full grid) and per-step stats."""
    u0 = W.sine_initial(2, N)
    fsp = W.sine_load_space(2, N)
    tab = product_tableau(name, s)
    stats = []
    with Solver(N, tab, dt, kappa=kappa, levels=levels, precond=kind, vcycle=prec, rtol=rtol) as sv:
        u = dev(u0)
        f = dev(fsp)
        for n in range(steps):
            t = n * dt
            coef = [W.sine_load_time(2, t + c * dt) for c in tab.c]
            stats.append(sv.step(u, u, f_space=f, f_coef=coef))
        return host(u), stats


def oracle_run(N, name, s, dt, steps, kappa=None):
    d = fem.Discretisation(2, N, kappa)
    ot = oracle_tableau(name, s)
    u0 = d.to_interior(W.sine_initial(2, N))
    Fs = d.to_interior(W.sine_load_space(2, N))
    uN, _ = rk.run(d, ot, dt, steps, u0, lambda t: W.sine_load_time(2, t) * Fs)
    return d, uN


def test_heat2d_32_radau2_exact_blocks():
    """32 x 32 Q1, RadauIIA(2), dt = 1/32, 10 steps, P_L with exact block solves (one level)."""
    N, dt, steps = 32, 1 / 32, 10
    u, stats = manufactured_run(N, "RadauIIA", 2, dt, steps, 1, "lower", "fp64", rtol=1e-12)
    d, uN = oracle_run(N, "RadauIIA", 2, dt, steps)
    assert rel(d.to_interior(u), uN) < 1e-10
    assert all(s["converged"] for s in stats)
    # at the tolerance the workload names (1e-10) the result still agrees closely
    u10, _ = manufactured_run(N, "RadauIIA", 2, dt, steps, 1, "lower", "fp64", rtol=1e-10)
    assert rel(d.to_interior(u10), uN) < 1e-8


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
@pytest.mark.parametrize("kind", ["diag", "lower"])
def test_variable_kappa_steps(prec, kind):
    N, dt, steps, levels = 128, 1 / 256, 3, 4
    kap = W.lognormal_kappa(2, N, 0.5, seed=0)
    u, stats = manufactured_run(N, "RadauIIA", 3, dt, steps, levels, kind, prec, kappa=kap)
    d, uN = oracle_run(N, "RadauIIA", 3, dt, steps, kappa=kap)
    assert rel(d.to_interior(u), uN) < 1e-10, rel(d.to_interior(u), uN)


@pytest.mark.parametrize("name,s", [("GaussLegendre", 2), ("GaussLegendre", 4), ("Alexander", 3)])
def test_other_tableaux(name, s):
    N, dt, steps = 48, 1 / 64, 2
    kap = W.lognormal_kappa(2, N, 0.5, seed=11)
    u, _ = manufactured_run(N, name, s, dt, steps, 2, "lower", "fp64", kappa=kap)
    d, uN = oracle_run(N, name, s, dt, steps, kappa=kap)
    assert rel(d.to_interior(u), uN) < 1e-10


@pytest.mark.parametrize("splitting", ["ai", "ia"])
@pytest.mark.parametrize("orth", ["cgs2", "dgks", "cgs"])
def test_restarted_fgmres(orth, splitting):
    """A short restart length forces several restart cycles; the result still matches the direct solve."""
    N, levels, s, dt = 48, 2, 3, 1 / 32
    kap = W.lognormal_kappa(2, N, 0.5, seed=30)
    d = fem.Discretisation(2, N, kap)
    ot = oracle_tableau("RadauIIA", s)
    r_full = W.random_nodal(2, N, seed=31, s=s)
    k_ref = rk.KroneckerSolver(d.M, d.K, ot.A, dt).solve(d.to_interior(r_full, s))
    with Solver(N, product_tableau("RadauIIA", s), dt, kappa=kap, levels=levels, precond="diag", restart=4,
                rtol=1e-12, orth=orth, splitting=splitting) as sv:
        k = np.empty(sv.n_nodes * s)
        st = sv.solve(r_full, k)
    assert st["converged"] and st["fgmres_its"] > 4
    assert rel(d.to_interior(k, s), k_ref) < 1e-10


@pytest.mark.parametrize("splitting", ["ai", "ia"])
@pytest.mark.parametrize("rtol", [1e-8, 1e-10, 1e-12])
def test_one_pass_gram_schmidt_reports_the_true_residual(splitting, rtol):
    """With one-pass classical Gram-Schmidt the reported residual is recomputed as ||r - S k|| / ||r||
    at convergence; it must meet rtol, and the solution must match the two-pass solve to that level."""
    N, levels, s, dt = 128, 4, 3, 1 / 64
    kap = W.lognormal_kappa(2, N, 0.5, seed=33)
    tab = product_tableau("RadauIIA", s)
    r = dev(W.random_nodal(2, N, seed=34, s=s))
    ks = {}
    for orth in ("cgs", "cgs2"):
        with Solver(N, tab, dt, kappa=kap, levels=levels, precond="lower", rtol=rtol, orth=orth,
                    splitting=splitting) as sv:
            k = torch.empty(sv.n_nodes * s, dtype=torch.float64, device="cuda")
            st = sv.solve(r, k)
            assert st["converged"] and st["rel_resid"] <= rtol
            if orth == "cgs":
                # the AI operator applied to k reproduces r (the IA solve returns k too)
                with Solver(N, tab, dt, kappa=kap, levels=levels, precond="lower") as ai:
                    y = torch.empty_like(k)
                    ai.apply_operator(k, y)
                true = float(torch.linalg.vector_norm(y - r) / torch.linalg.vector_norm(r))
                assert true <= 1.5 * rtol, (true, st["rel_resid"])
            ks[orth] = host(k)
    assert rel(ks["cgs"], ks["cgs2"]) < 1e3 * rtol


@pytest.mark.parametrize("prec", ["fp64", "bf16"])
def test_graph_replay_equals_eager_launches(prec, monkeypatch):
    """Each Arnoldi step runs as a captured CUDA graph; eager launches give the same bits."""
    N, s, dt = 64, 3, 1 / 64
    kap = W.lognormal_kappa(2, N, 0.5, seed=32)
    tab = product_tableau("RadauIIA", s)
    u0 = W.sine_initial(2, N)
    f = W.sine_load_space(2, N)
    outs = []
    for env in ("0", "1"):
        monkeypatch.setenv("IRK_NO_GRAPHS", env)
        with Solver(N, tab, dt, kappa=kap, levels=3, precond="lower", vcycle=prec) as sv:
            u = dev(u0)
            for n in range(3):  # later steps replay the graphs captured in the first
                sv.step(u, u, f_space=dev(f), f_coef=[W.sine_load_time(2, (n + c) * dt) for c in tab.c])
            outs.append(host(u))
    assert np.array_equal(outs[0], outs[1])


def test_stages_out_and_host_pointers():
    """Host (NumPy) buffers give the same result as device buffers."""
    N, s, dt = 40, 3, 0.01
    kap = W.lognormal_kappa(2, N, 0.5, seed=12)
    tab = product_tableau("RadauIIA", s)
    u0 = W.random_nodal(2, N, seed=13)
    F = W.random_nodal(2, N, seed=14, s=s)
    with Solver(N, tab, dt, kappa=kap, levels=2, rtol=1e-12) as sv:
        u1d = torch.empty(sv.n_nodes, dtype=torch.float64, device="cuda")
        kd = torch.empty(sv.n_nodes * s, dtype=torch.float64, device="cuda")
        sv.step(dev(u0), u1d, f_stages=dev(F), stages_out=kd)
        u1h = np.empty(sv.n_nodes)
        kh = np.empty(sv.n_nodes * s)
        sv.step(u0, u1h, f_stages=F, stages_out=kh)
    assert np.array_equal(host(u1d), u1h) and np.array_equal(host(kd), kh)
    d = fem.Discretisation(2, N, kap)
    ot = oracle_tableau("RadauIIA", s)
    solver = rk.KroneckerSolver(d.M, d.K, ot.A, dt)
    u_ref, k_ref = rk.step(solver, d.K, ot.b, dt, d.to_interior(u0), d.to_interior(F, s))
    assert rel(d.to_interior(u1h), u_ref) < 1e-10 and rel(d.to_interior(kh, s), k_ref) < 1e-10


def test_boundary_entries_of_inputs_are_ignored():
    N, s, dt = 24, 2, 0.05
    tab = product_tableau("RadauIIA", s)
    u0 = W.random_nodal(2, N, seed=15)
    u_dirty = u0.copy()
    u_dirty[W.boundary_mask(2, N)] = 7.0
    with Solver(N, tab, dt) as sv:
        a, b = np.empty(sv.n_nodes), np.empty(sv.n_nodes)
        sv.step(u0, a)
        sv.step(u_dirty, b)
    assert np.array_equal(a, b) and np.all(a[W.boundary_mask(2, N)] == 0.0)


def test_error_statuses():
    N, s, dt = 32, 2, 0.05
    tab = product_tableau("RadauIIA", s)
    u0 = W.random_nodal(2, N, seed=16)
    with Solver(N, tab, dt, levels=3, maxit=1, rtol=1e-14) as sv:
        out = np.empty(sv.n_nodes)
        with pytest.raises(IRKError) as e:
            sv.step(u0, out)
        assert e.value.code == -4
        st = sv.step(u0, out, allow_noconv=True)
        assert st["fgmres_its"] == 1 and not st["converged"]
        bad = u0.copy()
        bad[N + 3] = np.nan
        with pytest.raises(IRKError) as e:
            sv.step(bad, out)
        assert e.value.code == -5
        # the handle stays usable after an error
        st = sv.step(u0, out, allow_noconv=True)
        assert st["fgmres_its"] == 1


# ----------------------------------------------------------------------------
# discrete adjoint step
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("kind,prec", [("lower", "fp64"), ("diag", "fp32")])
def test_adjoint_step_matches_oracle(kind, prec):
    from oracle import adjoint as OA

    N, s, dt, steps = 32, 3, 0.01, 2
    kap = W.lognormal_kappa(2, N, 0.5, seed=17)
    d = fem.Discretisation(2, N, kap)
    ot = oracle_tableau("RadauIIA", s)
    u0 = d.to_interior(W.sine_initial(2, N))
    Fs = d.to_interior(W.sine_load_space(2, N))
    loads = np.stack([np.stack([W.sine_load_time(2, n * dt + c * dt) * Fs for c in ot.c]) for n in range(steps)])
    u_target = 0.5 * u0
    J, g_ref, lam0_ref = OA.gradient(2, N, kap, ot, dt, steps, u0, loads, u_target)
    tab = product_tableau("RadauIIA", s)
    with Solver(N, tab, dt, kappa=kap, levels=3, precond=kind, vcycle=prec, rtol=1e-13) as sv:
        us = [d.to_full(u0)]
        ks = []
        f = d.to_full(Fs)
        for n in range(steps):
            u1 = np.empty(sv.n_nodes)
            k = np.empty(sv.n_nodes * s)
            coef = [W.sine_load_time(2, n * dt + c * dt) for c in tab.c]
            sv.step(us[-1], u1, f_space=f, f_coef=coef, stages_out=k)
            us.append(u1)
            ks.append(k)
        lam = d.to_full(d.M @ (d.to_interior(us[-1]) - u_target))
        grad = np.zeros(N * N)
        for n in range(steps - 1, -1, -1):
            lam_n = np.empty(sv.n_nodes)
            sv.step_adjoint(us[n], ks[n], lam, lam_n, grad)
            lam = lam_n
    assert rel(grad, g_ref) < 1e-9, rel(grad, g_ref)
    assert rel(d.to_interior(lam), lam0_ref) < 1e-9
