"""GPU edge cases against the oracle: the smallest mesh, a zero right-hand side, extreme step sizes,
the deepest hierarchy, ragged tiles at every fused-leg tile size (and a ragged 1088^2 hierarchy whose
second level runs the large-tile legs), high-contrast diffusivity, and the
2048^2 long-horizon workload at full size (stage equations checked with the oracle's assembled system).
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

from paper_2403_08084_gb300 import Solver  # noqa: E402
from paper_2403_08084_gb300 import tableaux as PT  # noqa: E402
from parity import check_vcycle  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


@pytest.mark.parametrize("s", [1, 2, 3, 4])
@pytest.mark.parametrize("precond", ["diag", "lower", "monolithic"])
def test_smallest_mesh(s, precond):
    """N = 2: one interior node, one level (the exact coarsest solve is the whole preconditioner)."""
    N, dt = 2, 0.3
    kap = np.array([0.5, 2.0, 1.5, 0.8])
    d = fem.Discretisation(2, N, kap)
    ot, tab = OT.radau_iia(s), PT.radau_iia(s)
    u0 = W.random_nodal(2, N, seed=90)
    F = np.random.default_rng(91).standard_normal((s, d.n))
    u1_ref, k_ref = rk.step(rk.KroneckerSolver(d.M, d.K, ot.A, dt), d.K, ot.b, dt, d.to_interior(u0), F)
    with Solver(N, tab, dt, kappa=kap, levels=1, precond=precond, rtol=1e-14) as sv:
        u1, k = np.empty(sv.n_nodes), np.empty(sv.n_nodes * s)
        st = sv.step(u0, u1, f_stages=d.to_full(F, s) if s > 1 else d.to_full(F[0]), stages_out=k)
    assert st["converged"]
    assert rel(d.to_interior(u1), u1_ref) < 1e-13
    assert rel(d.to_interior(k, s), k_ref) < 1e-12


@pytest.mark.parametrize("splitting,orth", [("ai", "cgs2"), ("ia", "cgs"), ("ia", "cgs2")])
def test_zero_right_hand_side(splitting, orth):
    """u_n = 0 and no load: r = 0, FGMRES returns at once with k = 0 and u_{n+1} = 0."""
    N = 32
    with Solver(N, PT.radau_iia(3), 0.1, levels=3, splitting=splitting, orth=orth) as sv:
        u = np.zeros(sv.n_nodes)
        k = np.full(sv.n_nodes * 3, 5.0)
        st = sv.step(u, u, stages_out=k)
    assert st["converged"] and st["fgmres_its"] == 0
    assert np.all(u == 0.0) and np.all(k == 0.0)


@pytest.mark.parametrize("dt", [1e-8, 1e-3, 10.0, 1e3])
@pytest.mark.parametrize("splitting", ["ai", "ia"])
def test_extreme_step_sizes(dt, splitting):
    """Mass-dominated (dt -> 0) and stiffness-dominated (dt large) stage systems: the solve still
    matches the direct solve."""
    N, levels, s = 48, 3, 3
    kap = W.lognormal_kappa(2, N, 0.5, seed=92)
    d = fem.Discretisation(2, N, kap)
    ot = OT.radau_iia(s)
    r_full = W.random_nodal(2, N, seed=93, s=s)
    k_ref = rk.KroneckerSolver(d.M, d.K, ot.A, dt).solve(d.to_interior(r_full, s))
    with Solver(N, PT.radau_iia(s), dt, kappa=kap, levels=levels, precond="lower", rtol=1e-13, maxit=300,
                splitting=splitting) as sv:
        k = np.empty(sv.n_nodes * s)
        st = sv.solve(r_full, k)
    assert st["converged"]
    assert rel(d.to_interior(k, s), k_ref) < 1e-9


def test_deepest_hierarchy():
    """N = 256 on 8 levels: the coarsest grid has 2 x 2 cells (one interior node)."""
    N, levels, s, dt = 256, 8, 3, 1 / 128
    kap = W.lognormal_kappa(2, N, 0.5, seed=94)
    d = fem.Discretisation(2, N, kap)
    ot = OT.radau_iia(s)
    h = mg.Hierarchy(d, levels)
    P = krylov.BlockPreconditioner("lower", ot.A, d.K, dt, [mg.VCycle(h, dt * ot.A[i, i]) for i in range(s)])
    v_full = W.random_nodal(2, N, seed=95, s=s)
    z_ref = P(d.to_interior(v_full, s).reshape(-1))
    with Solver(N, PT.radau_iia(s), dt, kappa=kap, levels=levels, precond="lower") as sv:
        z = np.empty(sv.n_nodes * s)
        sv.apply_preconditioner(v_full, z)
    check_vcycle(d.to_interior(z, s).reshape(-1), z_ref, "fp64", "deepest-hierarchy 256^2 8 levels")


def oracle_lower_preconditioner(ot, dt, levels, splitting, v):
    """disc -> the oracle's P_L (AI) or IA lower block preconditioner with V-cycle blocks, applied to v."""
    s = ot.s

    def apply(d):
        h = mg.Hierarchy(d, levels)
        if splitting == "ai":
            P = krylov.BlockPreconditioner("lower", ot.A, d.K, dt, [mg.VCycle(h, dt * ot.A[i, i]) for i in range(s)])
        else:
            T = np.tril(ot.A)
            P = krylov.IABlockPreconditioner(T, d.M, dt, [mg.VCycle(h, dt * T[i, i]) for i in range(s)])
        return P(v)

    return apply


@pytest.mark.parametrize("splitting,prec", [("ai", "fp64"), ("ia", "fp64"), ("ia", "fp32"), ("ai", "fp32"),
                                            ("ai", "bf16"), ("ia", "bf16")])
def test_ragged_tiles_on_every_level(splitting, prec):
    """800^2 on 5 levels (800, 400, 200, 100, 50 cells): node counts per axis that fill none of the
    fused-leg tiles (32 x 16, 16 x 16 and 8 x 8 owned nodes) or the 32 x 8 sweep blocks exactly (FP32 /
    BF16 cycles run the finest level as fused legs too).  One application of the triangular
    preconditioner against the oracle's sparse V-cycles."""
    N, levels, s, dt = 800, 5, 3, 1 / 256
    kap = W.lognormal_kappa(2, N, 0.5, seed=96)
    d = fem.Discretisation(2, N, kap)
    ot = OT.radau_iia(s)
    v_full = W.random_nodal(2, N, seed=97, s=s)
    v = d.to_interior(v_full, s).reshape(-1)
    z_ref = oracle_lower_preconditioner(ot, dt, levels, splitting, v)(d)
    with Solver(N, PT.radau_iia(s), dt, kappa=kap, levels=levels, precond="lower", splitting=splitting,
                vcycle=prec) as sv:
        z = torch.empty(sv.n_nodes * s, dtype=torch.float64, device="cuda")
        sv.apply_preconditioner(torch.from_numpy(v_full).cuda(), z)
        z = z.cpu().numpy()
    check_vcycle(d.to_interior(z, s).reshape(-1), z_ref, prec, f"ragged-800 {splitting}")


@pytest.mark.parametrize("splitting", ["ai", "ia"])
def test_large_ragged_hierarchy_fp64(splitting):
    """1088^2 on 6 levels (1089, 545, 273, 137, 69, 35 nodes per axis): the FP64 triangular sweep with the
    finest level's scaled sweeps, the 545^2 level's large-tile legs with scaled-stencil sweeps, medium and
    small legs and the coarse solve, none of the tiles filled exactly.  One application against the oracle."""
    N, levels, s, dt = 1088, 6, 3, 1 / 256
    kap = W.lognormal_kappa(2, N, 0.5, seed=99)
    d = fem.Discretisation(2, N, kap)
    ot = OT.radau_iia(s)
    v_full = W.random_nodal(2, N, seed=100, s=s)
    v = d.to_interior(v_full, s).reshape(-1)
    z_ref = oracle_lower_preconditioner(ot, dt, levels, splitting, v)(d)
    with Solver(N, PT.radau_iia(s), dt, kappa=kap, levels=levels, precond="lower", splitting=splitting) as sv:
        z = torch.empty(sv.n_nodes * s, dtype=torch.float64, device="cuda")
        sv.apply_preconditioner(torch.from_numpy(v_full).cuda(), z)
        z = z.cpu().numpy()
    check_vcycle(d.to_interior(z, s).reshape(-1), z_ref, "fp64", f"ragged-1088 {splitting}")


@pytest.mark.parametrize("splitting", ["ai", "ia"])
def test_high_contrast_kappa(splitting):
    """log kappa ~ N(0, 2^2) per cell (contrasts above 1e5).  FGMRES stagnates near a relative residual
    of 1e-9 in FP64 here, so the solve runs to rtol 1e-8 and the stages are checked against the oracle's
    assembled stage equations (the true residual must meet the tolerance)."""
    N, levels, s, dt = 64, 3, 3, 1 / 64
    kap = W.lognormal_kappa(2, N, 2.0, seed=98)
    assert kap.max() / kap.min() > 1e5
    d = fem.Discretisation(2, N, kap)
    ot, tab = OT.radau_iia(s), PT.radau_iia(s)
    u0 = W.sine_initial(2, N)
    fsp = W.sine_load_space(2, N)
    coef = [W.sine_load_time(2, c * dt) for c in tab.c]
    with Solver(N, tab, dt, kappa=kap, levels=levels, precond="lower", rtol=1e-8, maxit=500,
                splitting=splitting) as sv:
        u1, k = np.empty(sv.n_nodes), np.empty(sv.n_nodes * s)
        st = sv.step(u0, u1, f_space=fsp, f_coef=coef, stages_out=k)
    assert st["converged"]
    S = rk.kronecker_operator(d.M, d.K, ot.A, dt)
    ui = d.to_interior(u0)
    r = np.stack([c * d.to_interior(fsp) for c in coef]) - (d.K @ ui)[None, :]
    ki = d.to_interior(k, s)
    assert np.linalg.norm(S @ ki.reshape(-1) - r.reshape(-1)) / np.linalg.norm(r) <= 1.5e-8
    assert np.linalg.norm(d.to_interior(u1) - (ui + dt * (ot.b @ ki))) <= 1e-14 * np.linalg.norm(ui)


def test_long_horizon_2048_stage_equations():
    """The 2048^2 workload (lognormal kappa seed 0, 7 levels, RadauIIA(3), dt = 1/100) at full size, in
    the benchmark's configuration (IA form, P_L, one-pass CGS): one step from the sine state; the stages
    satisfy the oracle's assembled stage system to the solver tolerance and u_{n+1} is the RK update."""
    wl = W.WORKLOADS["heat2d-2048-long"]
    N, s, dt = wl.N, wl.s, wl.dt
    kap = W.lognormal_kappa(2, N, 0.5, wl.kappa_seed)
    tab = PT.radau_iia(s)
    u0 = W.sine_initial(2, N)
    fsp = W.sine_load_space(2, N)
    coef = [W.sine_load_time(2, c * dt) for c in tab.c]
    with Solver(N, tab, dt, kappa=kap, levels=wl.levels, precond="lower", rtol=1e-12, splitting="ia",
                orth="cgs") as sv:
        u1, k = np.empty(sv.n_nodes), np.empty(sv.n_nodes * s)
        st = sv.step(u0, u1, f_space=fsp, f_coef=coef, stages_out=k)
    assert st["converged"]
    d = fem.Discretisation(2, N, kap)
    ot = OT.radau_iia(s)
    ui = d.to_interior(u0)
    r = np.stack([c * d.to_interior(fsp) for c in coef]) - (d.K @ ui)[None, :]
    ki = d.to_interior(k, s)
    # (I (x) M + dt A (x) K) k stage by stage (the assembled Kronecker matrix would hold 3.4e8 entries)
    Kk = np.stack([d.K @ ki[j] for j in range(s)])
    Sk = np.stack([d.M @ ki[i] + dt * (ot.A[i] @ Kk) for i in range(s)])
    res = np.linalg.norm(Sk - r) / np.linalg.norm(r)
    assert res <= 2e-12
    assert np.linalg.norm(d.to_interior(u1) - (ui + dt * (ot.b @ ki))) <= 1e-13 * np.linalg.norm(ui)
