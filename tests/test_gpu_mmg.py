"""GPU parity for monolithic multigrid (Sec. 3, monolithic multigrid): one V-cycle on the whole stage
system with stage-coupled point-block Jacobi relaxation, against the oracle's MonolithicVCycle."""
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
from paper_2403_08084_gb300 import tableaux as PT  # noqa: E402
from parity import VCYCLE_TOL, check_vcycle  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def setup(N, s, seed):
    kap = W.lognormal_kappa(2, N, 0.5, seed)
    d = fem.Discretisation(2, N, kap)
    return kap, d, OT.radau_iia(s), PT.radau_iia(s)


@pytest.mark.parametrize("N,levels,s", [(40, 3, 3), (64, 4, 2), (48, 2, 4), (32, 1, 3)])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
def test_mmg_cycle_matches_oracle(N, levels, s, prec):
    """One application of the preconditioner against the oracle's cycle (1 level: the exact solve)."""
    kap, d, ot, tab = setup(N, s, 80)
    dt = 1 / 48
    v_full = W.random_nodal(2, N, seed=81, s=s)
    v = d.to_interior(v_full, s)
    z_ref = mg.MonolithicVCycle(mg.Hierarchy(d, levels), ot.A, dt).cycle(v)
    with Solver(N, tab, dt, kappa=kap, levels=levels, precond="monolithic", vcycle=prec) as sv:
        z = torch.empty(sv.n_nodes * s, dtype=torch.float64, device="cuda")
        sv.apply_preconditioner(torch.from_numpy(v_full).cuda(), z)
        z = z.cpu().numpy()
    check_vcycle(d.to_interior(z, s), z_ref, prec, f"mmg {N}^2 levels={levels} s={s}")


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_mmg_solve_matches_direct_and_iteration_count(prec):
    N, levels, s, dt = 64, 3, 3, 1 / 64
    kap, d, ot, tab = setup(N, s, 82)
    r_full = W.random_nodal(2, N, seed=83, s=s)
    r = d.to_interior(r_full, s)
    k_ref = rk.KroneckerSolver(d.M, d.K, ot.A, dt).solve(r)
    with Solver(N, tab, dt, kappa=kap, levels=levels, precond="monolithic", vcycle=prec, rtol=1e-12) as sv:
        k = np.empty(sv.n_nodes * s)
        st = sv.solve(r_full, k)
    assert st["converged"] and rel(d.to_interior(k, s), k_ref) < 1e-10
    S = rk.kronecker_operator(d.M, d.K, ot.A, dt)
    _, its, _, _ = krylov.fgmres(lambda x: S @ x, r.reshape(-1), mg.MonolithicVCycle(mg.Hierarchy(d, levels), ot.A, dt),
                                 rtol=1e-12)
    assert abs(st["fgmres_its"] - its) <= (1 if prec == "fp64" else 2), (st["fgmres_its"], its)


def test_mmg_steps_match_oracle_and_iterations_flat_in_s():
    """RK steps with the monolithic preconditioner reproduce the oracle; iteration counts for
    RadauIIA(1..4) stay within two of each other (the paper's stage independence)."""
    N, levels, dt, steps = 48, 3, 1 / 32, 3
    kap = W.lognormal_kappa(2, N, 0.5, 84)
    d = fem.Discretisation(2, N, kap)
    its = {}
    for s in (1, 2, 3, 4):
        ot, tab = OT.radau_iia(s), PT.radau_iia(s)
        u0 = d.to_interior(W.sine_initial(2, N))
        Fs = d.to_interior(W.sine_load_space(2, N))
        uN, _ = rk.run(d, ot, dt, steps, u0, lambda t: W.sine_load_time(2, t) * Fs)
        with Solver(N, tab, dt, kappa=kap, levels=levels, precond="monolithic", rtol=1e-12) as sv:
            u = W.sine_initial(2, N)
            f = W.sine_load_space(2, N)
            n_its = []
            for n in range(steps):
                st = sv.step(u, u, f_space=f, f_coef=[W.sine_load_time(2, (n + c) * dt) for c in tab.c])
                n_its.append(st["fgmres_its"])
        assert rel(d.to_interior(u), uN) < 1e-10
        its[s] = max(n_its)
    assert max(its.values()) - min(its.values()) <= 2, its


@pytest.fixture(scope="module")
def ragged_800():
    """800^2 on 6 levels (801, 401, 201, 101, 51, 26 nodes per axis; coarsest 24^2 x 3 = 1728 coupled
    unknowns): node counts that fill none of the fused-leg tiles exactly, and the finest level large
    enough for the 32 x 16 tiles of the FP32 / BF16 legs."""
    N, levels, s, dt = 800, 6, 3, 1 / 256
    kap, d, ot, tab = setup(N, s, 90)
    v_full = W.random_nodal(2, N, seed=91, s=s)
    z_ref = mg.MonolithicVCycle(mg.Hierarchy(d, levels), ot.A, dt).cycle(d.to_interior(v_full, s))
    return N, levels, s, dt, kap, d, tab, v_full, z_ref


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
def test_mmg_cycle_ragged_tiles_on_every_level(ragged_800, prec):
    N, levels, s, dt, kap, d, tab, v_full, z_ref = ragged_800
    with Solver(N, tab, dt, kappa=kap, levels=levels, precond="monolithic", vcycle=prec) as sv:
        z = torch.empty(sv.n_nodes * s, dtype=torch.float64, device="cuda")
        sv.apply_preconditioner(torch.from_numpy(v_full).cuda(), z)
        z = z.cpu().numpy()
    check_vcycle(d.to_interior(z, s), z_ref, prec, "mmg ragged-800")


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_mmg_transposed_cycle_ragged(ragged_800, prec):
    """The transpose identity on the 800^2 hierarchy (every leg tile size, both relaxation orders)."""
    N, levels, s, dt, kap, d, tab, v_full, _ = ragged_800
    with Solver(N, tab, dt, kappa=kap, levels=levels, precond="monolithic", vcycle=prec) as sv:
        u = torch.from_numpy(v_full).cuda()
        v = torch.from_numpy(W.random_nodal(2, N, seed=92, s=s)).cuda()
        pu, pv = torch.empty_like(u), torch.empty_like(v)
        sv.apply_preconditioner(u, pu, transpose=True)
        sv.apply_preconditioner(v, pv)
        lhs, rhs = float(torch.dot(pu, v)), float(torch.dot(u, pv))
    print(f"PARITY mmg-transpose-identity ragged-800 {prec} rel={abs(lhs - rhs) / abs(rhs):.3e}")
    assert abs(lhs - rhs) <= VCYCLE_TOL[prec] * abs(rhs)


def test_mmg_rejects_unsupported_configurations():
    tab = PT.radau_iia(2)
    with pytest.raises(IRKError):
        Solver(16, tab, 0.1, precond="monolithic", splitting="ia")
    with pytest.raises(IRKError):
        Solver(16, tab, 0.1, dim=3, levels=2, precond="monolithic")
    with pytest.raises(IRKError):  # coupled coarsest system above 4096 unknowns
        Solver(128, PT.radau_iia(3), 0.1, levels=2, precond="monolithic")


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_mmg_transposed_cycle_is_the_transpose(prec):
    """<P^{-T} u, v> = <u, P^{-1} v> for random u, v: the transposed cycle (V(2,2) with A^T, D^{-T}, the
    transposed coarse inverse and the same transfer pair) is the exact transpose of the forward cycle."""
    N, levels, s, dt = 48, 3, 3, 1 / 32
    kap = W.lognormal_kappa(2, N, 0.5, 85)
    with Solver(N, PT.radau_iia(s), dt, kappa=kap, levels=levels, precond="monolithic", vcycle=prec) as sv:
        u = torch.from_numpy(W.random_nodal(2, N, seed=86, s=s)).cuda()
        v = torch.from_numpy(W.random_nodal(2, N, seed=87, s=s)).cuda()
        pu, pv = torch.empty_like(u), torch.empty_like(v)
        sv.apply_preconditioner(u, pu, transpose=True)
        sv.apply_preconditioner(v, pv)
        lhs, rhs = float(torch.dot(pu, v)), float(torch.dot(u, pv))
    print(f"PARITY mmg-transpose-identity 48^2 {prec} rel={abs(lhs - rhs) / abs(rhs):.3e}")
    assert abs(lhs - rhs) <= VCYCLE_TOL[prec] * abs(rhs)


def test_mmg_adjoint_gradient_matches_oracle():
    """The discrete adjoint with the transposed monolithic preconditioner gives the oracle's gradient."""
    from oracle import adjoint as OA
    from paper_2403_08084_gb300 import adjoint as AD

    N, dt, steps = 32, 1 / 50, 3
    kap = W.lognormal_kappa(2, N, 0.5, 88)
    tab, ot = PT.radau_iia(3), OT.radau_iia(3)
    sv = Solver(N, tab, dt, kappa=kap, levels=2, precond="monolithic", rtol=1e-13)
    u0 = torch.from_numpy(W.sine_initial(2, N)).cuda()
    f = torch.from_numpy(W.sine_load_space(2, N)).cuda()
    ut = torch.from_numpy(W.random_nodal(2, N, seed=89)).cuda()

    def coef(n):
        return [W.sine_load_time(2, (n + c) * dt) for c in tab.c]

    th = torch.from_numpy(np.log(kap)).cuda().requires_grad_(True)
    uN = AD.trajectory(sv, th, u0, steps, f_space=f, f_coef=coef, checkpoint=2)
    J = AD.mass_norm2(sv, uN - ut)
    J.backward()
    g = th.grad.cpu().numpy()
    sv.close()
    d = fem.Discretisation(2, N, kap)
    Fs = d.to_interior(W.sine_load_space(2, N))
    loads = np.stack([np.stack([W.sine_load_time(2, (n + c) * dt) * Fs for c in ot.c]) for n in range(steps)])
    J_ref, g_ref, _ = OA.gradient(2, N, kap, ot, dt, steps, d.to_interior(u0.cpu().numpy()), loads,
                                  d.to_interior(ut.cpu().numpy()))
    assert abs(J.item() - J_ref) <= 1e-10 * abs(J_ref)
    assert np.linalg.norm(g - g_ref) <= 1e-9 * np.linalg.norm(g_ref)
