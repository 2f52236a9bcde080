"""Parity at the full workload sizes, in the launch configuration bench.py times.

At 1024^2 the oracle solves the stage system directly through the eigen-
decomposition of A (s complex sparse LUs of M + dt lam_i K), and the GPU step in
the benchmark's form (IA, P_L, one-pass CGS; FP64 and FP32 V-cycles) must match
its stages and update element by element.  Where no direct factorisation fits,
the checks use properties that hold at any size: for kappa = 1 the sine
eigenmode stays an eigenmode, so the exact discrete solution is a(t_n) S with a
from the scalar RK recursion; for variable kappa the GPU stages must satisfy the
oracle's assembled stage equations.
"""
import numpy as np
import pytest

import workloads as W
from oracle import fem, rk
from oracle import manufactured as MF
from oracle import tableaux as OT

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("CUDA GPU required", allow_module_level=True)

from paper_2403_08084_gb300 import Solver  # noqa: E402
from paper_2403_08084_gb300 import tableaux as PT  # noqa: E402


@pytest.mark.parametrize("name,s,prec", [("GaussLegendre", 2, "fp32"), ("GaussLegendre", 4, "bf16"),
                                         ("RadauIIA", 3, "fp64")])
def test_heat3d_128_eigenmode(name, s, prec):
    """128^3 Q1, kappa = 1, dt = 1/64, 10 steps: u_n = a_n S exactly (scalar RK recursion)."""
    N, dt, steps, levels = 128, 1 / 64, 10, 5
    tab = PT.by_name(name, s)
    ot = OT.by_name(name, s)
    a = MF.scalar_rk_amplitudes(3, N, ot.A, ot.b, ot.c, dt, steps)
    S = W.sine_initial(3, N)
    with Solver(N, tab, dt, dim=3, levels=levels, precond="lower", vcycle=prec, rtol=1e-12) as sv:
        u = torch.from_numpy(S).cuda()
        f = torch.from_numpy(W.sine_load_space(3, N)).cuda()
        for n in range(steps):
            st = sv.step(u, u, f_space=f, f_coef=[W.sine_load_time(3, (n + c) * dt) for c in tab.c])
            assert st["converged"]
        ug = u.cpu().numpy()
    assert np.linalg.norm(ug - a[-1] * S) <= 1e-10 * np.linalg.norm(a[-1] * S)


@pytest.fixture(scope="module")
def direct_1024():
    """The oracle's direct solution of one step of the 1024^2 workload from the sine state."""
    wl = W.WORKLOADS["heat2d-1024-radau3"]
    N, s, dt = wl.N, wl.s, wl.dt
    kap = W.lognormal_kappa(2, N, 0.5, wl.kappa_seed)
    d = fem.Discretisation(2, N, kap)
    ot = OT.radau_iia(s)
    ui = d.to_interior(W.sine_initial(2, N))
    coef = [W.sine_load_time(2, c * dt) for c in ot.c]
    r = np.stack([c * d.to_interior(W.sine_load_space(2, N)) for c in coef]) - (d.K @ ui)[None, :]
    k = rk.EigenSolver(d.M, d.K, ot.A, dt).solve(r)
    return wl, kap, d, k, ui + dt * (ot.b @ k)


@pytest.mark.parametrize("prec,rtol,k_bound", [("fp64", 1e-14, 1e-10), ("fp32", 1e-14, 1e-10), ("fp64", 1e-12, 1e-9),
                                               ("fp64", 1e-10, 1e-7), ("fp32", 1e-10, 1e-7)])
def test_heat2d_1024_matches_direct_solve(direct_1024, prec, rtol, k_bound):
    """1024^2 Q1, lognormal kappa (seed 0), RadauIIA(3), dt = 1/256, 6 levels, one step from the sine state in
    the benchmark's form (IA, P_L, one-pass CGS).  Solved to rtol 1e-14 the stages and u_1 match the direct
    solve to 1e-10 (relative L2, and element-wise against the largest entry).  The stage system's condition
    number (~1e3 between the relative residual and the relative error of k here) makes a looser residual
    tolerance show in k: the runs at rtol 1e-12 and at the benchmark's 1e-10 are reported beside them with the
    bound that allows, u_1 staying within 1e-10 throughout."""
    wl, kap, d, k_ref, u1_ref = direct_1024
    N, s, dt = wl.N, wl.s, wl.dt
    tab = PT.radau_iia(s)
    coef = [W.sine_load_time(2, c * dt) for c in tab.c]
    with Solver(N, tab, dt, kappa=kap, levels=wl.levels, precond="lower", vcycle=prec, rtol=rtol, splitting="ia",
                orth="cgs", maxit=300) as sv:
        u1, k = np.empty(sv.n_nodes), np.empty(sv.n_nodes * s)
        st = sv.step(W.sine_initial(2, N), u1, f_space=W.sine_load_space(2, N), f_coef=coef, stages_out=k)
    assert st["converged"]
    ki, ui1 = d.to_interior(k, s), d.to_interior(u1)
    ek, eu = ki - k_ref, ui1 - u1_ref
    k_rel = np.linalg.norm(ek) / np.linalg.norm(k_ref)
    k_max = np.abs(ek).max() / np.abs(k_ref).max()
    u_rel = np.sqrt((eu @ (d.M @ eu)) / (u1_ref @ (d.M @ u1_ref)))
    u_max = np.abs(eu).max() / np.abs(u1_ref).max()
    print(f"{prec} rtol {rtol:g}: {st['fgmres_its']} its; k rel L2 {k_rel:.2e}, max {k_max:.2e}; "
          f"u1 rel L2_M {u_rel:.2e}, max {u_max:.2e}")
    assert k_rel <= k_bound and k_max <= k_bound
    assert u_rel <= 1e-10 and u_max <= 1e-10


@pytest.mark.parametrize("precond,prec", [("diag", "fp32")])
def test_heat2d_1024_stage_equations(precond, prec):
    """1024^2 Q1, lognormal kappa (seed 0), RadauIIA(3), dt = 1/256, 6 levels: one step from the sine
    state; the stages satisfy the oracle's assembled system to the solver tolerance."""
    wl = W.WORKLOADS["heat2d-1024-radau3"]
    N, s, dt = wl.N, wl.s, wl.dt
    kap = W.lognormal_kappa(2, N, 0.5, wl.kappa_seed)
    tab = PT.radau_iia(s)
    u0 = W.sine_initial(2, N)
    fsp = W.sine_load_space(2, N)
    coef = [W.sine_load_time(2, c * dt) for c in tab.c]
    with Solver(N, tab, dt, kappa=kap, levels=wl.levels, precond=precond, vcycle=prec, rtol=1e-12) as sv:
        u1 = np.empty(sv.n_nodes)
        k = np.empty(sv.n_nodes * s)
        st = sv.step(u0, u1, f_space=fsp, f_coef=coef, stages_out=k)
    assert st["converged"]
    d = fem.Discretisation(2, N, kap)
    ot = OT.radau_iia(s)
    S = rk.kronecker_operator(d.M, d.K, ot.A, dt)
    ui = d.to_interior(u0)
    r = np.stack([c * d.to_interior(fsp) for c in coef]) - (d.K @ ui)[None, :]
    ki = d.to_interior(k, s)
    res = np.linalg.norm(S @ ki.reshape(-1) - r.reshape(-1)) / np.linalg.norm(r)
    assert res <= 2e-12
    assert np.linalg.norm(d.to_interior(u1) - (ui + dt * (ot.b @ ki))) <= 1e-14 * np.linalg.norm(ui)
