"""Parity at the full workload sizes, in the launch configuration bench.py times.

The oracle cannot factor these systems, so the checks use properties that hold
at any size: for kappa = 1 the sine eigenmode stays an eigenmode, so the exact
discrete solution is a(t_n) S with a from the scalar RK recursion; for variable
kappa the GPU stages must satisfy the oracle's assembled stage equations.
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


@pytest.mark.parametrize("precond,prec", [("lower", "fp64"), ("diag", "fp32")])
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
