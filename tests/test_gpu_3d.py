"""GPU parity on 3D Q1 hexahedral grids (kappa = 1) against the FP64 CPU oracle."""
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
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


@pytest.mark.parametrize("N,s", [(6, 1), (12, 2), (9, 4)])
@pytest.mark.parametrize("transpose", [False, True])
def test_stage_operator_3d(N, s, transpose):
    d = fem.Discretisation(3, N)
    ot = OT.gauss_legendre(s)
    dt = 0.02
    x = W.random_nodal(3, N, seed=40, s=s)
    S = rk.kronecker_operator(d.M, d.K, ot.A.T if transpose else ot.A, dt)
    y_ref = d.to_full((S @ d.to_interior(x, s).reshape(-1)).reshape(s, -1), s)
    with Solver(N, PT.gauss_legendre(s), dt, dim=3, levels=1) as sv:
        y = np.empty(sv.n_nodes * s)
        sv.apply_operator(x, y, transpose=transpose)
    assert rel(y, y_ref) < 1e-14


@pytest.mark.parametrize("kind", ["diag", "lower", "upper"])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
def test_preconditioner_3d(kind, prec):
    N, levels, s, dt = 16, 3, 3, 1 / 64
    d = fem.Discretisation(3, N)
    ot = OT.radau_iia(s)
    v = W.random_nodal(3, N, seed=41, s=s)
    h = mg.Hierarchy(d, levels)
    for transpose in (False, True):
        solves = [mg.VCycle(h, dt * ot.A[i, i]) for i in range(s)]
        k = kind if not (transpose and kind != "diag") else ("upper" if kind == "lower" else "lower")
        P = krylov.BlockPreconditioner(k, ot.A.T if transpose else ot.A, d.K, dt, solves)
        z_ref = d.to_full(P(d.to_interior(v, s).reshape(-1)).reshape(s, -1), s)
        with Solver(N, PT.radau_iia(s), dt, dim=3, levels=levels, precond=kind, vcycle=prec) as sv:
            z = np.empty(sv.n_nodes * s)
            sv.apply_preconditioner(v, z, transpose=transpose)
        check_vcycle(z, z_ref, prec, f"preconditioner-3d {kind} transpose={transpose}")


@pytest.mark.parametrize("name,s", [("GaussLegendre", 2), ("GaussLegendre", 4), ("RadauIIA", 3)])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
def test_steps_3d(name, s, prec):
    N, dt, steps, levels = 16, 1 / 64, 3, 2
    d = fem.Discretisation(3, N)
    ot = OT.by_name(name, s)
    u0 = d.to_interior(W.sine_initial(3, N))
    Fs = d.to_interior(W.sine_load_space(3, N))
    uN, _ = rk.run(d, ot, dt, steps, u0, lambda t: W.sine_load_time(3, t) * Fs)
    tab = PT.by_name(name, s)
    with Solver(N, tab, dt, dim=3, levels=levels, precond="lower", vcycle=prec, rtol=1e-12) as sv:
        u = torch.from_numpy(W.sine_initial(3, N)).cuda()
        f = torch.from_numpy(W.sine_load_space(3, N)).cuda()
        for n in range(steps):
            st = sv.step(u, u, f_space=f, f_coef=[W.sine_load_time(3, (n + c) * dt) for c in tab.c])
            assert st["converged"]
        ug = u.cpu().numpy()
    assert rel(d.to_interior(ug), uN) < 1e-10
