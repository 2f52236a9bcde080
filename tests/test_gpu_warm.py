"""FGMRES warm start (irk_options.warm_start): the next step's solve starts from the last step's stages.

The paper's solver starts every Krylov solve from zero (Sec. 4.1); the option keeps the stopping test
relative to the step's right-hand side, so a warm-started run must reach the same accuracy against the
oracle's direct solves as a zero-started one, and once the initial transient has passed, in fewer
iterations.  A guess whose residual is not below the right-hand side's norm is dropped.  The first step,
and a step after a call that replaced the stored stages (a Dirichlet step, an adjoint step, an IA-form
irk_solve), start from zero and so equal a zero-started solver bit for bit.
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

from paper_2403_08084_gb300 import Solver  # noqa: E402
from paper_2403_08084_gb300 import tableaux as PT  # noqa: E402


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def run(N, dt, steps, levels, warm, split, prec, orth="cgs2", s=3, rtol=1e-12, precond="lower", dim=2):
    kap = W.lognormal_kappa(2, N, 0.5, seed=31) if dim == 2 else None
    tab = PT.radau_iia(s)
    with Solver(N, tab, dt, kappa=kap, levels=levels, precond=precond, vcycle=prec, splitting=split, orth=orth,
                rtol=rtol, warm_start=warm, dim=dim) as sv:
        u, f = dev(W.sine_initial(dim, N)), dev(W.sine_load_space(dim, N))
        stats = []
        for n in range(steps):
            coef = [W.sine_load_time(dim, (n + c) * dt) for c in tab.c]
            stats.append(sv.step(u, u, f_space=f, f_coef=coef))
        return host(u), stats


@pytest.mark.parametrize("split,prec,orth,precond", [("ai", "fp64", "cgs2", "lower"), ("ia", "fp64", "cgs", "lower"),
                                                     ("ia", "fp32", "cgs2", "lower"),
                                                     ("ai", "fp32", "cgs", "monolithic")])
def test_warm_start_matches_oracle_in_fewer_iterations(split, prec, orth, precond):
    N, dt, steps, levels = 256, 1 / 1024, 6, 5
    uw, sw = run(N, dt, steps, levels, True, split, prec, orth, precond=precond)
    uc, sc = run(N, dt, steps, levels, False, split, prec, orth, precond=precond)
    d = fem.Discretisation(2, N, W.lognormal_kappa(2, N, 0.5, seed=31))
    ot = OT.radau_iia(3)
    Fs = d.to_interior(W.sine_load_space(2, N))
    u_ref, _ = rk.run(d, ot, dt, steps, d.to_interior(W.sine_initial(2, N)), lambda t: W.sine_load_time(2, t) * Fs)
    assert rel(d.to_interior(uw), u_ref) < 1e-10 and rel(d.to_interior(uc), u_ref) < 1e-10
    assert all(st["converged"] and st["rel_resid"] <= 1e-12 for st in sw)
    its_w, its_c = [st["fgmres_its"] for st in sw], [st["fgmres_its"] for st in sc]
    assert its_w[0] == its_c[0]  # the first step has no previous stages
    # the fast modes of the initial state die out within the first steps, whose stages are then a poor guess
    # for the next; once the slow modes dominate, the previous stages are close to the next ones
    late = steps // 2
    assert sum(its_w[late:]) < sum(its_c[late:]), (its_w, its_c)


def test_warm_start_3d():
    """The 3D path (kappa = 1): the same accuracy as a zero start, fewer iterations once the transient is gone."""
    N, dt, steps, levels = 32, 1 / 256, 8, 3
    uw, sw = run(N, dt, steps, levels, True, "ia", "fp64", "cgs", dim=3)
    uc, sc = run(N, dt, steps, levels, False, "ia", "fp64", "cgs", dim=3)
    assert rel(uw, uc) < 1e-10
    its_w, its_c = [st["fgmres_its"] for st in sw], [st["fgmres_its"] for st in sc]
    assert its_w[0] == its_c[0] and sum(its_w[steps // 2:]) < sum(its_c[steps // 2:]), (its_w, its_c)


def test_first_step_equals_zero_start_bitwise():
    uw, _ = run(128, 1 / 256, 1, 4, True, "ia", "fp64")
    uc, _ = run(128, 1 / 256, 1, 4, False, "ia", "fp64")
    assert np.array_equal(uw, uc)


def test_repeated_step_converges_without_iterations():
    """The same step twice: with the one-pass Gram-Schmidt the first solve ends on a true residual below
    rtol, computed as the warm start's initial residual is, so the second solve takes no iteration and
    returns the same stages."""
    N, dt, s = 128, 1 / 256, 3
    tab = PT.radau_iia(s)
    with Solver(N, tab, dt, kappa=W.lognormal_kappa(2, N, 0.5, seed=32), levels=4, precond="lower",
                splitting="ia", orth="cgs", rtol=1e-10, warm_start=True) as sv:
        u0 = dev(W.sine_initial(2, N))
        f = dev(W.sine_load_space(2, N))
        u1, u2 = torch.empty_like(u0), torch.empty_like(u0)
        k1 = torch.empty(sv.n_nodes * s, dtype=torch.float64, device="cuda")
        k2 = torch.empty_like(k1)
        st1 = sv.step(u0, u1, f_space=f, stages_out=k1)
        st2 = sv.step(u0, u2, f_space=f, stages_out=k2)
    assert st1["fgmres_its"] > 0 and st2["fgmres_its"] == 0 and st2["vcycles"] == 0
    assert st2["converged"] and st2["rel_resid"] <= 1e-10
    assert torch.equal(u1, u2) and torch.equal(k1, k2)


def test_reset_initial_guess():
    """After irk_reset_initial_guess the same step repeats the zero-started solve bit for bit."""
    N, dt, s = 128, 1 / 256, 3
    with Solver(N, PT.radau_iia(s), dt, kappa=W.lognormal_kappa(2, N, 0.5, seed=35), levels=4, splitting="ia",
                orth="cgs", rtol=1e-10, warm_start=True) as sv:
        u0 = dev(W.sine_initial(2, N))
        f = dev(W.sine_load_space(2, N))
        u1, u2 = torch.empty_like(u0), torch.empty_like(u0)
        st1 = sv.step(u0, u1, f_space=f)
        sv.reset_initial_guess()
        st2 = sv.step(u0, u2, f_space=f)
    assert st1["fgmres_its"] == st2["fgmres_its"] > 0
    assert torch.equal(u1, u2)


@pytest.mark.parametrize("between", ["dirichlet", "adjoint", "solve_ia"])
def test_calls_that_replace_the_stages_restart_from_zero(between):
    """step, <call>, step on a warm-started handle equals the same sequence on a zero-started one."""
    N, dt, s = 64, 1 / 128, 3
    split = "ia" if between == "solve_ia" else "ai"
    tab = PT.radau_iia(s)
    kap = W.lognormal_kappa(2, N, 0.5, seed=33)
    out = []
    for warm in (True, False):
        with Solver(N, tab, dt, kappa=kap, levels=3, precond="lower", splitting=split, rtol=1e-10,
                    warm_start=warm) as sv:
            u = dev(W.sine_initial(2, N))
            f = dev(W.sine_load_space(2, N))
            k = torch.empty(sv.n_nodes * s, dtype=torch.float64, device="cuda")
            sv.step(u, u, f_space=f)
            if between == "dirichlet":
                g = torch.zeros(sv.n_nodes * s, dtype=torch.float64, device="cuda")
                sv.step_dirichlet(u, g, torch.empty_like(u), f_space=f)
            elif between == "adjoint":
                sv.step(u, torch.empty_like(u), f_space=f, stages_out=k)
                sv.step_adjoint(u, k, u.clone(), torch.empty_like(u))
            else:
                sv.solve(dev(W.random_nodal(2, N, seed=34, s=s)), k)
            st = sv.step(u, u, f_space=f)
            out.append((host(u), st["fgmres_its"]))
    assert np.array_equal(out[0][0], out[1][0]) and out[0][1] == out[1][1]


def test_warm_start_is_ignored_by_the_dirk_path():
    N, dt = 64, 1 / 128
    tab = PT.by_name("Alexander", 3)
    res = []
    for warm in (True, False):
        with Solver(N, tab, dt, levels=3, solver="dirk_cg", rtol=1e-10, warm_start=warm) as sv:
            u = dev(W.sine_initial(2, N))
            for _ in range(3):
                sv.step(u, u)
            res.append(host(u))
    assert np.array_equal(res[0], res[1])
