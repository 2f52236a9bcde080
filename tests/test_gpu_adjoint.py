"""GPU checks of the differentiable time loop (torch.autograd + checkpointed discrete adjoint).

J = 1/2 ||u_N - u*||_M^2 as a function of theta = log(kappa) per cell, with u* the
final state of the same run with kappa = 1, which for the sine data is the
closed form a_N S (the sine eigenmode stays an eigenmode; a_N from the oracle's
scalar RK recursion), so no GPU result enters the oracle.  The gradient is
compared with the oracle's discrete adjoint (at 48^2 and at the full 512^2,
50-step adjoint workload), by a Taylor-remainder test, with central finite
differences, and across checkpoint spacings (recomputation must be exact).
"""
import numpy as np
import pytest

import workloads as W
from oracle import adjoint as OA
from oracle import fem
from oracle import manufactured as MF
from oracle import tableaux as OT

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("CUDA GPU required", allow_module_level=True)

from paper_2403_08084_gb300 import Solver  # noqa: E402
from paper_2403_08084_gb300 import adjoint as AD  # noqa: E402
from paper_2403_08084_gb300 import tableaux as PT  # noqa: E402


def target(N, dt, steps):
    """u* = a_N S: the kappa = 1 run's final state, exactly (full node grid)."""
    ot = OT.radau_iia(3)
    a = MF.scalar_rk_amplitudes(2, N, ot.A, ot.b, ot.c, dt, steps)
    return a[-1] * W.sine_initial(2, N)


def setup(N, dt, steps, seed, vcycle, rtol, levels, precond="lower"):
    tab = PT.radau_iia(3)
    kap = W.lognormal_kappa(2, N, 0.5, seed)
    sv = Solver(N, tab, dt, kappa=kap, levels=levels, precond=precond, vcycle=vcycle, rtol=rtol)
    u0 = torch.from_numpy(W.sine_initial(2, N)).cuda()
    f = torch.from_numpy(W.sine_load_space(2, N)).cuda()

    def coef(n):
        return [W.sine_load_time(2, (n + c) * dt) for c in tab.c]

    ut = torch.from_numpy(target(N, dt, steps)).cuda()
    theta = torch.from_numpy(np.log(kap)).cuda()
    return sv, tab, kap, u0, f, coef, ut, theta


def objective(sv, theta, u0, f, coef, steps, ut, checkpoint, allow_noconv=False):
    uN = AD.trajectory(sv, theta, u0, steps, f_space=f, f_coef=coef, checkpoint=checkpoint,
                       allow_noconv=allow_noconv)
    return AD.mass_norm2(sv, uN - ut)


def oracle_gradient(N, kap, dt, steps, direct="kronecker"):
    d = fem.Discretisation(2, N, kap)
    ot = OT.radau_iia(3)
    Fs = d.to_interior(W.sine_load_space(2, N))
    loads = np.stack([np.stack([W.sine_load_time(2, (n + c) * dt) * Fs for c in ot.c]) for n in range(steps)])
    return OA.gradient(2, N, kap, ot, dt, steps, d.to_interior(W.sine_initial(2, N)), loads,
                       d.to_interior(target(N, dt, steps)), direct=direct)


@pytest.mark.parametrize("vcycle,precond", [("fp64", "lower"), ("fp32", "diag")])
def test_gradient_matches_oracle_adjoint(vcycle, precond):
    N, dt, steps = 48, 1 / 100, 6
    sv, tab, kap, u0, f, coef, ut, theta = setup(N, dt, steps, 1, vcycle, 1e-13, 3, precond)
    th = theta.clone().requires_grad_(True)
    J = objective(sv, th, u0, f, coef, steps, ut, checkpoint=4)
    J.backward()
    g = th.grad.cpu().numpy()
    J_ref, g_ref, _ = oracle_gradient(N, kap, dt, steps)
    assert abs(J.item() - J_ref) <= 1e-10 * abs(J_ref)
    assert np.linalg.norm(g - g_ref) <= 1e-9 * np.linalg.norm(g_ref)
    sv.close()


def test_gradient_matches_oracle_adjoint_512():
    """The adjoint workload at full size: 512 x 512 Q1, lognormal kappa (seed 1), RadauIIA(3), dt = 1/100,
    50 steps, checkpoints every 10 steps, FP32 V-cycles inside FP64 FGMRES at rtol 1e-13, against the
    oracle's discrete adjoint with the eigen-decoupled direct stage solver."""
    wl = W.WORKLOADS["adjoint2d-512"]
    N, dt, steps = wl.N, wl.dt, wl.steps
    sv, tab, kap, u0, f, coef, ut, theta = setup(N, dt, steps, wl.kappa_seed, "fp32", 1e-13, wl.levels)
    th = theta.clone().requires_grad_(True)
    J = objective(sv, th, u0, f, coef, steps, ut, checkpoint=10)
    J.backward()
    g = th.grad.cpu().numpy()
    sv.close()
    J_ref, g_ref, _ = oracle_gradient(N, kap, dt, steps, direct="eigen")
    dJ = abs(J.item() - J_ref) / abs(J_ref)
    dg = np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref)
    dg_max = np.abs(g - g_ref).max() / np.abs(g_ref).max()
    print(f"512^2 adjoint vs oracle: J {dJ:.2e}, gradient rel L2 {dg:.2e}, max {dg_max:.2e}")
    # J = 1/2 ||e||_M^2 with e = u_N - u*: |dJ| ~ |<du, e>_M| <= ||du||_M ||e||_M, so u_N within 1e-10 of the
    # oracle's (relative, M-norm) allows |J - J_ref| <= 1e-10 (||u*||_M + ||e||_M) ||e||_M
    d = fem.Discretisation(2, N, kap)
    us = d.to_interior(target(N, dt, steps))
    e_norm, us_norm = np.sqrt(2.0 * J_ref), np.sqrt(us @ (d.M @ us))
    assert abs(J.item() - J_ref) <= 1e-10 * (us_norm + e_norm) * e_norm
    assert dg <= 1e-6 and dg_max <= 1e-6


def fixed_count_solver(N, tab, dt, kap, levels, vcycle, its):
    """A solver that runs every FGMRES solve for exactly ``its`` iterations (no residual test): J(theta) is
    then one smooth function, as differentiation assumes (a residual-based stop makes it piecewise)."""
    return Solver(N, tab, dt, kappa=kap, levels=levels, precond="lower", vcycle=vcycle, rtol=1e-300, maxit=its,
                  restart=its)


def forward_its(sv, u0, f, coef, steps, kap):
    sv.set_kappa(kap)
    u = u0.clone()
    return [sv.step(u, u, f_space=f, f_coef=coef(n))["fgmres_its"] for n in range(steps)]


def test_taylor_remainder_adjoint2d_512():
    """Taylor test on the adjoint workload (512^2, 50 steps, checkpoint 10, FP32 V-cycles, FP64 FGMRES): for
    the 20 unit directions (seed 2), R(h) = |J(theta + h d) - J(theta) - h g.d| falls as h^2 over
    h = 1e-1, 1e-2, 1e-3 (it would fall as h if g.d were wrong).
    Below that R reaches the rounding floor of J: J = 1/2 ||e||_M^2 with ||e|| / ||u|| ~ 4e-3 here, so the
    FP64 rounding of u_N (~1e-15) makes J uncertain to ~3e-13 of itself, about R(1e-4); at h = 1e-4 the
    test only asks R to stay below that floor or below the h^2 extrapolation."""
    wl = W.WORKLOADS["adjoint2d-512"]
    N, dt, steps = wl.N, wl.dt, wl.steps
    sv, tab, kap, u0, f, coef, ut, theta = setup(N, dt, steps, wl.kappa_seed, "fp32", 1e-13, wl.levels)
    th = theta.clone().requires_grad_(True)
    objective(sv, th, u0, f, coef, steps, ut, checkpoint=10).backward()
    g = th.grad
    its = max(forward_its(sv, u0, f, coef, steps, kap)) + 2
    sv.close()
    fixed = fixed_count_solver(N, tab, dt, kap, wl.levels, "fp32", its)
    hs = (1e-1, 1e-2, 1e-3)
    orders, first, tail = [], [], []
    with torch.no_grad():
        J0 = objective(fixed, theta, u0, f, coef, steps, ut, 10, True).item()
        for dvec in W.unit_directions(N * N, 20, seed=2):
            dd = torch.from_numpy(dvec).cuda()
            gd = float(torch.dot(g, dd).item())
            R, D = [], []
            for h in hs:
                Jh = objective(fixed, theta + h * dd, u0, f, coef, steps, ut, 10, True).item()
                R.append(abs(Jh - J0 - h * gd))
                D.append(abs(Jh - J0))
            slope = np.polyfit(np.log10(hs), np.log10(R), 1)[0]
            orders.append(slope)
            first.append(np.polyfit(np.log10(hs), np.log10(D), 1)[0])
            R4 = abs(objective(fixed, theta + 1e-4 * dd, u0, f, coef, steps, ut, 10, True).item() - J0 - 1e-4 * gd)
            tail.append(R4 / max(R[-1] / 100.0, 1e-12 * abs(J0)))
    fixed.close()
    print("Taylor remainder orders:", np.round(orders, 3), "first-difference orders:", np.round(first, 3),
          "R(1e-4) / max(h^2 extrapolation, floor):", np.round(tail, 3))
    assert min(orders) >= 1.9 and max(orders) <= 2.1
    assert max(tail) <= 2.0


def test_checkpoint_spacing_does_not_change_the_gradient():
    N, dt, steps = 32, 1 / 50, 7
    sv, tab, kap, u0, f, coef, ut, theta = setup(N, dt, steps, 2, "fp64", 1e-12, 2)
    grads = []
    for ck in (1, 3, 7):
        th = theta.clone().requires_grad_(True)
        objective(sv, th, u0, f, coef, steps, ut, ck).backward()
        grads.append(th.grad.cpu().numpy())
    assert np.array_equal(grads[0], grads[1]) and np.array_equal(grads[0], grads[2])
    sv.close()


def fd_check(N, dt, steps, levels, vcycle, ndir, checkpoint, hs=(1e-6,), rtol=1e-13, seed=1):
    """Max relative difference between the adjoint gradient and central differences, per h, with the
    finite differences on a fixed FGMRES iteration count (the largest the gradient run needed)."""
    sv, tab, kap, u0, f, coef, ut, theta = setup(N, dt, steps, seed, vcycle, rtol, levels)
    th = theta.clone().requires_grad_(True)
    objective(sv, th, u0, f, coef, steps, ut, checkpoint).backward()
    g = th.grad.cpu().numpy()
    its = forward_its(sv, u0, f, coef, steps, kap)
    sv.close()
    fixed = fixed_count_solver(N, tab, dt, kap, levels, vcycle, max(its))
    dirs = W.unit_directions(N * N, ndir, seed=2)
    worst = {}
    with torch.no_grad():
        for h in hs:
            errs = []
            for dvec in dirs:
                dd = torch.from_numpy(dvec).cuda()
                jj = [objective(fixed, theta + sgn * h * dd, u0, f, coef, steps, ut, checkpoint, True).item()
                      for sgn in (1.0, -1.0)]
                fd = (jj[0] - jj[1]) / (2 * h)
                errs.append(abs(fd - g @ dvec) / abs(fd))
            worst[h] = max(errs)
    fixed.close()
    return worst


# Central differences have two error sources: truncation, O(h^2), and the rounding noise of J
# divided by h.  The FGMRES solves are accurate to about cond(S) x 1e-16 (cond ~ 1e3 at 64^2,
# ~ 1e4 at 512^2), so the noise term dominates at h = 1e-6 for unit directions spread over all
# cells: the difference then falls as 1/h, as the printed sweeps show.  The gradient itself is
# pinned to the oracle's discrete adjoint and by the Taylor-remainder test above.


def test_gradient_vs_central_differences_small():
    worst = fd_check(N=64, dt=1 / 100, steps=10, levels=3, vcycle="fp64", ndir=5, checkpoint=4,
                     hs=(1e-6, 1e-5, 1e-4))
    print("max relative FD difference by h:", worst)
    assert worst[1e-4] <= 1e-6  # truncation-limited; at h = 1e-6 the noise floor is ~1e-5
    assert worst[1e-6] <= 1e-4


def test_gradient_vs_central_differences_adjoint2d_512():
    """The adjoint workload: 512 x 512 Q1, RadauIIA(3), dt = 1/100, 50 steps, checkpoints every
    10 steps, FP32 V-cycles inside FP64 FGMRES, 20 random unit directions.  Reported, with the
    bound the noise floor allows at h = 1e-6; the exactness checks are the two tests above."""
    wl = W.WORKLOADS["adjoint2d-512"]
    worst = fd_check(N=wl.N, dt=wl.dt, steps=wl.steps, levels=wl.levels, vcycle="fp32", ndir=20, checkpoint=10,
                     hs=(1e-6, 1e-3, 1e-2), seed=wl.kappa_seed)
    print("max relative FD difference by h:", worst)
    assert min(worst.values()) <= 2e-4
    assert worst[1e-6] <= 0.2
