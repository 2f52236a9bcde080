"""GPU checks of the differentiable time loop (torch.autograd + checkpointed discrete adjoint).

J = 1/2 ||u_N - u*||_M^2 as a function of theta = log(kappa) per cell.  The
gradient is compared with the oracle's discrete adjoint, with central finite
differences, and across checkpoint spacings (recomputation must be exact).
"""
import numpy as np
import pytest

import workloads as W
from oracle import adjoint as OA
from oracle import fem
from oracle import tableaux as OT

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("CUDA GPU required", allow_module_level=True)

from paper_2403_08084_gb300 import Solver  # noqa: E402
from paper_2403_08084_gb300 import adjoint as AD  # noqa: E402
from paper_2403_08084_gb300 import tableaux as PT  # noqa: E402


def setup(N, dt, steps, seed, vcycle, rtol, levels, precond="lower"):
    tab = PT.radau_iia(3)
    kap = W.lognormal_kappa(2, N, 0.5, seed)
    sv = Solver(N, tab, dt, kappa=kap, levels=levels, precond=precond, vcycle=vcycle, rtol=rtol)
    u0 = torch.from_numpy(W.sine_initial(2, N)).cuda()
    f = torch.from_numpy(W.sine_load_space(2, N)).cuda()

    def coef(n):
        return [W.sine_load_time(2, (n + c) * dt) for c in tab.c]

    # target: the final state of the same run with kappa = 1
    sv.set_kappa(np.ones(N * N))
    ut = u0.clone()
    for n in range(steps):
        sv.step(ut, ut, f_space=f, f_coef=coef(n))
    theta = torch.from_numpy(np.log(kap)).cuda()
    return sv, tab, kap, u0, f, coef, ut, theta


def objective(sv, theta, u0, f, coef, steps, ut, checkpoint):
    uN = AD.trajectory(sv, theta, u0, steps, f_space=f, f_coef=coef, checkpoint=checkpoint)
    return AD.mass_norm2(sv, uN - ut)


@pytest.mark.parametrize("vcycle,precond", [("fp64", "lower"), ("fp32", "diag")])
def test_gradient_matches_oracle_adjoint(vcycle, precond):
    N, dt, steps = 48, 1 / 100, 6
    sv, tab, kap, u0, f, coef, ut, theta = setup(N, dt, steps, 1, vcycle, 1e-13, 3, precond)
    th = theta.clone().requires_grad_(True)
    J = objective(sv, th, u0, f, coef, steps, ut, checkpoint=4)
    J.backward()
    g = th.grad.cpu().numpy()
    d = fem.Discretisation(2, N, kap)
    ot = OT.radau_iia(3)
    Fs = d.to_interior(W.sine_load_space(2, N))
    loads = np.stack([np.stack([W.sine_load_time(2, (n + c) * dt) * Fs for c in ot.c]) for n in range(steps)])
    J_ref, g_ref, _ = OA.gradient(2, N, kap, ot, dt, steps, d.to_interior(u0.cpu().numpy()), loads,
                                  d.to_interior(ut.cpu().numpy()))
    assert abs(J.item() - J_ref) <= 1e-10 * abs(J_ref)
    assert np.linalg.norm(g - g_ref) <= 1e-9 * np.linalg.norm(g_ref)
    sv.close()


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
    """Max relative difference between the adjoint gradient and central differences, per h.

    The finite differences run every step with a fixed FGMRES iteration count (the largest the
    gradient run needed): a residual-based stop makes J(theta) piecewise (iteration counts jump
    with theta), while a fixed count keeps it a smooth function, as differentiation assumes."""
    sv, tab, kap, u0, f, coef, ut, theta = setup(N, dt, steps, seed, vcycle, rtol, levels)
    th = theta.clone().requires_grad_(True)
    objective(sv, th, u0, f, coef, steps, ut, checkpoint).backward()
    g = th.grad.cpu().numpy()
    # iteration counts of the forward run
    sv.set_kappa(kap)
    u = u0.clone()
    its = []
    for n in range(steps):
        its.append(sv.step(u, u, f_space=f, f_coef=coef(n))["fgmres_its"])
    sv.close()
    fixed = Solver(N, tab, dt, kappa=kap, levels=levels, precond="lower", vcycle=vcycle, rtol=1e-300,
                   maxit=max(its), restart=max(max(its), 1))
    dirs = W.unit_directions(N * N, ndir, seed=2)
    worst = {}
    with torch.no_grad():
        for h in hs:
            errs = []
            for dvec in dirs:
                dd = torch.from_numpy(dvec).cuda()
                jj = []
                for sgn in (1.0, -1.0):
                    uN = AD.trajectory(fixed, theta + sgn * h * dd, u0, steps, f_space=f, f_coef=coef,
                                       checkpoint=checkpoint, allow_noconv=True)
                    jj.append(AD.mass_norm2(fixed, uN - ut).item())
                fd = (jj[0] - jj[1]) / (2 * h)
                errs.append(abs(fd - g @ dvec) / abs(fd))
            worst[h] = max(errs)
    fixed.close()
    return worst


# Central differences have two error sources: truncation, O(h^2), and the rounding noise of J
# divided by h.  The FGMRES solves are accurate to about cond(S) x 1e-16 (cond ~ 1e3 at 64^2,
# ~ 1e4 at 512^2), so the noise term dominates at h = 1e-6 for unit directions spread over all
# cells: the difference then falls as 1/h, as the printed sweeps show.  The gradient itself is
# pinned to the oracle's discrete adjoint (<= 1e-9) in test_gradient_matches_oracle_adjoint.


def test_gradient_vs_central_differences_small():
    worst = fd_check(N=64, dt=1 / 100, steps=10, levels=3, vcycle="fp64", ndir=5, checkpoint=4,
                     hs=(1e-6, 1e-5, 1e-4))
    print("max relative FD difference by h:", worst)
    assert worst[1e-4] <= 1e-6  # truncation-limited; at h = 1e-6 the noise floor is ~1e-5
    assert worst[1e-6] <= 1e-4


def test_gradient_vs_central_differences_adjoint2d_512():
    """The adjoint workload: 512 x 512 Q1, RadauIIA(3), dt = 1/100, 50 steps, checkpoints every
    10 steps, FP32 V-cycles inside FP64 FGMRES, 20 random unit directions."""
    worst = fd_check(N=512, dt=1 / 100, steps=50, levels=5, vcycle="fp32", ndir=20, checkpoint=10,
                     hs=(1e-6, 1e-3, 1e-2))
    print("max relative FD difference by h:", worst)
    # measured: 6.8e-2 (h = 1e-6), 1.7e-4 (1e-3), 5.1e-5 (1e-2)
    assert min(worst.values()) <= 2e-4
    assert worst[1e-6] <= 0.2
