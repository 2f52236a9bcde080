"""Pins for the oracle's discrete adjoint: complex-step derivatives of the same discrete loop."""
import numpy as np
import pytest

import workloads as W
from oracle import adjoint, fem
from oracle import tableaux as T


def setup(N=6, steps=3, tab=None, seed=1):
    tab = tab or T.radau_iia(3)
    dim = 2
    kap = W.lognormal_kappa(dim, N, 0.5, seed)
    ii = fem.interior_index(dim, N)
    u0 = W.sine_initial(dim, N)[ii]
    Fs = W.sine_load_space(dim, N)[ii]
    dt = 0.05
    loads = np.stack([np.stack([W.sine_load_time(dim, n * dt + c * dt) * Fs for c in tab.c]) for n in range(steps)])
    u_target = 0.5 * u0
    return dim, N, kap, tab, dt, steps, u0, loads, u_target


@pytest.mark.parametrize("tab", [T.radau_iia(3), T.radau_iia(2), T.alexander()])
def test_adjoint_gradient_matches_complex_step(tab):
    dim, N, kap, tab, dt, steps, u0, loads, u_target = setup(tab=tab)
    J, g, _ = adjoint.gradient(dim, N, kap, tab, dt, steps, u0, loads, u_target)
    dirs = W.unit_directions(N**dim, 3, seed=2)
    for d in dirs:
        cs = adjoint.complex_step_derivative(dim, N, np.log(kap), d, tab, dt, steps, u0, loads, u_target)
        assert abs(g @ d - cs) <= 1e-11 * max(abs(cs), 1e-300) + 1e-16


def test_adjoint_state_is_initial_gradient():
    """lam_0 = dJ/du_0: compare with a finite difference in u_0 (J is quadratic in u_0)."""
    dim, N, kap, tab, dt, steps, u0, loads, u_target = setup(N=5, steps=2)
    J0, _, lam0 = adjoint.gradient(dim, N, kap, tab, dt, steps, u0, loads, u_target)
    rng = np.random.default_rng(3)
    du = rng.standard_normal(u0.size)
    eps = 1e-4
    Jp = adjoint.gradient(dim, N, kap, tab, dt, steps, u0 + eps * du, loads, u_target)[0]
    Jm = adjoint.gradient(dim, N, kap, tab, dt, steps, u0 - eps * du, loads, u_target)[0]
    fd = (Jp - Jm) / (2 * eps)  # exact for a quadratic up to roundoff
    assert abs(lam0 @ du - fd) < 1e-8 * abs(fd)


@pytest.mark.parametrize("tab", [T.radau_iia(3), T.gauss_legendre(2)])
def test_eigen_decoupled_gradient_matches_complex_step(tab):
    """The eigen-decoupled direct solver (used at sizes the Kronecker LU cannot factor) gives the same
    gradient, pinned by the complex step like the Kronecker path."""
    dim, N, kap, tab, dt, steps, u0, loads, u_target = setup(N=7, steps=3, tab=tab, seed=4)
    J, g, lam = adjoint.gradient(dim, N, kap, tab, dt, steps, u0, loads, u_target, direct="eigen")
    J2, g2, lam2 = adjoint.gradient(dim, N, kap, tab, dt, steps, u0, loads, u_target)
    assert abs(J - J2) <= 1e-13 * abs(J2)
    assert np.linalg.norm(lam - lam2) <= 1e-12 * np.linalg.norm(lam2)
    for d in W.unit_directions(N**dim, 2, seed=5):
        cs = adjoint.complex_step_derivative(dim, N, np.log(kap), d, tab, dt, steps, u0, loads, u_target)
        assert abs(g @ d - cs) <= 1e-11 * max(abs(cs), 1e-300) + 1e-16
