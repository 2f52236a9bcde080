"""Closed forms for the sine eigenmode of the Q1 heat problem (oracle pins).

TEST INFRASTRUCTURE: only tests, the smoke check and the CPU baseline use this.

On a uniform grid with homogeneous Dirichlet data the Q1 mass and stiffness
matrices (kappa = 1) are tensor products of the 1D matrices
M1 = h/6 tridiag(1, 4, 1) and K1 = 1/h tridiag(-1, 2, -1).  The nodal vector
S = prod_d sin(pi x_d) is an eigenvector of both 1D matrices, hence

    K S = lam_h M S,   lam_h = 6 d (1 - cos(pi h)) / (h^2 (2 + cos(pi h))),
    M S = m1^d S,      m1 = h (4 + 2 cos(pi h)) / 6.

With u0 = S and f = (d pi^2 - 1) e^{-t} prod sin(pi x_d), whose load vector is
(d pi^2 - 1) e^{-t} gamma^d S with gamma = 2 (1 - cos(pi h)) / (pi^2 h), the
semidiscrete solution stays a multiple a(t) S of S with

    a' = -lam_h a + beta e^{-t},  beta = (d pi^2 - 1) (gamma / m1)^d,  a(0) = 1,

whose exact solution is a(t) = (1 - beta/(lam_h - 1)) e^{-lam_h t} + beta/(lam_h - 1) e^{-t}.
An RK method (Sec. 2, eq. stageeq) applied to that scalar ODE gives stages from
(I + dt lam_h A) k = beta e^{-(t_n + c dt)} - lam_h a_n 1.
"""
from __future__ import annotations

import math

import numpy as np


def lam_h(dim: int, N: int) -> float:
    h = 1.0 / N
    return 6.0 * dim * (1.0 - math.cos(math.pi * h)) / (h * h * (2.0 + math.cos(math.pi * h)))


def m1(N: int) -> float:
    h = 1.0 / N
    return h * (4.0 + 2.0 * math.cos(math.pi * h)) / 6.0


def gamma(N: int) -> float:
    h = 1.0 / N
    return 2.0 * (1.0 - math.cos(math.pi * h)) / (math.pi**2 * h)


def beta(dim: int, N: int) -> float:
    return (dim * math.pi**2 - 1.0) * (gamma(N) / m1(N)) ** dim


def exact_amplitude(dim: int, N: int, t: float) -> float:
    lam, bet = lam_h(dim, N), beta(dim, N)
    q = bet / (lam - 1.0)
    return (1.0 - q) * math.exp(-lam * t) + q * math.exp(-t)


def scalar_rk_amplitudes(dim: int, N: int, A, b, c, dt: float, steps: int, a0: float = 1.0) -> np.ndarray:
    """a_0..a_steps from the RK recursion applied to the scalar eigenmode ODE."""
    A, b, c = np.asarray(A), np.asarray(b), np.asarray(c)
    lam, bet = lam_h(dim, N), beta(dim, N)
    s = len(b)
    a = [a0]
    t = 0.0
    for _ in range(steps):
        rhs = bet * np.exp(-(t + c * dt)) - lam * a[-1] * np.ones(s)
        k = np.linalg.solve(np.eye(s) + dt * lam * A, rhs)
        a.append(a[-1] + dt * float(b @ k))
        t += dt
    return np.array(a)
