"""Butcher tableaux for the solver (host-side data, float64).

Collocation methods are built from their simplifying conditions: with
abscissae c, the weights satisfy B(s), sum_j b_j c_j^(k-1) = 1/k, and the
matrix satisfies C(s), sum_j a_ij c_j^(k-1) = c_i^k / k, for k = 1..s; both are
s x s Vandermonde systems.  Abscissae:

* Gauss-Legendre(s): Gauss-Legendre nodes mapped from [-1, 1] to [0, 1];
* RadauIIA(s): zeros of P_s(2x-1) - P_{s-1}(2x-1) (P_k Legendre), which include
  x = 1 (App. A defines them equivalently through a derivative of
  x^(s-1) (x-1)^s).

Alexander's three-stage SDIRK follows App. A with its last-row entry read as
z = 3/2 x^2 - 5x + 5/4.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
from numpy.polynomial import legendre as npleg


@dataclass(frozen=True)
class ButcherTableau:
    name: str
    A: np.ndarray
    b: np.ndarray
    c: np.ndarray

    @property
    def s(self) -> int:
        return len(self.b)


def _from_abscissae(name: str, c: np.ndarray) -> ButcherTableau:
    s = len(c)
    V = np.vander(c, s, increasing=True).T  # V[k, j] = c_j^k
    k = np.arange(1, s + 1)
    b = np.linalg.solve(V, 1.0 / k)
    W = c[:, None] ** k[None, :] / k[None, :]  # W[i, k-1] = c_i^k / k
    A = np.linalg.solve(V, W.T).T  # A V^T = W, i.e. sum_j a_ij c_j^(k-1) = c_i^k / k
    return ButcherTableau(name, A, b, c)


def gauss_legendre(s: int) -> ButcherTableau:
    x, _ = npleg.leggauss(s)
    return _from_abscissae(f"GaussLegendre({s})", np.sort((x + 1.0) / 2.0))


def radau_iia(s: int) -> ButcherTableau:
    coef = np.zeros(s + 1)
    coef[s] = 1.0
    coef[s - 1] -= 1.0
    x = np.sort(np.real(npleg.legroots(coef)))
    # polish each root with Newton's method on the Legendre series
    d = npleg.legder(coef)
    for _ in range(3):
        x = x - npleg.legval(x, coef) / npleg.legval(x, d)
    c = (x + 1.0) / 2.0
    c[-1] = 1.0
    return _from_abscissae(f"RadauIIA({s})", c)


def alexander() -> ButcherTableau:
    r = np.roots([1.0, -3.0, 1.5, -1.0 / 6.0])
    x = float(np.real(r[(np.abs(np.imag(r)) < 1e-12) & (np.real(r) > 1 / 6) & (np.real(r) < 0.5)][0]))
    y = -1.5 * x * x + 4.0 * x - 0.25
    z = 1.5 * x * x - 5.0 * x + 1.25
    A = np.array([[x, 0.0, 0.0], [(1 - x) / 2, x, 0.0], [y, z, x]])
    return ButcherTableau("Alexander", A, np.array([y, z, x]), np.array([x, (1 + x) / 2, 1.0]))


def by_name(name: str, s: int | None = None) -> ButcherTableau:
    key = name.lower()
    if key in ("radauiia", "radau"):
        return radau_iia(int(s))
    if key in ("gausslegendre", "gauss", "gl"):
        return gauss_legendre(int(s))
    if key == "alexander":
        return alexander()
    raise KeyError(name)
