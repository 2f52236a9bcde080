"""Butcher tableaux (oracle side).

TEST INFRASTRUCTURE: only tests, the smoke check and the CPU baseline use this.

Collocation tableaux are built in 50-digit arithmetic (mpmath) from their
definition and rounded to float64 at the end:

* RadauIIA(s): the abscissae c_i are the roots of
  d^{s-1}/dx^{s-1} [ x^{s-1} (x-1)^s ]  (App. A, "Some Butcher tableaux").
* Gauss-Legendre(s): not printed in the paper; the abscissae are the roots of
  the shifted Legendre polynomial, i.e. of d^s/dx^s [ x^s (x-1)^s ] (Rodrigues).

For both, the paper states that b and A "follow programmatically" from the
points (App. A): with l_j the Lagrange basis on c,
a_ij = int_0^{c_i} l_j(t) dt and b_j = int_0^1 l_j(t) dt (collocation).

The printed tableaux (RadauIIA(1..3) and Alexander's SDIRK in App. A,
LobattoIIIC(2) in Sec. 2 eq. lobattotableau, WSODIRK433 in App. A) are typed in
as printed, with two readings of garbled entries:

* Alexander: the formula for z lost an exponent; read z = 3/2 x^2 - 5x + 5/4,
  which makes the last row sum to c_3 = 1.
* WSODIRK433: a_31 printed as +1.08354073 makes row 3 sum to 4.4989 instead of
  c_3 = 2.33179673; read a_31 = -1.08354073, which makes every row sum match.
"""
from __future__ import annotations

from dataclasses import dataclass

import mpmath
import numpy as np

_DPS = 50


@dataclass(frozen=True)
class Tableau:
    name: str
    A: np.ndarray  # (s, s)
    b: np.ndarray  # (s,)
    c: np.ndarray  # (s,)
    order: int  # classical order p
    stage_order: int  # q: C(q) holds

    @property
    def s(self) -> int:
        return len(self.b)


def _poly_derivative_roots(m: int, k: int, nder: int):
    """Roots of d^nder/dx^nder [ x^m (x-1)^k ] in mpmath precision (ascending)."""
    with mpmath.workdps(_DPS):
        # coefficients of x^m (x-1)^k, highest degree first
        p = [mpmath.mpf(1)]
        for _ in range(k):  # multiply by (x - 1)
            q = [mpmath.mpf(0)] * (len(p) + 1)
            for i, a in enumerate(p):
                q[i] += a
                q[i + 1] -= a
            p = q
        p = p + [mpmath.mpf(0)] * m  # multiply by x^m
        for _ in range(nder):  # differentiate
            deg = len(p) - 1
            p = [p[i] * (deg - i) for i in range(deg)]
        roots = mpmath.polyroots(p, maxsteps=500, extraprec=200)
        roots = sorted((mpmath.re(r) for r in roots))
        return roots


def _collocation(c):
    """A, b for the collocation method on abscissae c (mpmath numbers)."""
    s = len(c)
    with mpmath.workdps(_DPS):
        A = [[mpmath.mpf(0)] * s for _ in range(s)]
        b = [mpmath.mpf(0)] * s
        for j in range(s):
            # Lagrange basis l_j as polynomial coefficients (lowest degree first)
            coef = [mpmath.mpf(1)]
            denom = mpmath.mpf(1)
            for m in range(s):
                if m == j:
                    continue
                new = [mpmath.mpf(0)] * (len(coef) + 1)
                for i, a in enumerate(coef):
                    new[i] -= a * c[m]
                    new[i + 1] += a
                coef = new
                denom *= c[j] - c[m]
            coef = [a / denom for a in coef]

            def integral(x, coef=coef):
                return sum(a * x ** (i + 1) / (i + 1) for i, a in enumerate(coef))

            b[j] = integral(mpmath.mpf(1))
            for i in range(s):
                A[i][j] = integral(c[i])
        to = lambda v: np.array([float(x) for x in v], dtype=np.float64)  # noqa: E731
        return np.array([to(row) for row in A]), to(b), to(c)


def radau_iia(s: int) -> Tableau:
    """RadauIIA(s) by collocation (App. A); order 2s-1, stage order s (Sec. 4.1)."""
    if s < 1:
        raise ValueError("s must be >= 1")
    c = _poly_derivative_roots(s - 1, s, s - 1)
    A, b, cc = _collocation(c)
    cc[-1] = 1.0  # the last root is exactly 1
    return Tableau(f"RadauIIA({s})", A, b, cc, 2 * s - 1, s)


def gauss_legendre(s: int) -> Tableau:
    """Gauss-Legendre(s) by collocation at the shifted Legendre roots; order 2s, stage order s."""
    if s < 1:
        raise ValueError("s must be >= 1")
    c = _poly_derivative_roots(s, s, s)
    A, b, cc = _collocation(c)
    return Tableau(f"GaussLegendre({s})", A, b, cc, 2 * s, s)


def radau_iia_printed(s: int) -> Tableau:
    """The RadauIIA tableaux as printed in App. A (s = 1, 2, 3)."""
    if s == 1:
        A = np.array([[1.0]])
        b = np.array([1.0])
        c = np.array([1.0])
    elif s == 2:
        A = np.array([[5.0 / 12.0, -1.0 / 12.0], [3.0 / 4.0, 1.0 / 4.0]])
        b = np.array([3.0 / 4.0, 1.0 / 4.0])
        c = np.array([1.0 / 3.0, 1.0])
    elif s == 3:
        r6 = np.sqrt(6.0)
        A = np.array(
            [
                [11 / 45 - 7 * r6 / 360, 37 / 225 - 169 * r6 / 1800, -2 / 225 + r6 / 75],
                [37 / 225 + 169 * r6 / 1800, 11 / 45 + 7 * r6 / 360, -2 / 225 - r6 / 75],
                [4 / 9 - r6 / 36, 4 / 9 + r6 / 36, 1 / 9],
            ]
        )
        b = np.array([4 / 9 - r6 / 36, 4 / 9 + r6 / 36, 1 / 9])
        c = np.array([2 / 5 - r6 / 10, 2 / 5 + r6 / 10, 1.0])
    else:
        raise ValueError("printed RadauIIA only for s = 1, 2, 3")
    return Tableau(f"RadauIIA({s}) printed", A, b, c, 2 * s - 1, s)


def lobatto_iiic2() -> Tableau:
    """Two-stage LobattoIIIC (Sec. 2, eq. lobattotableau); order 2, stage order 1."""
    A = np.array([[0.5, -0.5], [0.5, 0.5]])
    b = np.array([0.5, 0.5])
    c = np.array([0.0, 1.0])
    return Tableau("LobattoIIIC(2)", A, b, c, 2, 1)


def alexander() -> Tableau:
    """Alexander's 3-stage L-stable SDIRK (App. A); order 3, stage order 1 (Sec. 4.1).

    x is the root of x^3 - 3x^2 + 3/2 x - 1/6 in (1/6, 1/2);
    y = -3/2 x^2 + 4x - 1/4 and z = 3/2 x^2 - 5x + 5/4 (garbled exponent restored).
    """
    with mpmath.workdps(_DPS):
        x = mpmath.findroot(lambda t: t**3 - 3 * t**2 + mpmath.mpf(3) / 2 * t - mpmath.mpf(1) / 6, mpmath.mpf("0.43"))
        y = -mpmath.mpf(3) / 2 * x**2 + 4 * x - mpmath.mpf(1) / 4
        z = mpmath.mpf(3) / 2 * x**2 - 5 * x + mpmath.mpf(5) / 4
        xf, yf, zf = float(x), float(y), float(z)
        half = float((1 + x) / 2)
        d = float((1 - x) / 2)
    A = np.array([[xf, 0.0, 0.0], [d, xf, 0.0], [yf, zf, xf]])
    b = np.array([yf, zf, xf])
    c = np.array([xf, half, 1.0])
    return Tableau("Alexander", A, b, c, 3, 1)


def wsodirk433() -> Tableau:
    """WSODIRK433 as printed (App. A) with a_31 read as -1.08354073 (8-digit data)."""
    A = np.array(
        [
            [0.13756544, 0.0, 0.0, 0.0],
            [0.56695123, 0.23483889, 0.0, 0.0],
            [-1.08354073, 2.96618224, 0.44915522, 0.0],
            [0.59761292, -0.43420998, -0.05305815, 0.88965521],
        ]
    )
    b = A[3].copy()
    c = np.array([0.13756544, 0.80179012, 2.33179673, 1.0])
    return Tableau("WSODIRK433", A, b, c, 3, 1)


def order_residuals_B(tab: Tableau, p: int) -> np.ndarray:
    """B(p): sum_i b_i c_i^(k-1) - 1/k for k = 1..p."""
    return np.array([tab.b @ tab.c ** (k - 1) - 1.0 / k for k in range(1, p + 1)])


def order_residuals_C(tab: Tableau, q: int) -> np.ndarray:
    """C(q): sum_j a_ij c_j^(k-1) - c_i^k / k for k = 1..q (max over i)."""
    return np.array([np.max(np.abs(tab.A @ tab.c ** (k - 1) - tab.c**k / k)) for k in range(1, q + 1)])


def by_name(name: str, s: int | None = None) -> Tableau:
    key = name.lower()
    if key in ("radauiia", "radau"):
        return radau_iia(int(s))
    if key in ("gausslegendre", "gauss", "gl"):
        return gauss_legendre(int(s))
    if key in ("alexander", "sdirk3"):
        return alexander()
    if key == "lobattoiiic2":
        return lobatto_iiic2()
    if key == "wsodirk433":
        return wsodirk433()
    raise KeyError(name)
