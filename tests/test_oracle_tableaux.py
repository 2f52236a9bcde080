"""Pins for the oracle's Butcher tableaux (App. A, Sec. 2, Sec. 4.1)."""
import json
import os

import numpy as np
import pytest

from oracle import tableaux as T

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "butcher_tableaux.json")))


@pytest.mark.parametrize("s", [1, 2, 3])
def test_collocation_radau_equals_printed(s):
    """RadauIIA built by collocation reproduces the tableaux printed in App. A."""
    g = GOLDEN[f"RadauIIA({s})"]
    t = T.radau_iia(s)
    assert np.allclose(t.A, g["A"], rtol=0, atol=2e-16)
    assert np.allclose(t.b, g["b"], rtol=0, atol=2e-16)
    assert np.allclose(t.c, g["c"], rtol=0, atol=2e-16)
    p = T.radau_iia_printed(s)
    assert np.allclose(p.A, g["A"], rtol=0, atol=2e-16)


@pytest.mark.parametrize("s", [1, 2, 3, 4, 5])
def test_radau_order_and_stage_order(s):
    """Order 2s-1 and stage order s (Sec. 4.1): B(2s-1), C(s) hold, B(2s), C(s+1) fail."""
    t = T.radau_iia(s)
    assert np.abs(t.A.sum(1) - t.c).max() < 1e-15
    assert abs(t.b.sum() - 1) < 1e-15
    assert np.abs(T.order_residuals_B(t, 2 * s - 1)).max() < 1e-14
    assert abs(T.order_residuals_B(t, 2 * s)[-1]) > 1e-6
    assert np.abs(T.order_residuals_C(t, s)).max() < 1e-14
    assert T.order_residuals_C(t, s + 1)[-1] > 1e-6
    # stiffly accurate: last row of A equals b, c_s = 1
    assert np.abs(t.A[-1] - t.b).max() < 1e-15 and t.c[-1] == 1.0


@pytest.mark.parametrize("s", [1, 2, 3, 4])
def test_gauss_legendre_order(s):
    t = T.gauss_legendre(s)
    assert np.abs(T.order_residuals_B(t, 2 * s)).max() < 1e-14
    assert abs(T.order_residuals_B(t, 2 * s + 1)[-1]) > 1e-6
    assert np.abs(T.order_residuals_C(t, s)).max() < 1e-14
    assert np.abs(t.c + t.c[::-1] - 1).max() < 1e-15  # symmetric abscissae


def stability_function(t, z):
    s = t.s
    return 1 + z * t.b @ np.linalg.solve(np.eye(s) - z * t.A, np.ones(s))


@pytest.mark.parametrize("z", [-0.3, -2.0, -17.5, 1.3 + 0.7j])
def test_stability_functions_are_pade(z):
    """Textbook closed forms: RadauIIA(1) 1/(1-z); RadauIIA(2) (1+z/3)/(1-2z/3+z^2/6);
    GL(2) (1+z/2+z^2/12)/(1-z/2+z^2/12)."""
    assert np.isclose(stability_function(T.radau_iia(1), z), 1 / (1 - z), rtol=1e-14)
    assert np.isclose(stability_function(T.radau_iia(2), z), (1 + z / 3) / (1 - 2 * z / 3 + z * z / 6), rtol=1e-14)
    gl = (1 + z / 2 + z * z / 12) / (1 - z / 2 + z * z / 12)
    assert np.isclose(stability_function(T.gauss_legendre(2), z), gl, rtol=1e-14)


def test_alexander_reading():
    """The z entry reading makes the method consistent, order 3 and L-stable (R(inf) = 0)."""
    t = T.alexander()
    x = t.A[0, 0]
    assert 1 / 6 < x < 1 / 2 and abs(x**3 - 3 * x**2 + 1.5 * x - 1 / 6) < 1e-15
    assert np.abs(t.A.sum(1) - t.c).max() < 1e-15
    assert np.abs(T.order_residuals_B(t, 3)).max() < 1e-15
    assert abs(t.b @ t.A @ t.c - 1 / 6) < 1e-15  # the remaining third-order condition
    r_inf = 1 - t.b @ np.linalg.solve(t.A, np.ones(3))
    assert abs(r_inf) < 1e-14


def test_wsodirk433_reading():
    t = T.wsodirk433()
    g = GOLDEN["WSODIRK433"]
    assert np.array_equal(t.A, np.array(g["A"])) and np.array_equal(t.c, np.array(g["c"]))
    assert np.abs(t.A.sum(1) - t.c).max() < 2e-8
    assert np.abs(T.order_residuals_B(t, 3)).max() < 2e-8
    assert abs(t.b @ t.A @ t.c - 1 / 6) < 1e-7


def test_lobatto_iiic2_printed():
    t = T.lobatto_iiic2()
    g = GOLDEN["LobattoIIIC(2)"]
    assert np.array_equal(t.A, np.array(g["A"]))
    assert np.abs(T.order_residuals_B(t, 2)).max() == 0 and np.abs(t.A.sum(1) - t.c).max() == 0
