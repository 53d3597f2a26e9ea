"""Pins of the oracle's adaptive-order sensor (§4.2) against closed forms and invariants."""
from math import factorial

import numpy as np
import pytest

from oracle import adapt, operators
from oracle.geometry import StructuredMesh


def _values_on_points(mesh, fn):
    """fn(reference coordinates xi of shape (n_points, d)) on every element, in buffer order."""
    _, _, xq = mesh.factors_flat()
    d = mesh.dim
    out = np.zeros(mesh.quad_off[-1])
    X = xq.reshape(-1)
    for e in range(mesh.E):
        q0, q1 = mesh.quad_off[e], mesh.quad_off[e + 1]
        nq = q1 - q0
        pts = np.stack([X[d * q0 + a * nq: d * q0 + (a + 1) * nq] for a in range(d)], axis=1)
        out[q0:q1] = fn(pts)
    return out


@pytest.mark.parametrize("dim,P", [(2, 2), (2, 5), (3, 3), (3, 4), (3, 6)])
def test_sensor_of_monomial_is_inverse_squared_leading_coefficient(dim, P):
    """u = xi_1^P on one affine element: its L2 projection error onto degree P-1 is the
    monic Legendre polynomial, so S = ||L_P / k_P||^2 / ||xi^P||^2 = 1 / k_P^2 with
    k_P = (2P)! / (2^P (P!)^2), both norms being 2 / (2P + 1) times the same factors."""
    mesh = StructuredMesh(dim, 1, P, amp=0.0, origin=-1.0, length=2.0)     # reference coordinates = x
    f = _values_on_points(mesh, lambda x: x[:, 0] ** P)
    u = operators.fwd_trans(mesh, f)                                       # exact: xi^P is in the space
    k = factorial(2 * P) / (2 ** P * factorial(P) ** 2)
    np.testing.assert_allclose(adapt.sensor(mesh, u), 1.0 / k ** 2, rtol=1e-9)


@pytest.mark.parametrize("dim,N,P,amp", [(3, 2, 4, 0.05), (2, 3, 3, 0.0), (3, 2, 2, 0.05)])
def test_sensor_vanishes_on_order_p_minus_1(dim, N, P, amp):
    """Modes of order P whose indices avoid the degree-P bubble (index P-1) in every
    direction span the degree <= P-1 space: the sensor is zero there."""
    mesh = StructuredMesh(dim, N, P, amp=amp)
    rng = np.random.default_rng(7)
    n = P + 1
    u = rng.uniform(-1, 1, mesh.coef_off[-1])
    idx = np.arange(n ** dim)
    digits = [(idx // n ** a) % n for a in range(dim)]
    top = np.any([dg == P - 1 for dg in digits], axis=0)
    for e in range(mesh.E):
        u[mesh.coef_off[e]: mesh.coef_off[e + 1]][top] = 0.0
    assert adapt.sensor(mesh, u).max() < 1e-20


def test_sensor_range_scale_and_variable_order():
    rng = np.random.default_rng(8)
    orders = rng.integers(2, 7, size=8)
    mesh = StructuredMesh(3, 2, orders, amp=0.05)
    u = rng.uniform(-1, 1, mesh.coef_off[-1])
    S = adapt.sensor(mesh, u)
    assert np.all(S > 0) and np.all(S < 1)
    np.testing.assert_allclose(adapt.sensor(mesh, 3.0 * u), S, rtol=1e-12)
    # each element alone gives the same value (no coupling between elements)
    for e in range(mesh.E):
        one = StructuredMesh(3, 2, int(orders[e]), amp=0.05)
        ue = np.zeros(one.coef_off[-1])
        ue[one.coef_off[e]: one.coef_off[e + 1]] = u[mesh.coef_off[e]: mesh.coef_off[e + 1]]
        Se = adapt.sensor(one, ue + 0.0)
        np.testing.assert_allclose(Se[e], S[e], rtol=1e-12)


def test_sensor_of_constant_is_zero_and_of_top_bubble_is_positive():
    mesh = StructuredMesh(3, 1, 3, amp=0.0)
    ones = operators.fwd_trans(mesh, np.ones(mesh.quad_off[-1]))
    assert adapt.sensor(mesh, ones)[0] < 1e-24
    u = np.zeros(mesh.coef_off[-1])
    u[2 + 4 * (2 + 4 * 2)] = 1.0      # the degree-3 bubble in every direction
    assert adapt.sensor(mesh, u)[0] > 0.5


def test_adapt_orders():
    S = np.array([1e-1, 1e-9, 1e-5, 1e-1, 1e-12])
    P = np.array([4, 4, 4, 8, 2])
    np.testing.assert_array_equal(adapt.adapt_orders(S, P, 1e-8, 1e-3, 2, 8), [5, 3, 4, 8, 2])
