"""GPU parity of the adaptive-order error sensor and order update (§4.2) against the oracle.

The GPU projects u_P onto the order-P modes that avoid the degree-P bubble
(preconditioned CG per element); the oracle projects onto the order P-1
modified basis itself (dense solve).  Both give the same S_e; agreement is
checked to 1e-9 relative (the projection's coefficients are ill-conditioned,
S_e itself is not: its error is about sqrt(cond(M_e)) 2^-52 / sqrt(S_e)).
"""
from math import factorial

import numpy as np
import pytest
import torch

import paper_1906_03489_gb300 as spx
from oracle import adapt, operators
from paper_1906_03489_gb300 import mesh, synth

from _cases import Case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("dim,N,P,amp", [(3, 3, 4, 0.05), (3, 2, 8, 0.05), (3, 3, 2, 0.05), (3, 2, 6, 0.05),
                                         (2, 5, 4, 0.05), (2, 3, 8, 0.0)])
def test_sensor_matches_oracle(dim, N, P, amp):
    c = Case(dim, N, P=P, amp=amp)
    u, ut = c.coef(21)
    S = spx.sensor(c.plan, ut).cpu().numpy()
    ref = adapt.sensor(c.om, u)
    np.testing.assert_allclose(S, ref, rtol=1e-9, atol=1e-15)
    assert c.plan.device_status() == 0


def test_sensor_variable_order_and_adapt():
    gen = synth.rng(22)
    orders = synth.orders(gen, 27, 2, 8)
    c = Case(3, 3, orders=orders, amp=0.05)
    u, ut = c.coef(23)
    # a smooth field for part of the elements: scale the top modes down so the sensor spreads out
    S = spx.sensor(c.plan, ut).cpu().numpy()
    ref = adapt.sensor(c.om, u)
    np.testing.assert_allclose(S, ref, rtol=1e-9, atol=1e-15)
    lower, upper = np.quantile(S, 0.3), np.quantile(S, 0.7)
    new = spx.adapt_orders(S, orders, lower, upper, 2, 8)
    np.testing.assert_array_equal(new, adapt.adapt_orders(ref, orders, lower, upper, 2, 8))
    assert np.any(new != orders)
    # the new orders feed the next variable-order plan: Helmholtz on it matches the oracle
    c2 = Case(3, 3, orders=new, amp=0.05)
    v, vt = c2.coef(24)
    y = spx.helmholtz(c2.plan, vt).cpu().numpy()
    ref2 = operators.helmholtz(c2.om, v)
    assert np.abs(y - ref2).max() <= 1e-12 * np.abs(ref2).max()


@pytest.mark.parametrize("dim,P", [(3, 3), (3, 5), (2, 6)])
def test_sensor_of_monomial(dim, P):
    """u = xi_1^P on the reference element: S = 1 / k_P^2, k_P = (2P)! / (2^P (P!)^2)."""
    plan = spx.Plan(dim, 1, order=P)
    g = spx.geom_factors(plan, mesh.structured_nodes(dim, 1, P, 0.0, origin=-1.0, length=2.0))
    plan.set_geometry(torch.float64, g["geom"], g["dxi"])
    x = g["xq"].reshape(dim, -1)[0]
    u = spx.fwd_trans(plan, (x ** P).contiguous())
    k = factorial(2 * P) / (2 ** P * factorial(P) ** 2)
    assert abs(float(spx.sensor(plan, u)[0]) - 1.0 / k ** 2) <= 1e-9 / k ** 2


def test_sensor_zero_on_lower_order_and_on_zero():
    c = Case(3, 2, P=5, amp=0.05)
    u, _ = c.coef(25)
    n = 6
    idx = np.arange(n ** 3)
    top = ((idx % n) == 4) | (((idx // n) % n) == 4) | ((idx // (n * n)) == 4)
    u = u.reshape(c.plan.E, -1)
    u[:, top] = 0.0
    S = spx.sensor(c.plan, torch.tensor(u.reshape(-1), device="cuda")).cpu().numpy()
    assert S.max() < 1e-20
    z = spx.sensor(c.plan, torch.zeros(c.plan.n_coef, dtype=torch.float64, device="cuda"))
    assert torch.count_nonzero(z) == 0


def test_sensor_rejects_order_one_and_fp32():
    c = Case(3, 2, P=1, amp=0.05)
    with pytest.raises(spx.SpxError):
        spx.sensor(c.plan, torch.zeros(c.plan.n_coef, dtype=torch.float64, device="cuda"))
    c = Case(3, 2, P=3, amp=0.05)
    with pytest.raises(TypeError):
        spx.sensor(c.plan, torch.zeros(c.plan.n_coef, dtype=torch.float32, device="cuda"))
