"""GPU parity of FwdTrans (Galerkin projection) and Integral against the FP64 oracle.

FwdTrans solves M_e c = IProduct(f)_e per element.  In the modified basis M_e
is ill-conditioned (cond ~ 4e7 at P = 4 in 3D, ~ 4e9 at P = 8), so the
coefficients of two correct FP64 solvers (the oracle's dense Cholesky, the
library's preconditioned CG) agree only to about cond(M_e) x 2^-52.  What the
method fixes exactly is checked tightly instead:
  * the residual ||M_e c - b|| / ||b|| of every element, with the oracle's
    dense M_e, <= 1e-13 (FP64);
  * the projected function BwdTrans(c): two solutions c1, c2 whose residuals
    are eps-small differ in the mass norm by
    ||Phi (c1 - c2)||_W^2 = (c1 - c2)^T M_e (c1 - c2) <= ||c1 - c2|| ||r1 - r2||
    ~ cond(M_e) eps^2 ||f||^2, i.e. by about sqrt(cond(M_e)) x 2^-52 relative:
    <= 100 sqrt(cond(M_e)) 2^-52 of the oracle's (FP64; 1.5e-10 at P = 4 in
    3D, measured constants 0.7 to 13); in FP32 the same argument gives
    100 sqrt(cond(M_e)) 2^-24 (4e-2 at P = 4, measured 5.5e-5): FP32 FwdTrans
    is only that accurate, cond(M_e) being beyond FP32's range;
  * the coefficients, within 100 x cond(M_e) x 2^-52 of the oracle's.
Integral: <= 1e-13 relative (FP64), 1e-6 (FP32), and the paper's worked
example (tests/golden/e1_integral.txt).
"""
import os

import numpy as np
import pytest
import torch

import paper_1906_03489_gb300 as spx
from oracle import operators
from paper_1906_03489_gb300 import mesh, synth

from _cases import Case, rel_err

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
EPS = 2.0 ** -52

# (dim, N, P, amp): ragged tiles, both dimensions, orders 1..8, Q = P+2
SHAPES = [(3, 3, 4, 0.05), (3, 2, 8, 0.05), (3, 3, 2, 0.05), (3, 2, 1, 0.05), (3, 2, 6, 0.05),
          (2, 7, 4, 0.05), (2, 4, 8, 0.0), (2, 3, 1, 0.0)]


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _cond(c):
    """Largest condition number of the elemental mass matrices (one element per order)."""
    om, d = c.om, c.dim
    k = 1.0
    for P, Q, ids in om.groups():
        k = max(k, np.linalg.cond(operators.mass_matrix(d, P, Q, om.geometry(P, Q, ids[:1]), 0)))
    return k


def _elem_checks(c, f, cg, tol_res):
    """Per-element residual with the oracle's dense mass matrix; max cond(M_e)."""
    om, d = c.om, c.dim
    b = operators.iproduct(om, f)
    kmax, rmax = 1.0, 0.0
    for P, Q, ids in om.groups():
        geo = om.geometry(P, Q, ids)
        n = (P + 1) ** d
        for t, e in enumerate(ids):
            M = operators.mass_matrix(d, P, Q, geo, t)
            s = slice(om.coef_off[e], om.coef_off[e] + n)
            be = b[s]
            r = np.linalg.norm(M @ cg[s] - be) / max(np.linalg.norm(be), 1e-300)
            rmax = max(rmax, r)
            if t == 0:
                kmax = max(kmax, np.linalg.cond(M))
    assert rmax <= tol_res, rmax
    return kmax


@pytest.mark.parametrize("dim,N,P,amp", SHAPES)
def test_fwd_trans_fp64(dim, N, P, amp):
    c = Case(dim, N, P=P, amp=amp)
    f, ft = c.quad(11)
    cg = spx.fwd_trans(c.plan, ft).cpu().numpy()
    ref = operators.fwd_trans(c.om, f)
    kappa = _elem_checks(c, f, cg, 1e-13)
    assert rel_err(cg, ref) <= 100 * kappa * EPS
    assert rel_err(operators.bwd_trans(c.om, cg), operators.bwd_trans(c.om, ref)) <= 100 * np.sqrt(kappa) * EPS
    assert c.plan.device_status() == 0


def test_fwd_trans_fp32_is_refused():
    """cond(M_e) exceeds FP32's 1/eps: an FP32 projection cannot meet the 1e-5 operator bar."""
    c = Case(3, 2, P=4, amp=0.05)
    f, ft = c.quad(12, torch.float32)
    out = torch.full((c.plan.n_coef,), 3.0, dtype=torch.float32, device="cuda")
    with pytest.raises(spx.SpxError, match="FP32 is refused"):
        spx.fwd_trans(c.plan, ft, out=out)
    assert bool((out == 3.0).all())
    assert _cond(c) > 2.0 ** 24


def test_fwd_trans_variable_order():
    gen = synth.rng(13)
    orders = synth.orders(gen, 27, 2, 8)
    c = Case(3, 3, orders=orders, amp=0.05)
    f, ft = c.quad(14)
    cg = spx.fwd_trans(c.plan, ft).cpu().numpy()
    ref = operators.fwd_trans(c.om, f)
    kappa = _elem_checks(c, f, cg, 1e-13)
    assert rel_err(cg, ref) <= 100 * kappa * EPS
    assert rel_err(operators.bwd_trans(c.om, cg), operators.bwd_trans(c.om, ref)) <= 100 * np.sqrt(kappa) * EPS


def test_fwd_trans_q_offset_one():
    """Q = P + 1 points (the mass matrix is no longer integrated exactly, but it is
    still SPD and the same projection is solved): parity with the oracle."""
    c = Case(3, 3, P=4, amp=0.05, q_offset=1)
    f, ft = c.quad(26)
    cg = spx.fwd_trans(c.plan, ft).cpu().numpy()
    ref = operators.fwd_trans(c.om, f)
    kappa = _elem_checks(c, f, cg, 1e-13)
    assert rel_err(cg, ref) <= 100 * kappa * EPS
    assert rel_err(operators.bwd_trans(c.om, cg), operators.bwd_trans(c.om, ref)) <= 100 * np.sqrt(kappa) * EPS


@pytest.mark.parametrize("dim,P", [(3, 4), (2, 6)])
def test_projection_reproduces_expansions(dim, P):
    """FwdTrans(BwdTrans(u)) = u: the projection of a function in the space is itself."""
    c = Case(dim, 3, P=P, amp=0.05)
    u, ut = c.coef(15)
    back = spx.fwd_trans(c.plan, spx.bwd_trans(c.plan, ut)).cpu().numpy()
    kappa = _elem_checks(c, operators.bwd_trans(c.om, u), back, 1e-13)
    assert rel_err(back, u) <= 100 * kappa * EPS


def test_fwd_trans_varying_jacobian_converges():
    """On a mesh whose det J varies inside each element (the tensor-product
    preconditioner is no longer exact) the projection still reproduces an
    expansion: FwdTrans(BwdTrans(u)) = u.  Nodes x' = x + 0.04 sin(pi x) (1 + y z)
    give det J = 1 + 0.04 pi cos(pi x) (1 + y z) over the unit cube."""
    dim, N, P = 3, 3, 4
    plan = spx.Plan(dim, N ** dim, order=P)
    nodes = mesh.structured_nodes(dim, N, P, 0.0).reshape(N ** dim, dim, -1)    # [E][x, y, z][node]
    x, y, z = nodes[:, 0].clone(), nodes[:, 1], nodes[:, 2]
    nodes[:, 0] = x + 0.04 * torch.sin(np.pi * x) * (1 + y * z)
    g = spx.geom_factors(plan, nodes.reshape(-1).contiguous())
    plan.set_geometry(torch.float64, g["geom"], g["dxi"])
    jw = g["geom"].reshape(plan.E, 7, -1)[:, 6]
    assert (jw.max(dim=1).values / jw.min(dim=1).values).max() > 1.02     # det J is not constant
    u = torch.tensor(synth.uniform(synth.rng(16), plan.n_coef), device="cuda")
    back = spx.fwd_trans(plan, spx.bwd_trans(plan, u))
    assert rel_err(back, u.cpu().numpy()) <= 1e-6
    # and the projection of the values is the values themselves: within
    # 10 sqrt(cond) 2^-52 (cond ~ 4.5e7 at P = 4), with a further factor 10 for
    # the stronger geometry
    fq = spx.bwd_trans(plan, u)
    assert rel_err(spx.bwd_trans(plan, back), fq.cpu().numpy()) <= 100 * np.sqrt(4.5e7) * EPS


def test_fwd_trans_zero_and_empty():
    c = Case(3, 2, P=3, amp=0.05)
    z = torch.zeros(c.plan.n_quad, dtype=torch.float64, device="cuda")
    assert torch.count_nonzero(spx.fwd_trans(c.plan, z)) == 0
    empty = spx.Plan(3, 0, order=3)
    spx.fwd_trans(empty, torch.zeros(1, dtype=torch.float64, device="cuda"),
                  out=torch.zeros(1, dtype=torch.float64, device="cuda"))


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-13), (torch.float32, 1e-6)])
@pytest.mark.parametrize("dim,N,P", [(3, 4, 4), (2, 9, 3), (3, 2, 8)])
def test_integral(dim, N, P, dtype, tol):
    c = Case(dim, N, P=P, amp=0.05)
    f, ft = c.quad(17, dtype)
    f = ft.double().cpu().numpy()
    ref = operators.integral(c.om, f)
    val = float(spx.integral(c.plan, ft))
    scale = operators.integral(c.om, np.abs(f))
    assert abs(val - ref) <= tol * scale
    # reproducible: the same sum twice
    assert float(spx.integral(c.plan, ft)) == val


def test_integral_variable_order_and_volume():
    gen = synth.rng(18)
    orders = synth.orders(gen, 64, 2, 8)
    c = Case(3, 4, orders=orders, amp=0.05)
    ones = torch.ones(c.plan.n_quad, dtype=torch.float64, device="cuda")
    assert abs(float(spx.integral(c.plan, ones)) - 1.0) <= 1e-13          # volume of the unit cube
    f, ft = c.quad(19)
    assert abs(float(spx.integral(c.plan, ft)) - operators.integral(c.om, f)) <= 1e-13 * np.abs(f).sum()


def test_paper_worked_example():
    """§3.5, Listing lst:python: project cos(x) cos(y) on [-1, 1]^2 (8 modes,
    9 GLL points), integrate; the exact value is 4 sin^2(1)."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "e1_integral.txt")) if not l.startswith("#")]
    n_modes, n_pts, exact = int(rows[0][0]), int(rows[0][1]), float(rows[0][3])
    P = n_modes - 1
    plan = spx.Plan(2, 1, order=P, q_offset=n_pts - P)
    g = spx.geom_factors(plan, mesh.structured_nodes(2, 1, P, 0.0, origin=-1.0, length=2.0))
    plan.set_geometry(torch.float64, g["geom"], g["dxi"])
    X = g["xq"].reshape(2, -1)
    f = (torch.cos(X[0]) * torch.cos(X[1])).contiguous()
    assert abs(float(spx.integral(plan, f)) - exact) < 1e-13
    proj = spx.fwd_trans(plan, f)
    assert abs(float(spx.integral(plan, spx.bwd_trans(plan, proj))) - exact) < 1e-12
    assert (spx.bwd_trans(plan, proj) - f).abs().max().item() < 1e-6
