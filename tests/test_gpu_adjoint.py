"""GPU parity of the adjoint kernel, the autograd bridge and the diagonal kernel.

Loss 0.5 ||H(lambda, kappa) u - f||^2 with lambda(x) = 1 + 0.5 sin(pi x),
kappa(x) = 1 + 0.3 cos(pi y) at the quadrature points (the differentiation
workload: 16^3 curved hexes, P = 6, Q = 8, FP64), u and f uniform[-1, 1).
Gradients are checked against the oracle's FP64 adjoint element by element
(1e-12) and against central differences of the GPU loss (h = 1e-6).
"""
import numpy as np
import pytest
import torch

import paper_1906_03489_gb300 as spx
from oracle import adjoint, operators
from paper_1906_03489_gb300 import synth

from _cases import Case, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def fields(c):
    xq = c.g["xq"].reshape(c.dim, -1) if c.plan.dim == 3 else None
    # xq layout: per element [dim][Q^d]; rebuild per-point x, y from blocks
    nq = c.plan.n_quad
    x = torch.empty(nq, dtype=torch.float64, device="cuda")
    y = torch.empty(nq, dtype=torch.float64, device="cuda")
    X = c.g["xq"]
    qo = c.plan.quad_off
    for e in range(c.plan.E):
        n = qo[e + 1] - qo[e]
        b = c.dim * qo[e]
        x[qo[e]:qo[e + 1]] = X[b:b + n]
        y[qo[e]:qo[e + 1]] = X[b + n:b + 2 * n]
    del xq
    lam = 1.0 + 0.5 * torch.sin(np.pi * x)
    kap = 1.0 + 0.3 * torch.cos(np.pi * y)
    return lam.contiguous(), kap.contiguous()


def fields_fast(c):
    """Same as fields() for uniform order, vectorised."""
    Q = c.plan.orders[0] + 2
    nq = Q ** c.dim
    X = c.g["xq"].reshape(c.plan.E, c.dim, nq)
    lam = 1.0 + 0.5 * torch.sin(np.pi * X[:, 0])
    kap = 1.0 + 0.3 * torch.cos(np.pi * X[:, 1])
    return lam.reshape(-1).contiguous(), kap.reshape(-1).contiguous()


@pytest.mark.parametrize("dim,N,P", [(3, 3, 3), (2, 4, 5), (3, 2, 6)])
def test_adjoint_matches_oracle(dim, N, P):
    c = Case(dim, N, P=P, amp=0.05)
    u, ut = c.coef(21)
    f, ftt = c.coef(22)
    lam, kap = fields_fast(c)
    _, gu, gl, gk = adjoint.gradients(c.om, u, f, lam.cpu().numpy(), kap.cpu().numpy())
    r = spx.helmholtz(c.plan, ut, lam_field=lam, kappa_field=kap) - ftt
    gl_gpu, gk_gpu = spx.helmholtz_adjoint(c.plan, ut, r)
    assert rel_err(gl_gpu, gl) <= 1e-12
    assert rel_err(gk_gpu, gk) <= 1e-12
    assert rel_err(spx.helmholtz(c.plan, r, lam_field=lam, kappa_field=kap), gu) <= 1e-12


def test_autograd_full_workload():
    """16^3 curved hexes, P = 6, Q = 8: autograd vs oracle adjoint and finite differences."""
    w = synth.WORKLOADS["hex3d_16_p6"]
    c = Case(3, w["N"], P=w["P"], amp=w["amp"])
    gen = synth.rng(w["seed"])
    u_np = synth.uniform(gen, c.plan.n_coef)
    f_np = synth.uniform(gen, c.plan.n_coef)
    lam, kap = fields_fast(c)
    u = torch.tensor(u_np, device="cuda", requires_grad=True)
    f = torch.tensor(f_np, device="cuda")
    lam_p = lam.clone().requires_grad_(True)
    kap_p = kap.clone().requires_grad_(True)
    y = spx.helmholtz_ad(c.plan, u, lam_p, kap_p)
    loss = 0.5 * ((y - f) ** 2).sum()
    loss.backward()
    L0, gu, gl, gk = adjoint.gradients(c.om, u_np, f_np, lam.cpu().numpy(), kap.cpu().numpy())
    assert abs(loss.item() - L0) <= 1e-12 * abs(L0)
    assert rel_err(u.grad, gu) <= 1e-12
    assert rel_err(lam_p.grad, gl) <= 1e-12
    assert rel_err(kap_p.grad, gk) <= 1e-12

    def gpu_loss(uu, ll, kk):
        return 0.5 * ((spx.helmholtz(c.plan, uu, lam_field=ll, kappa_field=kk) - f) ** 2).sum().item()

    h = 1e-6
    rng = np.random.default_rng(0)
    ud, ld, kd = u.detach(), lam.detach(), kap.detach()
    for idx in rng.choice(c.plan.n_coef, 4, replace=False):
        e = torch.zeros_like(ud)
        e[idx] = h
        fd = (gpu_loss(ud + e, ld, kd) - gpu_loss(ud - e, ld, kd)) / (2 * h)
        assert abs(fd - u.grad[idx].item()) <= 1e-6 * max(1.0, abs(fd)) + 1e-9 * abs(L0)
    for idx in rng.choice(c.plan.n_quad, 4, replace=False):
        e = torch.zeros_like(ld)
        e[idx] = h
        fd = (gpu_loss(ud, ld + e, kd) - gpu_loss(ud, ld - e, kd)) / (2 * h)
        assert abs(fd - lam_p.grad[idx].item()) <= 1e-5 * max(1.0, abs(fd)) + 1e-9 * abs(L0)
        fd = (gpu_loss(ud, ld, kd + e) - gpu_loss(ud, ld, kd - e)) / (2 * h)
        assert abs(fd - kap_p.grad[idx].item()) <= 1e-5 * max(1.0, abs(fd)) + 1e-9 * abs(L0)


def test_adjoint_variable_order():
    orders = synth.orders(synth.rng(23), 27, 2, 6)
    c = Case(3, 3, orders=orders, amp=0.05)
    u, ut = c.coef(24)
    g, gt = c.coef(25)
    lam, kap = fields(c)
    gl_gpu, gk_gpu = spx.helmholtz_adjoint(c.plan, ut, gt)
    # the adjoint with r = g: oracle gradients for f chosen so that H u - f = g
    Hu = operators.helmholtz(c.om, u, lam_field=lam.cpu().numpy(), kappa_field=kap.cpu().numpy())
    _, _, gl, gk = adjoint.gradients(c.om, u, Hu - g, lam.cpu().numpy(), kap.cpu().numpy())
    assert rel_err(gl_gpu, gl) <= 1e-12
    assert rel_err(gk_gpu, gk) <= 1e-12


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("dim,N,P", [(3, 2, 3), (2, 3, 4), (3, 2, 5)])
def test_diagonal(dim, N, P, dtype):
    c = Case(dim, N, P=P, amp=0.05)
    geo = c.om.geometry(P, P + 2, np.arange(c.om.E))
    ref = np.concatenate([np.diag(operators.helmholtz_matrix(dim, P, P + 2, geo, t, lam=1.3))
                          for t in range(c.om.E)])
    d = spx.helmholtz_diag(c.plan, dtype, lam=1.3)
    assert rel_err(d, ref) <= (1e-12 if dtype == torch.float64 else 1e-5)


def test_gather_and_assemble():
    from paper_1906_03489_gb300 import mesh
    c = Case(3, 3, P=3, amp=0.05)
    l2g, ng = mesh.periodic_l2g(3, 3, 3)
    xg = torch.tensor(synth.uniform(synth.rng(26), ng), device="cuda")
    loc = spx.gather(c.plan, l2g, xg)
    assert torch.equal(loc, xg[l2g.long()])
    yl = torch.tensor(synth.uniform(synth.rng(27), c.plan.n_coef), device="cuda")
    yg = spx.assemble(c.plan, l2g, yl, ng)
    ref = torch.zeros(ng, dtype=torch.float64, device="cuda").index_add_(0, l2g.long(), yl)
    assert rel_err(yg, ref.cpu().numpy()) <= 1e-15
    # an out-of-range index is skipped and reported, never read
    bad = l2g.clone()
    bad[5] = ng + 7
    loc = spx.gather(c.plan, bad, xg)
    assert loc[5].item() == 0.0
    assert c.plan.device_status() & 2
    assert c.plan.device_status() == 0
