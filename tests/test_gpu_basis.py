"""GPU parity with caller-supplied basis tables (spx_basis_desc) against the FP64 oracle.

* A permuted, sign-flipped modified basis (the vertex modes first, as some
  codes order them; generic kernels): if the caller's B' = B T1, the modal
  coefficients are u = T u' with T = T1 (x) T1 (x) T1, so H' = T^T H T; the
  oracle's H is applied to T u' and the result mapped by T^T.
* A rescaled modified basis B' = B diag(c) keeps the modified basis's parity
  (even-odd kernels, fed with the caller's numbers).
* The GLL nodal basis of §2.1 (oracle/nodal.py): on Q = P + 1 points it is
  the collocation basis B = I (collocation kernel, no B contractions); on
  Q = P + 2 points a general basis.
Tolerances: 1e-12 (FP64), 1e-5 (FP32), relative to the output's largest
entry, as for the library's own basis.
"""
import numpy as np
import pytest
import torch

import paper_1906_03489_gb300 as spx
from oracle import adjoint, basis, nodal, operators
from paper_1906_03489_gb300 import mesh, synth

from _cases import Case, rel_err

pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-12, torch.float32: 1e-5}
DTYPES = [torch.float64, torch.float32]


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def perm_matrix(P):
    """T1 with B' = B T1: new mode 0 = vertex 0, new mode 1 = vertex P, then the
    bubbles 1..P-1 in reverse order with alternating signs."""
    n = P + 1
    src = [0, P] + list(range(P - 1, 0, -1))
    T1 = np.zeros((n, n))
    for new, old in enumerate(src):
        T1[old, new] = -1.0 if (new >= 2 and new % 2) else 1.0
    return T1


def apply_axes(M, coef, off, n, dim):
    """Applies the n x n matrix M along every axis of each element's mode tensor."""
    out = np.empty_like(coef)
    for e in range(len(off) - 1):
        U = coef[off[e]: off[e + 1]].reshape((n,) * dim)      # [r][q][p] / [q][p], p fastest
        if dim == 3:
            U = np.einsum("ip,rqp->rqi", M, U)
            U = np.einsum("jq,rqi->rji", M, U)
            U = np.einsum("kr,rji->kji", M, U)
        else:
            U = np.einsum("ip,qp->qi", M, U)
            U = np.einsum("jq,qi->ji", M, U)
        out[off[e]: off[e + 1]] = U.reshape(-1)
    return out


def custom(P, Q, T1):
    t = spx.basis_tables(P, Q)
    return {"B": t["B"] @ T1, "dB": t["dB"] @ T1}


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("dim,N,P", [(3, 3, 4), (3, 3, 3), (3, 2, 6), (2, 5, 4)])
def test_permuted_modified_basis(dim, N, P, dtype):
    T1 = perm_matrix(P)
    c = Case(dim, N, P, basis={P: custom(P, P + 2, T1)})
    off = c.om.coef_off
    up, upt = c.coef(21, dtype)
    u = apply_axes(T1, up, off, P + 1, dim)                          # modal coefficients of the same function
    ref = apply_axes(T1.T, operators.helmholtz(c.om, u), off, P + 1, dim)
    assert rel_err(spx.helmholtz(c.plan, upt), ref) <= TOL[dtype]
    lam = 1.0 + 0.5 * synth.uniform(synth.rng(22), c.plan.n_quad)
    kap = 1.0 + 0.3 * synth.uniform(synth.rng(23), c.plan.n_quad)
    reff = apply_axes(T1.T, operators.helmholtz(c.om, u, lam_field=lam, kappa_field=kap), off, P + 1, dim)
    got = spx.helmholtz(c.plan, upt, lam_field=torch.tensor(lam, device="cuda", dtype=dtype),
                        kappa_field=torch.tensor(kap, device="cuda", dtype=dtype))
    assert rel_err(got, reff) <= TOL[dtype]
    # BwdTrans and IProduct of the same basis
    assert rel_err(spx.bwd_trans(c.plan, upt), operators.bwd_trans(c.om, u)) <= TOL[dtype]
    f, ft = c.quad(24, dtype)
    assert rel_err(spx.iproduct(c.plan, ft), apply_axes(T1.T, operators.iproduct(c.om, f), off, P + 1, dim)) \
        <= TOL[dtype]


@pytest.mark.parametrize("dim,N,P", [(3, 3, 3), (2, 4, 4)])
def test_permuted_basis_adjoint_fwdtrans_diag(dim, N, P):
    T1 = perm_matrix(P)
    c = Case(dim, N, P, basis={P: custom(P, P + 2, T1)})
    off, n = c.om.coef_off, P + 1
    up, upt = c.coef(25)
    gp, gpt = c.coef(26)
    u, g = apply_axes(T1, up, off, n, dim), apply_axes(T1, gp, off, n, dim)
    lam = 1.0 + 0.5 * synth.uniform(synth.rng(27), c.plan.n_quad)
    kap = 1.0 + 0.3 * synth.uniform(synth.rng(28), c.plan.n_quad)
    # with f = H u - g the oracle's residual is r = g: its gradients wrt lambda, kappa use (u, g)
    f = operators.helmholtz(c.om, u, lam_field=lam, kappa_field=kap) - g
    _, _, gl_ref, gk_ref = adjoint.gradients(c.om, u, f, lam, kap)
    gl, gk = spx.helmholtz_adjoint(c.plan, upt, gpt)
    assert rel_err(gl, gl_ref) <= 1e-12 and rel_err(gk, gk_ref) <= 1e-12
    # FwdTrans reproduces an expansion of the basis: BwdTrans(FwdTrans(BwdTrans u')) = BwdTrans u'
    fq = spx.bwd_trans(c.plan, upt)
    back = spx.bwd_trans(c.plan, spx.fwd_trans(c.plan, fq))
    assert rel_err(back, fq.cpu().numpy()) <= 1e-12
    # Jacobi diagonal of H' = T^T H T: diag = sum_kl T_kl^2 ... taken from the dense matrices
    d = spx.helmholtz_diag(c.plan).cpu().numpy()
    T = T1
    for P_, Q_, ids in c.om.groups():
        geo = c.om.geometry(P_, Q_, ids)
        Tt = np.kron(np.kron(T, T), T) if dim == 3 else np.kron(T, T)
        for t, e in enumerate(ids[:5]):
            H = operators.helmholtz_matrix(dim, P_, Q_, geo, t)
            ref = np.diag(Tt.T @ H @ Tt)
            assert rel_err(d[off[e]: off[e + 1]], ref) <= 1e-12


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("orders", [None, "var"])
def test_rescaled_modified_basis_keeps_parity_kernels(orders, dtype):
    rng = np.random.default_rng(5)
    if orders is None:
        P, ords = 4, None
        scales = {4: rng.uniform(0.5, 2.0, 5)}
    else:
        ords = synth.orders(synth.rng(31), 4 ** 3, 2, 8)
        scales = {p: rng.uniform(0.5, 2.0, p + 1) for p in range(2, 9)}
        P = None
    present = sorted(set([4] if ords is None else ords.tolist()))
    bas = {p: custom(p, p + 2, np.diag(scales[p])) for p in present}
    c = Case(3, 4, P, orders=ords, basis=bas)
    up, upt = c.coef(32, dtype)
    u = up.copy()
    ref = np.zeros_like(up)
    off = c.om.coef_off
    # per element: u = diag-scaled coefficients; H' = S H S
    Pe = c.om.P
    for e in range(c.om.E):
        n = Pe[e] + 1
        S = np.diag(scales[int(Pe[e])])
        sl = slice(off[e], off[e + 1])
        u[sl] = apply_axes(S, up[sl], np.array([0, n ** 3]), n, 3)
    y = operators.helmholtz(c.om, u)
    for e in range(c.om.E):
        n = Pe[e] + 1
        S = np.diag(scales[int(Pe[e])])
        sl = slice(off[e], off[e + 1])
        ref[sl] = apply_axes(S, y[sl], np.array([0, n ** 3]), n, 3)
    assert rel_err(spx.helmholtz(c.plan, upt), ref) <= TOL[dtype]


def nodal_basis(present, qoff):
    return {p: spx.nodal_basis_tables(p, p + qoff) for p in present}


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("dim,N,P,qoff", [(3, 3, 4, 1), (3, 3, 2, 1), (3, 2, 6, 1), (3, 2, 8, 1), (3, 3, 1, 1),
                                          (3, 2, 3, 2), (3, 2, 5, 2), (2, 5, 4, 1), (2, 4, 3, 2)])
def test_nodal_basis_helmholtz(dim, N, P, qoff, dtype):
    c = Case(dim, N, P, q_offset=qoff, basis=nodal_basis([P], qoff))
    u, ut = c.coef(41, dtype)
    assert rel_err(spx.helmholtz(c.plan, ut), nodal.helmholtz(c.om, u)) <= TOL[dtype]
    lam = 1.0 + 0.5 * synth.uniform(synth.rng(42), c.plan.n_quad)
    kap = 1.0 + 0.3 * synth.uniform(synth.rng(43), c.plan.n_quad)
    got = spx.helmholtz(c.plan, ut, lam_field=torch.tensor(lam, device="cuda", dtype=dtype),
                        kappa_field=torch.tensor(kap, device="cuda", dtype=dtype))
    assert rel_err(got, nodal.helmholtz(c.om, u, lam_field=lam, kappa_field=kap)) <= TOL[dtype]
    assert rel_err(spx.bwd_trans(c.plan, ut), nodal.bwd_trans(c.om, u)) <= TOL[dtype]
    f, ft = c.quad(44, dtype)
    assert rel_err(spx.iproduct(c.plan, ft), nodal.iproduct(c.om, f)) <= TOL[dtype]
    if qoff == 1:   # collocation: BwdTrans is the identity
        assert rel_err(spx.bwd_trans(c.plan, ut), u) <= TOL[dtype]


@pytest.mark.parametrize("dtype", DTYPES)
def test_nodal_basis_variable_order(dtype):
    ords = synth.orders(synth.rng(45), 4 ** 3, 1, 8)
    c = Case(3, 4, orders=ords, q_offset=1, basis=nodal_basis(sorted(set(ords.tolist())), 1))
    u, ut = c.coef(46, dtype)
    assert rel_err(spx.helmholtz(c.plan, ut), nodal.helmholtz(c.om, u)) <= TOL[dtype]


@pytest.mark.parametrize("dtype", DTYPES)
def test_nodal_collocation_full_workload_sampled(dtype):
    """32^3 curved hexes, P = 4, Q = 5 (collocation), autotuned tile; sampled elements vs the oracle."""
    from oracle import geometry
    N, P = 32, 4
    plan = spx.Plan(3, N ** 3, order=P, q_offset=1, basis=nodal_basis([P], 1))
    g = spx.geom_factors(plan, mesh.structured_nodes(3, N, P, 0.05))
    plan.set_geometry(torch.float64, g["geom"], g["dxi"])
    plan.set_geometry(torch.float32, g["geom32"], g["dxi32"])
    u = synth.uniform(synth.rng(2), plan.n_coef)
    ut = torch.tensor(u, device="cuda", dtype=dtype)
    y = torch.empty_like(ut)
    plan.autotune("helmholtz", dtype, ut, y, reps=2)
    y = spx.helmholtz(plan, ut).cpu().double().numpy()
    om = geometry.StructuredMesh(3, N, P, amp=0.05, nq=P + 1)
    ids = np.concatenate([[0, plan.E - 1], np.sort(np.random.default_rng(0).choice(plan.E, 40, replace=False))])
    geo = om.geometry(P, P + 1, ids)
    n = (P + 1) ** 3
    ref = np.concatenate([nodal.helmholtz_matrix(3, P, P + 1, geo, t) @ u[e * n:(e + 1) * n] for t, e in enumerate(ids)])
    got = np.concatenate([y[e * n:(e + 1) * n] for e in ids])
    assert rel_err(got, ref) <= TOL[dtype]


def test_device_memory_basis_tables_match_host():
    P = 3
    T1 = perm_matrix(P)
    host = custom(P, P + 2, T1)
    dev = {k: torch.tensor(v, device="cuda") for k, v in host.items()}
    a = Case(3, 2, P, basis={P: host})
    b = Case(3, 2, P, basis={P: dev})
    u, ut = a.coef(51)
    assert torch.equal(spx.helmholtz(a.plan, ut), spx.helmholtz(b.plan, ut))


def test_sensor_needs_the_modified_basis():
    P = 3
    c = Case(3, 2, P, basis={P: custom(P, P + 2, perm_matrix(P))})
    u, ut = c.coef(52)
    with pytest.raises(spx.SpxError) as ei:
        spx.sensor(c.plan, ut)
    assert "modified basis" in str(ei.value)


def test_nodal_periodic_solve_matches_dense_solve():
    """The assembled nodal (collocation) system on a 2^3 periodic mesh: CG vs a dense solve."""
    N, P = 2, 3
    c = Case(3, N, P, q_offset=1, basis=nodal_basis([P], 1))
    l2g, ng = mesh.periodic_l2g(3, N, P)
    l2g_np = l2g.cpu().numpy()
    n = (P + 1) ** 3
    A = np.zeros((ng, ng))
    geo = c.om.geometry(P, P + 1, np.arange(c.om.E))
    for e in range(c.om.E):
        H = nodal.helmholtz_matrix(3, P, P + 1, geo, e)
        idx = l2g_np[e * n:(e + 1) * n]
        A[np.ix_(idx, idx)] += H
    f = synth.uniform(synth.rng(53), ng)
    x_ref = np.linalg.solve(A, f)
    # x is fixed by the residual criterion only up to cond(A) x tol; cond(A) of
    # this 216-DOF system is below 1e3 (checked here), so 1e-8 holds at tol 1e-11
    ev = np.linalg.eigvalsh(A)
    assert ev.max() / ev.min() < 1e3
    for prec in ("f64", "f32_reliable"):
        x, info = spx.cg_solve(c.plan, 1.0, l2g, ng, torch.tensor(f, device="cuda"), tol=1e-11, precision=prec)
        assert info["status"] == 0
        assert rel_err(x, x_ref) <= 1e-8
