"""GPU parity of the collapsed-coordinate elements (triangles, prisms, tetrahedra) against the FP64 oracle.

Affine elements of a skewed grid with a seeded jitter of every vertex (so
that no two elements share a Jacobian), orders 1..8 on ragged tiles, both
precisions: geometric factors (1e-12), BwdTrans, IProductWRTBase, PhysDeriv
and the Helmholtz operator with constant and per-point lambda, kappa
(1e-12 FP64, 1e-5 FP32, relative to the output's largest entry), and the
full prism workload on sampled elements.
"""
import numpy as np
import pytest
import torch

import paper_1906_03489_gb300 as spx
from oracle import collapsed as C
from paper_1906_03489_gb300 import mesh, synth

from _cases import rel_err

pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-12, torch.float32: 1e-5}
DTYPES = [torch.float64, torch.float32]


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def make(shape, N, P, seed=60, jit=0.02):
    d = 2 if shape == "tri" else 3
    E = (6 if shape == "tet" else 2) * N ** d
    jitter = jit / N * synth.uniform(synth.rng(seed), E * (d + 1) * d).reshape(E, d + 1, d)
    plan = spx.Plan(d, E, order=P, shape=shape)
    g = spx.geom_factors(plan, mesh.collapsed_vertices(shape, N, jitter))
    plan.set_geometry(torch.float64, g["geom"], g["dxi"])
    plan.set_geometry(torch.float32, g["geom32"], g["dxi32"])
    skew = synth.SKEW2 if shape == "tri" else synth.SKEW3
    V = C.kuhn_vertices(N, skew, jitter) if shape == "tet" else C.structured_vertices(shape, N, skew, jitter)
    om = C.CollapsedMesh(shape, V, P)
    return plan, g, om


CASES = [("tri", 3, 1), ("tri", 3, 2), ("tri", 3, 4), ("tri", 2, 6), ("tri", 2, 8),
         ("prism", 2, 1), ("prism", 2, 2), ("prism", 2, 4), ("prism", 2, 6), ("prism", 1, 8),
         ("tet", 1, 1), ("tet", 2, 2), ("tet", 2, 3), ("tet", 2, 4), ("tet", 1, 6), ("tet", 1, 8)]


@pytest.mark.parametrize("shape,N,P", CASES)
def test_geometry_factors(shape, N, P):
    plan, g, om = make(shape, N, P)
    d = om.d
    K = C.deta_dx(om)                                           # (E, nq, a, m)
    G = om.JW[:, :, None, None] * np.einsum("eqam,eqbm->eqab", K, K)
    pairs = [(0, 0), (0, 1), (1, 1)] if d == 2 else [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
    ref = np.concatenate([np.stack([G[:, :, a, b] for a, b in pairs] + [om.JW], 1)], 0).reshape(-1)
    assert rel_err(g["geom"], ref) <= 1e-12
    refd = np.transpose(K, (0, 2, 3, 1)).reshape(-1)          # block a d + m
    assert rel_err(g["dxi"], refd) <= 1e-12
    assert rel_err(g["xq"], np.transpose(om.xq(), (0, 2, 1)).reshape(-1)) <= 1e-13


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("shape,N,P", CASES)
def test_operators(shape, N, P, dtype):
    plan, g, om = make(shape, N, P)
    u = synth.uniform(synth.rng(61), plan.n_coef)
    f = synth.uniform(synth.rng(62), plan.n_quad)
    ut = torch.tensor(u, device="cuda", dtype=dtype)
    ft = torch.tensor(f, device="cuda", dtype=dtype)
    assert rel_err(spx.bwd_trans(plan, ut), C.bwd_trans(om, u)) <= TOL[dtype]
    assert rel_err(spx.iproduct(plan, ft), C.iproduct(om, f)) <= TOL[dtype]
    got = spx.phys_deriv(plan, ft)
    for m, ref in enumerate(C.phys_deriv(om, f)):
        assert rel_err(got[m], ref) <= TOL[dtype] * 10, m
    assert rel_err(spx.helmholtz(plan, ut), C.helmholtz(om, u)) <= TOL[dtype]
    lam = 1.0 + 0.5 * synth.uniform(synth.rng(63), plan.n_quad)
    kap = 1.0 + 0.3 * synth.uniform(synth.rng(64), plan.n_quad)
    y = spx.helmholtz(plan, ut, lam_field=torch.tensor(lam, device="cuda", dtype=dtype),
                      kappa_field=torch.tensor(kap, device="cuda", dtype=dtype))
    assert rel_err(y, C.helmholtz(om, u, lam_field=lam, kappa_field=kap)) <= TOL[dtype]
    assert plan.device_status() == 0


@pytest.mark.parametrize("shape,N,P", [("prism", 2, 4), ("tet", 2, 3), ("tri", 3, 4)])
@pytest.mark.parametrize("eb", [1, 3, 5, 8])
def test_fp32_element_pairs_any_tile(shape, N, P, eb):
    """FP32 kernels hold two elements per value (pair p = elements p and
    p + npair of a tile): odd tile sizes and ragged last tiles leave the last
    pair half empty, and every operator must still match the oracle."""
    plan, g, om = make(shape, N, P, seed=66)
    for op in ("bwd_trans", "iproduct", "phys_deriv", "helmholtz"):
        plan.set_tile(op, torch.float32, eb, 128, 2)
    u = synth.uniform(synth.rng(67), plan.n_coef)
    f = synth.uniform(synth.rng(68), plan.n_quad)
    ut = torch.tensor(u, device="cuda", dtype=torch.float32)
    ft = torch.tensor(f, device="cuda", dtype=torch.float32)
    assert rel_err(spx.bwd_trans(plan, ut), C.bwd_trans(om, u)) <= 1e-5
    assert rel_err(spx.iproduct(plan, ft), C.iproduct(om, f)) <= 1e-5
    got = spx.phys_deriv(plan, ft)
    for m, ref in enumerate(C.phys_deriv(om, f)):
        assert rel_err(got[m], ref) <= 1e-4, m
    assert rel_err(spx.helmholtz(plan, ut), C.helmholtz(om, u)) <= 1e-5
    assert plan.device_status() == 0


def test_autotuned_tiles_and_integral():
    plan, g, om = make("prism", 3, 3)
    u = torch.tensor(synth.uniform(synth.rng(65), plan.n_coef), device="cuda")
    y = torch.empty_like(u)
    plan.autotune("helmholtz", torch.float64, u, y, reps=1)
    assert rel_err(spx.helmholtz(plan, u), C.helmholtz(om, u.cpu().numpy())) <= 1e-12
    one = torch.ones(plan.n_quad, dtype=torch.float64, device="cuda")
    assert abs(float(spx.integral(plan, one)) - om.JW.sum()) <= 1e-13 * om.JW.sum()


def test_unsupported_operators_are_refused():
    plan, g, om = make("tri", 2, 3)
    u = torch.zeros(plan.n_coef, dtype=torch.float64, device="cuda")
    with pytest.raises(spx.SpxError, match="not available"):
        spx.fwd_trans(plan, torch.zeros(plan.n_quad, dtype=torch.float64, device="cuda"))
    with pytest.raises(spx.SpxError, match="not available"):
        spx.helmholtz_diag(plan)


@pytest.mark.parametrize("dtype", DTYPES)
def test_prism_full_workload_sampled(dtype):
    w = synth.WORKLOADS["prism3d_24_p4"]
    N, P = w["N"], w["P"]
    plan = spx.Plan(3, 2 * N ** 3, order=P, shape="prism")
    V = mesh.collapsed_vertices("prism", N)
    g = spx.geom_factors(plan, V)
    plan.set_geometry(torch.float64, g["geom"], g["dxi"])
    plan.set_geometry(torch.float32, g["geom32"], g["dxi32"])
    u = synth.uniform(synth.rng(w["seed"]), plan.n_coef)
    ut = torch.tensor(u, device="cuda", dtype=dtype)
    y = torch.empty_like(ut)
    plan.autotune("helmholtz", dtype, ut, y, reps=1)
    y = spx.helmholtz(plan, ut).cpu().double().numpy()
    ids = np.concatenate([[0, plan.E - 1], np.sort(np.random.default_rng(0).choice(plan.E, 30, replace=False))])
    Vall = C.structured_vertices("prism", N, synth.SKEW3)
    om = C.CollapsedMesh("prism", Vall[ids], P)
    nm = om.nm
    ref = np.concatenate([om.helmholtz_matrix(t) @ u[e * nm:(e + 1) * nm] for t, e in enumerate(ids)])
    got = np.concatenate([y[e * nm:(e + 1) * nm] for e in ids])
    assert rel_err(got, ref) <= TOL[dtype]


@pytest.mark.parametrize("dtype", DTYPES)
def test_tet_full_workload_sampled(dtype):
    w = synth.WORKLOADS["tet3d_16_p4"]
    N, P = w["N"], w["P"]
    plan = spx.Plan(3, 6 * N ** 3, order=P, shape="tet")
    g = spx.geom_factors(plan, mesh.collapsed_vertices("tet", N))
    plan.set_geometry(torch.float64, g["geom"], g["dxi"])
    plan.set_geometry(torch.float32, g["geom32"], g["dxi32"])
    u = synth.uniform(synth.rng(w["seed"]), plan.n_coef)
    ut = torch.tensor(u, device="cuda", dtype=dtype)
    y = torch.empty_like(ut)
    plan.autotune("helmholtz", dtype, ut, y, reps=1)
    y = spx.helmholtz(plan, ut).cpu().double().numpy()
    ids = np.concatenate([[0, plan.E - 1], np.sort(np.random.default_rng(0).choice(plan.E, 30, replace=False))])
    om = C.CollapsedMesh("tet", C.kuhn_vertices(N, synth.SKEW3)[ids], P)
    nm = om.nm
    ref = np.concatenate([om.helmholtz_matrix(t) @ u[e * nm:(e + 1) * nm] for t, e in enumerate(ids)])
    got = np.concatenate([y[e * nm:(e + 1) * nm] for e in ids])
    assert rel_err(got, ref) <= TOL[dtype]
