"""Pins of the oracle's GLL nodal basis variant (collocation, classical spectral elements)."""
import numpy as np
import pytest

from oracle import basis, nodal, operators
from oracle.geometry import StructuredMesh, tensor_matrix


@pytest.mark.parametrize("dim,P", [(2, 3), (3, 2), (3, 4)])
def test_collocation_basis_is_identity_and_its_gradient_the_collocation_derivative(dim, P):
    Phi, dPhi = nodal.phi_matrices(dim, P, P + 1)
    np.testing.assert_allclose(Phi, np.eye((P + 1) ** dim), atol=1e-14)
    for a, D in enumerate(operators.collocation_matrices(dim, P + 1)):
        np.testing.assert_allclose(dPhi[a], D, atol=1e-12)


@pytest.mark.parametrize("dim,N,P,amp", [(3, 2, 3, 0.05), (2, 3, 4, 0.05)])
def test_collocated_mass_matrix_is_diagonal_jw(dim, N, P, amp):
    mesh = StructuredMesh(dim, N, P, amp=amp, nq=P + 1)
    for Pg, Qg, ids in mesh.groups():
        geo = mesh.geometry(Pg, Qg, ids)
        for t in range(len(ids)):
            M = nodal.helmholtz_matrix(dim, Pg, Qg, geo, t, lam=1.0, kappa=0.0)
            np.testing.assert_allclose(M, np.diag(geo["JW"][t]), atol=1e-15)


@pytest.mark.parametrize("dim,P,qoff", [(3, 3, 1), (3, 4, 2), (2, 5, 1), (2, 3, 2)])
def test_nodal_operator_is_the_modal_one_in_another_basis(dim, P, qoff):
    """Both bases span the same space: with T the modified basis evaluated at the
    P+1 GLL nodes (so that modal u maps to nodal T u), H_nodal = T^-T H_modal T^-1."""
    mesh = StructuredMesh(dim, 2, P, amp=0.05, nq=P + qoff)
    z, _ = basis.gll(P + 1)
    T = tensor_matrix(dim, [basis.modified_basis(P, z)] * dim)
    Ti = np.linalg.inv(T)
    rng = np.random.default_rng(3)
    for Pg, Qg, ids in mesh.groups():
        geo = mesh.geometry(Pg, Qg, ids)
        nq = geo["JW"].shape[1]
        lam, kap = rng.uniform(0.5, 2.0, nq), rng.uniform(0.5, 2.0, nq)
        for t in range(len(ids)):
            Hn = nodal.helmholtz_matrix(dim, Pg, Qg, geo, t, lam, kap)
            Hm = operators.helmholtz_matrix(dim, Pg, Qg, geo, t, lam, kap)
            np.testing.assert_allclose(Hn, Ti.T @ Hm @ Ti, rtol=1e-10, atol=1e-12 * np.abs(Hn).max())


@pytest.mark.parametrize("dim,P", [(3, 3), (2, 4)])
def test_constant_in_kernel_volume_symmetry(dim, P):
    mesh = StructuredMesh(dim, 2, P, amp=0.05, nq=P + 1)
    ones = np.ones((P + 1) ** dim)
    vol = 0.0
    for Pg, Qg, ids in mesh.groups():
        geo = mesh.geometry(Pg, Qg, ids)
        for t in range(len(ids)):
            L = nodal.helmholtz_matrix(dim, Pg, Qg, geo, t, lam=0.0, kappa=1.0)
            M = nodal.helmholtz_matrix(dim, Pg, Qg, geo, t, lam=1.0, kappa=0.0)
            np.testing.assert_allclose(L @ ones, 0.0, atol=1e-12)
            np.testing.assert_allclose(L, L.T, atol=1e-13)
            assert np.linalg.eigvalsh(L).min() > -1e-12
            vol += ones @ M @ ones
    assert abs(vol - 1.0) < 1e-13


def test_whole_mesh_apply_matches_elementwise():
    mesh = StructuredMesh(3, 2, 3, amp=0.05, nq=4)
    u = np.random.default_rng(4).uniform(-1, 1, mesh.coef_off[-1])
    y = nodal.helmholtz(mesh, u, lam=1.5, kappa=0.7)
    geo = mesh.geometry(3, 4, np.arange(mesh.E))
    for e in range(mesh.E):
        s = slice(mesh.coef_off[e], mesh.coef_off[e + 1])
        np.testing.assert_allclose(y[s], nodal.helmholtz_matrix(3, 3, 4, geo, e, 1.5, 0.7) @ u[s], atol=1e-13)


@pytest.mark.parametrize("dim,P,qoff", [(3, 3, 1), (3, 2, 2), (2, 4, 2)])
def test_nodal_bwd_trans_interpolates_and_iproduct_is_its_transpose(dim, P, qoff):
    """BwdTrans of nodal values of a polynomial of degree <= P per direction
    evaluates that polynomial at the quadrature points (the identity when the
    points are the nodes); IProduct satisfies <IProduct(f), u> = sum JW f (B u)."""
    mesh = StructuredMesh(dim, 2, P, amp=0.05, nq=P + qoff)
    rng = np.random.default_rng(9)
    c = rng.uniform(-1, 1, (P + 1,) * dim)          # coefficients of prod_a x_a^k_a in reference coordinates
    z, _ = basis.gll(P + 1)
    xi, _ = basis.gll(P + qoff)

    def poly(pts):
        V = [np.vander(pts[:, a], P + 1, increasing=True) for a in range(dim)]
        if dim == 2:
            return np.einsum("qi,qj,ij->q", V[0], V[1], c)
        return np.einsum("qi,qj,qk,ijk->q", V[0], V[1], V[2], c)
    from oracle.geometry import reference_points
    nod, quad = poly(reference_points(dim, z)), poly(reference_points(dim, xi))
    u = np.concatenate([nod] * mesh.E)
    np.testing.assert_allclose(nodal.bwd_trans(mesh, u), np.concatenate([quad] * mesh.E), atol=1e-12)
    if qoff == 1:
        np.testing.assert_array_equal(nodal.bwd_trans(mesh, u), u)
    f = rng.uniform(-1, 1, mesh.quad_off[-1])
    v = rng.uniform(-1, 1, mesh.coef_off[-1])
    JW = np.concatenate([mesh.geometry(P, P + qoff, np.array([e]))["JW"][0] for e in range(mesh.E)])
    lhs = nodal.iproduct(mesh, f) @ v
    rhs = np.sum(JW * f * nodal.bwd_trans(mesh, v))
    assert abs(lhs - rhs) <= 1e-13 * np.sum(np.abs(JW * f))


def test_nodal_helmholtz_fields_match_the_elemental_matrices():
    mesh = StructuredMesh(3, 2, 2, amp=0.05, nq=3)
    rng = np.random.default_rng(10)
    u = rng.uniform(-1, 1, mesh.coef_off[-1])
    lam = rng.uniform(0.5, 2, mesh.quad_off[-1])
    kap = rng.uniform(0.5, 2, mesh.quad_off[-1])
    y = nodal.helmholtz(mesh, u, lam_field=lam, kappa_field=kap)
    geo = mesh.geometry(2, 3, np.arange(mesh.E))
    for e in range(mesh.E):
        s = slice(mesh.coef_off[e], mesh.coef_off[e + 1])
        q = slice(mesh.quad_off[e], mesh.quad_off[e + 1])
        np.testing.assert_allclose(y[s], nodal.helmholtz_matrix(3, 2, 3, geo, e, lam[q], kap[q]) @ u[s], atol=1e-13)
    # lambda field = constant 1.5 reproduces the scalar form
    np.testing.assert_allclose(nodal.helmholtz(mesh, u, lam_field=np.full(mesh.quad_off[-1], 1.5)),
                               nodal.helmholtz(mesh, u, lam=1.5), atol=1e-13)
