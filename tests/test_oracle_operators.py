"""Pins of the oracle's elemental operators against closed forms and invariants.

Independent references used here: 1D mass/stiffness matrices integrated with
scipy's Gauss-Legendre rule and scipy's Jacobi polynomials; Kronecker
identities of affine elements; the paper's worked example (§3.5, Listing
lst:python); analytic derivatives of polynomials and of the coordinate map.
"""
import os

import numpy as np
import pytest
from numpy.polynomial import Polynomial
from scipy import special

from oracle import geometry, operators

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def ref_basis_1d(P, x):
    """phi_p from the paper's definition with scipy's Jacobi polynomials."""
    out = np.empty((x.size, P + 1))
    out[:, 0] = (1 - x) / 2
    out[:, P] = (1 + x) / 2
    for p in range(1, P):
        out[:, p] = (1 - x) * (1 + x) / 4 * special.eval_jacobi(p - 1, 1, 1, x)
    return out


def ref_mass_stiffness_1d(P):
    xg, wg = special.roots_legendre(40)
    B = ref_basis_1d(P, xg)
    dB = np.stack([Polynomial.fit(xg, B[:, p], P).deriv()(xg) for p in range(P + 1)], axis=1)
    return B.T @ (wg[:, None] * B), dB.T @ (wg[:, None] * dB)


def test_1d_p1_closed_form():
    M, K = ref_mass_stiffness_1d(1)
    np.testing.assert_allclose(M, [[2 / 3, 1 / 3], [1 / 3, 2 / 3]], atol=1e-14)
    np.testing.assert_allclose(K, [[0.5, -0.5], [-0.5, 0.5]], atol=1e-12)


@pytest.mark.parametrize("dim,P", [(2, 1), (2, 4), (2, 7), (3, 1), (3, 3), (3, 4), (3, 6)])
def test_affine_kronecker_identity(dim, P):
    N = 2
    h = 1.0 / N
    mesh = geometry.StructuredMesh(dim, N, P, amp=0.0)
    geo = mesh.geometry(P, P + 2, np.arange(mesh.E))
    M1, K1 = ref_mass_stiffness_1d(P)
    Me = operators.helmholtz_matrix(dim, P, P + 2, geo, 3, lam=1.0, kappa=0.0)
    Le = operators.helmholtz_matrix(dim, P, P + 2, geo, 3, lam=0.0, kappa=1.0)
    if dim == 2:
        Mref = (h / 2) ** 2 * np.kron(M1, M1)
        Lref = np.kron(M1, K1) + np.kron(K1, M1)
    else:
        Mref = (h / 2) ** 3 * np.kron(M1, np.kron(M1, M1))
        Lref = (h / 2) * (np.kron(M1, np.kron(M1, K1)) + np.kron(M1, np.kron(K1, M1))
                          + np.kron(K1, np.kron(M1, M1)))
    np.testing.assert_allclose(Me, Mref, atol=1e-13 * np.abs(Mref).max())
    np.testing.assert_allclose(Le, Lref, atol=1e-12 * np.abs(Lref).max())


def test_listing_quadrature_integrates_mass_exactly():
    """Reading of §3.5: 8 modes (order 7) need 9 GLL points for an exact mass matrix."""
    P = 7
    M1, _ = ref_mass_stiffness_1d(P)
    mesh = geometry.StructuredMesh(2, 1, P, nq=9, origin=-1.0, length=2.0)
    geo = mesh.geometry(P, 9, np.arange(1))
    np.testing.assert_allclose(operators.mass_matrix(2, P, 9, geo, 0), np.kron(M1, M1), atol=1e-14)
    mesh8 = geometry.StructuredMesh(2, 1, P, nq=8, origin=-1.0, length=2.0)
    geo8 = mesh8.geometry(P, 8, np.arange(1))
    assert np.abs(operators.mass_matrix(2, P, 8, geo8, 0) - np.kron(M1, M1)).max() > 1e-6


def curved(dim=3, N=2, P=4, amp=0.05):
    return geometry.StructuredMesh(dim, N, P, amp=amp)


@pytest.mark.parametrize("dim,P", [(2, 3), (3, 2), (3, 4)])
def test_symmetric_positive_definite(dim, P):
    mesh = curved(dim, 2, P)
    geo = mesh.geometry(P, P + 2, np.arange(mesh.E))
    for t in range(mesh.E):
        H = operators.helmholtz_matrix(dim, P, P + 2, geo, t)
        assert np.abs(H - H.T).max() <= 1e-14 * np.abs(H).max()
        assert np.linalg.eigvalsh(H).min() > 0
        M = operators.mass_matrix(dim, P, P + 2, geo, t)
        assert np.linalg.eigvalsh(M).min() > 0


@pytest.mark.parametrize("dim,P", [(2, 4), (3, 3), (3, 5)])
def test_constant_in_kernel_of_L_and_volume(dim, P):
    mesh = curved(dim, 2, P)
    geo = mesh.geometry(P, P + 2, np.arange(mesh.E))
    n = P + 1
    one = np.zeros(n ** dim)
    # the constant function = 1 on every vertex mode (p, q, r in {0, P}), 0 on the rest
    for loc in range(n ** dim):
        modes = [loc % n, (loc // n) % n, loc // (n * n)][:dim]
        if all(m in (0, P) for m in modes):
            one[loc] = 1.0
    h = 1.0 / mesh.N
    for t in range(mesh.E):
        L = operators.helmholtz_matrix(dim, P, P + 2, geo, t, lam=0.0, kappa=1.0)
        assert np.abs(L @ one).max() < 1e-13 * np.abs(L).max()
        M = operators.mass_matrix(dim, P, P + 2, geo, t)
        np.testing.assert_allclose(one @ M @ one, h ** dim, rtol=1e-13)
    # total area / volume of the periodic unit square / cube
    np.testing.assert_allclose(geo["JW"].sum(), 1.0, rtol=1e-13)


def test_shear_jacobian_is_constant():
    """For x' = x + f(y, z) the iso-parametric Jacobian has det J = (h/2)^3."""
    mesh = curved(3, 3, 4)
    geo = mesh.geometry(4, 6, np.arange(mesh.E))
    np.testing.assert_allclose(geo["detJ"], (1 / 6) ** 3, rtol=1e-13)


@pytest.mark.parametrize("dim,P", [(2, 4), (3, 4), (3, 2)])
def test_transpose_identity(dim, P):
    mesh = curved(dim, 2, P)
    rng = np.random.default_rng(0)
    u = rng.uniform(-1, 1, mesh.coef_off[-1])
    f = rng.uniform(-1, 1, mesh.quad_off[-1])
    lhs = operators.iproduct(mesh, f) @ u
    geom, _, _ = mesh.factors_flat()
    nf = 7 if dim == 3 else 4
    Q = P + 2
    JW = geom.reshape(mesh.E, nf, Q ** dim)[:, -1, :].reshape(-1)
    rhs = np.sum(JW * f * operators.bwd_trans(mesh, u))
    np.testing.assert_allclose(lhs, rhs, rtol=1e-13)


def test_projection_roundtrip_and_polynomial_reproduction():
    mesh = curved(3, 2, 3)
    rng = np.random.default_rng(1)
    u = rng.uniform(-1, 1, mesh.coef_off[-1])
    np.testing.assert_allclose(operators.fwd_trans(mesh, operators.bwd_trans(mesh, u)), u, atol=1e-12)
    # polynomial of degree <= P per axis on an affine mesh is reproduced
    P = 3
    aff = geometry.StructuredMesh(3, 2, P, amp=0.0)
    _, _, xq = aff.factors_flat()
    X = xq.reshape(aff.E, 3, -1)
    f = (X[:, 0] ** 3 - 2 * X[:, 1] ** 2 * X[:, 0] + X[:, 2] * X[:, 1] ** 3 + 0.5).reshape(-1)
    g = operators.bwd_trans(aff, operators.fwd_trans(aff, f))
    np.testing.assert_allclose(g, f, atol=1e-12)


def test_phys_deriv_of_coordinates_is_identity():
    mesh = curved(3, 2, 4)
    _, _, xq = mesh.factors_flat()
    X = xq.reshape(mesh.E, 3, -1)
    for m in range(3):
        d = operators.phys_deriv(mesh, X[:, m].reshape(-1))
        for k in range(3):
            np.testing.assert_allclose(d[k], 1.0 if k == m else 0.0, atol=1e-12)


@pytest.mark.parametrize("dim", [2, 3])
def test_phys_deriv_polynomial_exact(dim):
    P = 4
    aff = geometry.StructuredMesh(dim, 2, P, amp=0.0)
    _, _, xq = aff.factors_flat()
    X = xq.reshape(aff.E, dim, -1)
    x, y = X[:, 0], X[:, 1]
    z = X[:, 2] if dim == 3 else 0.0 * x
    f = x ** 4 * y ** 2 - 3 * y ** 5 + x * z ** 3 + 1.0
    grads = [4 * x ** 3 * y ** 2 + z ** 3, 2 * x ** 4 * y - 15 * y ** 4, 3 * x * z ** 2]
    out = operators.phys_deriv(aff, f.reshape(-1))
    for m in range(dim):
        np.testing.assert_allclose(out[m], grads[m].reshape(-1), atol=1e-11)


def test_paper_worked_example_integral():
    """§3.5, Listing lst:python: integral of cos(x) cos(y) on [-1, 1]^2 = 4 sin^2(1)."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "e1_integral.txt")) if not l.startswith("#")]
    n_modes, n_pts, _, exact = int(rows[0][0]), int(rows[0][1]), rows[0][2], float(rows[0][3])
    np.testing.assert_allclose(exact, 4 * np.sin(1) ** 2, rtol=1e-16)
    P = n_modes - 1
    mesh = geometry.StructuredMesh(2, 1, P, nq=n_pts, origin=-1.0, length=2.0)
    _, _, xq = mesh.factors_flat()
    X = xq.reshape(2, -1)
    f = np.cos(X[0]) * np.cos(X[1])
    assert abs(operators.integral(mesh, f) - exact) < 1e-13
    proj = operators.fwd_trans(mesh, f)
    assert abs(operators.integral(mesh, operators.bwd_trans(mesh, proj)) - exact) < 1e-12
    # the projection is close to f itself (order 7 approximation of an entire function)
    assert np.abs(operators.bwd_trans(mesh, proj) - f).max() < 1e-6


def test_variable_order_matches_uniform_groups():
    """A variable-order mesh applies each element with its own order."""
    rng = np.random.default_rng(3)
    orders = rng.integers(2, 6, size=8)
    mesh = geometry.StructuredMesh(3, 2, orders, amp=0.05)
    u = rng.uniform(-1, 1, mesh.coef_off[-1])
    y = operators.helmholtz(mesh, u)
    for e in range(mesh.E):
        P = int(orders[e])
        geo = mesh.geometry(P, P + 2, np.array([e]))
        H = operators.helmholtz_matrix(3, P, P + 2, geo, 0)
        ue = u[mesh.coef_off[e]: mesh.coef_off[e + 1]]
        np.testing.assert_allclose(y[mesh.coef_off[e]: mesh.coef_off[e + 1]], H @ ue, atol=1e-14)
