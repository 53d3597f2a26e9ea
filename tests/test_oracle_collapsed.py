"""Pins of the collapsed-coordinate oracle (triangles, prisms) against closed
forms, brute force and invariants: Gauss-Radau exactness, the span of the
basis (all polynomials of total degree <= P, nothing more), the vertex modes
as barycentric coordinates, vanishing of edge and interior modes, exact
integrals of monomials over the reference triangle, the P = 1 mass and
stiffness matrices of an arbitrary triangle, finite-difference derivatives,
symmetry / definiteness / constants, and PhysDeriv of the coordinates."""
import math

import numpy as np
import pytest

from oracle import basis, collapsed as C


@pytest.mark.parametrize("Q", [2, 3, 4, 6, 9])
def test_gauss_radau_rule(Q):
    x, w = C.gauss_radau(Q)
    assert x[0] == -1.0 and x[-1] < 1.0 and np.all(np.diff(x) > 0) and np.all(w > 0)
    for k in range(2 * Q - 1):
        exact = (1.0 - (-1.0) ** (k + 1)) / (k + 1)
        assert abs(np.sum(w * x ** k) - exact) < 1e-13
    k = 2 * Q - 1
    assert abs(np.sum(w * x ** k) - (1.0 - (-1.0) ** (k + 1)) / (k + 1)) > 1e-6


def test_gauss_radau_two_points_closed_form():
    x, w = C.gauss_radau(2)
    np.testing.assert_allclose(x, [-1.0, 1.0 / 3.0], atol=1e-15)
    np.testing.assert_allclose(w, [0.5, 1.5], atol=1e-15)


def _tri_points(n, seed):
    rng = np.random.default_rng(seed)
    s = rng.uniform(0.02, 0.98, (n, 2))
    s = s[s.sum(1) < 0.98]
    xi = 2.0 * s - 1.0                       # inside T: xi1 + xi2 <= 0
    eta1 = 2.0 * (1.0 + xi[:, 0]) / (1.0 - xi[:, 1]) - 1.0
    return xi, np.stack([eta1, xi[:, 1]], axis=-1)


def _monomials_tri(xi, P):
    return np.stack([xi[:, 0] ** a * xi[:, 1] ** b for a in range(P + 1) for b in range(P + 1 - a)], axis=-1)


@pytest.mark.parametrize("P", [1, 2, 3, 5, 8])
def test_triangle_basis_spans_total_degree_p(P):
    xi, eta = _tri_points(400, P)
    Phi, _ = C.basis_at(C.TRI, P, eta)
    assert Phi.shape[1] == (P + 1) * (P + 2) // 2
    Mono = _monomials_tri(xi, P)
    coef, *_ = np.linalg.lstsq(Mono, Phi, rcond=None)
    assert np.abs(Mono @ coef - Phi).max() < 1e-10          # every mode is a polynomial of degree <= P
    assert np.linalg.matrix_rank(Phi, tol=1e-10) == Phi.shape[1]   # and they are independent


@pytest.mark.parametrize("P", [1, 3, 6])
def test_triangle_vertex_modes_are_barycentric(P):
    xi, eta = _tri_points(50, 7)
    Phi, _ = C.basis_at(C.TRI, P, eta)
    modes = C.tri_modes(P)
    v0, v1, v2 = modes.index((0, 0)), modes.index((P, 0)), modes.index((0, P))
    np.testing.assert_allclose(Phi[:, v0], -(xi[:, 0] + xi[:, 1]) / 2, atol=1e-14)
    np.testing.assert_allclose(Phi[:, v1], (1 + xi[:, 0]) / 2, atol=1e-14)
    np.testing.assert_allclose(Phi[:, v2], (1 + xi[:, 1]) / 2, atol=1e-14)


def test_triangle_edge_and_interior_modes_vanish_where_they_must():
    P = 5
    t = np.linspace(-1, 1, 11)[1:-1]
    # the three edges in collapsed coordinates: bottom eta2 = -1, left eta1 = -1, hypotenuse eta1 = 1
    edges = {"bottom": np.stack([t, -np.ones_like(t)], -1), "left": np.stack([-np.ones_like(t), t], -1),
             "hyp": np.stack([np.ones_like(t), t], -1)}
    vals = {k: C.basis_at(C.TRI, P, v)[0] for k, v in edges.items()}
    for k, (p, q) in enumerate(C.tri_modes(P)):
        if (p, q) in [(0, 0), (P, 0), (0, P)]:
            continue
        on = {"bottom": 0 < p < P and q == 0, "left": p == 0 and 0 < q < P, "hyp": p == P and 0 < q < P}
        for edge, V in vals.items():
            if not on[edge]:
                assert np.abs(V[:, k]).max() < 1e-13, (p, q, edge)
            else:
                assert np.abs(V[:, k]).max() > 1e-3, (p, q, edge)


def _tri_monomial_integral(a, b):
    """int over T of xi1^a xi2^b, with s = 1 + xi1, t = 1 + xi2 on the simplex s + t <= 2
    (int s^i t^j = 2^(i+j+2) i! j! / (i+j+2)!), summed in exact rational arithmetic."""
    from fractions import Fraction
    tot = Fraction(0)
    for i in range(a + 1):
        for j in range(b + 1):
            c = math.comb(a, i) * math.comb(b, j) * (-1) ** (a - i + b - j)
            tot += c * Fraction(2 ** (i + j + 2) * math.factorial(i) * math.factorial(j), math.factorial(i + j + 2))
    return float(tot)


@pytest.mark.parametrize("P", [1, 3, 6])
def test_triangle_quadrature_integrates_degree_2p(P):
    _, xi, w = C.quadrature(C.TRI, P + 2)
    assert abs(w.sum() - 2.0) < 1e-14
    for a in range(2 * P + 1):
        for b in range(2 * P + 1 - a):
            got = np.sum(w * xi[:, 0] ** a * xi[:, 1] ** b)
            assert abs(got - _tri_monomial_integral(a, b)) < 1e-13, (a, b)


def test_p1_triangle_mass_and_stiffness_closed_forms():
    V = np.array([[[0.1, 0.2], [1.3, 0.0], [0.4, 0.9]]])
    m = C.CollapsedMesh(C.TRI, V, 1)
    modes = C.tri_modes(1)          # (0,0)=V0, (0,1)=V2 (collapsed vertex), (1,0)=V1
    order = [modes.index((0, 0)), modes.index((1, 0)), modes.index((0, 1))]
    M = m.mass_matrix(0)[np.ix_(order, order)]
    L = m.helmholtz_matrix(0, 0.0, 1.0)[np.ix_(order, order)]
    P0, P1, P2 = V[0]
    area = 0.5 * abs((P1[0] - P0[0]) * (P2[1] - P0[1]) - (P2[0] - P0[0]) * (P1[1] - P0[1]))
    np.testing.assert_allclose(M, area / 12.0 * np.array([[2, 1, 1], [1, 2, 1], [1, 1, 2]]), atol=1e-14)
    # stiffness of linear elements: K_ij = (b_i b_j + c_i c_j) / (4 area)
    x, y = V[0][:, 0], V[0][:, 1]
    b = np.array([y[1] - y[2], y[2] - y[0], y[0] - y[1]])
    c = np.array([x[2] - x[1], x[0] - x[2], x[1] - x[0]])
    np.testing.assert_allclose(L, (np.outer(b, b) + np.outer(c, c)) / (4 * area), atol=1e-13)


@pytest.mark.parametrize("P", [2, 4])
def test_triangle_derivatives_match_finite_differences(P):
    xi, eta = _tri_points(30, 11)
    _, dPhi = C.basis_at(C.TRI, P, eta)
    h = 1e-6
    for a in range(2):
        dx = np.zeros(2)
        dx[a] = h
        fp, fm = xi + dx, xi - dx
        to_eta = lambda X: np.stack([2 * (1 + X[:, 0]) / (1 - X[:, 1]) - 1, X[:, 1]], -1)
        num = (C.basis_at(C.TRI, P, to_eta(fp))[0] - C.basis_at(C.TRI, P, to_eta(fm))[0]) / (2 * h)
        np.testing.assert_allclose(dPhi[a], num, atol=1e-7)


def _prism_points(n, seed):
    xi2, eta2 = _tri_points(n, seed)
    x1 = np.random.default_rng(seed + 1).uniform(-0.98, 0.98, xi2.shape[0])
    xi = np.stack([x1, xi2[:, 0], xi2[:, 1]], -1)
    eta = np.stack([x1, eta2[:, 0], eta2[:, 1]], -1)
    return xi, eta


@pytest.mark.parametrize("P", [1, 2, 4])
def test_prism_basis_spans_segment_times_triangle(P):
    xi, eta = _prism_points(900, P)
    Phi, dPhi = C.basis_at(C.PRISM, P, eta)
    Mono = np.stack([xi[:, 0] ** a * xi[:, 1] ** b * xi[:, 2] ** c for a in range(P + 1)
                     for b in range(P + 1) for c in range(P + 1 - b)], axis=-1)
    coef, *_ = np.linalg.lstsq(Mono, Phi, rcond=None)
    assert np.abs(Mono @ coef - Phi).max() < 1e-10
    assert np.linalg.matrix_rank(Phi, tol=1e-10) == Phi.shape[1] == (P + 1) ** 2 * (P + 2) // 2
    # derivatives by finite differences in xi
    h = 1e-6
    def to_eta(X):
        return np.stack([X[:, 0], 2 * (1 + X[:, 1]) / (1 - X[:, 2]) - 1, X[:, 2]], -1)
    for a in range(3):
        dx = np.zeros(3)
        dx[a] = h
        num = (C.basis_at(C.PRISM, P, to_eta(xi + dx))[0] - C.basis_at(C.PRISM, P, to_eta(xi - dx))[0]) / (2 * h)
        np.testing.assert_allclose(dPhi[a], num, atol=1e-7)


def test_prism_p1_mass_is_segment_times_triangle():
    V = np.array([[[0, 0, 0], [2.0, 0, 0], [0, 1.0, 0], [0, 0, 1.0]]])   # affine: xi -> (1 + xi)/2 scaled
    m = C.CollapsedMesh(C.PRISM, V, 1)
    tri = C.CollapsedMesh(C.TRI, np.array([[[0, 0], [1.0, 0], [0, 1.0]]]), 1)
    seg = np.array([[2.0, 1.0], [1.0, 2.0]]) / 6.0 * 2.0                   # 1D linear mass on a length-2 segment
    np.testing.assert_allclose(m.mass_matrix(0), np.kron(tri.mass_matrix(0), seg), atol=1e-14)


@pytest.mark.parametrize("shape,P", [(C.TRI, 3), (C.TRI, 6), (C.PRISM, 2), (C.PRISM, 4)])
def test_symmetry_definiteness_constants_volume(shape, P):
    rng = np.random.default_rng(3)
    d = C.dim_of(shape)
    V = np.zeros((1, d + 1, d))
    V[0, 0] = rng.uniform(-0.2, 0.2, d)
    for c in range(d):
        V[0, c + 1] = V[0, 0] + np.eye(d)[c] + rng.uniform(-0.2, 0.2, d)
    m = C.CollapsedMesh(shape, V, P)
    H = m.helmholtz_matrix(0, 1.0, 1.0)
    M, L = m.mass_matrix(0), m.helmholtz_matrix(0, 0.0, 1.0)
    np.testing.assert_allclose(H, H.T, atol=1e-12 * np.abs(H).max())
    assert np.linalg.eigvalsh(M).min() > 0
    # the constant function: coefficients of the vertex modes (all 1)
    one = np.linalg.lstsq(m.Phi, np.ones(m.nq), rcond=None)[0]
    np.testing.assert_allclose(m.Phi @ one, 1.0, atol=1e-12)
    np.testing.assert_allclose(L @ one, 0.0, atol=1e-11)
    vol = abs(np.linalg.det(m.J[0])) * (2.0 if shape == C.TRI else 4.0)
    assert abs(one @ M @ one - vol) < 1e-12


@pytest.mark.parametrize("shape", [C.TRI, C.PRISM])
def test_phys_deriv_of_coordinates_is_identity(shape):
    rng = np.random.default_rng(4)
    d = C.dim_of(shape)
    V = np.zeros((3, d + 1, d))
    for e in range(3):
        V[e, 0] = rng.uniform(-1, 1, d)
        for c in range(d):
            V[e, c + 1] = V[e, 0] + np.eye(d)[c] + rng.uniform(-0.3, 0.3, d)
    m = C.CollapsedMesh(shape, V, 3)
    X = m.xq()
    for k in range(d):
        grads = C.phys_deriv(m, X[:, :, k].reshape(-1))
        for mm in range(d):
            np.testing.assert_allclose(grads[mm], 1.0 if mm == k else 0.0, atol=1e-11)


def test_transpose_identity_and_polynomial_bwd():
    rng = np.random.default_rng(5)
    V = np.array([[[0, 0, 0], [1.0, 0.1, 0], [0.2, 1.0, 0], [0, 0.1, 1.0]]])
    m = C.CollapsedMesh(C.PRISM, V, 3)
    u = rng.uniform(-1, 1, m.nm)
    f = rng.uniform(-1, 1, m.nq)
    lhs = C.iproduct(m, f) @ u
    rhs = np.sum(m.JW[0] * f * C.bwd_trans(m, u))
    assert abs(lhs - rhs) < 1e-13


@pytest.mark.parametrize("shape", [C.TRI, C.PRISM])
def test_structured_elements_tile_the_skewed_cell_volume(shape):
    """The two elements of every cell cover it: total volume = det(skew) (the skewed unit square / cube)."""
    skew = np.array([[1.0, 0.2], [0.1, 1.0]]) if shape == C.TRI else \
        np.array([[1.0, 0.2, 0.1], [0.0, 1.0, 0.15], [0.05, 0.0, 1.0]])
    V = C.structured_vertices(shape, 3, skew)
    m = C.CollapsedMesh(shape, V, 2)
    assert np.all(m.detJ > 0)
    assert abs(m.JW.sum() - np.linalg.det(skew)) < 1e-13


def _tet_points(n, seed):
    rng = np.random.default_rng(seed)
    s = rng.uniform(0.02, 0.98, (n, 3))
    s = s[s.sum(1) < 0.98]
    xi = 2.0 * s - 1.0                       # inside A: xi1 + xi2 + xi3 <= -1
    return xi, _tet_eta(xi)


def _tet_eta(xi):
    e1 = 2.0 * (1.0 + xi[:, 0]) / (-xi[:, 1] - xi[:, 2]) - 1.0
    e2 = 2.0 * (1.0 + xi[:, 1]) / (1.0 - xi[:, 2]) - 1.0
    return np.stack([e1, e2, xi[:, 2]], -1)


@pytest.mark.parametrize("P", [1, 2, 3, 5, 8])
def test_tet_basis_spans_total_degree_p(P):
    xi, eta = _tet_points(2500, P)
    Phi, _ = C.basis_at(C.TET, P, eta)
    assert Phi.shape[1] == (P + 1) * (P + 2) * (P + 3) // 6
    Mono = np.stack([xi[:, 0] ** a * xi[:, 1] ** b * xi[:, 2] ** c for a in range(P + 1)
                     for b in range(P + 1 - a) for c in range(P + 1 - a - b)], axis=-1)
    coef, *_ = np.linalg.lstsq(Mono, Phi, rcond=None)
    assert np.abs(Mono @ coef - Phi).max() < 1e-9
    assert np.linalg.matrix_rank(Phi, tol=1e-10) == Phi.shape[1]


@pytest.mark.parametrize("P", [1, 3, 6])
def test_tet_vertex_modes_are_barycentric(P):
    xi, eta = _tet_points(200, 9)
    Phi, _ = C.basis_at(C.TET, P, eta)
    modes, tm = C.tet_modes(P), C.tri_modes(P)
    col = lambda tri: modes.index((tm.index(tri), 0))
    np.testing.assert_allclose(Phi[:, col((0, 0))], -(1 + xi.sum(1)) / 2, atol=1e-14)
    np.testing.assert_allclose(Phi[:, col((P, 0))], (1 + xi[:, 0]) / 2, atol=1e-14)
    np.testing.assert_allclose(Phi[:, col((0, P))], (1 + xi[:, 1]) / 2, atol=1e-14)
    np.testing.assert_allclose(Phi[:, modes.index(("apex", 0))], (1 + xi[:, 2]) / 2, atol=1e-14)


@pytest.mark.parametrize("P", [2, 4])
def test_tet_derivatives_match_finite_differences(P):
    xi, eta = _tet_points(300, 12)
    _, dPhi = C.basis_at(C.TET, P, eta)
    h = 1e-6
    for a in range(3):
        dx = np.zeros(3)
        dx[a] = h
        num = (C.basis_at(C.TET, P, _tet_eta(xi + dx))[0] - C.basis_at(C.TET, P, _tet_eta(xi - dx))[0]) / (2 * h)
        np.testing.assert_allclose(dPhi[a], num, atol=2e-7)


def _tet_monomial_integral(a, b, c):
    """int over A of xi1^a xi2^b xi3^c: s = 1 + xi on the simplex s1 + s2 + s3 <= 2,
    int s^i s^j s^k = 2^(i+j+k+3) i! j! k! / (i+j+k+3)!, in exact arithmetic."""
    from fractions import Fraction
    tot = Fraction(0)
    for i in range(a + 1):
        for j in range(b + 1):
            for k in range(c + 1):
                co = math.comb(a, i) * math.comb(b, j) * math.comb(c, k) * (-1) ** (a - i + b - j + c - k)
                tot += co * Fraction(2 ** (i + j + k + 3) * math.factorial(i) * math.factorial(j) * math.factorial(k),
                                     math.factorial(i + j + k + 3))
    return float(tot)


@pytest.mark.parametrize("P", [1, 3])
def test_tet_quadrature_integrates_degree_2p(P):
    _, xi, w = C.quadrature(C.TET, P + 2)
    assert abs(w.sum() - 4.0 / 3.0) < 1e-14
    for a in range(2 * P + 1):
        for b in range(2 * P + 1 - a):
            for c in range(2 * P + 1 - a - b):
                got = np.sum(w * xi[:, 0] ** a * xi[:, 1] ** b * xi[:, 2] ** c)
                assert abs(got - _tet_monomial_integral(a, b, c)) < 1e-13, (a, b, c)


def test_p1_tet_mass_and_stiffness_closed_forms():
    V = np.array([[[0.1, 0.0, 0.2], [1.2, 0.1, 0.0], [0.2, 0.9, 0.1], [0.0, 0.2, 1.1]]])
    m = C.CollapsedMesh(C.TET, V, 1)
    modes, tm = C.tet_modes(1), C.tri_modes(1)
    order = [modes.index((tm.index((0, 0)), 0)), modes.index((tm.index((1, 0)), 0)),
             modes.index((tm.index((0, 1)), 0)), modes.index(("apex", 0))]
    M = m.mass_matrix(0)[np.ix_(order, order)]
    L = m.helmholtz_matrix(0, 0.0, 1.0)[np.ix_(order, order)]
    X = V[0]
    vol = abs(np.linalg.det(np.stack([X[1] - X[0], X[2] - X[0], X[3] - X[0]], -1))) / 6.0
    np.testing.assert_allclose(M, vol / 20.0 * (np.ones((4, 4)) + np.eye(4)), atol=1e-14)
    # linear stiffness: grad lambda_i are the rows of the inverse of [1 x y z]
    A = np.hstack([np.ones((4, 1)), X])
    G = np.linalg.inv(A)[1:, :]          # column i = grad of barycentric lambda_i
    np.testing.assert_allclose(L, vol * G.T @ G, atol=1e-12)


def test_tet_constants_volume_and_kuhn_mesh():
    skew = np.array([[1.0, 0.2, 0.1], [0.0, 1.0, 0.15], [0.05, 0.0, 1.0]])
    V = C.kuhn_vertices(2, skew)
    m = C.CollapsedMesh(C.TET, V, 3)
    assert np.all(m.detJ > 0)
    assert abs(m.JW.sum() - np.linalg.det(skew)) < 1e-13
    one = np.linalg.lstsq(m.Phi, np.ones(m.nq), rcond=None)[0]
    for e in range(0, m.E, 7):
        L = m.helmholtz_matrix(e, 0.0, 1.0)
        H = m.helmholtz_matrix(e)
        np.testing.assert_allclose(L @ one, 0.0, atol=1e-11)
        np.testing.assert_allclose(H, H.T, atol=1e-12 * np.abs(H).max())
    X = m.xq()
    grads = C.phys_deriv(m, X[:, :, 1].reshape(-1))
    np.testing.assert_allclose(grads[1], 1.0, atol=1e-11)
    np.testing.assert_allclose(grads[0], 0.0, atol=1e-11)
