"""Collapsed-coordinate elements: triangles, prisms and tetrahedra (FP64, numpy).

Test infrastructure only (see ``oracle/__init__.py``).

Follows §2.1: the triangle T = {xi in [-1,1]^2 | xi1 + xi2 <= 0} and the
prism R = {xi in [-1,1]^3 | xi2 + xi3 <= 0} of Table t:refregions are the
images of the square / cube under the collapse (Duffy map, Fig. f:duffy)
    triangle: xi1 = (1 + eta1)(1 - eta2)/2 - 1,  xi2 = eta2
    prism:    xi1 = eta1,  xi2 = (1 + eta2)(1 - eta3)/2 - 1,  xi3 = eta3
so that a tensor product of 1D functions of the collapsed coordinates eta
can span the polynomials on the element.  The paper defers the collapsed
basis itself to Karniadakis & Sherwin (2005); the construction here is the
modified C0 one restated from its mathematics (the reading is recorded with
the build's readings):

* principal functions in eta1 (and in the uncollapsed prism direction): the
  modified 1D basis psi^a_p of §2.1 (``basis.modified_basis``);
* in the collapsed direction z = eta2 (triangle) / eta3 (prism):
    psi^b_{pq}(z) = psi^a_q(z)                                  p = 0 or p = P
                  = ((1-z)/2)^(p+1)                              0 < p < P, q = 0
                  = ((1-z)/2)^(p+1) (1+z)/2 P^{(2p+1,1)}_{q-1}(z) 0 < p < P, q >= 1
  so that psi^a_p(eta1) psi^b_{pq}(eta2) is a polynomial in xi of total
  degree <= P for the modes below;
* triangle modes, in storage order (p outer, q inner):
    p = 0: q = 0..P     p = 1..P-1: q = 0..P-1-p     p = P: q = 0..P-1
  with the mode (0, P) the collapsed vertex xi = (-1, 1): the function
  (1 + eta2)/2 = psi^a_0(eta1) psi^a_P(eta2) + psi^a_P(eta1) psi^a_P(eta2);
  (P+1)(P+2)/2 modes: 3 vertices, 3 (P-1) edge and (P-1)(P-2)/2 interior;
* prism modes: psi^a_a(xi1) times a triangle mode in (eta2, eta3), index
  a + (P+1) m (a fastest, m the triangle mode's storage index).

Quadrature on Q points per direction: Gauss-Lobatto-Legendre in the
uncollapsed directions, Gauss-Radau-Legendre in the collapsed one (the
points include -1 and omit +1, the collapsed vertex, where the inverse map is
singular; §2.1 names Gauss-Radau points for this).  The weights carry the
Duffy Jacobian (1 - eta2)/2 (triangle) / (1 - eta3)/2 (prism).  Point index
i + Q j (+ Q^2 k), first direction fastest.

Elements are affine images x = V0 + sum_c (V_c - V0)(1 + xi_c)/2 of the
reference shape (V_c the image of the reference vertex one step along xi_c
from (-1, ..., -1)); derivatives with respect to xi follow from those with
respect to eta by the chain rule of the collapse, and the physical ones from
the constant Jacobian.  Every operator is a dense matrix built from these
definitions; no sum-factorisation.
"""
import numpy as np

from . import basis

TRI, PRISM = "tri", "prism"


# ---------------------------------------------------------------------------
# 1D pieces
# ---------------------------------------------------------------------------

def gauss_radau(Q):
    """Q Gauss-Radau-Legendre points (ascending, x_0 = -1, all < 1) and weights.

    The points are the zeros of P_{Q-1}(x) + P_Q(x) (which vanishes at -1);
    weights w_0 = 2 / Q^2 and w_i = (1 - x_i) / (Q^2 P_{Q-1}(x_i)^2).  The rule
    integrates polynomials of degree <= 2Q - 2 exactly on [-1, 1].
    """
    c = np.zeros(Q + 1)
    c[Q - 1] = 1.0
    c[Q] = 1.0
    x = np.sort(np.real(np.polynomial.legendre.legroots(c)))
    x[0] = -1.0
    Pm1, _ = basis.legendre(Q - 1, x)
    w = (1.0 - x) / (Q * Q * Pm1 ** 2)
    w[0] = 2.0 / (Q * Q)
    return x, w


def psi_b(P, p, z, deriv=False):
    """Values (or derivatives) of psi^b_{pq}(z), q over the mode range of p; shape (len(z), nq)."""
    z = np.atleast_1d(np.asarray(z, dtype=np.float64))
    if p == 0 or p == P:
        m = P + 1 if p == 0 else P
        B = basis.modified_basis_deriv(P, z) if deriv else basis.modified_basis(P, z)
        return B[:, :m]
    nq = P - p
    out = np.empty((z.size, nq))
    L, R = 0.5 * (1.0 - z), 0.5 * (1.0 + z)
    dL, dR = -0.5, 0.5
    for q in range(nq):
        if q == 0:
            f = L ** (p + 1)
            df = (p + 1) * L ** p * dL
        else:
            J = basis.jacobi(q - 1, 2 * p + 1, 1, z)
            dJ = basis.jacobi_deriv(q - 1, 2 * p + 1, 1, z)
            f = L ** (p + 1) * R * J
            df = (p + 1) * L ** p * dL * R * J + L ** (p + 1) * dR * J + L ** (p + 1) * R * dJ
        out[:, q] = df if deriv else f
    return out


def tri_modes(P):
    """Storage order of the triangle modes: list of (p, q)."""
    m = [(0, q) for q in range(P + 1)]
    for p in range(1, P):
        m += [(p, q) for q in range(P - p)]
    m += [(P, q) for q in range(P)]
    return m


def n_tri(P):
    return (P + 1) * (P + 2) // 2


def tri_basis(P, e1, e2):
    """Triangle modes at collapsed points (e1[k], e2[k]): values and d/d eta1, d/d eta2.

    Returns (Phi, dPhi1, dPhi2), each (npts, n_tri(P)).
    """
    e1 = np.atleast_1d(np.asarray(e1, dtype=np.float64))
    e2 = np.atleast_1d(np.asarray(e2, dtype=np.float64))
    A, dA = basis.modified_basis(P, e1), basis.modified_basis_deriv(P, e1)
    Phi = np.empty((e1.size, n_tri(P)))
    D1, D2 = np.empty_like(Phi), np.empty_like(Phi)
    cols = {}
    for p in range(P + 1):
        cols[p] = (psi_b(P, p, e2), psi_b(P, p, e2, deriv=True))
    for k, (p, q) in enumerate(tri_modes(P)):
        if (p, q) == (0, P):     # collapsed vertex: (1 + eta2) / 2, independent of eta1
            Phi[:, k] = 0.5 * (1.0 + e2)
            D1[:, k] = 0.0
            D2[:, k] = 0.5
            continue
        b, db = cols[p]
        Phi[:, k] = A[:, p] * b[:, q]
        D1[:, k] = dA[:, p] * b[:, q]
        D2[:, k] = A[:, p] * db[:, q]
    return Phi, D1, D2


def n_modes(shape, P):
    return {TRI: n_tri(P), PRISM: (P + 1) * n_tri(P), TET: n_tet(P)}[shape]


def dim_of(shape):
    return 2 if shape == TRI else 3


def quadrature(shape, Q):
    """Collapsed points eta (npts, d), reference points xi (npts, d) and weights
    including the Duffy Jacobian, point index i + Q j (+ Q^2 k)."""
    g, wg = basis.gll(Q)
    r, wr = gauss_radau(Q)
    if shape == TRI:
        E2, E1 = np.meshgrid(r, g, indexing="ij")
        W2, W1 = np.meshgrid(wr, wg, indexing="ij")
        eta = np.stack([E1.ravel(), E2.ravel()], axis=-1)
        w = (W1 * W2).ravel() * 0.5 * (1.0 - eta[:, 1])
        xi = np.stack([0.5 * (1.0 + eta[:, 0]) * (1.0 - eta[:, 1]) - 1.0, eta[:, 1]], axis=-1)
        return eta, xi, w
    if shape == TET:
        E3, E2, E1 = np.meshgrid(r, r, g, indexing="ij")
        W3, W2, W1 = np.meshgrid(wr, wr, wg, indexing="ij")
        eta = np.stack([E1.ravel(), E2.ravel(), E3.ravel()], axis=-1)
        w = (W1 * W2 * W3).ravel() * 0.5 * (1.0 - eta[:, 1]) * (0.5 * (1.0 - eta[:, 2])) ** 2
        xi = np.stack([0.25 * (1.0 + eta[:, 0]) * (1.0 - eta[:, 1]) * (1.0 - eta[:, 2]) - 1.0,
                       0.5 * (1.0 + eta[:, 1]) * (1.0 - eta[:, 2]) - 1.0, eta[:, 2]], axis=-1)
        return eta, xi, w
    E3, E2, E1 = np.meshgrid(r, g, g, indexing="ij")
    W3, W2, W1 = np.meshgrid(wr, wg, wg, indexing="ij")
    eta = np.stack([E1.ravel(), E2.ravel(), E3.ravel()], axis=-1)
    w = (W1 * W2 * W3).ravel() * 0.5 * (1.0 - eta[:, 2])
    xi = np.stack([eta[:, 0], 0.5 * (1.0 + eta[:, 1]) * (1.0 - eta[:, 2]) - 1.0, eta[:, 2]], axis=-1)
    return eta, xi, w


def _deta_dxi(shape, eta):
    """K[q, a, c] = d eta_a / d xi_c of the collapse at the points eta."""
    npt = eta.shape[0]
    d = 2 if shape == TRI else 3
    K = np.zeros((npt, d, d))
    if shape == TRI:
        s = 1.0 / (1.0 - eta[:, 1])
        K[:, 0, 0] = 2.0 * s
        K[:, 0, 1] = (1.0 + eta[:, 0]) * s
        K[:, 1, 1] = 1.0
    elif shape == PRISM:
        s = 1.0 / (1.0 - eta[:, 2])
        K[:, 0, 0] = 1.0
        K[:, 1, 1] = 2.0 * s
        K[:, 1, 2] = (1.0 + eta[:, 1]) * s
        K[:, 2, 2] = 1.0
    else:
        s23 = 1.0 / ((1.0 - eta[:, 1]) * (1.0 - eta[:, 2]))
        s3 = 1.0 / (1.0 - eta[:, 2])
        K[:, 0, 0] = 4.0 * s23
        K[:, 0, 1] = 2.0 * (1.0 + eta[:, 0]) * s23
        K[:, 0, 2] = 2.0 * (1.0 + eta[:, 0]) * s23
        K[:, 1, 1] = 2.0 * s3
        K[:, 1, 2] = (1.0 + eta[:, 1]) * s3
        K[:, 2, 2] = 1.0
    return K


def basis_at(shape, P, eta):
    """Phi (npts, nm) and [d Phi / d xi_a] at collapsed points, by the chain rule of the collapse."""
    if shape == TET:
        Phi, d1, d2, d3 = tet_basis(P, eta)
        K = _deta_dxi(TET, eta)
        dEta = [d1, d2, d3]
        return Phi, [sum(K[:, a, c][:, None] * dEta[a] for a in range(3)) for c in range(3)]
    if shape == TRI:
        T, T1, T2 = tri_basis(P, eta[:, 0], eta[:, 1])
        s = 1.0 / (1.0 - eta[:, 1])
        d_xi1 = (2.0 * s)[:, None] * T1
        d_xi2 = ((1.0 + eta[:, 0]) * s)[:, None] * T1 + T2
        return T, [d_xi1, d_xi2]
    A, dA = basis.modified_basis(P, eta[:, 0]), basis.modified_basis_deriv(P, eta[:, 0])
    T, T1, T2 = tri_basis(P, eta[:, 1], eta[:, 2])
    n = P + 1
    prod = lambda X, Y: (X[:, :, None] * Y[:, None, :]).transpose(0, 2, 1).reshape(X.shape[0], -1)
    # column a + n m: X[:, a] Y[:, m] -> reshape with a fastest
    Phi = prod(A, T)
    s = 1.0 / (1.0 - eta[:, 2])
    d1 = prod(dA, T)
    d2 = prod(A, (2.0 * s)[:, None] * T1)
    d3 = prod(A, ((1.0 + eta[:, 1]) * s)[:, None] * T1 + T2)
    assert Phi.shape[1] == n * n_tri(P)
    return Phi, [d1, d2, d3]


class CollapsedMesh:
    """Affine triangles or prisms.

    ``verts``: (E, d+1, d) array, element e's defining vertices V0..Vd (V_c the
    image of the reference vertex one step along xi_c from (-1, ..., -1)).
    Buffers follow the library's layouts: element-major coefficients (n_modes
    per element), quadrature values (Q^d per element)."""

    def __init__(self, shape, verts, P, Q=None):
        self.shape, self.d = shape, dim_of(shape)
        self.V = np.asarray(verts, dtype=np.float64)
        self.E = self.V.shape[0]
        self.P, self.Q = P, (P + 2 if Q is None else Q)
        self.nm, self.nq = n_modes(shape, P), self.Q ** self.d
        self.eta, self.xi, self.w = quadrature(shape, self.Q)
        self.Phi, self.dPhi = basis_at(shape, P, self.eta)
        d = self.d
        self.J = np.stack([(self.V[:, c + 1] - self.V[:, 0]) / 2.0 for c in range(d)], axis=-1)  # J[e, m, c]
        self.detJ = np.linalg.det(self.J)
        self.Jinv = np.linalg.inv(self.J)           # Jinv[e, c, m] = d xi_c / d x_m
        self.JW = self.w[None, :] * self.detJ[:, None]

    def xq(self):
        """Physical coordinates of the quadrature points: (E, nq, d)."""
        return self.V[:, None, 0, :] + np.einsum("emc,qc->eqm", self.J, self.xi + 1.0)

    def helmholtz_matrix(self, e, lam=1.0, kappa=1.0):
        """Dense H_e = M_e(lambda) + L_e(kappa) (lambda, kappa scalars or per-point arrays)."""
        lam_q = np.broadcast_to(np.asarray(lam, dtype=np.float64), (self.nq,))
        kap_q = np.broadcast_to(np.asarray(kappa, dtype=np.float64), (self.nq,))
        W = self.JW[e]
        M = self.Phi.T @ ((W * lam_q)[:, None] * self.Phi)
        Ci = self.Jinv[e]
        grad = [sum(Ci[c, m] * self.dPhi[c] for c in range(self.d)) for m in range(self.d)]   # d Phi / d x_m
        L = sum(grad[m].T @ ((W * kap_q)[:, None] * grad[m]) for m in range(self.d))
        return M + L

    def mass_matrix(self, e):
        return self.helmholtz_matrix(e, 1.0, 0.0)


def bwd_trans(mesh, coef):
    U = np.asarray(coef, dtype=np.float64).reshape(mesh.E, mesh.nm)
    return (U @ mesh.Phi.T).reshape(-1)


def iproduct(mesh, f):
    F = np.asarray(f, dtype=np.float64).reshape(mesh.E, mesh.nq)
    return ((mesh.JW * F) @ mesh.Phi).reshape(-1)


def helmholtz(mesh, coef, lam=1.0, lam_field=None, kappa_field=None):
    U = np.asarray(coef, dtype=np.float64).reshape(mesh.E, mesh.nm)
    out = np.empty_like(U)
    for e in range(mesh.E):
        la = lam if lam_field is None else np.asarray(lam_field).reshape(mesh.E, mesh.nq)[e]
        ka = 1.0 if kappa_field is None else np.asarray(kappa_field).reshape(mesh.E, mesh.nq)[e]
        out[e] = mesh.helmholtz_matrix(e, la, ka) @ U[e]
    return out.reshape(-1)


def collocation_matrices(shape, Q):
    """Dense Q^d x Q^d derivative along each collapsed direction of the Lagrange
    interpolant through the quadrature grid (GLL / Gauss-Radau points)."""
    g, _ = basis.gll(Q)
    r, _ = gauss_radau(Q)
    Dg = basis.lagrange(g, g)[1]
    Dr = basis.lagrange(r, r)[1]
    I = np.eye(Q)
    from .geometry import tensor_matrix
    if shape == TRI:
        return [tensor_matrix(2, [Dg, I]), tensor_matrix(2, [I, Dr])]
    if shape == TET:
        return [tensor_matrix(3, [Dg, I, I]), tensor_matrix(3, [I, Dr, I]), tensor_matrix(3, [I, I, Dr])]
    return [tensor_matrix(3, [Dg, I, I]), tensor_matrix(3, [I, Dg, I]), tensor_matrix(3, [I, I, Dr])]


def deta_dx(mesh):
    """d eta_a / d x_m at the quadrature points: (E, nq, d, d), by the chain
    rule d eta / d xi (the collapse) times d xi / d x (the affine map)."""
    K = _deta_dxi(mesh.shape, mesh.eta)     # K[q, a, c] = d eta_a / d xi_c
    return np.einsum("qac,ecm->eqam", K, mesh.Jinv)


def phys_deriv(mesh, f):
    """d f / d x_m at the quadrature points from quadrature values f: a list of d flat arrays."""
    F = np.asarray(f, dtype=np.float64).reshape(mesh.E, mesh.nq)
    Dm = collocation_matrices(mesh.shape, mesh.Q)
    ref = [F @ Dm[a].T for a in range(mesh.d)]          # d f / d eta_a
    K = deta_dx(mesh)
    return [sum(K[:, :, a, m] * ref[a] for a in range(mesh.d)).reshape(-1) for m in range(mesh.d)]


def structured_vertices(shape, N, skew, jitter=None):
    """Affine elements of a skewed N^d grid on the unit square / cube, two per cell.

    Grid node (i, j[, k]) sits at skew @ ((i, j[, k]) / N).  Cell c = ex + N(ey
    [+ N ez]) holds elements 2c and 2c + 1:
      triangles  (n(ex,ey), n(ex+1,ey), n(ex,ey+1)) and (n(ex+1,ey+1), n(ex,ey+1), n(ex+1,ey));
      prisms     (n(i,j,k), n(i+1,j,k), n(i,j+1,k), n(i,j,k+1)) and
                 (n(i,j+1,k+1), n(i+1,j+1,k+1), n(i,j,k+1), n(i,j+1,k)),
    each listed as its defining vertices V0..Vd.  ``jitter`` (E, d+1, d) is added."""
    S = np.asarray(skew, dtype=np.float64)
    d = S.shape[0]
    out = []
    rng_cells = [(ex, ey) for ey in range(N) for ex in range(N)] if d == 2 else \
        [(i, j, k) for k in range(N) for j in range(N) for i in range(N)]
    node = lambda *c: S @ (np.array(c, dtype=np.float64) / N)
    for c in rng_cells:
        if d == 2:
            ex, ey = c
            out.append([node(ex, ey), node(ex + 1, ey), node(ex, ey + 1)])
            out.append([node(ex + 1, ey + 1), node(ex, ey + 1), node(ex + 1, ey)])
        else:
            i, j, k = c
            out.append([node(i, j, k), node(i + 1, j, k), node(i, j + 1, k), node(i, j, k + 1)])
            out.append([node(i, j + 1, k + 1), node(i + 1, j + 1, k + 1), node(i, j, k + 1), node(i, j + 1, k)])
    V = np.array(out)
    if jitter is not None:
        V = V + np.asarray(jitter).reshape(V.shape)
    return V


# ---------------------------------------------------------------------------
# Tetrahedra: A = {xi in [-1,1]^3 | xi1 + xi2 + xi3 <= -1} (Table t:refregions),
# collapsed by  xi1 = (1 + eta1)(1 - eta2)(1 - eta3)/4 - 1,
#               xi2 = (1 + eta2)(1 - eta3)/2 - 1,  xi3 = eta3.
# At height eta3 the cross-section is the triangle of (eta1, eta2) scaled by
# (1 - eta3)/2, so a triangle mode T_m of degree k_m (in the triangle's own
# coordinates) times ((1 - eta3)/2)^k_m is a polynomial of degree k_m on the
# tetrahedron.  Modes, in storage order: for every triangle mode m (its own
# storage order), r = 0..P - k_m:
#     T_m(eta1, eta2) ((1 - eta3)/2)^k_m                        r = 0
#     T_m(eta1, eta2) ((1 - eta3)/2)^k_m (1 + eta3)/2 P^{(2 k_m - 1, 1)}_{r-1}(eta3)   r >= 1
# then the apex (xi = (-1, -1, 1)) mode (1 + eta3)/2.  k_m: 1 for the three
# triangle vertices, p + 1 (bottom edge), q + 1 (side edges), p + q + 1
# (interior).  (P+1)(P+2)(P+3)/6 modes.  Quadrature: GLL in eta1, Gauss-Radau
# in eta2 and eta3, weights times (1 - eta2)/2 ((1 - eta3)/2)^2.
# ---------------------------------------------------------------------------
TET = "tet"


def tri_degree(P, p, q):
    """Polynomial degree of triangle mode (p, q) in the triangle's coordinates."""
    if (p, q) in ((0, 0), (P, 0), (0, P)):
        return 1
    if p == 0 or p == P:
        return q + 1
    if q == 0:
        return p + 1
    return p + q + 1


def n_tet(P):
    return (P + 1) * (P + 2) * (P + 3) // 6


def tet_modes(P):
    """Storage order: list of (triangle mode index m, r), then ('apex', 0)."""
    out = []
    for m, (p, q) in enumerate(tri_modes(P)):
        k = tri_degree(P, p, q)
        out += [(m, r) for r in range(P - k + 1)]
    out.append(("apex", 0))
    return out


def psi_c(k, r, z, deriv=False):
    """((1-z)/2)^k (r = 0) or ((1-z)/2)^k (1+z)/2 P^{(2k-1,1)}_{r-1}(z), or its derivative."""
    z = np.atleast_1d(np.asarray(z, dtype=np.float64))
    L, R = 0.5 * (1.0 - z), 0.5 * (1.0 + z)
    if r == 0:
        return -0.5 * k * L ** (k - 1) if deriv else L ** k
    J = basis.jacobi(r - 1, 2 * k - 1, 1, z)
    dJ = basis.jacobi_deriv(r - 1, 2 * k - 1, 1, z)
    if not deriv:
        return L ** k * R * J
    dLk = -0.5 * k * L ** (k - 1) if k > 0 else np.zeros_like(z)
    return dLk * R * J + L ** k * 0.5 * J + L ** k * R * dJ


def tet_basis(P, eta):
    """Tetrahedron modes at collapsed points eta (npts, 3): values and d/d eta_a (a = 1, 2, 3)."""
    T, T1, T2 = tri_basis(P, eta[:, 0], eta[:, 1])
    z = eta[:, 2]
    modes = tri_modes(P)
    out = np.empty((eta.shape[0], n_tet(P)))
    d1, d2, d3 = np.empty_like(out), np.empty_like(out), np.empty_like(out)
    for c, (m, r) in enumerate(tet_modes(P)):
        if m == "apex":
            out[:, c] = 0.5 * (1.0 + z)
            d1[:, c] = d2[:, c] = 0.0
            d3[:, c] = 0.5
            continue
        k = tri_degree(P, *modes[m])
        g, dg = psi_c(k, r, z), psi_c(k, r, z, deriv=True)
        out[:, c] = T[:, m] * g
        d1[:, c] = T1[:, m] * g
        d2[:, c] = T2[:, m] * g
        d3[:, c] = T[:, m] * dg
    return out, d1, d2, d3


def kuhn_vertices(N, skew, jitter=None):
    """Affine tetrahedra of a skewed N^3 grid, six per cube (Kuhn split along the
    main diagonal): for the permutation (a, b, c) of the axes, the tet
    (n0, n0 + e_a, n0 + e_a + e_b, n0 + e_a + e_b + e_c), listed as defining
    vertices V0..V3 with V1 and V2 swapped where needed for a positive
    orientation.  Cube c = i + N(j + N k) holds elements 6c..6c+5 in the order
    of the permutations (0,1,2), (0,2,1), (1,0,2), (1,2,0), (2,0,1), (2,1,0)."""
    S = np.asarray(skew, dtype=np.float64)
    perms = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
    E = np.eye(3)
    out = []
    for k in range(N):
        for j in range(N):
            for i in range(N):
                n0 = np.array([i, j, k], dtype=np.float64)
                for (a, b, c) in perms:
                    v = [n0, n0 + E[a], n0 + E[a] + E[b], n0 + E[a] + E[b] + E[c]]
                    v = [S @ (x / N) for x in v]
                    if np.linalg.det(np.stack([v[1] - v[0], v[2] - v[0], v[3] - v[0]], -1)) < 0:
                        v[1], v[2] = v[2], v[1]
                    out.append(v)
    V = np.array(out)
    if jitter is not None:
        V = V + np.asarray(jitter).reshape(V.shape)
    return V
