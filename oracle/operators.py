"""Dense elemental operators of the spectral/hp method (FP64, numpy).

Test infrastructure only (see ``oracle/__init__.py``).

Every operator is written as the dense matrix its definition gives; there is
no sum-factorisation.  Definitions followed:

* Tensor-product expansion u(xi) = sum_pqr u_pqr phi_p(xi1) phi_q(xi2) phi_r(xi3)
  (§2.1 tensorial basis; §3.3 interpolation display).  Phi is the dense
  Q^d x n^d matrix of basis values at the quadrature points; d_a Phi uses
  phi' along axis a.
* BwdTrans:        u_q = (Phi u_hat)_q                      (§3.3, "transformations")
* IProductWRTBase: y = Phi^T W f,  W = diag(w det J)        (§3.3, "inner products")
* PhysDeriv:       (du/dx_m)_q = sum_a (dxi_a/dx_m)_q (D_a u)_q, with D_a the
                   dense collocation derivative along axis a (§2.1 StdRegions
                   differentiation composed with the map chi_e).
* Helmholtz:       H_e = M_e(lambda) + L_e(kappa),
                   M_e = Phi^T diag(w detJ lambda) Phi,
                   L_e = sum_ab (d_a Phi)^T diag(w detJ kappa (Jinv Jinv^T)_ab) (d_b Phi),
                   the Galerkin matrix of the bilinear form
                   a(u,v) = int lambda u v + kappa grad u . grad v  (eq:var, e:bilinear);
                   eq:filtereq is the case lambda = 1, kappa = (Delta lambda / 2 pi)^2.
* FwdTrans:        u_hat = M_e^{-1} IProduct(f)  (Galerkin projection, Listing lst:python)
* Integral:        sum_q w_q det J_q f_q          (Listing lst:python)
"""
import numpy as np

from . import basis
from .geometry import tensor_matrix


def phi_matrices(dim, P, Q):
    """(Phi, [d_0 Phi, ..., d_{dim-1} Phi]) on the Q^d GLL points, each (Q^d, n^d)."""
    xi, _ = basis.gll(Q)
    B = basis.modified_basis(P, xi)
    dB = basis.modified_basis_deriv(P, xi)
    Phi = tensor_matrix(dim, [B] * dim)
    dPhi = [tensor_matrix(dim, [dB if b == a else B for b in range(dim)]) for a in range(dim)]
    return Phi, dPhi


def collocation_matrices(dim, Q):
    """Dense Q^d x Q^d collocation derivative along each axis."""
    D1 = basis.collocation_derivative(Q)
    I = np.eye(Q)
    return [tensor_matrix(dim, [D1 if b == a else I for b in range(dim)]) for a in range(dim)]


def _field(val, shape):
    """A scalar coefficient or a per-quadrature-point field, as an array of ``shape``."""
    if val is None:
        return np.ones(shape)
    return np.broadcast_to(np.asarray(val, dtype=np.float64), shape)


def helmholtz_matrix(dim, P, Q, geo, t, lam=1.0, kappa=1.0):
    """Dense H_e = M_e + L_e of element ``t`` of a geometry group (n^d x n^d)."""
    Phi, dPhi = phi_matrices(dim, P, Q)
    JW, Jinv = geo["JW"][t], geo["Jinv"][t]
    nq = JW.size
    lam_q = _field(lam, (nq,))
    kap_q = _field(kappa, (nq,))
    M = Phi.T @ (JW[:, None] * lam_q[:, None] * Phi)
    L = np.zeros_like(M)
    for a in range(dim):
        for b in range(dim):
            gab = np.einsum("qm,qm->q", Jinv[:, a, :], Jinv[:, b, :])
            L += dPhi[a].T @ ((JW * kap_q * gab)[:, None] * dPhi[b])
    return M + L


def mass_matrix(dim, P, Q, geo, t):
    return helmholtz_matrix(dim, P, Q, geo, t, lam=1.0, kappa=0.0)


# ----------------------------------------------------------------------------
# Whole-mesh operators on the flat, element-major buffers.  Each loops over the
# distinct (P, Q) groups of the mesh and applies the dense matrices as dense
# mat-vecs (one matmul over all elements of a group).
# ----------------------------------------------------------------------------

def _gather(buf, off, ids, size):
    return np.stack([buf[off[e]: off[e] + size] for e in ids]) if len(ids) else np.zeros((0, size))


def _scatter(out, off, ids, vals):
    for t, e in enumerate(ids):
        out[off[e]: off[e] + vals.shape[1]] = vals[t]


def bwd_trans(mesh, coef):
    d = mesh.dim
    out = np.zeros(mesh.quad_off[-1])
    for P, Q, ids in mesh.groups():
        Phi, _ = phi_matrices(d, P, Q)
        U = _gather(coef, mesh.coef_off, ids, (P + 1) ** d)
        _scatter(out, mesh.quad_off, ids, U @ Phi.T)
    return out


def iproduct(mesh, f):
    d = mesh.dim
    out = np.zeros(mesh.coef_off[-1])
    for P, Q, ids in mesh.groups():
        Phi, _ = phi_matrices(d, P, Q)
        geo = mesh.geometry(P, Q, ids)
        F = _gather(f, mesh.quad_off, ids, Q ** d)
        _scatter(out, mesh.coef_off, ids, (geo["JW"] * F) @ Phi)
    return out


def phys_deriv(mesh, f):
    """Returns a list of ``dim`` flat arrays, d f / d x_m at the quadrature points."""
    d = mesh.dim
    outs = [np.zeros(mesh.quad_off[-1]) for _ in range(d)]
    for P, Q, ids in mesh.groups():
        Dm = collocation_matrices(d, Q)
        geo = mesh.geometry(P, Q, ids)
        F = _gather(f, mesh.quad_off, ids, Q ** d)
        ref = [F @ Dm[a].T for a in range(d)]          # d f / d xi_a
        for m in range(d):
            dm = sum(geo["Jinv"][:, :, a, m] * ref[a] for a in range(d))
            _scatter(outs[m], mesh.quad_off, ids, dm)
    return outs


def helmholtz(mesh, coef, lam=1.0, lam_field=None, kappa_field=None):
    """y_e = H_e(lambda, kappa) u_e for every element, as dense mat-vecs.

    ``lam`` scales the mass term; ``lam_field`` / ``kappa_field`` are optional
    flat per-quadrature-point fields (lambda(x) replaces the constant ``lam``
    when given; kappa defaults to 1).
    """
    d = mesh.dim
    out = np.zeros(mesh.coef_off[-1])
    for P, Q, ids in mesh.groups():
        Phi, dPhi = phi_matrices(d, P, Q)
        geo = mesh.geometry(P, Q, ids)
        nq = Q ** d
        U = _gather(coef, mesh.coef_off, ids, (P + 1) ** d)
        lam_q = _gather(lam_field, mesh.quad_off, ids, nq) if lam_field is not None else lam
        kap_q = _gather(kappa_field, mesh.quad_off, ids, nq) if kappa_field is not None else 1.0
        u = U @ Phi.T
        du = [U @ dPhi[a].T for a in range(d)]
        y = (geo["JW"] * lam_q * u) @ Phi
        for a in range(d):
            g = np.zeros_like(u)
            for b in range(d):
                g += np.einsum("eqm,eqm->eq", geo["Jinv"][:, :, a, :], geo["Jinv"][:, :, b, :]) * du[b]
            y += (geo["JW"] * kap_q * g) @ dPhi[a]
        _scatter(out, mesh.coef_off, ids, y)
    return out


def fwd_trans(mesh, f):
    """Galerkin projection: u_hat_e = M_e^{-1} IProduct(f)_e (dense Cholesky)."""
    d = mesh.dim
    rhs = iproduct(mesh, f)
    out = np.zeros_like(rhs)
    for P, Q, ids in mesh.groups():
        geo = mesh.geometry(P, Q, ids)
        n = (P + 1) ** d
        for t, e in enumerate(ids):
            M = mass_matrix(d, P, Q, geo, t)
            c = np.linalg.cholesky(M)
            b = rhs[mesh.coef_off[e]: mesh.coef_off[e] + n]
            out[mesh.coef_off[e]: mesh.coef_off[e] + n] = np.linalg.solve(c.T, np.linalg.solve(c, b))
    return out


def integral(mesh, f):
    """Sum over elements and quadrature points of w det J f."""
    d = mesh.dim
    total = 0.0
    for P, Q, ids in mesh.groups():
        geo = mesh.geometry(P, Q, ids)
        F = _gather(f, mesh.quad_off, ids, Q ** d)
        total += float(np.sum(geo["JW"] * F))
    return total
