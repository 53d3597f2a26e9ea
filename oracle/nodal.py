"""The GLL nodal (classical spectral element) basis variant (FP64, numpy).

Test infrastructure only (see ``oracle/__init__.py``).

§2.1, right after the display of the modified basis phi_p: the same 1D
functions may instead be taken as the Lagrange polynomials through the
Gauss-Lobatto-Legendre points, which gives the traditional spectral element
method, with tensor products of either basis on quadrilaterals and
hexahedra (the p-adaptivity paragraph of §4.2 notes that both admit the
boundary-interior decomposition C0 assembly uses).  Nodal basis of order P,
read here as: the Lagrange polynomials l_m through the P+1 GLL points, in the
library's tensor-product index order (m along xi_1 fastest).  On Q = P+1 GLL quadrature points (collocation) the
basis matrix is the identity, its reference gradient the collocation
derivative, and the mass matrix diag(w det J); with more points the same
definitions apply with the Lagrange values at those points.  The elemental
Helmholtz matrix is built exactly as for the modified basis (dense, from the
bilinear form), only with this basis.
"""
import numpy as np

from . import basis
from .geometry import tensor_matrix


def phi_matrices(dim, P, Q):
    """(Phi, [d_0 Phi, ...]) of the nodal basis of order P on the Q^d GLL points, each (Q^d, (P+1)^d)."""
    z, _ = basis.gll(P + 1)
    xi, _ = basis.gll(Q)
    L, dL = basis.lagrange(z, xi)
    Phi = tensor_matrix(dim, [L] * dim)
    dPhi = [tensor_matrix(dim, [dL if b == a else L for b in range(dim)]) for a in range(dim)]
    return Phi, dPhi


def helmholtz_matrix(dim, P, Q, geo, t, lam=1.0, kappa=1.0):
    """Dense H_e = M_e(lambda) + L_e(kappa) of element ``t`` of a geometry group, nodal basis."""
    Phi, dPhi = phi_matrices(dim, P, Q)
    JW, Jinv = geo["JW"][t], geo["Jinv"][t]
    M = Phi.T @ ((lam * JW)[:, None] * Phi)
    L = np.zeros_like(M)
    for a in range(dim):
        for b in range(dim):
            gab = np.einsum("qm,qm->q", Jinv[:, a, :], Jinv[:, b, :])
            L += dPhi[a].T @ ((kappa * JW * gab)[:, None] * dPhi[b])
    return M + L


def helmholtz(mesh, coef, lam=1.0, kappa=1.0, lam_field=None, kappa_field=None):
    """y_e = H_e u_e for every element (nodal coefficients, element-major buffers).

    ``lam_field`` / ``kappa_field``: optional flat per-quadrature-point fields
    that replace the constants ``lam`` / ``kappa``."""
    d = mesh.dim
    out = np.zeros_like(np.asarray(coef, dtype=np.float64))
    for P, Q, ids in mesh.groups():
        geo = mesh.geometry(P, Q, ids)
        n = (P + 1) ** d
        nq = Q ** d
        for t, e in enumerate(ids):
            s = slice(mesh.coef_off[e], mesh.coef_off[e] + n)
            q = slice(mesh.quad_off[e], mesh.quad_off[e] + nq)
            la = lam if lam_field is None else np.asarray(lam_field)[q]
            ka = kappa if kappa_field is None else np.asarray(kappa_field)[q]
            out[s] = helmholtz_matrix(d, P, Q, geo, t, la, ka) @ coef[s]
    return out


def bwd_trans(mesh, coef):
    """u_q = (Phi u_hat)_q per element with the nodal basis."""
    d = mesh.dim
    out = np.zeros(mesh.quad_off[-1])
    for P, Q, ids in mesh.groups():
        Phi, _ = phi_matrices(d, P, Q)
        n, nq = (P + 1) ** d, Q ** d
        for e in ids:
            out[mesh.quad_off[e]: mesh.quad_off[e] + nq] = Phi @ coef[mesh.coef_off[e]: mesh.coef_off[e] + n]
    return out


def iproduct(mesh, f):
    """y = Phi^T diag(w det J) f per element with the nodal basis."""
    d = mesh.dim
    out = np.zeros(mesh.coef_off[-1])
    for P, Q, ids in mesh.groups():
        Phi, _ = phi_matrices(d, P, Q)
        geo = mesh.geometry(P, Q, ids)
        n, nq = (P + 1) ** d, Q ** d
        for t, e in enumerate(ids):
            out[mesh.coef_off[e]: mesh.coef_off[e] + n] = Phi.T @ (geo["JW"][t] * f[mesh.quad_off[e]: mesh.quad_off[e] + nq])
    return out
