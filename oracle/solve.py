"""Periodic C0 assembly and linear solves (FP64, numpy).

Test infrastructure only (see ``oracle/__init__.py``).

Assembly (§2.1 assembly paragraph: the C0 assembly operator sums the
contributions of neighbouring elements).  On the structured periodic mesh all
elements are translates of one another, so no orientation signs arise: mode p
of element e along one axis maps to global index (e P + p) mod (N P); the
right-vertex mode p = P of element e therefore coincides with the left-vertex
mode p = 0 of element e+1.  In 2D/3D the map is the tensor product of the 1D
maps.  The assembled operator is A = sum_e R_e^T H_e R_e, applied matrix-free
from the dense elemental operators.

Solvers: Jacobi-preconditioned conjugate gradients (Hestenes-Stiefel) and,
for tiny meshes, a dense Cholesky solve of the explicitly assembled matrix.
"""
import numpy as np

from . import operators


def local_to_global(mesh):
    """int64 array l2g (length sum_e n_e^d) for a uniform-order periodic mesh."""
    P = int(mesh.P[0])
    if not np.all(mesh.P == P):
        raise ValueError("periodic assembly map needs a uniform order")
    N, d = mesh.N, mesh.dim
    NP = N * P
    n = P + 1
    l2g = np.empty(mesh.coef_off[-1], dtype=np.int64)
    for e in range(mesh.E):
        pos = mesh.element_index(e)
        base = mesh.coef_off[e]
        for loc in range(n ** d):
            modes = [loc % n, (loc // n) % n] + ([loc // (n * n)] if d == 3 else [])
            g = [(pos[a] * P + modes[a]) % NP for a in range(d)]
            gi = g[0] + NP * g[1] + (NP * NP * g[2] if d == 3 else 0)
            l2g[base + loc] = gi
    return l2g


def n_global(mesh):
    return (mesh.N * int(mesh.P[0])) ** mesh.dim


def scatter_add(l2g, y_local, n):
    """Assembly R^T: global[g] = sum of local entries mapped to g."""
    out = np.zeros(n)
    np.add.at(out, l2g, y_local)
    return out


def apply_assembled(mesh, l2g, x, lam=1.0):
    """A x = R^T H R x."""
    return scatter_add(l2g, operators.helmholtz(mesh, x[l2g], lam=lam), x.size)


def jacobi_diagonal(mesh, l2g, lam=1.0):
    """diag(A)_g = sum over local entries l with l2g(l) = g of (H_e)_{ll}.

    (H_e)_{ll} = sum_q JW_q lam Phi_ql^2
                 + sum_ab sum_q JW_q (Jinv Jinv^T)_ab,q (d_a Phi)_ql (d_b Phi)_ql,
    the diagonal of the dense forms in ``operators.helmholtz_matrix``.
    """
    d = mesh.dim
    diag_local = np.zeros(mesh.coef_off[-1])
    for P, Q, ids in mesh.groups():
        Phi, dPhi = operators.phi_matrices(d, P, Q)
        geo = mesh.geometry(P, Q, ids)
        diag = lam * geo["JW"] @ (Phi ** 2)
        for a in range(d):
            for b in range(d):
                gab = np.einsum("eqm,eqm->eq", geo["Jinv"][:, :, a, :], geo["Jinv"][:, :, b, :])
                diag += (geo["JW"] * gab) @ (dPhi[a] * dPhi[b])
        n = (P + 1) ** d
        for t, e in enumerate(ids):
            diag_local[mesh.coef_off[e]: mesh.coef_off[e] + n] = diag[t]
    return scatter_add(l2g, diag_local, n_global(mesh))


def pcg(apply_A, b, diag, tol=1e-10, maxit=10000, x0=None):
    """Jacobi-preconditioned CG.  Stops when ||b - A x||_2 / ||b||_2 <= tol.

    Returns (x, iterations, relative residual of the recurrence).
    """
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - apply_A(x)
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return x, 0, 0.0
    z = r / diag
    p = z.copy()
    rz = r @ z
    it = 0
    rel = np.linalg.norm(r) / nb
    while rel > tol and it < maxit:
        Ap = apply_A(p)
        alpha = rz / (p @ Ap)
        x += alpha * p
        r -= alpha * Ap
        z = r / diag
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
        it += 1
        rel = np.linalg.norm(r) / nb
    return x, it, rel


def assembled_matrix(mesh, l2g, lam=1.0):
    """Explicit dense A = sum_e R_e^T H_e R_e (tiny meshes only)."""
    d = mesh.dim
    n = n_global(mesh)
    A = np.zeros((n, n))
    for P, Q, ids in mesh.groups():
        geo = mesh.geometry(P, Q, ids)
        nl = (P + 1) ** d
        for t, e in enumerate(ids):
            H = operators.helmholtz_matrix(d, P, Q, geo, t, lam=lam)
            g = l2g[mesh.coef_off[e]: mesh.coef_off[e] + nl]
            A[np.ix_(g, g)] += H
    return A


def manufactured_rhs(mesh, l2g, lam=1.0):
    """Assembled RHS and exact solution for u* = sin(2 pi x) sin(2 pi y) [sin(2 pi z)].

    -Laplace u* + lam u* = (lam + 4 pi^2 d) u* =: f*; the RHS is the assembled
    IProductWRTBase of f* sampled at the physical quadrature points.
    Returns (rhs_global, u_star_at_quad_points_flat).
    """
    d = mesh.dim
    _, _, xq = mesh.factors_flat()
    xq = xq.reshape(-1)
    u_star = np.zeros(mesh.quad_off[-1])
    for P, Q, ids in mesh.groups():
        nq = Q ** d
        for e in ids:
            o = mesh.quad_off[e]
            X = xq[d * o: d * (o + nq)].reshape(d, nq)
            u_star[o: o + nq] = np.prod(np.sin(2 * np.pi * X), axis=0)
    f_star = (lam + 4 * np.pi ** 2 * d) * u_star
    rhs = scatter_add(l2g, operators.iproduct(mesh, f_star), n_global(mesh))
    return rhs, u_star
