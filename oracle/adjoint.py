"""Loss and gradients of 0.5 ||H(lambda, kappa) u - f||^2 (FP64, numpy).

Test infrastructure only (see ``oracle/__init__.py``).

H is the unassembled, per-element Helmholtz operator of eq. e:bilinear with a
per-quadrature-point reaction field lambda(x) and diffusivity kappa(x):
    (H u)_e = Phi^T diag(JW lambda) Phi u_e
              + sum_ab (d_a Phi)^T diag(JW kappa (Jinv Jinv^T)_ab) (d_b Phi) u_e.
H is linear in u, in lambda and in kappa separately, so with r = H u - f:
    dL/du        = H^T r = H r                                (H symmetric)
    dL/dlambda_q = JW_q (Phi r)_q (Phi u)_q
    dL/dkappa_q  = JW_q sum_ab (Jinv Jinv^T)_ab,q (d_a Phi r)_q (d_b Phi u)_q
"""
import numpy as np

from . import operators


def loss(mesh, u, f, lam_field, kappa_field):
    r = operators.helmholtz(mesh, u, lam_field=lam_field, kappa_field=kappa_field) - f
    return 0.5 * float(r @ r)


def gradients(mesh, u, f, lam_field, kappa_field):
    """Returns (loss, g_u, g_lambda, g_kappa) on the flat buffers."""
    d = mesh.dim
    r = operators.helmholtz(mesh, u, lam_field=lam_field, kappa_field=kappa_field) - f
    g_u = operators.helmholtz(mesh, r, lam_field=lam_field, kappa_field=kappa_field)
    g_lam = np.zeros(mesh.quad_off[-1])
    g_kap = np.zeros(mesh.quad_off[-1])
    for P, Q, ids in mesh.groups():
        Phi, dPhi = operators.phi_matrices(d, P, Q)
        geo = mesh.geometry(P, Q, ids)
        nl = (P + 1) ** d
        U = np.stack([u[mesh.coef_off[e]: mesh.coef_off[e] + nl] for e in ids])
        R = np.stack([r[mesh.coef_off[e]: mesh.coef_off[e] + nl] for e in ids])
        gl = geo["JW"] * (R @ Phi.T) * (U @ Phi.T)
        dR = [R @ dPhi[a].T for a in range(d)]
        dU = [U @ dPhi[b].T for b in range(d)]
        gk = np.zeros_like(gl)
        for a in range(d):
            for b in range(d):
                gab = np.einsum("eqm,eqm->eq", geo["Jinv"][:, :, a, :], geo["Jinv"][:, :, b, :])
                gk += gab * dR[a] * dU[b]
        gk *= geo["JW"]
        nq = Q ** d
        for t, e in enumerate(ids):
            g_lam[mesh.quad_off[e]: mesh.quad_off[e] + nq] = gl[t]
            g_kap[mesh.quad_off[e]: mesh.quad_off[e] + nq] = gk[t]
    return 0.5 * float(r @ r), g_u, g_lam, g_kap
