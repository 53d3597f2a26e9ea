"""Adaptive polynomial order: the element error sensor and the order update (FP64, numpy).

Test infrastructure only (see ``oracle/__init__.py``).

Follows §4.2 (adaptive polynomial order paragraph and its display of S_e):
for the solution u_P of order P on element Omega_e,

    S_e = ||u_P - u_{P-1}||_2^2 / ||u_P||_2^2,

where u_{P-1} is the projection of u_P onto polynomials of order P - 1 and
||.||_2 the L^2 norm on the element.  Read here as: u_{P-1} is the L^2
projection onto the tensor-product space of degree <= P - 1 per direction,
spanned by the modified basis of order P - 1, and every integral is the
element's quadrature with the weights w det J of u_P's own Q points (which
integrate u_P u_{P-1} exactly on affine elements, degree 2P - 1 <= 2Q - 3).
After each sensor evaluation, P is raised by one where S_e is above a chosen
threshold, lowered by one where it is below another, and kept within
[P_min, P_max].  Orders P >= 2 (order 0 has no modified basis).  Where
u_P = 0 the ratio is undefined; S_e = 0 is taken there (nothing to refine).
"""
import numpy as np

from . import basis
from .geometry import tensor_matrix


def sensor(mesh, coef):
    """S_e for every element of ``mesh`` from the coefficients ``coef`` (dense)."""
    d = mesh.dim
    S = np.zeros(mesh.E)
    for P, Q, ids in mesh.groups():
        if P < 2:
            raise ValueError("the sensor needs P >= 2")
        geo = mesh.geometry(P, Q, ids)
        xi, _ = basis.gll(Q)
        PhiP = tensor_matrix(d, [basis.modified_basis(P, xi)] * d)          # order P at the Q^d points
        PhiL = tensor_matrix(d, [basis.modified_basis(P - 1, xi)] * d)      # order P - 1, same points
        n = (P + 1) ** d
        for t, e in enumerate(ids):
            W = geo["JW"][t]
            u = PhiP @ coef[mesh.coef_off[e]: mesh.coef_off[e] + n]
            ML = PhiL.T @ (W[:, None] * PhiL)                                 # mass matrix of order P - 1
            c = np.linalg.solve(ML, PhiL.T @ (W * u))                        # L^2 projection
            r = u - PhiL @ c
            uu = float(W @ (u * u))
            S[e] = float(W @ (r * r)) / uu if uu > 0 else 0.0      # no content: nothing to refine
    return S


def adapt_orders(S, orders, lower, upper, p_min, p_max):
    """New orders: P + 1 where S_e > upper, P - 1 where S_e < lower, clamped to [p_min, p_max]."""
    S = np.asarray(S, dtype=np.float64)
    P = np.asarray(orders, dtype=np.int64).copy()
    P[S > upper] += 1
    P[S < lower] -= 1
    return np.clip(P, p_min, p_max).astype(np.int32)
