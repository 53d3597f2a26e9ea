"""Structured quad/hex meshes and their iso-parametric geometry (FP64, numpy).

Test infrastructure only (see ``oracle/__init__.py``).

Follows §2.1 (mapping paragraph): each element Omega_e is the image of the
reference region [-1,1]^d (Table t:refregions, StdQuad / StdHex) under a
parametric map x = chi_e(xi).  Curvature is represented iso-parametrically:
chi_e is the Lagrange interpolant, through the element's (P+1)^d GLL nodes,
of the exact map evaluated at those nodes.  The Jacobian J = dx/dxi at the
quadrature points is the derivative of that interpolant, evaluated with the
dense tensor-product Lagrange matrices (no sum factorisation).

Synthetic mesh: N^d elements tiling [o, o+l]^d (default [0,1]^d), element
e = ex + N(ey + N ez) (x fastest), element width h = l/N, then the shear
    3D: x' = x + amp sin(2 pi y) sin(2 pi z),  y' = y,  z' = z
    2D: x' = x + amp sin(2 pi y),              y' = y
which maps the periodic unit cube (square) onto itself.
"""
import numpy as np

from . import basis


def shear_map(dim, amp, X):
    """Exact curved map applied to affine coordinates X of shape (..., dim)."""
    Y = np.array(X, dtype=np.float64, copy=True)
    if amp != 0.0:
        if dim == 3:
            Y[..., 0] += amp * np.sin(2 * np.pi * X[..., 1]) * np.sin(2 * np.pi * X[..., 2])
        else:
            Y[..., 0] += amp * np.sin(2 * np.pi * X[..., 1])
    return Y


def tensor_matrix(dim, mats):
    """Dense tensor-product matrix of 1D matrices, one per axis.

    ``mats[a]`` has shape (rows_a, cols_a); the result maps a tensor with
    column index c0 + cols0 (c1 + cols1 c2) (axis 0 fastest) to one with row
    index r0 + rows0 (r1 + rows1 r2).  Entry = prod_a mats[a][r_a, c_a].
    """
    if dim == 2:
        A0, A1 = mats
        T = np.einsum("jq,ip->jiqp", A1, A0)
        return T.reshape(A1.shape[0] * A0.shape[0], A1.shape[1] * A0.shape[1])
    A0, A1, A2 = mats
    T = np.einsum("kr,jq,ip->kjirqp", A2, A1, A0)
    r = A2.shape[0] * A1.shape[0] * A0.shape[0]
    c = A2.shape[1] * A1.shape[1] * A0.shape[1]
    return T.reshape(r, c)


def reference_points(dim, pts):
    """Tensor grid of 1D points as an array (len(pts)^dim, dim), axis 0 fastest."""
    if dim == 2:
        X1, X0 = np.meshgrid(pts, pts, indexing="ij")
        return np.stack([X0.ravel(), X1.ravel()], axis=-1)
    X2, X1, X0 = np.meshgrid(pts, pts, pts, indexing="ij")
    return np.stack([X0.ravel(), X1.ravel(), X2.ravel()], axis=-1)


class StructuredMesh:
    """N^d elements on the unit cube with per-element order P_e and Q_e points.

    Buffers follow the library's layouts: element-major, mode index
    p + n(q + n r), quadrature index i + Q(j + Q k), with offsets
    ``coef_off`` / ``quad_off`` (length E+1) for variable order.
    """

    def __init__(self, dim, N, orders, amp=0.0, nq=None, origin=0.0, length=1.0):
        if dim not in (2, 3):
            raise ValueError("dim must be 2 or 3")
        self.dim, self.N, self.amp = dim, N, float(amp)
        self.origin, self.length = float(origin), float(length)
        self.E = N ** dim
        self.P = np.broadcast_to(np.asarray(orders, dtype=np.int64), (self.E,)).copy()
        if nq is None:
            self.Q = self.P + 2
        else:
            self.Q = np.broadcast_to(np.asarray(nq, dtype=np.int64), (self.E,)).copy()
        n = self.P + 1
        self.coef_off = np.concatenate([[0], np.cumsum(n ** dim)])
        self.quad_off = np.concatenate([[0], np.cumsum(self.Q ** dim)])
        self._geo = {}

    # element index -> integer position (ex, ey[, ez])
    def element_index(self, e):
        e = np.asarray(e)
        idx = [e % self.N, (e // self.N) % self.N]
        if self.dim == 3:
            idx.append(e // (self.N * self.N))
        return np.stack(idx, axis=-1)

    def groups(self):
        """Distinct (P, Q) pairs and the element ids that carry them."""
        out = []
        for P, Q in sorted(set(zip(self.P.tolist(), self.Q.tolist()))):
            ids = np.nonzero((self.P == P) & (self.Q == Q))[0]
            out.append((int(P), int(Q), ids))
        return out

    def physical(self, ids, ref):
        """Exact physical coordinates chi(ref) for elements ``ids``: (E, npts, dim)."""
        h = self.length / self.N
        org = self.origin + self.element_index(ids).astype(np.float64) * h
        X = org[:, None, :] + 0.5 * h * (ref[None, :, :] + 1.0)
        return shear_map(self.dim, self.amp, X)

    def nodes(self, P, ids):
        """Iso-parametric node coordinates at the (P+1)^d GLL nodes: (E, dim, n^d)."""
        z, _ = basis.gll(P + 1)
        return np.transpose(self.physical(ids, reference_points(self.dim, z)), (0, 2, 1))

    def geometry(self, P, Q, ids):
        """Geometry at the Q^d GLL quadrature points of elements ``ids``.

        Returns a dict with
          xq   (E, dim, Q^d)        physical coordinates of the quadrature points
          J    (E, Q^d, dim, dim)   J[m, a] = d x_m / d xi_a
          detJ (E, Q^d)
          Jinv (E, Q^d, dim, dim)   Jinv[a, m] = d xi_a / d x_m
          JW   (E, Q^d)             w_i w_j (w_k) det J   (weights folded in)
          G    (E, Q^d, dim, dim)   JW * (Jinv Jinv^T)    (weights folded in)
        """
        key = (P, Q, ids.tobytes())
        if key in self._geo:
            return self._geo[key]
        d = self.dim
        z, _ = basis.gll(P + 1)
        xi, w = basis.gll(Q)
        L1, dL1 = basis.lagrange(z, xi)
        Lint = tensor_matrix(d, [L1] * d)
        dL = [tensor_matrix(d, [dL1 if b == a else L1 for b in range(d)]) for a in range(d)]
        X = self.nodes(P, ids)                          # (E, d, n^d)
        xq = np.einsum("qn,emn->emq", Lint, X)
        J = np.stack([np.einsum("qn,emn->eqm", dL[a], X) for a in range(d)], axis=-1)
        detJ = np.linalg.det(J)
        Jinv = np.linalg.inv(J)
        W = tensor_matrix(d, [np.diag(w)] * d).diagonal()
        JW = W[None, :] * detJ
        G = JW[:, :, None, None] * np.einsum("eqam,eqbm->eqab", Jinv, Jinv)
        g = dict(xq=xq, J=J, detJ=detJ, Jinv=Jinv, JW=JW, G=G)
        self._geo[key] = g
        return g

    def factors_flat(self):
        """Geometric factors in the library's flat layout.

        geom   : concat over elements of [G11,G12,G13,G22,G23,G33,JW] x Q^3
                 (2D: [G11,G12,G22,JW] x Q^2)
        dxi_dx : concat over elements of [d xi_a / d x_m, index a*d + m] x Q^d
        xq     : concat over elements of [x, y(, z)] x Q^d
        """
        d = self.dim
        nf = 7 if d == 3 else 4
        pairs = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)] if d == 3 else [(0, 0), (0, 1), (1, 1)]
        geom = np.empty(nf * self.quad_off[-1])
        dxi = np.empty(d * d * self.quad_off[-1])
        xq = np.empty(d * self.quad_off[-1])
        for P, Q, ids in self.groups():
            g = self.geometry(P, Q, ids)
            nq = Q ** d
            for t, e in enumerate(ids):
                o = self.quad_off[e]
                blk = [g["G"][t, :, a, b] for a, b in pairs] + [g["JW"][t]]
                geom[nf * o: nf * (o + nq)] = np.concatenate(blk)
                dxi[d * d * o: d * d * (o + nq)] = np.transpose(g["Jinv"][t], (1, 2, 0)).reshape(-1)
                xq[d * o: d * (o + nq)] = g["xq"][t].reshape(-1)
        return geom, dxi, xq
