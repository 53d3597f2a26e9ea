"""Synthetic structured meshes for the library's tests and benchmark.

N^d elements on [o, o+l]^d (default the unit cube), element index
ex + N(ey + N ez), each element's nodal coordinates sampled at its (P+1)^d GLL
nodes (node index = mode index p + n(q + n r)) from the map
    3D: x' = x + amp sin(2 pi y) sin(2 pi z),  2D: x' = x + amp sin(2 pi y),
which is the iso-parametric description of the curved mesh the geometry
kernel consumes.  GLL nodes come from the library's own basis tables.
"""
import numpy as np
import torch

from . import synth
from .binding import basis_tables


def structured_nodes(dim, N, orders, amp=0.0, origin=0.0, length=1.0, device="cuda"):
    """FP64 tensor of nodal coordinates in the library's node layout."""
    E = N ** dim
    orders = np.broadcast_to(np.asarray(orders, dtype=np.int64), (E,))
    n_e = (orders + 1) ** dim
    off = np.concatenate([[0], np.cumsum(n_e)])
    out = torch.empty(dim * int(off[-1]), dtype=torch.float64, device=device)
    h = length / N
    e_all = np.arange(E)
    pos = np.stack([e_all % N, (e_all // N) % N] + ([e_all // (N * N)] if dim == 3 else []), axis=1)
    for P in np.unique(orders):
        P = int(P)
        ids = np.nonzero(orders == P)[0]
        z = torch.tensor(basis_tables(P, P + 1)["xi"], dtype=torch.float64, device=device)
        n = P + 1
        if dim == 3:
            r, q, p = torch.meshgrid(z, z, z, indexing="ij")
            ref = [p.reshape(-1), q.reshape(-1), r.reshape(-1)]
        else:
            q, p = torch.meshgrid(z, z, indexing="ij")
            ref = [p.reshape(-1), q.reshape(-1)]
        org = origin + torch.tensor(pos[ids], dtype=torch.float64, device=device) * h   # (Eg, dim)
        X = [org[:, a:a + 1] + 0.5 * h * (ref[a][None, :] + 1.0) for a in range(dim)]    # (Eg, n^d) each
        if amp != 0.0:
            if dim == 3:
                X[0] = X[0] + amp * torch.sin(2 * np.pi * X[1]) * torch.sin(2 * np.pi * X[2])
            else:
                X[0] = X[0] + amp * torch.sin(2 * np.pi * X[1])
        blk = torch.stack(X, dim=1).reshape(len(ids), dim * n ** dim)                     # (Eg, dim*n^d)
        starts = torch.tensor(dim * off[ids], dtype=torch.int64, device=device)
        idx = starts[:, None] + torch.arange(dim * n ** dim, device=device)[None, :]
        out[idx.reshape(-1)] = blk.reshape(-1)
    return out


def periodic_l2g(dim, N, P, device="cuda"):
    """int32 local-to-global map of the periodic C0 assembly of a uniform-order mesh.

    Mode p of element e along an axis maps to (e P + p) mod (N P); the map is
    the tensor product over axes (no orientation signs: all elements are
    translates of one another).
    """
    n = P + 1
    NP = N * P
    e = torch.arange(N ** dim, device=device)
    pos = [e % N, (e // N) % N] + ([e // (N * N)] if dim == 3 else [])
    loc = torch.arange(n ** dim, device=device)
    modes = [loc % n, (loc // n) % n] + ([loc // (n * n)] if dim == 3 else [])
    g = [(pos[a][:, None] * P + modes[a][None, :]) % NP for a in range(dim)]
    gi = g[0] + NP * g[1] + (NP * NP * g[2] if dim == 3 else 0)
    return gi.reshape(-1).to(torch.int32).contiguous(), NP ** dim


def collapsed_vertices(shape, N, jitter=None, device="cuda"):
    """Defining vertices V0..Vd of affine triangles ("tri", 2 N^2), prisms
    ("prism", 2 N^3) or tetrahedra ("tet", 6 N^3, the Kuhn split of every cube
    along its main diagonal): FP64 tensor (E, d+1, d), the library's vertex layout.

    Grid nodes (i, j[, k]) / N pass through the skew synth.SKEW2 / SKEW3.  Each
    square (cube) holds two elements, element 2 c + t for cell c = ex + N(ey
    [+ N ez]): a triangle V0 = n(ex, ey), V1 = n(ex+1, ey), V2 = n(ex, ey+1) and
    V0 = n(ex+1, ey+1), V1 = n(ex, ey+1), V2 = n(ex+1, ey); a prism over the
    (y, z) triangle V0 = n(i, j, k), V1 = n(i+1, j, k), V2 = n(i, j+1, k),
    V3 = n(i, j, k+1) and V0 = n(i, j+1, k+1), V1 = n(i+1, j+1, k+1),
    V2 = n(i, j, k+1), V3 = n(i, j+1, k).  ``jitter``: optional (E, d+1, d)
    array added to the vertices (elements stay affine, the mesh need not stay
    conforming)."""
    h = 1.0 / N
    if shape == "tri":
        S = np.array(synth.SKEW2)
        ey, ex = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
        ex, ey = ex.ravel(), ey.ravel()
        node = lambda i, j: (np.stack([i, j], -1) * h) @ S.T
        lo = np.stack([node(ex, ey), node(ex + 1, ey), node(ex, ey + 1)], 1)
        up = np.stack([node(ex + 1, ey + 1), node(ex, ey + 1), node(ex + 1, ey)], 1)
    elif shape == "prism":
        S = np.array(synth.SKEW3)
        ez, ey, ex = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
        i, j, k = ex.ravel(), ey.ravel(), ez.ravel()
        node = lambda a, b, c: (np.stack([a, b, c], -1) * h) @ S.T
        lo = np.stack([node(i, j, k), node(i + 1, j, k), node(i, j + 1, k), node(i, j, k + 1)], 1)
        up = np.stack([node(i, j + 1, k + 1), node(i + 1, j + 1, k + 1), node(i, j, k + 1), node(i, j + 1, k)], 1)
    elif shape == "tet":
        # six tetrahedra per cube along its main diagonal: for the axis order
        # (a, b, c), n0, n0 + e_a, n0 + e_a + e_b, n0 + e_a + e_b + e_c; the
        # second and third vertex swapped where that gives a positive volume
        S = np.array(synth.SKEW3)
        ez, ey, ex = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
        n0 = np.stack([ex.ravel(), ey.ravel(), ez.ravel()], -1).astype(np.float64)
        E3 = np.eye(3)
        tets = []
        for a, b, c in ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)):
            v = [n0, n0 + E3[a], n0 + E3[a] + E3[b], n0 + E3[a] + E3[b] + E3[c]]
            v = [(x * h) @ S.T for x in v]
            det = np.linalg.det(np.stack([v[1] - v[0], v[2] - v[0], v[3] - v[0]], -1))
            swap = det < 0
            v1 = np.where(swap[:, None], v[2], v[1])
            v2 = np.where(swap[:, None], v[1], v[2])
            tets.append(np.stack([v[0], v1, v2, v[3]], 1))
        V = np.stack(tets, 1).reshape(-1, 4, 3)
        if jitter is not None:
            V = V + np.asarray(jitter).reshape(V.shape)
        return torch.tensor(V, dtype=torch.float64, device=device).contiguous()
    else:
        raise ValueError("shape must be 'tri', 'prism' or 'tet'")
    V = np.stack([lo, up], 1).reshape(-1, lo.shape[1], lo.shape[2])
    if jitter is not None:
        V = V + np.asarray(jitter).reshape(V.shape)
    return torch.tensor(V, dtype=torch.float64, device=device).contiguous()
