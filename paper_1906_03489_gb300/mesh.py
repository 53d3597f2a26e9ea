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
