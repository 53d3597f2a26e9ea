"""Shared builders for the GPU parity tests (seeded inputs; oracle on the CPU)."""
import numpy as np
import torch

import paper_1906_03489_gb300 as spx
from oracle import geometry
from paper_1906_03489_gb300 import mesh, synth

DEV = "cuda"


def rel_err(y, ref):
    y = y.detach().cpu().double().numpy() if isinstance(y, torch.Tensor) else np.asarray(y)
    den = np.abs(ref).max()
    return float(np.abs(y - ref).max() / (den if den > 0 else 1.0))


class Case:
    """A structured mesh on both sides: GPU plan + geometry, oracle mesh."""

    def __init__(self, dim, N, P=None, orders=None, amp=0.05, q_offset=2, basis=None):
        self.dim, self.N, self.amp = dim, N, amp
        E = N ** dim
        if orders is None:
            self.plan = spx.Plan(dim, E, order=P, q_offset=q_offset, basis=basis)
            ords = P
        else:
            self.plan = spx.Plan(dim, E, orders=orders, q_offset=q_offset, basis=basis)
            ords = orders
        self.nodes = mesh.structured_nodes(dim, N, ords, amp, device=DEV)
        self.g = spx.geom_factors(self.plan, self.nodes)
        self.plan.set_geometry(torch.float64, self.g["geom"], self.g["dxi"])
        self.plan.set_geometry(torch.float32, self.g["geom32"], self.g["dxi32"])
        self.om = geometry.StructuredMesh(dim, N, ords, amp=amp,
                                          nq=None if q_offset == 2 else np.asarray(ords) + q_offset)

    def coef(self, seed, dtype=torch.float64):
        u = synth.uniform(synth.rng(seed), self.plan.n_coef)
        return u, torch.tensor(u, device=DEV, dtype=dtype)

    def quad(self, seed, dtype=torch.float64):
        f = synth.uniform(synth.rng(seed), self.plan.n_quad)
        return f, torch.tensor(f, device=DEV, dtype=dtype)
