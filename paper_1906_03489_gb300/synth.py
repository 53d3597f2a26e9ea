"""Seeded synthetic inputs shared by the CUDA path's tests/benchmark and the oracle.

This module holds only random draws and workload sizes; it contains none of
the method's arithmetic (no basis, quadrature, geometry or operator).  Both
sides call it to obtain identical inputs:

* coefficient / field buffers: i.i.d. uniform[-1, 1) FP64 from
  ``numpy.random.default_rng(seed)``, drawn in buffer order;
* per-element orders for variable-order meshes: ``rng.integers(lo, hi + 1, E)``
  drawn first from the same generator, before any coefficient.

Workloads (structured meshes of the unit cube / square, element index
ex + N(ey + N ez); the curved ones use the shear
x' = x + amp sin(2 pi y) sin(2 pi z)):
"""
import numpy as np

WORKLOADS = {
    # 2D quads, 16x16 affine elements, P=4, Q=6: correctness workload
    "quad2d_16x16_p4": dict(dim=2, N=16, P=4, Q=6, amp=0.0, seed=1),
    # 3D hexes, 32^3 curved elements, P=4, Q=6: Helmholtz / PhysDeriv throughput
    "hex3d_32_p4": dict(dim=3, N=32, P=4, Q=6, amp=0.05, seed=2),
    # 3D hexes, 24^3 curved elements, P_e uniform in {2..8}, Q_e = P_e + 2
    "hex3d_24_varp": dict(dim=3, N=24, P=(2, 8), Q=None, amp=0.05, seed=3),
    # 3D hexes, 16^3 curved elements, P=6, Q=8: gradients of the Helmholtz loss
    "hex3d_16_p6": dict(dim=3, N=16, P=6, Q=8, amp=0.05, seed=4),
    # 3D hexes, 48^3 curved elements, P=4, Q=6: periodic C0 solve
    "hex3d_48_p4": dict(dim=3, N=48, P=4, Q=6, amp=0.05, seed=5),
    # collapsed elements: 2 N^3 affine prisms (each cube of a skewed N^3 grid cut
    # along a (y, z) diagonal), P=4, Q=6 (GLL, GLL, Gauss-Radau)
    "prism3d_24_p4": dict(dim=3, N=24, P=4, Q=6, shape="prism", seed=6),
    # 2 N^2 affine triangles of a skewed N^2 grid, P=4, Q=6 (GLL, Gauss-Radau)
    "tri2d_128_p4": dict(dim=2, N=128, P=4, Q=6, shape="tri", seed=7),
    # 6 N^3 affine tetrahedra (Kuhn split of every cube of a skewed N^3 grid),
    # P=4, Q=6 (GLL, Gauss-Radau, Gauss-Radau)
    "tet3d_16_p4": dict(dim=3, N=16, P=4, Q=6, shape="tet", seed=8),
}

# Skew of the collapsed-element grids (node (i, j[, k]) h maps to SKEW applied
# to it): the elements are then affine but not right-angled.
SKEW2 = ((1.0, 0.2), (0.1, 1.0))
SKEW3 = ((1.0, 0.2, 0.1), (0.0, 1.0, 0.15), (0.05, 0.0, 1.0))


def rng(seed):
    return np.random.default_rng(seed)


def uniform(gen, n):
    """n i.i.d. uniform[-1, 1) FP64 draws from generator ``gen``."""
    return gen.uniform(-1.0, 1.0, int(n))


def orders(gen, n_elem, lo=2, hi=8):
    """Per-element polynomial orders, uniform on {lo, ..., hi}."""
    return gen.integers(lo, hi + 1, size=int(n_elem)).astype(np.int32)
