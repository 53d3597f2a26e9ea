"""GB300 (sm_103a) spectral/hp element operators of arXiv 1906.03489.

BwdTrans, IProductWRTBase, PhysDeriv and the Helmholtz operator H = lambda M + L
evaluated over all elements of quad/hex meshes by sum-factorised CUDA kernels
behind a C ABI (include/spx.h); FwdTrans (Galerkin projection) and Integral;
the adaptive-order error sensor and order update;
adjoint of H with respect to its coefficient fields behind ``torch.autograd``;
periodic C0 assembly and a mixed-precision Jacobi-PCG solver.
"""
from ._lib import SpxError, lib  # noqa: F401
from .binding import (Plan, assemble, basis_tables, bwd_trans, cg_solve, cg_workspace_bytes, dot,  # noqa: F401
                      fwd_trans, gather, gauss_radau, geom_factors, helmholtz, helmholtz_adjoint, helmholtz_diag, integral,
                      iproduct, nodal_basis_tables, phys_deriv, sensor, adapt_orders)
from .autograd import HelmholtzFn, helmholtz_ad  # noqa: F401
