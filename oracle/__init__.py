"""Dense FP64 CPU oracle for the spectral/hp element operators (arXiv 1906.03489).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` use it.  It shares no code, table or helper with the CUDA path
in ``paper_1906_03489_gb300``; the only thing both sides consume is the seeded
input generator ``paper_1906_03489_gb300/synth.py`` (random draws, no method
arithmetic).

What it computes, and the passage each part follows:

* ``basis``      GLL points/weights (Listing lst:python, §3.5), Jacobi
                 polynomials, the modified C0 basis phi_p (§2.1 display of
                 phi_p) and Lagrange interpolation/derivative matrices.
* ``geometry``   structured (optionally curved) meshes, the iso-parametric map
                 chi_e and its Jacobian at quadrature points (§2.1, mapping
                 paragraph; reference regions Table t:refregions).
* ``operators``  dense elemental matrices Phi, d_a Phi, M_e, L_e, H_e = M + L
                 and the four operators BwdTrans, IProductWRTBase, PhysDeriv,
                 Helmholtz, plus FwdTrans and Integral (§2.1 weak form
                 eq:var / e:bilinear; §3.3 operator list; §3.4 eq:filtereq).
                 No sum-factorisation anywhere: every operator is a dense
                 matrix (or dense mat-vec) built from the definitions.
* ``solve``      periodic C0 assembly (§2.1 assembly paragraph), Jacobi PCG
                 and a dense Cholesky solve for tiny meshes.
* ``adapt``      the element error sensor S_e = ||u_P - u_{P-1}||^2 / ||u_P||^2
                 of the adaptive polynomial order procedure and its order
                 update (§4.2), with u_{P-1} the dense L^2 projection onto the
                 order P - 1 basis.
* ``nodal``      the GLL nodal (Lagrange, classical spectral element) basis
                 variant of the elemental Helmholtz matrix (§2.1 names the
                 Lagrange interpolant basis beside the modified one).
* ``collapsed``  collapsed-coordinate triangles and prisms (§2.1, Fig.
                 f:duffy, Table t:refregions): the modified C0 basis in
                 collapsed coordinates, Gauss-Radau quadrature in the
                 collapsed direction, affine elements, dense BwdTrans,
                 IProductWRTBase, PhysDeriv and Helmholtz.
* ``adjoint``    gradients of 0.5*||H(lambda,kappa)u - f||^2 with respect to
                 u, lambda(x) and kappa(x), by differentiating the dense
                 forms of eq. e:bilinear.

Pins (independent checks of this oracle against closed forms, invariants,
the paper's worked example and brute force) live in ``tests/test_oracle_*.py``.
Parity: every function here is pinned; none is "parity unpinned".
"""
