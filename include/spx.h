/*
 * spx.h -- C ABI of the GB300 (sm_103a) spectral/hp element operator library.
 *
 * The library evaluates, over every element of a quadrilateral (2D) or
 * hexahedral (3D) mesh at once, the elemental operators of the spectral/hp
 * element method of arXiv 1906.03489 (Nektar++ 5.0): BwdTrans,
 * IProductWRTBase, PhysDeriv and the Helmholtz operator H = lambda M + L,
 * with the modified C0 basis (§2.1) on Gauss-Lobatto-Legendre points, by
 * sum-factorisation (§3.3) in hand-written CUDA kernels; FwdTrans (Galerkin
 * projection) and Integral (§3.5 worked example); the adjoint of H with
 * respect to its coefficient fields; the adaptive-order error sensor (§4.2);
 * periodic C0 assembly and a Jacobi-preconditioned CG solver (§2.1,
 * implicit-type methods).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Only plain C types cross the ABI.  "device" pointers are CUDA device
 *   memory of the current device; "host" pointers are ordinary host memory.
 * - Ownership: the caller owns every data buffer.  The library never frees a
 *   caller pointer and allocates no buffer of the size of a field; a plan owns
 *   only small metadata (per-element offsets and a work list, O(E) words;
 *   per-order 1D tables and a few kilobytes of reduction partials).
 * - Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *   stream).  All device work is enqueued on it and the call returns without
 *   synchronising, unless stated otherwise.
 * - Errors: every call returns an spx_status; on any status other than SPX_OK,
 *   spx_last_error() returns a message for the calling thread.  Arguments are
 *   validated before anything is launched; nothing is launched on error.
 * - Layouts (element-major, FP64 or FP32 as selected by spx_dtype):
 *     coefficients  element e at coef_off[e], n^d values (n = P_e + 1),
 *                   mode index p + n (q + n r) (p along xi_1 fastest);
 *     quad values   element e at quad_off[e], Q^d values,
 *                   point index i + Q (j + Q k);
 *     geometry      element e at nf * quad_off[e], nf blocks of Q^d values:
 *                   3D nf = 7: G11 G12 G13 G22 G23 G33 JW,
 *                   2D nf = 4: G11 G12 G22 JW,
 *                   with JW = w_i w_j w_k det J and
 *                   G_ab = JW * sum_m (dxi_a/dx_m)(dxi_b/dx_m);
 *     dxi_dx        element e at d*d*quad_off[e], d*d blocks of Q^d values,
 *                   block a*d + m holds dxi_a/dx_m;
 *     nodes         element e at d*coef_off[e], d blocks of n^d values (the
 *                   x, y(, z) coordinates of the element's GLL nodes, node
 *                   index as the mode index).
 *   Here P_e is the element's polynomial order, Q_e = P_e + q_offset its
 *   number of GLL points per direction; coef_off / quad_off are the running
 *   sums of n^d and Q^d (see spx_plan_offsets).
 * - Supported orders: 1 <= P <= 8, q_offset in {1, 2}; 2D and 3D.
 *   Variable order (per-element P) is supported by every operator.
 * - Device buffers must be aligned to their element size; 16-byte alignment
 *   (every torch / cudaMalloc allocation) gives the fastest path.
 */
#ifndef SPX_H
#define SPX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SPX_OK = 0,
  SPX_ERR_INVALID_ARG = 1,   /* a NULL, out-of-range or inconsistent argument */
  SPX_ERR_UNSUPPORTED = 2,   /* valid request the library does not implement */
  SPX_ERR_CUDA = 3,          /* a CUDA runtime call or kernel launch failed */
  SPX_ERR_NOT_CONVERGED = 4, /* iteration limit reached before the tolerance */
  SPX_ERR_NONFINITE = 5,     /* NaN or Inf met in a residual */
  SPX_ERR_NO_MEMORY = 6,     /* host allocation or caller workspace too small */
  SPX_ERR_TIMEOUT = 7        /* a bounded device-side wait gave up */
} spx_status;

typedef enum { SPX_F64 = 0, SPX_F32 = 1 } spx_dtype;

/* Operator identifiers for spx_autotune / spx_plan_set_tile. */
typedef enum {
  SPX_OP_BWD_TRANS = 0,
  SPX_OP_IPRODUCT = 1,
  SPX_OP_PHYS_DERIV = 2,
  SPX_OP_HELMHOLTZ = 3,
  SPX_OP_HELMHOLTZ_ADJOINT = 4,
  SPX_OP_HELMHOLTZ_DIAG = 5,
  SPX_OP_FWD_TRANS = 6,
  SPX_OP_SENSOR = 7,
  SPX_OP_COUNT = 8
} spx_op;

typedef struct spx_plan spx_plan;

/* Thread-local message describing the last non-OK status of this thread. */
const char *spx_last_error(void);

/* Library version string. */
const char *spx_version(void);

/* ---------------------------------------------------------------------------
 * Basis tables (§2.1 modified basis display; §3.5 Listing lst:python GLL
 * points).  Host FP64, any output may be NULL:
 *   xi[Q], w[Q]    GLL points (ascending) and weights on [-1, 1];
 *   B[Q][P+1]      B[i][p] = phi_p(xi_i), phi_0 = (1-x)/2, phi_P = (1+x)/2,
 *                  phi_p = (1-x)/2 (1+x)/2 P^{1,1}_{p-1}(x) for 0 < p < P
 *                  (Jacobi polynomial in the standard normalisation);
 *   dB[Q][P+1]     dB[i][p] = phi_p'(xi_i);
 *   D[Q][Q]        D[i][j] = l_j'(xi_i), the collocation derivative of the
 *                  Lagrange interpolant through the GLL points.
 * Row-major, first index slowest.  Requires 1 <= P, 2 <= Q <= 16.
 * ------------------------------------------------------------------------- */
spx_status spx_basis_tables(int P, int Q, double *xi, double *w, double *B, double *dB, double *D);

/* Tables of the GLL nodal basis (§2.1, the Lagrange polynomials through the
 * P + 1 GLL points, the traditional spectral element basis), for use as a
 * caller-supplied basis (spx_basis_desc).  Host FP64, either output may be
 * NULL:
 *   B[Q][P+1]   B[i][m] = l_m(xi_i), l_m the Lagrange polynomial of node m
 *               (nodes ascending) at the Q GLL points xi_i;
 *   dB[Q][P+1]  dB[i][m] = l_m'(xi_i).
 * With Q = P + 1 the nodes are the quadrature points: B = I (collocation)
 * and dB = D.  Requires 1 <= P, 2 <= Q <= 16. */
spx_status spx_nodal_basis_tables(int P, int Q, double *B, double *dB);

/* Gauss-Radau-Legendre points x[Q] (ascending, x[0] = -1, all < 1) and
 * weights w[Q] on [-1, 1], exact for polynomials of degree <= 2Q - 2: the
 * rule of the collapsed direction of triangles and prisms (§2.1, Gauss-Radau
 * points omitting the collapsed vertex).  Host FP64; 2 <= Q <= 16. */
spx_status spx_gauss_radau(int Q, double *x, double *w);

/* ---------------------------------------------------------------------------
 * Plans: the mesh's element count, dimension and per-element orders
 * (Collections groups of same-shape, same-basis elements, §3.3; variable
 * order per element, §4.2).
 * ------------------------------------------------------------------------- */
/* Basis tables of one order supplied by the caller (the paper's BasisKey,
 * §3.5 Listing lst:python, with the basis functions of §2.1 given by their
 * values): the 1D functions phi_p, p = 0..P, of the tensor-product
 * expansion, evaluated at the Q GLL quadrature points.  FP64, row-major,
 * first index slowest:
 *   B[Q][P+1]   B[i][p] = phi_p(xi_i)                               (required)
 *   dB[Q][P+1]  dB[i][p] = phi_p'(xi_i); NULL: computed as D B.  The kernels
 *               differentiate by D B (exact for P <= Q - 1), so a given dB
 *               must equal D B to 1e-10 relative (else SPX_ERR_INVALID_ARG).
 *   D[Q][Q]     collocation derivative; NULL or the GLL one
 *   w[Q]        quadrature weights; NULL or the GLL ones
 * The quadrature is the GLL rule on Q = P + q_offset points (the geometric
 * factors fold its weights in), so D and w, when given, must equal the GLL
 * tables of spx_basis_tables to 1e-12 (else SPX_ERR_UNSUPPORTED).  Any basis
 * spanning the polynomials of degree <= P is accepted, e.g. a permutation or
 * rescaling of the modified basis, or the Lagrange (nodal) basis through the
 * P + 1 GLL points of §2.1 (the classical spectral element method; with
 * q_offset = 1 its B is the identity, which selects a collocation kernel
 * that skips every B contraction).  The library classifies each basis: the
 * modified basis's parity phi_0(-x) = phi_P(x), phi_b(-x) = (-1)^(b-1)
 * phi_b(x) selects the even-odd kernels, B = I the collocation kernels, any
 * other basis the generic sum-factorised kernels.  FP32 calls use the tables
 * rounded to FP32.  The adaptive-order sensor needs the library's own
 * modified basis (SPX_ERR_UNSUPPORTED otherwise). */
typedef struct {
  int P;                 /* order, 1..8 */
  int Q;                 /* points per direction, must be P + q_offset */
  const double *B;
  const double *dB;
  const double *D;
  const double *w;
} spx_basis_desc;

typedef enum { SPX_MEM_HOST = 0, SPX_MEM_DEVICE = 1 } spx_memory;

/* Element shapes (Table t:refregions).  Triangles T = {xi in [-1,1]^2 |
 * xi1 + xi2 <= 0} and prisms R = {xi in [-1,1]^3 | xi2 + xi3 <= 0} use the
 * collapsed coordinates of §2.1 (Fig. f:duffy): triangle xi1 = (1 + eta1)
 * (1 - eta2)/2 - 1, xi2 = eta2; prism xi1 = eta1, xi2 = (1 + eta2)(1 - eta3)/2
 * - 1, xi3 = eta3, and the modified C0 basis in those coordinates:
 *   triangle modes (p, q), p outer: p = 0: q = 0..P; p = 1..P-1: q = 0..P-1-p;
 *     p = P: q = 0..P-1 (n_T = (P+1)(P+2)/2 per element), function
 *     psi^a_p(eta1) psi^b_pq(eta2) with psi^a the modified basis of
 *     spx_basis_tables, psi^b_pq = psi^a_q for p = 0, P, ((1-z)/2)^(p+1) for
 *     q = 0 and ((1-z)/2)^(p+1) (1+z)/2 P^(2p+1,1)_(q-1)(z) otherwise; the mode
 *     (0, P) is the collapsed vertex, the function (1 + eta2)/2;
 *   prism modes a + (P+1) m: psi^a_a(xi1) times triangle mode m in (eta2, eta3);
 *   tetrahedra A = {xi in [-1,1]^3 | xi1 + xi2 + xi3 <= -1}: xi1 = (1 + eta1)
 *     (1 - eta2)(1 - eta3)/4 - 1, xi2 = (1 + eta2)(1 - eta3)/2 - 1, xi3 = eta3;
 *     for every triangle mode m (storage order) of degree k_m (1 vertices,
 *     p + 1 bottom edge, q + 1 side edges, p + q + 1 interior), r = 0..P - k_m:
 *     T_m(eta1, eta2) ((1 - eta3)/2)^k_m times 1 (r = 0) or (1 + eta3)/2
 *     P^(2 k_m - 1, 1)_(r-1)(eta3), then the apex mode (1 + eta3)/2
 *     ((P+1)(P+2)(P+3)/6 per element); Gauss-Radau in eta2 and eta3.
 * Quadrature: Q = P + 2 points per direction, GLL in the uncollapsed
 * directions, Gauss-Radau (spx_gauss_radau; it omits the collapsed vertex) in
 * the collapsed one; point index i + Q j (+ Q^2 k) over (eta1, eta2[, eta3]).
 * The geometry layout is that of quads / hexes with eta in place of xi:
 * G_ab = JW sum_m (d eta_a/dx_m)(d eta_b/dx_m), JW = w det(dx/deta) (the
 * Duffy factor included), dxi_dx block a d + m = d eta_a / d x_m.  Plans of
 * these shapes: uniform order (1..8), q_offset 2, the library's basis; the
 * operators BwdTrans, IProductWRTBase, PhysDeriv, Helmholtz (constant or
 * per-point lambda, kappa) and Integral (others: SPX_ERR_UNSUPPORTED);
 * spx_geom_factors takes straight-sided (affine) elements by their vertices. */
typedef enum { SPX_SHAPE_TENSOR = 0, SPX_SHAPE_TRI = 1, SPX_SHAPE_PRISM = 2, SPX_SHAPE_TET = 3 } spx_shape;

typedef struct {
  int dim;                    /* 2 or 3 */
  int64_t n_elem;             /* E >= 0 */
  const int32_t *elem_order;  /* host [E] orders P_e, or NULL for uniform order */
  int uniform_order;          /* P for every element when elem_order == NULL */
  int q_offset;               /* Q_e = P_e + q_offset; 1 or 2 (0 selects 2) */
  int n_basis;                /* 0: the library's modified basis (§2.1) for every order;
                                 else the number of entries of `basis` */
  const spx_basis_desc *basis; /* host array, one entry per order present (orders not
                                 present may be given too); the tables are copied */
  int basis_memory;           /* spx_memory of the table pointers B, dB, D, w */
  int shape;                  /* spx_shape: SPX_SHAPE_TENSOR (0) quadrilaterals (dim 2) /
                                 hexahedra (dim 3); SPX_SHAPE_TRI triangles (dim 2);
                                 SPX_SHAPE_PRISM prisms (dim 3) */
} spx_plan_desc;

/* Creates a plan (copies the orders and basis tables; builds offsets and the
 * launch work list on the current device).  *out receives the plan.  A
 * zero-initialised descriptor tail (n_basis = 0) selects the modified basis. */
spx_status spx_plan_create(spx_plan **out, const spx_plan_desc *desc);
/* Frees a plan (NULL is accepted). */
spx_status spx_plan_destroy(spx_plan *plan);
/* Total coefficient and quadrature-point counts (sum n^d, sum Q^d). */
spx_status spx_plan_sizes(const spx_plan *plan, int64_t *n_coef, int64_t *n_quad);
/* Host copies of the offsets, each of length E+1 (either may be NULL). */
spx_status spx_plan_offsets(const spx_plan *plan, int64_t *coef_off, int64_t *quad_off);

/* Reads the plan's device status word (synchronises the device): bit 0 set
 * means a kernel of this plan gave up a bounded wait for its input copies and
 * left its outputs incomplete; bit 1 means an index argument was out of
 * range; bit 2 means an elemental solve (FwdTrans, sensor) stopped at its
 * step cap above its tolerance.  reset != 0 clears the word afterwards.
 * (The paper has no device-side status; this reports on the collective
 * operations of §3.3 and the elemental projections of §3.5 / §4.2.) */
spx_status spx_plan_device_status(spx_plan *plan, int *status, int reset);

/* Registers caller-owned geometry buffers (device, layout above) for one
 * precision.  geom is required by IProduct, Helmholtz and the adjoint,
 * dxi_dx by PhysDeriv; either may be NULL if the operator is not used.
 * The plan keeps the pointers, not the data: the buffers must stay alive
 * and unchanged while operators run. */
spx_status spx_plan_set_geometry(spx_plan *plan, spx_dtype dtype, const void *geom, const void *dxi_dx);

/* Launch tiles: the GPU counterpart of the Collections strategy choice that
 * §3.3 makes at start-up (autotuning, COLLECTIONS DEFAULT="auto"): here the
 * strategy is fixed (sum-factorisation over element tiles) and its tile
 * shape per operator, precision and order is what is chosen.
 *
 * Overrides the launch tile of one operator/precision/order: elements per
 * batch `eb` (1..64), threads per block `nthreads` (32..512, multiple of
 * 32) and pipeline depth `stages` (1..4).  order = -1 sets every order.
 * Three kinds of kernel derive their block size from eb instead:
 *  - FP64 3D Helmholtz (and any precision with a collocation basis): eb * Q^2
 *    threads; there stages 0 reads the geometric factors from L2 (the tile's
 *    factors are prefetched when it starts) instead of staging them in shared
 *    memory, which leaves room for larger tiles, and `nthreads` (32..1024)
 *    picks the register budget of a uniform-order plan (<= 512: 128
 *    registers per thread, above: 72, for more CTAs per SM);
 *  - FP32 3D Helmholtz (element-pair kernel): ceil(eb / 2) * Q^2 threads;
 *    there `nthreads` (32..1024) is the number of threads per SM that the
 *    register budget must allow (<= 512: 128 registers per thread, <= 640:
 *    96, else 80) and `stages` (0..4) the L2 prefetch distance in tiles.  In
 *    a variable-order plan (one kernel at 128 registers, orders above the
 *    threshold one element per thread) `nthreads` picks the highest order
 *    run two elements per thread instead: <= 512: 5, <= 640: 6, else 8;
 *  - FP32 3D BwdTrans and IProductWRTBase of a uniform-order plan with the
 *    modified basis (the same element-pair layout): ceil(eb / 2) * Q^2
 *    threads, `nthreads` (32..2048) the threads per SM of the register budget
 *    (<= 768: 80 registers, <= 1024: 64, <= 1280: 48, else 40), `stages`
 *    (0..4) the L2 prefetch distance in tiles. */
spx_status spx_plan_set_tile(spx_plan *plan, spx_op op, spx_dtype dtype, int order, int eb, int nthreads,
                             int stages);

/* Times the candidate tiles of `op` for every order present in the plan on
 * the given buffers (device, sized for the operator's input and output; for
 * PhysDeriv `out` holds the d outputs one after another) and
 * keeps the fastest per order.  Synchronises the stream.  `reps` timed runs
 * per candidate (>= 1).  Autotuning at start-up, §3.3 (COLLECTIONS auto). */
spx_status spx_autotune(spx_plan *plan, spx_op op, spx_dtype dtype, const void *in, void *out, int reps,
                        void *stream);

/* Reads back the tile chosen for (op, dtype, order) (§3.3 autotuning, as
 * above). */
spx_status spx_plan_get_tile(const spx_plan *plan, spx_op op, spx_dtype dtype, int order, int *eb,
                             int *nthreads, int *stages);

/* ---------------------------------------------------------------------------
 * Geometry (§2.1 mapping paragraph): iso-parametric map chi_e given by the
 * element's nodal coordinates at its (P+1)^d GLL nodes.  For triangle and
 * prism plans the elements are affine, x = V0 + sum_c (V_c - V0)(1 + xi_c)/2,
 * and `nodes` holds element e's d + 1 vertices V0..Vd at (d + 1) d e
 * (vertex-major, V_c the image of the reference vertex one step along xi_c
 * from (-1, ..., -1)).  FP64 kernel computing,
 * at every quadrature point, J = dx/dxi of the nodal interpolant, det J,
 * J^{-1} and the folded factors of the layout above.
 *   nodes   device FP64 in  (layout above)
 *   geom    device FP64 out [nf * n_quad]          (may be NULL)
 *   dxi_dx  device FP64 out [d * d * n_quad]       (may be NULL)
 *   xq      device FP64 out [d * n_quad], physical coordinates of the
 *           quadrature points, block m = coordinate x_m   (may be NULL)
 *   geom32  device FP32 out, FP32 copy of geom      (may be NULL)
 *   dxi32   device FP32 out, FP32 copy of dxi_dx    (may be NULL)
 * ------------------------------------------------------------------------- */
spx_status spx_geom_factors(const spx_plan *plan, const double *nodes, double *geom, double *dxi_dx, double *xq,
                            float *geom32, float *dxi32, void *stream);

/* ---------------------------------------------------------------------------
 * Elemental operators, all elements at once (Collections SumFac, §3.3).
 * dtype selects FP64 or FP32 buffers, arithmetic and registered geometry.
 * ------------------------------------------------------------------------- */

/* BwdTrans (§3.3 interpolation display): u_ijk = sum_pqr B_ip B_jq B_kr c_pqr.
 * coef: device in [n_coef]; phys: device out [n_quad]. */
spx_status spx_bwd_trans(const spx_plan *plan, spx_dtype dtype, const void *coef, void *phys, void *stream);

/* IProductWRTBase (§3.3, inner products): y_pqr = sum_ijk B_ip B_jq B_kr JW_ijk f_ijk.
 * phys: device in [n_quad]; coef: device out [n_coef].  Needs geom. */
spx_status spx_iproduct(const spx_plan *plan, spx_dtype dtype, const void *phys, void *coef, void *stream);

/* PhysDeriv (§2.1, StdRegions differentiation composed with chi_e):
 * du/dx_m = sum_a (dxi_a/dx_m) D_a u at the quadrature points.
 * phys: device in [n_quad]; d0, d1 (, d2 in 3D; NULL in 2D): device out
 * [n_quad] each.  Needs dxi_dx. */
spx_status spx_phys_deriv(const spx_plan *plan, spx_dtype dtype, const void *phys, void *d0, void *d1, void *d2,
                          void *stream);

/* Helmholtz operator (eq. e:bilinear with a(u,v) = int lambda u v +
 * kappa grad u . grad v; eq. eq:filtereq is lambda = 1): per element,
 * unassembled, y_e = (M_e(lambda) + L_e(kappa)) u_e.
 *   lambda        constant reaction coefficient, used when lambda_field is NULL;
 *   lambda_field  device [n_quad] per-point lambda(x) or NULL;
 *   kappa_field   device [n_quad] per-point kappa(x) or NULL (kappa = 1);
 *   coef_in       device in [n_coef]; coef_out: device out [n_coef]
 *                 (must not alias coef_in).
 * Fields have the dtype of the call.  Needs geom. */
spx_status spx_helmholtz(const spx_plan *plan, spx_dtype dtype, double lambda, const void *lambda_field,
                         const void *kappa_field, const void *coef_in, void *coef_out, void *stream);

/* Adjoint of the Helmholtz operator with respect to its coefficient fields
 * (FP64).  For the loss 0.5 ||H(lambda,kappa) u - f||^2 with r = H u - f
 * passed as g:
 *   grad_lambda[q] = JW_q (B g)_q (B u)_q
 *   grad_kappa[q]  = sum_ab G_ab,q (d_a g)_q (d_b u)_q
 * (d_a = derivative along xi_a of the expansion).  The gradient with respect
 * to u is H g, i.e. spx_helmholtz applied to g (H is symmetric).
 * u, g: device [n_coef]; grad_lambda, grad_kappa: device out [n_quad], either
 * may be NULL.  BwdTrans of u and g is recomputed, nothing is stored by the
 * forward call.  Needs FP64 geom. */
spx_status spx_helmholtz_adjoint(const spx_plan *plan, const double *u, const double *g, double *grad_lambda,
                                 double *grad_kappa, void *stream);

/* FwdTrans: Galerkin projection of quadrature-point values onto the
 * expansion (§3.5, Listing lst:python, the FwdTrans call), per element
 *   c_e = M_e^{-1} IProductWRTBase(f)_e,  M_e = Phi^T diag(JW) Phi.
 * Solved in one launch by a preconditioned CG per element (matrix-free, in
 * shared memory), preconditioned by (1 / Jbar_e) (M1^{-1})^{(x)d} with M1 the
 * 1D mass matrix B^T diag(w) B and Jbar_e the element's mean Jacobian: exact,
 * so one step, when det J is constant on the element.  Each element stops at
 * ||M_e c - b||_2 <= tol ||b||_2 (tol 1e-14 FP64, 1e-6 FP32) or after 64 steps
 * (then bit 2 of the plan's device status word is set).
 * The coefficients are as ill-conditioned as M_e (cond about 4e7 at P = 4 in
 * 3D in this basis); the projected function BwdTrans(c) only by the square
 * root: about sqrt(cond) x unit roundoff, ~1e-12 in FP64.  In FP32 that
 * would be ~1e-4, far from the FP32 operators' 1e-5, so SPX_F32 is refused
 * (SPX_ERR_UNSUPPORTED): FwdTrans is FP64 only.
 * phys: device in [n_quad]; coef: device out [n_coef] (must not alias phys).
 * Needs geom. */
spx_status spx_fwd_trans(const spx_plan *plan, spx_dtype dtype, const void *phys, void *coef, void *stream);

/* Integral over the mesh (§3.5, Listing lst:python, the Integral call):
 * sum over elements and quadrature points of JW_q f_q, i.e. of w det J f.
 * phys: device in [n_quad] of the call's dtype; result: device, one FP64
 * value, written by the stream's work (read it after synchronising).  Sums in
 * FP64 in a fixed order (reproducible).  Calls on one plan that overlap on the
 * GPU race on the plan's partial-sum buffer: serialise them.  Needs geom. */
spx_status spx_integral(const spx_plan *plan, spx_dtype dtype, const void *phys, double *result, void *stream);

/* ---------------------------------------------------------------------------
 * Adaptive polynomial order (§4.2, adaptive polynomial order paragraph).
 * ------------------------------------------------------------------------- */

/* Element error sensor S_e = ||u_P - u_{P-1}||^2 / ||u_P||^2 of §4.2, for every
 * element of order P: u_P the expansion with coefficients `coef`, u_{P-1}
 * its L2 projection onto polynomials of degree <= P-1 per direction, norms
 * L2 on the element (quadrature with w det J).  u_{P-1} is computed in the
 * span of the order-P modes that avoid the degree-P bubble in every
 * direction (the same space), by preconditioned CG per element in one launch;
 * S_e = 0 where u_P = 0.  FP64 only.  coef: device [n_coef]; S: device out
 * [n_elem], indexed by element.  Orders >= 2 (SPX_ERR_UNSUPPORTED if an
 * element has order 1).  Needs FP64 geom. */
spx_status spx_sensor(const spx_plan *plan, const double *coef, double *S, void *stream);

/* Order update of §4.2 (host): new_orders[e] = orders[e] + 1 where S[e] >
 * upper, orders[e] - 1 where S[e] < lower, else unchanged, then clamped to
 * [p_min, p_max] (2 <= p_min <= p_max <= 8).  All arrays host, n_elem
 * entries.  The new orders define the next variable-order plan. */
spx_status spx_adapt_orders(int64_t n_elem, const double *S, const int32_t *orders, double lower, double upper,
                            int p_min, int p_max, int32_t *new_orders);

/* Diagonal of the elemental Helmholtz matrices, diag(H_e)_l for every local
 * mode: the diagonal of the elemental Galerkin matrix of the bilinear form
 * a(u, v) of §2.1 (eq. e:bilinear with the Helmholtz integrand), summed over
 * shared modes by spx_assemble it is the Jacobi preconditioner of the
 * assembled system (§2.1, implicit-type methods).  dtype selects FP64 or
 * FP32 output and geometry; lambda as in spx_helmholtz (kappa = 1).
 * out: device [n_coef].  Needs geom. */
spx_status spx_helmholtz_diag(const spx_plan *plan, spx_dtype dtype, double lambda, void *out, void *stream);

/* ---------------------------------------------------------------------------
 * C0 assembly (§2.1 assembly paragraph) and the linear solve.
 * l2g: device int32 [n_coef], global index of every local mode.
 * ------------------------------------------------------------------------- */

/* local[l] = global[l2g[l]] (dtype of the buffers); global has n_global
 * entries.  An entry of l2g outside [0, n_global) reads nothing, writes 0 and
 * sets bit 1 (value 2) of the plan's device status word. */
spx_status spx_gather(const spx_plan *plan, spx_dtype dtype, const int32_t *l2g, int64_t n_global,
                      const void *global, void *local, void *stream);

/* global[g] = sum of local[l] over l with l2g[l] = g (global is
 * overwritten; n_global entries).  Sums with FP atomics, so the order of the
 * additions (and the last bits of the result) may vary between calls; the CG
 * solver uses its own deterministic assembly.  Out-of-range entries of l2g
 * are skipped and set bit 1 of the plan's device status word. */
spx_status spx_assemble(const spx_plan *plan, spx_dtype dtype, const int32_t *l2g, int64_t n_global,
                        const void *local, void *global, void *stream);

/* Inner product <a, b> = sum_i a_i b_i of two device vectors of n values of
 * the call's dtype, at FP64 accuracy: the reductions of the conjugate-
 * gradient method for the assembled system (§2.1, implicit-type methods),
 * computed the way the solver computes them: per-thread partials (FP64 for
 * FP64 data; an unevaluated float pair, hi + lo, for FP32 data, so that no
 * FP64 instruction is spent per term), then FP64 sums across threads in a
 * fixed order, so the result is reproducible bit for bit.  For FP32 data the
 * error is about (terms per thread)^2 2^-48 + (tree depth) 2^-53 times
 * sum |a_i b_i|.  result: device, one FP64 value written by the stream's
 * work.  Uses the plan's reduction buffers: calls on one plan that overlap
 * on the GPU (this and spx_integral) race on them; serialise them. */
spx_status spx_dot(const spx_plan *plan, spx_dtype dtype, int64_t n, const void *a, const void *b, double *result,
                   void *stream);

/* Options of spx_cg_solve. */
typedef struct {
  double tol;        /* relative residual ||f - A x||_2 / ||f||_2 to reach (e.g. 1e-10) */
  int maxit;         /* iteration cap: FP64 CG (0), each inner FP32 solve (1), all FP32 iterations (2) */
  int precision;     /* 0 = all-FP64 CG; 1 = FP32 inner CG inside FP64 refinement, restarted after
                        every refinement step; 2 = FP32 CG with reliable updates: one FP32 run whose
                        recurrence residual is replaced by the FP64 residual of the corrected x
                        (x += the FP32 correction) each time it has fallen by inner_tol */
  double inner_tol;  /* residual reduction of each FP32 run between FP64 residuals (1, 2); a run
                        also stops once its residual is below half of what tol still asks */
  int max_outer;     /* cap on refinement steps / FP64 residual replacements (1, 2) */
  int use_graph;     /* 1: capture the iteration in a CUDA graph */
  int check_every;   /* iterations between host-side convergence checks (>= 1) */
} spx_cg_opts;

typedef struct {
  int iters;            /* total CG iterations (FP32 iterations for precisions 1, 2) */
  int outer_iters;      /* refinement steps / residual replacements (precisions 1, 2), else 0 */
  double rel_residual;  /* final ||f - A x||_2 / ||f||_2 computed in FP64 */
} spx_cg_result;

/* Workspace bytes spx_cg_solve needs for this plan and n_global. */
spx_status spx_cg_workspace_bytes(const spx_plan *plan, int64_t n_global, const spx_cg_opts *opts, size_t *bytes);

/* Solves A x = f with A = sum_e R_e^T H_e(lambda) R_e (assembled through
 * l2g) by Jacobi-preconditioned CG.  f: device FP64 [n_global]; x: device
 * FP64 [n_global], initial guess in, solution out.  workspace: device,
 * >= spx_cg_workspace_bytes, 256-byte aligned.  Needs geometry for FP64
 * (and FP32 when precision = 1 or 2).  Synchronises the stream (it reads residual
 * norms on the host).  Returns SPX_ERR_NOT_CONVERGED with `result` filled if
 * the caps are reached, SPX_ERR_NONFINITE on a NaN/Inf residual. */
spx_status spx_cg_solve(const spx_plan *plan, double lambda, const int32_t *l2g, int64_t n_global, const double *f,
                        double *x, void *workspace, size_t workspace_bytes, const spx_cg_opts *opts,
                        spx_cg_result *result, void *stream);

/* ---------------------------------------------------------------------------
 * Allocation-free solve.  The paper has no counterpart: this entry point
 * exists for callers that must not allocate device memory during a solve:
 * for example a program whose device memory is entirely owned by another
 * pool allocator, a latency-critical loop that cannot afford the implicit
 * device synchronisation of cudaMalloc/cudaFree, or an embedding that may
 * only use memory reserved when the library is loaded.
 *
 * Same arguments and results as spx_cg_solve, minus the workspace: the
 * solver's scratch lives in a fixed array of SPX_CG_NOALLOC_BYTES inside
 * this library's own device memory.  That array exists on every GPU that
 * loads the library, from load until the process exits.
 *   - Limit: problems whose spx_cg_workspace_bytes exceeds
 *     SPX_CG_NOALLOC_BYTES are rejected with SPX_ERR_NO_MEMORY before any
 *     work is enqueued.
 *   - Nothing is allocated or created by the call: no cudaMalloc/cudaFree,
 *     no stream, event or graph; all work runs on `stream` (use_graph is
 *     ignored) and the call synchronises that stream.
 *   - The plan's launch tiles must already exist: run spx_cg_solve once, or
 *     spx_helmholtz in each precision used and spx_helmholtz_diag in FP64,
 *     on the plan first; otherwise SPX_ERR_INVALID_ARG, x untouched.
 *   - The array is reserved on a device when this library's solver code is
 *     loaded there.  spx_plan_create loads it and looks up the array's
 *     device address with that device current (once per device and CUDA
 *     context), so a solve on a plan's device finds everything in place.
 *     Only a first call in a context where no plan was created does that
 *     set-up itself (and may reserve the array then); make such a first
 *     call before any stream capture.
 *   - Every call on a device shares the one array and it keeps the previous
 *     call's contents (the solver re-initialises what it needs); calls that
 *     overlap on the GPU (other threads or streams) race on it and must be
 *     serialised by the caller.
 * ------------------------------------------------------------------------- */
#define SPX_CG_NOALLOC_BYTES (32u * 1024u * 1024u)
spx_status spx_cg_solve_noalloc(const spx_plan *plan, double lambda, const int32_t *l2g, int64_t n_global,
                                const double *f, double *x, const spx_cg_opts *opts, spx_cg_result *result,
                                void *stream);

#ifdef __cplusplus
}
#endif

#endif /* SPX_H */
