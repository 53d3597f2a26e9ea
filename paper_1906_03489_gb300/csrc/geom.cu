// Geometric factors of the iso-parametric map (§2.1, mapping paragraph) in FP64.
//
// Each element's map chi_e is the Lagrange interpolant through its (P+1)^d
// GLL nodes.  Its value and first derivatives at the Q^d GLL quadrature
// points are obtained by sum-factorisation with the 1D matrices
//   L[i][a] = l_a(xi_i),  dL[i][a] = l_a'(xi_i)
// (Lagrange basis through the P+1 GLL nodes, evaluated at the Q GLL points),
// then at every point: J[m][a] = d x_m / d xi_a, det J, J^{-1} and the folded
// factors JW = w det J, G_ab = JW sum_m J^{-1}_{am} J^{-1}_{bm}.
#include <cmath>
#include <vector>

#include "op_kernel.cuh"
#include "dot_acc.cuh"
#include "spx_internal.h"

namespace spx {

template <int P, int Q>
struct GeomParams {
  double L[Q * (P + 1)];
  double dL[Q * (P + 1)];
  double w[Q];
  const int32_t* ids;   // element ids (nullptr: first + j)
  int64_t first;
  int64_t count;
  int eb;
  const int64_t* coef_off;  // nullptr: uniform
  const int64_t* quad_off;
  const double* nodes;
  double* geom;
  double* dxi;
  double* xq;
  float* geom32;
  float* dxi32;
};

template <int DIM, int P, int Q>
__global__ void __launch_bounds__(256) geom_kernel(const __grid_constant__ GeomParams<P, Q> p) {
  constexpr int n = P + 1;
  constexpr int S1 = Q | 1;
  constexpr int S2 = DIM == 3 ? S1 * Q : 0;
  constexpr int WS = DIM == 3 ? S1 * Q * Q : S1 * Q;
  constexpr int ND = DIM == 3 ? n * n * n : n * n;
  constexpr int QD = DIM == 3 ? Q * Q * Q : Q * Q;
  constexpr int NFIELD = DIM == 3 ? 12 : 6;  // x_m and J[m][a]
  extern __shared__ __align__(16) double gsm[];
  // per element: nodes [DIM][ND] | fields [NFIELD][WS] | temps [5][WS]
  constexpr int PER = DIM * ND + (NFIELD + 5) * WS;
  const int tid = threadIdx.x, nthr = blockDim.x;
  __shared__ int64_t s_eid[64];
  for (int64_t t0 = int64_t(blockIdx.x) * p.eb; t0 < p.count; t0 += int64_t(gridDim.x) * p.eb) {
    const int ne = static_cast<int>(p.count - t0 < p.eb ? p.count - t0 : p.eb);
    __syncthreads();
    for (int j = tid; j < ne; j += nthr) s_eid[j] = p.ids ? p.ids[p.first + t0 + j] : p.first + t0 + j;
    __syncthreads();
    // load nodes
    for (int x = tid; x < ne * DIM * ND; x += nthr) {
      const int j = x / (DIM * ND);
      const int r = x - j * DIM * ND;
      const int64_t e = s_eid[j];
      const int64_t co = p.coef_off ? p.coef_off[e] : e * ND;
      gsm[j * PER + r] = p.nodes[DIM * co + r];
    }
    __syncthreads();
    for (int m = 0; m < DIM; ++m) {
      const double* X = gsm + m * ND;  // element stride PER
      double* F = gsm + DIM * ND;      // fields, field f of element j at j*PER + f*WS
      double* Tm = F + NFIELD * WS;    // temps
      auto fld = [&](int f) { return F + f * WS; };
      if (DIM == 3) {
        // axis 0: L -> T0, dL -> T1   (Q, n, n)
        contract_g<0, n, n, n, Q, false, 0, false, n, n * n, S1, S2>(X, BaseStride{PER}, X, BaseStride{PER}, Tm,
                                                                      BaseStride{PER}, p.L, ne, tid, nthr);
        contract_g<0, n, n, n, Q, false, 0, false, n, n * n, S1, S2>(X, BaseStride{PER}, X, BaseStride{PER},
                                                                      Tm + WS, BaseStride{PER}, p.dL, ne, tid, nthr);
        __syncthreads();
        // axis 1: T0 -L-> T2 (LL), T0 -dL-> T3 (LD), T1 -L-> T4 (DL)   (Q, Q, n)
        contract_g<1, Q, n, n, Q, false, 0, false, S1, S2, S1, S2>(Tm, BaseStride{PER}, Tm, BaseStride{PER},
                                                                    Tm + 2 * WS, BaseStride{PER}, p.L, ne, tid, nthr);
        contract_g<1, Q, n, n, Q, false, 0, false, S1, S2, S1, S2>(Tm, BaseStride{PER}, Tm, BaseStride{PER},
                                                                    Tm + 3 * WS, BaseStride{PER}, p.dL, ne, tid, nthr);
        contract_g<1, Q, n, n, Q, false, 0, false, S1, S2, S1, S2>(Tm + WS, BaseStride{PER}, Tm, BaseStride{PER},
                                                                    Tm + 4 * WS, BaseStride{PER}, p.L, ne, tid, nthr);
        __syncthreads();
        // axis 2: LL -L-> x_m, LL -dL-> J[m][2], LD -L-> J[m][1], DL -L-> J[m][0]
        // field index: x_m at m, J[m][a] at DIM + m*DIM + a
        contract_g<2, Q, Q, n, Q, false, 0, false, S1, S2, S1, S2>(Tm + 2 * WS, BaseStride{PER}, Tm, BaseStride{PER},
                                                                    fld(m), BaseStride{PER}, p.L, ne, tid, nthr);
        contract_g<2, Q, Q, n, Q, false, 0, false, S1, S2, S1, S2>(Tm + 2 * WS, BaseStride{PER}, Tm, BaseStride{PER},
                                                                    fld(DIM + m * DIM + 2), BaseStride{PER}, p.dL, ne,
                                                                    tid, nthr);
        contract_g<2, Q, Q, n, Q, false, 0, false, S1, S2, S1, S2>(Tm + 3 * WS, BaseStride{PER}, Tm, BaseStride{PER},
                                                                    fld(DIM + m * DIM + 1), BaseStride{PER}, p.L, ne,
                                                                    tid, nthr);
        contract_g<2, Q, Q, n, Q, false, 0, false, S1, S2, S1, S2>(Tm + 4 * WS, BaseStride{PER}, Tm, BaseStride{PER},
                                                                    fld(DIM + m * DIM + 0), BaseStride{PER}, p.L, ne,
                                                                    tid, nthr);
        __syncthreads();
      } else {
        contract_g<0, n, n, 1, Q, false, 0, false, n, 0, S1, 0>(X, BaseStride{PER}, X, BaseStride{PER}, Tm,
                                                                 BaseStride{PER}, p.L, ne, tid, nthr);
        contract_g<0, n, n, 1, Q, false, 0, false, n, 0, S1, 0>(X, BaseStride{PER}, X, BaseStride{PER}, Tm + WS,
                                                                 BaseStride{PER}, p.dL, ne, tid, nthr);
        __syncthreads();
        contract_g<1, Q, n, 1, Q, false, 0, false, S1, 0, S1, 0>(Tm, BaseStride{PER}, Tm, BaseStride{PER}, fld(m),
                                                                  BaseStride{PER}, p.L, ne, tid, nthr);
        contract_g<1, Q, n, 1, Q, false, 0, false, S1, 0, S1, 0>(Tm, BaseStride{PER}, Tm, BaseStride{PER},
                                                                  fld(DIM + m * DIM + 1), BaseStride{PER}, p.dL, ne,
                                                                  tid, nthr);
        contract_g<1, Q, n, 1, Q, false, 0, false, S1, 0, S1, 0>(Tm + WS, BaseStride{PER}, Tm, BaseStride{PER},
                                                                  fld(DIM + m * DIM + 0), BaseStride{PER}, p.L, ne,
                                                                  tid, nthr);
        __syncthreads();
      }
    }
    // pointwise
    for (int x = tid; x < ne * QD; x += nthr) {
      const int j = x / QD;
      const int q = x - j * QD;
      const int i0 = q % Q, i1 = (q / Q) % Q, i2 = DIM == 3 ? q / (Q * Q) : 0;
      const int w = j * PER + DIM * ND + i0 + i1 * S1 + i2 * S2;
      const int64_t e = s_eid[j];
      const int64_t qo = (p.quad_off ? p.quad_off[e] : e * QD) + q;
      double J[3][3], Ji[3][3];
      for (int m = 0; m < DIM; ++m)
        for (int a = 0; a < DIM; ++a) J[m][a] = gsm[w + (DIM + m * DIM + a) * WS];
      double det, wq;
      if (DIM == 3) {
        Ji[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
        Ji[0][1] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
        Ji[0][2] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
        Ji[1][0] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
        Ji[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
        Ji[1][2] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
        Ji[2][0] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
        Ji[2][1] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
        Ji[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        det = J[0][0] * Ji[0][0] + J[0][1] * Ji[1][0] + J[0][2] * Ji[2][0];
        wq = p.w[i0] * p.w[i1] * p.w[i2];
      } else {
        Ji[0][0] = J[1][1];
        Ji[0][1] = -J[0][1];
        Ji[1][0] = -J[1][0];
        Ji[1][1] = J[0][0];
        det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        wq = p.w[i0] * p.w[i1];
      }
      // J^{-1}[a][m] = d xi_a / d x_m
      const double inv = 1.0 / det;
      for (int a = 0; a < DIM; ++a)
        for (int m = 0; m < DIM; ++m) Ji[a][m] *= inv;
      const double jw = wq * det;
      constexpr int nf = DIM == 3 ? 7 : 4;
      double gv[7];
      int f = 0;
      for (int a = 0; a < DIM; ++a)
        for (int b = a; b < DIM; ++b) {
          double s = 0.0;
          for (int m = 0; m < DIM; ++m) s += Ji[a][m] * Ji[b][m];
          gv[f++] = jw * s;
        }
      gv[f] = jw;
      if (p.geom || p.geom32) {
        const int64_t gb = nf * (qo - q) + q;  // element block start + point
        for (int k = 0; k < nf; ++k) {
          if (p.geom) p.geom[gb + int64_t(k) * QD] = gv[k];
          if (p.geom32) p.geom32[gb + int64_t(k) * QD] = static_cast<float>(gv[k]);
        }
      }
      if (p.dxi || p.dxi32) {
        const int64_t db = DIM * DIM * (qo - q) + q;
        for (int a = 0; a < DIM; ++a)
          for (int m = 0; m < DIM; ++m) {
            if (p.dxi) p.dxi[db + int64_t(a * DIM + m) * QD] = Ji[a][m];
            if (p.dxi32) p.dxi32[db + int64_t(a * DIM + m) * QD] = static_cast<float>(Ji[a][m]);
          }
      }
      if (p.xq) {
        const int64_t xb = DIM * (qo - q) + q;
        for (int m = 0; m < DIM; ++m) p.xq[xb + int64_t(m) * QD] = gsm[w + m * WS];
      }
    }
  }
}

// Lagrange matrices through the P+1 GLL nodes at the Q GLL points.
static void lagrange_tables(int P, int Q, std::vector<double>& L, std::vector<double>& dL, std::vector<double>& w) {
  const int n = P + 1;
  std::vector<double> z(n), x(Q);
  w.assign(Q, 0.0);
  basis_tables(P, n, z.data(), nullptr, nullptr, nullptr, nullptr);
  basis_tables(P, Q, x.data(), w.data(), nullptr, nullptr, nullptr);
  std::vector<double> lam(n, 1.0);  // barycentric weights of the nodes
  for (int a = 0; a < n; ++a)
    for (int k = 0; k < n; ++k)
      if (k != a) lam[a] /= (z[a] - z[k]);
  L.assign(Q * n, 0.0);
  dL.assign(Q * n, 0.0);
  for (int i = 0; i < Q; ++i) {
    int hit = -1;
    for (int a = 0; a < n; ++a)
      if (x[i] == z[a]) hit = a;
    if (hit >= 0) {
      // point coincides with node `hit`: l_a = delta; l_a' from the
      // differentiation-matrix formula
      for (int a = 0; a < n; ++a) L[i * n + a] = a == hit ? 1.0 : 0.0;
      double diag = 0.0;
      for (int a = 0; a < n; ++a) {
        if (a == hit) continue;
        const double v = (lam[a] / lam[hit]) / (z[hit] - z[a]);
        dL[i * n + a] = v;
        diag -= v;
      }
      dL[i * n + hit] = diag;
    } else {
      // l_a(x) = ell(x) lam_a / (x - z_a), ell(x) = prod_k (x - z_k);
      // l_a'(x) = l_a(x) (sum_{k != a} 1 / (x - z_k))
      double ell = 1.0;
      for (int k = 0; k < n; ++k) ell *= (x[i] - z[k]);
      for (int a = 0; a < n; ++a) {
        const double la = ell * lam[a] / (x[i] - z[a]);
        double s = 0.0;
        for (int k = 0; k < n; ++k)
          if (k != a) s += 1.0 / (x[i] - z[k]);
        L[i * n + a] = la;
        dL[i * n + a] = la * s;
      }
    }
  }
}

template <int DIM, int P, int Q>
static spx_status geom_launch(const spx_plan* plan, const int32_t* ids, int64_t first, int64_t count,
                              const double* nodes, double* geom, double* dxi, double* xq, float* geom32, float* dxi32,
                              cudaStream_t st) {
  GeomParams<P, Q> p{};
  std::vector<double> L, dL, w;
  lagrange_tables(P, Q, L, dL, w);
  for (int i = 0; i < Q * (P + 1); ++i) {
    p.L[i] = L[i];
    p.dL[i] = dL[i];
  }
  for (int i = 0; i < Q; ++i) p.w[i] = w[i];
  p.ids = ids;
  p.first = first;
  p.count = count;
  p.coef_off = plan->uniform ? nullptr : plan->d_coef_off;
  p.quad_off = plan->uniform ? nullptr : plan->d_quad_off;
  p.nodes = nodes;
  p.geom = geom;
  p.dxi = dxi;
  p.xq = xq;
  p.geom32 = geom32;
  p.dxi32 = dxi32;
  constexpr int n = P + 1, S1 = Q | 1;
  constexpr int WS = DIM == 3 ? S1 * Q * Q : S1 * Q;
  constexpr int ND = DIM == 3 ? n * n * n : n * n;
  constexpr int NFIELD = DIM == 3 ? 12 : 6;
  const size_t per = (DIM * ND + (NFIELD + 5) * WS) * sizeof(double);
  int eb = static_cast<int>(std::min<size_t>(64, std::max<size_t>(1, (96 * 1024) / per)));
  p.eb = eb;
  const size_t smem = eb * per;
  if (smem > plan->max_smem) return fail(SPX_ERR_UNSUPPORTED, "geometry tile does not fit in shared memory");
  auto kern = geom_kernel<DIM, P, Q>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(geom)");
  const int64_t tiles = (count + eb - 1) / eb;
  const int grid = static_cast<int>(std::min<int64_t>(tiles, int64_t(plan->num_sms) * 8));
  if (grid == 0) return SPX_OK;
  kern<<<grid, 256, smem, st>>>(p);
  e = cudaGetLastError();
  return e == cudaSuccess ? SPX_OK : cuda_fail(e, "geometry kernel launch");
}

template <int DIM, int QOFF>
static spx_status geom_dispatch(int P, const spx_plan* plan, const int32_t* ids, int64_t first, int64_t count,
                                const double* nodes, double* geom, double* dxi, double* xq, float* g32, float* d32,
                                cudaStream_t st) {
  switch (P) {
#define SPX_G(PP) \
  case PP: return geom_launch<DIM, PP, PP + QOFF>(plan, ids, first, count, nodes, geom, dxi, xq, g32, d32, st);
    SPX_G(1) SPX_G(2) SPX_G(3) SPX_G(4) SPX_G(5) SPX_G(6) SPX_G(7) SPX_G(8)
#undef SPX_G
    default: return fail(SPX_ERR_UNSUPPORTED, "order out of range");
  }
}

// ---- gather: local[l] = global[l2g[l]] -------------------------------------
template <typename T>
__global__ void gather_kernel(const int32_t* __restrict__ l2g, const T* __restrict__ g, T* __restrict__ loc,
                              int64_t n, int64_t ng, int* status) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const int32_t k = l2g[i];
    if (k >= 0 && k < ng) {
      loc[i] = g[k];
    } else {  // out-of-range index: no read, zero written, status raised
      loc[i] = T(0);
      atomicOr(status, kStatusBadIndex);
    }
  }
}

template <typename T>
__global__ void assemble_atomic(const int32_t* __restrict__ l2g, const T* __restrict__ loc, T* __restrict__ g,
                                int64_t n, int64_t ng, int* status) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const int32_t k = l2g[i];
    if (k >= 0 && k < ng)
      atomicAdd(&g[k], loc[i]);
    else
      atomicOr(status, kStatusBadIndex);
  }
}

// ---- integral: sum over elements and quadrature points of JW f -----------
// One warp per element (elements warp, warp + all warps, ...), lanes over the
// element's points; sums at FP64 accuracy in a fixed order (per-thread
// partials as in dot_acc.cuh, then FP64: warp
// shuffles, per-warp then per-block sums, and the last block to finish sums
// the block partials with all its threads), so the result is reproducible
// for a given GPU.
constexpr int kIntThreads = 256;
template <typename T>
__global__ void __launch_bounds__(kIntThreads) integral_kernel(const T* __restrict__ f, const T* __restrict__ geom,
                                                               const int64_t* __restrict__ quad_off, int64_t qd_uniform,
                                                               int nf, int64_t E, double* partials,
                                                               unsigned int* ticket, double* out) {
  __shared__ double ws[kIntThreads / 32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t gw = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  DotAcc<T> part;   // FP64, or a compensated float pair for FP32 data (no FP64 instruction per term)
  if (!quad_off) {
    // uniform order: a warp takes four elements at a time (e, e + nw, e + 2 nw,
    // e + 3 nw), with the loads of all four issued before their terms are added
    const int64_t qd = qd_uniform;
    for (int64_t e = gw; e < E; e += 4 * nw) {
      for (int64_t q = lane; q < qd; q += 32) {
        T a[4], b[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int64_t ej = e + j * nw;
          a[j] = ej < E ? geom[int64_t(nf) * ej * qd + int64_t(nf - 1) * qd + q] : T(0);
          b[j] = ej < E ? f[ej * qd + q] : T(0);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) part.add(a[j], b[j]);
      }
    }
  } else {
    for (int64_t e = gw; e < E; e += nw) {
      const int64_t q0 = quad_off[e];
      const int64_t qd = quad_off[e + 1] - q0;
      const T* jw = geom + int64_t(nf) * q0 + int64_t(nf - 1) * qd;
      const T* fe = f + q0;
      for (int64_t q = lane; q < qd; q += 32) part.add(jw[q], fe[q]);
    }
  }
  double acc = part.value();
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) ws[w] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int i = 0; i < kIntThreads / 32; ++i) b += ws[i];
    partials[blockIdx.x] = b;
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;   // uniform across the block
  __threadfence();
  // the block sums the partials: thread t takes t, t + blockDim, ... in order,
  // then warp shuffles and the warp sums in warp order (a fixed order)
  double t = 0.0;
  for (unsigned i = threadIdx.x; i < gridDim.x; i += blockDim.x) t += static_cast<volatile const double*>(partials)[i];
  for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  __syncthreads();
  if (lane == 0) ws[w] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int i = 0; i < kIntThreads / 32; ++i) b += ws[i];
    *out = b;
    *ticket = 0;
  }
}

}  // namespace spx

using namespace spx;

extern "C" spx_status spx_integral(const spx_plan* plan, spx_dtype dt, const void* phys, double* result,
                                   void* stream) {
  if (!plan || !result || (plan->n_quad && !phys)) return fail(SPX_ERR_INVALID_ARG, "integral: NULL argument");
  if (dt != SPX_F64 && dt != SPX_F32) return fail(SPX_ERR_INVALID_ARG, "integral: bad dtype");
  const void* geom = plan->geom[dt];
  if (plan->E && !geom) return fail(SPX_ERR_INVALID_ARG, "integral: geometry not registered for this dtype");
  const size_t a = dt == SPX_F64 ? 8 : 4;
  if ((reinterpret_cast<uintptr_t>(phys) % a) || (reinterpret_cast<uintptr_t>(result) % 8))
    return fail(SPX_ERR_INVALID_ARG, "integral: buffer not aligned to its element size");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int nf = plan->dim == 3 ? 7 : 4;
  const int Q = plan->uP + plan->qoff;
  const int64_t qd = plan->uniform ? (plan->dim == 3 ? int64_t(Q) * Q * Q : int64_t(Q) * Q) : 0;
  const int64_t* qoff = plan->uniform ? nullptr : plan->d_quad_off;
  const int grid = plan->num_sms * kIntegralBlocksPerSM;
  if (dt == SPX_F64)
    integral_kernel<double><<<grid, kIntThreads, 0, st>>>(static_cast<const double*>(phys),
                                                           static_cast<const double*>(geom), qoff, qd, nf, plan->E,
                                                           plan->d_partials, plan->d_ticket, result);
  else
    integral_kernel<float><<<grid, kIntThreads, 0, st>>>(static_cast<const float*>(phys),
                                                          static_cast<const float*>(geom), qoff, qd, nf, plan->E,
                                                          plan->d_partials, plan->d_ticket, result);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SPX_OK : cuda_fail(e, "integral kernel launch");
}

extern "C" spx_status spx_geom_factors(const spx_plan* plan, const double* nodes, double* geom, double* dxi,
                                       double* xq, float* geom32, float* dxi32, void* stream) {
  if (!plan) return fail(SPX_ERR_INVALID_ARG, "geom_factors: NULL plan");
  if (plan->E == 0) return SPX_OK;
  if (!nodes) return fail(SPX_ERR_INVALID_ARG, "geom_factors: NULL nodes");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (plan->shape) return collapsed_geom(plan, nodes, geom, dxi, xq, geom32, dxi32, st);
  for (int P = 1; P <= kMaxP; ++P) {
    if (!plan->present[P]) continue;
    const int32_t* ids = plan->uniform ? nullptr : plan->d_ids;
    const int64_t first = plan->uniform ? 0 : plan->bucket_start[P];
    const int64_t count = plan->uniform ? plan->E : plan->bucket_start[P + 1] - plan->bucket_start[P];
    spx_status s;
    if (plan->dim == 3)
      s = plan->qoff == 1 ? geom_dispatch<3, 1>(P, plan, ids, first, count, nodes, geom, dxi, xq, geom32, dxi32, st)
                          : geom_dispatch<3, 2>(P, plan, ids, first, count, nodes, geom, dxi, xq, geom32, dxi32, st);
    else
      s = plan->qoff == 1 ? geom_dispatch<2, 1>(P, plan, ids, first, count, nodes, geom, dxi, xq, geom32, dxi32, st)
                          : geom_dispatch<2, 2>(P, plan, ids, first, count, nodes, geom, dxi, xq, geom32, dxi32, st);
    if (s != SPX_OK) return s;
  }
  return SPX_OK;
}

extern "C" spx_status spx_gather(const spx_plan* plan, spx_dtype dt, const int32_t* l2g, int64_t n_global,
                                 const void* global, void* local, void* stream) {
  if (!plan || !l2g || (plan->n_coef && (!global || !local))) return fail(SPX_ERR_INVALID_ARG, "gather: NULL argument");
  if (n_global < 0) return fail(SPX_ERR_INVALID_ARG, "gather: n_global < 0");
  if (plan->n_coef == 0) return SPX_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t n = plan->n_coef;
  const int grid = static_cast<int>(std::min<int64_t>((n + 255) / 256, int64_t(plan->num_sms) * 16));
  if (dt == SPX_F64)
    gather_kernel<double><<<grid, 256, 0, st>>>(l2g, static_cast<const double*>(global), static_cast<double*>(local), n,
                                                n_global, plan->d_status);
  else if (dt == SPX_F32)
    gather_kernel<float><<<grid, 256, 0, st>>>(l2g, static_cast<const float*>(global), static_cast<float*>(local), n,
                                               n_global, plan->d_status);
  else
    return fail(SPX_ERR_INVALID_ARG, "gather: bad dtype");
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SPX_OK : cuda_fail(e, "gather kernel launch");
}

extern "C" spx_status spx_assemble(const spx_plan* plan, spx_dtype dt, const int32_t* l2g, int64_t n_global,
                                   const void* local, void* global, void* stream) {
  if (!plan || !l2g || n_global < 0 || (plan->n_coef && !local) || (n_global && !global))
    return fail(SPX_ERR_INVALID_ARG, "assemble: bad argument");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t sz = dt == SPX_F64 ? 8 : 4;
  if (dt != SPX_F64 && dt != SPX_F32) return fail(SPX_ERR_INVALID_ARG, "assemble: bad dtype");
  cudaError_t e = cudaMemsetAsync(global, 0, n_global * sz, st);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
  const int64_t n = plan->n_coef;
  if (n == 0) return SPX_OK;
  const int grid = static_cast<int>(std::min<int64_t>((n + 255) / 256, int64_t(plan->num_sms) * 16));
  if (dt == SPX_F64)
    assemble_atomic<double><<<grid, 256, 0, st>>>(l2g, static_cast<const double*>(local), static_cast<double*>(global),
                                                  n, n_global, plan->d_status);
  else
    assemble_atomic<float><<<grid, 256, 0, st>>>(l2g, static_cast<const float*>(local), static_cast<float*>(global), n,
                                                 n_global, plan->d_status);
  e = cudaGetLastError();
  return e == cudaSuccess ? SPX_OK : cuda_fail(e, "assemble kernel launch");
}
