// FP32 Helmholtz operator H = lambda M + L on hexahedra, two elements per
// thread in packed f32x2 arithmetic (§3.3 collective evaluation, SumFac
// strategy; sum-factorisation display of §3.3 for the three 1D contractions).
//
// Every value a thread handles is a float2 holding the same entry of two
// elements of the tile (an element pair), so each FFMA2 / LDS.64 / STS.64
// does the work of two scalar instructions: the kernel is issue bound on
// CUDA cores (the contractions are 5x6 / 6x6 matrices, too small for the
// tensor cores to pay), and the pair layout halves its instruction count per
// element.  Thread (a, b) of a pair plays the column / pencil roles of the
// role-based body: column owner of quadrature column (i, j) = (a, b) (xi_3
// contractions, xi_3 gradient and the pointwise geometric factors in
// registers), pencil owner along xi_1 at (j, k) = (b, a) and along xi_2 at
// (i, k) = (a, b).  Nine phases, one CTA barrier each, through three
// shared-memory buffers per pair laid out free of bank conflicts
// (PairLayout in kernel_params.h).
//
// Each tile's geometric factors (86% of the bytes) are staged into one
// shared-memory slot by a 1D bulk copy (TMA) that thread 0 issues as soon as
// the previous tile's pointwise phase has released the slot, so it has eight
// phases to land; the wait for it is bounded (a copy that never lands sets the
// plan's status word, nothing hangs).  Coefficients are read straight from
// HBM (coalesced, read once), outputs stored straight to HBM.  Optionally one
// thread issues L2 prefetches of the tiles `pf` tiles ahead.
#pragma once
#include "op_kernel.cuh"

namespace spx {

__device__ __forceinline__ float2 f2fma(float a, float2 x, float2 y) { return __ffma2_rn(make_float2(a, a), x, y); }
__device__ __forceinline__ float2 f2fmav(float2 a, float2 x, float2 y) { return __ffma2_rn(a, x, y); }
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }

// L2 prefetch of [g, g + bytes): the 16-byte aligned interior only.
__device__ __forceinline__ void prefetch_l2(const void* g, uint64_t bytes) {
  const uintptr_t a0 = (reinterpret_cast<uintptr_t>(g) + 15) & ~uintptr_t(15);
  const uintptr_t a1 = (reinterpret_cast<uintptr_t>(g) + bytes) & ~uintptr_t(15);
  for (uintptr_t a = a0; a < a1;) {
    const uint32_t n = static_cast<uint32_t>(a1 - a > (1u << 20) ? (1u << 20) : a1 - a);
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"(n) : "memory");
    a += n;
  }
}

template <int PLO, int PHI, int QOFF>
struct PairParams {
  KParams<float, PLO, PHI, QOFF> k;
  int pf;                          // L2 prefetch distance in tiles (0: none)
  uint32_t off_a, off_c, off_f;    // byte offsets of the work buffers
  uint32_t off_geo;                // byte offset of the geometry slot
};

// L2 prefetch of every input range of tile `ti`.
template <int DIM, class Prm>
__device__ __forceinline__ void prefetch_tile(const Prm& p, int ti, int QOFF) {
  const Tile t = p.tiles[ti];
  const int P = t.P, Q = P + QOFF;
  const int64_t nd = int64_t(P + 1) * (P + 1) * (P + 1), qd = int64_t(Q) * Q * Q;
  for (int j = 0; j < t.count; ++j) {
    const int64_t e = elem_id(p, t, j);
    const int64_t co = coef_off_of<DIM>(p, e, P), qo = quad_off_of<DIM>(p, e, Q);
    prefetch_l2(p.in0 + co, nd * 4);
    prefetch_l2(p.geom + 7 * qo, 7 * qd * 4);
    if (p.lam_f) prefetch_l2(p.lam_f + qo, qd * 4);
    if (p.kap_f) prefetch_l2(p.kap_f + qo, qd * 4);
  }
}

// Geometry of tile `ti` into the slot (thread 0): one 1D bulk copy of a
// contiguous tile's [count][7][Q^3] range (one instruction keeps thread 0's
// detour short: the other warps wait for it at the next barrier), else one
// copy per element into regions of geo_erb bytes (kernel_params.h).  Ragged
// head / tail words (< 16 bytes, when a range is not 16-byte aligned in HBM)
// are copied by geo_fixup once the bulk part has landed.
template <class Prm>
__device__ void geo_issue(const Prm& p, char* slot, uint64_t* bar, int ti, int QOFF) {
  const Tile t = p.tiles[ti];
  const int P = t.P, Q = P + QOFF;
  const uint32_t eblk = geo_eblk(Q), erb = geo_erb(Q);
  if (t.contig) {
    const float* g0 = p.geom + 7 * quad_off_of<3>(p, elem_id(p, t, 0), Q);
    mbar_arrive_expect_tx(bar, stage_bytes(g0, t.count * eblk));
    stage_issue(slot, g0, t.count * eblk, bar);
    return;
  }
  uint32_t tx = 0;
  for (int j = 0; j < t.count; ++j) tx += stage_bytes(p.geom + 7 * quad_off_of<3>(p, elem_id(p, t, j), Q), eblk);
  mbar_arrive_expect_tx(bar, tx);
  for (int j = 0; j < t.count; ++j)
    stage_issue(slot + j * erb, p.geom + 7 * quad_off_of<3>(p, elem_id(p, t, j), Q), eblk, bar);
}

// Shared-memory address of element j's staged geometry block.
template <class Prm>
__device__ __forceinline__ const float* geo_staged(const Prm& p, const char* slot, const Tile& t, int j, int Q) {
  if (t.contig) {
    const float* g0 = p.geom + 7 * quad_off_of<3>(p, elem_id(p, t, 0), Q);
    return reinterpret_cast<const float*>(slot + (reinterpret_cast<uintptr_t>(g0) & 15) + j * geo_eblk(Q));
  }
  const float* g = p.geom + 7 * quad_off_of<3>(p, elem_id(p, t, j), Q);
  return reinterpret_cast<const float*>(slot + j * geo_erb(Q) + (reinterpret_cast<uintptr_t>(g) & 15));
}

// Head / tail words of the staged blocks, by the threads of the tile.
template <class Prm>
__device__ __forceinline__ void geo_fixup(const Prm& p, char* slot, const Tile& t, int Q, int tid, int nthr) {
  const uint32_t eblk = geo_eblk(Q), erb = geo_erb(Q);
  if (t.contig) {
    const float* g0 = p.geom + 7 * quad_off_of<3>(p, elem_id(p, t, 0), Q);
    stage_fixup<4>(slot, g0, t.count * eblk, tid, nthr);
    return;
  }
  for (int j = tid / 8; j < t.count; j += nthr / 8)
    stage_fixup<4>(slot + j * erb, p.geom + 7 * quad_off_of<3>(p, elem_id(p, t, j), Q), eblk, tid % 8, 8);
}

// Coefficients of this thread's S1 pencil (a, b < n) of element pair pi of
// tile t (for the prefetch of the next tile's inputs into registers).
template <int P, class Prm>
__device__ __forceinline__ void load_coef_pencil(const Prm& p, const Tile& t, int pi, int a, int b, float2* v) {
  constexpr int n = P + 1;
  const int np = (t.count + 1) / 2;
  if (pi < np && a < n && b < n) {
    const int64_t e0 = elem_id(p, t, pi);
    const int64_t e1 = pi + np < t.count ? elem_id(p, t, pi + np) : e0;
    const float* u0 = p.in0 + coef_off_of<3>(p, e0, P) + (b * n + a) * n;
    const float* u1 = p.in0 + coef_off_of<3>(p, e1, P) + (b * n + a) * n;
#pragma unroll
    for (int k = 0; k < n; ++k) v[k] = make_float2(__ldcs(u0 + k), __ldcs(u1 + k));
  }
}

// One tile of order P (Q = P + QOFF): ceil(count / 2) pairs, Q^2 threads each;
// pair pi holds elements pi and pi + npair of the tile.
// Thread cc = a + Q b of pair pi; buffers (layout in PairLayout):
//   A: X (S1 -> S2), then U / g0 in place (S3 -> S7)
//   C: Y (S2 -> S3), then Y3 (S7 -> S8)
//   F: U' / g1 in place (S3 -> S7), then Y2 (S8 -> S9)
// The next tile's S1 writes only A, which no thread reads in S9.
// pre: this thread's S1 coefficients (n float2), already loaded when
// have_pre; on return they hold those of the next tile if it has the same
// order (next_loaded).  Returns false if the geometry copy did not land
// within the wait limit (the CTA then stops; the status word records it).
template <int P, int Q, class Prm>
__device__ __forceinline__ bool helm_pair_tile(const Prm& p, const float* tab, const Tile& t, char* sm,
                                               const uint32_t* offs, uint64_t* bar, uint32_t parity, int tid,
                                               int nthr, float2* pre, bool have_pre, bool* next_loaded) {
  using L = PairLayout<P, Q>;
  constexpr int n = P + 1, XS = L::XS, YS = L::YS, US = L::US, GS = L::GS, ZS = L::ZS;
  constexpr int Q2 = Q * Q, Q3 = Q * Q * Q;
  const float* B = tab;              // B[Q][n]
  const float* D = tab + 2 * Q * n;  // D[Q][Q]
  const int pi = tid / Q2;
  const int cc = tid - pi * Q2;
  const int a = cc % Q, b = cc / Q;
  const int npair = (t.count + 1) / 2;
  const int j0 = pi, j1 = pi + npair;  // pair pi = elements (j0, j1) of the tile
  const bool act = pi < npair;
  const bool two = j1 < t.count;
  float2* A = reinterpret_cast<float2*>(sm + offs[0]) + pi * L::WA;
  float2* C = reinterpret_cast<float2*>(sm + offs[1]) + pi * L::WC;
  float2* F = reinterpret_cast<float2*>(sm + offs[2]) + pi * L::WF;
  char* slot = sm + offs[3];
  int64_t c0 = 0, c1 = 0, q0 = 0, q1 = 0;
  if (act) {
    const int64_t e0 = elem_id(p, t, j0);
    const int64_t e1 = two ? elem_id(p, t, j1) : e0;
    c0 = coef_off_of<3>(p, e0, P);
    c1 = coef_off_of<3>(p, e1, P);
    q0 = quad_off_of<3>(p, e0, Q);
    q1 = quad_off_of<3>(p, e1, Q);
  }
  // S1: pencil along p at (q, r) = (a, b): X(q, r, i) = sum_p B[i][p] u[r][q][p] -> A
  if (act && a < n && b < n) {
    float2 v[n];
    if (have_pre) {
#pragma unroll
      for (int k = 0; k < n; ++k) v[k] = pre[k];
    } else {
      load_coef_pencil<P>(p, t, pi, a, b, v);
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int k = 0; k < n; ++k) acc = f2fma(B[i * n + k], v[k], acc);
      A[a + Q * b + XS * i] = acc;
    }
  }
  __syncthreads();
  // S2: pencil along q at (i, r) = (a, b): Y(i, r, j) = sum_q B[j][q] X(q, r, i) -> C
  if (act && b < n) {
    float2 v[n];
#pragma unroll
    for (int q = 0; q < n; ++q) v[q] = A[q + Q * b + XS * a];
#pragma unroll
    for (int j = 0; j < Q; ++j) {
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int q = 0; q < n; ++q) acc = f2fma(B[j * n + q], v[q], acc);
      C[a + Q * b + YS * j] = acc;
    }
  }
  __syncthreads();
  // S3: column (i, j) = (a, b): u = B y along xi_3 -> U in A and U' in F; d2 = D u in registers
  float2 u[Q], g2[Q];
  if (act) {
    float2 y[n];
#pragma unroll
    for (int r = 0; r < n; ++r) y[r] = C[a + Q * r + YS * b];
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int r = 0; r < n; ++r) acc = f2fma(B[k * n + r], y[r], acc);
      u[k] = acc;
      A[a + Q * b + US * k] = acc;
      F[a + Q * b + GS * k] = acc;
    }
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int m = 0; m < Q; ++m) acc = f2fma(D[k * Q + m], u[m], acc);
      g2[k] = acc;
    }
  }
  __syncthreads();
  // S4: gradient pencils, in place: along xi_1 at (j, k) = (b, a) in A (U -> d0),
  // along xi_2 at (i, k) = (a, b) in F (U' -> d1)
  if (act) {
    float2 v[Q];
    float2* g = A + Q * b + US * a;
#pragma unroll
    for (int m = 0; m < Q; ++m) v[m] = g[m];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int m = 0; m < Q; ++m) acc = f2fma(D[i * Q + m], v[m], acc);
      g[i] = acc;
    }
    g = F + a + GS * b;
#pragma unroll
    for (int m = 0; m < Q; ++m) v[m] = g[Q * m];
#pragma unroll
    for (int j = 0; j < Q; ++j) {
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int m = 0; m < Q; ++m) acc = f2fma(D[j * Q + m], v[m], acc);
      g[Q * j] = acc;
    }
  }
  // the tile's geometry: wait for its bulk copy, copy the ragged words
  const bool landed = mbar_wait(bar, parity);
  if (landed) geo_fixup(p, slot, t, Q, tid, nthr);
  if (__syncthreads_or(!landed)) return false;
  // S5: column (i, j) = (a, b): pointwise geometric factors; g0 -> A, g1 -> F, g2 and
  // lambda JW u in registers; then z = lambda JW u + D^T g2 along xi_3
  float2 z[Q];
  if (act) {
    const float* G0 = geo_staged(p, slot, t, j0, Q) + b * Q + a;
    const float* G1 = geo_staged(p, slot, t, two ? j1 : j0, Q) + b * Q + a;
    const float lam = static_cast<float>(p.lam);
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      const int w0 = a + Q * b + US * k, w1 = a + Q * b + GS * k;
      const float2 d0 = A[w0], d1 = F[w1], d2 = g2[k];
      const int o = k * Q2;
      const float2 g00 = make_float2(G0[o], G1[o]);
      const float2 g01 = make_float2(G0[o + Q3], G1[o + Q3]);
      const float2 g02 = make_float2(G0[o + 2 * Q3], G1[o + 2 * Q3]);
      const float2 g11 = make_float2(G0[o + 3 * Q3], G1[o + 3 * Q3]);
      const float2 g12 = make_float2(G0[o + 4 * Q3], G1[o + 4 * Q3]);
      const float2 g22 = make_float2(G0[o + 5 * Q3], G1[o + 5 * Q3]);
      const float2 jw = make_float2(G0[o + 6 * Q3], G1[o + 6 * Q3]);
      float2 r0 = f2fmav(g02, d2, f2fmav(g01, d1, f2mul(g00, d0)));
      float2 r1 = f2fmav(g12, d2, f2fmav(g11, d1, f2mul(g01, d0)));
      float2 r2 = f2fmav(g22, d2, f2fmav(g12, d1, f2mul(g02, d0)));
      if (p.kap_f) {
        const float2 kk = make_float2(__ldcs(p.kap_f + q0 + o + b * Q + a), __ldcs(p.kap_f + q1 + o + b * Q + a));
        r0 = f2mul(kk, r0);
        r1 = f2mul(kk, r1);
        r2 = f2mul(kk, r2);
      }
      float2 lj;
      if (p.lam_f) {
        const float2 ll = make_float2(__ldcs(p.lam_f + q0 + o + b * Q + a), __ldcs(p.lam_f + q1 + o + b * Q + a));
        lj = f2mul(ll, jw);
      } else {
        lj = f2mul(make_float2(lam, lam), jw);
      }
      A[w0] = r0;
      F[w1] = r1;
      g2[k] = r2;
      u[k] = f2mul(lj, u[k]);
    }
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      float2 acc = u[k];
#pragma unroll
      for (int m = 0; m < Q; ++m) acc = f2fma(D[m * Q + k], g2[m], acc);
      z[k] = acc;
    }
  }
  __syncthreads();
  // every thread is done with the geometry slot: stage the next tile's; load
  // the next tile's coefficients into registers if it has this order
  const int tn = offs[4];
  if (tid == 0 && tn < p.n_tiles) {
    fence_proxy_async();
    geo_issue(p, slot, bar, tn, Q - P);
  }
  *next_loaded = false;
  if (tn < p.n_tiles) {
    const Tile t2 = p.tiles[tn];
    if (t2.P == P) {
      load_coef_pencil<P>(p, t2, pi, a, b, pre);
      *next_loaded = true;
    }
  }
  // S6: transposed-gradient pencils, in place (same roles as S4)
  if (act) {
    float2 v[Q];
    float2* g = A + Q * b + US * a;
#pragma unroll
    for (int m = 0; m < Q; ++m) v[m] = g[m];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int m = 0; m < Q; ++m) acc = f2fma(D[m * Q + i], v[m], acc);
      g[i] = acc;
    }
    g = F + a + GS * b;
#pragma unroll
    for (int m = 0; m < Q; ++m) v[m] = g[Q * m];
#pragma unroll
    for (int j = 0; j < Q; ++j) {
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int m = 0; m < Q; ++m) acc = f2fma(D[m * Q + j], v[m], acc);
      g[Q * j] = acc;
    }
  }
  __syncthreads();
  // S7: column (i, j) = (a, b): z += both contributions; B^T along xi_3 -> Y3(i, j, r) in C
  if (act) {
#pragma unroll
    for (int k = 0; k < Q; ++k) z[k] = f2add(z[k], f2add(A[a + Q * b + US * k], F[a + Q * b + GS * k]));
#pragma unroll
    for (int r = 0; r < n; ++r) {
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int k = 0; k < Q; ++k) acc = f2fma(B[k * n + r], z[k], acc);
      C[a + Q * r + YS * b] = acc;
    }
  }
  __syncthreads();
  // S8: pencil along j at (i, r) = (a, b): Y2(i, q, r) = sum_j B[j][q] Y3(i, j, r) -> F
  if (act && b < n) {
    float2 v[Q];
#pragma unroll
    for (int j = 0; j < Q; ++j) v[j] = C[a + Q * b + YS * j];
#pragma unroll
    for (int q = 0; q < n; ++q) {
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int j = 0; j < Q; ++j) acc = f2fma(B[j * n + q], v[j], acc);
      F[a + Q * b + ZS * q] = acc;
    }
  }
  __syncthreads();
  // S9: pencil along i at (q, r) = (a, b): y[r][q][p] = sum_i B[i][p] Y2(i, q, r) -> HBM
  if (act && a < n && b < n) {
    float2 v[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) v[i] = F[i + Q * b + ZS * a];
    float* y0 = p.out0 + c0 + (b * n + a) * n;
    float* y1 = p.out0 + c1 + (b * n + a) * n;
#pragma unroll
    for (int k = 0; k < n; ++k) {
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int i = 0; i < Q; ++i) acc = f2fma(B[i * n + k], v[i], acc);
      __stcs(y0 + k, acc.x);
      if (two) __stcs(y1 + k, acc.y);
    }
  }
  return true;
}

template <int PLO, int PHI, int QOFF, class Prm>
__device__ __forceinline__ bool pair_dispatch(int P, const Prm& p, const Tile& t, char* sm, const uint32_t* offs,
                                              uint64_t* bar, uint32_t parity, int tid, int nthr, float2* pre,
                                              bool have_pre, bool* next_loaded) {
  if constexpr (PLO <= PHI) {
    if (P == PLO)
      return helm_pair_tile<PLO, PLO + QOFF>(p, p.tab + Prm::Layout::off(PLO), t, sm, offs, bar, parity, tid, nthr,
                                             pre, have_pre, next_loaded);
    return pair_dispatch<PLO + 1, PHI, QOFF>(P, p, t, sm, offs, bar, parity, tid, nthr, pre, have_pre, next_loaded);
  }
  return true;
}

// REG: register budget per thread (occupancy class chosen by the autotuner).
template <int PLO, int PHI, int QOFF, int REG>
__global__ void __maxnreg__(REG) helm_pair_kernel(const __grid_constant__ PairParams<PLO, PHI, QOFF> pp) {
  extern __shared__ __align__(128) char sm[];
  const auto& p = pp.k;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm);
  const int tid = threadIdx.x, nthr = blockDim.x;
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_barrier_init();
  }
  __syncthreads();
  if (tid == 0) {
    if (blockIdx.x < p.n_tiles) geo_issue(p, sm + pp.off_geo, bar, blockIdx.x, QOFF);
    for (int j = 1; j <= pp.pf; ++j) {
      const int ti = blockIdx.x + j * gridDim.x;
      if (ti < p.n_tiles) prefetch_tile<3>(p, ti, QOFF);
    }
  }
  uint32_t offs[5] = {pp.off_a, pp.off_c, pp.off_f, pp.off_geo, 0};
  // the next tile's S1 coefficients, prefetched into registers (uniform order:
  // sized for it; several orders: sized for the highest)
  float2 pre[PHI + 1];
  bool have_pre = false;
  for (int k = 0;; ++k) {
    const int ti = blockIdx.x + k * gridDim.x;
    if (ti >= p.n_tiles) break;
    if (tid == 0 && pp.pf > 0) {
      const int tn = ti + (pp.pf + 1) * gridDim.x;
      if (tn < p.n_tiles) prefetch_tile<3>(p, tn, QOFF);
    }
    offs[4] = ti + gridDim.x;  // the tile staged after this one's S5
    const Tile t = p.tiles[ti];
    bool next_loaded = false;
    if (!pair_dispatch<PLO, PHI, QOFF>(t.P, p, t, sm, offs, bar, k & 1, tid, nthr, pre, have_pre, &next_loaded)) {
      if (tid == 0) atomicOr(p.status, kStatusTimeout);
      return;
    }
    have_pre = next_loaded;
  }
}

}  // namespace spx
