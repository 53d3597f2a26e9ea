// FP32 Helmholtz operator H = lambda M + L on hexahedra (§3.3 collective
// evaluation, SumFac strategy; sum-factorisation display of §3.3 for the
// three 1D contractions), two elements per thread in packed f32x2 arithmetic.
//
// Every value a thread handles is a float2 holding the same entry of two
// elements of the tile (an element pair), so each FFMA2 / LDS.64 / STS.64
// does the work of two scalar instructions: the operator is issue / latency
// bound on CUDA cores (the contractions are 5x6 / 6x6 matrices, too small for
// the tensor cores to pay), and the pair layout halves its instruction count
// per element.  (The body is generic in the value type: `float`, one element
// per thread, serves the high orders of a variable-order launch, whose single
// kernel allocates registers for its largest body.)  Thread (a, b) of a pair
// plays the column / pencil roles of the role-based body: column owner of
// quadrature column (i, j) = (a, b) (xi_3 contractions, xi_3 gradient and the
// pointwise geometric factors in registers), pencil owner along xi_1 at
// (j, k) = (b, a) and along xi_2 at (i, k) = (a, b).  Nine phases, one CTA
// barrier each, through three shared-memory buffers per pair laid out free of
// bank conflicts (PairLayout in kernel_params.h).
//
// Each tile's geometric factors (86% of the bytes) are staged into one
// shared-memory slot by 1D bulk copies (TMA) issued as soon as the previous
// tile's pointwise phase has released the slot, so they have eight phases to
// land; the wait for them is bounded (a copy that never lands sets the plan's
// status word, nothing hangs).  Two kernels:
//  * helm_pair_kernel (one order): warp 0 issues the copies; the next tile's
//    S1 coefficients are loaded into registers during S6..S9;
//  * helm_varp_kernel (several orders, elements of one order scattered
//    through the mesh): a producer warp outside the compute barriers writes
//    each tile's element offsets into shared memory and stages its geometry;
//    every CTA keeps to the tiles of one order, so that each order's body
//    runs in a loop of its own.
// Coefficients are read straight from HBM (coalesced, read once), outputs
// stored straight to HBM.
#pragma once
#include <type_traits>

#include "lanes.cuh"
#include "op_kernel.cuh"

namespace spx {

template <int PLO, int PHI, int QOFF>
struct PairParams {
  KParams<float, PLO, PHI, QOFF> k;
  int pf;                          // L2 prefetch distance in tiles (0: none)
  uint32_t off_a, off_c, off_f;    // byte offsets of the work buffers
  uint32_t off_geo;                // byte offset of the geometry slot
  uint32_t off_meta;               // byte offset of the tile metadata (variable order)
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

// Geometry of tile `ti` into the slot, by the 32 lanes of warp 0 (all must
// call): one 1D bulk copy of a contiguous tile's [count][7][Q^3] range, else
// one copy per element (lane j issues elements j, j + 32, ...) into regions of
// geo_erb bytes (kernel_params.h).  Ragged head / tail words (< 16 bytes,
// when a range is not 16-byte aligned in HBM) are copied by geo_fixup once the
// bulk part has landed.
template <class Prm>
__device__ void geo_issue_warp(const Prm& p, char* slot, uint64_t* bar, int ti, int QOFF, int lane) {
  const Tile t = p.tiles[ti];
  const int P = t.P, Q = P + QOFF;
  const uint32_t eblk = geo_eblk(Q), erb = geo_erb(Q);
  if (t.contig) {
    if (lane == 0) {
      fence_proxy_async();
      const float* g0 = p.geom + 7 * quad_off_of<3>(p, elem_id(p, t, 0), Q);
      mbar_arrive_expect_tx(bar, stage_bytes(g0, t.count * eblk));
      stage_issue(slot, g0, t.count * eblk, bar);
    }
    return;
  }
  fence_proxy_async();
  uint32_t tx = 0;
  for (int j = lane; j < t.count; j += 32) tx += stage_bytes(p.geom + 7 * quad_off_of<3>(p, elem_id(p, t, j), Q), eblk);
  for (int o = 16; o > 0; o >>= 1) tx += __shfl_xor_sync(0xffffffffu, tx, o);
  if (lane == 0) mbar_arrive_expect_tx(bar, tx);
  __syncwarp();
  for (int j = lane; j < t.count; j += 32)
    stage_issue(slot + j * erb, p.geom + 7 * quad_off_of<3>(p, elem_id(p, t, j), Q), eblk, bar);
}

// Shared-memory address of the staged geometry of element j of tile t, whose
// quadrature offset is qj.
__device__ __forceinline__ const float* geo_staged(const float* geom, const char* slot, const Tile& t, int j,
                                                   int64_t qj, int Q) {
  const uintptr_t g = reinterpret_cast<uintptr_t>(geom + 7 * qj);
  if (t.contig) return reinterpret_cast<const float*>(slot + ((g - j * geo_eblk(Q)) & 15) + j * geo_eblk(Q));
  return reinterpret_cast<const float*>(slot + j * geo_erb(Q) + (g & 15));
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

// Inputs of a thread's element group carried from one tile to the next: its
// S1 coefficients.
template <int NMAX, bool ON>
struct GroupPrefetch {
  static constexpr bool kOn = ON;
  float2 v[NMAX];
};
// (variable-order launches keep nothing across tiles: the registers held by
// the carried inputs would make the highest-order bodies spill)
template <int NMAX>
struct GroupPrefetch<NMAX, false> {
  static constexpr bool kOn = false;
  float2 v[1];
};

// Offsets {c0, c1, q0, q1} and S1 coefficients (a, b < n) of element group gi
// of tile t of order P (Q points per direction); nothing for gi outside it.
template <int P, int Q, class V, class Prm>
__device__ __forceinline__ void load_group(const Prm& p, const Tile& t, int gi, int a, int b, V* v, int64_t* off) {
  constexpr int n = P + 1, LN = Lane<V>::L;
  const int ng = (t.count + LN - 1) / LN;
  if (gi < ng) {
    const int64_t e0 = elem_id(p, t, gi);
    const int64_t e1 = (LN == 2 && gi + ng < t.count) ? elem_id(p, t, gi + ng) : e0;
    off[0] = coef_off_of<3>(p, e0, P);
    off[1] = coef_off_of<3>(p, e1, P);
    off[2] = quad_off_of<3>(p, e0, Q);
    off[3] = quad_off_of<3>(p, e1, Q);
    if (a < n && b < n) {
      const float* u0 = p.in0 + off[0] + (b * n + a) * n;
      const float* u1 = p.in0 + off[1] + (b * n + a) * n;
#pragma unroll
      for (int k = 0; k < n; ++k) v[k] = Lane<V>::ldcs2(u0 + k, u1 + k);
    }
  }
}

// One tile of order P (Q = P + QOFF) in value type V: ceil(count / L) element
// groups of Q^2 threads each (L = 2 for float2, 1 for float); group pi holds
// elements pi and pi + ngroup of the tile.
// Thread cc = a + Q b of group pi; buffers (layout in PairLayout):
//   A: X (S1 -> S2), then U / g0 in place (S3 -> S7)
//   C: Y (S2 -> S3), then Y3 (S7 -> S8)
//   F: U' / g1 in place (S3 -> S7), then Y2 (S8 -> S9)
// The next tile's S1 writes only A, which no thread reads in S9.
// `ctl` provides the barriers, the inputs, the geometry slot and what happens
// once the slot is released (DirectCtl / ProducerCtl below).  Returns false
// if a bounded wait gave up (the CTA then stops; the status word records it).
template <int P, int Q, class V, class Prm, class Ctl>
__device__ __forceinline__ bool helm_pair_tile(const Prm& p, Ctl& ctl, const float* tab, const Tile& t) {
  using Vt = Lane<V>;
  using L = PairLayout<P, Q, Vt::M>;
  constexpr int n = P + 1, XS = L::XS, YS = L::YS, US = L::US, GS = L::GS, ZS = L::ZS;
  constexpr int Q2 = Q * Q, Q3 = Q * Q * Q;
  const int tid = ctl.tid;
  const int pi = tid / Q2;
  const int cc = tid - pi * Q2;
  const int a = cc % Q, b = cc / Q;
  const int npair = (t.count + Vt::L - 1) / Vt::L;
  const int j0 = pi, j1 = pi + npair;  // group pi = elements (j0, j1) of the tile
  const bool act = pi < npair;
  const bool two = Vt::L == 2 && j1 < t.count;
  // (buffers addressed from the dynamic shared array itself, so that the
  // compiler keeps 32-bit shared-window addressing)
  extern __shared__ __align__(128) char dsm[];
  V* A = reinterpret_cast<V*>(dsm + ctl.offs[0]) + pi * L::WA;
  V* C = reinterpret_cast<V*>(dsm + ctl.offs[1]) + pi * L::WC;
  V* F = reinterpret_cast<V*>(dsm + ctl.offs[2]) + pi * L::WF;
  // element offsets {c0, c1, q0, q1} and this thread's S1 coefficients
  V v1[n];
  int64_t off[4] = {0, 0, 0, 0};
  ctl.template inputs<P, Q, V>(p, t, pi, a, b, act, j0, j1, two, v1, off);
  const int64_t c0 = off[0], c1 = off[1], q0 = off[2], q1 = off[3];
  // S1: pencil along p at (q, r) = (a, b): X(q, r, i) = sum_p B[i][p] u[r][q][p] -> A
  if (act && a < n && b < n) {
    V x[Q];
    eo_b<P, Q>(tab, v1, x);
#pragma unroll
    for (int i = 0; i < Q; ++i) A[a + Q * b + XS * i] = x[i];
  }
  ctl.sync();
  // S2: pencil along q at (i, r) = (a, b): Y(i, r, j) = sum_q B[j][q] X(q, r, i) -> C
  if (act && b < n) {
    V v[n], y[Q];
#pragma unroll
    for (int q = 0; q < n; ++q) v[q] = A[q + Q * b + XS * a];
    eo_b<P, Q>(tab, v, y);
#pragma unroll
    for (int j = 0; j < Q; ++j) C[a + Q * b + YS * j] = y[j];
  }
  ctl.sync();
  // S3: column (i, j) = (a, b): u = B y along xi_3 -> U in A and U' in F; d2 = dB y in registers
  V u[Q], g2[Q];
  if (act) {
    V y[n];
#pragma unroll
    for (int r = 0; r < n; ++r) y[r] = C[a + Q * r + YS * b];
    eo_b<P, Q>(tab, y, u);
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      A[a + Q * b + US * k] = u[k];
      F[a + Q * b + GS * k] = u[k];
    }
    eo_db<P, Q>(tab, y, g2);
  }
  ctl.sync();
  // S4: gradient pencils, in place: along xi_1 at (j, k) = (b, a) in A (U -> d0),
  // along xi_2 at (i, k) = (a, b) in F (U' -> d1)
  if (act) {
    V v[Q], d[Q];
    V* g = A + Q * b + US * a;
#pragma unroll
    for (int m = 0; m < Q; ++m) v[m] = g[m];
    eo_d<P, Q, false>(tab, v, d);
#pragma unroll
    for (int i = 0; i < Q; ++i) g[i] = d[i];
    g = F + a + GS * b;
#pragma unroll
    for (int m = 0; m < Q; ++m) v[m] = g[Q * m];
    eo_d<P, Q, false>(tab, v, d);
#pragma unroll
    for (int j = 0; j < Q; ++j) g[Q * j] = d[j];
  }
  // the tile's geometry: wait for it to land (ends the phase with a barrier)
  if (!ctl.geo_wait(p, t, Q)) return false;
  // S5: column (i, j) = (a, b): pointwise geometric factors; g0 -> A, g1 -> F, g2 and
  // lambda JW in registers; then z = D^T g2 + lambda JW u along xi_3
  V z[Q];
  if (act) {
    const float* G0 = geo_staged(p.geom, dsm + ctl.offs[3], t, j0, q0, Q) + b * Q + a;
    const float* G1 = geo_staged(p.geom, dsm + ctl.offs[3], t, two ? j1 : j0, two ? q1 : q0, Q) + b * Q + a;
    const float lam = static_cast<float>(p.lam);
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      const int w0 = a + Q * b + US * k, w1 = a + Q * b + GS * k;
      const V d0 = A[w0], d1 = F[w1], d2 = g2[k];
      const int o = k * Q2;
      const V g00 = Vt::pair(G0[o], G1[o]);
      const V g01 = Vt::pair(G0[o + Q3], G1[o + Q3]);
      const V g02 = Vt::pair(G0[o + 2 * Q3], G1[o + 2 * Q3]);
      const V g11 = Vt::pair(G0[o + 3 * Q3], G1[o + 3 * Q3]);
      const V g12 = Vt::pair(G0[o + 4 * Q3], G1[o + 4 * Q3]);
      const V g22 = Vt::pair(G0[o + 5 * Q3], G1[o + 5 * Q3]);
      const V jw = Vt::pair(G0[o + 6 * Q3], G1[o + 6 * Q3]);
      V r0 = Vt::fmav(g02, d2, Vt::fmav(g01, d1, Vt::mul(g00, d0)));
      V r1 = Vt::fmav(g12, d2, Vt::fmav(g11, d1, Vt::mul(g01, d0)));
      V r2 = Vt::fmav(g22, d2, Vt::fmav(g12, d1, Vt::mul(g02, d0)));
      if (p.kap_f) {
        const V kk = Vt::ldcs2(p.kap_f + q0 + o + b * Q + a, p.kap_f + q1 + o + b * Q + a);
        r0 = Vt::mul(kk, r0);
        r1 = Vt::mul(kk, r1);
        r2 = Vt::mul(kk, r2);
      }
      A[w0] = r0;
      F[w1] = r1;
      g2[k] = r2;
      (void)jw;
    }
    eo_d<P, Q, true>(tab, g2, z);
    // mass term: lambda JW u, with JW read again from the staged slot (holding
    // lambda JW in registers across the D^T contraction made the combined
    // variable-order kernel spill)
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      const int o = k * Q2 + 6 * Q3;
      const V jw = Vt::pair(G0[o], G1[o]);
      V lj;
      if (p.lam_f) {
        const int oq = k * Q2 + b * Q + a;
        lj = Vt::mul(Vt::ldcs2(p.lam_f + q0 + oq, p.lam_f + q1 + oq), jw);
      } else {
        lj = Vt::mul(Vt::bcast(lam), jw);
      }
      z[k] = Vt::fmav(lj, u[k], z[k]);
    }
  }
  ctl.sync();
  // every thread is done with the geometry slot
  ctl.template slot_released<P, Q, V>(p, pi, a, b);
  // S6: transposed-gradient pencils, in place (same roles as S4)
  if (act) {
    V v[Q], d[Q];
    V* g = A + Q * b + US * a;
#pragma unroll
    for (int m = 0; m < Q; ++m) v[m] = g[m];
    eo_d<P, Q, true>(tab, v, d);
#pragma unroll
    for (int i = 0; i < Q; ++i) g[i] = d[i];
    g = F + a + GS * b;
#pragma unroll
    for (int m = 0; m < Q; ++m) v[m] = g[Q * m];
    eo_d<P, Q, true>(tab, v, d);
#pragma unroll
    for (int j = 0; j < Q; ++j) g[Q * j] = d[j];
  }
  ctl.sync();
  // S7: column (i, j) = (a, b): z += both contributions; B^T along xi_3 -> Y3(i, j, r) in C
  if (act) {
    V y3[n];
#pragma unroll
    for (int k = 0; k < Q; ++k) z[k] = Vt::add(z[k], Vt::add(A[a + Q * b + US * k], F[a + Q * b + GS * k]));
    eo_bt<P, Q>(tab, z, y3);
#pragma unroll
    for (int r = 0; r < n; ++r) C[a + Q * r + YS * b] = y3[r];
  }
  ctl.sync();
  // S8: pencil along j at (i, r) = (a, b): Y2(i, q, r) = sum_j B[j][q] Y3(i, j, r) -> F
  if (act && b < n) {
    V v[Q], y2[n];
#pragma unroll
    for (int j = 0; j < Q; ++j) v[j] = C[a + Q * b + YS * j];
    eo_bt<P, Q>(tab, v, y2);
#pragma unroll
    for (int q = 0; q < n; ++q) F[a + Q * b + ZS * q] = y2[q];
  }
  ctl.sync();
  // S9: pencil along i at (q, r) = (a, b): y[r][q][p] = sum_i B[i][p] Y2(i, q, r) -> HBM
  if (act && a < n && b < n) {
    V v[Q], y[n];
#pragma unroll
    for (int i = 0; i < Q; ++i) v[i] = F[i + Q * b + ZS * a];
    eo_bt<P, Q>(tab, v, y);
    float* y0 = p.out0 + c0 + (b * n + a) * n;
    float* y1 = p.out0 + c1 + (b * n + a) * n;
#pragma unroll
    for (int k = 0; k < n; ++k) Vt::stcs2(y0 + k, y1 + k, y[k], two);
  }
  return true;
}

// Body of order P, selected at run time from the tile (orders <= THR packed
// two elements per thread).  (Bodies called out of line, each with its own
// register allocation, measured 40% slower on the variable-order workload:
// the calls' register saves cost more than the spills of the union.)
template <int PLO, int PHI, int QOFF, int THR, class Prm, class Ctl>
__device__ __forceinline__ bool pair_dispatch(int P, const Prm& p, Ctl& ctl, const Tile& t) {
  if constexpr (PLO <= PHI) {
    using V = typename std::conditional<pair_lanes(PLO, THR) == 2, float2, float>::type;
    if (P == PLO) return helm_pair_tile<PLO, PLO + QOFF, V>(p, ctl, p.tab + Prm::Layout::off(PLO), t);
    return pair_dispatch<PLO + 1, PHI, QOFF, THR>(P, p, ctl, t);
  }
  return true;
}

// ---- Direct control: every thread computes; warp 0 stages the next tile's
// geometry as soon as S5 has released the slot; inputs read from HBM; a
// uniform-order kernel carries the next tile's S1 coefficients in registers.
template <int NMAX, bool PREF>
struct DirectCtl {
  char* sm;
  uint32_t offs[4];   // A, C, F, geometry slot
  uint64_t* bar;      // geometry mbarrier
  uint32_t parity;
  int tid, nthr;
  int next_tile;
  GroupPrefetch<NMAX, PREF> pre;
  bool have_pre = false, next_loaded = false;

  __device__ __forceinline__ void sync() { __syncthreads(); }
  __device__ __forceinline__ char* slot() const { return sm + offs[3]; }

  template <int P, int Q, class V, class Prm>
  __device__ __forceinline__ void inputs(const Prm& p, const Tile& t, int gi, int a, int b, bool act, int j0, int j1,
                                         bool two, V* v, int64_t* off) {
    constexpr int n = P + 1;
    if (PREF && have_pre) {
      // carried coefficients; offsets of a uniform plan are arithmetic
#pragma unroll
      for (int k = 0; k < n; ++k) v[k] = Lane<V>::from2(pre.v[k]);
      if (act) {
        const int64_t e0 = elem_id(p, t, j0), e1 = two ? elem_id(p, t, j1) : e0;
        off[0] = coef_off_of<3>(p, e0, P);
        off[1] = coef_off_of<3>(p, e1, P);
        off[2] = quad_off_of<3>(p, e0, Q);
        off[3] = quad_off_of<3>(p, e1, Q);
      }
    } else if (act) {
      load_group<P, Q>(p, t, gi, a, b, v, off);
    }
  }

  // wait for the tile's geometry, copy its ragged words, barrier
  template <class Prm>
  __device__ __forceinline__ bool geo_wait(const Prm& p, const Tile& t, int Q) {
    const bool landed = mbar_wait(bar, parity);
    if (landed) geo_fixup(p, slot(), t, Q, tid, nthr);
    return !__syncthreads_or(!landed);
  }

  template <int P, int Q, class V, class Prm>
  __device__ __forceinline__ void slot_released(const Prm& p, int gi, int a, int b) {
    if (tid < 32 && next_tile < p.n_tiles) geo_issue_warp(p, slot(), bar, next_tile, Q - P, tid);
    next_loaded = false;
    if (PREF && next_tile < p.n_tiles) {
      const Tile t2 = p.tiles[next_tile];
      if (t2.P == P) {
        constexpr int n = P + 1;
        V v2[n];
        int64_t o2[4] = {0, 0, 0, 0};
        load_group<P, Q>(p, t2, gi, a, b, v2, o2);
#pragma unroll
        for (int k = 0; k < n; ++k) pre.v[k] = Lane<V>::to2(v2[k]);
        next_loaded = true;
      }
    }
  }
};

// REG: register budget per thread (occupancy class chosen by the autotuner);
// orders <= THR run two elements per thread, the others one.
template <int PLO, int PHI, int QOFF, int REG, int THR>
__global__ void __maxnreg__(REG) helm_pair_kernel(const __grid_constant__ PairParams<PLO, PHI, QOFF> pp) {
  extern __shared__ __align__(128) char sm[];
  const auto& p = pp.k;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm);
  const int tid = threadIdx.x, nthr = blockDim.x;
  if (p.skip && *p.skip) return;   // uniform across the grid: nothing started yet
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_barrier_init();
  }
  __syncthreads();
  if (tid < 32 && blockIdx.x < p.n_tiles) geo_issue_warp(p, sm + pp.off_geo, bar, blockIdx.x, QOFF, tid);
  if (tid == 0) {
    for (int j = 1; j <= pp.pf; ++j) {
      const int ti = blockIdx.x + j * gridDim.x;
      if (ti < p.n_tiles) prefetch_tile<3>(p, ti, QOFF);
    }
  }
  DirectCtl<PHI + 1, PLO == PHI> ctl{sm, {pp.off_a, pp.off_c, pp.off_f, pp.off_geo}, bar, 0u, tid, nthr, 0};
  for (int k = 0;; ++k) {
    const int ti = blockIdx.x + k * gridDim.x;
    if (ti >= p.n_tiles) break;
    if (tid == 0 && pp.pf > 0) {
      const int tn = ti + (pp.pf + 1) * gridDim.x;
      if (tn < p.n_tiles) prefetch_tile<3>(p, tn, QOFF);
    }
    ctl.next_tile = ti + gridDim.x;  // the tile staged after this one's S5
    ctl.parity = k & 1;
    const Tile t = p.tiles[ti];
    if (!pair_dispatch<PLO, PHI, QOFF, THR>(t.P, p, ctl, t)) {
      if (tid == 0) atomicOr(p.status, kStatusTimeout);
      return;
    }
    ctl.have_pre = ctl.next_loaded;
  }
}

// ---- Producer control (variable order): warp `ncompute / 32` of the CTA is
// a producer that never joins the compute barriers.  For every tile it writes
// the tile and its elements' coefficient / quadrature offsets into one of two
// metadata buffers (released to the compute warps through an mbarrier), and
// stages the tile's geometry (ragged words by plain copies, the rest by bulk
// copies) as soon as the compute warps have passed S5 of the previous tile
// (named barrier 2, arrive / sync).  Compute warps synchronise on named
// barrier 1.  Non-contiguous tiles (elements of one order scattered through
// the mesh) then cost the compute warps no dependent global loads.
struct TileMeta {
  Tile t;
  int64_t coff[kMaxEB];
  int64_t qoff[kMaxEB];
};

__device__ __forceinline__ void named_sync(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }
__device__ __forceinline__ void named_arrive(int id, int n) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ bool named_sync_or(int id, int n, bool x) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 q, %1, 0;\n\tbar.red.or.pred p, %2, %3, q;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(r)
      : "r"(uint32_t(x)), "r"(id), "r"(n)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

struct ProducerCtl {
  char* sm;
  uint32_t offs[4];
  uint64_t* bar;          // geometry mbarrier
  uint32_t parity;
  int tid, nthr;          // nthr = compute threads
  const TileMeta* meta;   // this tile's
  int* abort;

  __device__ __forceinline__ void sync() { named_sync(1, nthr); }
  __device__ __forceinline__ char* slot() const { return sm + offs[3]; }

  template <int P, int Q, class V, class Prm>
  __device__ __forceinline__ void inputs(const Prm& p, const Tile&, int, int a, int b, bool act, int j0, int j1,
                                         bool two, V* v, int64_t* off) {
    constexpr int n = P + 1;
    if (!act) return;
    off[0] = meta->coff[j0];
    off[1] = meta->coff[two ? j1 : j0];
    off[2] = meta->qoff[j0];
    off[3] = meta->qoff[two ? j1 : j0];
    if (a < n && b < n) {
      const float* u0 = p.in0 + off[0] + (b * n + a) * n;
      const float* u1 = p.in0 + off[1] + (b * n + a) * n;
#pragma unroll
      for (int k = 0; k < n; ++k) v[k] = Lane<V>::ldcs2(u0 + k, u1 + k);
    }
  }

  // the producer copied the ragged words before releasing the copy
  template <class Prm>
  __device__ __forceinline__ bool geo_wait(const Prm&, const Tile&, int) {
    const bool landed = mbar_wait(bar, parity);
    if (named_sync_or(1, nthr, !landed)) {
      if (tid == 0) *abort = 1;
      named_arrive(2, nthr + 32);   // let the producer see the abort
      return false;
    }
    return true;
  }

  template <int P, int Q, class V, class Prm>
  __device__ __forceinline__ void slot_released(const Prm&, int, int, int) {
    named_arrive(2, nthr + 32);
  }
};

// Producer: metadata of tile ti into buffer m, then arrive on mbar.
template <int QOFF, class Prm>
__device__ __forceinline__ void produce_meta(const Prm& p, TileMeta* m, uint64_t* mbar, int ti, int lane) {
  const Tile t = p.tiles[ti];
  const int Q = t.P + QOFF;
  for (int j = lane; j < t.count; j += 32) {
    const int64_t e = elem_id(p, t, j);
    m->coff[j] = coef_off_of<3>(p, e, t.P);
    m->qoff[j] = quad_off_of<3>(p, e, Q);
  }
  if (lane == 0) m->t = t;
  __syncwarp();
  if (lane == 0) mbar_arrive(mbar);
}

// Producer: geometry of the tile described by m into the slot: ragged words
// by plain copies, then the expected bytes, then the bulk copies.
template <int QOFF, class Prm>
__device__ __forceinline__ void produce_geo(const Prm& p, const TileMeta* m, char* slot, uint64_t* bar, int lane) {
  const Tile t = m->t;
  const int Q = t.P + QOFF;
  const uint32_t eblk = geo_eblk(Q), erb = geo_erb(Q);
  fence_proxy_async();
  uint32_t tx = 0;
  if (t.contig) {
    const float* g0 = p.geom + 7 * m->qoff[0];
    stage_fixup<4>(slot, g0, t.count * eblk, lane, 32);
    tx = lane == 0 ? stage_bytes(g0, t.count * eblk) : 0;
  } else {
    for (int j = lane; j < t.count; j += 32) {
      const float* g = p.geom + 7 * m->qoff[j];
      stage_fixup<4>(slot + j * erb, g, eblk, 0, 1);
      tx += stage_bytes(g, eblk);
    }
  }
  for (int o = 16; o > 0; o >>= 1) tx += __shfl_xor_sync(0xffffffffu, tx, o);
  __syncwarp();
  if (lane == 0) mbar_arrive_expect_tx(bar, tx);
  __syncwarp();
  if (t.contig) {
    if (lane == 0) stage_issue(slot, p.geom + 7 * m->qoff[0], t.count * eblk, bar);
  } else {
    for (int j = lane; j < t.count; j += 32) stage_issue(slot + j * erb, p.geom + 7 * m->qoff[j], eblk, bar);
  }
}

// Compute warps of a CTA that keeps to order P: its tiles t0, t0 + G, ...
// below t1.  The loop sits inside the order's branch: a loop around the
// dispatch over all orders made the compiler keep values of every body live
// across it (spills that no single body has).
template <int P, int QOFF, int THR, class Prm>
__device__ __forceinline__ void varp_compute(const Prm& pp, ProducerCtl& ctl, uint64_t* mbar, TileMeta* meta, int t0,
                                             int t1, int G) {
  using V = typename std::conditional<pair_lanes(P, THR) == 2, float2, float>::type;
  const auto& p = pp.k;
  const int tid = ctl.tid, nc = ctl.nthr;
  for (int k = 0;; ++k) {
    const int ti = t0 + k * G;
    if (ti >= t1) break;
    const bool ok = mbar_wait(&mbar[k & 1], (k >> 1) & 1);
    if (named_sync_or(1, nc, !ok)) {
      if (tid == 0) {
        *ctl.abort = 1;
        atomicOr(p.status, kStatusTimeout);
      }
      named_arrive(2, nc + 32);
      return;
    }
    ctl.meta = &meta[k & 1];
    ctl.parity = k & 1;
    const Tile t = ctl.meta->t;
    if (!helm_pair_tile<P, P + QOFF, V>(p, ctl, p.tab + std::decay_t<decltype(p)>::Layout::off(P), t)) {
      if (tid == 0) atomicOr(p.status, kStatusTimeout);
      return;
    }
  }
}

template <int PLO, int PHI, int QOFF, int THR, class Prm>
__device__ __forceinline__ void varp_dispatch(int P, const Prm& pp, ProducerCtl& ctl, uint64_t* mbar, TileMeta* meta,
                                              int t0, int t1, int G) {
  if constexpr (PLO <= PHI) {
    if (P == PLO) varp_compute<PLO, QOFF, THR>(pp, ctl, mbar, meta, t0, t1, G);
    else varp_dispatch<PLO + 1, PHI, QOFF, THR>(P, pp, ctl, mbar, meta, t0, t1, G);
  }
}

template <int PLO, int PHI, int QOFF, int REG, int THR>
__global__ void __maxnreg__(REG) helm_varp_kernel(const __grid_constant__ PairParams<PLO, PHI, QOFF> pp) {
  extern __shared__ __align__(128) char sm[];
  const auto& p = pp.k;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm);         // geometry
  uint64_t* mbar = bar + 1;                                // metadata buffers 0, 1
  int* abort = reinterpret_cast<int*>(bar + 3);
  TileMeta* meta = reinterpret_cast<TileMeta*>(sm + pp.off_meta);
  const int tid = threadIdx.x;
  const int nc = blockDim.x - 32;                          // compute threads
  if (p.skip && *p.skip) return;   // uniform across the grid: nothing started yet
  // this CTA's run of tiles (one order)
  const TileRun run = tile_run(p);
  const int G = run.G, t0 = run.t0, t1 = run.t1;
  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    *abort = 0;
    fence_barrier_init();
  }
  __syncthreads();
  if (tid >= nc) {   // producer warp
    const int lane = tid - nc;
    if (t0 < t1) {
      produce_meta<QOFF>(p, &meta[0], &mbar[0], t0, lane);
      produce_geo<QOFF>(p, &meta[0], sm + pp.off_geo, bar, lane);
      if (t0 + G < t1) produce_meta<QOFF>(p, &meta[1], &mbar[1], t0 + G, lane);
    }
    for (int k = 0;; ++k) {
      const int ti = t0 + k * G;
      if (ti >= t1) break;
      named_sync(2, nc + 32);   // compute warps are past S5 of tile k
      if (*reinterpret_cast<volatile int*>(abort)) break;
      if (ti + G < t1) produce_geo<QOFF>(p, &meta[(k + 1) & 1], sm + pp.off_geo, bar, lane);
      if (ti + 2 * G < t1) produce_meta<QOFF>(p, &meta[k & 1], &mbar[k & 1], ti + 2 * G, lane);
    }
    return;
  }
  ProducerCtl ctl{sm, {pp.off_a, pp.off_c, pp.off_f, pp.off_geo}, bar, 0u, tid, nc, nullptr, abort};
  varp_dispatch<PLO, PHI, QOFF, THR>(run.P, pp, ctl, mbar, meta, t0, t1, G);
}

}  // namespace spx
