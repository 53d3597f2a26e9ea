// FP32 BwdTrans and IProductWRTBase on hexahedra in the element-pair layout
// of the Helmholtz pair kernel (§3.3 collective evaluation, SumFac strategy:
// the three 1D contractions of the sum-factorisation display of §3.3).
//
// Both operators stream: BwdTrans reads n^3 coefficients and writes Q^3
// values per element, IProductWRTBase reads Q^3 values and the Q^3 Jacobian
// weights JW and writes n^3 coefficients.  Every value a thread handles is a
// float2 holding the same entry of two elements (FFMA2, LDS.64 / STS.64), and
// thread (a, b) of a pair plays the roles of the Helmholtz body's phases:
//   BwdTrans:        S1 pencil along xi_1, S2 pencil along xi_2, S3 column
//                    (i, j) = (a, b) along xi_3, stored straight to HBM;
//   IProductWRTBase: column (i, j) = (a, b): JW f, then B^T along xi_3, S8
//                    pencil along xi_2, S9 pencil along xi_1, stored to HBM.
// Two barriers per tile.  Each CTA walks its tiles persistently, in one of
// two input modes (the launch's `stages`):
//  * 0: the next tile's inputs are loaded into registers while the current
//    tile's later phases run (one tile of look-ahead), with an L2 prefetch
//    two tiles further ahead;
//  * S >= 1: a ring of S shared-memory slots, each filled with one tile's
//    inputs by 1D bulk copies (TMA) that thread 0 issues as soon as the slot
//    has been read (S tiles of look-ahead, no registers held); ragged words
//    of ranges that are not 16-byte aligned are copied by thread 0 with plain
//    loads before it arms the slot's mbarrier, whose wait is bounded (a copy
//    that never lands sets the plan's status word, nothing hangs).
#pragma once
#include "helm_pair.cuh"

namespace spx {

template <int P, int QOFF>
struct SfParams {
  KParams<float, P, P, QOFF> k;
  int stages;                        // ring slots (0: inputs carried in registers)
  int eb;                            // elements per tile
  uint32_t off_a, off_c, off_f;      // byte offsets of the work buffers
  uint32_t off_ring, slot_bytes;     // input ring: byte offset, bytes per slot
};

// Inputs of one tile carried in registers: BwdTrans the S1 coefficients
// (n values), IProductWRTBase the column's f and JW (Q values each).
template <int OP, int P, int Q>
struct SfCarry {
  static constexpr int N = OP == OP_BWD ? P + 1 : 2 * Q;
  float2 v[N];
};

template <int OP, int P, int Q>
__device__ __forceinline__ void sf_load(const KParams<float, P, P, Q - P>& p, const Tile& t, int pi, int a, int b,
                                        SfCarry<OP, P, Q>& cr) {
  constexpr int n = P + 1, Q2 = Q * Q, Q3 = Q * Q * Q;
  constexpr int64_t n3 = int64_t(n) * n * n;
  const int npair = (t.count + 1) / 2;
  if (pi >= npair) return;
  const int64_t e0 = int64_t(t.first) + pi;
  const int64_t e1 = pi + npair < t.count ? e0 + npair : e0;
  if constexpr (OP == OP_BWD) {
    if (a < n && b < n) {
      const float* u0 = p.in0 + e0 * n3 + (b * n + a) * n;
      const float* u1 = p.in0 + e1 * n3 + (b * n + a) * n;
#pragma unroll
      for (int k = 0; k < n; ++k) cr.v[k] = Lane<float2>::ldcs2(u0 + k, u1 + k);
    }
  } else {
    const float* f0 = p.in0 + e0 * Q3 + b * Q + a;
    const float* f1 = p.in0 + e1 * Q3 + b * Q + a;
    const float* w0 = p.geom + 7 * e0 * Q3 + 6 * Q3 + b * Q + a;
    const float* w1 = p.geom + 7 * e1 * Q3 + 6 * Q3 + b * Q + a;
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      cr.v[k] = Lane<float2>::ldcs2(f0 + k * Q2, f1 + k * Q2);
      cr.v[Q + k] = Lane<float2>::ldcs2(w0 + k * Q2, w1 + k * Q2);
    }
  }
}

// L2 prefetch of tile ti's input ranges (contiguous in a uniform plan).
template <int OP, int P, int Q>
__device__ __forceinline__ void sf_prefetch(const KParams<float, P, P, Q - P>& p, int ti) {
  constexpr int64_t n3 = int64_t(P + 1) * (P + 1) * (P + 1), Q3 = int64_t(Q) * Q * Q;
  const Tile t = p.tiles[ti];
  if constexpr (OP == OP_BWD) {
    prefetch_l2(p.in0 + int64_t(t.first) * n3, t.count * n3 * 4);
  } else {
    prefetch_l2(p.in0 + int64_t(t.first) * Q3, t.count * Q3 * 4);
    for (int j = 0; j < t.count; ++j) prefetch_l2(p.geom + 7 * (int64_t(t.first) + j) * Q3 + 6 * Q3, Q3 * 4);
  }
}

// Shared-memory slot of the input ring: BwdTrans the tile's coefficient
// range; IProductWRTBase the tile's f range, then one region per element for
// its JW block.  Each range lands at (its address mod 16) into its region.
template <int OP, int P, int Q>
struct SfSlot {
  static constexpr uint32_t n3 = uint32_t(P + 1) * (P + 1) * (P + 1), Q3 = uint32_t(Q) * Q * Q;
  __host__ __device__ static constexpr uint32_t jw_rb() { return ((Q3 * 4 + 15) & ~15u) + 16; }
  __host__ __device__ static constexpr uint32_t f_rb(int eb) { return ((eb * (OP == OP_BWD ? n3 : Q3) * 4 + 15) & ~15u) + 16; }
  __host__ __device__ static constexpr uint32_t bytes(int eb) {
    return OP == OP_BWD ? f_rb(eb) : f_rb(eb) + eb * jw_rb();
  }
};

// Thread 0: inputs of tile ti into a ring slot.  Ragged words by plain copies
// first (released to the consumers by the arrive), then the expected bytes,
// then the bulk copies.
template <int OP, int P, int Q>
__device__ __forceinline__ void sf_issue(const KParams<float, P, P, Q - P>& p, int ti, char* slot, uint64_t* bar,
                                         int eb) {
  using S = SfSlot<OP, P, Q>;
  const Tile t = p.tiles[ti];
  const int64_t e0 = t.first;
  const uint32_t nv = OP == OP_BWD ? S::n3 : S::Q3;
  const float* gf = p.in0 + e0 * nv;
  const uint32_t bf = t.count * nv * 4;
  fence_proxy_async();
  stage_fixup<4>(slot, gf, bf, 0, 1);
  uint32_t tx = stage_bytes(gf, bf);
  if constexpr (OP == OP_IPROD) {
    for (int j = 0; j < t.count; ++j) {
      const float* gw = p.geom + (7 * (e0 + j) + 6) * S::Q3;
      char* r = slot + S::f_rb(eb) + j * S::jw_rb();
      stage_fixup<4>(r, gw, S::Q3 * 4, 0, 1);
      tx += stage_bytes(gw, S::Q3 * 4);
    }
  }
  mbar_arrive_expect_tx(bar, tx);
  stage_issue(slot, gf, bf, bar);
  if constexpr (OP == OP_IPROD) {
    for (int j = 0; j < t.count; ++j) {
      const float* gw = p.geom + (7 * (e0 + j) + 6) * S::Q3;
      stage_issue(slot + S::f_rb(eb) + j * S::jw_rb(), gw, S::Q3 * 4, bar);
    }
  }
}

// Inputs of thread (a, b) of pair pi from a landed slot: BwdTrans its S1
// coefficients (n values), IProductWRTBase its column's JW f (Q values).
template <int OP, int P, int Q>
__device__ __forceinline__ void sf_from_slot(const KParams<float, P, P, Q - P>& p, const Tile& t, const char* slot,
                                             int eb, int pi, int a, int b, float2* v) {
  using S = SfSlot<OP, P, Q>;
  constexpr int n = P + 1, Q2 = Q * Q;
  const int npair = (t.count + 1) / 2;
  if (pi >= npair) return;
  const int j0 = pi, j1 = pi + npair < t.count ? pi + npair : pi;
  const int64_t e0 = t.first;
  const uint32_t nv = OP == OP_BWD ? S::n3 : S::Q3;
  const float* f = reinterpret_cast<const float*>(slot + (reinterpret_cast<uintptr_t>(p.in0 + e0 * nv) & 15));
  if constexpr (OP == OP_BWD) {
    if (a < n && b < n) {
      const float* u0 = f + j0 * nv + (b * n + a) * n;
      const float* u1 = f + j1 * nv + (b * n + a) * n;
#pragma unroll
      for (int k = 0; k < n; ++k) v[k] = make_float2(u0[k], u1[k]);
    }
  } else {
    const float* w0 = reinterpret_cast<const float*>(
        slot + S::f_rb(eb) + j0 * S::jw_rb() + (reinterpret_cast<uintptr_t>(p.geom + (7 * (e0 + j0) + 6) * S::Q3) & 15));
    const float* w1 = reinterpret_cast<const float*>(
        slot + S::f_rb(eb) + j1 * S::jw_rb() + (reinterpret_cast<uintptr_t>(p.geom + (7 * (e0 + j1) + 6) * S::Q3) & 15));
    const float* f0 = f + j0 * nv + b * Q + a;
    const float* f1 = f + j1 * nv + b * Q + a;
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      const int o = k * Q2 + b * Q + a;
      v[k] = Lane<float2>::mul(make_float2(w0[o], w1[o]), make_float2(f0[k * Q2], f1[k * Q2]));
    }
  }
}

// One tile of order P: ceil(count / 2) element pairs of Q^2 threads; pair pi
// holds elements pi and pi + npair of the tile.  `in`: this thread's inputs
// (BwdTrans: its S1 coefficients; IProductWRTBase: its column's JW f).
// `after_sync` runs right after the first barrier, once every thread has
// consumed its inputs; the barrier also ORs `fail` over the CTA, and a true
// result aborts the tile (returns false) before anything is stored.
template <int OP, int P, int Q, class After>
__device__ __forceinline__ bool sf_pair_tile(const KParams<float, P, P, Q - P>& p, const Tile& t, const float2* in,
                                             const uint32_t* offs, int tid, bool fail, After after_sync) {
  using Vt = Lane<float2>;
  using L = PairLayout<P, Q, Vt::M>;
  constexpr int n = P + 1, XS = L::XS, YS = L::YS, ZS = L::ZS;
  constexpr int Q2 = Q * Q, Q3 = Q * Q * Q;
  constexpr int64_t n3 = int64_t(n) * n * n;
  const float* tab = p.tab;
  const int pi = tid / Q2;
  const int cc = tid - pi * Q2;
  const int a = cc % Q, b = cc / Q;
  const int npair = (t.count + 1) / 2;
  const bool act = pi < npair;
  const bool two = pi + npair < t.count;
  const int64_t e0 = int64_t(t.first) + pi, e1 = two ? e0 + npair : e0;
  extern __shared__ __align__(128) char dsm[];
  float2* A = reinterpret_cast<float2*>(dsm + offs[0]) + pi * L::WX;
  float2* C = reinterpret_cast<float2*>(dsm + offs[1]) + pi * L::WC;
  float2* F = reinterpret_cast<float2*>(dsm + offs[2]) + pi * L::WZ;
  if constexpr (OP == OP_BWD) {
    // S1: pencil along p at (q, r) = (a, b): X(q, r, i) = sum_p B[i][p] u[r][q][p] -> A
    if (act && a < n && b < n) {
      float2 x[Q];
      eo_b<P, Q>(tab, in, x);
#pragma unroll
      for (int i = 0; i < Q; ++i) A[a + Q * b + XS * i] = x[i];
    }
    if (__syncthreads_or(fail)) return false;
    after_sync();
    // S2: pencil along q at (i, r) = (a, b): Y(i, r, j) = sum_q B[j][q] X(q, r, i) -> C
    if (act && b < n) {
      float2 v[n], y[Q];
#pragma unroll
      for (int q = 0; q < n; ++q) v[q] = A[q + Q * b + XS * a];
      eo_b<P, Q>(tab, v, y);
#pragma unroll
      for (int j = 0; j < Q; ++j) C[a + Q * b + YS * j] = y[j];
    }
    __syncthreads();
    // S3: column (i, j) = (a, b): u = B y along xi_3 -> HBM
    if (act) {
      float2 y[n], u[Q];
#pragma unroll
      for (int r = 0; r < n; ++r) y[r] = C[a + Q * r + YS * b];
      eo_b<P, Q>(tab, y, u);
      float* o0 = p.out0 + e0 * Q3 + b * Q + a;
      float* o1 = p.out0 + e1 * Q3 + b * Q + a;
#pragma unroll
      for (int k = 0; k < Q; ++k) Vt::stcs2(o0 + k * Q2, o1 + k * Q2, u[k], two);
    }
  } else {
    // S7: column (i, j) = (a, b): B^T (JW f) along xi_3 -> Y3(i, j, r) in C
    if (act) {
      float2 y3[n];
      eo_bt<P, Q>(tab, in, y3);
#pragma unroll
      for (int r = 0; r < n; ++r) C[a + Q * r + YS * b] = y3[r];
    }
    if (__syncthreads_or(fail)) return false;
    after_sync();
    // S8: pencil along j at (i, r) = (a, b): Y2(i, q, r) = sum_j B[j][q] Y3(i, j, r) -> F
    if (act && b < n) {
      float2 v[Q], y2[n];
#pragma unroll
      for (int j = 0; j < Q; ++j) v[j] = C[a + Q * b + YS * j];
      eo_bt<P, Q>(tab, v, y2);
#pragma unroll
      for (int q = 0; q < n; ++q) F[a + Q * b + ZS * q] = y2[q];
    }
    __syncthreads();
    // S9: pencil along i at (q, r) = (a, b): y[r][q][p] = sum_i B[i][p] Y2(i, q, r) -> HBM
    if (act && a < n && b < n) {
      float2 v[Q], y[n];
#pragma unroll
      for (int i = 0; i < Q; ++i) v[i] = F[i + Q * b + ZS * a];
      eo_bt<P, Q>(tab, v, y);
      float* y0 = p.out0 + e0 * n3 + (b * n + a) * n;
      float* y1 = p.out0 + e1 * n3 + (b * n + a) * n;
#pragma unroll
      for (int k = 0; k < n; ++k) Vt::stcs2(y0 + k, y1 + k, y[k], two);
    }
  }
  return true;
}

// Persistent kernel of one order (uniform plan, contiguous tiles).  REG:
// register budget per thread (occupancy class chosen by the autotuner).
template <int OP, int P, int QOFF, int REG>
__global__ void __maxnreg__(REG) sf_pair_kernel(const __grid_constant__ SfParams<P, QOFF> pp) {
  constexpr int Q = P + QOFF;
  constexpr int NV = OP == OP_BWD ? P + 1 : Q;
  extern __shared__ __align__(128) char sm[];
  const auto& p = pp.k;
  const int tid = threadIdx.x;
  const int G = gridDim.x;
  if (p.skip && *p.skip) return;   // uniform across the grid
  if (blockIdx.x >= p.n_tiles) return;
  const uint32_t offs[3] = {pp.off_a, pp.off_c, pp.off_f};
  const int Q2 = Q * Q;
  const int pi = tid / Q2, a = (tid % Q2) % Q, b = (tid % Q2) / Q;
  const int S = pp.stages;
  if (S == 0) {
    if (tid == 0) {
      for (int j = 1; j <= 2; ++j)
        if (blockIdx.x + j * G < p.n_tiles) sf_prefetch<OP, P, Q>(p, blockIdx.x + j * G);
    }
    SfCarry<OP, P, Q> cr;
    sf_load<OP, P, Q>(p, p.tiles[blockIdx.x], pi, a, b, cr);
    for (int ti = blockIdx.x; ti < p.n_tiles; ti += G) {
      if (tid == 0 && ti + 3 * G < p.n_tiles) sf_prefetch<OP, P, Q>(p, ti + 3 * G);
      const int tn = ti + G < p.n_tiles ? ti + G : -1;
      const Tile t = p.tiles[ti];
      float2 v[NV];
      if constexpr (OP == OP_BWD) {
#pragma unroll
        for (int k = 0; k < NV; ++k) v[k] = cr.v[k];
      } else {
#pragma unroll
        for (int k = 0; k < NV; ++k) v[k] = Lane<float2>::mul(cr.v[Q + k], cr.v[k]);
      }
      sf_pair_tile<OP, P, Q>(p, t, v, offs, tid, false, [&] {
        if (tn >= 0) sf_load<OP, P, Q>(p, p.tiles[tn], pi, a, b, cr);
      });
    }
    return;
  }
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm);   // one mbarrier per slot
  const int eb = pp.eb;
  if (tid == 0) {
    for (int s = 0; s < S; ++s) mbar_init(&bar[s], 1);
    fence_barrier_init();
  }
  __syncthreads();
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      const int ti = blockIdx.x + s * G;
      if (ti < p.n_tiles) sf_issue<OP, P, Q>(p, ti, sm + pp.off_ring + s * pp.slot_bytes, &bar[s], eb);
    }
  }
  for (int k = 0;; ++k) {
    const int ti = blockIdx.x + k * G;
    if (ti >= p.n_tiles) break;
    const int s = k % S;
    char* slot = sm + pp.off_ring + s * pp.slot_bytes;
    const bool ok = mbar_wait(&bar[s], (k / S) & 1);
    const Tile t = p.tiles[ti];
    float2 v[NV];
    if (ok) sf_from_slot<OP, P, Q>(p, t, slot, eb, pi, a, b, v);
    const int tn = ti + S * G;
    const bool go = sf_pair_tile<OP, P, Q>(p, t, v, offs, tid, !ok, [&] {
      if (tid == 0 && tn < p.n_tiles) sf_issue<OP, P, Q>(p, tn, slot, &bar[s], eb);
    });
    if (!go) {
      // a copy never landed: record it, then wait (bounded) for the copies
      // still in flight into the other slots before the CTA exits
      if (tid == 0) atomicOr(p.status, kStatusTimeout);
      for (int j = 1; j < S && ti + j * G < p.n_tiles; ++j) mbar_wait(&bar[(k + j) % S], ((k + j) / S) & 1);
      return;
    }
  }
}

}  // namespace spx
