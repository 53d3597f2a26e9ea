// Persistent, tile-based kernel for the elemental operators (§3.3 Collections,
// SumFac strategy re-designed for one GB300).
//
// Work is a list of tiles; a tile is up to `eb` elements of one order P
// (elements bucketed by order, §4.2).  Every CTA walks the tiles
// blockIdx.x, blockIdx.x + gridDim.x, ... and keeps `stages` tiles in flight:
// one thread stages the next tiles' input blocks (coefficients, geometric
// factors, coefficient fields) into a ring of shared-memory slots with 1D bulk
// copies, while all threads evaluate the current tile by sum-factorisation
// through padded shared-memory work buffers.  Outputs are stored straight to
// HBM.  Basis tables B, dB, D of every order the kernel handles travel in the
// kernel parameter block (constant bank).
#pragma once
#include "device_common.cuh"
#include "kernel_params.h"
#include "lanes.cuh"

namespace spx {

// ---------------------------------------------------------------------------
// Streams: which element blocks an operator reads.
// ---------------------------------------------------------------------------
template <typename T>
struct StreamDesc {
  const T* base;   // nullptr: stream absent
  int64_t len;     // values copied per element
  int mult;        // element offset multiplier (block = mult * off_e values)
  int64_t boff;    // offset of the copied part inside the element block
  bool quad;       // off_e from quad offsets (else coefficient offsets)
  bool whole;      // copies the entire block: consecutive elements are contiguous
};

template <typename T, int DIM, int OP, class Prm>
__device__ __forceinline__ int op_streams(const Prm& p, int P, int Q, StreamDesc<T>* s) {
  const int64_t nd = DIM == 3 ? int64_t(P + 1) * (P + 1) * (P + 1) : int64_t(P + 1) * (P + 1);
  const int64_t qd = DIM == 3 ? int64_t(Q) * Q * Q : int64_t(Q) * Q;
  constexpr int nf = DIM == 3 ? 7 : 4;
  int k = 0;
  switch (OP) {
    case OP_BWD:
      s[k++] = {p.in0, nd, 1, 0, false, true};
      break;
    case OP_IPROD:
      s[k++] = {p.in0, qd, 1, 0, true, true};
      s[k++] = {p.geom, qd, nf, (nf - 1) * qd, true, false};
      break;
    case OP_DERIV:
      s[k++] = {p.in0, qd, 1, 0, true, true};
      s[k++] = {p.geom, DIM * DIM * qd, DIM * DIM, 0, true, true};
      break;
    case OP_HELM:
      s[k++] = {p.in0, nd, 1, 0, false, true};
      s[k++] = {p.geo_direct ? nullptr : p.geom, nf * qd, nf, 0, true, true};
      s[k++] = {p.lam_f, qd, 1, 0, true, true};
      s[k++] = {p.kap_f, qd, 1, 0, true, true};
      break;
    case OP_ADJ:
      s[k++] = {p.in0, nd, 1, 0, false, true};
      s[k++] = {p.in1, nd, 1, 0, false, true};
      s[k++] = {p.geom, nf * qd, nf, 0, true, true};
      s[k++] = {p.lam_f, qd, 1, 0, true, true};
      s[k++] = {p.kap_f, qd, 1, 0, true, true};
      break;
    case OP_FWD:
      s[k++] = {p.in0, qd, 1, 0, true, true};
      s[k++] = {p.geom, qd, nf, (nf - 1) * qd, true, false};
      break;
    case OP_SENSOR:
      s[k++] = {p.in0, nd, 1, 0, false, true};
      s[k++] = {p.geom, qd, nf, (nf - 1) * qd, true, false};
      break;
    case OP_DIAG:
      s[k++] = {p.geom, nf * qd, nf, 0, true, true};
      s[k++] = {p.lam_f, qd, 1, 0, true, true};
      break;
  }
  return k;
}

// element offsets (uniform plans have no offset arrays)
template <int DIM, class Prm>
__device__ __forceinline__ int64_t coef_off_of(const Prm& p, int64_t e, int P) {
  const int64_t n = P + 1;
  return p.coef_off ? p.coef_off[e] : e * (DIM == 3 ? n * n * n : n * n);
}
template <int DIM, class Prm>
__device__ __forceinline__ int64_t quad_off_of(const Prm& p, int64_t e, int Q) {
  return p.quad_off ? p.quad_off[e] : e * (DIM == 3 ? int64_t(Q) * Q * Q : int64_t(Q) * Q);
}
template <class Prm>
__device__ __forceinline__ int64_t elem_id(const Prm& p, const Tile& t, int j) {
  return t.contig ? int64_t(p.ids ? p.ids[t.first] : t.first) + j : int64_t(p.ids ? p.ids[t.first + j] : t.first + j);
}

__device__ __forceinline__ uint32_t erb_bytes(int64_t len, int sz) {  // per-element region bytes
  return static_cast<uint32_t>(((len * sz + 15) & ~int64_t(15)) + 16);
}

// Producer: stage tile `ti` into slot `slot` (thread 0 only).
template <typename T, int DIM, int OP, int QOFF, class Prm>
__device__ void issue_tile(const Prm& p, char* sm, uint64_t* bars, int slot, int ti) {
  const Tile t = p.tiles[ti];
  const int P = t.P, Q = t.P + QOFF;
  StreamDesc<T> sd[5];
  const int ns = op_streams<T, DIM, OP>(p, P, Q, sd);
  char* slotp = sm + p.slot_base + slot * p.slot_bytes;
  uint32_t tx = 0;
  for (int pass = 0; pass < 2; ++pass) {
    if (pass == 1) mbar_arrive_expect_tx(&bars[slot], tx);
#pragma unroll
    for (int s = 0; s < 5; ++s) {
      if (s >= ns || !sd[s].base) continue;
      char* region = slotp + p.region_off[s];
      if (t.contig && sd[s].whole) {
        const int64_t e0 = elem_id(p, t, 0);
        const int64_t off = sd[s].quad ? quad_off_of<DIM>(p, e0, Q) : coef_off_of<DIM>(p, e0, P);
        const T* g = sd[s].base + sd[s].mult * off + sd[s].boff;
        const uint32_t bytes = static_cast<uint32_t>(t.count * sd[s].len * sizeof(T));
        if (pass == 0) tx += stage_bytes(g, bytes);
        else stage_issue(region, g, bytes, &bars[slot]);
      } else {
        const uint32_t erb = erb_bytes(sd[s].len, sizeof(T));
        for (int j = 0; j < t.count; ++j) {
          const int64_t e = elem_id(p, t, j);
          const int64_t off = sd[s].quad ? quad_off_of<DIM>(p, e, Q) : coef_off_of<DIM>(p, e, P);
          const T* g = sd[s].base + sd[s].mult * off + sd[s].boff;
          const uint32_t bytes = static_cast<uint32_t>(sd[s].len * sizeof(T));
          if (pass == 0) tx += stage_bytes(g, bytes);
          else stage_issue(region + j * erb, g, bytes, &bars[slot]);
        }
      }
    }
  }
}

// Per-tile context handed to the operator bodies.
template <typename T>
struct Ctx {
  char* sm;
  T* work[8];
  const uint32_t* soff;   // [5][kMaxEB] value offsets of staged element data (relative to sm)
  const int64_t* gcoef;   // [kMaxEB] coefficient offsets of the tile's elements
  const int64_t* gquad;   // [kMaxEB] quadrature offsets
  int ne, tid, nthr;
  int* tab_order;         // order whose tables are in work buffer 4 (shared)
  T* extra;               // kFwdExtra values after the tile metadata (FwdTrans)
  int* status;            // the plan's device status word
  bool has_lam, has_kap;
  T lam;
  const T* geom_g;        // geometry in global memory when it is not staged (geo_direct), else nullptr
  __device__ const T* staged(int s, int j) const { return reinterpret_cast<const T*>(sm) + soff[s * kMaxEB + j]; }
};

// Input / output element bases for the contraction loops.
struct BaseStride {   // element e at e * es
  int es;
  __device__ __forceinline__ int64_t operator()(int e) const { return int64_t(e) * es; }
};
struct BaseTable32 {  // element e at t[e]
  const uint32_t* t;
  __device__ __forceinline__ int64_t operator()(int e) const { return t[e]; }
};
struct BaseTable64 {
  const int64_t* t;
  __device__ __forceinline__ int64_t operator()(int e) const { return t[e]; }
};

// General contraction (see device_common.cuh for the index convention) with
// per-element bases, optional elementwise product of two inputs (PROD) and
// store / accumulate (MODE 0 / 1).
template <int AX, int N0, int N1, int N2, int M, bool TR, int MODE, bool PROD, int IS1, int IS2, int OS1, int OS2,
          typename T, class IB, class IB2, class OB>
__device__ __forceinline__ void contract_g(const T* __restrict__ in, IB ib, const T* __restrict__ in2, IB2 ib2,
                                           T* __restrict__ out, OB ob, const T* __restrict__ A, int ne, int tid,
                                           int nthr) {
  constexpr int NA = AX == 0 ? N0 : (AX == 1 ? N1 : N2);
  constexpr int OA = AX == 0 ? N1 : N0;
  constexpr int OB_ = AX == 2 ? N1 : N2;
  constexpr int NP = OA * OB_;
  constexpr int ISA = AX == 0 ? 1 : (AX == 1 ? IS1 : IS2);
  constexpr int OSA = AX == 0 ? 1 : (AX == 1 ? OS1 : OS2);
  constexpr int ISa = AX == 0 ? IS1 : 1;
  constexpr int OSa = AX == 0 ? OS1 : 1;
  constexpr int ISb = AX == 2 ? IS1 : IS2;
  constexpr int OSb = AX == 2 ? OS1 : OS2;
  for (int pc = tid; pc < ne * NP; pc += nthr) {
    const int e = pc / NP;
    const int r = pc - e * NP;
    const int b = r / OA;
    const int a = r - b * OA;
    const int lo = a * ISa + b * ISb;
    const T* src = in + ib(e) + lo;
    T* dst = out + ob(e) + a * OSa + b * OSb;
    T v[NA];
    if (PROD) {
      const T* src2 = in2 + ib2(e) + lo;
#pragma unroll
      for (int c = 0; c < NA; ++c) v[c] = src[c * ISA] * src2[c * ISA];
    } else {
#pragma unroll
      for (int c = 0; c < NA; ++c) v[c] = src[c * ISA];
    }
#pragma unroll
    for (int m = 0; m < M; ++m) {
      T acc = MODE == 1 ? dst[m * OSA] : T(0);
#pragma unroll
      for (int c = 0; c < NA; ++c) acc = fma(TR ? A[c * M + m] : A[m * NA + c], v[c], acc);
      dst[m * OSA] = acc;
    }
  }
}

// Fused pencil along axis 2 (3D) or axis 1 (2D): u = B v (n -> Q) stored to
// U, and d = D u stored to Dd.
template <int AX, int N0, int N1, int N2, int Q, int S1, int S2, int ES, typename T>
__device__ __forceinline__ void bwd_and_deriv_pencil(const T* __restrict__ in, T* __restrict__ U, T* __restrict__ Dd,
                                                     const T* __restrict__ B, const T* __restrict__ D, int ne,
                                                     int tid, int nthr) {
  // input extents (N0, N1, N2) with N_AX = n; output extent Q on AX.
  constexpr int NA = AX == 1 ? N1 : N2;
  constexpr int OA = N0;
  constexpr int OB_ = AX == 2 ? N1 : N2;
  constexpr int NP = OA * OB_;
  constexpr int SA = AX == 1 ? S1 : S2;
  constexpr int Sb = AX == 2 ? S1 : S2;
  for (int pc = tid; pc < ne * NP; pc += nthr) {
    const int e = pc / NP;
    const int r = pc - e * NP;
    const int b = r / OA;
    const int a = r - b * OA;
    const int base = e * ES + a + b * Sb;
    T v[NA];
#pragma unroll
    for (int c = 0; c < NA; ++c) v[c] = in[base + c * SA];
    T u[Q];
#pragma unroll
    for (int m = 0; m < Q; ++m) {
      T acc = T(0);
#pragma unroll
      for (int c = 0; c < NA; ++c) acc = fma(B[m * NA + c], v[c], acc);
      u[m] = acc;
      U[base + m * SA] = acc;
    }
#pragma unroll
    for (int m = 0; m < Q; ++m) {
      T acc = T(0);
#pragma unroll
      for (int c = 0; c < Q; ++c) acc = fma(D[m * Q + c], u[c], acc);
      Dd[base + m * SA] = acc;
    }
  }
}

// Fused pencil along the last axis for the transposed half of Helmholtz:
// r = R + D^T G (Q values), z = B^T r (n values) stored to Z.
template <int AX, int N0, int N1, int Q, int n, int S1, int S2, int ES, typename T>
__device__ __forceinline__ void dt_and_bt_pencil(const T* __restrict__ R, const T* __restrict__ G, T* __restrict__ Z,
                                                 const T* __restrict__ B, const T* __restrict__ D, int ne, int tid,
                                                 int nthr) {
  constexpr int OA = N0;
  constexpr int OB_ = AX == 2 ? N1 : 1;
  constexpr int NP = OA * OB_;
  constexpr int SA = AX == 1 ? S1 : S2;
  constexpr int Sb = AX == 2 ? S1 : S2;
  for (int pc = tid; pc < ne * NP; pc += nthr) {
    const int e = pc / NP;
    const int r = pc - e * NP;
    const int b = r / OA;
    const int a = r - b * OA;
    const int base = e * ES + a + b * Sb;
    T g[Q], rr[Q];
#pragma unroll
    for (int c = 0; c < Q; ++c) {
      g[c] = G[base + c * SA];
      rr[c] = R[base + c * SA];
    }
#pragma unroll
    for (int m = 0; m < Q; ++m) {
      T acc = rr[m];
#pragma unroll
      for (int c = 0; c < Q; ++c) acc = fma(D[c * Q + m], g[c], acc);
      rr[m] = acc;
    }
#pragma unroll
    for (int m = 0; m < n; ++m) {
      T acc = T(0);
#pragma unroll
      for (int c = 0; c < Q; ++c) acc = fma(B[c * n + m], rr[c], acc);
      Z[base + m * SA] = acc;
    }
  }
}

// ===========================================================================
// Operator bodies.  Each returns after its last store; `release()` is called
// once the staged inputs of the tile are no longer needed.
// Table layout per order: B[Q][n], dB[Q][n], D[Q][Q].
// ===========================================================================
template <typename T, int DIM, int P, int Q>
struct Shape {
  static constexpr int n = P + 1;
  static constexpr int S1 = Q | 1;                    // odd padded row stride
  static constexpr int S2 = DIM == 3 ? S1 * Q : 0;
  static constexpr int WS = DIM == 3 ? S1 * Q * Q : S1 * Q;
  static constexpr int ND = DIM == 3 ? n * n * n : n * n;
  static constexpr int QD = DIM == 3 ? Q * Q * Q : Q * Q;
};

#define SPX_SYNC() __syncthreads()

// ---- BwdTrans -------------------------------------------------------------
template <typename T, int DIM, int P, int Q, class Rel>
__device__ void body_bwd(const T* tab, const Ctx<T>& c, T* out, Rel release) {
  using S = Shape<T, DIM, P, Q>;
  constexpr int n = S::n;
  const T* B = tab;
  BaseTable32 in0{c.soff};
  if (DIM == 3) {
    contract_g<0, n, n, n, Q, false, 0, false, n, n * n, S::S1, S::S2>(
        reinterpret_cast<const T*>(c.sm), in0, (const T*)nullptr, in0, c.work[0], BaseStride{S::WS}, B, c.ne, c.tid,
        c.nthr);
    SPX_SYNC();
    release();
    contract_g<1, Q, n, n, Q, false, 0, false, S::S1, S::S2, S::S1, S::S2>(
        c.work[0], BaseStride{S::WS}, (const T*)nullptr, BaseStride{0}, c.work[1], BaseStride{S::WS}, B, c.ne, c.tid,
        c.nthr);
    SPX_SYNC();
    contract_g<2, Q, Q, n, Q, false, 0, false, S::S1, S::S2, Q, Q * Q>(
        c.work[1], BaseStride{S::WS}, (const T*)nullptr, BaseStride{0}, out, BaseTable64{c.gquad}, B, c.ne, c.tid,
        c.nthr);
  } else {
    contract_g<0, n, n, 1, Q, false, 0, false, n, 0, S::S1, 0>(reinterpret_cast<const T*>(c.sm), in0,
                                                               (const T*)nullptr, in0, c.work[0], BaseStride{S::WS},
                                                               B, c.ne, c.tid, c.nthr);
    SPX_SYNC();
    release();
    contract_g<1, Q, n, 1, Q, false, 0, false, S::S1, 0, Q, 0>(c.work[0], BaseStride{S::WS}, (const T*)nullptr,
                                                               BaseStride{0}, out, BaseTable64{c.gquad}, B, c.ne,
                                                               c.tid, c.nthr);
  }
}

// ---- IProductWRTBase --------------------------------------------------------
template <typename T, int DIM, int P, int Q, class Rel>
__device__ void body_iprod(const T* tab, const Ctx<T>& c, T* out, Rel release) {
  using S = Shape<T, DIM, P, Q>;
  constexpr int n = S::n;
  const T* B = tab;
  BaseTable32 f{c.soff}, jw{c.soff + kMaxEB};
  const T* sm = reinterpret_cast<const T*>(c.sm);
  if (DIM == 3) {
    // (f * JW) contracted along axis 2 with B^T
    contract_g<2, Q, Q, Q, n, true, 0, true, Q, Q * Q, S::S1, S::S2>(sm, f, sm, jw, c.work[0], BaseStride{S::WS}, B,
                                                                      c.ne, c.tid, c.nthr);
    SPX_SYNC();
    release();
    contract_g<1, Q, Q, n, n, true, 0, false, S::S1, S::S2, S::S1, S::S2>(
        c.work[0], BaseStride{S::WS}, (const T*)nullptr, BaseStride{0}, c.work[1], BaseStride{S::WS}, B, c.ne, c.tid,
        c.nthr);
    SPX_SYNC();
    contract_g<0, Q, n, n, n, true, 0, false, S::S1, S::S2, n, n * n>(
        c.work[1], BaseStride{S::WS}, (const T*)nullptr, BaseStride{0}, out, BaseTable64{c.gcoef}, B, c.ne, c.tid,
        c.nthr);
  } else {
    contract_g<1, Q, Q, 1, n, true, 0, true, Q, 0, S::S1, 0>(sm, f, sm, jw, c.work[0], BaseStride{S::WS}, B, c.ne,
                                                              c.tid, c.nthr);
    SPX_SYNC();
    release();
    contract_g<0, Q, n, 1, n, true, 0, false, S::S1, 0, n, 0>(c.work[0], BaseStride{S::WS}, (const T*)nullptr,
                                                              BaseStride{0}, out, BaseTable64{c.gcoef}, B, c.ne,
                                                              c.tid, c.nthr);
  }
}

// ---- PhysDeriv --------------------------------------------------------------
template <typename T, int DIM, int P, int Q, class Rel>
__device__ void body_deriv(const T* tab, const Ctx<T>& c, T* o0, T* o1, T* o2, Rel release) {
  using S = Shape<T, DIM, P, Q>;
  constexpr int n = S::n;
  const T* D = tab + 2 * Q * n;
  BaseTable32 f{c.soff};
  const T* sm = reinterpret_cast<const T*>(c.sm);
  constexpr int QD = S::QD;
  if (DIM == 3) {
    contract_g<0, Q, Q, Q, Q, false, 0, false, Q, Q * Q, S::S1, S::S2>(sm, f, sm, f, c.work[0], BaseStride{S::WS},
                                                                        D, c.ne, c.tid, c.nthr);
    contract_g<1, Q, Q, Q, Q, false, 0, false, Q, Q * Q, S::S1, S::S2>(sm, f, sm, f, c.work[1], BaseStride{S::WS},
                                                                        D, c.ne, c.tid, c.nthr);
    contract_g<2, Q, Q, Q, Q, false, 0, false, Q, Q * Q, S::S1, S::S2>(sm, f, sm, f, c.work[2], BaseStride{S::WS},
                                                                        D, c.ne, c.tid, c.nthr);
  } else {
    contract_g<0, Q, Q, 1, Q, false, 0, false, Q, 0, S::S1, 0>(sm, f, sm, f, c.work[0], BaseStride{S::WS}, D, c.ne,
                                                               c.tid, c.nthr);
    contract_g<1, Q, Q, 1, Q, false, 0, false, Q, 0, S::S1, 0>(sm, f, sm, f, c.work[1], BaseStride{S::WS}, D, c.ne,
                                                               c.tid, c.nthr);
  }
  SPX_SYNC();
  T* outs[3] = {o0, o1, o2};
  for (int pt = c.tid; pt < c.ne * QD; pt += c.nthr) {
    const int e = pt / QD;
    const int q = pt - e * QD;
    const int i = q % Q;
    const int j = (q / Q) % Q;
    const int k = DIM == 3 ? q / (Q * Q) : 0;
    const int w = e * S::WS + i + j * S::S1 + k * S::S2;
    const T* X = c.staged(1, e) + q;  // dxi_a/dx_m blocks
    T r[DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a) r[a] = c.work[a][w];
#pragma unroll
    for (int m = 0; m < DIM; ++m) {
      T acc = T(0);
#pragma unroll
      for (int a = 0; a < DIM; ++a) acc = fma(X[(a * DIM + m) * QD], r[a], acc);
      outs[m][c.gquad[e] + q] = acc;
    }
  }
  (void)release;
}

// ---- Helmholtz --------------------------------------------------------------
template <typename T, int DIM, int P, int Q, class Rel>
__device__ void body_helm(const T* tab, const Ctx<T>& c, T* out, Rel release) {
  using S = Shape<T, DIM, P, Q>;
  constexpr int n = S::n, S1 = S::S1, S2 = S::S2, WS = S::WS, QD = S::QD;
  const T* B = tab;
  const T* D = tab + 2 * Q * n;
  BaseTable32 in0{c.soff};
  const T* sm = reinterpret_cast<const T*>(c.sm);
  T *W0 = c.work[0], *W1 = c.work[1], *W2 = c.work[2], *W3 = c.work[3];
  if (DIM == 3) {
    contract_g<0, n, n, n, Q, false, 0, false, n, n * n, S1, S2>(sm, in0, sm, in0, W0, BaseStride{WS}, B, c.ne,
                                                                  c.tid, c.nthr);
    SPX_SYNC();
    contract_g<1, Q, n, n, Q, false, 0, false, S1, S2, S1, S2>(W0, BaseStride{WS}, W0, BaseStride{WS}, W1,
                                                                BaseStride{WS}, B, c.ne, c.tid, c.nthr);
    SPX_SYNC();
    bwd_and_deriv_pencil<2, Q, Q, n, Q, S1, S2, WS>(W1, W2, W3, B, D, c.ne, c.tid, c.nthr);  // U -> W2, d2 -> W3
    SPX_SYNC();
    contract_g<0, Q, Q, Q, Q, false, 0, false, S1, S2, S1, S2>(W2, BaseStride{WS}, W2, BaseStride{WS}, W0,
                                                                BaseStride{WS}, D, c.ne, c.tid, c.nthr);
    contract_g<1, Q, Q, Q, Q, false, 0, false, S1, S2, S1, S2>(W2, BaseStride{WS}, W2, BaseStride{WS}, W1,
                                                                BaseStride{WS}, D, c.ne, c.tid, c.nthr);
    SPX_SYNC();
  } else {
    contract_g<0, n, n, 1, Q, false, 0, false, n, 0, S1, 0>(sm, in0, sm, in0, W0, BaseStride{WS}, B, c.ne, c.tid,
                                                             c.nthr);
    SPX_SYNC();
    bwd_and_deriv_pencil<1, Q, n, 1, Q, S1, 0, WS>(W0, W2, W3, B, D, c.ne, c.tid, c.nthr);  // U -> W2, d1 -> W3
    SPX_SYNC();
    contract_g<0, Q, Q, 1, Q, false, 0, false, S1, 0, S1, 0>(W2, BaseStride{WS}, W2, BaseStride{WS}, W0,
                                                              BaseStride{WS}, D, c.ne, c.tid, c.nthr);
    SPX_SYNC();
  }
  // pointwise: W2 <- lambda JW u; (W0, W1, W3) <- kappa G grad u  (2D: W0, W3)
  constexpr int nf = DIM == 3 ? 7 : 4;
  for (int pt = c.tid; pt < c.ne * QD; pt += c.nthr) {
    const int e = pt / QD;
    const int q = pt - e * QD;
    const int i = q % Q;
    const int j = (q / Q) % Q;
    const int k = DIM == 3 ? q / (Q * Q) : 0;
    const int w = e * WS + i + j * S1 + k * S2;
    const T* G = c.staged(1, e) + q;
    const T kap = c.has_kap ? c.staged(3, e)[q] : T(1);
    const T lam = c.has_lam ? c.staged(2, e)[q] : c.lam;
    if (DIM == 3) {
      const T d0 = W0[w], d1 = W1[w], d2 = W3[w];
      const T g00 = G[0], g01 = G[QD], g02 = G[2 * QD], g11 = G[3 * QD], g12 = G[4 * QD], g22 = G[5 * QD];
      const T jw = G[6 * QD];
      W0[w] = kap * (g00 * d0 + g01 * d1 + g02 * d2);
      W1[w] = kap * (g01 * d0 + g11 * d1 + g12 * d2);
      W3[w] = kap * (g02 * d0 + g12 * d1 + g22 * d2);
      W2[w] = lam * jw * W2[w];
    } else {
      const T d0 = W0[w], d1 = W3[w];
      const T g00 = G[0], g01 = G[QD], g11 = G[2 * QD], jw = G[3 * QD];
      W0[w] = kap * (g00 * d0 + g01 * d1);
      W3[w] = kap * (g01 * d0 + g11 * d1);
      W2[w] = lam * jw * W2[w];
    }
  }
  (void)nf;
  SPX_SYNC();
  release();
  if (DIM == 3) {
    contract_g<0, Q, Q, Q, Q, true, 1, false, S1, S2, S1, S2>(W0, BaseStride{WS}, W0, BaseStride{WS}, W2,
                                                               BaseStride{WS}, D, c.ne, c.tid, c.nthr);
    SPX_SYNC();
    contract_g<1, Q, Q, Q, Q, true, 1, false, S1, S2, S1, S2>(W1, BaseStride{WS}, W1, BaseStride{WS}, W2,
                                                               BaseStride{WS}, D, c.ne, c.tid, c.nthr);
    SPX_SYNC();
    dt_and_bt_pencil<2, Q, Q, Q, n, S1, S2, WS>(W2, W3, W0, B, D, c.ne, c.tid, c.nthr);  // -> W0 (Q,Q,n)
    SPX_SYNC();
    contract_g<1, Q, Q, n, n, true, 0, false, S1, S2, S1, S2>(W0, BaseStride{WS}, W0, BaseStride{WS}, W1,
                                                               BaseStride{WS}, B, c.ne, c.tid, c.nthr);
    SPX_SYNC();
    contract_g<0, Q, n, n, n, true, 0, false, S1, S2, n, n * n>(W1, BaseStride{WS}, W1, BaseStride{WS}, out,
                                                                 BaseTable64{c.gcoef}, B, c.ne, c.tid, c.nthr);
  } else {
    contract_g<0, Q, Q, 1, Q, true, 1, false, S1, 0, S1, 0>(W0, BaseStride{WS}, W0, BaseStride{WS}, W2,
                                                             BaseStride{WS}, D, c.ne, c.tid, c.nthr);
    SPX_SYNC();
    dt_and_bt_pencil<1, Q, 1, Q, n, S1, 0, WS>(W2, W3, W1, B, D, c.ne, c.tid, c.nthr);  // -> W1 (Q,n)
    SPX_SYNC();
    contract_g<0, Q, n, 1, n, true, 0, false, S1, 0, n, 0>(W1, BaseStride{WS}, W1, BaseStride{WS}, out,
                                                            BaseTable64{c.gcoef}, B, c.ne, c.tid, c.nthr);
  }
}

// ---- Helmholtz, 3D: Q^2 threads per element, column and pencil roles -------
// Thread (a, b) of element `el` (a, b in [0, Q)) plays three roles:
//  * column owner of (i, j) = (a, b): the contractions along xi_3, the
//    gradient along xi_3 and the pointwise geometric factors, in registers;
//  * pencil owner along xi_1 at (j, k) = (a, b) and along xi_2 at
//    (i, k) = (a, b) for the gradient and transposed gradient;
//  * the BwdTrans / IProduct contractions along xi_1, xi_2 (S1, S2, S8, S9)
//    have fewer pencils than an element has threads: their work items are
//    numbered densely over the whole CTA instead.
// Data moves between roles through shared memory with odd row strides S, so
// that the scalar accesses of consecutive threads fall in distinct banks.
// Matrices are indexed with compile-time indices only (constant bank).
// Buffers per element (row stride S = Q | 1, plane stride Q*S):
//   W0: X[r][q][i] (S1 -> S2), U[k][j][i] (S3 -> S4), Y3[r][i][j] (S7 -> S8)
//   W1: Y[j][i][r] (rows of n, stride SN = n | 1; S2 -> S3), then Y2[r][q][i] (S8 -> S9)
//   W2: d0 (S4 -> S5), g0 (S5 -> S6), D^T-contracted g0 (S6 -> S7), same layout
//   W3: d1, g1, D^T-contracted g1
template <typename T, int P, int Q>
struct RoleShape {
  static constexpr int n = P + 1;
  static constexpr int S = Q | 1;
  static constexpr int SN = n | 1;
  static constexpr int PL = Q * S;                              // plane stride of Q x Q fields
  static constexpr int WS0 = n * Q * S > n * n * S ? n * Q * S : n * n * S;
  static constexpr int WS1 = Q * Q * SN > n * n * S ? Q * Q * SN : n * n * S;
  static constexpr int WS = Q * PL > WS0 ? (Q * PL > WS1 ? Q * PL : WS1) : (WS0 > WS1 ? WS0 : WS1);
};

// Middle phases of the 3D Helmholtz bodies with Q^2 threads per element
// (RoleShape buffers; PL = Q S plane stride): from U[k][j][i] in W2 (the
// caller's U buffer; W3, W4 are the caller's two gradient buffers) and the
// column's u, d2 = du/dxi_3 in registers, the gradient pencils along xi_1,
// xi_2 (S4), the pointwise geometric factors (S5), the transposed-gradient
// pencils (S6).  Returns after the S6 barrier with z = D^T g2 + lambda JW u
// (the column's xi_3 part and the mass term) in registers and the xi_1, xi_2
// transposed parts in W3, W4 at (k, j, i) = k PL + j S + i.
template <typename T, int P, int Q, class Rel>
__device__ __forceinline__ void helm_mid(const T* tab, const Ctx<T>& c, int el, int a, int b, bool act, T* W2, T* W3,
                                         T* W4, T (&u)[Q], T (&g2)[Q], T (&z)[Q], Rel& release) {
  using S_ = RoleShape<T, P, Q>;
  constexpr int S = S_::S, PL = S_::PL;
  constexpr int Q2 = Q * Q, Q3 = Q * Q * Q;
  // S4: gradient pencils: along xi_1 at (j, k) = (a, b) -> W3, along xi_2 at (i, k) = (a, b) -> W4
  if (act) {
    T v[Q], d[Q];
#pragma unroll
    for (int m = 0; m < Q; ++m) v[m] = W2[b * PL + a * S + m];
    eo_d<P, Q, false>(tab, v, d);
#pragma unroll
    for (int i = 0; i < Q; ++i) W3[b * PL + a * S + i] = d[i];
#pragma unroll
    for (int m = 0; m < Q; ++m) v[m] = W2[b * PL + m * S + a];
    eo_d<P, Q, false>(tab, v, d);
#pragma unroll
    for (int j = 0; j < Q; ++j) W4[b * PL + j * S + a] = d[j];
  }
  SPX_SYNC();
  // S5: column (i, j) = (a, b): pointwise; g0 -> W3, g1 -> W4, g2 and lambda JW in
  // registers; then z = D^T g2 + lambda JW u along xi_3
  if (act) {
    // geometric factors: staged in shared memory, or read from L2 (prefetched at the tile's start)
    const T* G = (c.geom_g ? c.geom_g + 7 * c.gquad[el] : c.staged(1, el)) + b * Q + a;
    const T* lf = c.has_lam ? c.staged(2, el) + b * Q + a : nullptr;
    const T* kf = c.has_kap ? c.staged(3, el) + b * Q + a : nullptr;
    T lj[Q];
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      const int w = k * PL + b * S + a;
      const T d0 = W3[w], d1 = W4[w], d2 = g2[k];
      const T* g = G + k * Q2;
      const T g00 = g[0], g01 = g[Q3], g02 = g[2 * Q3], g11 = g[3 * Q3], g12 = g[4 * Q3], g22 = g[5 * Q3];
      const T jw = g[6 * Q3];
      T r0 = fma(g02, d2, fma(g01, d1, g00 * d0));
      T r1 = fma(g12, d2, fma(g11, d1, g01 * d0));
      T r2 = fma(g22, d2, fma(g12, d1, g02 * d0));
      if (kf) {
        const T kk = kf[k * Q2];
        r0 *= kk;
        r1 *= kk;
        r2 *= kk;
      }
      W3[w] = r0;
      W4[w] = r1;
      g2[k] = r2;
      lj[k] = (lf ? lf[k * Q2] : c.lam) * jw;
    }
    eo_d<P, Q, true>(tab, g2, z);
#pragma unroll
    for (int k = 0; k < Q; ++k) z[k] = fma(lj[k], u[k], z[k]);
  }
  SPX_SYNC();
  release();
  // S6: transposed-gradient pencils, in place: along xi_1 at (j, k) = (a, b) in W3,
  // along xi_2 at (i, k) = (a, b) in W4
  if (act) {
    T v[Q], d[Q];
#pragma unroll
    for (int m = 0; m < Q; ++m) v[m] = W3[b * PL + a * S + m];
    eo_d<P, Q, true>(tab, v, d);
#pragma unroll
    for (int i = 0; i < Q; ++i) W3[b * PL + a * S + i] = d[i];
#pragma unroll
    for (int m = 0; m < Q; ++m) v[m] = W4[b * PL + m * S + a];
    eo_d<P, Q, true>(tab, v, d);
#pragma unroll
    for (int j = 0; j < Q; ++j) W4[b * PL + j * S + a] = d[j];
  }
  SPX_SYNC();
}

template <typename T, int P, int Q, class Rel>
__device__ void body_helm_role(const T* tab, const Ctx<T>& c, T* out, Rel release) {
  using S_ = RoleShape<T, P, Q>;
  constexpr int n = S_::n, S = S_::S, SN = S_::SN, PL = S_::PL, WS = S_::WS;
  constexpr int Q2 = Q * Q;
  const int el = c.tid / Q2;
  const int cc = c.tid - el * Q2;
  const int a = cc % Q, b = cc / Q;
  const bool act = el < c.ne;
  const int ne = c.ne, tid = c.tid;
  T* W0 = c.work[0];
  T* W1 = c.work[1];
  // S1, S2, S8 and S9 have fewer pencils than the element has threads; their
  // work items are numbered densely over the CTA's threads (item t -> thread
  // t), so that the idle threads form whole idle warps: a warp with a few
  // active lanes costs the FP64 pipe as much as a full one.
  // S1: pencil along p at (q, r): X[r][q][i] = sum_p B[i][p] C[r][q][p]   (ne n^2 items)
  if (tid < ne * n * n) {
    const int e1 = tid / (n * n), qr = tid - e1 * n * n;
    const T* C = c.staged(0, e1) + qr * n;
    T v[n], x[Q];
#pragma unroll
    for (int p = 0; p < n; ++p) v[p] = C[p];
    eo_b<P, Q>(tab, v, x);
    T* dst = W0 + e1 * WS + qr * S;
#pragma unroll
    for (int i = 0; i < Q; ++i) dst[i] = x[i];
  }
  SPX_SYNC();
  // S2: pencil along q at (i, r): Y[j][i][r] = sum_q B[j][q] X[r][q][i]   (ne Q n items)
  if (tid < ne * Q * n) {
    const int e2 = tid / (Q * n), ir = tid - e2 * Q * n;
    const int i = ir % Q, r = ir / Q;
    const T* X = W0 + e2 * WS;
    T v[n], y[Q];
#pragma unroll
    for (int q = 0; q < n; ++q) v[q] = X[(r * n + q) * S + i];
    eo_b<P, Q>(tab, v, y);
    T* Y = W1 + e2 * WS;
#pragma unroll
    for (int j = 0; j < Q; ++j) Y[(j * Q + i) * SN + r] = y[j];
  }
  SPX_SYNC();
  // S3: column (i, j) = (a, b): u = B y (xi_3), d2 = dB y; U[k][j][i] = u (in W0)
  T* U = W0 + el * WS;
  T u[Q], g2[Q];
  if (act) {
    T y[n];
#pragma unroll
    for (int r = 0; r < n; ++r) y[r] = W1[el * WS + (b * Q + a) * SN + r];
    eo_b<P, Q>(tab, y, u);
#pragma unroll
    for (int k = 0; k < Q; ++k) U[k * PL + b * S + a] = u[k];
    eo_db<P, Q>(tab, y, g2);
  }
  SPX_SYNC();
  T* W2 = c.work[2] + el * WS;
  T* W3 = c.work[3] + el * WS;
  T z[Q];
  helm_mid<T, P, Q>(tab, c, el, a, b, act, U, W2, W3, u, g2, z, release);
  // S7: column (i, j) = (a, b): z += both contributions; y3 = B^T z (xi_3) -> Y3[r][i][j] (in W0)
  if (act) {
    T y3[n];
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      const int w = k * PL + b * S + a;
      z[k] += W2[w] + W3[w];
    }
    eo_bt<P, Q>(tab, z, y3);
#pragma unroll
    for (int r = 0; r < n; ++r) U[(r * Q + a) * S + b] = y3[r];
  }
  SPX_SYNC();
  // S8: pencil along j at (i, r): Y2[r][q][i] = sum_j B[j][q] Y3[r][i][j]   (ne Q n items)
  if (tid < ne * Q * n) {
    const int e2 = tid / (Q * n), ir = tid - e2 * Q * n;
    const int i = ir % Q, r = ir / Q;
    const T* Y3 = W0 + e2 * WS;
    T v[Q], y2[n];
#pragma unroll
    for (int j = 0; j < Q; ++j) v[j] = Y3[(r * Q + i) * S + j];
    eo_bt<P, Q>(tab, v, y2);
    T* Y2 = W1 + e2 * WS;
#pragma unroll
    for (int q = 0; q < n; ++q) Y2[(r * n + q) * S + i] = y2[q];
  }
  SPX_SYNC();
  // S9: pencil along i at (q, r): y[p][q][r] = sum_i B[i][p] Y2[r][q][i] -> HBM   (ne n^2 items)
  if (tid < ne * n * n) {
    const int e1 = tid / (n * n), qr = tid - e1 * n * n;
    const T* Y2 = W1 + e1 * WS + qr * S;
    T v[Q], y[n];
#pragma unroll
    for (int i = 0; i < Q; ++i) v[i] = Y2[i];
    eo_bt<P, Q>(tab, v, y);
    T* dst = out + c.gcoef[e1] + qr * n;
#pragma unroll
    for (int p = 0; p < n; ++p) dst[p] = y[p];
  }
}

// ---- Helmholtz, 3D, collocation (B = I) ----------------------------------
// The basis is the Lagrange basis through the Q = P + 1 GLL points that are
// also the quadrature points (the classical spectral element method, §2.1:
// nodal basis on GLL points), so BwdTrans and IProductWRTBase are the
// identity: the coefficients are the values at the quadrature points, the
// mass term is lambda JW u pointwise, and only the collocation derivatives
// and the geometric factors remain.  Q^2 threads per element, column (i, j) =
// (a, b) as in body_helm_role; five phases instead of nine.
template <typename T, int P, int Q, class Rel>
__device__ void body_helm_col(const T* tab, const Ctx<T>& c, T* out, Rel release) {
  static_assert(Q == P + 1, "collocation needs one GLL quadrature point per mode and direction");
  using S_ = RoleShape<T, P, Q>;
  constexpr int S = S_::S, PL = S_::PL, WS = S_::WS;
  constexpr int Q2 = Q * Q;
  const int el = c.tid / Q2;
  const int cc = c.tid - el * Q2;
  const int a = cc % Q, b = cc / Q;
  const bool act = el < c.ne;
  T* U = c.work[0] + el * WS;
  T* W2 = c.work[2] + el * WS;
  T* W3 = c.work[3] + el * WS;
  // C1: column (i, j) = (a, b): u = the column's coefficients; U[k][j][i] = u; d2 = D u
  T u[Q], g2[Q];
  if (act) {
    const T* C = c.staged(0, el) + b * Q + a;
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      u[k] = C[k * Q2];
      U[k * PL + b * S + a] = u[k];
    }
    eo_d<P, Q, false>(tab, u, g2);
  }
  SPX_SYNC();
  T z[Q];
  helm_mid<T, P, Q>(tab, c, el, a, b, act, U, W2, W3, u, g2, z, release);
  // C5: column (i, j) = (a, b): y = z + both transposed parts -> HBM
  if (act) {
    T* dst = out + c.gcoef[el] + b * Q + a;
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      const int w = k * PL + b * S + a;
      dst[k * Q2] = z[k] + (W2[w] + W3[w]);
    }
  }
}

// ---- BwdTrans and reference gradient of one staged coefficient stream -----
// U -> Wu, d_a -> Wd[a]; 3D uses scratch Wt.
template <typename T, int DIM, int P, int Q>
__device__ void bwd_grad(const T* tab, const Ctx<T>& c, BaseTable32 src, T* Wt, T* Wu, T* Wd0, T* Wd1, T* Wd2) {
  using S = Shape<T, DIM, P, Q>;
  constexpr int n = S::n, S1 = S::S1, S2 = S::S2, WS = S::WS;
  const T* B = tab;
  const T* D = tab + 2 * Q * n;
  const T* sm = reinterpret_cast<const T*>(c.sm);
  if (DIM == 3) {
    contract_g<0, n, n, n, Q, false, 0, false, n, n * n, S1, S2>(sm, src, sm, src, Wt, BaseStride{WS}, B, c.ne,
                                                                  c.tid, c.nthr);
    SPX_SYNC();
    contract_g<1, Q, n, n, Q, false, 0, false, S1, S2, S1, S2>(Wt, BaseStride{WS}, Wt, BaseStride{WS}, Wd0,
                                                                BaseStride{WS}, B, c.ne, c.tid, c.nthr);
    SPX_SYNC();
    bwd_and_deriv_pencil<2, Q, Q, n, Q, S1, S2, WS>(Wd0, Wu, Wd2, B, D, c.ne, c.tid, c.nthr);
    SPX_SYNC();
    contract_g<0, Q, Q, Q, Q, false, 0, false, S1, S2, S1, S2>(Wu, BaseStride{WS}, Wu, BaseStride{WS}, Wd0,
                                                                BaseStride{WS}, D, c.ne, c.tid, c.nthr);
    contract_g<1, Q, Q, Q, Q, false, 0, false, S1, S2, S1, S2>(Wu, BaseStride{WS}, Wu, BaseStride{WS}, Wd1,
                                                                BaseStride{WS}, D, c.ne, c.tid, c.nthr);
    SPX_SYNC();
  } else {
    contract_g<0, n, n, 1, Q, false, 0, false, n, 0, S1, 0>(sm, src, sm, src, Wt, BaseStride{WS}, B, c.ne, c.tid,
                                                             c.nthr);
    SPX_SYNC();
    bwd_and_deriv_pencil<1, Q, n, 1, Q, S1, 0, WS>(Wt, Wu, Wd1, B, D, c.ne, c.tid, c.nthr);
    SPX_SYNC();
    contract_g<0, Q, Q, 1, Q, false, 0, false, S1, 0, S1, 0>(Wu, BaseStride{WS}, Wu, BaseStride{WS}, Wd0,
                                                              BaseStride{WS}, D, c.ne, c.tid, c.nthr);
    SPX_SYNC();
  }
  (void)Wd2;
}

// ---- Adjoint with respect to lambda(x) and kappa(x) ----------------------
template <typename T, int DIM, int P, int Q, class Rel>
__device__ void body_adj(const T* tab, const Ctx<T>& c, T* glam, T* gkap, Rel release) {
  using S = Shape<T, DIM, P, Q>;
  constexpr int S1 = S::S1, S2 = S::S2, WS = S::WS, QD = S::QD;
  T** W = const_cast<T**>(c.work);
  // u: U -> W[1], grad -> W[2..4]; g: U -> W[5], grad -> W[6], W[7], W[0]
  bwd_grad<T, DIM, P, Q>(tab, c, BaseTable32{c.soff}, W[0], W[1], W[2], W[3], W[4]);
  bwd_grad<T, DIM, P, Q>(tab, c, BaseTable32{c.soff + kMaxEB}, W[0], W[5], W[6], W[7], W[0]);
  // in 2D the g gradient lives in W[6], W[7]; in 3D d2 of g was written to W[0]
  for (int pt = c.tid; pt < c.ne * QD; pt += c.nthr) {
    const int e = pt / QD;
    const int q = pt - e * QD;
    const int i = q % Q;
    const int j = (q / Q) % Q;
    const int k = DIM == 3 ? q / (Q * Q) : 0;
    const int w = e * WS + i + j * S1 + k * S2;
    const T* G = c.staged(2, e) + q;
    const int64_t o = c.gquad[e] + q;
    if (DIM == 3) {
      const T du0 = W[2][w], du1 = W[3][w], du2 = W[4][w];
      const T dg0 = W[6][w], dg1 = W[7][w], dg2 = W[0][w];
      const T g00 = G[0], g01 = G[QD], g02 = G[2 * QD], g11 = G[3 * QD], g12 = G[4 * QD], g22 = G[5 * QD];
      const T jw = G[6 * QD];
      if (glam) glam[o] = jw * W[5][w] * W[1][w];
      if (gkap)
        gkap[o] = dg0 * (g00 * du0 + g01 * du1 + g02 * du2) + dg1 * (g01 * du0 + g11 * du1 + g12 * du2) +
                  dg2 * (g02 * du0 + g12 * du1 + g22 * du2);
    } else {
      const T du0 = W[2][w], du1 = W[3][w];
      const T dg0 = W[6][w], dg1 = W[7][w];
      const T g00 = G[0], g01 = G[QD], g11 = G[2 * QD], jw = G[3 * QD];
      if (glam) glam[o] = jw * W[5][w] * W[1][w];
      if (gkap) gkap[o] = dg0 * (g00 * du0 + g01 * du1) + dg1 * (g01 * du0 + g11 * du1);
    }
  }
  (void)release;
}

// ---- Diagonal of the elemental Helmholtz matrices ------------------------
// diag_pqr = sum_ijk F_t[ijk] A0_t[i,p] A1_t[j,q] A2_t[k,r] over the terms
// t: lambda JW with (B^2, B^2, B^2) and G_ab with (dB^2 or B dB in the
// differentiated directions, B^2 elsewhere), off-diagonal G_ab counted twice.
template <typename T, int DIM, int P, int Q, class Rel>
__device__ void body_diag(const T* tab, const Ctx<T>& c, T* out, Rel release) {
  using S = Shape<T, DIM, P, Q>;
  constexpr int n = S::n, S1 = S::S1, S2 = S::S2, WS = S::WS, QD = S::QD;
  // squared tables in work buffer 4: BB, dd, Bd each [Q][n]
  T* tabs = c.work[4];
  for (int t = c.tid; t < Q * n; t += c.nthr) {
    const T b = tab[t], d = tab[Q * n + t];
    tabs[t] = b * b;
    tabs[Q * n + t] = d * d;
    tabs[2 * Q * n + t] = b * d;
  }
  const T* BB = tabs;
  const T* dd = tabs + Q * n;
  const T* Bd = tabs + 2 * Q * n;
  T *W0 = c.work[0], *W1 = c.work[1], *W2 = c.work[2], *W3 = c.work[3];
  constexpr int NT = DIM == 3 ? 7 : 4;
  for (int term = 0; term < NT; ++term) {
    SPX_SYNC();
    // field of this term into W3 (padded layout)
    for (int pt = c.tid; pt < c.ne * QD; pt += c.nthr) {
      const int e = pt / QD;
      const int q = pt - e * QD;
      const int i = q % Q;
      const int j = (q / Q) % Q;
      const int k = DIM == 3 ? q / (Q * Q) : 0;
      const T* G = c.staged(0, e) + q;
      T v;
      if (DIM == 3) {
        const int fi[7] = {6, 0, 3, 5, 1, 2, 4};
        v = G[fi[term] * QD];
        if (term == 0) v *= c.has_lam ? c.staged(1, e)[q] : c.lam;
        if (term >= 4) v *= T(2);
      } else {
        const int fi[4] = {3, 0, 2, 1};
        v = G[fi[term] * QD];
        if (term == 0) v *= c.has_lam ? c.staged(1, e)[q] : c.lam;
        if (term == 3) v *= T(2);
      }
      W3[e * WS + i + j * S1 + k * S2] = v;
    }
    SPX_SYNC();
    // matrices per axis for this term
    const T* A0;
    const T* A1;
    const T* A2;
    if (DIM == 3) {
      switch (term) {
        case 0: A0 = BB; A1 = BB; A2 = BB; break;
        case 1: A0 = dd; A1 = BB; A2 = BB; break;   // G00
        case 2: A0 = BB; A1 = dd; A2 = BB; break;   // G11
        case 3: A0 = BB; A1 = BB; A2 = dd; break;   // G22
        case 4: A0 = Bd; A1 = Bd; A2 = BB; break;   // G01
        case 5: A0 = Bd; A1 = BB; A2 = Bd; break;   // G02
        default: A0 = BB; A1 = Bd; A2 = Bd; break;  // G12
      }
      contract_g<2, Q, Q, Q, n, true, 0, false, S1, S2, S1, S2>(W3, BaseStride{WS}, W3, BaseStride{WS}, W0,
                                                                 BaseStride{WS}, A2, c.ne, c.tid, c.nthr);
      SPX_SYNC();
      contract_g<1, Q, Q, n, n, true, 0, false, S1, S2, S1, S2>(W0, BaseStride{WS}, W0, BaseStride{WS}, W1,
                                                                 BaseStride{WS}, A1, c.ne, c.tid, c.nthr);
      SPX_SYNC();
      if (term == 0)
        contract_g<0, Q, n, n, n, true, 0, false, S1, S2, S1, S2>(W1, BaseStride{WS}, W1, BaseStride{WS}, W2,
                                                                   BaseStride{WS}, A0, c.ne, c.tid, c.nthr);
      else
        contract_g<0, Q, n, n, n, true, 1, false, S1, S2, S1, S2>(W1, BaseStride{WS}, W1, BaseStride{WS}, W2,
                                                                   BaseStride{WS}, A0, c.ne, c.tid, c.nthr);
    } else {
      switch (term) {
        case 0: A0 = BB; A1 = BB; break;
        case 1: A0 = dd; A1 = BB; break;
        case 2: A0 = BB; A1 = dd; break;
        default: A0 = Bd; A1 = Bd; break;
      }
      A2 = nullptr;
      contract_g<1, Q, Q, 1, n, true, 0, false, S1, 0, S1, 0>(W3, BaseStride{WS}, W3, BaseStride{WS}, W1,
                                                               BaseStride{WS}, A1, c.ne, c.tid, c.nthr);
      SPX_SYNC();
      if (term == 0)
        contract_g<0, Q, n, 1, n, true, 0, false, S1, 0, S1, 0>(W1, BaseStride{WS}, W1, BaseStride{WS}, W2,
                                                                 BaseStride{WS}, A0, c.ne, c.tid, c.nthr);
      else
        contract_g<0, Q, n, 1, n, true, 1, false, S1, 0, S1, 0>(W1, BaseStride{WS}, W1, BaseStride{WS}, W2,
                                                                 BaseStride{WS}, A0, c.ne, c.tid, c.nthr);
    }
    (void)A2;
  }
  SPX_SYNC();
  release();
  constexpr int ND = S::ND;
  for (int pt = c.tid; pt < c.ne * ND; pt += c.nthr) {
    const int e = pt / ND;
    const int l = pt - e * ND;
    const int p = l % n;
    const int q = (l / n) % n;
    const int r = DIM == 3 ? l / (n * n) : 0;
    out[c.gcoef[e] + l] = W2[e * WS + p + q * S1 + r * S2];
  }
}

// ===========================================================================
// The kernel.
// ===========================================================================
// ---- FwdTrans ---------------------------------------------------------------
// Galerkin projection of quadrature-point values f onto the expansion (the
// FwdTrans of §3.5, Listing lst:python): u_e = M_e^{-1} b_e with
// b_e = IProduct(f)_e and M_e = Phi^T diag(JW) Phi the elemental mass matrix.
// Solved per element by preconditioned CG, all elements of the tile in
// lockstep with their own step lengths, matrix-free (M_e p = IProduct(JW
// BwdTrans(p)) by sum-factorisation through shared memory).  Preconditioner:
// K_e^{-1} = (1 / Jbar_e) (M1^{-1} (x) M1^{-1} (x) M1^{-1}), with M1 = B^T
// diag(w) B the 1D mass matrix (host-inverted table `mi`) and Jbar_e =
// sum_q JW_q / 2^d the element's mean Jacobian, since M_e = Jbar_e M1^{(x)d}
// whenever det J is constant on the element: then one step solves it, and a
// varying det J only adds steps.  An element stops at ||r|| <= tol ||b||
// (1e-14 FP64, 1e-6 FP32); a tile whose elements have not all converged
// after 64 steps stops there and sets bit 2 of the plan's status word.
// Per-element dot products: one warp per element, lanes in a fixed order
// (reproducible).
template <typename T>
__device__ __forceinline__ T warp_sum_t(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return __shfl_sync(0xffffffffu, v, 0);
}

// <a, b> over element e's ND modes (buffers [ne][WS], compact modal layout)
template <typename T, int ND, int WS>
__device__ __forceinline__ T elem_dot(const T* a, const T* b, int e, int lane) {
  T s = T(0);
  for (int m = lane; m < ND; m += 32) s = fma(a[e * WS + m], b[e * WS + m], s);
  return warp_sum_t(s);
}

// SENSOR = false: FwdTrans (above).  SENSOR = true: the adaptive-order sensor
// of §4.2, S_e = ||u_P - u_{P-1}||^2 / ||u_P||^2 (L2 norms by the element's
// quadrature, w det J): the input is the coefficients u_P, u_{P-1} is the L2
// projection onto degree <= P-1, i.e. onto the order-P modes that avoid the
// top bubble index P-1 in every direction (which span that space), computed
// by the same PCG restricted to those modes (the table `mi` is then the
// inverse of the restricted 1D mass matrix, zero on row and column P-1); then
// S_e = d^T M_e d / u^T M_e u with d = u_P - u_{P-1} (0 where u_P = 0),
// written to out[e] (the metadata slot gquad holds element ids for this op).
template <typename T, int DIM, int P, int Q, bool SENSOR = false>
__device__ void body_fwd(const T* tab, const Ctx<T>& c, const T* __restrict__ mi_g, T* out) {
  using S = Shape<T, DIM, P, Q>;
  constexpr int n = S::n, S1 = S::S1, S2 = S::S2, WS = S::WS, ND = S::ND, QD = S::QD;
  constexpr T kTol2 = sizeof(T) == 8 ? T(1e-28) : T(1e-12);
  constexpr int kMaxIt = 64;
  const T* B = tab;
  T *W0 = c.work[0], *W1 = c.work[1], *X = c.work[2], *R = c.work[3], *Pd = c.work[4], *AP = c.work[5],
    *Z = c.work[6];
  T* jb = c.extra;          // 1 / Jbar_e
  T* rz = jb + kMaxEB;      // <r, K^{-1} r>
  T* bb = rz + kMaxEB;      // <b, b>  (sensor: later u^T M u)
  T* al = bb + kMaxEB;      // step length (0 once converged)
  T* be = al + kMaxEB;      // direction update (< 0: converged)
  T* uMu = be + kMaxEB;     // (sensor) u^T M u
  T* mi = uMu + kMaxEB;     // [n][n]
  const int ne = c.ne, tid = c.tid, nthr = c.nthr;
  const int lane = tid & 31, warp = tid >> 5, nwarp = (nthr + 31) >> 5;
  BaseTable32 in0{c.soff}, jw{c.soff + kMaxEB};
  const T* sm = reinterpret_cast<const T*>(c.sm);
  const T* nul = nullptr;
  // mode m kept in the restricted space (sensor): no index equal to P - 1
  auto kept = [](int m) {
    const int a = m % n, b = (m / n) % n, q = DIM == 3 ? m / (n * n) : 0;
    return !(a == P - 1 || b == P - 1 || (DIM == 3 && q == P - 1));
  };
  for (int t = tid; t < n * n; t += nthr) mi[t] = mi_g[t];
  // AP = M_e v for a modal vector v (element base vb(e)): BwdTrans to the
  // quadrature points (compact layout in W0), then IProduct of JW * u
  auto mass_apply = [&](const T* v, auto vb) {
    if constexpr (DIM == 3) {
      contract_g<0, n, n, n, Q, false, 0, false, n, n * n, S1, S2>(v, vb, nul, BaseStride{0}, W0, BaseStride{WS}, B,
                                                                    ne, tid, nthr);
      SPX_SYNC();
      contract_g<1, Q, n, n, Q, false, 0, false, S1, S2, S1, S2>(W0, BaseStride{WS}, nul, BaseStride{0}, W1,
                                                                  BaseStride{WS}, B, ne, tid, nthr);
      SPX_SYNC();
      contract_g<2, Q, Q, n, Q, false, 0, false, S1, S2, Q, Q * Q>(W1, BaseStride{WS}, nul, BaseStride{0}, W0,
                                                                    BaseStride{WS}, B, ne, tid, nthr);
      SPX_SYNC();
      contract_g<2, Q, Q, Q, n, true, 0, true, Q, Q * Q, S1, S2>(W0, BaseStride{WS}, sm, jw, W1, BaseStride{WS}, B,
                                                                  ne, tid, nthr);
      SPX_SYNC();
      contract_g<1, Q, Q, n, n, true, 0, false, S1, S2, S1, S2>(W1, BaseStride{WS}, nul, BaseStride{0}, W0,
                                                                 BaseStride{WS}, B, ne, tid, nthr);
      SPX_SYNC();
      contract_g<0, Q, n, n, n, true, 0, false, S1, S2, n, n * n>(W0, BaseStride{WS}, nul, BaseStride{0}, AP,
                                                                   BaseStride{WS}, B, ne, tid, nthr);
    } else {
      contract_g<0, n, n, 1, Q, false, 0, false, n, 0, S1, 0>(v, vb, nul, BaseStride{0}, W0, BaseStride{WS}, B, ne,
                                                              tid, nthr);
      SPX_SYNC();
      contract_g<1, Q, n, 1, Q, false, 0, false, S1, 0, Q, 0>(W0, BaseStride{WS}, nul, BaseStride{0}, W1,
                                                              BaseStride{WS}, B, ne, tid, nthr);
      SPX_SYNC();
      contract_g<1, Q, Q, 1, n, true, 0, true, Q, 0, S1, 0>(W1, BaseStride{WS}, sm, jw, W0, BaseStride{WS}, B, ne,
                                                            tid, nthr);
      SPX_SYNC();
      contract_g<0, Q, n, 1, n, true, 0, false, S1, 0, n, 0>(W0, BaseStride{WS}, nul, BaseStride{0}, AP,
                                                             BaseStride{WS}, B, ne, tid, nthr);
    }
    SPX_SYNC();
  };
  // Z = (M1^{-1})^{(x)d} R (unscaled; the 1 / Jbar_e factor is applied by the callers)
  auto precond = [&]() {
    if constexpr (DIM == 3) {
      contract_g<0, n, n, n, n, false, 0, false, n, n * n, n, n * n>(R, BaseStride{WS}, nul, BaseStride{0}, W0,
                                                                     BaseStride{WS}, mi, ne, tid, nthr);
      SPX_SYNC();
      contract_g<1, n, n, n, n, false, 0, false, n, n * n, n, n * n>(W0, BaseStride{WS}, nul, BaseStride{0}, W1,
                                                                     BaseStride{WS}, mi, ne, tid, nthr);
      SPX_SYNC();
      contract_g<2, n, n, n, n, false, 0, false, n, n * n, n, n * n>(W1, BaseStride{WS}, nul, BaseStride{0}, Z,
                                                                     BaseStride{WS}, mi, ne, tid, nthr);
    } else {
      contract_g<0, n, n, 1, n, false, 0, false, n, 0, n, 0>(R, BaseStride{WS}, nul, BaseStride{0}, W0,
                                                             BaseStride{WS}, mi, ne, tid, nthr);
      SPX_SYNC();
      contract_g<1, n, n, 1, n, false, 0, false, n, 0, n, 0>(W0, BaseStride{WS}, nul, BaseStride{0}, Z,
                                                             BaseStride{WS}, mi, ne, tid, nthr);
    }
    SPX_SYNC();
  };
  if constexpr (SENSOR) {
    // b = restriction of M_e u_P; u^T M u for the denominator
    mass_apply(sm, in0);
    for (int e = warp; e < ne; e += nwarp) {
      const T* u = c.staged(0, e);
      T s = T(0);
      for (int m = lane; m < ND; m += 32) s = fma(u[m], AP[e * WS + m], s);
      s = warp_sum_t(s);
      if (lane == 0) uMu[e] = s;
    }
    for (int t = tid; t < ne * ND; t += nthr) {
      const int e = t / ND, m = t - e * ND;
      R[e * WS + m] = kept(m) ? AP[e * WS + m] : T(0);
    }
  } else {
    // b = IProduct(f) -> R
    if constexpr (DIM == 3) {
      contract_g<2, Q, Q, Q, n, true, 0, true, Q, Q * Q, S1, S2>(sm, in0, sm, jw, W0, BaseStride{WS}, B, ne, tid,
                                                                  nthr);
      SPX_SYNC();
      contract_g<1, Q, Q, n, n, true, 0, false, S1, S2, S1, S2>(W0, BaseStride{WS}, nul, BaseStride{0}, W1,
                                                                 BaseStride{WS}, B, ne, tid, nthr);
      SPX_SYNC();
      contract_g<0, Q, n, n, n, true, 0, false, S1, S2, n, n * n>(W1, BaseStride{WS}, nul, BaseStride{0}, R,
                                                                   BaseStride{WS}, B, ne, tid, nthr);
    } else {
      contract_g<1, Q, Q, 1, n, true, 0, true, Q, 0, S1, 0>(sm, in0, sm, jw, W0, BaseStride{WS}, B, ne, tid, nthr);
      SPX_SYNC();
      contract_g<0, Q, n, 1, n, true, 0, false, S1, 0, n, 0>(W0, BaseStride{WS}, nul, BaseStride{0}, R,
                                                             BaseStride{WS}, B, ne, tid, nthr);
    }
  }
  for (int e = warp; e < ne; e += nwarp) {  // 1 / Jbar_e = 2^d / sum_q JW_q
    const T* J = c.staged(1, e);
    T s = T(0);
    for (int q = lane; q < QD; q += 32) s += J[q];
    s = warp_sum_t(s);
    if (lane == 0) jb[e] = T(1 << DIM) / s;
  }
  SPX_SYNC();
  precond();
  // X = 0, Z = K^{-1} R, Pd = Z; rz = <R, Z>, bb = <R, R>
  for (int t = tid; t < ne * ND; t += nthr) {
    const int e = t / ND, m = t - e * ND;
    const T z = jb[e] * Z[e * WS + m];
    X[e * WS + m] = T(0);
    Z[e * WS + m] = z;
    Pd[e * WS + m] = z;
  }
  SPX_SYNC();
  for (int e = warp; e < ne; e += nwarp) {
    const T a = elem_dot<T, ND, WS>(R, Z, e, lane), b2 = elem_dot<T, ND, WS>(R, R, e, lane);
    if (lane == 0) {
      rz[e] = a;
      bb[e] = b2;
      be[e] = b2 > T(0) ? T(0) : T(-1);   // a zero right-hand side is converged at x = 0
    }
  }
  SPX_SYNC();
  for (int it = 0; it < kMaxIt; ++it) {
    mass_apply(Pd, BaseStride{WS});
    if constexpr (SENSOR) {   // restrict to the kept modes
      for (int t = tid; t < ne * ND; t += nthr) {
        const int e = t / ND, m = t - e * ND;
        if (!kept(m)) AP[e * WS + m] = T(0);
      }
      SPX_SYNC();
    }
    for (int e = warp; e < ne; e += nwarp) {
      const T pap = elem_dot<T, ND, WS>(Pd, AP, e, lane);
      if (lane == 0) al[e] = be[e] < T(0) ? T(0) : rz[e] / pap;
    }
    SPX_SYNC();
    for (int t = tid; t < ne * ND; t += nthr) {
      const int e = t / ND, m = t - e * ND;
      X[e * WS + m] = fma(al[e], Pd[e * WS + m], X[e * WS + m]);
      R[e * WS + m] = fma(-al[e], AP[e * WS + m], R[e * WS + m]);
    }
    SPX_SYNC();
    precond();
    bool active = false;
    for (int e = warp; e < ne; e += nwarp) {
      const T rr = elem_dot<T, ND, WS>(R, R, e, lane);
      const T rzn = jb[e] * elem_dot<T, ND, WS>(R, Z, e, lane);
      if (lane == 0) {
        if (be[e] >= T(0) && rr <= kTol2 * bb[e]) be[e] = T(-1);
        if (be[e] >= T(0)) {
          be[e] = rzn / rz[e];
          rz[e] = rzn;
          active = true;
        }
      }
    }
    if (!__syncthreads_or(active)) break;
    if (it == kMaxIt - 1) {   // step cap reached with elements still above the tolerance
      if (tid == 0) atomicOr(c.status, kStatusNotConverged);
      break;
    }
    for (int t = tid; t < ne * ND; t += nthr) {
      const int e = t / ND, m = t - e * ND;
      if (be[e] >= T(0)) Pd[e * WS + m] = fma(be[e], Pd[e * WS + m], jb[e] * Z[e * WS + m]);
    }
    SPX_SYNC();
  }
  if constexpr (SENSOR) {
    // d = u_P - u_{P-1}; S_e = d^T M d / u^T M u
    for (int t = tid; t < ne * ND; t += nthr) {
      const int e = t / ND, m = t - e * ND;
      Pd[e * WS + m] = c.staged(0, e)[m] - X[e * WS + m];
    }
    SPX_SYNC();
    mass_apply(Pd, BaseStride{WS});
    for (int e = warp; e < ne; e += nwarp) {
      const T dmd = elem_dot<T, ND, WS>(Pd, AP, e, lane);
      if (lane == 0) out[c.gquad[e]] = uMu[e] > T(0) ? dmd / uMu[e] : T(0);
    }
  } else {
    for (int t = tid; t < ne * ND; t += nthr) {
      const int e = t / ND, m = t - e * ND;
      out[c.gcoef[e] + m] = X[e * WS + m];
    }
  }
}

// BK: the basis kind of the plan (3D Helmholtz only): 0 the modified basis's
// parity (even-odd role body), 1 any basis (generic body), 2 collocation,
// B = I (collocation body).
template <typename T, int DIM, int OP, int P, int Q, int BK, class Prm, class Rel>
__device__ __forceinline__ void run_body(const Prm& p, const Ctx<T>& c, Rel rel) {
  const T* tab = p.tab + Prm::Layout::off(P);
  if constexpr (OP == OP_BWD) body_bwd<T, DIM, P, Q>(tab, c, p.out0, rel);
  else if constexpr (OP == OP_IPROD) body_iprod<T, DIM, P, Q>(tab, c, p.out0, rel);
  else if constexpr (OP == OP_DERIV) body_deriv<T, DIM, P, Q>(tab, c, p.out0, p.out1, p.out2, rel);
  else if constexpr (OP == OP_HELM && DIM == 3 && BK == 0) body_helm_role<T, P, Q>(tab, c, p.out0, rel);
  else if constexpr (OP == OP_HELM && DIM == 3 && BK == 2) body_helm_col<T, P, Q>(tab, c, p.out0, rel);
  else if constexpr (OP == OP_HELM) body_helm<T, DIM, P, Q>(tab, c, p.out0, rel);
  else if constexpr (OP == OP_ADJ) body_adj<T, DIM, P, Q>(tab, c, p.out0, p.out1, rel);
  else if constexpr (OP == OP_FWD) body_fwd<T, DIM, P, Q>(tab, c, p.in1 + mass1d_off(P), p.out0);
  else if constexpr (OP == OP_SENSOR)
    body_fwd<T, DIM, P, Q, true>(tab, c, p.in1 + mass1d_off(kMaxP + 1) + mass1d_off(P), p.out0);
  else body_diag<T, DIM, P, Q>(tab, c, p.out0, rel);
}

// The tiles of this CTA's run (order P, compile time): tiles t0, t0 + G, ...
// below t1, through the staging ring.  The loop sits inside the order's
// branch (op_dispatch): a loop around a dispatch over every order made the
// compiler keep values of all the bodies live across it (spills that no
// single body has).
// P == 0 (FP64 variable order): the run is the whole tile list, every order
// in it, and each tile's body is chosen at run time.  The FP64 bodies are
// bound by the FP64 pipe: there the balance of every CTA walking every order
// (heaviest first) measured 3-7% faster than one order per CTA, spills and all.
template <typename T, int DIM, int OP, int PLO, int PHI, int QOFF, int BK, class Prm, class Rel>
__device__ __forceinline__ void body_of_order(int P, const Prm& p, const Ctx<T>& c, Rel rel) {
  if constexpr (PLO <= PHI) {
    if (P == PLO) run_body<T, DIM, OP, PLO, PLO + QOFF, BK>(p, c, rel);
    else body_of_order<T, DIM, OP, PLO + 1, PHI, QOFF, BK>(P, p, c, rel);
  }
}

template <typename T, int DIM, int OP, int P, int QOFF, int BK, class Prm, int PLO = P, int PHI = P>
__device__ __forceinline__ void op_run(const Prm& p, char* sm, uint64_t* bars, uint32_t* soff, int64_t* gcoef,
                                       int64_t* gquad, Ctx<T>& c, int t0, int t1, int G) {
  const int tid = c.tid, nthr = c.nthr;
  const int S = p.stages;
  for (int k = 0;; ++k) {
    const int ti = t0 + k * G;
    if (ti >= t1) break;
    const int slot = k % S;
    const bool ok = mbar_wait(&bars[slot], (k / S) & 1);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) atomicOr(p.status, kStatusTimeout);
      return;
    }
    const Tile t = p.tiles[ti];
    const int TP = P ? P : t.P, Q = TP + QOFF;   // this tile's order
    c.ne = t.count;
    // per-tile metadata: element offsets and staged-data offsets
    StreamDesc<T> sd[5];
    const int ns = op_streams<T, DIM, OP>(p, TP, Q, sd);
    char* slotp = sm + p.slot_base + slot * p.slot_bytes;
    for (int j = tid; j < t.count; j += nthr) {
      const int64_t e = elem_id(p, t, j);
      gcoef[j] = coef_off_of<DIM>(p, e, TP);
      gquad[j] = quad_off_of<DIM>(p, e, Q);
#pragma unroll
      for (int s = 0; s < 5; ++s) {
        if (s >= ns || !sd[s].base) continue;
        char* region = slotp + p.region_off[s];
        const int64_t off = sd[s].quad ? gquad[j] : gcoef[j];
        const T* g = sd[s].base + sd[s].mult * off + sd[s].boff;
        char* at;
        if (t.contig && sd[s].whole) {
          const int64_t e0 = elem_id(p, t, 0);
          const int64_t off0 = sd[s].quad ? quad_off_of<DIM>(p, e0, Q) : coef_off_of<DIM>(p, e0, TP);
          const T* g0 = sd[s].base + sd[s].mult * off0 + sd[s].boff;
          at = region + (reinterpret_cast<uintptr_t>(g0) & 15) + (g - g0) * sizeof(T);
          // head / tail words of the whole-tile range
          if (j == 0)
            stage_fixup<sizeof(T)>(region, g0, static_cast<uint32_t>(t.count * sd[s].len * sizeof(T)), 0, 1);
        } else {
          char* r = region + j * erb_bytes(sd[s].len, sizeof(T));
          at = r + (reinterpret_cast<uintptr_t>(g) & 15);
          stage_fixup<sizeof(T)>(r, g, static_cast<uint32_t>(sd[s].len * sizeof(T)), 0, 1);
        }
        soff[s * kMaxEB + j] = static_cast<uint32_t>((at - sm) / sizeof(T));
      }
      if constexpr (OP == OP_SENSOR) gquad[j] = e;   // its output is one value per element
    }
    __syncthreads();
    if (OP == OP_HELM && DIM == 3 && p.geo_direct && tid == 0) {   // this tile's geometry into L2 while S1..S4 run
      if (t.contig) prefetch_l2(p.geom + 7 * gquad[0], uint64_t(t.count) * 7 * Q * Q * Q * sizeof(T));
      else
        for (int j = 0; j < t.count; ++j) prefetch_l2(p.geom + 7 * gquad[j], uint64_t(7) * Q * Q * Q * sizeof(T));
    }
    bool released = false;
    auto rel = [&]() {
      if (!released) {
        released = true;
        if (tid == 0 && ti + S * G < t1) {
          fence_proxy_async();
          issue_tile<T, DIM, OP, QOFF>(p, sm, bars, slot, ti + S * G);
        }
      }
    };
    if constexpr (P != 0) run_body<T, DIM, OP, P, P + QOFF, BK>(p, c, rel);
    else body_of_order<T, DIM, OP, PLO, PHI, QOFF, BK>(TP, p, c, rel);
    __syncthreads();
    rel();
  }
}

template <typename T, int DIM, int OP, int PLO, int PHI, int QOFF, int BK, class Prm>
__device__ __forceinline__ void op_dispatch(int P, const Prm& p, char* sm, uint64_t* bars, uint32_t* soff,
                                            int64_t* gcoef, int64_t* gquad, Ctx<T>& c, int t0, int t1, int G) {
  if constexpr (PLO <= PHI) {
    if (P == PLO) op_run<T, DIM, OP, PLO, QOFF, BK>(p, sm, bars, soff, gcoef, gquad, c, t0, t1, G);
    else op_dispatch<T, DIM, OP, PLO + 1, PHI, QOFF, BK>(P, p, sm, bars, soff, gcoef, gquad, c, t0, t1, G);
  }
}

// REG: register budget per thread (128 lets a 512-thread block run; the 3D
// Helmholtz bodies with Q^2 threads per element also come with 72, for more
// CTAs per SM).  Each CTA walks one run of the tile list (one order).
template <typename T, int DIM, int OP, int PLO, int PHI, int QOFF, int BK = 0, int REG = 128>
__global__ void __maxnreg__(REG) op_kernel(const __grid_constant__ KParams<T, PLO, PHI, QOFF> p) {
  extern __shared__ __align__(128) char sm[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm);
  uint32_t* soff = reinterpret_cast<uint32_t*>(sm + p.meta_base);
  int64_t* gcoef = reinterpret_cast<int64_t*>(sm + p.meta_base + 5 * kMaxEB * 4);
  int64_t* gquad = gcoef + kMaxEB;
  int* tab_order = reinterpret_cast<int*>(gquad + kMaxEB);
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int S = p.stages;
  if (p.skip && *p.skip) return;   // uniform across the grid: nothing started yet
  const TileRun run = tile_run(p);
  if (tid == 0) {
    for (int s = 0; s < S; ++s) mbar_init(&bars[s], 1);
    fence_barrier_init();
    *tab_order = -1;
  }
  __syncthreads();
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      const int ti = run.t0 + s * run.G;
      if (ti < run.t1) issue_tile<T, DIM, OP, QOFF>(p, sm, bars, s, ti);
    }
  }
  Ctx<T> c;
  c.sm = sm;
  for (int w = 0; w < 8; ++w) c.work[w] = reinterpret_cast<T*>(sm + p.work_base + size_t(w) * p.work_bytes);
  c.soff = soff;
  c.tab_order = tab_order;
  c.extra = reinterpret_cast<T*>(sm + p.meta_base + 5 * kMaxEB * 4 + 2 * kMaxEB * 8 + 16);
  c.status = p.status;
  c.gcoef = gcoef;
  c.gquad = gquad;
  c.tid = tid;
  c.nthr = nthr;
  c.has_lam = p.lam_f != nullptr;
  c.has_kap = p.kap_f != nullptr;
  c.lam = static_cast<T>(p.lam);
  c.geom_g = (OP == OP_HELM && p.geo_direct) ? p.geom : nullptr;
  if constexpr (sizeof(T) == 8 && PLO < PHI)   // FP64 variable order: one run, every order (see body_of_order)
    op_run<T, DIM, OP, 0, QOFF, BK, KParams<T, PLO, PHI, QOFF>, PLO, PHI>(p, sm, bars, soff, gcoef, gquad, c, run.t0,
                                                                         run.t1, run.G);
  else
    op_dispatch<T, DIM, OP, PLO, PHI, QOFF, BK>(run.P, p, sm, bars, soff, gcoef, gquad, c, run.t0, run.t1, run.G);
}

}  // namespace spx
