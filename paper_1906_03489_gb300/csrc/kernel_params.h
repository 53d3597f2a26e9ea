// Parameter block of the operator kernel, shared by host and device code.
#pragma once
#include <cstdint>

namespace spx {

constexpr int kMaxEB = 64;  // elements per tile (upper bound)
constexpr int kMaxP = 8;    // highest supported order
constexpr int kMaxP1 = 9;   // orders 0..8 index per-order tables

enum OpKind {
  OP_BWD = 0, OP_IPROD = 1, OP_DERIV = 2, OP_HELM = 3, OP_ADJ = 4, OP_DIAG = 5, OP_FWD = 6, OP_SENSOR = 7, OP_KINDS = 8
};

// Offset of order P's [n][n] inverse 1D mass matrix in the per-order table
// array (orders 1, 2, ... stored one after the other; the sensor's restricted
// inverses follow at mass1d_off(kMaxP + 1)).
__host__ __device__ constexpr int mass1d_off(int P) {
  int o = 0;
  for (int p = 1; p < P; ++p) o += (p + 1) * (p + 1);
  return o;
}
// Values of the FwdTrans / sensor body's scratch region after the tile
// metadata: six per-element scalars and one order's [n][n] table.
constexpr int kFwdExtra = 6 * kMaxEB + 81;

// A tile: `count` elements of order P.  contig != 0: the elements are
// id(first), id(first)+1, ...; else ids[first + j].  Without an id array
// id(x) = x.
struct Tile {
  int32_t P;
  int32_t count;
  int32_t first;
  int32_t contig;
};

// Per-order table: B[Q][n], dB[Q][n], D[Q][Q], then the even-odd
// coefficients (EOLayout): Bs[Hc], Bd[Hc], Dp[H][H], Dm[H][H], Tp[H][H],
// Tm[H][H], Gs[Hc], Gd[Hc] with H = Q / 2, Hc = (Q + 1) / 2.
__host__ __device__ constexpr int eo_len(int Q) { return 4 * ((Q + 1) / 2) + 4 * (Q / 2) * (Q / 2); }
__host__ __device__ constexpr int tab_len(int P, int QOFF) {
  return 2 * (P + QOFF) * (P + 1) + (P + QOFF) * (P + QOFF) + eo_len(P + QOFF);
}

// Even-odd form of the 1D operators (symmetric GLL points xi_{Q-1-i} = -xi_i):
// the modified basis has phi_0(-x) = phi_P(x) and phi_b(-x) = (-1)^(b-1)
// phi_b(x) for the bubbles, and the collocation derivative D is
// centro-antisymmetric, D[Q-1-i][Q-1-j] = -D[i][j].  With e = v_0 + v_P,
// o = v_0 - v_P, s_j = v_j + v_{Q-1-j}, d_j = v_j - v_{Q-1-j}:
//   (B v)_i, (B v)_{Q-1-i} = S_i +- D_i,  S_i = Bs_i e + sum_{b odd} B_ib v_b,
//                                           D_i = Bd_i o + sum_{b even} B_ib v_b
//   (D v)_i, (D v)_{Q-1-i} = E_i +- F_i,  E_i = sum_j Dm_ij d_j,
//                                           F_i = sum_j Dp_ij s_j (+ D_iM v_M, Q odd)
// with Bs_i = (B_i0 + B_iP) / 2, Bd_i = (B_i0 - B_iP) / 2,
// Dp_ij = (D_ij + D_i,Q-1-j) / 2, Dm_ij = (D_ij - D_i,Q-1-j) / 2 and Tp, Tm the
// same for D^T; the transposed contractions follow by the same symmetry.
// The derivatives of the basis have the opposite parity, phi_0'(-x) =
// -phi_P'(x) and phi_b'(-x) = (-1)^b phi_b'(x), so
//   (dB v)_i, (dB v)_{Q-1-i} = S'_i +- A'_i,  S'_i = Gd_i o + sum_{b even} dB_ib v_b,
//                                               A'_i = Gs_i e + sum_{b odd} dB_ib v_b
// with Gs_i = (dB_i0 + dB_iP) / 2, Gd_i = (dB_i0 - dB_iP) / 2.
template <int P, int Q>
struct EOLayout {
  static constexpr int n = P + 1, H = Q / 2, Hc = (Q + 1) / 2;
  static constexpr int Bs = 2 * Q * n + Q * Q, Bd = Bs + Hc, Dp = Bd + Hc, Dm = Dp + H * H, Tp = Dm + H * H,
                       Tm = Tp + H * H, Gs = Tm + H * H, Gd = Gs + Hc;
};

// Shared-memory layout of the FP32 3D Helmholtz kernel (helm_pair.cuh), in
// units of its value type: float2 (two elements per thread, 8-byte accesses,
// bank modulus M = 16 per half-warp) or float (one element per thread, M = 32
// per warp).  Thread cc = a + Q b of an element group takes roles (a, b);
// every array is laid out so that the role coordinate a thread varies with
// `a` has stride 1 and the one it varies with `b` stride Q (mod M), and the
// group stride is Q^2 (mod M): the lanes of a wavefront then touch distinct
// banks in every phase (no bank conflicts).
//   X (q, r, i)  = q + Q r + XS i     Y, Y3 (i, r, j) = i + Q r + YS j
//   U, G0 (i, j, k) = i + Q j + US k  U', G1 (i, j, k) = i + Q j + GS k
//   Y2 (i, q, r) = i + Q r + ZS q
__host__ __device__ constexpr int upm(int x, int r, int M) { return x + (((r % M) - (x % M)) % M + M) % M; }

template <int P, int Q, int M>
struct PairLayout {
  static constexpr int n = P + 1;
  static constexpr int XS = upm((n - 1) + Q * (n - 1) + 1, 1, M);
  static constexpr int YS = upm(Q * n, Q, M);
  static constexpr int US = upm(Q * Q, 1, M);
  static constexpr int GS = upm(Q * Q, Q, M);
  static constexpr int ZS = upm(Q * n, 1, M);
  static constexpr int mx(int a, int b) { return a > b ? a : b; }
  // group strides of the three buffers: A holds X then U / g0, C holds Y then
  // Y3, F holds U' / g1 then Y2
  static constexpr int WA = upm(mx((n - 1) + Q * (n - 1) + XS * (Q - 1) + 1, Q * Q + US * (Q - 1)), Q * Q, M);
  static constexpr int WC = upm((Q - 1) + Q * (n - 1) + YS * (Q - 1) + 1, Q * Q, M);
  static constexpr int WF = upm(mx(Q * Q + GS * (Q - 1), (Q - 1) + Q * (n - 1) + ZS * (n - 1) + 1), Q * Q, M);
  // group strides of the streaming operators (pair_ops.cuh): X alone in A
  // (BwdTrans), Y2 alone in F (IProductWRTBase)
  static constexpr int WX = upm((n - 1) + Q * (n - 1) + XS * (Q - 1) + 1, Q * Q, M);
  static constexpr int WZ = upm((Q - 1) + Q * (n - 1) + ZS * (n - 1) + 1, Q * Q, M);
};

// Highest order packed two elements per thread in a variable-order launch by
// default (measured on 24^3, P = 2..8: pairs up to 5 0.070 ms, up to 6 or 8
// 0.081 ms; the launch's threads class selects the others).
constexpr int kPairThrVar = 5;

// Elements per thread of order P in a kernel that packs orders <= thr in pairs.
__host__ __device__ constexpr int pair_lanes(int P, int thr) { return P <= thr ? 2 : 1; }

// Group strides of order P in bytes at runtime (host side): {WA, WC, WF}.
inline void pair_ws_bytes(int P, int QOFF, int lanes, uint64_t w[3]) {
  w[0] = w[1] = w[2] = 0;
  switch ((P * 4 + QOFF) * 2 + (lanes == 2)) {
#define SPX_PWS_(p, q, l, m)                                                                                         \
  case (p * 4 + (q - p)) * 2 + (l == 2):                                                                              \
    w[0] = 4u * l * PairLayout<p, q, m>::WA; w[1] = 4u * l * PairLayout<p, q, m>::WC; w[2] = 4u * l * PairLayout<p, q, m>::WF; \
    break;
#define SPX_PWS(p) SPX_PWS_(p, p + 1, 1, 32) SPX_PWS_(p, p + 1, 2, 16) SPX_PWS_(p, p + 2, 1, 32) SPX_PWS_(p, p + 2, 2, 16)
    SPX_PWS(1) SPX_PWS(2) SPX_PWS(3) SPX_PWS(4) SPX_PWS(5) SPX_PWS(6) SPX_PWS(7) SPX_PWS(8)
#undef SPX_PWS
#undef SPX_PWS_
    default: break;
  }
}

// Group strides in bytes of the streaming pair kernels (pair_ops.cuh, two
// elements per thread): {WX, WC, WZ}.
inline void pair_sf_bytes(int P, int QOFF, uint64_t w[3]) {
  w[0] = w[1] = w[2] = 0;
  switch (P * 4 + QOFF) {
#define SPX_PSF_(p, q) \
  case p * 4 + (q - p): \
    w[0] = 8u * PairLayout<p, q, 16>::WX; w[1] = 8u * PairLayout<p, q, 16>::WC; w[2] = 8u * PairLayout<p, q, 16>::WZ; \
    break;
#define SPX_PSF(p) SPX_PSF_(p, p + 1) SPX_PSF_(p, p + 2)
    SPX_PSF(1) SPX_PSF(2) SPX_PSF(3) SPX_PSF(4) SPX_PSF(5) SPX_PSF(6) SPX_PSF(7) SPX_PSF(8)
#undef SPX_PSF
#undef SPX_PSF_
    default: break;
  }
}

// Bytes of one element's FP32 3D geometry block, and the stride of the
// per-element regions of the Helmholtz pair kernel's geometry slot: at least
// the block rounded to 16 bytes plus 16 bytes of alignment slack, and for
// even Q congruent to 4 Q^2 modulo 128 bytes, so that element j starts Q^2 j
// words (mod 32) into the banks: the column reads of element pairs
// (j, j + npair) then follow the thread index (no bank conflicts).
__host__ __device__ constexpr uint32_t geo_eblk(int Q) { return 7u * Q * Q * Q * 4u; }
__host__ __device__ constexpr uint32_t geo_erb(int Q) {
  return (Q % 2) ? ((geo_eblk(Q) + 15u) & ~15u) + 16u
                 : (((geo_eblk(Q) + 15u) & ~15u) + 16u) +
                       (((4u * Q * Q) % 128u + 128u - ((((geo_eblk(Q) + 15u) & ~15u) + 16u) % 128u)) % 128u);
}

template <int PLO, int PHI, int QOFF>
struct TabLayout {
  __host__ __device__ static constexpr int off(int P) {
    int o = 0;
    for (int p = PLO; p < P; ++p) o += tab_len(p, QOFF);
    return o;
  }
  static constexpr int total = off(PHI + 1);
};

template <typename T, int PLO, int PHI, int QOFF>
struct KParams {
  using Layout = TabLayout<PLO, PHI, QOFF>;
  const Tile* tiles;
  const int32_t* ids;
  const int64_t* coef_off;  // nullptr for uniform plans
  const int64_t* quad_off;
  const T* in0;
  const T* in1;
  const T* geom;
  const T* lam_f;
  const T* kap_f;
  T* out0;
  T* out1;
  T* out2;
  int* status;
  const int* skip;          // non-null and nonzero at launch time: the launch does nothing
  double lam;
  int n_tiles;
  int stages;
  int geo_direct;          // 3D Helmholtz bodies: geometry read from global memory (L2-prefetched), not staged
  uint32_t slot_base;      // byte offset of slot 0
  uint32_t slot_bytes;
  uint32_t region_off[5];  // per stream, inside a slot
  uint32_t work_base;
  uint32_t work_bytes;     // per work buffer
  uint32_t meta_base;
  // runs of the tile list, one order each (a uniform plan has one): CTAs
  // [grp_cta[g], grp_cta[g + 1]) walk run g (order grp_P[g], tiles
  // [grp_tile[g], grp_tile[g + 1])) and nothing else
  int ngrp;
  int grp_P[kMaxP];
  int grp_tile[kMaxP + 1];
  int grp_cta[kMaxP + 1];
  // layers > 1: grp_cta counts SM slots instead of CTAs; CTA b sits in slot
  // b mod nslot of layer b / nslot, and run g owns its slots in every layer
  // (the CTAs a persistent grid places on one SM then share an order)
  int layers, nslot;
  T tab[Layout::total];
};

// This CTA's run of tiles: tiles t0, t0 + G, ... below t1, all of order P.
struct TileRun {
  int P, t0, t1, G;
};
#ifdef __CUDACC__
template <class Prm>
__device__ __forceinline__ TileRun tile_run(const Prm& p) {
  const int b = blockIdx.x;
  const int slot = p.layers > 1 ? b % p.nslot : b, layer = p.layers > 1 ? b / p.nslot : 0;
  int g = 0;
  while (g + 1 < p.ngrp && slot >= p.grp_cta[g + 1]) ++g;
  const int width = p.grp_cta[g + 1] - p.grp_cta[g];
  return TileRun{p.grp_P[g], p.grp_tile[g] + layer * width + slot - p.grp_cta[g], p.grp_tile[g + 1],
                 width * (p.layers > 1 ? p.layers : 1)};
}
#endif

}  // namespace spx
