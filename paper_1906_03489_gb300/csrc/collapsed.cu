// Collapsed-coordinate elements: triangles (2D), prisms and tetrahedra (3D), §2.1
// (Fig. f:duffy: the Duffy map from the square / cube onto the reference
// shape, Table t:refregions) with the sum-factorisation of §3.3.
//
// In collapsed coordinates eta the modal basis is a product of 1D functions
// whose collapsed-direction factor psi^b_{pq} depends on the mode index p of
// the direction before it, so the contraction along the collapsed direction
// runs over a p-dependent range of q ("ragged" but still one direction at a
// time, O(P^{d+1}) work):
//   triangle  u(eta1_i, eta2_j) = sum_p psi^a_p(eta1_i) sum_q c_{pq} psi^b_{pq}(eta2_j)
//   prism     u(xi1_i, eta2_j, eta3_k) = sum_a psi^a_a(xi1_i) sum_p psi^a_p(eta2_j)
//                                         sum_q c_{a,pq} psi^b_{pq}(eta3_k)
//   tetrahedron  u(eta1_i, eta2_j, eta3_k) = sum_p psi^a_p(eta1_i) sum_q psi^b_{pq}(eta2_j)
//                sum_r c_{(pq),r} psi^c_{k(pq),r}(eta3_k)  (+ the apex (1 + eta3)/2):
//                the eta3 factor of triangle mode m of degree k_m is
//                ((1-z)/2)^k_m times 1 or (1+z)/2 P^{(2k_m-1,1)}_{r-1}(z), r <= P - k_m,
//                and both eta2 and eta3 use Gauss-Radau points
// Mode (p, q) = (0, P) is the collapsed vertex: its function (1 + z)/2 equals
// psi^a_0 psi^a_P + psi^a_P psi^a_P, so its coefficient also enters the
// p = P row of the collapsed-direction contraction (and, transposed, its
// inner product collects both rows).  Quadrature: Q = P + 2 Gauss-Lobatto
// points in the uncollapsed directions, Gauss-Radau in the collapsed one
// (the collapsed vertex is not a point); the Duffy Jacobian is folded into
// the geometric factors, which hold d eta / d x (not d xi / d x) so that the
// gradient is taken along the collapsed directions with the 1D collocation
// derivatives and the folded factors do the rest, as for quads / hexes.
//
// One kernel per (shape, operator, order, precision): a CTA walks tiles of
// consecutive elements; the basis tables are copied to shared memory once per
// CTA (the collapsed-direction stages index them with run-time mode indices);
// inputs are loaded with coalesced reads, every stage is a loop of independent
// work items over the tile's elements (the dense tensor-direction stages one
// thread per pencil), outputs are stored straight to HBM.  FP32 kernels hold
// two elements per value (float2, FFMA2), FP64 kernels one.
#include <algorithm>
#include <mutex>
#include <type_traits>
#include <vector>

#include "device_common.cuh"
#include "spx_internal.h"

namespace spx {
namespace {

constexpr int kTri = 1, kPrism = 2, kTet = 3;

template <int P>
struct Tri {
  // first storage index of the modes of row p (p = 0..P) and their count
  __host__ __device__ static constexpr int off(int p) {
    return p == 0 ? 0 : (P + 1) + (p - 1) * P - (p - 1) * p / 2;
  }
  __host__ __device__ static constexpr int cnt(int p) { return p == 0 ? P + 1 : (p == P ? P : P - p); }
  static constexpr int nm = (P + 1) * (P + 2) / 2;
};

template <typename T, int P>
struct CParams {
  static constexpr int n = P + 1, Q = P + 2, nt = (P + 1) * (P + 2) / 2;
  T B1[Q * n];       // psi^a at the GLL points, [i][p]
  T Bb[n * Q * n];   // psi^b_{pq} at the Radau points, [p][k][q]
  T Bc[n * Q * n];   // tetrahedra: psi^c_{k,r} at the Radau points, [k][k3][r]; [0][k3][0] = (1 + z)/2 (apex)
  T D1[Q * Q];       // collocation derivative, GLL points
  T D2[Q * Q];       // collocation derivative, Radau points
  short toff[nt + 1];  // tetrahedra: first mode of triangle mode m (r = 0) and the apex at toff[nt]
  short tdeg[nt];      // tetrahedra: degree k_m of triangle mode m
  const Tile* tiles;
  int n_tiles;
  int eb;            // elements per tile (buffer stride)
  const T* in0;
  const T* geom;     // folded factors (nf blocks of Q^d) or d eta / d x (d^2 blocks)
  const T* lam_f;
  const T* kap_f;
  T* out0;
  T* out1;
  T* out2;
  double lam;
};

// shared-memory carve-up per element (values of T)
template <int SHAPE, int P>
struct CLayout {
  static_assert(SHAPE == kTri || SHAPE == kPrism || SHAPE == kTet, "triangles, prisms and tetrahedra");
  static constexpr int n = P + 1, Q = P + 2, nt = Tri<P>::nm;
  static constexpr int NQ = SHAPE == kTri ? Q * Q : Q * Q * Q;    // quadrature points
  static constexpr int NM = SHAPE == kTri ? nt : (SHAPE == kPrism ? n * nt : (P + 1) * (P + 2) * (P + 3) / 6);
  // after the first (collapsed-direction) stage: tri [p][k], prism [a][p][k], tet [m][k3]
  static constexpr int NF = SHAPE == kTri ? n * Q : (SHAPE == kPrism ? n * n * Q : nt * Q);
  static constexpr int NH = SHAPE == kTri ? 0 : n * Q * Q;       // after the second stage
  // the buffers of quadrature-point values (U, G0, G1, G2, V) hold rows along
  // eta1 of QP >= Q values.  Triangles take QP odd: pencils along eta1 then
  // start in distinct shared-memory banks (a row of an even Q puts them 2Q
  // words apart).  Measured (FP32, P = 4): triangles 0.0168 -> 0.0150 ms;
  // prisms the same and tetrahedra slower (the larger buffers cost tiles), so
  // they keep QP = Q.
  static constexpr int QP = (SHAPE != kTri || Q % 2) ? Q : Q + 1;
  static constexpr int NQP = SHAPE == kTri ? QP * Q : QP * Q * Q;
  __host__ __device__ static constexpr int sq(int q) { return q % Q + QP * (q / Q); }   // point q in a buffer
  // buffers: C (modes), F, H, U, G0, G1, G2, V
  static constexpr int per_elem = NM + NF + NH + 5 * NQP;
  // tables: B1, Bb, Bc, D1, D2 (values of T), then the tet mode tables (ints, rounded up)
  static constexpr int tables = Q * n + 2 * n * Q * n + 2 * Q * Q + (2 * nt + 2);
};

// ---- values: one element (T) or an element pair (float2, FP32) --------------
// FP32 kernels hold every value as a float2 of the same entry of two elements
// of the tile (pair p = elements p and p + npair), so each FFMA2 does two
// elements' work; the 1D tables stay scalar (a broadcast operand).
template <typename T>
struct ValueOf {
  using type = T;
};
template <>
struct ValueOf<float> {
  using type = float2;
};

__device__ __forceinline__ double vfma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float2 vfma(float a, float2 x, float2 c) { return __ffma2_rn(make_float2(a, a), x, c); }
__device__ __forceinline__ float2 vfma(float2 x, float a, float2 c) { return __ffma2_rn(x, make_float2(a, a), c); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ double vmul(double a, double b) { return a * b; }
__device__ __forceinline__ float2 vmul(float a, float2 x) { return __fmul2_rn(make_float2(a, a), x); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ double vadd(double a, double b) { return a + b; }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
template <typename V>
__device__ __forceinline__ V vzero() {
  if constexpr (std::is_same_v<V, float2>) return make_float2(0.f, 0.f);
  else return V(0);
}
template <typename V>
__device__ __forceinline__ V vfill(double a) {
  if constexpr (std::is_same_v<V, float2>) return make_float2(float(a), float(a));
  else return V(a);
}

// Where the values of (pair-)element e of a tile live in global memory: the
// elements first + e and, for pairs, first + e + npair (if below count).
struct PairMap {
  int64_t first;
  int npair, count;
};

template <typename T>
__device__ __forceinline__ typename ValueOf<T>::type vload(const T* g, int64_t stride, const PairMap& pm, int e,
                                                           int64_t off) {
  if constexpr (std::is_same_v<T, double>) {
    return g[(pm.first + e) * stride + off];
  } else {
    const float x = __ldg(g + (pm.first + e) * stride + off);
    const float y = e + pm.npair < pm.count ? __ldg(g + (pm.first + e + pm.npair) * stride + off) : 0.f;
    return make_float2(x, y);
  }
}
template <typename T>
__device__ __forceinline__ void vstore(T* g, int64_t stride, const PairMap& pm, int e, int64_t off,
                                       typename ValueOf<T>::type v) {
  if constexpr (std::is_same_v<T, double>) {
    g[(pm.first + e) * stride + off] = v;
  } else {
    g[(pm.first + e) * stride + off] = v.x;
    if (e + pm.npair < pm.count) g[(pm.first + e + pm.npair) * stride + off] = v.y;
  }
}

// shared-memory carve-up: the tables (T, then the tet mode tables as ints,
// rounded up to an even count of words) and the (pair-)elements' buffers (V)
template <typename T, int SHAPE, int P>
struct Bufs {
  using L = CLayout<SHAPE, P>;
  using V = typename ValueOf<T>::type;
  T *B1, *Bb, *Bc, *D1, *D2;
  V *C, *F, *H, *U, *G0, *G1, *G2, *Vb;
  int* toff;   // [nt + 1]
  int* tdeg;   // [nt]
  static constexpr int table_words = (L::tables + 1) & ~1;
  __device__ Bufs(T* sm, int npe) {
    B1 = sm;
    Bb = B1 + L::Q * L::n;
    Bc = Bb + L::n * L::Q * L::n;
    D1 = Bc + L::n * L::Q * L::n;
    D2 = D1 + L::Q * L::Q;
    toff = reinterpret_cast<int*>(D2 + L::Q * L::Q);
    tdeg = toff + L::nt + 1;
    C = reinterpret_cast<V*>(sm + table_words);
    F = C + npe * L::NM;
    H = F + npe * L::NF;
    U = H + npe * L::NH;
    G0 = U + npe * L::NQP;
    G1 = G0 + npe * L::NQP;
    G2 = G1 + npe * L::NQP;
    Vb = G2 + npe * L::NQP;
  }
};

// ---- collapsed-direction stages ------------------------------------------
// forward: F[e][.. p ..][k] = sum_q C[e][mode(p, q)] Bb[p][k][q] (+ the collapsed vertex in row P);
// `outer` = the number of leading mode blocks (1 triangle, n prism: mode a + n m).
template <typename T, typename V, int P, int OUTER>
__device__ __forceinline__ void stage_b_fwd(const V* C, V* F, const T* Bb, int ne, int tid, int nthr) {
  constexpr int n = P + 1, Q = P + 2, nt = Tri<P>::nm;
  constexpr int items = OUTER * n * Q;
  for (int w = tid; w < ne * items; w += nthr) {
    const int e = w / items, r = w - e * items;
    const int a = r % OUTER, pk = r / OUTER;     // a fastest
    const int p = pk % n, k = pk / n;
    const V* c = C + e * OUTER * nt + a;         // mode m at c[OUTER * m]
    const T* b = Bb + (p * Q + k) * n;
    const int o = Tri<P>::off(p), m = Tri<P>::cnt(p);
    V acc = vzero<V>();
#pragma unroll
    for (int q = 0; q < n; ++q)
      if (q < m) acc = vfma(c[OUTER * (o + q)], b[q], acc);
    if (p == P) acc = vfma(c[OUTER * P], Bb[k * n + P], acc);   // collapsed vertex (0, P)
    F[e * OUTER * n * Q + a + OUTER * (p + n * k)] = acc;
  }
}

// transposed: out[e][mode(p, q)] = sum_k Bb[p][k][q] F[e][.. p ..][k] (+ row P for the collapsed vertex)
template <typename T, typename V, int P, int OUTER>
__device__ __forceinline__ void stage_b_bwd(const V* F, T* out, const PairMap& pm, const T* Bb, int ne, int tid,
                                            int nthr) {
  constexpr int n = P + 1, Q = P + 2, nt = Tri<P>::nm;
  constexpr int items = OUTER * nt;
  for (int w = tid; w < ne * items; w += nthr) {
    const int e = w / items, r = w - e * items;
    const int a = r % OUTER, mi = r / OUTER;
    int p = 0;
#pragma unroll
    for (int pp = 1; pp <= P; ++pp)
      if (mi >= Tri<P>::off(pp)) p = pp;
    const int q = mi - Tri<P>::off(p);
    const V* f = F + e * OUTER * n * Q + a + OUTER * p;
    V acc = vzero<V>();
#pragma unroll
    for (int k = 0; k < Q; ++k) acc = vfma(f[OUTER * n * k], Bb[(p * Q + k) * n + q], acc);
    if (p == 0 && q == P) {   // collapsed vertex: also row P
      const V* fP = F + e * OUTER * n * Q + a + OUTER * P;
#pragma unroll
      for (int k = 0; k < Q; ++k) acc = vfma(fP[OUTER * n * k], Bb[k * n + P], acc);
    }
    vstore(out, OUTER * nt, pm, e, r, acc);
  }
}

// ---- tetrahedra: the eta3 stage over the triangle modes ---------------------
// forward: F[e][m][k3] = sum_r C[e][toff[m] + r] Bc[k_m][k3][r]
//          (+ the apex coefficient for the three triangle vertex modes, whose sum is 1)
template <typename T, typename V, int P>
__device__ __forceinline__ void stage_c_fwd(const V* C, V* F, const T* Bc, const int* toff, const int* tdeg, int ne,
                                            int tid, int nthr) {
  constexpr int n = P + 1, Q = P + 2, nt = Tri<P>::nm, NM = (P + 1) * (P + 2) * (P + 3) / 6;
  constexpr int items = nt * Q;
  for (int w = tid; w < ne * items; w += nthr) {
    const int e = w / items, r0 = w - e * items;
    const int m = r0 % nt, k3 = r0 / nt;
    const int k = tdeg[m], o = toff[m];
    const V* c = C + e * NM;
    const T* b = Bc + (k * Q + k3) * n;
    V acc = vzero<V>();
#pragma unroll
    for (int r = 0; r < n; ++r)
      if (r <= P - k) acc = vfma(c[o + r], b[r], acc);
    if (m == 0 || m == P || m == Tri<P>::off(P)) acc = vfma(c[NM - 1], Bc[k3 * n], acc);   // apex
    F[e * nt * Q + m + nt * k3] = acc;
  }
}

// forward, eta2: H[e][p][j][k3] = sum_q F[e][(p, q)][k3] Bb[p][j][q] (+ row P for the triangle's collapsed vertex)
template <typename T, typename V, int P>
__device__ __forceinline__ void stage_tb_fwd(const V* F, V* H, const T* Bb, int ne, int tid, int nthr) {
  constexpr int n = P + 1, Q = P + 2, nt = Tri<P>::nm;
  constexpr int items = n * Q * Q;
  for (int w = tid; w < ne * items; w += nthr) {
    const int e = w / items, r0 = w - e * items;
    const int p = r0 % n, j = (r0 / n) % Q, k3 = r0 / (n * Q);
    const V* f = F + e * nt * Q + nt * k3;
    const T* b = Bb + (p * Q + j) * n;
    const int o = Tri<P>::off(p), mc = Tri<P>::cnt(p);
    V acc = vzero<V>();
#pragma unroll
    for (int q = 0; q < n; ++q)
      if (q < mc) acc = vfma(f[o + q], b[q], acc);
    if (p == P) acc = vfma(f[P], Bb[j * n + P], acc);
    H[e * n * Q * Q + r0] = acc;
  }
}

// transposed, eta2: F[e][(p, q)][k3] = sum_j Bb[p][j][q] H[e][p][j][k3] (+ row P into (0, P))
template <typename T, typename V, int P>
__device__ __forceinline__ void stage_tb_bwd(const V* H, V* F, const T* Bb, int ne, int tid, int nthr) {
  constexpr int n = P + 1, Q = P + 2, nt = Tri<P>::nm;
  constexpr int items = nt * Q;
  for (int w = tid; w < ne * items; w += nthr) {
    const int e = w / items, r0 = w - e * items;
    const int mi = r0 % nt, k3 = r0 / nt;
    int p = 0;
#pragma unroll
    for (int pp = 1; pp <= P; ++pp)
      if (mi >= Tri<P>::off(pp)) p = pp;
    const int q = mi - Tri<P>::off(p);
    const V* h = H + e * n * Q * Q + p + n * Q * k3;
    V acc = vzero<V>();
#pragma unroll
    for (int j = 0; j < Q; ++j) acc = vfma(h[n * j], Bb[(p * Q + j) * n + q], acc);
    if (p == 0 && q == P) {
      const V* hP = H + e * n * Q * Q + P + n * Q * k3;
#pragma unroll
      for (int j = 0; j < Q; ++j) acc = vfma(hP[n * j], Bb[j * n + P], acc);
    }
    F[e * nt * Q + mi + nt * k3] = acc;
  }
}

// transposed, eta3: out[e][toff[m] + r] = sum_k3 Bc[k_m][k3][r] F[e][m][k3]; the apex
// collects the three triangle vertex modes against (1 + z)/2
template <typename T, typename V, int P>
__device__ __forceinline__ void stage_c_bwd(const V* F, T* out, const PairMap& pm, const T* Bc, const int* toff,
                                            const int* tdeg, int ne, int tid, int nthr) {
  constexpr int n = P + 1, Q = P + 2, nt = Tri<P>::nm, NM = (P + 1) * (P + 2) * (P + 3) / 6;
  for (int w = tid; w < ne * NM; w += nthr) {
    const int e = w / NM, mi = w - e * NM;
    const V* f = F + e * nt * Q;
    V acc = vzero<V>();
    if (mi == NM - 1) {
      const int v1 = P, v2 = Tri<P>::off(P);
#pragma unroll
      for (int k3 = 0; k3 < Q; ++k3)
        acc = vfma(vadd(vadd(f[nt * k3], f[v1 + nt * k3]), f[v2 + nt * k3]), Bc[k3 * n], acc);
    } else {
      int m = 0;
      for (int mm = 1; mm < nt; ++mm)
        if (mi >= toff[mm]) m = mm;
      const int r = mi - toff[m], k = tdeg[m];
#pragma unroll
      for (int k3 = 0; k3 < Q; ++k3) acc = vfma(f[m + nt * k3], Bc[(k * Q + k3) * n + r], acc);
    }
    vstore(out, NM, pm, e, mi, acc);
  }
}

// ---- dense 1D stages on the tensor part ------------------------------------
// y[e][.. i along axis ..] = sum_c A[i][c] x[e][.. c ..] (TR: A[c][i]); extents
// (N0, N1, N2) in and the same with axis AX resized to M out, axis 0 fastest.
// One thread per pencil along AX: its NA inputs are read once into registers
// and every output of the pencil is formed from them, with A at compile-time
// indices.  FP32 kernels pass A in the kernel's parameter block (a
// constant-bank operand of the FMA, no load per multiply-add); FP64 kernels
// pass the shared-memory copy (a broadcast load per multiply-add, hidden by
// the FP64 pipe; constant-bank FP64 operands made the compiler hold many
// table values in registers and spill).  OUT_G: y is the operator's output in
// global memory, written through the pair map.
// X0, Y0: the row strides (axis-0 extents as stored) of x and y, at least
// N0 and the output's axis-0 extent (padded buffers, CLayout::QP).
template <int AX, int N0, int N1, int N2, int M, bool TR, bool ACC, bool OUT_G = false, int X0 = N0,
          int Y0 = (AX == 0 ? M : N0), typename T, typename V, typename Y>
__device__ __forceinline__ void stage_dense(const V* x, Y* y, const T* A, int ne, int tid, int nthr,
                                            const PairMap* pm = nullptr) {
  constexpr int NA = AX == 0 ? N0 : (AX == 1 ? N1 : N2);
  constexpr int O0 = AX == 0 ? M : N0, O1 = AX == 1 ? M : N1, O2 = AX == 2 ? M : N2;
  static_assert(X0 >= N0 && Y0 >= O0 && (!OUT_G || Y0 == O0), "row strides");
  constexpr int XS = X0 * N1 * N2, YS = Y0 * O1 * O2;
  constexpr int SA = AX == 0 ? 1 : (AX == 1 ? X0 : X0 * N1);
  constexpr int SO = AX == 0 ? 1 : (AX == 1 ? Y0 : Y0 * O1);
  constexpr int NP = N0 * N1 * N2 / NA;   // pencils per element
  for (int w = tid; w < ne * NP; w += nthr) {
    const int e = w / NP, r = w - e * NP;
    // the pencil's two other coordinates (the same extents in x and y), fastest first
    const int i0 = AX == 0 ? 0 : r % N0;
    const int i1 = AX == 1 ? 0 : (AX == 0 ? r % N1 : (r / N0) % N1);
    const int i2 = AX == 2 ? 0 : (AX == 0 ? r / N1 : r / N0);
    const V* xe = x + e * XS + i0 + X0 * (i1 + N1 * i2);
    const int yo = i0 + Y0 * (i1 + O1 * i2);
    V v[NA];
#pragma unroll
    for (int c = 0; c < NA; ++c) v[c] = xe[c * SA];
    auto put = [&](int m, V acc) {
      if constexpr (OUT_G) {
        vstore(y, YS, *pm, e, yo + m * SO, acc);
      } else {
        V* ye = y + e * YS + yo + m * SO;
        if (ACC) *ye = vadd(*ye, acc);
        else *ye = acc;
      }
    };
    if constexpr (sizeof(T) == 4) {   // A in the parameter block: every index a constant
#pragma unroll
      for (int m = 0; m < M; ++m) {
        V acc = vmul(TR ? A[m] : A[m * NA], v[0]);
#pragma unroll
        for (int c = 1; c < NA; ++c) acc = vfma(TR ? A[c * M + m] : A[m * NA + c], v[c], acc);
        put(m, acc);
      }
    } else {   // A in shared memory: one output at a time keeps the table loads few
#pragma unroll 1
      for (int m = 0; m < M; ++m) {
        V acc = vmul(TR ? A[m] : A[m * NA], v[0]);
#pragma unroll
        for (int c = 1; c < NA; ++c) acc = vfma(TR ? A[c * M + m] : A[m * NA + c], v[c], acc);
        put(m, acc);
      }
    }
  }
}

// a tile's quadrature-point values (NQ per element) into a padded buffer
template <typename T, typename V, int Q, int QP>
__device__ __forceinline__ void load_tile_q(const T* g, V* s, int NQ, int NQP, const PairMap& pm) {
  for (int i = threadIdx.x; i < pm.npair * NQ; i += blockDim.x) {
    const int e = i / NQ, q = i - e * NQ;
    s[e * NQP + q % Q + QP * (q / Q)] = vload(g, NQ, pm, e, q);
  }
}

// a tile's inputs (len values per element, consecutive elements) into the
// (pair-)element buffer s
template <typename T, typename V>
__device__ __forceinline__ void load_tile(const T* g, V* s, int len, const PairMap& pm) {
  for (int i = threadIdx.x; i < pm.npair * len; i += blockDim.x) {
    const int e = i / len;
    s[i] = vload(g, len, pm, e, i - e * len);
  }
}

// ---- the kernel -------------------------------------------------------------
// OP: OP_BWD, OP_IPROD, OP_DERIV, OP_HELM.  FP32: element pairs (ValueOf).
template <typename T, int SHAPE, int OP, int P>
__global__ void __launch_bounds__(512) collapsed_kernel(const __grid_constant__ CParams<T, P> p) {
  using L = CLayout<SHAPE, P>;
  using V = typename ValueOf<T>::type;
  constexpr int LN = std::is_same_v<V, T> ? 1 : 2;   // elements per value
  constexpr int n = L::n, Q = L::Q, nt = L::nt, NQ = L::NQ, NM = L::NM, QP = L::QP, NQP = L::NQP;
  constexpr int DIM = SHAPE == kTri ? 2 : 3;
  constexpr int NFG = DIM == 3 ? 7 : 4;
  extern __shared__ __align__(16) unsigned char csm[];
  Bufs<T, SHAPE, P> b(reinterpret_cast<T*>(csm), (p.eb + LN - 1) / LN);
  const int tid = threadIdx.x, nthr = blockDim.x;
  // tables of the dense stages (see stage_dense)
  constexpr bool kParamTab = sizeof(T) == 4;
  const T* tB1 = kParamTab ? p.B1 : b.B1;
  const T* tD1 = kParamTab ? p.D1 : b.D1;
  const T* tD2 = kParamTab ? p.D2 : b.D2;
  for (int i = tid; i < Q * n; i += nthr) b.B1[i] = p.B1[i];
  for (int i = tid; i < n * Q * n; i += nthr) {
    b.Bb[i] = p.Bb[i];
    b.Bc[i] = p.Bc[i];
  }
  for (int i = tid; i < Q * Q; i += nthr) {
    b.D1[i] = p.D1[i];
    b.D2[i] = p.D2[i];
  }
  for (int i = tid; i <= nt; i += nthr) b.toff[i] = p.toff[i];
  for (int i = tid; i < nt; i += nthr) b.tdeg[i] = p.tdeg[i];
  __syncthreads();
  for (int ti = blockIdx.x; ti < p.n_tiles; ti += gridDim.x) {
    const Tile t = p.tiles[ti];
    const int ne = (t.count + LN - 1) / LN;   // (pair-)elements of the tile
    const PairMap pm{t.first, ne, t.count};
    // the next tile's inputs and geometric factors into L2 while this one runs
    // (its tile load and pointwise reads then wait on L2, not HBM)
    if (tid == 0 && ti + int(gridDim.x) < p.n_tiles) {
      const Tile tn = p.tiles[ti + gridDim.x];
      const int64_t in_len = (OP == OP_BWD || OP == OP_HELM) ? NM : NQ;
      prefetch_l2(p.in0 + tn.first * in_len, uint64_t(tn.count) * in_len * sizeof(T));
      if (OP == OP_IPROD) {   // JW only
        for (int j = 0; j < tn.count; ++j)
          prefetch_l2(p.geom + ((tn.first + j) * NFG + NFG - 1) * int64_t(NQ), uint64_t(NQ) * sizeof(T));
      } else if (OP != OP_BWD) {
        const int64_t g_len = OP == OP_DERIV ? int64_t(DIM) * DIM * NQ : int64_t(NFG) * NQ;
        prefetch_l2(p.geom + tn.first * g_len, uint64_t(tn.count) * g_len * sizeof(T));
      }
    }
    if constexpr (OP == OP_BWD || OP == OP_HELM) {
      load_tile(p.in0, b.C, NM, pm);
      __syncthreads();
      // collapsed direction, then the tensor directions -> U (or straight to HBM)
      constexpr bool G = OP == OP_BWD;
      if constexpr (SHAPE == kTri) {
        stage_b_fwd<T, V, P, 1>(b.C, b.F, b.Bb, ne, tid, nthr);
        __syncthreads();
        if constexpr (G) stage_dense<0, n, Q, 1, Q, false, false, true>(b.F, p.out0, tB1, ne, tid, nthr, &pm);
        else stage_dense<0, n, Q, 1, Q, false, false, false, n, QP>(b.F, b.U, tB1, ne, tid, nthr);   // u[i][j]
      } else if constexpr (SHAPE == kTet) {
        stage_c_fwd<T, V, P>(b.C, b.F, b.Bc, b.toff, b.tdeg, ne, tid, nthr);   // F[m][k3]
        __syncthreads();
        stage_tb_fwd<T, V, P>(b.F, b.H, b.Bb, ne, tid, nthr);   // H[p][j][k3]
        __syncthreads();
        if constexpr (G) stage_dense<0, n, Q, Q, Q, false, false, true>(b.H, p.out0, tB1, ne, tid, nthr, &pm);
        else stage_dense<0, n, Q, Q, Q, false, false, false, n, QP>(b.H, b.U, tB1, ne, tid, nthr);   // u[i][j][k3]
      } else {
        stage_b_fwd<T, V, P, n>(b.C, b.F, b.Bb, ne, tid, nthr);   // F[a][p][k]
        __syncthreads();
        stage_dense<1, n, n, Q, Q, false, false>(b.F, b.H, tB1, ne, tid, nthr);   // H[a][j][k]
        __syncthreads();
        if constexpr (G) stage_dense<0, n, Q, Q, Q, false, false, true>(b.H, p.out0, tB1, ne, tid, nthr, &pm);
        else stage_dense<0, n, Q, Q, Q, false, false, false, n, QP>(b.H, b.U, tB1, ne, tid, nthr);   // u[i][j][k]
      }
      __syncthreads();
    } else {
      load_tile_q<T, V, Q, QP>(p.in0, OP == OP_DERIV ? b.U : b.Vb, NQ, NQP, pm);
      __syncthreads();
    }
    if constexpr (OP == OP_DERIV || OP == OP_HELM) {
      // gradient along the collapsed directions: G0, G1 (, G2)
      if constexpr (SHAPE == kTri) {
        stage_dense<0, Q, Q, 1, Q, false, false, false, QP, QP>(b.U, b.G0, tD1, ne, tid, nthr);
        stage_dense<1, Q, Q, 1, Q, false, false, false, QP, QP>(b.U, b.G1, tD2, ne, tid, nthr);
      } else {   // eta2 on GLL points (prism) or Gauss-Radau points (tetrahedron)
        stage_dense<0, Q, Q, Q, Q, false, false, false, QP, QP>(b.U, b.G0, tD1, ne, tid, nthr);
        stage_dense<1, Q, Q, Q, Q, false, false, false, QP, QP>(b.U, b.G1, SHAPE == kTet ? tD2 : tD1, ne, tid,
                                                                nthr);
        stage_dense<2, Q, Q, Q, Q, false, false, false, QP, QP>(b.U, b.G2, tD2, ne, tid, nthr);
      }
      __syncthreads();
    }
    if constexpr (OP == OP_DERIV) {
      T* outs[3] = {p.out0, p.out1, p.out2};
      constexpr int64_t KS = int64_t(DIM) * DIM * NQ;   // d eta_a / d x_m: block a d + m
      for (int w = tid; w < ne * NQ; w += nthr) {
        const int e = w / NQ, q = w - e * NQ, sw = e * NQP + L::sq(q);
        V d[DIM];
        d[0] = b.G0[sw];
        d[1] = b.G1[sw];
        if (DIM == 3) d[DIM - 1] = b.G2[sw];
#pragma unroll
        for (int m = 0; m < DIM; ++m) {
          V acc = vmul(vload(p.geom, KS, pm, e, int64_t(m) * NQ + q), d[0]);
#pragma unroll
          for (int a = 1; a < DIM; ++a) acc = vfma(vload(p.geom, KS, pm, e, int64_t(a * DIM + m) * NQ + q), d[a], acc);
          vstore(outs[m], NQ, pm, e, q, acc);
        }
      }
      __syncthreads();
      continue;
    }
    if constexpr (OP == OP_HELM) {
      // pointwise: g_a = kappa sum_b G_ab d_b (into G0, G1, G2), V = lambda JW u
      constexpr int64_t GS = int64_t(NFG) * NQ;
      for (int w0 = tid; w0 < ne * NQ; w0 += nthr) {
        const int e = w0 / NQ, q = w0 - e * NQ, w = e * NQP + L::sq(q);
        auto g = [&](int f) { return vload(p.geom, GS, pm, e, int64_t(f) * NQ + q); };
        const V kk = p.kap_f ? vload(p.kap_f, NQ, pm, e, q) : vfill<V>(1.0);
        const V ll = p.lam_f ? vload(p.lam_f, NQ, pm, e, q) : vfill<V>(p.lam);
        if constexpr (DIM == 2) {
          const V d0 = b.G0[w], d1 = b.G1[w];
          const V g00 = g(0), g01 = g(1), g11 = g(2), jw = g(3);
          b.G0[w] = vmul(kk, vfma(g01, d1, vmul(g00, d0)));
          b.G1[w] = vmul(kk, vfma(g11, d1, vmul(g01, d0)));
          b.Vb[w] = vmul(vmul(ll, jw), b.U[w]);
        } else {
          const V d0 = b.G0[w], d1 = b.G1[w], d2 = b.G2[w];
          const V g00 = g(0), g01 = g(1), g02 = g(2), g11 = g(3), g12 = g(4), g22 = g(5), jw = g(6);
          b.G0[w] = vmul(kk, vfma(g02, d2, vfma(g01, d1, vmul(g00, d0))));
          b.G1[w] = vmul(kk, vfma(g12, d2, vfma(g11, d1, vmul(g01, d0))));
          b.G2[w] = vmul(kk, vfma(g22, d2, vfma(g12, d1, vmul(g02, d0))));
          b.Vb[w] = vmul(vmul(ll, jw), b.U[w]);
        }
      }
      __syncthreads();
      // transposed gradient added to V
      if constexpr (SHAPE == kTri) {
        stage_dense<0, Q, Q, 1, Q, true, true, false, QP, QP>(b.G0, b.Vb, tD1, ne, tid, nthr);
        __syncthreads();
        stage_dense<1, Q, Q, 1, Q, true, true, false, QP, QP>(b.G1, b.Vb, tD2, ne, tid, nthr);
      } else {
        stage_dense<0, Q, Q, Q, Q, true, true, false, QP, QP>(b.G0, b.Vb, tD1, ne, tid, nthr);
        __syncthreads();
        stage_dense<1, Q, Q, Q, Q, true, true, false, QP, QP>(b.G1, b.Vb, SHAPE == kTet ? tD2 : tD1, ne, tid,
                                                              nthr);
        __syncthreads();
        stage_dense<2, Q, Q, Q, Q, true, true, false, QP, QP>(b.G2, b.Vb, tD2, ne, tid, nthr);
      }
      __syncthreads();
    }
    if constexpr (OP == OP_IPROD) {
      constexpr int64_t GS = int64_t(NFG) * NQ;
      for (int w = tid; w < ne * NQ; w += nthr) {
        const int e = w / NQ, q = w - e * NQ, sw = e * NQP + L::sq(q);
        b.Vb[sw] = vmul(b.Vb[sw], vload(p.geom, GS, pm, e, int64_t(NFG - 1) * NQ + q));
      }
      __syncthreads();
    }
    if constexpr (OP == OP_IPROD || OP == OP_HELM) {
      // transposed tensor directions, then the collapsed direction -> HBM
      if constexpr (SHAPE == kTri) {
        stage_dense<0, Q, Q, 1, n, true, false, false, QP>(b.Vb, b.F, tB1, ne, tid, nthr);   // F[p][k]
        __syncthreads();
        stage_b_bwd<T, V, P, 1>(b.F, p.out0, pm, b.Bb, ne, tid, nthr);
      } else if constexpr (SHAPE == kTet) {
        stage_dense<0, Q, Q, Q, n, true, false, false, QP>(b.Vb, b.H, tB1, ne, tid, nthr);   // H[p][j][k3]
        __syncthreads();
        stage_tb_bwd<T, V, P>(b.H, b.F, b.Bb, ne, tid, nthr);   // F[m][k3]
        __syncthreads();
        stage_c_bwd<T, V, P>(b.F, p.out0, pm, b.Bc, b.toff, b.tdeg, ne, tid, nthr);
      } else {
        stage_dense<0, Q, Q, Q, n, true, false, false, QP>(b.Vb, b.H, tB1, ne, tid, nthr);   // H[a][j][k]
        __syncthreads();
        stage_dense<1, n, Q, Q, n, true, false>(b.H, b.F, tB1, ne, tid, nthr);   // F[a][p][k]
        __syncthreads();
        stage_b_bwd<T, V, P, n>(b.F, p.out0, pm, b.Bb, ne, tid, nthr);
      }
    }
    __syncthreads();   // the tile's buffers are reused by the next tile
  }
  (void)nt;
}

}  // namespace
}  // namespace spx

// ===========================================================================
// Host side
// ===========================================================================
namespace spx {

// Shared-memory bytes of a collapsed-element launch: tables + eb elements' buffers.
template <typename T, int SHAPE, int P>
size_t collapsed_smem_t(int eb) {
  using L = CLayout<SHAPE, P>;
  constexpr int LN = sizeof(T) == 4 ? 2 : 1;   // FP32: buffers of element pairs (float2)
  const int npe = (eb + LN - 1) / LN;
  return size_t(((L::tables + 1) & ~1) + npe * LN * L::per_elem) * sizeof(T);
}

#if defined(SPX_CT)
namespace {
template <typename T, int SHAPE, int OP, int P>
spx_status launch_c(const LaunchReq& r) {
  using Prm = CParams<T, P>;
  const spx_plan* plan = r.plan;
  const LaunchCfg& cfg = plan->cfg[OP][r.dtype];
  const TileList& tl = plan->tiles[OP][r.dtype];
  if (tl.n == 0) return SPX_OK;
  Prm prm{};
  constexpr int n = P + 1, Q = P + 2;
  const std::vector<double>& ct = plan->ctab;   // B1, Bb, D1, D2, Bc (FP64)
  int o = 0;
  for (int i = 0; i < Q * n; ++i) prm.B1[i] = static_cast<T>(ct[o++]);
  for (int i = 0; i < n * Q * n; ++i) prm.Bb[i] = static_cast<T>(ct[o++]);
  for (int i = 0; i < Q * Q; ++i) prm.D1[i] = static_cast<T>(ct[o++]);
  for (int i = 0; i < Q * Q; ++i) prm.D2[i] = static_cast<T>(ct[o++]);
  for (int i = 0; i < n * Q * n; ++i) prm.Bc[i] = static_cast<T>(ct[o++]);
  // tetrahedra: first mode and degree of every triangle mode (storage order p outer, q inner)
  constexpr int nt = (P + 1) * (P + 2) / 2;
  int m = 0, acc = 0;
  for (int pp = 0; pp <= P; ++pp) {
    const int cnt = pp == 0 ? P + 1 : (pp == P ? P : P - pp);
    for (int q = 0; q < cnt; ++q, ++m) {
      int k;
      if ((pp == 0 && (q == 0 || q == P)) || (pp == P && q == 0)) k = 1;
      else if (pp == 0 || pp == P) k = q + 1;
      else k = q == 0 ? pp + 1 : pp + q + 1;
      prm.tdeg[m] = static_cast<short>(k);
      prm.toff[m] = static_cast<short>(acc);
      acc += P - k + 1;
    }
  }
  prm.toff[nt] = static_cast<short>(acc);   // the apex
  prm.tiles = tl.d;
  prm.n_tiles = tl.n;
  prm.eb = cfg.order[P].eb;
  prm.in0 = static_cast<const T*>(r.in0);
  prm.geom = static_cast<const T*>(r.geom);
  prm.lam_f = static_cast<const T*>(r.lam_f);
  prm.kap_f = static_cast<const T*>(r.kap_f);
  prm.out0 = static_cast<T*>(r.out0);
  prm.out1 = static_cast<T*>(r.out1);
  prm.out2 = static_cast<T*>(r.out2);
  prm.lam = r.lam;
  const size_t smem = collapsed_smem_t<T, SHAPE, P>(prm.eb);
  if (smem > plan->max_smem) return fail(SPX_ERR_UNSUPPORTED, "collapsed tile does not fit in shared memory");
  auto kern = collapsed_kernel<T, SHAPE, OP, P>;
  static std::mutex mu;
  static bool configured = false;
  {
    std::lock_guard<std::mutex> g(mu);
    if (!configured) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           static_cast<int>(plan->max_smem));
      if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
      configured = true;
    }
  }
  const int nthr = cfg.nthreads;
  int nb = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, nthr, smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  if (nb < 1) return fail(SPX_ERR_UNSUPPORTED, "collapsed tile does not fit on an SM");
  const int grid = static_cast<int>(std::min<int64_t>(tl.n, int64_t(nb) * plan->num_sms));
  kern<<<grid, nthr, smem, r.stream>>>(prm);
  e = cudaGetLastError();
  return e == cudaSuccess ? SPX_OK : cuda_fail(e, "collapsed kernel launch");
}

template <typename T, int SHAPE, int OP>
spx_status launch_orders(const LaunchReq& r) {
  switch (r.plan->uP) {
    case 1: return launch_c<T, SHAPE, OP, 1>(r);
    case 2: return launch_c<T, SHAPE, OP, 2>(r);
    case 3: return launch_c<T, SHAPE, OP, 3>(r);
    case 4: return launch_c<T, SHAPE, OP, 4>(r);
    case 5: return launch_c<T, SHAPE, OP, 5>(r);
    case 6: return launch_c<T, SHAPE, OP, 6>(r);
    case 7: return launch_c<T, SHAPE, OP, 7>(r);
    case 8: return launch_c<T, SHAPE, OP, 8>(r);
    default: return fail(SPX_ERR_UNSUPPORTED, "order out of range");
  }
}

template <int SHAPE, int P>
size_t smem_orders_t(int dtype, int eb) {
  return dtype == 0 ? collapsed_smem_t<double, SHAPE, P>(eb) : collapsed_smem_t<float, SHAPE, P>(eb);
}
}  // namespace

#define SPX_C_CAT_(a, b, c) a##b##_##c
#define SPX_C_CAT(a, b, c) SPX_C_CAT_(a, b, c)
#define SPX_C_T_f32 float
#define SPX_C_T_f64 double
#define SPX_C_TYPE_(tn) SPX_C_T_##tn
#define SPX_C_TYPE(tn) SPX_C_TYPE_(tn)
// launch_collapsed_<tn>_<shape>: the operators of one precision and shape
spx_status SPX_C_CAT(launch_collapsed_, SPX_CT, SPX_CS)(const LaunchReq& r) {
  using T = SPX_C_TYPE(SPX_CT);
  switch (r.op) {
    case OP_BWD: return launch_orders<T, SPX_CS, OP_BWD>(r);
    case OP_IPROD: return launch_orders<T, SPX_CS, OP_IPROD>(r);
    case OP_DERIV: return launch_orders<T, SPX_CS, OP_DERIV>(r);
    case OP_HELM: return launch_orders<T, SPX_CS, OP_HELM>(r);
    default: return fail(SPX_ERR_UNSUPPORTED, "operator not available for triangles / prisms");
  }
}
#endif  // SPX_CT

#if defined(SPX_CGEOM)
// Shared-memory bytes of a collapsed-element launch (api.cu's tile checks).
size_t collapsed_smem_bytes(const spx_plan* plan, int dtype, int eb) {
  const int P = plan->uP;
  switch (plan->shape * 16 + P) {
#define SPX_CSM(S, Pv) \
  case S * 16 + Pv: return dtype == 0 ? collapsed_smem_t<double, S, Pv>(eb) : collapsed_smem_t<float, S, Pv>(eb);
    SPX_CSM(1, 1) SPX_CSM(1, 2) SPX_CSM(1, 3) SPX_CSM(1, 4) SPX_CSM(1, 5) SPX_CSM(1, 6) SPX_CSM(1, 7) SPX_CSM(1, 8)
    SPX_CSM(2, 1) SPX_CSM(2, 2) SPX_CSM(2, 3) SPX_CSM(2, 4) SPX_CSM(2, 5) SPX_CSM(2, 6) SPX_CSM(2, 7) SPX_CSM(2, 8)
    SPX_CSM(3, 1) SPX_CSM(3, 2) SPX_CSM(3, 3) SPX_CSM(3, 4) SPX_CSM(3, 5) SPX_CSM(3, 6) SPX_CSM(3, 7) SPX_CSM(3, 8)
#undef SPX_CSM
    default: return SIZE_MAX;
  }
}

spx_status launch_collapsed_f64_1(const LaunchReq& r);
spx_status launch_collapsed_f64_2(const LaunchReq& r);
spx_status launch_collapsed_f64_3(const LaunchReq& r);
spx_status launch_collapsed_f32_1(const LaunchReq& r);
spx_status launch_collapsed_f32_2(const LaunchReq& r);
spx_status launch_collapsed_f32_3(const LaunchReq& r);

spx_status launch_collapsed(const LaunchReq& r) {
  const int sh = r.plan->shape;
  if (r.dtype == 0) return sh == kTri ? launch_collapsed_f64_1(r) : (sh == kPrism ? launch_collapsed_f64_2(r)
                                                                                  : launch_collapsed_f64_3(r));
  return sh == kTri ? launch_collapsed_f32_1(r) : (sh == kPrism ? launch_collapsed_f32_2(r) : launch_collapsed_f32_3(r));
}

// ---- geometric factors of affine collapsed elements (FP64) ------------------
// One thread per quadrature point: J = [(V_c - V0) / 2]_c (constant on the
// element), d eta / d x = (d eta / d xi) J^{-1} with the collapse's chain rule,
// JW = w det J including the Duffy factor, G = JW (d eta/dx)(d eta/dx)^T.
struct CGeomParams {
  const double* verts;     // [E][d+1][d]
  double* geom;            // [E][nf][Q^d] or NULL
  double* dxi;             // [E][d*d][Q^d] or NULL
  double* xq;              // [E][d][Q^d] or NULL
  float* geom32;
  float* dxi32;
  int64_t E;
  int d, Q;
  int tet;                 // 3D: tetrahedra (else prisms)
  double xg[16], wg[16], xr[16], wr[16];
};

__global__ void collapsed_geom_kernel(const __grid_constant__ CGeomParams g) {
  const int d = g.d, Q = g.Q;
  const int NQ = d == 2 ? Q * Q : Q * Q * Q;
  const int nf = d == 2 ? 4 : 7;
  const int64_t total = g.E * NQ;
  for (int64_t w = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; w < total; w += int64_t(gridDim.x) * blockDim.x) {
    const int64_t e = w / NQ;
    const int q = static_cast<int>(w - e * NQ);
    const double* V = g.verts + e * (d + 1) * d;
    double J[3][3] = {}, Ji[3][3] = {};
    for (int m = 0; m < d; ++m)
      for (int c = 0; c < d; ++c) J[m][c] = 0.5 * (V[(c + 1) * d + m] - V[m]);
    double det;
    if (d == 2) {
      det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
      Ji[0][0] = J[1][1] / det;
      Ji[0][1] = -J[0][1] / det;
      Ji[1][0] = -J[1][0] / det;
      Ji[1][1] = J[0][0] / det;
    } else {
      det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
            J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {   // inverse = adjugate / det
          const int i1 = (j + 1) % 3, i2 = (j + 2) % 3, j1 = (i + 1) % 3, j2 = (i + 2) % 3;
          Ji[i][j] = (J[i1][j1] * J[i2][j2] - J[i1][j2] * J[i2][j1]) / det;
        }
    }
    // collapsed point, reference point, weight, d eta / d xi
    double eta[3] = {}, xi[3] = {}, K[3][3] = {}, wt;
    if (d == 2) {
      const int i = q % Q, j = q / Q;
      eta[0] = g.xg[i];
      eta[1] = g.xr[j];
      const double s = 1.0 / (1.0 - eta[1]);
      xi[0] = 0.5 * (1.0 + eta[0]) * (1.0 - eta[1]) - 1.0;
      xi[1] = eta[1];
      K[0][0] = 2.0 * s;
      K[0][1] = (1.0 + eta[0]) * s;
      K[1][1] = 1.0;
      wt = g.wg[i] * g.wr[j] * 0.5 * (1.0 - eta[1]);
    } else if (g.tet) {
      const int i = q % Q, j = (q / Q) % Q, k = q / (Q * Q);
      eta[0] = g.xg[i];
      eta[1] = g.xr[j];
      eta[2] = g.xr[k];
      const double s23 = 1.0 / ((1.0 - eta[1]) * (1.0 - eta[2])), s3 = 1.0 / (1.0 - eta[2]);
      xi[0] = 0.25 * (1.0 + eta[0]) * (1.0 - eta[1]) * (1.0 - eta[2]) - 1.0;
      xi[1] = 0.5 * (1.0 + eta[1]) * (1.0 - eta[2]) - 1.0;
      xi[2] = eta[2];
      K[0][0] = 4.0 * s23;
      K[0][1] = 2.0 * (1.0 + eta[0]) * s23;
      K[0][2] = 2.0 * (1.0 + eta[0]) * s23;
      K[1][1] = 2.0 * s3;
      K[1][2] = (1.0 + eta[1]) * s3;
      K[2][2] = 1.0;
      const double h3 = 0.5 * (1.0 - eta[2]);
      wt = g.wg[i] * g.wr[j] * g.wr[k] * 0.5 * (1.0 - eta[1]) * h3 * h3;
    } else {
      const int i = q % Q, j = (q / Q) % Q, k = q / (Q * Q);
      eta[0] = g.xg[i];
      eta[1] = g.xg[j];
      eta[2] = g.xr[k];
      const double s = 1.0 / (1.0 - eta[2]);
      xi[0] = eta[0];
      xi[1] = 0.5 * (1.0 + eta[1]) * (1.0 - eta[2]) - 1.0;
      xi[2] = eta[2];
      K[0][0] = 1.0;
      K[1][1] = 2.0 * s;
      K[1][2] = (1.0 + eta[1]) * s;
      K[2][2] = 1.0;
      wt = g.wg[i] * g.wg[j] * g.wr[k] * 0.5 * (1.0 - eta[2]);
    }
    double Kx[3][3] = {};   // d eta_a / d x_m
    for (int a = 0; a < d; ++a)
      for (int m = 0; m < d; ++m) {
        double acc = 0.0;
        for (int c = 0; c < d; ++c) acc += K[a][c] * Ji[c][m];
        Kx[a][m] = acc;
      }
    const double jw = wt * det;
    const int64_t base = e * NQ;
    if (g.geom || g.geom32) {
      double f[7];
      int t = 0;
      for (int a = 0; a < d; ++a)
        for (int b2 = a; b2 < d; ++b2) {
          double acc = 0.0;
          for (int m = 0; m < d; ++m) acc += Kx[a][m] * Kx[b2][m];
          f[t++] = jw * acc;
        }
      f[t++] = jw;
      for (int s2 = 0; s2 < nf; ++s2) {
        if (g.geom) g.geom[(base * nf) + s2 * NQ + q] = f[s2];
        if (g.geom32) g.geom32[(base * nf) + s2 * NQ + q] = static_cast<float>(f[s2]);
      }
    }
    if (g.dxi || g.dxi32)
      for (int a = 0; a < d; ++a)
        for (int m = 0; m < d; ++m) {
          const int64_t o = base * d * d + (a * d + m) * int64_t(NQ) + q;
          if (g.dxi) g.dxi[o] = Kx[a][m];
          if (g.dxi32) g.dxi32[o] = static_cast<float>(Kx[a][m]);
        }
    if (g.xq)
      for (int m = 0; m < d; ++m) {
        double x = V[m];
        for (int c = 0; c < d; ++c) x += J[m][c] * (xi[c] + 1.0);
        g.xq[base * d + m * int64_t(NQ) + q] = x;
      }
  }
}

spx_status collapsed_geom(const spx_plan* plan, const double* verts, double* geom, double* dxi, double* xq,
                          float* geom32, float* dxi32, cudaStream_t st) {
  CGeomParams g{};
  g.verts = verts;
  g.geom = geom;
  g.dxi = dxi;
  g.xq = xq;
  g.geom32 = geom32;
  g.dxi32 = dxi32;
  g.E = plan->E;
  g.d = plan->dim;
  g.Q = plan->uP + 2;
  g.tet = plan->shape == kTet ? 1 : 0;
  spx_status s = collapsed_tables(plan->uP, g.Q, nullptr, nullptr, nullptr, nullptr, g.xg, g.wg, g.xr, g.wr);
  if (s != SPX_OK) return s;
  const int64_t total = plan->E * (plan->dim == 2 ? g.Q * g.Q : g.Q * g.Q * g.Q);
  const int grid = static_cast<int>(std::min<int64_t>((total + 255) / 256, int64_t(plan->num_sms) * 32));
  collapsed_geom_kernel<<<grid, 256, 0, st>>>(g);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SPX_OK : cuda_fail(e, "collapsed geometry kernel launch");
}
#endif  // SPX_CGEOM

}  // namespace spx
