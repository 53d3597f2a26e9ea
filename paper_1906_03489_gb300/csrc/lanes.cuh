// Value types of the operator kernels and the even-odd evaluation of their
// 1D contractions (sum-factorisation display of §3.3, one direction at a time).
#pragma once
#include <cuda_runtime.h>

#include "kernel_params.h"

namespace spx {

// Value types of the kernel: float2 = the same entry of two elements (packed
// f32x2 arithmetic, 8-byte shared accesses, bank modulus 16 per half-warp);
// float = one element (bank modulus 32 per warp).
template <class V>
struct Lane;
template <>
struct Lane<float2> {
  static constexpr int L = 2, M = 16;
  static __device__ __forceinline__ float2 zero() { return make_float2(0.f, 0.f); }
  static __device__ __forceinline__ float2 bcast(float a) { return make_float2(a, a); }
  static __device__ __forceinline__ float2 fma(float a, float2 x, float2 y) { return __ffma2_rn(make_float2(a, a), x, y); }
  static __device__ __forceinline__ float2 fmav(float2 a, float2 x, float2 y) { return __ffma2_rn(a, x, y); }
  static __device__ __forceinline__ float2 mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
  static __device__ __forceinline__ float2 add(float2 a, float2 b) { return __fadd2_rn(a, b); }
  static __device__ __forceinline__ float2 pair(float x, float y) { return make_float2(x, y); }
  static __device__ __forceinline__ float2 ldcs2(const float* p0, const float* p1) {
    return make_float2(__ldcs(p0), __ldcs(p1));
  }
  static __device__ __forceinline__ void stcs2(float* y0, float* y1, float2 v, bool two) {
    __stcs(y0, v.x);
    if (two) __stcs(y1, v.y);
  }
  static __device__ __forceinline__ float2 from2(float2 v) { return v; }
  static __device__ __forceinline__ float2 to2(float2 v) { return v; }
};
template <>
struct Lane<float> {
  static constexpr int L = 1, M = 32;
  static __device__ __forceinline__ float zero() { return 0.f; }
  static __device__ __forceinline__ float bcast(float a) { return a; }
  static __device__ __forceinline__ float fma(float a, float x, float y) { return fmaf(a, x, y); }
  static __device__ __forceinline__ float fmav(float a, float x, float y) { return fmaf(a, x, y); }
  static __device__ __forceinline__ float mul(float a, float b) { return a * b; }
  static __device__ __forceinline__ float add(float a, float b) { return a + b; }
  static __device__ __forceinline__ float pair(float x, float) { return x; }
  static __device__ __forceinline__ float ldcs2(const float* p0, const float*) { return __ldcs(p0); }
  static __device__ __forceinline__ void stcs2(float* y0, float*, float v, bool) { __stcs(y0, v); }
  static __device__ __forceinline__ float from2(float2 v) { return v.x; }
  static __device__ __forceinline__ float2 to2(float v) { return make_float2(v, 0.f); }
};
template <>
struct Lane<double> {
  static constexpr int L = 1, M = 16;
  static __device__ __forceinline__ double zero() { return 0.0; }
  static __device__ __forceinline__ double bcast(double a) { return a; }
  static __device__ __forceinline__ double fma(double a, double x, double y) { return ::fma(a, x, y); }
  static __device__ __forceinline__ double fmav(double a, double x, double y) { return ::fma(a, x, y); }
  static __device__ __forceinline__ double mul(double a, double b) { return a * b; }
  static __device__ __forceinline__ double add(double a, double b) { return a + b; }
};

// Shared by the three value types: a - b, and a scalar times a value.
__device__ __forceinline__ float2 vsub(float2 a, float2 b) { return __ffma2_rn(make_float2(-1.f, -1.f), b, a); }
__device__ __forceinline__ float vsub(float a, float b) { return a - b; }
__device__ __forceinline__ double vsub(double a, double b) { return a - b; }
__device__ __forceinline__ float2 vscale(float a, float2 x) { return __fmul2_rn(make_float2(a, a), x); }
__device__ __forceinline__ float vscale(float a, float x) { return a * x; }
__device__ __forceinline__ double vscale(double a, double x) { return a * x; }

// ---------------------------------------------------------------------------
// Even-odd contractions (EOLayout in kernel_params.h).  `tab` is the order's
// table in the kernel's scalar type S, indexed with compile-time constants
// (constant bank); V the value type.  Register arrays in and out.
// ---------------------------------------------------------------------------

// u[Q] = B v[n]   (modal -> quadrature along one direction)
template <int P, int Q, class V, class S>
__device__ __forceinline__ void eo_b(const S* tab, const V* v, V* u) {
  using E = EOLayout<P, Q>;
  using Vt = Lane<V>;
  constexpr int n = P + 1, H = Q / 2;
  const S* B = tab;
  const V e = Vt::add(v[0], v[P]);
  const V o = vsub(v[0], v[P]);
#pragma unroll
  for (int i = 0; i < E::Hc; ++i) {
    V s = vscale(tab[E::Bs + i], e);
#pragma unroll
    for (int b = 1; b < P; b += 2) s = Vt::fma(B[i * n + b], v[b], s);
    if (i == H) {  // middle point of an odd Q: the antisymmetric part vanishes
      u[i] = s;
    } else {
      V d = vscale(tab[E::Bd + i], o);
#pragma unroll
      for (int b = 2; b < P; b += 2) d = Vt::fma(B[i * n + b], v[b], d);
      u[i] = Vt::add(s, d);
      u[Q - 1 - i] = vsub(s, d);
    }
  }
}

// u[Q] = dB v[n]   (derivative of the expansion at the quadrature points along
// one direction; the opposite parity of B, EOLayout)
template <int P, int Q, class V, class S>
__device__ __forceinline__ void eo_db(const S* tab, const V* v, V* u) {
  using E = EOLayout<P, Q>;
  using Vt = Lane<V>;
  constexpr int n = P + 1, H = Q / 2;
  const S* dB = tab + Q * n;
  const V e = Vt::add(v[0], v[P]);
  const V o = vsub(v[0], v[P]);
#pragma unroll
  for (int i = 0; i < E::Hc; ++i) {
    V s = vscale(tab[E::Gd + i], o);
#pragma unroll
    for (int b = 2; b < P; b += 2) s = Vt::fma(dB[i * n + b], v[b], s);
    if (i == H) {  // middle point of an odd Q: the antisymmetric part vanishes
      u[i] = s;
    } else {
      V a = vscale(tab[E::Gs + i], e);
#pragma unroll
      for (int b = 1; b < P; b += 2) a = Vt::fma(dB[i * n + b], v[b], a);
      u[i] = Vt::add(s, a);
      u[Q - 1 - i] = vsub(s, a);
    }
  }
}

// y[n] = B^T w[Q]   (quadrature -> modal, the inner product along one direction)
template <int P, int Q, class V, class S>
__device__ __forceinline__ void eo_bt(const S* tab, const V* w, V* y) {
  using E = EOLayout<P, Q>;
  using Vt = Lane<V>;
  constexpr int n = P + 1, H = Q / 2, Hc = E::Hc;
  const S* B = tab;
  V sv[Hc], dv[H];
#pragma unroll
  for (int i = 0; i < H; ++i) {
    sv[i] = Vt::add(w[i], w[Q - 1 - i]);
    dv[i] = vsub(w[i], w[Q - 1 - i]);
  }
  if (Hc > H) sv[H] = w[H];
  V a = Vt::zero(), c = Vt::zero();
#pragma unroll
  for (int i = 0; i < Hc; ++i) a = Vt::fma(tab[E::Bs + i], sv[i], a);
#pragma unroll
  for (int i = 0; i < H; ++i) c = Vt::fma(tab[E::Bd + i], dv[i], c);
  y[0] = Vt::add(a, c);
  y[P] = vsub(a, c);
#pragma unroll
  for (int b = 1; b < P; ++b) {
    V acc = Vt::zero();
    if (b & 1) {
#pragma unroll
      for (int i = 0; i < Hc; ++i) acc = Vt::fma(B[i * n + b], sv[i], acc);
    } else {
#pragma unroll
      for (int i = 0; i < H; ++i) acc = Vt::fma(B[i * n + b], dv[i], acc);
    }
    y[b] = acc;
  }
}

// y[Q] = D v[Q] (TR = false) or D^T v[Q] (TR = true)
template <int P, int Q, bool TR, class V, class S>
__device__ __forceinline__ void eo_d(const S* tab, const V* v, V* y) {
  using E = EOLayout<P, Q>;
  using Vt = Lane<V>;
  constexpr int n = P + 1, H = Q / 2, M = Q / 2;
  const S* D = tab + 2 * Q * n;
  const S* Xp = tab + (TR ? E::Tp : E::Dp);
  const S* Xm = tab + (TR ? E::Tm : E::Dm);
  V sv[H], dv[H];
#pragma unroll
  for (int j = 0; j < H; ++j) {
    sv[j] = Vt::add(v[j], v[Q - 1 - j]);
    dv[j] = vsub(v[j], v[Q - 1 - j]);
  }
#pragma unroll
  for (int i = 0; i < H; ++i) {
    V e = Vt::zero(), f = Vt::zero();
#pragma unroll
    for (int j = 0; j < H; ++j) {
      e = Vt::fma(Xm[i * H + j], dv[j], e);
      f = Vt::fma(Xp[i * H + j], sv[j], f);
    }
    if (Q & 1) f = Vt::fma(TR ? D[M * Q + i] : D[i * Q + M], v[M], f);
    y[i] = Vt::add(e, f);
    y[Q - 1 - i] = vsub(e, f);
  }
  if (Q & 1) {  // middle row: only the antisymmetric part of v contributes
    V m = Vt::zero();
#pragma unroll
    for (int j = 0; j < H; ++j) m = Vt::fma(TR ? D[j * Q + M] : D[M * Q + j], dv[j], m);
    y[M] = m;
  }
}

}  // namespace spx
