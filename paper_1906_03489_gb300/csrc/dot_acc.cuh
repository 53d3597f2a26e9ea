// Per-thread accumulation of dot products and sums at FP64 accuracy (shared
// by the solver's vector kernels and the integral reduction).
#pragma once
#include <cuda_runtime.h>

namespace spx {

// Per-thread partial sums of the dot products.  FP64 vectors: plain FP64.
// FP32 vectors: an unevaluated float pair hi + lo (double-float) that keeps
// FP64-level accuracy without FP64 instructions (an FP32 -> FP64 conversion
// and a DFMA per term would run on the FP64 pipe, 1/64 of the FP32 rate on
// this part, and bound the kernels).  Each product a b is split exactly into
// p + e (p = fl(a b), e = fma(a, b, -p)); p is added to hi by Knuth's TwoSum,
// which also yields the exact rounding error of that addition; both errors go
// into lo.  The pair's relative error is about (terms) x 2^-48.  The partial
// sums are then reduced across threads in FP64 (grid_reduce2).
template <typename T>
struct DotAcc {
  double s = 0.0;
  __device__ __forceinline__ void add(T a, T b) { s = fma(static_cast<double>(a), static_cast<double>(b), s); }
  __device__ __forceinline__ double value() const { return s; }
};
template <>
struct DotAcc<float> {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float a, float b) {
    const float p = __fmul_rn(a, b);
    const float e = __fmaf_rn(a, b, -p);
    const float t = __fadd_rn(hi, p);
    const float bp = __fsub_rn(t, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bp)), __fsub_rn(p, bp));
    hi = t;
    lo = __fadd_rn(lo, __fadd_rn(err, e));
  }
  __device__ __forceinline__ double value() const { return static_cast<double>(hi) + static_cast<double>(lo); }
};

}  // namespace spx
