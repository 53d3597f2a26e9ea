// Arithmetic throughput probe of the GPU the library runs on (a measurement
// tool of the benchmark, not part of the operator library; built into its own
// shared object, libspx_probe.so).
//
// The FP64 operators of this library (the Helmholtz apply in FP64, the
// adjoint, FwdTrans, the sensor) are bound by the FP64 pipe rather than by
// HBM on this part, so their rooflines need a measured FP64 peak.  Each probe
// runs independent chains of one instruction kind in every thread of a grid
// that fills the GPU and reports the flops it executed and its CUDA-event
// time on the caller's stream:
//   kind 0  DFMA          (fma on double; 2 flop)
//   kind 1  DMMA m8n8k4   (mma.sync f64, 512 flop per warp instruction)
//   kind 2  DMMA m16n8k16 (mma.sync f64, 4096 flop per warp instruction)
//   kind 3  FFMA          (fmaf; 2 flop)
//   kind 4  FFMA2         (packed f32x2 fma; 4 flop)
//   kind 5  DFMA and DMMA m8n8k4 in alternate warps: whether the two kinds
//           share one FP64 unit.  If they do, the mixed kernel takes about
//           as long as its two halves at the rates of kinds 0 and 1 added;
//           with separate units, about as long as the slower half.
// Every chain converges to a bounded fixed point (no overflow, no
// subnormals), and the results feed a store guarded by a comparison the
// compiler cannot decide, so no work is removed.
#include <cuda_runtime.h>

#include <cstdint>

namespace {

constexpr int kThreads = 256;
constexpr int kUnroll = 16;

// `never` is a run-time value no chain reaches (the caller passes -1); the
// compiler cannot prove the store dead, so the chains are kept.
__device__ __forceinline__ void keep(double s, double* out, double never) {
  if (s == never) out[0] = s;
}

template <int CH>
__global__ void __launch_bounds__(kThreads) dfma_loop(double* out, int iters, double b, double c, double never) {
  double a[CH];
#pragma unroll
  for (int k = 0; k < CH; ++k) a[k] = 1e-3 * threadIdx.x + k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int k = 0; k < CH; ++k) a[k] = fma(a[k], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < CH; ++k) s += a[k];
  keep(s, out, never);
}

template <int CH>
__global__ void __launch_bounds__(kThreads) ffma_loop(double* out, int iters, float b, float c, double never) {
  float a[CH];
#pragma unroll
  for (int k = 0; k < CH; ++k) a[k] = 1e-3f * threadIdx.x + k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int k = 0; k < CH; ++k) a[k] = fmaf(a[k], b, c);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < CH; ++k) s += a[k];
  keep(s, out, never);
}

template <int CH>
__global__ void __launch_bounds__(kThreads) ffma2_loop(double* out, int iters, float b, float c, double never) {
  float2 a[CH];
  const float2 bb = make_float2(b, b), cc = make_float2(c, c);
#pragma unroll
  for (int k = 0; k < CH; ++k) a[k] = make_float2(1e-3f * threadIdx.x + k, 2e-3f * threadIdx.x - k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int k = 0; k < CH; ++k) a[k] = __ffma2_rn(a[k], bb, cc);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < CH; ++k) s += a[k].x + a[k].y;
  keep(s, out, never);
}

// D = A B + C on 8x8x4 (f64); per thread A, B one value each, C/D two.
__device__ __forceinline__ void dmma_884(double& c0, double& c1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
               : "+d"(c0), "+d"(c1)
               : "d"(a), "d"(b));
}

// D = A B + C on 16x8x16 (f64); per thread A eight values, B four, C/D four.
__device__ __forceinline__ void dmma_16816(double (&c)[4], const double (&a)[8], const double (&b)[4]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f64.f64.f64.f64 {%0, %1, %2, %3}, {%4, %5, %6, %7, %8, %9, %10, %11}, "
      "{%12, %13, %14, %15}, {%0, %1, %2, %3};"
      : "+d"(c[0]), "+d"(c[1]), "+d"(c[2]), "+d"(c[3])
      : "d"(a[0]), "d"(a[1]), "d"(a[2]), "d"(a[3]), "d"(a[4]), "d"(a[5]), "d"(a[6]), "d"(a[7]), "d"(b[0]),
        "d"(b[1]), "d"(b[2]), "d"(b[3]));
}

// The accumulators grow by at most 4 a b (resp. 16 a b) per instruction; with
// |a|, |b| <= 1e-4 they stay far from overflow for any iteration count used.
template <int CH>
__global__ void __launch_bounds__(kThreads) dmma884_loop(double* out, int iters, double a, double b, double never) {
  double c0[CH], c1[CH];
#pragma unroll
  for (int k = 0; k < CH; ++k) c0[k] = c1[k] = 0.0;
  const double av = a * (1 + (threadIdx.x & 3)), bv = b;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int k = 0; k < CH; ++k) dmma_884(c0[k], c1[k], av, bv);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < CH; ++k) s += c0[k] + c1[k];
  keep(s, out, never);
}

template <int CH>
__global__ void __launch_bounds__(kThreads) dmma16816_loop(double* out, int iters, double a, double b, double never) {
  double c[CH][4], av[8], bv[4];
#pragma unroll
  for (int k = 0; k < CH; ++k)
#pragma unroll
    for (int j = 0; j < 4; ++j) c[k][j] = 0.0;
#pragma unroll
  for (int j = 0; j < 8; ++j) av[j] = a * (1 + ((threadIdx.x + j) & 3));
#pragma unroll
  for (int j = 0; j < 4; ++j) bv[j] = b;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll / 4; ++u)
#pragma unroll
      for (int k = 0; k < CH; ++k) dmma_16816(c[k], av, bv);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < CH; ++k) s += c[k][0] + c[k][1] + c[k][2] + c[k][3];
  keep(s, out, never);
}

// even warps DFMA, odd warps DMMA m8n8k4, the same instruction count per warp
template <int CH>
__global__ void __launch_bounds__(kThreads) mixed_loop(double* out, int iters, double b, double c, double never) {
  const int w = threadIdx.x >> 5;
  if (w & 1) {
    double c0[CH], c1[CH];
#pragma unroll
    for (int k = 0; k < CH; ++k) c0[k] = c1[k] = 0.0;
    const double av = 1e-4 * (1 + (threadIdx.x & 3));
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int u = 0; u < kUnroll; ++u)
#pragma unroll
        for (int k = 0; k < CH; ++k) dmma_884(c0[k], c1[k], av, 1e-4);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < CH; ++k) s += c0[k] + c1[k];
    keep(s, out, never);
  } else {
    double a[CH];
#pragma unroll
    for (int k = 0; k < CH; ++k) a[k] = 1e-3 * threadIdx.x + k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int u = 0; u < kUnroll; ++u)
#pragma unroll
        for (int k = 0; k < CH; ++k) a[k] = fma(a[k], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < CH; ++k) s += a[k];
    keep(s, out, never);
  }
}

}  // namespace

extern "C" {

// Runs probe `kind` (0..5, above) with `blocks_per_sm` blocks of 256 threads
// on every SM, `iters` outer iterations, on `stream` (a cudaStream_t, NULL =
// legacy default stream), synchronising it.  Writes the flops executed and
// the kernel's CUDA-event time in milliseconds.  Returns 0, or a cudaError_t
// value, or -1 for a bad argument.
int spx_probe_rate(int kind, int blocks_per_sm, int iters, void* stream, double* flops, float* ms) {
  if (kind < 0 || kind > 5 || blocks_per_sm < 1 || blocks_per_sm > 32 || iters < 1 || !flops || !ms) return -1;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return static_cast<int>(e);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double* out = nullptr;
  if ((e = cudaMalloc(&out, sizeof(double))) != cudaSuccess) return static_cast<int>(e);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int grid = sms * blocks_per_sm;
  const double threads = double(grid) * kThreads, warps = threads / 32.0;
  constexpr int CH = 8;
  double fl = 0.0;
  cudaEventRecord(e0, st);
  switch (kind) {
    case 0:
      dfma_loop<CH><<<grid, kThreads, 0, st>>>(out, iters, 0.999999, 1e-6, -1.0);
      fl = 2.0 * threads * CH * kUnroll * iters;
      break;
    case 1:
      dmma884_loop<CH><<<grid, kThreads, 0, st>>>(out, iters, 1e-4, 1e-4, -1.0);
      fl = 512.0 * warps * CH * kUnroll * iters;
      break;
    case 2:
      dmma16816_loop<4><<<grid, kThreads, 0, st>>>(out, iters, 1e-4, 1e-4, -1.0);
      fl = 4096.0 * warps * 4 * (kUnroll / 4) * iters;
      break;
    case 3:
      ffma_loop<CH><<<grid, kThreads, 0, st>>>(out, iters, 0.999999f, 1e-6f, -1.0);
      fl = 2.0 * threads * CH * kUnroll * iters;
      break;
    case 4:
      ffma2_loop<CH><<<grid, kThreads, 0, st>>>(out, iters, 0.999999f, 1e-6f, -1.0);
      fl = 4.0 * threads * CH * kUnroll * iters;
      break;
    default:
      mixed_loop<4><<<grid, kThreads, 0, st>>>(out, iters, 0.999999, 1e-6, -1.0);
      fl = (2.0 * 32.0 + 512.0) * (warps / 2.0) * 4 * kUnroll * iters;
      break;
  }
  cudaEventRecord(e1, st);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess) return static_cast<int>(e);
  *flops = fl;
  *ms = t;
  return 0;
}

}  // extern "C"
