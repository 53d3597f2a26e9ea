// C0 assembly and the Jacobi-preconditioned conjugate-gradient solve of the
// assembled Helmholtz system A x = f, A = sum_e R_e^T H_e R_e (§2.1:
// implicit-type methods lead to a linear system; assembly sums neighbouring
// elemental contributions for C0 continuity).
//
// Everything runs on the device:
//  * the transpose of the local-to-global map (CSR: for every global index
//    the local indices that map to it, in increasing order) is built once per
//    solve, so assembly is a deterministic gather-sum (no atomics on values);
//  * the Jacobi diagonal is the assembled diagonal of the elemental matrices;
//  * each PCG iteration is gather -> elemental Helmholtz -> assembly (+ <p,Ap>)
//    -> update (+ <r,z>, <r,r>) -> direction update; dot products accumulate
//    in FP64 in fixed order (per-block partials summed by the last block), so
//    results are bitwise reproducible;
//  * iterations are captured once per solve in a CUDA graph of `check_every`
//    iterations and replayed until the device-side `done` flag is set (the
//    Helmholtz launches of iterations past that point return at once);
//  * precision 1: FP32 PCG on the correction equation inside FP64 iterative
//    refinement (outer residual, its norm and x += d in FP64), restarted from
//    the new residual after every refinement step;
//  * precision 2: the same FP32 PCG with reliable updates: after each
//    refinement step its recurrence residual is replaced by the new FP64
//    residual and the run continues along its current search direction
//    instead of restarting (residual replacement, Sleijpen & van der Vorst
//    1996; its mixed-precision use by Clark et al. 2010).
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <cuda.h>

#include "dot_acc.cuh"
#include "spx_internal.h"

namespace spx {
namespace {

constexpr int kRedThreads = 256;

struct Scalars {
  double rz, rz_new, rz_prev, pAp, alpha, beta, rr, ff, tol2, scale;
  int it, done, maxit, nonfinite;
  unsigned int ticket;
};

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Grid reduction of two values in a fixed order (bitwise reproducible for a
// given grid): warp shuffles, per-warp sums in warp order, per-block partials
// partials[2 * blockIdx.x + k]; the last block to finish (ticket) then sums
// all partials with all its threads (thread t takes partials t, t + blockDim,
// ... in order, then the same warp / block pattern).  Returns true in thread 0
// of the last block, with the totals in *ta, *tb.
__device__ bool grid_reduce2(double a, double b, double* partials, unsigned int* ticket, double* ta, double* tb) {
  __shared__ double sa[kRedThreads / 32], sb[kRedThreads / 32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  a = warp_sum(a);
  b = warp_sum(b);
  if (lane == 0) {
    sa[w] = a;
    sb[w] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double x = 0.0, y = 0.0;
    for (int i = 0; i < nw; ++i) {
      x += sa[i];
      y += sb[i];
    }
    partials[2 * blockIdx.x] = x;
    partials[2 * blockIdx.x + 1] = y;
    __threadfence();
    const unsigned t = atomicAdd(ticket, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return false;   // uniform across the block
  __threadfence();
  double x = 0.0, y = 0.0;
  for (int i = threadIdx.x; i < static_cast<int>(gridDim.x); i += blockDim.x) {
    x += static_cast<volatile const double*>(partials)[2 * i];
    y += static_cast<volatile const double*>(partials)[2 * i + 1];
  }
  x = warp_sum(x);
  y = warp_sum(y);
  __syncthreads();
  if (lane == 0) {
    sa[w] = x;
    sb[w] = y;
  }
  __syncthreads();
  if (threadIdx.x != 0) return false;
  x = 0.0;
  y = 0.0;
  for (int i = 0; i < nw; ++i) {
    x += sa[i];
    y += sb[i];
  }
  *ta = x;
  *tb = y;
  return true;
}

// ---- CSR transpose of l2g ------------------------------------------------
__global__ void csr_count(const int32_t* l2g, int64_t nl, int32_t* cnt) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < nl; i += int64_t(gridDim.x) * blockDim.x)
    atomicAdd(&cnt[l2g[i]], 1);
}

__global__ void check_l2g(const int32_t* l2g, int64_t nl, int64_t ng, int* bad) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < nl; i += int64_t(gridDim.x) * blockDim.x)
    if (l2g[i] < 0 || l2g[i] >= ng) atomicOr(bad, 1);
}

// exclusive scan, pass 1: per-chunk scan, chunk totals
constexpr int kScanChunk = 1024;
__global__ void scan_chunks(const int32_t* in, int32_t* out, int64_t n, int32_t* totals) {
  __shared__ int32_t s[kScanChunk];
  const int64_t base = int64_t(blockIdx.x) * kScanChunk;
  const int t = threadIdx.x;  // blockDim = kScanChunk
  s[t] = base + t < n ? in[base + t] : 0;
  __syncthreads();
  for (int o = 1; o < kScanChunk; o <<= 1) {
    int32_t v = t >= o ? s[t - o] : 0;
    __syncthreads();
    s[t] += v;
    __syncthreads();
  }
  if (base + t < n) out[base + t] = s[t] - (base + t < n ? in[base + t] : 0);
  if (t == kScanChunk - 1) totals[blockIdx.x] = s[t];
}

// pass 2 (one block): exclusive scan of chunk totals, written in place
__global__ void scan_totals(int32_t* totals, int nchunks, int32_t* grand) {
  if (threadIdx.x != 0) return;
  int32_t run = 0;
  for (int i = 0; i < nchunks; ++i) {
    const int32_t v = totals[i];
    totals[i] = run;
    run += v;
  }
  *grand = run;
}

__global__ void scan_add(int32_t* out, int64_t n, const int32_t* totals) {
  const int64_t i = int64_t(blockIdx.x) * kScanChunk + threadIdx.x;
  if (i < n) out[i] += totals[blockIdx.x];
}

__global__ void csr_fill(const int32_t* l2g, int64_t nl, const int32_t* row_ptr, int32_t* cursor, int32_t* cols) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < nl; i += int64_t(gridDim.x) * blockDim.x) {
    const int32_t g = l2g[i];
    const int32_t k = atomicAdd(&cursor[g], 1);
    cols[row_ptr[g] + k] = static_cast<int32_t>(i);
  }
}

__global__ void csr_sort(const int32_t* row_ptr, int32_t* cols, int64_t ng) {
  for (int64_t g = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; g < ng; g += int64_t(gridDim.x) * blockDim.x) {
    const int32_t a = row_ptr[g], b = row_ptr[g + 1];
    for (int32_t i = a + 1; i < b; ++i) {
      const int32_t v = cols[i];
      int32_t j = i - 1;
      while (j >= a && cols[j] > v) {
        cols[j + 1] = cols[j];
        --j;
      }
      cols[j + 1] = v;
    }
  }
}

// ---- assembly and vector kernels ----------------------------------------
// Global vectors are processed in packs of V = 16 / sizeof(T) consecutive
// values (one 16-byte access per vector and pack) when every pointer of the
// launch is 16-byte aligned, else one value at a time (V = 1).  The values
// past the last whole pack are handled one by one after the pack loop.
template <typename T, int V>
struct Pack {
  T v[V];
};

template <typename T, int V>
__device__ __forceinline__ Pack<T, V> ldp(const T* __restrict__ a, int64_t i) {
  Pack<T, V> r;
  if constexpr (V == 1) {
    r.v[0] = a[i];
  } else if constexpr (sizeof(T) == 4) {
    static_assert(V == 4, "FP32 packs hold 4 values");
    const float4 x = reinterpret_cast<const float4*>(a)[i];
    r.v[0] = x.x; r.v[1] = x.y; r.v[2] = x.z; r.v[3] = x.w;
  } else {
    static_assert(V == 2, "FP64 packs hold 2 values");
    const double2 x = reinterpret_cast<const double2*>(a)[i];
    r.v[0] = x.x; r.v[1] = x.y;
  }
  return r;
}

template <typename T, int V>
__device__ __forceinline__ void stp(T* __restrict__ a, int64_t i, const Pack<T, V>& r) {
  if constexpr (V == 1) {
    a[i] = r.v[0];
  } else if constexpr (sizeof(T) == 4) {
    reinterpret_cast<float4*>(a)[i] = make_float4(r.v[0], r.v[1], r.v[2], r.v[3]);
  } else {
    reinterpret_cast<double2*>(a)[i] = make_double2(r.v[0], r.v[1]);
  }
}

template <typename T>
__global__ void assemble_plain(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ cols,
                               const T* __restrict__ yl, T* __restrict__ yg, int64_t ng) {
  for (int64_t g = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; g < ng; g += int64_t(gridDim.x) * blockDim.x) {
    T s = T(0);
    for (int32_t k = row_ptr[g]; k < row_ptr[g + 1]; ++k) s += yl[cols[k]];
    yg[g] = s;
  }
}

// Programmatic dependent launch (sm_90+): the iteration's vector kernels are
// launched with programmatic stream serialisation, so a kernel's blocks may be
// scheduled while its predecessor drains.  Each of them first waits for the
// predecessor grid to complete with its memory visible (griddep_wait: a no-op
// without a programmatic predecessor), and lets its own successor launch once
// its main loop is done (griddep_launch).
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// loc = g[l2g] (skipped once the solve is done).  One entry per thread and
// trip: the lanes of a warp read consecutive l2g entries, whose global
// indices run in short consecutive stretches (the modes of an element row).
template <typename T>
__global__ void gather_if(const int32_t* __restrict__ l2g, const T* __restrict__ g, T* __restrict__ loc, int64_t n,
                          const Scalars* sc) {
  griddep_wait();
  if (sc->done) return;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    loc[i] = g[l2g[i]];
}

// q = assemble(ql); pAp = <p, q>; alpha = rz / pAp.  A thread sums the rows
// g, g + S, ... (S = all threads), kRowsA of them in lockstep, each row in CSR
// order; the lanes of a warp take consecutive rows.
constexpr int kRowsA = 4;
template <typename T>
__global__ void __launch_bounds__(kRedThreads) assemble_dot(const int32_t* __restrict__ row_ptr,
                                                            const int32_t* __restrict__ cols,
                                                            const T* __restrict__ ql, T* __restrict__ q,
                                                            const T* __restrict__ p, int64_t ng, Scalars* sc,
                                                            double* partials) {
  griddep_wait();
  if (sc->done) return;
  DotAcc<T> acc;
  const int64_t S = int64_t(gridDim.x) * blockDim.x;
  for (int64_t g0 = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; g0 < ng; g0 += kRowsA * S) {
    int32_t k0[kRowsA], k1[kRowsA];
    T pv[kRowsA], sv[kRowsA];
    int len = 0;
#pragma unroll
    for (int u = 0; u < kRowsA; ++u) {
      const int64_t g = g0 + u * S;
      k0[u] = k1[u] = 0;
      pv[u] = T(0);
      sv[u] = T(0);
      if (g < ng) {
        k0[u] = row_ptr[g];
        k1[u] = row_ptr[g + 1];
        pv[u] = p[g];
      }
      len = max(len, k1[u] - k0[u]);
    }
    for (int j = 0; j < len; ++j) {
#pragma unroll
      for (int u = 0; u < kRowsA; ++u)
        if (k0[u] + j < k1[u]) sv[u] += ql[cols[k0[u] + j]];
    }
#pragma unroll
    for (int u = 0; u < kRowsA; ++u) {
      const int64_t g = g0 + u * S;
      if (g < ng) {
        q[g] = sv[u];
        acc.add(pv[u], sv[u]);
      }
    }
  }
  griddep_launch();
  double pAp, unused;
  if (grid_reduce2(acc.value(), 0.0, partials, &sc->ticket, &pAp, &unused)) {
    sc->pAp = pAp;
    sc->alpha = sc->rz / pAp;
    sc->ticket = 0;
  }
}

// x += alpha p; r -= alpha q; z = minv r; rz_new = <r,z>; rr = <r,r>.
// Ends the run (done) on convergence of the recurrence residual
// (rr <= tol2 ff), the iteration cap or a non-finite value.
template <typename T, int V>
__global__ void __launch_bounds__(kRedThreads) cg_update(T* __restrict__ x, T* __restrict__ r, T* __restrict__ z,
                                                         const T* __restrict__ p, const T* __restrict__ q,
                                                         const T* __restrict__ minv, int64_t ng, Scalars* sc,
                                                         double* partials) {
  griddep_wait();
  if (sc->done) return;
  constexpr int U = V == 1 ? 4 : 1;   // packs per trip (loads in flight per thread)
  const T alpha = static_cast<T>(sc->alpha);
  DotAcc<T> arz, arr;
  const int64_t S = int64_t(gridDim.x) * blockDim.x, t0 = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  const int64_t np = ng / V;
  for (int64_t i0 = t0; i0 < np; i0 += U * S) {
    Pack<T, V> xv[U], rv[U], pv[U], qv[U], mv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = i0 + u * S;
      if (i < np) {
        xv[u] = ldp<T, V>(x, i);
        rv[u] = ldp<T, V>(r, i);
        pv[u] = ldp<T, V>(p, i);
        qv[u] = ldp<T, V>(q, i);
        mv[u] = ldp<T, V>(minv, i);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = i0 + u * S;
      if (i < np) {
        Pack<T, V> zv;
#pragma unroll
        for (int c = 0; c < V; ++c) {
          xv[u].v[c] = xv[u].v[c] + alpha * pv[u].v[c];
          const T rn = rv[u].v[c] - alpha * qv[u].v[c];
          rv[u].v[c] = rn;
          zv.v[c] = mv[u].v[c] * rn;
          arz.add(rn, zv.v[c]);
          arr.add(rn, rn);
        }
        stp<T, V>(x, i, xv[u]);
        stp<T, V>(r, i, rv[u]);
        stp<T, V>(z, i, zv);
      }
    }
  }
  for (int64_t g = np * V + t0; g < ng; g += S) {
    x[g] = x[g] + alpha * p[g];
    const T rn = r[g] - alpha * q[g];
    r[g] = rn;
    const T zv = minv[g] * rn;
    z[g] = zv;
    arz.add(rn, zv);
    arr.add(rn, rn);
  }
  griddep_launch();
  double rz, rr;
  if (grid_reduce2(arz.value(), arr.value(), partials, &sc->ticket, &rz, &rr)) {
    sc->rz_new = rz;
    sc->beta = rz / sc->rz;
    sc->rz_prev = sc->rz;
    sc->rz = rz;
    sc->rr = rr;
    sc->it += 1;
    if (!isfinite(rr) || !isfinite(rz)) {
      sc->nonfinite = 1;
      sc->done = 1;
    } else if (rr <= sc->tol2 * sc->ff || sc->it >= sc->maxit) {
      sc->done = 1;
    }
    sc->ticket = 0;
  }
}

// p = z + beta p
template <typename T, int V>
__global__ void cg_direction(T* __restrict__ p, const T* __restrict__ z, int64_t ng, const Scalars* sc) {
  griddep_wait();
  if (sc->done) return;
  const T beta = static_cast<T>(sc->beta);
  const int64_t S = int64_t(gridDim.x) * blockDim.x, t0 = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  const int64_t np = ng / V;
  for (int64_t i = t0; i < np; i += S) {
    Pack<T, V> pv = ldp<T, V>(p, i);
    const Pack<T, V> zv = ldp<T, V>(z, i);
#pragma unroll
    for (int c = 0; c < V; ++c) pv.v[c] = zv.v[c] + beta * pv.v[c];
    stp<T, V>(p, i, pv);
  }
  for (int64_t g = np * V + t0; g < ng; g += S) p[g] = z[g] + beta * p[g];
}

// Start of a PCG run from residual r (x not touched): z = minv r; p = z;
// rz = <r,z>; it = 0; done unless there is work (rr > tol2 ff, maxit > 0).
template <typename T, int V>
__global__ void __launch_bounds__(kRedThreads) cg_start(const T* __restrict__ r, T* __restrict__ z,
                                                        T* __restrict__ p, const T* __restrict__ minv, int64_t ng,
                                                        Scalars* sc, double* partials) {
  DotAcc<T> arz, arr;
  const int64_t S = int64_t(gridDim.x) * blockDim.x, t0 = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  const int64_t np = ng / V;
  for (int64_t i = t0; i < np; i += S) {
    const Pack<T, V> rv = ldp<T, V>(r, i), mv = ldp<T, V>(minv, i);
    Pack<T, V> zv;
#pragma unroll
    for (int c = 0; c < V; ++c) {
      zv.v[c] = mv.v[c] * rv.v[c];
      arz.add(rv.v[c], zv.v[c]);
      arr.add(rv.v[c], rv.v[c]);
    }
    stp<T, V>(z, i, zv);
    stp<T, V>(p, i, zv);
  }
  for (int64_t g = np * V + t0; g < ng; g += S) {
    const T rv = r[g], zv = minv[g] * rv;
    z[g] = zv;
    p[g] = zv;
    arz.add(rv, zv);
    arr.add(rv, rv);
  }
  double rz, rr;
  if (grid_reduce2(arz.value(), arr.value(), partials, &sc->ticket, &rz, &rr)) {
    sc->rz = rz;
    sc->rr = rr;
    sc->it = 0;
    sc->nonfinite = (!isfinite(rr) || !isfinite(rz)) ? 1 : 0;
    sc->done = (sc->nonfinite || rr <= sc->tol2 * sc->ff || sc->maxit <= 0) ? 1 : 0;
    sc->ticket = 0;
  }
}

// r = f - y (FP64; y = nullptr: y = 0); rr = <r,r>; ff = <f,f>
__global__ void __launch_bounds__(kRedThreads) residual64(const double* __restrict__ f, const double* __restrict__ y,
                                                          double* __restrict__ r, int64_t ng, Scalars* sc,
                                                          double* partials) {
  double arr = 0.0, aff = 0.0;
  for (int64_t g = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; g < ng; g += int64_t(gridDim.x) * blockDim.x) {
    const double rv = y ? f[g] - y[g] : f[g];
    r[g] = rv;
    arr += rv * rv;
    aff += f[g] * f[g];
  }
  double rr, ff;
  if (grid_reduce2(arr, aff, partials, &sc->ticket, &rr, &ff)) {
    sc->rr = rr;
    sc->ff = ff;
    sc->ticket = 0;
  }
}

// scale = <x, x> (FP64): tells whether the initial guess is zero
__global__ void __launch_bounds__(kRedThreads) sumsq64(const double* __restrict__ x, int64_t ng, Scalars* sc,
                                                       double* partials) {
  double a = 0.0;
  for (int64_t g = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; g < ng; g += int64_t(gridDim.x) * blockDim.x)
    a += x[g] * x[g];
  double xx, unused;
  if (grid_reduce2(a, 0.0, partials, &sc->ticket, &xx, &unused)) {
    sc->scale = xx;
    sc->ticket = 0;
  }
}

// r32 = r64 * s, d32 = 0
__global__ void to_f32_scaled(const double* __restrict__ r, float* __restrict__ r32, float* __restrict__ d32,
                              int64_t ng, const Scalars* sc) {
  const double s = 1.0 / sqrt(sc->rr);
  for (int64_t g = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; g < ng; g += int64_t(gridDim.x) * blockDim.x) {
    r32[g] = static_cast<float>(r[g] * s);
    d32[g] = 0.f;
  }
}

// Residual replacement of a reliable update (precision 2).  The FP32 run
// stopped after the update of iteration i (its direction update not done);
// the FP64 residual r64 of the corrected x replaces the recurrence residual,
// rescaled so that ||r32|| = 1: r32 = r64 / s_new, d32 = 0, z32 = minv r32,
// rz = <r32, z32>.  Rescaling multiplies every vector of the old scaled system
// by c = s_old / s_new, so the direction update that follows,
// p = z32 + beta' p, takes beta' = c * rz / (c^2 rz_prev) (rz_prev = <r_i, z_i>
// of the old scaling).  The run then continues with tol2 / ff / maxit as set
// by the host beforehand.
__global__ void __launch_bounds__(kRedThreads) reliable_restart(const double* __restrict__ r64,
                                                                float* __restrict__ r32, float* __restrict__ d32,
                                                                float* __restrict__ z32,
                                                                const float* __restrict__ minv, int64_t ng,
                                                                double inv_s_new, double c, Scalars* sc,
                                                                double* partials) {
  DotAcc<float> arz, arr;
  for (int64_t g = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; g < ng; g += int64_t(gridDim.x) * blockDim.x) {
    const float rv = static_cast<float>(r64[g] * inv_s_new);
    const float zv = minv[g] * rv;
    r32[g] = rv;
    d32[g] = 0.f;
    z32[g] = zv;
    arz.add(rv, zv);
    arr.add(rv, rv);
  }
  double rz, rr;
  if (grid_reduce2(arz.value(), arr.value(), partials, &sc->ticket, &rz, &rr)) {
    sc->beta = rz / (c * sc->rz_prev);
    sc->rz = rz;
    sc->rr = rr;
    sc->nonfinite = (!isfinite(rr) || !isfinite(rz) || !isfinite(sc->beta)) ? 1 : 0;
    sc->done = (sc->nonfinite || sc->it >= sc->maxit) ? 1 : 0;
    sc->ticket = 0;
  }
}

// x += scale d32
__global__ void add_correction(double* __restrict__ x, const float* __restrict__ d32, int64_t ng, double scale) {
  for (int64_t g = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; g < ng; g += int64_t(gridDim.x) * blockDim.x)
    x[g] += scale * static_cast<double>(d32[g]);
}

template <typename T>
__global__ void invert_diag(const double* __restrict__ dg, T* __restrict__ minv, int64_t ng) {
  for (int64_t g = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; g < ng; g += int64_t(gridDim.x) * blockDim.x)
    minv[g] = static_cast<T>(1.0 / dg[g]);
}

template <typename T>
__global__ void fill_zero(T* v, int64_t n) {
  for (int64_t g = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; g < n; g += int64_t(gridDim.x) * blockDim.x)
    v[g] = T(0);
}
// ---------------------------------------------------------------------------
struct Workspace {
  int32_t *row_ptr, *cols, *cursor, *totals, *grand;
  int* bad;
  Scalars* sc;
  double* partials;
  double *r64, *z64, *p64, *q64, *minv64, *pl64, *ql64, *diag64;
  float *r32, *z32, *p32, *q32, *d32, *minv32, *pl32, *ql32;
  size_t bytes;
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

Workspace carve(char* base, int64_t ng, int64_t nl, int nred, int precision) {
  Workspace w{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* p = base ? base + off : nullptr;
    off += align256(bytes);
    return p;
  };
  const int64_t nchunks = (ng + 1 + kScanChunk - 1) / kScanChunk;
  w.row_ptr = reinterpret_cast<int32_t*>(take((ng + 1) * 4));
  w.cols = reinterpret_cast<int32_t*>(take(nl * 4));
  w.cursor = reinterpret_cast<int32_t*>(take((ng + 1) * 4));
  w.totals = reinterpret_cast<int32_t*>(take(nchunks * 4));
  w.grand = reinterpret_cast<int32_t*>(take(16));
  w.bad = reinterpret_cast<int*>(take(16));
  w.sc = reinterpret_cast<Scalars*>(take(sizeof(Scalars)));
  w.partials = reinterpret_cast<double*>(take(2 * nred * sizeof(double)));
  w.diag64 = reinterpret_cast<double*>(take(nl * 8));   // local diagonal, then global diagonal
  w.r64 = reinterpret_cast<double*>(take(ng * 8));
  w.minv64 = reinterpret_cast<double*>(take(ng * 8));
  w.pl64 = reinterpret_cast<double*>(take(nl * 8));
  w.ql64 = reinterpret_cast<double*>(take(nl * 8));
  w.q64 = reinterpret_cast<double*>(take(ng * 8));
  if (precision == 0) {
    w.z64 = reinterpret_cast<double*>(take(ng * 8));
    w.p64 = reinterpret_cast<double*>(take(ng * 8));
  } else {
    w.r32 = reinterpret_cast<float*>(take(ng * 4));
    w.z32 = reinterpret_cast<float*>(take(ng * 4));
    w.p32 = reinterpret_cast<float*>(take(ng * 4));
    w.q32 = reinterpret_cast<float*>(take(ng * 4));
    w.d32 = reinterpret_cast<float*>(take(ng * 4));
    w.minv32 = reinterpret_cast<float*>(take(ng * 4));
    w.pl32 = reinterpret_cast<float*>(take(nl * 4));
    w.ql32 = reinterpret_cast<float*>(take(nl * 4));
  }
  w.bytes = off;
  return w;
}

struct Solver {
  const spx_plan* plan;
  const int32_t* l2g;
  int64_t ng, nl;
  cudaStream_t st;
  int grid_v;    // grid of element-wise kernels
  int nred;      // upper bound of the reduction kernels' grids (partials buffer)
  int grid_dir;  // grid of the direction update
  Workspace w;
  double lam;
};

#define SPX_CK(expr)                                          \
  do {                                                        \
    cudaError_t e_ = (expr);                                  \
    if (e_ != cudaSuccess) return cuda_fail(e_, #expr);       \
  } while (0)

// Grid of a reduction kernel: one wave, every block resident at once (SMs x
// the kernel's occupancy, at most s.nred).  It is a property of the compiled
// kernel and the GPU, so each kernel's grid, and with it the order of every
// sum, is the same at every launch.
template <class K>
int one_wave(const Solver& s, K kern) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kRedThreads, 0) != cudaSuccess || nb < 1) nb = 1;
  return std::min(s.nred, s.plan->num_sms * nb);
}

spx_status build_csr(Solver& s) {
  Workspace& w = s.w;
  SPX_CK(cudaMemsetAsync(w.cursor, 0, (s.ng + 1) * 4, s.st));
  SPX_CK(cudaMemsetAsync(w.bad, 0, 4, s.st));
  check_l2g<<<s.grid_v, 256, 0, s.st>>>(s.l2g, s.nl, s.ng, w.bad);
  int bad = 0;
  SPX_CK(cudaMemcpyAsync(&bad, w.bad, 4, cudaMemcpyDeviceToHost, s.st));
  SPX_CK(cudaStreamSynchronize(s.st));
  if (bad) return fail(SPX_ERR_INVALID_ARG, "cg_solve: l2g has an entry outside [0, n_global)");
  csr_count<<<s.grid_v, 256, 0, s.st>>>(s.l2g, s.nl, w.cursor);
  const int64_t n = s.ng + 1;
  const int nchunks = static_cast<int>((n + kScanChunk - 1) / kScanChunk);
  scan_chunks<<<nchunks, kScanChunk, 0, s.st>>>(w.cursor, w.row_ptr, n, w.totals);
  scan_totals<<<1, 32, 0, s.st>>>(w.totals, nchunks, w.grand);
  scan_add<<<nchunks, kScanChunk, 0, s.st>>>(w.row_ptr, n, w.totals);
  SPX_CK(cudaMemsetAsync(w.cursor, 0, (s.ng + 1) * 4, s.st));
  csr_fill<<<s.grid_v, 256, 0, s.st>>>(s.l2g, s.nl, w.row_ptr, w.cursor, w.cols);
  csr_sort<<<s.grid_v, 256, 0, s.st>>>(w.row_ptr, w.cols, s.ng);
  SPX_CK(cudaGetLastError());
  return SPX_OK;
}

bool a16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

// Launch with programmatic stream serialisation (see griddep_wait).
template <typename... KArgs, typename... Args>
void pdl_launch(void (*kern)(KArgs...), int grid, int block, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// y_global = A x_global in precision T (using pl / ql local buffers)
template <typename T>
spx_status apply_A(Solver& s, int dt, const T* xg, T* pl, T* ql, T* yg) {
  spx_status st = spx_gather(s.plan, static_cast<spx_dtype>(dt), s.l2g, s.ng, xg, pl, s.st);
  if (st != SPX_OK) return st;
  st = helmholtz_unless(s.plan, dt, s.lam, pl, ql, nullptr, s.st);
  if (st != SPX_OK) return st;
  assemble_plain<T><<<s.grid_v, 256, 0, s.st>>>(s.w.row_ptr, s.w.cols, ql, yg, s.ng);
  SPX_CK(cudaGetLastError());
  return SPX_OK;
}

// The vectors and launches of one PCG run in precision T: x += alpha p,
// r -= alpha A p, z = minv r, p = z + beta p.  One iteration is gather ->
// Helmholtz (skipped once the run is done) -> assembly + <p, Ap> -> update +
// <r, z>, <r, r> -> direction.  With use_graph, `check_every` iterations are
// captured once in a CUDA graph that every chunk of the run replays (the
// buffers never change); else they are launched eagerly.
template <typename T>
struct PcgRun {
  static constexpr int V = 16 / sizeof(T);
  Solver* s;
  int dt;
  T *x, *r, *z, *p, *q;
  const T* minv;
  T *pl, *ql;
  int check_every = 1;
  cudaGraphExec_t exec = nullptr;

  ~PcgRun() {
    if (exec) cudaGraphExecDestroy(exec);
  }

  spx_status enqueue_iteration() {
    Workspace& w = s->w;
    cudaStream_t st = s->st;
    pdl_launch(gather_if<T>, s->grid_v, 256, st, s->l2g, p, pl, s->nl, w.sc);
    spx_status e = helmholtz_unless(s->plan, dt, s->lam, pl, ql, &w.sc->done, st);
    if (e != SPX_OK) return e;
    pdl_launch(assemble_dot<T>, one_wave(*s, assemble_dot<T>), kRedThreads, st, w.row_ptr, w.cols, ql, q, p, s->ng,
               w.sc, w.partials);
    if (a16(x) && a16(r) && a16(z) && a16(p) && a16(q) && a16(minv))
      pdl_launch(cg_update<T, V>, one_wave(*s, cg_update<T, V>), kRedThreads, st, x, r, z, p, q, minv, s->ng, w.sc,
                 w.partials);
    else
      pdl_launch(cg_update<T, 1>, one_wave(*s, cg_update<T, 1>), kRedThreads, st, x, r, z, p, q, minv, s->ng, w.sc,
                 w.partials);
    direction();
    SPX_CK(cudaGetLastError());
    return SPX_OK;
  }

  void direction() {
    if (a16(p) && a16(z)) pdl_launch(cg_direction<T, V>, s->grid_dir, 256, s->st, p, static_cast<const T*>(z), s->ng,
                                     static_cast<const Scalars*>(s->w.sc));
    else pdl_launch(cg_direction<T, 1>, s->grid_dir, 256, s->st, p, static_cast<const T*>(z), s->ng,
                    static_cast<const Scalars*>(s->w.sc));
  }

  // z = minv r; p = z; rz (scalars ff / tol2 / maxit set by the caller)
  spx_status start() {
    Workspace& w = s->w;
    if (a16(r) && a16(z) && a16(p) && a16(minv))
      cg_start<T, V><<<one_wave(*s, cg_start<T, V>), kRedThreads, 0, s->st>>>(r, z, p, minv, s->ng, w.sc,
                                                                                w.partials);
    else
      cg_start<T, 1><<<one_wave(*s, cg_start<T, 1>), kRedThreads, 0, s->st>>>(r, z, p, minv, s->ng, w.sc,
                                                                                w.partials);
    SPX_CK(cudaGetLastError());
    return SPX_OK;
  }

  spx_status prepare(bool use_graph, int every) {
    check_every = every;
    // one eager apply first, so that every launch attribute of the operator
    // kernel is set before any stream capture
    spx_status e = helmholtz_unless(s->plan, dt, s->lam, pl, ql, nullptr, s->st);
    if (e != SPX_OK || !use_graph) return e;
    cudaGraph_t graph;
    SPX_CK(cudaStreamBeginCapture(s->st, cudaStreamCaptureModeThreadLocal));
    for (int k = 0; k < check_every && e == SPX_OK; ++k) e = enqueue_iteration();
    cudaError_t ce = cudaStreamEndCapture(s->st, &graph);
    if (e != SPX_OK) return e;
    SPX_CK(ce);
    ce = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    SPX_CK(ce);
    return SPX_OK;
  }

  // Iterates until the device sets `done`; the final scalars land in *h.
  spx_status run(Scalars* h) {
    for (;;) {
      if (exec) {
        SPX_CK(cudaGraphLaunch(exec, s->st));
      } else {
        for (int k = 0; k < check_every; ++k) {
          spx_status e = enqueue_iteration();
          if (e != SPX_OK) return e;
        }
      }
      SPX_CK(cudaMemcpyAsync(h, s->w.sc, sizeof(Scalars), cudaMemcpyDeviceToHost, s->st));
      SPX_CK(cudaStreamSynchronize(s->st));
      if (h->done) return SPX_OK;
    }
  }
};

spx_status set_scalars(Solver& s, double ff, double tol, int maxit) {
  Scalars h{};
  h.ff = ff;
  h.tol2 = tol * tol;
  h.maxit = maxit;
  SPX_CK(cudaMemcpyAsync(s.w.sc, &h, sizeof(Scalars), cudaMemcpyHostToDevice, s.st));
  SPX_CK(cudaStreamSynchronize(s.st));
  return SPX_OK;
}

spx_status read_scalars(Solver& s, Scalars* h) {
  SPX_CK(cudaMemcpyAsync(h, s.w.sc, sizeof(Scalars), cudaMemcpyDeviceToHost, s.st));
  SPX_CK(cudaStreamSynchronize(s.st));
  return SPX_OK;
}

// FP64 residual r = f - A x; returns ||r||^2 and ||f||^2 (sets rr, ff).
// x_zero: x is known to be zero, so r = f without an apply.
spx_status residual(Solver& s, const double* f, const double* x, double* rr, double* ff, bool x_zero = false) {
  Workspace& w = s.w;
  if (!x_zero) {
    spx_status st = apply_A<double>(s, SPX_F64, x, w.pl64, w.ql64, w.q64);
    if (st != SPX_OK) return st;
  }
  residual64<<<one_wave(s, residual64), kRedThreads, 0, s.st>>>(f, x_zero ? nullptr : w.q64, w.r64, s.ng, w.sc,
                                                                 w.partials);
  spx_status st;
  SPX_CK(cudaGetLastError());
  Scalars h;
  st = read_scalars(s, &h);
  if (st != SPX_OK) return st;
  *rr = h.rr;
  *ff = h.ff;
  return SPX_OK;
}

}  // namespace
}  // namespace spx

using namespace spx;

extern "C" spx_status spx_cg_workspace_bytes(const spx_plan* plan, int64_t n_global, const spx_cg_opts* o,
                                             size_t* bytes) {
  if (!plan || !o || !bytes || n_global < 0) return fail(SPX_ERR_INVALID_ARG, "cg_workspace_bytes: bad argument");
  if (o->precision < 0 || o->precision > 2) return fail(SPX_ERR_INVALID_ARG, "cg: precision must be 0, 1 or 2");
  const int nred = plan->num_sms * 8;
  *bytes = carve(nullptr, n_global, plan->n_coef, nred, o->precision).bytes;
  return SPX_OK;
}

namespace spx {
namespace {

// The solve.  own_resources = true (spx_cg_solve): the call may build the
// plan's tile lists, runs on a private stream ordered after the caller's and
// may capture its iterations in CUDA graphs.  own_resources = false
// (spx_cg_solve_noalloc): nothing is created or allocated; the work runs
// eagerly on the caller's stream and the tile lists must already exist.
spx_status cg_solve_impl(const spx_plan* plan, double lambda, const int32_t* l2g, int64_t n_global, const double* f,
                         double* x, void* workspace, size_t ws_bytes, const spx_cg_opts* o, spx_cg_result* res,
                         void* stream, bool own_resources) {
  if (!plan || !o || !res) return fail(SPX_ERR_INVALID_ARG, "cg_solve: NULL argument");
  std::memset(res, 0, sizeof(*res));
  if (plan->shape) return fail(SPX_ERR_UNSUPPORTED, "cg_solve: triangles / prisms are not supported by the solver");
  if (n_global < 0 || n_global > (int64_t(1) << 31) - 2 || plan->n_coef > (int64_t(1) << 31) - 1)
    return fail(SPX_ERR_INVALID_ARG, "cg_solve: sizes exceed the int32 index range");
  if (n_global == 0) return SPX_OK;
  if (!l2g || !f || !x || !workspace) return fail(SPX_ERR_INVALID_ARG, "cg_solve: NULL buffer");
  if (o->precision < 0 || o->precision > 2) return fail(SPX_ERR_INVALID_ARG, "cg_solve: precision must be 0, 1 or 2");
  if (!(o->tol > 0) || o->maxit < 1 || o->check_every < 1)
    return fail(SPX_ERR_INVALID_ARG, "cg_solve: tol > 0, maxit >= 1, check_every >= 1 required");
  if (o->precision >= 1 && (!(o->inner_tol > 0) || o->max_outer < 1))
    return fail(SPX_ERR_INVALID_ARG, "cg_solve: inner_tol > 0 and max_outer >= 1 required");
  if (!plan->geom[SPX_F64] || (o->precision >= 1 && !plan->geom[SPX_F32]))
    return fail(SPX_ERR_INVALID_ARG, "cg_solve: geometry not registered for the precision(s) used");
  if (reinterpret_cast<uintptr_t>(workspace) % 256) return fail(SPX_ERR_INVALID_ARG, "cg_solve: workspace not 256-byte aligned");
  Solver s{};
  s.plan = plan;
  s.l2g = l2g;
  s.ng = n_global;
  s.nl = plan->n_coef;
  s.lam = lambda;
  s.nred = plan->num_sms * 8;   // 256-thread blocks: at most 8 per SM
  {
    int nd = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nd, cg_direction<float, 4>, 256, 0) != cudaSuccess || nd < 1)
      nd = 4;
    s.grid_dir = plan->num_sms * std::min(8, nd);
  }
  s.grid_v = plan->num_sms * 8;
  s.w = carve(static_cast<char*>(workspace), n_global, plan->n_coef, s.nred, o->precision);
  if (ws_bytes < s.w.bytes) return fail(SPX_ERR_NO_MEMORY, "cg_solve: workspace smaller than cg_workspace_bytes");
  spx_plan* mp = const_cast<spx_plan*>(plan);
  spx_status st;
  cudaStream_t user = static_cast<cudaStream_t>(stream);
  cudaEvent_t ev = nullptr;
  bool use_graph = o->use_graph != 0;
  if (own_resources) {
    if ((st = ensure_tiles(mp, OP_HELM, 0)) != SPX_OK) return st;
    if ((st = ensure_tiles(mp, OP_HELM, 1)) != SPX_OK) return st;
    // private stream ordered after the caller's
    SPX_CK(cudaStreamCreateWithFlags(&s.st, cudaStreamNonBlocking));
    SPX_CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  } else {
    if (plan->tiles[OP_HELM][SPX_F64].dirty || plan->tiles[OP_DIAG][SPX_F64].dirty ||
        (o->precision >= 1 && plan->tiles[OP_HELM][SPX_F32].dirty))
      return fail(SPX_ERR_INVALID_ARG,
                  "cg_solve_noalloc: the plan's Helmholtz / diagonal launch tiles are not built yet (run "
                  "spx_helmholtz in each precision used and spx_helmholtz_diag in FP64 once on this plan, or "
                  "spx_cg_solve once, before the first allocation-free solve)");
    s.st = user;
    use_graph = false;
  }
  auto finish = [&](spx_status r) {
    if (own_resources) {
      cudaEventRecord(ev, s.st);
      cudaStreamWaitEvent(user, ev, 0);
      cudaStreamSynchronize(s.st);
      cudaEventDestroy(ev);
      cudaStreamDestroy(s.st);
    } else {
      cudaStreamSynchronize(s.st);
    }
    return r;
  };
  if (own_resources) {
    cudaEventRecord(ev, user);
    cudaStreamWaitEvent(s.st, ev, 0);
  }
  Workspace& w = s.w;
  SPX_CK(cudaMemsetAsync(w.sc, 0, sizeof(Scalars), s.st));
  if ((st = build_csr(s)) != SPX_OK) return finish(st);
  // Jacobi diagonal: assembled diag(H_e)
  if ((st = spx_helmholtz_diag(plan, SPX_F64, lambda, w.diag64, s.st)) != SPX_OK) return finish(st);
  assemble_plain<double><<<s.grid_v, 256, 0, s.st>>>(w.row_ptr, w.cols, w.diag64, w.r64, s.ng);
  if (o->precision == 0) invert_diag<double><<<s.grid_v, 256, 0, s.st>>>(w.r64, w.minv64, s.ng);
  else invert_diag<float><<<s.grid_v, 256, 0, s.st>>>(w.r64, w.minv32, s.ng);
  if (cudaGetLastError() != cudaSuccess) return finish(fail(SPX_ERR_CUDA, "cg setup kernels"));

  // initial residual; a zero initial guess needs no apply
  sumsq64<<<one_wave(s, sumsq64), kRedThreads, 0, s.st>>>(x, s.ng, w.sc, w.partials);
  if (cudaGetLastError() != cudaSuccess) return finish(fail(SPX_ERR_CUDA, "cg initial guess norm"));
  Scalars h0{};
  if ((st = read_scalars(s, &h0)) != SPX_OK) return finish(st);
  double rr, ff;
  if ((st = residual(s, f, x, &rr, &ff, h0.scale == 0.0)) != SPX_OK) return finish(st);
  if (ff == 0.0) {
    fill_zero<double><<<s.grid_v, 256, 0, s.st>>>(x, s.ng);
    return finish(SPX_OK);
  }
  const double tol = o->tol;
  int total_it = 0;
  if (o->precision == 0) {
    // all-FP64 PCG; restart from the true residual if the recurrence drifted
    PcgRun<double> run{&s, SPX_F64, x, w.r64, w.z64, w.p64, w.q64, w.minv64, w.pl64, w.ql64};
    if ((st = run.prepare(use_graph, o->check_every)) != SPX_OK) return finish(st);
    for (int restart = 0; restart < 4; ++restart) {
      if (!std::isfinite(rr)) return finish(fail(SPX_ERR_NONFINITE, "cg_solve: non-finite residual"));
      if (std::sqrt(rr / ff) <= tol) break;
      if ((st = set_scalars(s, ff, tol, o->maxit - total_it)) != SPX_OK) return finish(st);
      Scalars h{};
      if ((st = run.start()) != SPX_OK || (st = run.run(&h)) != SPX_OK) return finish(st);
      total_it += h.it;
      if (h.nonfinite) return finish(fail(SPX_ERR_NONFINITE, "cg_solve: non-finite residual"));
      if ((st = residual(s, f, x, &rr, &ff)) != SPX_OK) return finish(st);
      if (total_it >= o->maxit) break;
    }
    res->iters = total_it;
    res->rel_residual = std::sqrt(rr / ff);
  } else {
    // FP32 PCG on the scaled correction equation A d = r / ||r|| (from d = 0),
    // x += ||r|| d and the FP64 residual r = f - A x after every FP32 run.
    // precision 1 restarts the FP32 PCG from the new residual (p = z);
    // precision 2 replaces the FP32 recurrence residual by the new one and
    // continues the same run (reliable update, reliable_restart).  An FP32
    // run stops once its residual fell by inner_tol, or by half of what the
    // outer tolerance still asks if that is less.
    PcgRun<float> run{&s, SPX_F32, w.d32, w.r32, w.z32, w.p32, w.q32, w.minv32, w.pl32, w.ql32};
    if ((st = run.prepare(use_graph, o->check_every)) != SPX_OK) return finish(st);
    int outer = 0;
    double s_old = 0.0;
    for (; outer < o->max_outer; ++outer) {
      if (!std::isfinite(rr)) return finish(fail(SPX_ERR_NONFINITE, "cg_solve: non-finite residual"));
      const double rel = std::sqrt(rr / ff);
      if (rel <= tol) break;
      if (o->precision == 2 && total_it >= o->maxit) break;
      const double s_new = std::sqrt(rr);
      const double itol = std::max(o->inner_tol, 0.5 * tol / rel);
      Scalars h{};
      if (o->precision == 1 || outer == 0) {
        to_f32_scaled<<<s.grid_v, 256, 0, s.st>>>(w.r64, w.r32, w.d32, s.ng, w.sc);
        // right-hand side norm of the scaled system is 1
        if ((st = set_scalars(s, 1.0, itol, o->maxit)) != SPX_OK) return finish(st);
        if ((st = run.start()) != SPX_OK) return finish(st);
      } else {
        if ((st = read_scalars(s, &h)) != SPX_OK) return finish(st);
        h.ff = 1.0;
        h.tol2 = itol * itol;
        h.ticket = 0;
        SPX_CK(cudaMemcpyAsync(w.sc, &h, sizeof(Scalars), cudaMemcpyHostToDevice, s.st));
        reliable_restart<<<one_wave(s, reliable_restart), kRedThreads, 0, s.st>>>(
            w.r64, w.r32, w.d32, w.z32, w.minv32, s.ng, 1.0 / s_new, s_old / s_new, w.sc, w.partials);
        run.direction();
        SPX_CK(cudaGetLastError());
      }
      s_old = s_new;
      if ((st = run.run(&h)) != SPX_OK) return finish(st);
      total_it = o->precision == 1 ? total_it + h.it : h.it;
      if (h.nonfinite) return finish(fail(SPX_ERR_NONFINITE, "cg_solve: non-finite inner residual"));
      add_correction<<<s.grid_v, 256, 0, s.st>>>(x, w.d32, s.ng, s_new);
      if ((st = residual(s, f, x, &rr, &ff)) != SPX_OK) return finish(st);
    }
    res->iters = total_it;
    res->outer_iters = outer;
    res->rel_residual = std::sqrt(rr / ff);
  }
  if (!std::isfinite(res->rel_residual)) return finish(fail(SPX_ERR_NONFINITE, "cg_solve: non-finite residual"));
  if (res->rel_residual > tol)
    return finish(fail(SPX_ERR_NOT_CONVERGED, "cg_solve: tolerance not reached within the iteration caps"));
  return finish(SPX_OK);
}

// ---------------------------------------------------------------------------
// <a, b> at FP64 accuracy (the PCG inner products, exposed on their own):
// per-thread DotAcc partials, the fixed-order grid reduction, the result
// written by the last block.  Fixed grid (2 blocks per SM): reproducible.
template <typename T, int V>
__global__ void __launch_bounds__(kRedThreads) dot_kernel(const T* __restrict__ a, const T* __restrict__ b,
                                                          int64_t n, double* partials, unsigned int* ticket,
                                                          double* out) {
  DotAcc<T> acc;
  const int64_t S = int64_t(gridDim.x) * blockDim.x, t0 = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  const int64_t np = n / V;
  for (int64_t i = t0; i < np; i += S) {
    const Pack<T, V> av = ldp<T, V>(a, i), bv = ldp<T, V>(b, i);
#pragma unroll
    for (int c = 0; c < V; ++c) acc.add(av.v[c], bv.v[c]);
  }
  for (int64_t g = np * V + t0; g < n; g += S) acc.add(a[g], b[g]);
  double r, unused;
  if (grid_reduce2(acc.value(), 0.0, partials, ticket, &r, &unused)) {
    *out = r;
    *ticket = 0;
  }
}

// ---------------------------------------------------------------------------
// Allocation-free solve: the workspace is a fixed array in the module's own
// device memory.  It exists on every device that loads this library, from
// module load until process exit, and is shared by every call on that device.
// ---------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_noalloc_ws[SPX_CG_NOALLOC_BYTES];

std::mutex g_noalloc_mu;
constexpr int kMaxDevices = 64;
struct NoallocAddr {
  unsigned long long ctx_id = 0;   // CUDA context the address belongs to (0: none yet)
  void* addr = nullptr;
};
NoallocAddr g_noalloc[kMaxDevices];

}  // namespace

// Device address of g_noalloc_ws on the current device, looked up with that
// device current (the host-side symbol is only a handle, never a device
// pointer) once per device and context: the cache is keyed on the context's
// unique id, so a context created after a cudaDeviceReset gets a fresh
// lookup instead of a stale address.  The lookup loads this file's device
// code on the device if it is not loaded yet, which is when the array is
// reserved; spx_plan_create calls this, so a solve on a plan's device finds
// the address cached.
spx_status noalloc_workspace(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return fail(SPX_ERR_UNSUPPORTED, "no-alloc workspace: device ordinal too large");
  e = cudaFree(nullptr);   // makes the device's primary context current (allocates nothing)
  if (e != cudaSuccess) return cuda_fail(e, "cudaFree(NULL)");
  // driver entry points through the runtime (the library does not link the
  // driver library itself, so it still loads where no driver is installed)
  using GetCurrentFn = CUresult (*)(CUcontext*);
  using GetIdFn = CUresult (*)(CUcontext, unsigned long long*);
  static GetCurrentFn get_current = nullptr;
  static GetIdFn get_id = nullptr;
  {
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    if (!get_current || !get_id) {
      void* f0 = nullptr;
      void* f1 = nullptr;
      cudaDriverEntryPointQueryResult q0, q1;
      if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f0, 12000, cudaEnableDefault, &q0) != cudaSuccess ||
          cudaGetDriverEntryPointByVersion("cuCtxGetId", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
          q0 != cudaDriverEntryPointSuccess || q1 != cudaDriverEntryPointSuccess || !f0 || !f1)
        return fail(SPX_ERR_CUDA, "no-alloc workspace: driver entry points cuCtxGetCurrent / cuCtxGetId not found");
      get_current = reinterpret_cast<GetCurrentFn>(f0);
      get_id = reinterpret_cast<GetIdFn>(f1);
    }
  }
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
    return fail(SPX_ERR_CUDA, "no-alloc workspace: no current CUDA context");
  std::lock_guard<std::mutex> g(g_noalloc_mu);
  NoallocAddr& c = g_noalloc[dev];
  if (c.ctx_id != id || !c.addr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_ws);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-alloc workspace)");
    c.ctx_id = id;
    c.addr = p;
  }
  *out = c.addr;
  return SPX_OK;
}

}  // namespace spx

extern "C" spx_status spx_dot(const spx_plan* plan, spx_dtype dt, int64_t n, const void* a, const void* b,
                              double* result, void* stream) {
  if (!plan || !result || n < 0 || (n && (!a || !b))) return fail(SPX_ERR_INVALID_ARG, "dot: bad argument");
  if (dt != SPX_F64 && dt != SPX_F32) return fail(SPX_ERR_INVALID_ARG, "dot: bad dtype");
  const size_t sz = dt == SPX_F64 ? 8 : 4;
  if ((reinterpret_cast<uintptr_t>(a) % sz) || (reinterpret_cast<uintptr_t>(b) % sz) ||
      (reinterpret_cast<uintptr_t>(result) % 8))
    return fail(SPX_ERR_INVALID_ARG, "dot: buffer not aligned to its element size");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int grid = plan->num_sms * 2;   // 2 partials per block fit the plan's num_sms * 4 values
  const bool v16 = !(reinterpret_cast<uintptr_t>(a) & 15) && !(reinterpret_cast<uintptr_t>(b) & 15);
  if (dt == SPX_F64) {
    const double *x = static_cast<const double*>(a), *y = static_cast<const double*>(b);
    if (v16) dot_kernel<double, 2><<<grid, kRedThreads, 0, st>>>(x, y, n, plan->d_partials, plan->d_ticket, result);
    else dot_kernel<double, 1><<<grid, kRedThreads, 0, st>>>(x, y, n, plan->d_partials, plan->d_ticket, result);
  } else {
    const float *x = static_cast<const float*>(a), *y = static_cast<const float*>(b);
    if (v16) dot_kernel<float, 4><<<grid, kRedThreads, 0, st>>>(x, y, n, plan->d_partials, plan->d_ticket, result);
    else dot_kernel<float, 1><<<grid, kRedThreads, 0, st>>>(x, y, n, plan->d_partials, plan->d_ticket, result);
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SPX_OK : cuda_fail(e, "dot kernel launch");
}

extern "C" spx_status spx_cg_solve(const spx_plan* plan, double lambda, const int32_t* l2g, int64_t n_global,
                                   const double* f, double* x, void* workspace, size_t ws_bytes,
                                   const spx_cg_opts* o, spx_cg_result* res, void* stream) {
  return cg_solve_impl(plan, lambda, l2g, n_global, f, x, workspace, ws_bytes, o, res, stream, true);
}

extern "C" spx_status spx_cg_solve_noalloc(const spx_plan* plan, double lambda, const int32_t* l2g,
                                           int64_t n_global, const double* f, double* x, const spx_cg_opts* o,
                                           spx_cg_result* res, void* stream) {
  if (!plan || !o || !res) return fail(SPX_ERR_INVALID_ARG, "cg_solve_noalloc: NULL argument");
  size_t need = 0;
  spx_status st = spx_cg_workspace_bytes(plan, n_global, o, &need);
  if (st != SPX_OK) return st;
  if (need > SPX_CG_NOALLOC_BYTES)
    return fail(SPX_ERR_NO_MEMORY, "cg_solve_noalloc: this problem needs " + std::to_string(need) +
                                       " bytes of solver workspace; the built-in workspace holds " +
                                       std::to_string(size_t(SPX_CG_NOALLOC_BYTES)) +
                                       " (use spx_cg_solve with a caller workspace)");
  void* ws = nullptr;
  if ((st = noalloc_workspace(&ws)) != SPX_OK) return st;
  return cg_solve_impl(plan, lambda, l2g, n_global, f, x, ws, SPX_CG_NOALLOC_BYTES, o, res, stream, false);
}
