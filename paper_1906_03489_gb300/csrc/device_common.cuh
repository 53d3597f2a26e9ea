// Device building blocks shared by the operator kernels (sm_103a).
//
//  * bulk-copy pipeline: 1D TMA copies (cp.async.bulk) of element blocks from
//    HBM into shared memory, completion tracked by one mbarrier per stage, with
//    bounded waits (a wait that gives up raises a status flag instead of
//    hanging);
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace spx {

constexpr unsigned long long kWaitNs = 4000000000ull;  // a staged copy not landed after 4 s is abandoned
constexpr int kStatusTimeout = 1;     // bit set in the plan's device status word
constexpr int kStatusBadIndex = 2;    // bit set when an index argument is out of range
constexpr int kStatusNotConverged = 4;  // bit set when an elemental iteration hit its step cap

// ---------------------------------------------------------------------------
// PTX helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t tx) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(tx)
               : "memory");
}

// 1D bulk copy global -> shared; dst, src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait bounded in wall-clock time; returns false if it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (unsigned i = 1;; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 63u) == 0 && global_ns() - t0 > kWaitNs) return false;
  }
}

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

// ---------------------------------------------------------------------------
// Staging of element blocks into shared memory.
//
// A "range" is a contiguous byte interval [g, g + bytes) of global memory
// that lands in shared memory at region + (g mod 16) (region 16-byte
// aligned), so that the 16-byte aligned interior can be moved by one bulk
// copy and the ragged head and tail (< 16 bytes each, whole words) by plain
// loads once the copy has landed.
// ---------------------------------------------------------------------------
struct RangeSplit {
  uintptr_t g0, a0, a1, g1;  // [g0,a0) head, [a0,a1) bulk, [a1,g1) tail
};

__device__ __forceinline__ RangeSplit split_range(const void* g, uint32_t bytes) {
  RangeSplit s;
  s.g0 = reinterpret_cast<uintptr_t>(g);
  s.g1 = s.g0 + bytes;
  s.a0 = (s.g0 + 15) & ~uintptr_t(15);
  s.a1 = s.g1 & ~uintptr_t(15);
  if (s.a1 <= s.a0) {  // no aligned interior: everything by plain loads
    s.a0 = s.g1;
    s.a1 = s.g1;
  }
  return s;
}

// Producer side: issue the bulk part, return its byte count (for expect_tx).
__device__ __forceinline__ uint32_t stage_issue(char* region, const void* g, uint32_t bytes, uint64_t* bar) {
  RangeSplit s = split_range(g, bytes);
  uint32_t n = static_cast<uint32_t>(s.a1 - s.a0);
  // the range's data starts at region + (g0 mod 16); global a0 lands at
  // region + (g0 mod 16) + (a0 - g0) = region + (a0 - floor16(g0)), 16-byte aligned
  if (n) bulk_g2s(region + (s.g0 & 15) + (s.a0 - s.g0), reinterpret_cast<const void*>(s.a0), n, bar);
  return n;
}

// Bulk bytes of a range without issuing (for expect_tx computed up front).
__device__ __forceinline__ uint32_t stage_bytes(const void* g, uint32_t bytes) {
  RangeSplit s = split_range(g, bytes);
  return static_cast<uint32_t>(s.a1 - s.a0);
}

// Consumer side: copy head and tail words of a range (any thread may call;
// `lane` in [0, nlanes) selects the word).  Word size W (4 or 8 bytes).
template <int W>
__device__ __forceinline__ void stage_fixup(char* region, const void* g, uint32_t bytes, int lane, int nlanes) {
  RangeSplit s = split_range(g, bytes);
  char* dst0 = region + (s.g0 & 15);
  const int nhead = static_cast<int>((s.a0 - s.g0) / W);
  const int ntail = static_cast<int>((s.g1 - s.a1) / W);
  for (int w = lane; w < nhead + ntail; w += nlanes) {
    uintptr_t src = w < nhead ? s.g0 + uintptr_t(w) * W : s.a1 + uintptr_t(w - nhead) * W;
    char* dst = dst0 + (src - s.g0);
    if (W == 8)
      *reinterpret_cast<unsigned long long*>(dst) = __ldg(reinterpret_cast<const unsigned long long*>(src));
    else
      *reinterpret_cast<unsigned*>(dst) = __ldg(reinterpret_cast<const unsigned*>(src));
  }
}

// Shared-memory address of the data of a staged range.
template <typename T>
__device__ __forceinline__ T* staged_ptr(char* region, const void* g) {
  return reinterpret_cast<T*>(region + (reinterpret_cast<uintptr_t>(g) & 15));
}

}  // namespace spx
