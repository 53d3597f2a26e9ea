// Parameter block of the operator kernel, shared by host and device code.
#pragma once
#include <cstdint>

namespace spx {

constexpr int kMaxEB = 64;  // elements per tile (upper bound)
constexpr int kMaxP = 8;    // highest supported order
constexpr int kMaxP1 = 9;   // orders 0..8 index per-order tables

enum OpKind { OP_BWD = 0, OP_IPROD = 1, OP_DERIV = 2, OP_HELM = 3, OP_ADJ = 4, OP_DIAG = 5, OP_KINDS = 6 };

// A tile: `count` elements of order P.  contig != 0: the elements are
// id(first), id(first)+1, ...; else ids[first + j].  Without an id array
// id(x) = x.
struct Tile {
  int32_t P;
  int32_t count;
  int32_t first;
  int32_t contig;
};

__host__ __device__ constexpr int tab_len(int P, int QOFF) {
  // B[Q][n], dB[Q][n], D[Q][Q]
  return 2 * (P + QOFF) * (P + 1) + (P + QOFF) * (P + QOFF);
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
  double lam;
  int n_tiles;
  int stages;
  uint32_t slot_base;      // byte offset of slot 0
  uint32_t slot_bytes;
  uint32_t region_off[5];  // per stream, inside a slot
  uint32_t work_base;
  uint32_t work_bytes;     // per work buffer
  uint32_t meta_base;
  T tab[Layout::total];
};

}  // namespace spx
