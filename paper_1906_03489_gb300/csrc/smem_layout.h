// Shared-memory layout of the operator kernel (host side).
#pragma once
#include <algorithm>
#include <cstdint>

#include "spx_internal.h"

namespace spx {

inline int n_work_buffers(int op) {
  switch (op) {
    case OP_BWD: return 2;
    case OP_IPROD: return 2;
    case OP_DERIV: return 3;
    case OP_HELM: return 4;
    case OP_ADJ: return 8;
    case OP_FWD: return 7;
    case OP_SENSOR: return 7;
    default: return 5;
  }
}

// Host mirror of op_streams(): value counts per element of each stream slot,
// 0 when the stream is absent.
inline void stream_lens(int op, int dim, int P, int Q, bool lam_f, bool kap_f, int64_t lens[5]) {
  const int64_t nd = dim == 3 ? int64_t(P + 1) * (P + 1) * (P + 1) : int64_t(P + 1) * (P + 1);
  const int64_t qd = dim == 3 ? int64_t(Q) * Q * Q : int64_t(Q) * Q;
  const int nf = dim == 3 ? 7 : 4;
  for (int s = 0; s < 5; ++s) lens[s] = 0;
  switch (op) {
    case OP_BWD: lens[0] = nd; break;
    case OP_IPROD: lens[0] = qd; lens[1] = qd; break;
    case OP_FWD: lens[0] = qd; lens[1] = qd; break;
    case OP_SENSOR: lens[0] = nd; lens[1] = qd; break;
    case OP_DERIV: lens[0] = qd; lens[1] = dim * dim * qd; break;
    case OP_HELM:
      lens[0] = nd; lens[1] = nf * qd; lens[2] = lam_f ? qd : 0; lens[3] = kap_f ? qd : 0;
      break;
    case OP_ADJ:
      lens[0] = nd; lens[1] = nd; lens[2] = nf * qd; lens[3] = lam_f ? qd : 0; lens[4] = kap_f ? qd : 0;
      break;
    default: lens[0] = nf * qd; lens[1] = lam_f ? qd : 0; break;
  }
}

struct SmemLayout {
  uint32_t slot_base, slot_bytes, region_off[5], work_base, work_bytes, meta_base, total;
};

inline uint32_t up128(uint64_t x) { return static_cast<uint32_t>((x + 127) & ~uint64_t(127)); }

// stages 0 selects, for the 3D Helmholtz bodies with Q^2 threads per element,
// geometry read from L2 instead of staged (no geometry region) and one slot.
inline bool geo_direct(const spx_plan* plan, int op, const LaunchCfg& cfg) {
  return op == OP_HELM && plan->dim == 3 && plan->bkind != BK_GENERAL && cfg.stages == 0;
}

inline SmemLayout smem_layout(const spx_plan* plan, int op, int sz, const LaunchCfg& cfg, bool lam_f, bool kap_f) {
  SmemLayout L{};
  const bool direct = geo_direct(plan, op, cfg);
  uint64_t region[5] = {0, 0, 0, 0, 0};
  uint64_t work = 0;
  for (int P = 1; P <= kMaxP; ++P) {
    if (!plan->present[P]) continue;
    const int Q = P + plan->qoff;
    const int eb = cfg.order[P].eb;
    int64_t lens[5];
    stream_lens(op, plan->dim, P, Q, lam_f, kap_f, lens);
    if (direct) lens[1] = 0;
    for (int s = 0; s < 5; ++s)
      if (lens[s]) region[s] = std::max<uint64_t>(region[s], uint64_t(eb) * (((lens[s] * sz + 15) & ~int64_t(15)) + 16));
    const int S1 = Q | 1;
    uint64_t ws = plan->dim == 3 ? uint64_t(S1) * Q * Q : uint64_t(S1) * Q;
    if (op == OP_HELM && plan->dim == 3 && plan->bkind != BK_GENERAL) {  // column / pencil role layout
      const uint64_t n = P + 1, S = Q | 1, SN = n | 1;
      ws = std::max<uint64_t>({ws, n * Q * S, n * n * S, uint64_t(Q) * Q * SN, uint64_t(Q) * Q * S});
    }
    work = std::max<uint64_t>(work, uint64_t(eb) * ws * sz);
    if (op == OP_DIAG) work = std::max<uint64_t>(work, uint64_t(3) * Q * (P + 1) * sz);
  }
  L.slot_base = 128;
  uint64_t off = 0;
  for (int s = 0; s < 5; ++s) {
    L.region_off[s] = static_cast<uint32_t>(off);
    off += up128(region[s]);
  }
  L.slot_bytes = static_cast<uint32_t>(off);
  L.work_base = L.slot_base + (cfg.stages < 1 ? 1 : cfg.stages) * L.slot_bytes;
  L.work_bytes = up128(work);
  L.meta_base = L.work_base + n_work_buffers(op) * L.work_bytes;
  L.total = L.meta_base + 5 * kMaxEB * 4 + 2 * kMaxEB * 8 + 16 + (op == OP_FWD || op == OP_SENSOR ? kFwdExtra * sz : 0);
  return L;
}

// Launch shape of the FP32 3D Helmholtz kernel (helm_pair.cuh): orders
// P <= thr run two elements per thread, the others one; a tile of eb elements
// is ceil(eb / lanes) element groups of Q^2 threads each.  Shared memory: an
// mbarrier, the three work buffers A, C, F (PairLayout strides per group) and
// one geometry slot holding the tile's [eb][7][Q^3] factors.
struct PairShape {
  int nthreads;                  // compute threads
  uint32_t off_a, off_c, off_f;  // byte offsets of the work buffers
  uint32_t off_geo;              // byte offset of the geometry slot
  uint32_t off_meta;             // byte offset of the two tile-metadata buffers (variable order)
  uint32_t slot_bytes;           // BwdTrans / IProductWRTBase: bytes per input-ring slot (at off_geo)
  uint32_t smem;
};

// Tile metadata buffer of the variable-order kernel's producer warp (Tile +
// coefficient and quadrature offsets of up to kMaxEB elements).
constexpr uint32_t kTileMetaBytes = 16 + 2 * 8 * kMaxEB;

// BwdTrans / IProductWRTBase in the pair layout (pair_ops.cuh, uniform
// order): the work buffers of their phases, then `stages` input-ring slots
// (SfSlot) in place of the geometry slot.
inline PairShape pair_shape(const spx_plan* plan, const LaunchCfg& cfg, int thr, int op = OP_HELM) {
  PairShape s{};
  uint64_t wa = 0, wc = 0, wf = 0, geo = 0;
  const bool sf = op == OP_BWD || op == OP_IPROD;
  for (int P = 1; P <= kMaxP; ++P) {
    if (!plan->present[P]) continue;
    const int Q = P + plan->qoff;
    const int eb = cfg.order[P].eb;
    const int lanes = sf ? 2 : pair_lanes(P, thr);
    const int groups = (eb + lanes - 1) / lanes;
    uint64_t w[3];
    if (sf) {
      pair_sf_bytes(P, plan->qoff, w);
      if (op == OP_BWD) w[2] = 0;   // A (X) and C (Y)
      else w[0] = 0;                // C (Y3) and F (Y2)
    } else {
      pair_ws_bytes(P, plan->qoff, lanes, w);
    }
    s.nthreads = std::max(s.nthreads, groups * Q * Q);
    wa = std::max<uint64_t>(wa, groups * w[0]);
    wc = std::max<uint64_t>(wc, groups * w[1]);
    wf = std::max<uint64_t>(wf, groups * w[2]);
    if (!sf) geo = std::max<uint64_t>(geo, uint64_t(eb) * geo_erb(Q));   // per element regions
  }
  s.nthreads = (s.nthreads + 31) / 32 * 32;
  if (sf) {
    const int P = plan->uP, Q = P + plan->qoff, eb = cfg.order[P].eb;
    const uint64_t nv = op == OP_BWD ? uint64_t(P + 1) * (P + 1) * (P + 1) : uint64_t(Q) * Q * Q;
    const uint64_t f_rb = ((eb * nv * 4 + 15) & ~uint64_t(15)) + 16;
    const uint64_t jw_rb = ((uint64_t(Q) * Q * Q * 4 + 15) & ~uint64_t(15)) + 16;
    s.slot_bytes = static_cast<uint32_t>(up128(op == OP_BWD ? f_rb : f_rb + eb * jw_rb));
    geo = uint64_t(cfg.stages) * s.slot_bytes;
  }
  s.off_a = 128;
  s.off_c = s.off_a + up128(wa);
  s.off_f = s.off_c + up128(wc);
  s.off_geo = s.off_f + up128(wf);
  s.off_meta = s.off_geo + up128(geo);
  s.smem = s.off_meta + (plan->uniform ? 0 : up128(2 * kTileMetaBytes));
  return s;
}

// Orders packed two per thread: all of them in a uniform-order plan; in a
// variable-order launch (one kernel for every order, registers allocated for
// the largest body) the launch's `nthreads` class picks the highest packed
// order: <= 512: 5, <= 640: 6, else 8 (pairs of P = 7, 8 spill a little at
// 128 registers).
inline int pair_threshold(const spx_plan* plan, const LaunchCfg& cfg) {
  if (plan->uniform) return kMaxP;
  return cfg.nthreads <= 512 ? kPairThrVar : (cfg.nthreads <= 640 ? 6 : 8);
}

inline bool uses_pair_kernel(const spx_plan* plan, int op, int dtype) {
  if ((op == OP_BWD || op == OP_IPROD) && dtype == 1 && plan->dim == 3 && plan->bkind == BK_PARITY && !plan->shape &&
      plan->uniform)
    return true;
  return op == OP_HELM && dtype == 1 && plan->dim == 3 && plan->bkind == BK_PARITY && !plan->shape;
}

}  // namespace spx
