// Host launcher of the operator kernel for one (precision, dimension, operator).
#pragma once
#include <algorithm>
#include <mutex>

#include <type_traits>

#include "helm_pair.cuh"
#include "op_kernel.cuh"
#include "pair_ops.cuh"
#include "smem_layout.h"
#include "spx_internal.h"

namespace spx {

template <class K, class Prm>
spx_status launch_pair_kernel(K kern, const Prm& pp, int nthreads, uint32_t smem, const spx_plan* plan, int n_tiles,
                              cudaStream_t stream, bool* configured, std::mutex* mu) {
  {
    std::lock_guard<std::mutex> g(*mu);
    if (!*configured) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           static_cast<int>(plan->max_smem));
      if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
      *configured = true;
    }
  }
  int nb = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, nthreads, smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  if (nb < 1) return fail(SPX_ERR_UNSUPPORTED, "pair-kernel tile does not fit on an SM");
  const int grid = std::min<int64_t>(n_tiles, int64_t(nb) * plan->num_sms);
  kern<<<grid, nthreads, smem, stream>>>(pp);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "pair kernel launch");
  return SPX_OK;
}

template <int PLO, int PHI, int QOFF, int REG, int THR>
spx_status launch_pair_reg(const PairParams<PLO, PHI, QOFF>& pp, const PairShape& s, const spx_plan* plan, int n_tiles,
                           cudaStream_t stream) {
  static std::mutex mu;
  static bool configured = false;
  return launch_pair_kernel(helm_pair_kernel<PLO, PHI, QOFF, REG, THR>, pp, s.nthreads, s.smem, plan, n_tiles,
                            stream, &configured, &mu);
}

// Splits `grid` CTAs among the runs of a variable-order tile list in
// proportion to their algorithmic bytes (every run gets at least one CTA and
// no more than its tiles), into grp_cta.
inline int varp_split_ctas(const TileList& tl, int grid, int* grp_cta) {
  if (tl.grp_P.empty()) {   // uniform order: one run over the whole list
    grp_cta[0] = 0;
    grp_cta[1] = std::max(1, std::min(grid, tl.n));
    return grp_cta[1];
  }
  const int ng = static_cast<int>(tl.grp_P.size());
  double W = 0.0;
  for (double b : tl.grp_bytes) W += b;
  std::vector<int> cnt(ng);
  int used = 0;
  for (int g = 0; g < ng; ++g) {
    const int nt = tl.grp_tile[g + 1] - tl.grp_tile[g];
    cnt[g] = std::max(1, std::min(nt, static_cast<int>(grid * tl.grp_bytes[g] / std::max(W, 1.0))));
    used += cnt[g];
  }
  // hand out what rounding left over to the runs with the most bytes per CTA
  while (used < grid) {
    int best = -1;
    double bw = 0.0;
    for (int g = 0; g < ng; ++g) {
      const int nt = tl.grp_tile[g + 1] - tl.grp_tile[g];
      if (cnt[g] >= nt) continue;
      const double w = tl.grp_bytes[g] / cnt[g];
      if (w > bw) {
        bw = w;
        best = g;
      }
    }
    if (best < 0) break;
    ++cnt[best];
    ++used;
  }
  grp_cta[0] = 0;
  for (int g = 0; g < ng; ++g) grp_cta[g + 1] = grp_cta[g] + cnt[g];
  return grp_cta[ng];
}

// The runs of a launch's tile list into the kernel parameters (one per order
// present, or one for a uniform plan) and the grid split among them; returns
// the grid size (0 if the list is malformed).
template <class KP>
int set_runs(KP& k, const spx_plan* plan, const TileList& tl, int grid, bool one_run = false, int layers = 1) {
  k.layers = 0;
  k.nslot = 0;
  if (one_run) {   // every CTA walks the whole list (orders mixed, heaviest first)
    k.ngrp = 1;
    k.grp_P[0] = 0;
    k.grp_tile[0] = 0;
    k.grp_tile[1] = tl.n;
    k.grp_cta[0] = 0;
    k.grp_cta[1] = std::max(1, std::min(grid, tl.n));
    return k.grp_cta[1];
  }
  if (tl.grp_P.empty()) {
    k.ngrp = 1;
    k.grp_P[0] = plan->uP;
    k.grp_tile[0] = 0;
    k.grp_tile[1] = tl.n;
  } else {
    const int ng = static_cast<int>(tl.grp_P.size());
    if (ng > kMaxP) return 0;
    k.ngrp = ng;
    for (int g = 0; g < ng; ++g) k.grp_P[g] = tl.grp_P[g];
    for (int g = 0; g <= ng; ++g) k.grp_tile[g] = tl.grp_tile[g];
    if (layers > 1 && grid / layers >= ng) {   // split SM slots; every layer repeats the split
      const int nslot = varp_split_ctas(tl, grid / layers, k.grp_cta);
      k.layers = layers;
      k.nslot = nslot;
      return nslot * layers;
    }
    grid = std::max(grid, ng);
  }
  return varp_split_ctas(tl, grid, k.grp_cta);
}

// variable order: compute threads + one producer warp; the grid is split
// among the orders' runs of tiles (KParams::grp_*)
template <int PLO, int PHI, int QOFF, int REG, int THR>
spx_status launch_varp_reg(PairParams<PLO, PHI, QOFF>& pp, const PairShape& s, const spx_plan* plan,
                           const TileList& tl, cudaStream_t stream) {
  static std::mutex mu;
  static bool configured = false;
  auto kern = helm_varp_kernel<PLO, PHI, QOFF, REG, THR>;
  const int nthreads = s.nthreads + 32;
  if (nthreads > 1024) return fail(SPX_ERR_UNSUPPORTED, "Helmholtz tile needs too many threads");
  {
    std::lock_guard<std::mutex> g(mu);
    if (!configured) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           static_cast<int>(plan->max_smem));
      if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
      configured = true;
    }
  }
  int nb = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, nthreads, s.smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  if (nb < 1) return fail(SPX_ERR_UNSUPPORTED, "pair-kernel tile does not fit on an SM");
  const int grid = set_runs(pp.k, plan, tl, nb * plan->num_sms, false, nb);
  if (grid < 1) return fail(SPX_ERR_UNSUPPORTED, "tile list has no order runs");
  kern<<<grid, nthreads, s.smem, stream>>>(pp);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "Helmholtz kernel launch");
  return SPX_OK;
}

// FP32 Helmholtz on hexahedra (helm_pair.cuh).  `stages` of the launch
// configuration is its L2 prefetch distance in tiles; `nthreads` the number
// of threads per SM that the register budget must allow: 128 registers up to
// 512, 96 up to 640, else 80 (uniform order).  Variable-order launches run the
// producer-warp kernel at 128 registers; there `nthreads` picks the highest
// order run in pairs (pair_threshold).
template <int PLO, int PHI, int QOFF>
spx_status launch_pair(const LaunchReq& r) {
  const spx_plan* plan = r.plan;
  const LaunchCfg& cfg = plan->cfg[OP_HELM][1];
  const TileList& tl = plan->tiles[OP_HELM][1];
  if (tl.n == 0) return SPX_OK;
  PairParams<PLO, PHI, QOFF> pp{};
  auto& p = pp.k;
  for (int P = PLO; P <= PHI; ++P) {
    if (!plan->present[P]) continue;
    const std::vector<double>& t = plan->tab[P];
    const int off = TabLayout<PLO, PHI, QOFF>::off(P);
    for (int i = 0; i < tab_len(P, QOFF); ++i) p.tab[off + i] = static_cast<float>(t[i]);
  }
  p.tiles = tl.d;
  p.ids = plan->uniform ? nullptr : plan->d_ids;
  p.coef_off = plan->uniform ? nullptr : plan->d_coef_off;
  p.quad_off = plan->uniform ? nullptr : plan->d_quad_off;
  p.in0 = static_cast<const float*>(r.in0);
  p.geom = static_cast<const float*>(r.geom);
  p.lam_f = static_cast<const float*>(r.lam_f);
  p.kap_f = static_cast<const float*>(r.kap_f);
  p.out0 = static_cast<float*>(r.out0);
  p.status = plan->d_status;
  p.skip = r.skip;
  p.lam = r.lam;
  p.n_tiles = tl.n;
  const int thr = pair_threshold(plan, cfg);
  const PairShape s = pair_shape(plan, cfg, thr);
  if (s.nthreads > 512) return fail(SPX_ERR_UNSUPPORTED, "Helmholtz tile needs more than 512 threads");
  if (s.smem > plan->max_smem) return fail(SPX_ERR_UNSUPPORTED, "Helmholtz tile does not fit in shared memory");
  pp.pf = cfg.stages;
  pp.off_a = s.off_a;
  pp.off_c = s.off_c;
  pp.off_f = s.off_f;
  pp.off_geo = s.off_geo;
  if constexpr (PLO == PHI) {
    const int budget = cfg.nthreads;
    if (budget <= 512) return launch_pair_reg<PLO, PHI, QOFF, 128, kMaxP>(pp, s, plan, tl.n, r.stream);
    if (budget <= 640) return launch_pair_reg<PLO, PHI, QOFF, 96, kMaxP>(pp, s, plan, tl.n, r.stream);
    return launch_pair_reg<PLO, PHI, QOFF, 80, kMaxP>(pp, s, plan, tl.n, r.stream);
  } else {
    pp.off_meta = s.off_meta;
    if (thr == kPairThrVar) return launch_varp_reg<PLO, PHI, QOFF, 128, kPairThrVar>(pp, s, plan, tl, r.stream);
    if (thr == 6) return launch_varp_reg<PLO, PHI, QOFF, 128, 6>(pp, s, plan, tl, r.stream);
    return launch_varp_reg<PLO, PHI, QOFF, 128, 8>(pp, s, plan, tl, r.stream);
  }
}

template <int OP, int P, int QOFF, int REG>
spx_status launch_sf_reg(const SfParams<P, QOFF>& pp, const PairShape& s, const spx_plan* plan, int n_tiles,
                         cudaStream_t stream) {
  static std::mutex mu;
  static bool configured = false;
  return launch_pair_kernel(sf_pair_kernel<OP, P, QOFF, REG>, pp, s.nthreads, s.smem, plan, n_tiles, stream,
                            &configured, &mu);
}

// FP32 BwdTrans / IProductWRTBase on hexahedra of one order in the pair
// layout (pair_ops.cuh).  `nthreads` of the launch configuration is the
// number of threads per SM the register budget must allow (80 registers up
// to 768, 64 up to 1024, 48 up to 1280, else 40); `stages` the slots of the
// shared-memory input ring (0: inputs carried in registers).
template <int OP, int P, int QOFF>
spx_status launch_sf_pair(const LaunchReq& r) {
  const spx_plan* plan = r.plan;
  const LaunchCfg& cfg = plan->cfg[OP][1];
  const TileList& tl = plan->tiles[OP][1];
  if (tl.n == 0) return SPX_OK;
  SfParams<P, QOFF> pp{};
  auto& p = pp.k;
  const std::vector<double>& t = plan->tab[P];
  for (int i = 0; i < tab_len(P, QOFF); ++i) p.tab[i] = static_cast<float>(t[i]);
  p.tiles = tl.d;
  p.in0 = static_cast<const float*>(r.in0);
  p.geom = static_cast<const float*>(r.geom);
  p.out0 = static_cast<float*>(r.out0);
  p.status = plan->d_status;
  p.skip = r.skip;
  p.n_tiles = tl.n;
  const PairShape s = pair_shape(plan, cfg, kMaxP, OP);
  if (s.nthreads > 1024) return fail(SPX_ERR_UNSUPPORTED, "operator tile needs more than 1024 threads");
  if (s.smem > plan->max_smem) return fail(SPX_ERR_UNSUPPORTED, "operator tile does not fit in shared memory");
  pp.stages = cfg.stages;
  pp.eb = cfg.order[P].eb;
  pp.off_a = s.off_a;
  pp.off_c = s.off_c;
  pp.off_f = s.off_f;
  pp.off_ring = s.off_geo;
  pp.slot_bytes = s.slot_bytes;
  const int budget = cfg.nthreads;
  if (budget <= 768) return launch_sf_reg<OP, P, QOFF, 80>(pp, s, plan, tl.n, r.stream);
  if (budget <= 1024) return launch_sf_reg<OP, P, QOFF, 64>(pp, s, plan, tl.n, r.stream);
  if (budget <= 1280) return launch_sf_reg<OP, P, QOFF, 48>(pp, s, plan, tl.n, r.stream);
  return launch_sf_reg<OP, P, QOFF, 40>(pp, s, plan, tl.n, r.stream);
}

template <typename T, int DIM, int OP, int PLO, int PHI, int QOFF, int BK = 0>
spx_status launch_impl(const LaunchReq& r) {
  const spx_plan* plan = r.plan;
  const int dt = r.dtype;
  const LaunchCfg& cfg = plan->cfg[OP][dt];
  const TileList& tl = plan->tiles[OP][dt];
  if (tl.n == 0) return SPX_OK;
  KParams<T, PLO, PHI, QOFF> p{};
  for (int P = PLO; P <= PHI; ++P) {
    if (!plan->present[P]) continue;
    const std::vector<double>& t = plan->tab[P];
    const int off = TabLayout<PLO, PHI, QOFF>::off(P);
    for (int i = 0; i < tab_len(P, QOFF); ++i) p.tab[off + i] = static_cast<T>(t[i]);
  }
  p.tiles = tl.d;
  p.ids = plan->uniform ? nullptr : plan->d_ids;
  p.coef_off = plan->uniform ? nullptr : plan->d_coef_off;
  p.quad_off = plan->uniform ? nullptr : plan->d_quad_off;
  p.in0 = static_cast<const T*>(r.in0);
  p.in1 = static_cast<const T*>(r.in1);
  p.geom = static_cast<const T*>(r.geom);
  p.lam_f = static_cast<const T*>(r.lam_f);
  p.kap_f = static_cast<const T*>(r.kap_f);
  p.out0 = static_cast<T*>(r.out0);
  p.out1 = static_cast<T*>(r.out1);
  p.out2 = static_cast<T*>(r.out2);
  p.status = plan->d_status;
  p.skip = r.skip;
  p.lam = r.lam;
  p.n_tiles = tl.n;
  // stages 0 (3D Helmholtz with Q^2 threads per element): geometry read from L2, one slot for the rest
  p.geo_direct = (OP == OP_HELM && DIM == 3 && BK != 1 && cfg.stages == 0) ? 1 : 0;
  p.stages = cfg.stages < 1 ? 1 : cfg.stages;
  const SmemLayout L = smem_layout(plan, OP, sizeof(T), cfg, r.lam_f != nullptr, r.kap_f != nullptr);
  if (L.total > plan->max_smem)
    return fail(SPX_ERR_UNSUPPORTED, "operator tile needs " + std::to_string(L.total) +
                                         " bytes of shared memory (limit " + std::to_string(plan->max_smem) + ")");
  p.slot_base = L.slot_base;
  p.slot_bytes = L.slot_bytes;
  for (int s = 0; s < 5; ++s) p.region_off[s] = L.region_off[s];
  p.work_base = L.work_base;
  p.work_bytes = L.work_bytes;
  p.meta_base = L.meta_base;
  // 3D Helmholtz bodies with Q^2 threads per element, one order: `nthreads`
  // above 512 selects the 72-register class (more CTAs per SM)
  constexpr bool kRole = OP == OP_HELM && DIM == 3 && BK != 1 && PLO == PHI;
  const bool low_regs = kRole && cfg.nthreads > 512;
  auto kern = op_kernel<T, DIM, OP, PLO, PHI, QOFF, BK>;
  if constexpr (kRole) {
    if (low_regs) kern = op_kernel<T, DIM, OP, PLO, PHI, QOFF, BK, 72>;
  }
  // raise the dynamic shared-memory limit once per kernel
  static std::mutex mu;
  static size_t configured[2] = {0, 0};
  {
    std::lock_guard<std::mutex> g(mu);
    if (L.total > configured[low_regs]) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           static_cast<int>(plan->max_smem));
      if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
      configured[low_regs] = plan->max_smem;
    }
  }
  int nthr = cfg.nthreads;
  if (OP == OP_HELM && DIM == 3 && BK != 1) {  // one thread per quadrature column
    nthr = 0;
    for (int P = PLO; P <= PHI; ++P)
      if (plan->present[P]) nthr = std::max(nthr, cfg.order[P].eb * (P + QOFF) * (P + QOFF));
    nthr = (nthr + 31) / 32 * 32;
    if (nthr > 512) return fail(SPX_ERR_UNSUPPORTED, "Helmholtz tile needs more than 512 threads");
  }
  int nb = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, nthr, L.total);
  if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  if (nb < 1) return fail(SPX_ERR_UNSUPPORTED, "operator tile does not fit on an SM");
  // variable order: one order per CTA, except FP64 (one run over the mixed list; op_kernel.cuh body_of_order)
  constexpr bool kOneRun = std::is_same_v<T, double> && PLO < PHI;
  const int grid = set_runs(p, plan, tl, nb * plan->num_sms, kOneRun, kOneRun ? 1 : nb);
  if (grid < 1) return fail(SPX_ERR_UNSUPPORTED, "tile list has no order runs");
  kern<<<grid, nthr, L.total, r.stream>>>(p);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "operator kernel launch");
  return SPX_OK;
}

// Kernel of one (precision, dimension, operator) over orders PLO..PHI; BK is
// the plan's basis kind (3D Helmholtz: 0 even-odd, 1 generic, 2 collocation).
template <typename T, int DIM, int OP, int PLO, int PHI, int QOFF, int BK = 0>
spx_status launch_any(const LaunchReq& r) {
  if constexpr (std::is_same_v<T, float> && DIM == 3 && OP == OP_HELM && BK == 0) return launch_pair<PLO, PHI, QOFF>(r);
  else if constexpr (std::is_same_v<T, float> && DIM == 3 && (OP == OP_BWD || OP == OP_IPROD) && BK == 0 && PLO == PHI)
    return r.plan->bkind == BK_PARITY ? launch_sf_pair<OP, PLO, QOFF>(r) : launch_impl<T, DIM, OP, PLO, PHI, QOFF, BK>(r);
  else return launch_impl<T, DIM, OP, PLO, PHI, QOFF, BK>(r);
}

template <typename T, int DIM, int OP, int QOFF, int BK = 0>
spx_status launch_uniform(const LaunchReq& r) {
  switch (r.plan->uP) {
    case 1: return launch_any<T, DIM, OP, 1, 1, QOFF, BK>(r);
    case 2: return launch_any<T, DIM, OP, 2, 2, QOFF, BK>(r);
    case 3: return launch_any<T, DIM, OP, 3, 3, QOFF, BK>(r);
    case 4: return launch_any<T, DIM, OP, 4, 4, QOFF, BK>(r);
    case 5: return launch_any<T, DIM, OP, 5, 5, QOFF, BK>(r);
    case 6: return launch_any<T, DIM, OP, 6, 6, QOFF, BK>(r);
    case 7: return launch_any<T, DIM, OP, 7, 7, QOFF, BK>(r);
    case 8: return launch_any<T, DIM, OP, 8, 8, QOFF, BK>(r);
    default: return fail(SPX_ERR_UNSUPPORTED, "order out of range");
  }
}

template <typename T, int DIM, int OP, int BK = 0>
spx_status launch_typed(const LaunchReq& r) {
  if constexpr (BK == 2) {   // collocation: Q = P + 1 only
    if (r.plan->qoff != 1) return fail(SPX_ERR_UNSUPPORTED, "collocation kernel needs q_offset = 1");
    return r.plan->uniform ? launch_uniform<T, DIM, OP, 1, BK>(r) : launch_any<T, DIM, OP, 1, kMaxP, 1, BK>(r);
  } else {
    if (r.plan->uniform) {
      return r.plan->qoff == 1 ? launch_uniform<T, DIM, OP, 1, BK>(r) : launch_uniform<T, DIM, OP, 2, BK>(r);
    }
    return r.plan->qoff == 1 ? launch_any<T, DIM, OP, 1, kMaxP, 1, BK>(r) : launch_any<T, DIM, OP, 1, kMaxP, 2, BK>(r);
  }
}

}  // namespace spx

#define SPX_DEFINE_LAUNCH_(TN, T, DIM, OP) \
  spx_status spx::launch_##TN##_##DIM##_##OP(const spx::LaunchReq& r) { return spx::launch_typed<T, DIM, OP>(r); }
#define SPX_DEFINE_LAUNCH(TN, T, DIM, OP) SPX_DEFINE_LAUNCH_(TN, T, DIM, OP)
// 3D Helmholtz for the other basis kinds (1 generic, 2 collocation)
#define SPX_DEFINE_LAUNCH_BK_(TN, T, BK) \
  spx_status spx::launch_##TN##_helm3_bk##BK(const spx::LaunchReq& r) { return spx::launch_typed<T, 3, spx::OP_HELM, BK>(r); }
#define SPX_DEFINE_LAUNCH_BK(TN, T, BK) SPX_DEFINE_LAUNCH_BK_(TN, T, BK)
