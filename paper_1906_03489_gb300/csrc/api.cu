// C ABI of the spx library: plans, tiles, operator dispatch, autotuning.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "smem_layout.h"
#include "spx_internal.h"

namespace spx {

static thread_local std::string g_last_error;

spx_status fail(spx_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

spx_status cuda_fail(cudaError_t e, const char* what) {
  return fail(SPX_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

static bool op_needs_geom(int op) { return op != OP_BWD; }

static int default_eb(int dim, int Q) {
  const int per = dim == 3 ? Q * Q : Q;
  return std::max(1, std::min(kMaxEB, 256 / per));
}

size_t op_smem_bytes(const spx_plan* plan, int op, int dtype, const LaunchCfg& cfg) {
  if (plan->shape) return collapsed_smem_bytes(plan, dtype, cfg.order[plan->uP].eb);
  if (uses_pair_kernel(plan, op, dtype)) {
    const PairShape s = pair_shape(plan, cfg, pair_threshold(plan, cfg), op);
    return s.nthreads > (op == OP_HELM ? 512 : 1024) ? SIZE_MAX : s.smem;
  }
  // worst case: coefficient fields present
  return smem_layout(plan, op, dtype == 0 ? 8 : 4, cfg, true, true).total;
}

spx_status ensure_tiles(spx_plan* plan, int op, int dtype) {
  TileList& tl = plan->tiles[op][dtype];
  if (!tl.dirty) return SPX_OK;
  const LaunchCfg& cfg = plan->cfg[op][dtype];
  std::vector<Tile> tiles;
  if (plan->uniform) {
    const int eb = cfg.order[plan->uP].eb;
    for (int64_t e0 = 0; e0 < plan->E; e0 += eb)
      tiles.push_back(Tile{plan->uP, static_cast<int32_t>(std::min<int64_t>(eb, plan->E - e0)),
                           static_cast<int32_t>(e0), 1});
  } else {
    // heaviest orders first: round-robin assignment then balances the CTAs
    tl.grp_P.clear();
    tl.grp_tile.clear();
    tl.grp_bytes.clear();
    for (int P = kMaxP; P >= 1; --P) {
      if (!plan->present[P]) continue;
      const int eb = cfg.order[P].eb;
      const int64_t b0 = plan->bucket_start[P], b1 = plan->bucket_start[P + 1];
      const double n = P + 1, Q = P + plan->qoff;
      tl.grp_P.push_back(P);
      tl.grp_tile.push_back(static_cast<int>(tiles.size()));
      tl.grp_bytes.push_back(double(b1 - b0) * (2 * n * n * n + 7 * Q * Q * Q));
      for (int64_t s = b0; s < b1; s += eb) {
        const int cnt = static_cast<int>(std::min<int64_t>(eb, b1 - s));
        bool contig = true;
        for (int j = 1; j < cnt; ++j)
          if (plan->ids[s + j] != plan->ids[s] + j) contig = false;
        tiles.push_back(Tile{P, cnt, static_cast<int32_t>(s), contig ? 1 : 0});
      }
    }
    tl.grp_tile.push_back(static_cast<int>(tiles.size()));
  }
  if (tl.d) cudaFree(tl.d);
  tl.d = nullptr;
  tl.n = static_cast<int>(tiles.size());
  if (tl.n) {
    cudaError_t e = cudaMalloc(&tl.d, tiles.size() * sizeof(Tile));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(tiles)");
    e = cudaMemcpy(tl.d, tiles.data(), tiles.size() * sizeof(Tile), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(tiles)");
  }
  tl.dirty = false;
  return SPX_OK;
}

spx_status launch_op(const LaunchReq& r) {
  if (r.plan->shape) return launch_collapsed(r);
  if (r.op == OP_HELM && r.plan->dim == 3 && r.plan->bkind != BK_PARITY) {
    const bool col = r.plan->bkind == BK_COLLOCATION;
    if (r.dtype == 0) return col ? launch_f64_helm3_bk2(r) : launch_f64_helm3_bk1(r);
    return col ? launch_f32_helm3_bk2(r) : launch_f32_helm3_bk1(r);
  }
  const int key = r.dtype * 100 + r.plan->dim * 10 + r.op;
  switch (key) {
#define SPX_CASE(DT, TN, DIM, OP) \
  case DT * 100 + DIM * 10 + OP: return launch_##TN##_##DIM##_##OP(r);
#define SPX_CASES(DT, TN, DIM) \
  SPX_CASE(DT, TN, DIM, 0) SPX_CASE(DT, TN, DIM, 1) SPX_CASE(DT, TN, DIM, 2) \
  SPX_CASE(DT, TN, DIM, 3) SPX_CASE(DT, TN, DIM, 4) SPX_CASE(DT, TN, DIM, 5) SPX_CASE(DT, TN, DIM, 6) \
  SPX_CASE(DT, TN, DIM, 7)
    SPX_CASES(0, f64, 2)
    SPX_CASES(0, f64, 3)
    SPX_CASES(1, f32, 2)
    SPX_CASES(1, f32, 3)
#undef SPX_CASES
#undef SPX_CASE
    default: return fail(SPX_ERR_UNSUPPORTED, "no kernel for this operator");
  }
}

// Helmholtz apply for the solver (spx_internal.h).
spx_status helmholtz_unless(const spx_plan* cp, int dtype, double lambda, const void* in, void* out, const int* skip,
                            cudaStream_t stream) {
  spx_plan* p = const_cast<spx_plan*>(cp);
  if (p->E == 0) return SPX_OK;
  const void* geom = p->geom[dtype];
  if (!geom) return fail(SPX_ERR_INVALID_ARG, "geometry not registered for this dtype");
  spx_status s = ensure_tiles(p, OP_HELM, dtype);
  if (s != SPX_OK) return s;
  LaunchReq r{p, OP_HELM, dtype, in, nullptr, geom, nullptr, nullptr, out, nullptr, nullptr, lambda, stream, skip};
  return launch_op(r);
}
// Caller-supplied basis tables (spx_basis_desc): copied into the plan's
// per-order tables after checks against the GLL quadrature, then classified
// for the 3D Helmholtz kernels (BasisKind).  Host-memory tables are checked
// before any device call.
static spx_status load_basis(spx_plan* p, const spx_plan_desc* d) {
  if (d->n_basis == 0) return SPX_OK;
  if (d->n_basis < 0 || d->n_basis > 64 || !d->basis)
    return fail(SPX_ERR_INVALID_ARG, "plan_create: n_basis must be 0..64 with a basis array");
  if (d->basis_memory != SPX_MEM_HOST && d->basis_memory != SPX_MEM_DEVICE)
    return fail(SPX_ERR_INVALID_ARG, "plan_create: basis_memory must be SPX_MEM_HOST or SPX_MEM_DEVICE");
  bool given[kMaxP1] = {};
  auto fetch = [&](const double* src, size_t count, std::vector<double>& dst) -> spx_status {
    dst.resize(count);
    if (d->basis_memory == SPX_MEM_HOST) {
      std::memcpy(dst.data(), src, count * sizeof(double));
      return SPX_OK;
    }
    const cudaError_t e = cudaMemcpy(dst.data(), src, count * sizeof(double), cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? SPX_OK : cuda_fail(e, "plan_create: cudaMemcpy(basis tables)");
  };
  for (int t = 0; t < d->n_basis; ++t) {
    const spx_basis_desc& b = d->basis[t];
    if (b.P < 1 || b.P > kMaxP) return fail(SPX_ERR_INVALID_ARG, "plan_create: basis order outside 1..8");
    if (given[b.P]) return fail(SPX_ERR_INVALID_ARG, "plan_create: two basis descriptions for one order");
    given[b.P] = true;
    const int P = b.P, n = P + 1, Q = P + p->qoff;
    if (b.Q != Q) return fail(SPX_ERR_INVALID_ARG, "plan_create: basis Q must equal P + q_offset");
    if (!b.B) return fail(SPX_ERR_INVALID_ARG, "plan_create: basis table B is required");
    std::vector<double> B, dB, D, w;
    spx_status st;
    if ((st = fetch(b.B, size_t(Q) * n, B)) != SPX_OK) return st;
    double bmax = 0.0;
    for (double v : B) {
      if (!std::isfinite(v)) return fail(SPX_ERR_INVALID_ARG, "plan_create: basis table B not finite");
      bmax = std::max(bmax, std::fabs(v));
    }
    if (bmax == 0.0) return fail(SPX_ERR_INVALID_ARG, "plan_create: basis table B is zero");
    std::vector<double>& tab = p->tab[P];   // holds the library's GLL tables of this order
    const double* Dg = tab.data() + 2 * Q * n;
    std::vector<double> wg(Q);
    basis_tables(P, Q, nullptr, wg.data(), nullptr, nullptr, nullptr);
    if (b.D) {
      if ((st = fetch(b.D, size_t(Q) * Q, D)) != SPX_OK) return st;
      double dm = 0.0;
      for (int i = 0; i < Q * Q; ++i) dm = std::max(dm, std::fabs(Dg[i]));
      for (int i = 0; i < Q * Q; ++i)
        if (!(std::fabs(D[i] - Dg[i]) <= 1e-12 * dm))
          return fail(SPX_ERR_UNSUPPORTED, "plan_create: D must be the GLL collocation derivative (the quadrature "
                                           "is the GLL rule the geometric factors are built on)");
    }
    if (b.w) {
      if ((st = fetch(b.w, size_t(Q), w)) != SPX_OK) return st;
      for (int i = 0; i < Q; ++i)
        if (!(std::fabs(w[i] - wg[i]) <= 1e-12 * 2.0))
          return fail(SPX_ERR_UNSUPPORTED, "plan_create: w must be the GLL weights (the quadrature is the GLL "
                                           "rule the geometric factors are built on)");
    }
    // dB as the kernels use it: D B (exact for P <= Q - 1)
    std::vector<double> DB(size_t(Q) * n, 0.0);
    for (int i = 0; i < Q; ++i)
      for (int q = 0; q < n; ++q) {
        double acc = 0.0;
        for (int j = 0; j < Q; ++j) acc += Dg[i * Q + j] * B[j * n + q];
        DB[i * n + q] = acc;
      }
    if (b.dB) {
      if ((st = fetch(b.dB, size_t(Q) * n, dB)) != SPX_OK) return st;
      double dm = 0.0;
      for (double v : DB) dm = std::max(dm, std::fabs(v));
      for (int i = 0; i < Q * n; ++i)
        if (!(std::fabs(dB[i] - DB[i]) <= 1e-10 * std::max(dm, bmax)))
          return fail(SPX_ERR_INVALID_ARG, "plan_create: dB must be the derivative of B (D B to 1e-10)");
      DB = dB;
    }
    // differs from the library's modified basis?
    for (int i = 0; i < Q * n; ++i)
      if (std::fabs(B[i] - tab[i]) > 1e-15 * bmax) p->custom_basis = true;
    std::copy(B.begin(), B.end(), tab.begin());
    std::copy(DB.begin(), DB.end(), tab.begin() + Q * n);
    eo_tables(P, Q, tab.data());
  }
  for (int P = 1; P <= kMaxP; ++P)
    if (p->present[P] && !given[P])
      return fail(SPX_ERR_INVALID_ARG, "plan_create: no basis description for an order present in the mesh");
  if (!p->custom_basis) return SPX_OK;
  // classification over the orders present
  bool parity = true, ident = true;
  for (int P = 1; P <= kMaxP; ++P) {
    if (!p->present[P]) continue;
    const int n = P + 1, Q = P + p->qoff;
    const double* B = p->tab[P].data();
    double bmax = 0.0;
    for (int i = 0; i < Q * n; ++i) bmax = std::max(bmax, std::fabs(B[i]));
    const double tol = 1e-13 * bmax;
    for (int i = 0; i < Q; ++i) {
      const double* r = B + i * n;
      const double* m = B + (Q - 1 - i) * n;   // mirrored point
      if (std::fabs(m[0] - r[P]) > tol || std::fabs(m[P] - r[0]) > tol) parity = false;
      for (int q = 1; q < P; ++q)
        if (std::fabs(m[q] - ((q - 1) % 2 ? -r[q] : r[q])) > tol) parity = false;
      for (int q = 0; q < n; ++q)
        if (Q != n || std::fabs(r[q] - (q == i ? 1.0 : 0.0)) > 1e-14) ident = false;
    }
  }
  p->bkind = parity ? BK_PARITY : (ident ? BK_COLLOCATION : BK_GENERAL);
  return SPX_OK;
}

}  // namespace spx

using namespace spx;

extern "C" {

const char* spx_last_error(void) { return g_last_error.c_str(); }

const char* spx_version(void) { return "spx 0.1 (sm_103a)"; }

spx_status spx_basis_tables(int P, int Q, double* xi, double* w, double* B, double* dB, double* D) {
  return basis_tables(P, Q, xi, w, B, dB, D);
}

spx_status spx_nodal_basis_tables(int P, int Q, double* B, double* dB) { return nodal_basis_tables(P, Q, B, dB); }

spx_status spx_gauss_radau(int Q, double* x, double* w) {
  if (!x || !w) return fail(SPX_ERR_INVALID_ARG, "gauss_radau: NULL output");
  return gauss_radau(Q, x, w);
}

spx_status spx_plan_create(spx_plan** out, const spx_plan_desc* d) {
  if (!out || !d) return fail(SPX_ERR_INVALID_ARG, "plan_create: NULL argument");
  *out = nullptr;
  if (d->dim != 2 && d->dim != 3) return fail(SPX_ERR_INVALID_ARG, "plan_create: dim must be 2 or 3");
  if (d->n_elem < 0 || d->n_elem > (int64_t(1) << 31) - 1)
    return fail(SPX_ERR_INVALID_ARG, "plan_create: n_elem out of range");
  const int qoff = d->q_offset == 0 ? 2 : d->q_offset;
  if (qoff != 1 && qoff != 2) return fail(SPX_ERR_UNSUPPORTED, "plan_create: q_offset must be 1 or 2");
  if (d->shape != SPX_SHAPE_TENSOR && d->shape != SPX_SHAPE_TRI && d->shape != SPX_SHAPE_PRISM &&
      d->shape != SPX_SHAPE_TET)
    return fail(SPX_ERR_INVALID_ARG, "plan_create: unknown element shape");
  if (d->shape != SPX_SHAPE_TENSOR) {
    if ((d->shape == SPX_SHAPE_TRI) != (d->dim == 2))
      return fail(SPX_ERR_INVALID_ARG, "plan_create: triangles are 2D, prisms and tetrahedra 3D");
    if (d->elem_order || qoff != 2 || d->n_basis)
      return fail(SPX_ERR_UNSUPPORTED, "plan_create: triangles / prisms take a uniform order, q_offset 2 and the "
                                       "library's basis");
  }
  spx_plan* p = new (std::nothrow) spx_plan();
  if (!p) return fail(SPX_ERR_NO_MEMORY, "plan_create: out of host memory");
  p->dim = d->dim;
  p->E = d->n_elem;
  p->qoff = qoff;
  p->shape = d->shape;
  p->orders.resize(p->E);
  if (d->elem_order) {
    for (int64_t e = 0; e < p->E; ++e) {
      const int P = d->elem_order[e];
      if (P < 1 || P > kMaxP) {
        delete p;
        return fail(SPX_ERR_INVALID_ARG, "plan_create: element order outside 1..8");
      }
      p->orders[e] = P;
    }
  } else {
    if (d->uniform_order < 1 || d->uniform_order > kMaxP) {
      delete p;
      return fail(SPX_ERR_INVALID_ARG, "plan_create: uniform_order outside 1..8");
    }
    std::fill(p->orders.begin(), p->orders.end(), d->uniform_order);
  }
  for (int64_t e = 0; e < p->E; ++e) p->present[p->orders[e]] = true;
  int npresent = 0;
  for (int P = 1; P <= kMaxP; ++P) npresent += p->present[P];
  p->uniform = npresent <= 1;
  p->uP = d->elem_order ? (p->E ? p->orders[0] : 1) : d->uniform_order;
  if (p->E == 0) p->present[p->uP] = true;
  p->coef_off.resize(p->E + 1);
  p->quad_off.resize(p->E + 1);
  p->coef_off[0] = p->quad_off[0] = 0;
  for (int64_t e = 0; e < p->E; ++e) {
    const int64_t n = p->orders[e] + 1, Q = p->orders[e] + qoff;
    const int64_t nt = n * (n + 1) / 2;   // triangle modes
    const int64_t nm = p->shape == SPX_SHAPE_TRI     ? nt
                       : p->shape == SPX_SHAPE_PRISM ? n * nt
                       : p->shape == SPX_SHAPE_TET   ? n * (n + 1) * (n + 2) / 6
                                                     : (p->dim == 3 ? n * n * n : n * n);
    p->coef_off[e + 1] = p->coef_off[e] + nm;
    p->quad_off[e + 1] = p->quad_off[e] + (p->dim == 3 ? Q * Q * Q : Q * Q);
  }
  if (p->shape) {   // tables of the collapsed kernels: B1[Q][n], Bb[n][Q][n], D1[Q][Q], D2[Q][Q], Bc[n][Q][n]
    const int P = p->uP, n = P + 1, Q = P + 2;
    p->ctab.assign(Q * n + 2 * n * Q * n + 2 * Q * Q, 0.0);
    double* t = p->ctab.data();
    const spx_status cs = collapsed_tables(P, Q, t, t + Q * n, t + Q * n + n * Q * n, t + Q * n + n * Q * n + Q * Q,
                                           nullptr, nullptr, nullptr, nullptr, t + Q * n + n * Q * n + 2 * Q * Q);
    if (cs != SPX_OK) {
      delete p;
      return cs;
    }
  }
  p->n_coef = p->coef_off[p->E];
  p->n_quad = p->quad_off[p->E];
  for (int P = 1; P <= kMaxP; ++P) {
    const int Q = P + qoff, n = P + 1;
    p->tab[P].assign(tab_len(P, qoff), 0.0);
    basis_tables(P, Q, nullptr, nullptr, p->tab[P].data(), p->tab[P].data() + Q * n, p->tab[P].data() + 2 * Q * n);
    eo_tables(P, Q, p->tab[P].data());
  }
  {
    const spx_status bs = load_basis(p, d);
    if (bs != SPX_OK) {
      delete p;
      return bs;
    }
  }
  cudaError_t e = cudaGetDevice(&p->device);
  if (e != cudaSuccess) {
    delete p;
    return cuda_fail(e, "cudaGetDevice");
  }
  cudaDeviceProp prop;
  e = cudaGetDeviceProperties(&prop, p->device);
  if (e != cudaSuccess) {
    delete p;
    return cuda_fail(e, "cudaGetDeviceProperties");
  }
  p->num_sms = prop.multiProcessorCount;
  p->max_smem = prop.sharedMemPerBlockOptin;
  p->smem_per_sm = prop.sharedMemPerMultiprocessor;
  // device metadata
  auto cleanup = [&](cudaError_t err, const char* what) {
    spx_plan_destroy(p);
    return cuda_fail(err, what);
  };
  if ((e = cudaMalloc(&p->d_status, sizeof(int))) != cudaSuccess) return cleanup(e, "cudaMalloc(status)");
  if ((e = cudaMemset(p->d_status, 0, sizeof(int))) != cudaSuccess) return cleanup(e, "cudaMemset(status)");
  {  // inverse 1D mass matrices of every order (FwdTrans preconditioner)
    // full inverses of orders 1..8, then the sensor's restricted ones (order 1: unused zeros)
    std::vector<double> a64(2 * mass1d_off(kMaxP + 1), 0.0);
    for (int P = 1; P <= kMaxP; ++P) {
      mass1d_inverse(P, P + qoff, p->tab[P].data(), a64.data() + mass1d_off(P));
      if (P >= 2 && !p->custom_basis)   // the restricted space is the modified basis's (sensor)
        mass1d_inverse(P, P + qoff, p->tab[P].data(), a64.data() + mass1d_off(kMaxP + 1) + mass1d_off(P), true);
    }
    std::vector<float> a32(a64.begin(), a64.end());
    if ((e = cudaMalloc(&p->d_aux64, a64.size() * sizeof(double))) != cudaSuccess) return cleanup(e, "cudaMalloc(aux)");
    if ((e = cudaMalloc(&p->d_aux32, a32.size() * sizeof(float))) != cudaSuccess) return cleanup(e, "cudaMalloc(aux)");
    if ((e = cudaMemcpy(p->d_aux64, a64.data(), a64.size() * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(p->d_aux32, a32.data(), a32.size() * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess)
      return cleanup(e, "cudaMemcpy(aux)");
    if ((e = cudaMalloc(&p->d_partials, size_t(p->num_sms) * kIntegralBlocksPerSM * sizeof(double))) != cudaSuccess)
      return cleanup(e, "cudaMalloc(partials)");
    if ((e = cudaMalloc(&p->d_ticket, sizeof(unsigned int))) != cudaSuccess) return cleanup(e, "cudaMalloc(ticket)");
    if ((e = cudaMemset(p->d_ticket, 0, sizeof(unsigned int))) != cudaSuccess) return cleanup(e, "cudaMemset(ticket)");
  }
  if (!p->uniform) {
    p->bucket_start.assign(kMaxP + 2, 0);
    for (int64_t i = 0; i < p->E; ++i) p->bucket_start[p->orders[i] + 1]++;
    for (int P = 1; P <= kMaxP + 1; ++P) p->bucket_start[P] += p->bucket_start[P - 1];
    p->ids.resize(p->E);
    std::vector<int64_t> fill(p->bucket_start.begin(), p->bucket_start.end());
    for (int64_t i = 0; i < p->E; ++i) p->ids[fill[p->orders[i]]++] = static_cast<int32_t>(i);
    if ((e = cudaMalloc(&p->d_ids, p->E * sizeof(int32_t))) != cudaSuccess) return cleanup(e, "cudaMalloc(ids)");
    if ((e = cudaMalloc(&p->d_coef_off, (p->E + 1) * sizeof(int64_t))) != cudaSuccess)
      return cleanup(e, "cudaMalloc(coef_off)");
    if ((e = cudaMalloc(&p->d_quad_off, (p->E + 1) * sizeof(int64_t))) != cudaSuccess)
      return cleanup(e, "cudaMalloc(quad_off)");
    e = cudaMemcpy(p->d_ids, p->ids.data(), p->E * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(p->d_coef_off, p->coef_off.data(), (p->E + 1) * sizeof(int64_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(p->d_quad_off, p->quad_off.data(), (p->E + 1) * sizeof(int64_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cleanup(e, "cudaMemcpy(plan metadata)");
  }
  {  // the allocation-free solver's workspace: reserved here (module load), not inside a solve
    void* ws = nullptr;
    const spx_status st = noalloc_workspace(&ws);
    if (st != SPX_OK) {
      spx_plan_destroy(p);
      return st;
    }
  }
  // default tiles: fit shared memory with 2 stages
  for (int op = 0; op < OP_KINDS; ++op) {
    for (int dt = 0; dt < 2; ++dt) {
      LaunchCfg& c = p->cfg[op][dt];
      c.nthreads = 256;
      c.stages = 2;
      for (int P = 1; P <= kMaxP; ++P) c.order[P].eb = default_eb(p->dim, P + qoff);
      for (int P = 1; P <= kMaxP; ++P) {
        if (!p->present[P]) continue;
        while (c.order[P].eb > 1 && op_smem_bytes(p, op, dt, c) > p->max_smem) c.order[P].eb /= 2;
      }
    }
  }
  *out = p;
  return SPX_OK;
}

spx_status spx_plan_destroy(spx_plan* p) {
  if (!p) return SPX_OK;
  for (int op = 0; op < OP_KINDS; ++op)
    for (int dt = 0; dt < 2; ++dt)
      if (p->tiles[op][dt].d) cudaFree(p->tiles[op][dt].d);
  if (p->d_ids) cudaFree(p->d_ids);
  if (p->d_coef_off) cudaFree(p->d_coef_off);
  if (p->d_quad_off) cudaFree(p->d_quad_off);
  if (p->d_status) cudaFree(p->d_status);
  if (p->d_aux64) cudaFree(p->d_aux64);
  if (p->d_aux32) cudaFree(p->d_aux32);
  if (p->d_partials) cudaFree(p->d_partials);
  if (p->d_ticket) cudaFree(p->d_ticket);
  delete p;
  return SPX_OK;
}

spx_status spx_plan_sizes(const spx_plan* p, int64_t* n_coef, int64_t* n_quad) {
  if (!p) return fail(SPX_ERR_INVALID_ARG, "plan_sizes: NULL plan");
  if (n_coef) *n_coef = p->n_coef;
  if (n_quad) *n_quad = p->n_quad;
  return SPX_OK;
}

spx_status spx_plan_offsets(const spx_plan* p, int64_t* coef_off, int64_t* quad_off) {
  if (!p) return fail(SPX_ERR_INVALID_ARG, "plan_offsets: NULL plan");
  if (coef_off) std::memcpy(coef_off, p->coef_off.data(), (p->E + 1) * sizeof(int64_t));
  if (quad_off) std::memcpy(quad_off, p->quad_off.data(), (p->E + 1) * sizeof(int64_t));
  return SPX_OK;
}

spx_status spx_plan_set_geometry(spx_plan* p, spx_dtype dt, const void* geom, const void* dxi) {
  if (!p) return fail(SPX_ERR_INVALID_ARG, "set_geometry: NULL plan");
  if (dt != SPX_F64 && dt != SPX_F32) return fail(SPX_ERR_INVALID_ARG, "set_geometry: bad dtype");
  p->geom[dt] = geom;
  p->dxi[dt] = dxi;
  return SPX_OK;
}

spx_status spx_plan_device_status(spx_plan* p, int* status, int reset) {
  if (!p || !status) return fail(SPX_ERR_INVALID_ARG, "plan_device_status: NULL argument");
  cudaError_t e = cudaMemcpy(status, p->d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(status)");
  if (reset && (e = cudaMemset(p->d_status, 0, sizeof(int))) != cudaSuccess) return cuda_fail(e, "cudaMemset");
  return SPX_OK;
}

spx_status spx_plan_set_tile(spx_plan* p, spx_op op, spx_dtype dt, int order, int eb, int nthreads, int stages) {
  if (!p) return fail(SPX_ERR_INVALID_ARG, "set_tile: NULL plan");
  if (op < 0 || op >= OP_KINDS || (dt != SPX_F64 && dt != SPX_F32))
    return fail(SPX_ERR_INVALID_ARG, "set_tile: bad operator or dtype");
  // pair kernels: nthreads is the threads-per-SM class of the register budget
  // stages 0: the FP32 3D pair kernel's L2 prefetch distance, or the other 3D
  // Helmholtz bodies with Q^2 threads per element reading geometry from L2
  const bool role3 = op == OP_HELM && p->dim == 3 && p->bkind != BK_GENERAL && !p->shape;
  const int max_nt = uses_pair_kernel(p, op, dt) ? (op == OP_HELM ? 1024 : 2048) : (role3 ? 1024 : 512);
  const int min_st = (uses_pair_kernel(p, op, dt) || role3) ? 0 : 1;
  if (eb < 1 || eb > kMaxEB || nthreads < 32 || nthreads > max_nt || nthreads % 32 || stages < min_st || stages > 4)
    return fail(SPX_ERR_INVALID_ARG, "set_tile: eb 1..64, nthreads 32..512 (3D Helmholtz: 1024; FP32 BwdTrans / "
                                     "IProductWRTBase pair kernels of one order: 2048), multiple of 32, stages 1..4 "
                                     "(0..4 for the 3D Helmholtz and the pair kernels)");
  if (order != -1 && (order < 1 || order > kMaxP)) return fail(SPX_ERR_INVALID_ARG, "set_tile: order outside 1..8");
  LaunchCfg c = p->cfg[op][dt];
  c.nthreads = nthreads;
  c.stages = stages;
  for (int P = 1; P <= kMaxP; ++P)
    if (order == -1 || order == P) c.order[P].eb = eb;
  if (op_smem_bytes(p, op, dt, c) > p->max_smem)
    return fail(SPX_ERR_UNSUPPORTED, "set_tile: tile does not fit in shared memory");
  p->cfg[op][dt] = c;
  p->tiles[op][dt].dirty = true;
  return ensure_tiles(p, op, dt);
}

spx_status spx_plan_get_tile(const spx_plan* p, spx_op op, spx_dtype dt, int order, int* eb, int* nthreads,
                             int* stages) {
  if (!p || op < 0 || op >= OP_KINDS || (dt != SPX_F64 && dt != SPX_F32) || order < 1 || order > kMaxP)
    return fail(SPX_ERR_INVALID_ARG, "get_tile: bad argument");
  const LaunchCfg& c = p->cfg[op][dt];
  if (eb) *eb = c.order[order].eb;
  if (nthreads) *nthreads = c.nthreads;
  if (stages) *stages = c.stages;
  return SPX_OK;
}

// ---------------------------------------------------------------------------
static spx_status run_op(const spx_plan* cp, int op, spx_dtype dt, const void* in0, const void* in1,
                         const void* lam_f, const void* kap_f, void* o0, void* o1, void* o2, double lam,
                         void* stream) {
  spx_plan* p = const_cast<spx_plan*>(cp);
  if (!p) return fail(SPX_ERR_INVALID_ARG, "NULL plan");
  if (dt != SPX_F64 && dt != SPX_F32) return fail(SPX_ERR_INVALID_ARG, "bad dtype");
  if (p->E == 0) return SPX_OK;
  const void* geom = op == OP_DERIV ? p->dxi[dt] : p->geom[dt];
  if (op_needs_geom(op) && !geom)
    return fail(SPX_ERR_INVALID_ARG, op == OP_DERIV ? "dxi_dx not registered for this dtype"
                                                    : "geometry not registered for this dtype");
  const size_t a = dt == SPX_F64 ? 8 : 4;
  const void* ptrs[] = {in0, in1, lam_f, kap_f, o0, o1, o2};
  for (const void* q : ptrs)
    if (q && (reinterpret_cast<uintptr_t>(q) % a)) return fail(SPX_ERR_INVALID_ARG, "buffer not aligned to its element size");
  if (p->shape && op != OP_BWD && op != OP_IPROD && op != OP_DERIV && op != OP_HELM)
    return fail(SPX_ERR_UNSUPPORTED, "operator not available for triangles / prisms");
  spx_status s = ensure_tiles(p, op, dt);
  if (s != SPX_OK) return s;
  LaunchReq r{p, op, dt, in0, in1, geom, lam_f, kap_f, o0, o1, o2, lam, static_cast<cudaStream_t>(stream)};
  return launch_op(r);
}

spx_status spx_bwd_trans(const spx_plan* p, spx_dtype dt, const void* coef, void* phys, void* stream) {
  if (p && p->E && (!coef || !phys)) return fail(SPX_ERR_INVALID_ARG, "bwd_trans: NULL buffer");
  return run_op(p, OP_BWD, dt, coef, nullptr, nullptr, nullptr, phys, nullptr, nullptr, 0.0, stream);
}

spx_status spx_iproduct(const spx_plan* p, spx_dtype dt, const void* phys, void* coef, void* stream) {
  if (p && p->E && (!coef || !phys)) return fail(SPX_ERR_INVALID_ARG, "iproduct: NULL buffer");
  return run_op(p, OP_IPROD, dt, phys, nullptr, nullptr, nullptr, coef, nullptr, nullptr, 0.0, stream);
}

spx_status spx_phys_deriv(const spx_plan* p, spx_dtype dt, const void* phys, void* d0, void* d1, void* d2,
                          void* stream) {
  if (p && p->E && (!phys || !d0 || !d1 || (p->dim == 3 && !d2)))
    return fail(SPX_ERR_INVALID_ARG, "phys_deriv: NULL buffer");
  return run_op(p, OP_DERIV, dt, phys, nullptr, nullptr, nullptr, d0, d1, p && p->dim == 3 ? d2 : nullptr, 0.0,
                stream);
}

spx_status spx_helmholtz(const spx_plan* p, spx_dtype dt, double lambda, const void* lam_f, const void* kap_f,
                         const void* in, void* out, void* stream) {
  if (p && p->E && (!in || !out)) return fail(SPX_ERR_INVALID_ARG, "helmholtz: NULL buffer");
  if (in && in == out) return fail(SPX_ERR_INVALID_ARG, "helmholtz: coef_out must not alias coef_in");
  if (!std::isfinite(lambda)) return fail(SPX_ERR_INVALID_ARG, "helmholtz: lambda not finite");
  return run_op(p, OP_HELM, dt, in, nullptr, lam_f, kap_f, out, nullptr, nullptr, lambda, stream);
}

spx_status spx_helmholtz_adjoint(const spx_plan* p, const double* u, const double* g, double* glam, double* gkap,
                                 void* stream) {
  if (p && p->E && (!u || !g)) return fail(SPX_ERR_INVALID_ARG, "helmholtz_adjoint: NULL input");
  if (!glam && !gkap) return SPX_OK;
  return run_op(p, OP_ADJ, SPX_F64, u, g, nullptr, nullptr, glam, gkap, nullptr, 0.0, stream);
}

spx_status spx_fwd_trans(const spx_plan* p, spx_dtype dt, const void* phys, void* coef, void* stream) {
  if (dt == SPX_F32)
    return fail(SPX_ERR_UNSUPPORTED, "fwd_trans: FP32 is refused: the elemental mass matrix's condition number "
                                     "(about 4e7 at P = 4 in 3D) exceeds FP32's 1 / epsilon, so no FP32 solve "
                                     "reaches the FP32 operator tolerance; use SPX_F64");
  if (p && p->E && (!coef || !phys)) return fail(SPX_ERR_INVALID_ARG, "fwd_trans: NULL buffer");
  if (p && phys && phys == coef) return fail(SPX_ERR_INVALID_ARG, "fwd_trans: coef must not alias phys");
  const void* aux = !p ? nullptr : (dt == SPX_F64 ? static_cast<const void*>(p->d_aux64) : p->d_aux32);
  return run_op(p, OP_FWD, dt, phys, aux, nullptr, nullptr, coef, nullptr, nullptr, 0.0, stream);
}

spx_status spx_sensor(const spx_plan* p, const double* coef, double* S, void* stream) {
  if (p && p->E && (!coef || !S)) return fail(SPX_ERR_INVALID_ARG, "sensor: NULL buffer");
  if (p && p->present[1]) return fail(SPX_ERR_UNSUPPORTED, "sensor: elements of order 1 (the sensor needs P >= 2)");
  if (p && p->custom_basis)
    return fail(SPX_ERR_UNSUPPORTED, "sensor: needs the library's modified basis (its top bubble spans degree P)");
  return run_op(p, OP_SENSOR, SPX_F64, coef, p ? p->d_aux64 : nullptr, nullptr, nullptr, S, nullptr, nullptr, 0.0,
                stream);
}

spx_status spx_adapt_orders(int64_t n_elem, const double* S, const int32_t* orders, double lower, double upper,
                            int p_min, int p_max, int32_t* new_orders) {
  if (n_elem < 0 || (n_elem && (!S || !orders || !new_orders)))
    return fail(SPX_ERR_INVALID_ARG, "adapt_orders: bad argument");
  if (p_min < 2 || p_max > kMaxP || p_min > p_max || !(lower <= upper))
    return fail(SPX_ERR_INVALID_ARG, "adapt_orders: need 2 <= p_min <= p_max <= 8 and lower <= upper");
  for (int64_t e = 0; e < n_elem; ++e) {
    int P = orders[e];
    if (S[e] > upper) ++P;
    else if (S[e] < lower) --P;
    new_orders[e] = std::min(p_max, std::max(p_min, P));
  }
  return SPX_OK;
}

spx_status spx_helmholtz_diag(const spx_plan* p, spx_dtype dt, double lambda, void* out, void* stream) {
  if (p && p->E && !out) return fail(SPX_ERR_INVALID_ARG, "helmholtz_diag: NULL buffer");
  return run_op(p, OP_DIAG, dt, nullptr, nullptr, nullptr, nullptr, out, nullptr, nullptr, lambda, stream);
}

// ---------------------------------------------------------------------------
// Autotuning (§3.3: the fastest strategy is picked at start-up).
// ---------------------------------------------------------------------------
// Reads a buffer larger than the L2 (16-byte words, cached in L2 only), so
// that the next launch finds none of its operands there; the lines it leaves
// are clean (no write-back charged to the timed launch).  The buffer is
// zeroed, so the sink is never written.
__global__ void l2_evict_kernel(const uint4* __restrict__ buf, size_t n, unsigned* sink) {
  unsigned x = 0;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) {
    const uint4 v = __ldcg(buf + i);
    x ^= v.x ^ v.y ^ v.z ^ v.w;
  }
  if (x == 0x9e3779b9u) *sink = x;
}

// Device buffer of twice the L2 for l2_evict_kernel, held for one autotune call.
struct EvictBuf {
  uint4* d = nullptr;
  size_t n = 0;
  ~EvictBuf() {
    if (d) cudaFree(d);
  }
  spx_status init(cudaStream_t st) {
    int dev = 0, l2 = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
    if (e != cudaSuccess) return cuda_fail(e, "autotune: L2 size");
    n = 2 * size_t(std::max(l2, 1 << 20)) / sizeof(uint4);
    if ((e = cudaMalloc(&d, (n + 1) * sizeof(uint4))) != cudaSuccess) return cuda_fail(e, "cudaMalloc(evict)");
    if ((e = cudaMemsetAsync(d, 0, (n + 1) * sizeof(uint4), st)) != cudaSuccess) return cuda_fail(e, "cudaMemset");
    return SPX_OK;
  }
  void evict(int num_sms, cudaStream_t st) const {
    l2_evict_kernel<<<num_sms * 4, 512, 0, st>>>(d, n, reinterpret_cast<unsigned*>(d + n));
  }
};

// Mean time of one launch with the L2 evicted before each (the operands of
// a streaming operator then come from HBM, as on a mesh larger than the L2).
static float time_op(spx_plan* p, int op, spx_dtype dt, const void* in, void* out, int reps, cudaStream_t st,
                     const EvictBuf& ev, spx_status* err) {
  void* o[3] = {out, nullptr, nullptr};
  const void* in1 = nullptr;
  size_t qbytes = (dt == SPX_F64 ? 8 : 4) * static_cast<size_t>(p->n_quad);
  if (op == OP_DERIV) {  // three outputs packed in `out`
    o[1] = static_cast<char*>(out) + qbytes;
    o[2] = p->dim == 3 ? static_cast<char*>(out) + 2 * qbytes : nullptr;
  }
  if (op == OP_FWD || op == OP_SENSOR) in1 = dt == SPX_F64 ? static_cast<const void*>(p->d_aux64) : p->d_aux32;
  if (op == OP_ADJ) {
    in1 = in;
    o[1] = static_cast<char*>(out) + qbytes;
  }
  std::vector<cudaEvent_t> ev0(reps), ev1(reps);
  for (int i = 0; i < reps; ++i) {
    cudaEventCreate(&ev0[i]);
    cudaEventCreate(&ev1[i]);
  }
  *err = run_op(p, op, dt, in, in1, nullptr, nullptr, o[0], o[1], o[2], 1.0, st);  // warm-up
  for (int i = 0; i < reps && *err == SPX_OK; ++i) {
    ev.evict(p->num_sms, st);
    cudaEventRecord(ev0[i], st);
    *err = run_op(p, op, dt, in, in1, nullptr, nullptr, o[0], o[1], o[2], 1.0, st);
    cudaEventRecord(ev1[i], st);
  }
  cudaError_t ce = cudaEventSynchronize(ev1[reps - 1]);
  float total = 0.f;
  for (int i = 0; i < reps; ++i) {
    float ms = 0.f;
    if (ce == cudaSuccess && *err == SPX_OK) cudaEventElapsedTime(&ms, ev0[i], ev1[i]);
    total += ms;
    cudaEventDestroy(ev0[i]);
    cudaEventDestroy(ev1[i]);
  }
  if (ce != cudaSuccess && *err == SPX_OK) *err = cuda_fail(ce, "autotune timing");
  return total / reps;
}

// Threads (compute threads plus the producer warp of the variable-order FP32
// Helmholtz kernel) and shared memory of a CTA whose largest tile is order
// P's, with eb elements (every other order at one element).
static void tile_footprint(const spx_plan* p, int op, int dt, const LaunchCfg& base, int P, int eb, int* thr,
                           size_t* smem) {
  LaunchCfg c = base;
  for (int o = 1; o <= kMaxP; ++o) c.order[o].eb = 1;
  c.order[P].eb = eb;
  const int Q = P + p->qoff;
  if (uses_pair_kernel(p, op, dt)) {
    const PairShape s = pair_shape(p, c, pair_threshold(p, c), op);
    *thr = s.nthreads + (p->uniform ? 0 : 32);
    *smem = s.smem;
  } else {
    *thr = (op == OP_HELM && p->dim == 3 && p->bkind != BK_GENERAL && !p->shape) ? (eb * Q * Q + 31) / 32 * 32
                                                                                  : c.nthreads;
    *smem = op_smem_bytes(p, op, dt, c);
  }
}

spx_status spx_autotune(spx_plan* p, spx_op op, spx_dtype dt, const void* in, void* out, int reps, void* stream) {
  if (!p || !in || !out || op < 0 || op >= SPX_OP_COUNT || (dt != SPX_F64 && dt != SPX_F32) || reps < 1)
    return fail(SPX_ERR_INVALID_ARG, "autotune: bad argument");
  if (p->E == 0) return SPX_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  EvictBuf ev;
  if (spx_status es = ev.init(st); es != SPX_OK) return es;
  const int ebs[] = {1, 2, 3, 4, 5, 6, 7, 8, 12, 16, 24, 32};
  const bool pair = uses_pair_kernel(p, op, dt);
  // bodies with Q^2 threads per element take their block size from eb
  const bool role = op == OP_HELM && p->dim == 3 && p->bkind != BK_GENERAL && !pair && !p->shape;
  // the pair kernels derive their CTA size from eb: there `nthreads` picks the
  // register budget (threads per SM) and `stages` the L2 prefetch distance
  const bool sf = pair && (op == OP_BWD || op == OP_IPROD);
  const std::vector<int> nts = sf     ? std::vector<int>{768, 1024, 1280, 1536}
                               : pair ? std::vector<int>{512, 640, 768}
                                      : (role ? (p->uniform ? std::vector<int>{512, 896} : std::vector<int>{512})
                                              : std::vector<int>{64, 128, 192, 256, 384, 512});
  // (BwdTrans / IProductWRTBase pair kernels: slots of the input ring, 0 = registers)
  const std::vector<int> sts = sf ? std::vector<int>{0, 2, 3}
                                  : ((pair || role) ? std::vector<int>{0, 1, 2} : std::vector<int>{1, 2, 3});
  LaunchCfg best = p->cfg[op][dt];
  // Variable order: one launch serves every order, so its CTA is sized by the
  // largest order's tile (threads and shared memory); an order whose tile
  // uses fewer threads leaves them idle at every phase barrier, and one large
  // tile caps the CTAs per SM for all orders.  First pass: for a target of T
  // threads per CTA and k CTAs per SM, every order takes the largest tile
  // (any size up to kMaxEB) that stays within T threads and 1 / k of the SM's
  // shared memory, which evens out the orders' thread counts; the fastest
  // (T, k) is the start of the per-order search below.
  if (!p->uniform) {
    float kms = 1e30f;
    LaunchCfg kbest = best;
    std::vector<std::vector<int>> seen;
    for (int T : {64, 96, 128, 160, 192, 224, 256, 320, 384, 448, 512}) {
      for (int k = 1; k <= 3; ++k) {
        LaunchCfg c = best;
        const size_t smax = std::min(p->max_smem, p->smem_per_sm / k - 1024);
        std::vector<int> key;
        for (int P = 1; P <= kMaxP; ++P) {
          if (!p->present[P]) continue;
          int pick = 1;
          for (int eb = 1; eb <= kMaxEB; ++eb) {
            int thr = 0;
            size_t sm = 0;
            tile_footprint(p, op, dt, c, P, eb, &thr, &sm);
            if (thr > T + (pair ? 32 : 0) || sm > smax) break;
            pick = eb;
          }
          c.order[P].eb = pick;
          key.push_back(pick);
        }
        if (std::find(seen.begin(), seen.end(), key) != seen.end()) continue;
        seen.push_back(key);
        if (op_smem_bytes(p, op, dt, c) > p->max_smem) continue;
        p->cfg[op][dt] = c;
        p->tiles[op][dt].dirty = true;
        spx_status s;
        const float ms = time_op(p, op, dt, in, out, reps, st, ev, &s);
        if (s != SPX_OK) {
          p->cfg[op][dt] = best;
          p->tiles[op][dt].dirty = true;
          if (s == SPX_ERR_UNSUPPORTED) continue;
          return s;
        }
        if (ms < kms) {
          kms = ms;
          kbest = c;
        }
      }
    }
    best = kbest;
  }
  // orders one at a time (other orders keep their current tile); the same
  // thread count and depth serve the whole launch, so they are tuned last.
  float best_ms = 1e30f;
  for (int P = 1; P <= kMaxP; ++P) {
    if (!p->present[P]) continue;
    float bms = 1e30f;
    int beb = best.order[P].eb, bsg = best.stages;
    // bodies with Q^2 threads per element: the tile size, the staging depth
    // and the register class decide the CTAs per SM together (staged geometry
    // is most of the shared memory), so they are searched jointly
    const std::vector<int> sgs = role ? sts : std::vector<int>{best.stages};
    const std::vector<int> ntl = role ? nts : std::vector<int>{best.nthreads};
    int bnt = best.nthreads;
    for (int nt : ntl)
    for (int eb : ebs) {
      for (int sg : sgs) {
        LaunchCfg c = best;
        c.order[P].eb = eb;
        c.stages = sg;
        c.nthreads = nt;
        if (op_smem_bytes(p, op, dt, c) > p->max_smem) continue;
        p->cfg[op][dt] = c;
        p->tiles[op][dt].dirty = true;
        spx_status s;
        float ms = time_op(p, op, dt, in, out, reps, st, ev, &s);
        if (s != SPX_OK) {
          p->cfg[op][dt] = best;
          p->tiles[op][dt].dirty = true;
          if (s == SPX_ERR_UNSUPPORTED) continue;
          return s;
        }
        if (ms < bms) {
          bms = ms;
          beb = eb;
          bsg = sg;
          bnt = nt;
        }
      }
    }
    best.order[P].eb = beb;
    best.stages = bsg;
    best.nthreads = bnt;
    best_ms = bms;
  }
  for (int nt : role ? std::vector<int>{} : nts) {
    for (int sg : sts) {
      LaunchCfg c = best;
      c.nthreads = nt;
      c.stages = sg;
      if (op_smem_bytes(p, op, dt, c) > p->max_smem) continue;
      p->cfg[op][dt] = c;
      p->tiles[op][dt].dirty = true;
      spx_status s;
      float ms = time_op(p, op, dt, in, out, reps, st, ev, &s);
      if (s != SPX_OK) {
        if (s == SPX_ERR_UNSUPPORTED) continue;
        p->cfg[op][dt] = best;
        p->tiles[op][dt].dirty = true;
        return s;
      }
      if (ms < best_ms) {
        best_ms = ms;
        best.nthreads = nt;
        best.stages = sg;
      }
    }
  }
  p->cfg[op][dt] = best;
  p->tiles[op][dt].dirty = true;
  return ensure_tiles(p, op, dt);
}

}  // extern "C"
