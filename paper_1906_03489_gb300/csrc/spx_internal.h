// Internal host-side declarations of the spx library (not part of the ABI).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/spx.h"
#include "kernel_params.h"

namespace spx {

spx_status fail(spx_status s, const std::string& msg);   // records the message, returns s
spx_status cuda_fail(cudaError_t e, const char* what);    // maps a CUDA error

struct TileCfg {
  int eb = 0;  // elements per tile for this order
};

struct LaunchCfg {
  int nthreads = 256;
  int stages = 2;
  TileCfg order[kMaxP1];
};

struct TileList {
  Tile* d = nullptr;   // device
  int n = 0;
  bool dirty = true;
  // variable order: the list holds one contiguous run of tiles per order
  // (heaviest order first); run g has order grp_P[g], tiles
  // [grp_tile[g], grp_tile[g + 1]) and grp_bytes[g] algorithmic bytes
  std::vector<int> grp_P, grp_tile;
  std::vector<double> grp_bytes;
};

}  // namespace spx

struct spx_plan {
  int dim = 3;
  int64_t E = 0;
  int qoff = 2;
  bool uniform = true;
  int uP = 0;                            // order of a uniform plan
  std::vector<int32_t> orders;           // host [E]
  std::vector<int64_t> coef_off, quad_off;  // host [E+1]
  int64_t n_coef = 0, n_quad = 0;
  bool present[spx::kMaxP1] = {};
  std::vector<int32_t> ids;              // host: element ids bucketed by order (var plans)
  std::vector<int64_t> bucket_start;     // host: start of each order's bucket in ids
  int device = 0;
  int num_sms = 0;
  size_t max_smem = 0;                   // shared memory per block (opt-in limit)
  size_t smem_per_sm = 0;                // shared memory per SM
  // device metadata (owned)
  int64_t* d_coef_off = nullptr;
  int64_t* d_quad_off = nullptr;
  int32_t* d_ids = nullptr;
  int* d_status = nullptr;
  // small device buffers (owned): per-order inverse 1D mass matrices for
  // FwdTrans and the sensor (FP64 at aux64, FP32 at aux32; layout
  // mass1d_off in kernel_params.h), and the partial sums of spx_integral
  double* d_aux64 = nullptr;
  float* d_aux32 = nullptr;
  double* d_partials = nullptr;
  unsigned int* d_ticket = nullptr;
  // per operator and precision
  spx::LaunchCfg cfg[spx::OP_KINDS][2];
  spx::TileList tiles[spx::OP_KINDS][2];
  // caller-owned geometry, per precision
  const void* geom[2] = {nullptr, nullptr};
  const void* dxi[2] = {nullptr, nullptr};
  // host basis tables (FP64) per order: B[Q][n], dB[Q][n], D[Q][Q], then the
  // even-odd coefficients (EOLayout)
  std::vector<double> tab[spx::kMaxP1];
  int shape = 0;                         // spx_shape
  std::vector<double> ctab;              // collapsed shapes: B1, Bb, D1, D2 (FP64, collapsed.cu)
  int bkind = 0;                         // BasisKind of the 3D Helmholtz kernels
  bool custom_basis = false;             // tables differ from the library's modified basis
};

namespace spx {

// Launch request for one operator call.
struct LaunchReq {
  const spx_plan* plan;
  int op;
  int dtype;  // 0 FP64, 1 FP32
  const void* in0;
  const void* in1;
  const void* geom;
  const void* lam_f;
  const void* kap_f;
  void* out0;
  void* out1;
  void* out2;
  double lam;
  cudaStream_t stream;
  const int* skip = nullptr;  // device flag read by every CTA at launch (KParams::skip)
};

// Builds (if needed) the tile list of (op, dtype) on the device.  Synchronous.
spx_status ensure_tiles(spx_plan* plan, int op, int dtype);

// Per-(T, DIM, OP) launchers; each lives in its own translation unit.
#define SPX_DECL_LAUNCH(TN, DIM, OP) spx_status launch_##TN##_##DIM##_##OP(const LaunchReq& r);
#define SPX_DECL_ALL_OPS(TN, DIM) \
  SPX_DECL_LAUNCH(TN, DIM, 0)     \
  SPX_DECL_LAUNCH(TN, DIM, 1)     \
  SPX_DECL_LAUNCH(TN, DIM, 2)     \
  SPX_DECL_LAUNCH(TN, DIM, 3)     \
  SPX_DECL_LAUNCH(TN, DIM, 4)     \
  SPX_DECL_LAUNCH(TN, DIM, 5)     \
  SPX_DECL_LAUNCH(TN, DIM, 6)     \
  SPX_DECL_LAUNCH(TN, DIM, 7)
SPX_DECL_ALL_OPS(f64, 2)
SPX_DECL_ALL_OPS(f64, 3)
SPX_DECL_ALL_OPS(f32, 2)
SPX_DECL_ALL_OPS(f32, 3)

// 3D Helmholtz of the other basis kinds (generic body, collocation body).
spx_status launch_f64_helm3_bk1(const LaunchReq& r);
spx_status launch_f64_helm3_bk2(const LaunchReq& r);
spx_status launch_f32_helm3_bk1(const LaunchReq& r);
spx_status launch_f32_helm3_bk2(const LaunchReq& r);

spx_status launch_op(const LaunchReq& r);

// Triangles and prisms (collapsed.cu): operator launch, shared memory of a
// tile of eb elements, affine geometric factors.
spx_status launch_collapsed(const LaunchReq& r);
size_t collapsed_smem_bytes(const spx_plan* plan, int dtype, int eb);
spx_status collapsed_geom(const spx_plan* plan, const double* verts, double* geom, double* dxi, double* xq,
                          float* geom32, float* dxi32, cudaStream_t st);

// Helmholtz apply for the solver: as spx_helmholtz (constant lambda, kappa =
// 1), but the launch does nothing when *skip != 0 at the time it runs.
spx_status helmholtz_unless(const spx_plan* p, int dtype, double lambda, const void* in, void* out,
                            const int* skip, cudaStream_t stream);

// Shared-memory footprint of (op, dtype) with the plan's current tile
// configuration; 0 if the tile does not fit.
size_t op_smem_bytes(const spx_plan* plan, int op, int dtype, const LaunchCfg& cfg);

// Basis tables (host FP64): fills B, dB, D as documented in spx.h.
spx_status basis_tables(int P, int Q, double* xi, double* w, double* B, double* dB, double* D);

// Gauss-Radau-Legendre points (including -1) and weights.
spx_status gauss_radau(int Q, double* x, double* w);
// Tables of the collapsed-coordinate kernels (basis_host.cpp).
spx_status collapsed_tables(int P, int Q, double* B1, double* Bb, double* D1, double* D2, double* xg, double* wg,
                            double* xr, double* wr, double* Bc = nullptr);

// Nodal (Lagrange through the P + 1 GLL points) basis at the Q GLL points.
spx_status nodal_basis_tables(int P, int Q, double* B, double* dB);

// Even-odd coefficients appended to a per-order table (EOLayout).
void eo_tables(int P, int Q, double* tab);

// Device address of the allocation-free solver's built-in workspace on the
// current device (looked up once per device and CUDA context; cg.cu).
spx_status noalloc_workspace(void** out);

// Blocks per SM of the spx_integral reduction (fixed: its sums are
// reproducible); the plan's partials buffer holds one FP64 value per block.
constexpr int kIntegralBlocksPerSM = 4;

// Inverse of the 1D mass matrix B^T diag(w) B of the tables B [Q][n] (order P,
// Q GLL points, weights w), [n][n].  restricted: the matrix without row and
// column P - 1 (the degree-P bubble of the modified basis), inverted, with
// zeros in that row and column (P >= 2).
void mass1d_inverse(int P, int Q, const double* B, double* minv, bool restricted = false);

// Basis kinds of a plan (3D Helmholtz kernels): the modified basis's parity
// (even-odd bodies), any basis (generic body), collocation B = I.
enum BasisKind { BK_PARITY = 0, BK_GENERAL = 1, BK_COLLOCATION = 2 };

}  // namespace spx
