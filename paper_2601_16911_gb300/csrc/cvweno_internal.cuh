// Internal declarations of the GB300 cell-vertex WENO library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "../../include/cvweno.h"

namespace cvw {

// An NVTX range over a host scope: every entry point that enqueues kernels names its
// work (and every RK stage its launch), so that a profiler can select a call's kernels
// (ncu --nvtx --nvtx-include "cvweno_step/").  Without an attached tool the push and
// pop cost one predictable branch each.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

constexpr int kMaxP = 4;
constexpr int kMaxMarks = 24;  // timing events per step: 3 stages x (up to 6 kernels + 1) + 1

// Status bits raised by kernels in the mesh's device status word.
enum : int { kStatNonfinite = 1, kStatPositivity = 2, kStatTimeout = 4, kStatCheck = 8 };

// Bounds checks of the checked build (compiled with -DCVWENO_CHECK): before each global
// load or store of a stage kernel, and each shared-memory store whose offset depends on
// the data's alignment, the span [first, first + count) is checked against the extent of
// its array; a failed check raises kStatCheck in the status word (CVWENO_ERR_CHECK at the
// next status check) and the access is skipped.  Nothing traps.  In the normal build
// CVW_SPAN is the constant true and costs nothing.
#if defined(CVWENO_CHECK) && defined(__CUDACC__)
__device__ __forceinline__ bool cvw_span(int* status, long long first, long long count, long long lim) {
  if (first >= 0 && count >= 0 && first + count <= lim) return true;
  atomicOr(status, kStatCheck);
  return false;
}
#define CVW_SPAN(status, first, count, lim) \
  ::cvw::cvw_span((status), (long long)(first), (long long)(count), (long long)(lim))
#define CVW_EXTENT(a, field) ((a).field)
#else
#define CVW_SPAN(status, first, count, lim) true
#define CVW_EXTENT(a, field) int64_t(0)
#endif

// Reference-cell tabulations of one (dim, p) pair, FP64 on the host rounded once to
// FP32, passed to the kernels by value (__grid_constant__), so that every warp reads
// them through the constant bank with uniform addresses (the entries read with per-lane
// indices come from TabImage instead).
//   E[k][m]     = P_m^(k)(+1); the value at -1 is (-1)^(m+k) E[k][m]
//   B[q][m]     = P_m(xi_q), Bd[q][m] = P_m'(xi_q) at the n Gauss-Legendre nodes xi_q
//   Bk[k][q][m] = P_m^(k)(xi_q) (pointwise semi-norm at quadrature nodes, stage d)
//   w[q]        Gauss weights on [-1,1]
//   sigma[k]    weights of the pointwise semi-norm in reference derivatives:
//               ||u||_x^2 = sum_{k != 0} sigma_k (d_ref^k u)^2  (eq. pointsnorm)
//   R[i][j]     upper-triangular Cholesky factor of the element semi-norm Gram matrix
//               on Legendre modes 1..ND-1: ||u||_e = |R c[1:]|     (eq. snorm)
//   A[l][i][j]  R times the Taylor->Legendre map of corner l, on derivative orders
//               1..ND-1: ||u*_vertex||_e-vector = A[l] t*[1:]       (Sec. 3.2 remark)
//   tscale[k]   (2/dx)^kx (2/dy)^ky: reference -> physical derivative
template <int DIM, int P>
struct DgTables {
  static constexpr int N = P + 1;
  static constexpr int ND = DIM == 2 ? N * N : N;
  static constexpr int NS = ND - 1;
  static constexpr int NC = 1 << DIM;
  float E[N][N];
  float B[N][N];
  float Bd[N][N];
  float Bk[N][N][N];
  float w[N];
  float sigma[ND];
  float tscale[ND];
  float R[NS][NS];
  float A[NC][NS][NS];
};

// Device image of the tabulations that the stage kernels index with a different value in
// every lane (A padded to NSP columns, B, Bd, Bk, w), in the order they take in shared
// memory: a tile stages it with 16-byte copies from global memory, where reading the
// by-value tables with per-lane indices would serialise in the constant bank.  Built on
// the device from DgTables by launch_tab_image (once per mesh).
template <int DIM, int P>
struct TabImage {
  using Tb = DgTables<DIM, P>;
  static constexpr int N = P + 1, NS = Tb::NS, NC = Tb::NC;
  static constexpr int NSP = (NS + 3) / 4 * 4;
  static constexpr int A = 0;                  // [NC][NS][NSP], columns >= NS zero
  static constexpr int B = A + NC * NS * NSP;  // [N][N]
  static constexpr int BD = B + N * N;         // [N][N]
  static constexpr int BK = BD + N * N;        // [N][N][N]
  static constexpr int W = BK + N * N * N;     // [N]
  static constexpr int FLOATS = (W + N + 3) / 4 * 4;  // whole 16-byte chunks (the CUDA-core kernels' part)
  // The tensor-core form of the sensor's corner products (2D, p = 3): A[l] split into TF32
  // hi and lo parts, zero-padded to TCK x TCK, in the canonical K-major operand layout
  // [part][corner l][K chunk of 4][row i][4] (tc_tf32.cuh).
  static constexpr bool HAS_TC = DIM == 2 && P == 3;
  static constexpr int TCK = (NS + 15) / 16 * 16;
  static constexpr int TC = FLOATS;
  static constexpr int FLOATS_ALL = FLOATS + (HAS_TC ? 2 * NC * TCK * TCK : 0);
};
constexpr int imax(int a, int b) { return a > b ? a : b; }
constexpr int kMaxTabImage = imax(TabImage<2, kMaxP>::FLOATS_ALL, TabImage<2, 3>::FLOATS_ALL);
inline int tab_image_floats(int dim, int p) {
  switch (dim * 10 + p) {
    case 11: return TabImage<1, 1>::FLOATS_ALL;
    case 12: return TabImage<1, 2>::FLOATS_ALL;
    case 13: return TabImage<1, 3>::FLOATS_ALL;
    case 14: return TabImage<1, 4>::FLOATS_ALL;
    case 21: return TabImage<2, 1>::FLOATS_ALL;
    case 22: return TabImage<2, 2>::FLOATS_ALL;
    case 23: return TabImage<2, 3>::FLOATS_ALL;
    case 24: return TabImage<2, 4>::FLOATS_ALL;
    default: return 0;
  }
}

// CG tabulations (Gauss-Lobatto-Legendre nodal basis l_a on [-1,1]):
//   V[m][a]   Legendre mode m of l_a: (2m+1)/2 int P_m l_a      (nodal -> modal)
//   Lq[q][a]  l_a(xi_q) and Ldq[q][a] = l_a'(xi_q) at the Gauss nodes
//   M1[a][b]  int l_a l_b (1D reference mass), wl[a] = int l_a (GLL weight)
//   xg[a]     GLL nodes
//   Em[a][m]  int l_a P_m and Dm[a][m] = int l_a P_m' (local integrals of a Legendre
//             expansion against the nodal basis)
//   iml[a]    1 / (m_a wl[a]), m_a = 2 for the vertex node a = 0 (shared by two cells
//             along the line), else 1: the inverse 1D lumped mass of local node a
template <int DIM, int P>
struct CgTables {
  static constexpr int N = P + 1;
  float V[N][N];
  float Lq[N][N];
  float Ldq[N][N];
  float M1[N][N];
  float Em[N][N];
  float Dm[N][N];
  float wl[N];
  float iml[N];
  float xg[N];
};

// Run-time arguments of one stage launch.
struct StageArgs {
  const float* u_in;   // state the residual is evaluated on
  const float* u_n;    // RK: state at the start of the step (may alias u_out)
  float* u_out;        // RK result or dudt
  float* gamma_out;    // optional [ncell]
  float* nu_out;       // optional [ncell]
  float* alpha_out;    // optional [ncell][nvar][nq]
  int32_t* troubled_out;          // optional [ncell]
  const int32_t* troubled_override;  // optional [ncell]
  float* tstar_out;    // optional [nvert][ND] (physical derivatives)
  float* lambda_out;   // optional [ncell] wave speed lambda_e
  int* status;         // device status word
  int nx, ny;          // cells
  int perx, pery;      // periodic flags
  int vx;              // vertices per row (nx if periodic in x, nx+1 otherwise)
  int mode;            // kMode* flags
  // u_out = rk_a u_n + rk_b (u_in + dt L(u_in)) with rk_a = 1 - rk_b, evaluated as the
  // increment u_n + rk_b (w - u_n): 1/3 + 2/3 rounded to float sum to 1 + 3e-8, a growth
  // that compounds over thousands of steps; the increment form keeps constants exact.
  // rk_a == 0 selects u_out = w.
  float rk_a, rk_b, dt;
  float two_dx, two_dy;  // 2/dx, 2/dy
  float nu_scale;        // h_e / (2p)
  float eps, gamma_vertex, c_gamma, q, lambda_const;
  int r;
  int sc, sensor_mode;
  int limit_all;       // kModeLimit: limit every cell, not only gamma_e < c_gamma
  // surrogate sensor (2D DG scalar): packed network weights (MlpPacked) or null, the
  // confidence below which the plain sensor decides, a fallback counter (may be null),
  // and the features output of kModeFeatures ([ncell][12])
  const void* mlp;
  float mlp_conf_min;
  unsigned int* mlp_fallbacks;
  float* feat_out;
  float* norm_out;     // kModeFeatures: ||u^e||_e per cell (may be null)
  float h_e;           // cell diameter
  const float* tab_img;  // TabImage of the mesh's tabulations (device)
  float adv_vx, adv_vy;
  float gas_gamma;
  // CG only: nodal lattice and the per-stage work arrays
  int nnx, nny;
  float* rloc;  // [ncell][nd] cell-local residuals
  float* rnode; // [nnode] assembled residual (1D)
  float* du;    // [nnode] du/dt iterate (1D)
  float* du2;   // [nnode] second defect-correction iterate (1D)
#ifdef CVWENO_CHECK
  // extents for the bounds checks of the checked build (absent from the normal build, whose
  // kernels then see the same arguments as without the checks)
  int64_t lim_in;      // floats readable at u_in and u_n
  int64_t lim_out;     // floats writable at u_out
  int64_t lim_cell;    // cells: the extent of the per-cell outputs and of rloc (in cells)
#endif
};

// Sets the extents of the checked build's bounds checks (nothing in the normal build).
inline void set_check_extents(StageArgs& a, int64_t nstate, int64_t ncell) {
#ifdef CVWENO_CHECK
  a.lim_in = a.lim_out = nstate;
  a.lim_cell = ncell;
#else
  (void)a, (void)nstate, (void)ncell;
#endif
}

// The three SSP-RK3 stages of a step, each a full StageArgs (kModeRK), repeated nsteps
// times by the one-launch step kernel of a 1D mesh that is a single tile.
struct StepArgs {
  StageArgs st[3];
  int nsteps;
};

// Cells of a 1D tile: a 1D DG mesh of at most this many cells is one CTA.
constexpr int kTile1D = 128;

enum : int {
  kModeResidual = 1,   // write dudt to u_out
  kModeRK = 2,         // write u_n + rk_b (u_in + dt L - u_n) (or u_in + dt L) to u_out
  kModeSensorOnly = 4, // stop after stage (c) (gamma, nu, lambda outputs)
  kModeLimit = 8,      // HWENO limiter: write u_in or its reconstruction u^{e,*} to u_out
  kModeFeatures = 16,  // surrogate inputs to feat_out and the computed gamma_e to gamma_out
};

}  // namespace cvw

struct cvweno_mesh_s {
  cvweno_mesh_desc desc;
  int device;
  int dim, p, n, nd, nvar, nq, ncorner;
  int nx, ny, vx, vy;
  int64_t ncell, nvert, nstate;
  double dx, dy, h;
  // host tables
  int32_t* cell_vertices;  // [ncell][ncorner]
  int32_t* vertex_cells;   // [nvert][ncorner]
  int32_t* colour;         // [ncell]
  // reference tabulations, one per (dim, p) -- only the matching one is filled
  void* tables;            // host copy of DgTables<dim, p>
  size_t tables_bytes;
  float* d_tabimg;         // TabImage<dim, p> (device)
  // CG: nodal lattice, tabulations and stage work arrays
  int kind;
  int nnx, nny;
  int64_t nnode;
  void* cg_tables;         // host copy of CgTables<dim, p>
  size_t cg_tables_bytes;
  float* d_rloc;
  float* d_r;
  float* d_du;
  float* d_du2;
  double cg_xg[cvw::kMaxP + 1];  // GLL nodes (host, FP64)
  double cg_wl[cvw::kMaxP + 1];  // GLL weights (host, FP64)
  float* d_cg_xg;           // GLL nodes (device)
  double* d_cg_ml;          // 1D lumped masses by local node index, x then y (device)
  // device scratch
  float* d_u1;
  float* d_u2;
  float* d_lambda;         // [ncell]
  double* d_red;           // reduction scratch
  int* d_status;
  int* h_status;           // pinned
  // surrogate sensor (cvweno_mesh_set_surrogate): packed weights owned by the network
  // object, the confidence threshold and an optional device fallback counter
  const void* surrogate;
  float surrogate_conf_min;
  unsigned int* surrogate_fallbacks;
  // cvweno_mesh_set_tensor_cores: 1 = the stage kernel's tcgen05 variant (2D DG scalar Q3)
  int tensor_cores;
  // cvweno_mesh_set_check_extents: the checked build's extents (-1: nstate and ncell)
  int64_t chk_state, chk_cell;
  // optional per-launch timing (cvweno_mesh_set_kernel_timing): events recorded
  // between the kernels of one step, read back by cvweno_kernel_times
  int timing;
  int tcount;
  cudaEvent_t tev[cvw::kMaxMarks];
  double* h_red;           // pinned
};

namespace cvw {
// tables.cpp
cvweno_status build_tables(cvweno_mesh m);
// The reference-cell tabulations DgTables<dim, p> of a dx x dy cell into out (host, at
// least capacity bytes; *bytes receives their size), with no allocation.
cvweno_status fill_dg_tables(int dim, int p, double dx, double dy, void* out, size_t capacity, size_t* bytes);
constexpr int kMaxGaussRule = 16;                    // largest rule gauss_rule builds
bool gauss_rule(int n, double* x, double* w);         // Gauss-Legendre on [-1,1], ascending; false unless 1 <= n <= 16
void legendre_values(double x, int mmax, double* out);  // P_0..P_mmax at x
// dg_scalar.cu / dg_euler.cu
cudaError_t launch_stage(const cvweno_mesh_s* m, const StageArgs& a, cudaStream_t s);
cudaError_t launch_stage_euler(const cvweno_mesh_s* m, const StageArgs& a, cudaStream_t s);
// dg_scalar_1d.cu: nsteps whole SSP-RK3 steps of a 1D scalar DG mesh of at most kTile1D
// cells in one launch (cudaErrorNotSupported for any other mesh)
cudaError_t launch_steps_1d_tile(const cvweno_mesh_s* m, const StepArgs& a, cudaStream_t s);
// dg_euler.cu: the positivity limiter on a.u_in -> a.u_out (may alias), theta per cell
cudaError_t launch_positivity(const cvweno_mesh_s* m, const StageArgs& a, float* theta, cudaStream_t s);
// dg_scalar_2d.cu: writes TabImage<dim, p> of the host tables t (DgTables<dim, p>) to
// dst (device, tab_image_floats(dim, p) floats), stream-ordered on s
cudaError_t launch_tab_image(int dim, int p, const void* t, float* dst, cudaStream_t s);
// cg_scalar.cu
cudaError_t launch_stage_cg(const cvweno_mesh_s* m, const StageArgs& a, cudaStream_t s);
// api.cu: the stage arguments common to every launch on mesh m (no state pointers, no RK)
StageArgs stage_base_args(const cvweno_mesh_s* m);
// api.cu: with kernel timing on, records the next timing event of the step on s
void kernel_mark(const cvweno_mesh_s* m, cudaStream_t s);
}  // namespace cvw
