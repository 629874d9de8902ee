// C ABI of the cell-vertex WENO library: mesh lifecycle, stage dispatch, SSP-RK3,
// projection of analytic initial data and the FP64 reductions (conservation totals
// and CFL wave speed -- the only FP64 arithmetic on the device).
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "cvweno_internal.cuh"

using namespace cvw;

namespace {

constexpr int kRedThreads = 256;
constexpr int kRedBlocks = 304;  // 2 x 152 SMs
constexpr int kProjN = 12;       // projection rule points per direction

inline cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

inline cvweno_status cuda_status(cudaError_t e) { return e == cudaSuccess ? CVWENO_OK : CVWENO_ERR_CUDA; }

// ---- analytic initial data --------------------------------------------------------------

struct ProjTables {
  float x[kProjN], w[kProjN];
  float P[kProjN][kMaxP + 1];  // Legendre values at the projection nodes
};

struct ProjArgs {
  float* u;
  int nx, ny, dim, nd, n, nvar, type;
  double x0, y0, dx, dy, lx, ly, gas_gamma;
  float prm[64];
};

__device__ void prim_to_cons(float g, float rho, float vx, float vy, float p, float* U) {
  U[0] = rho;
  U[1] = rho * vx;
  U[2] = rho * vy;
  U[3] = p / (g - 1.0f) + 0.5f * rho * (vx * vx + vy * vy);
}

__device__ void ic_eval(const ProjArgs& a, float x, float y, float* U) {
  const float* P = a.prm;
  const float twopi = 6.28318530717958647692f;
  switch (a.type) {
    case CVWENO_IC_CONST:
      for (int v = 0; v < 4; ++v) U[v] = P[v];
      break;
    case CVWENO_IC_SINE_STEP:
      U[0] = P[0] * sinf(twopi * P[1] * (x - (float)a.x0) / (float)a.lx) + (x >= P[3] ? P[2] : 0.0f);
      break;
    case CVWENO_IC_CIRCLE: {
      float rx = x - P[0], ry = y - P[1];
      U[0] = (rx * rx + ry * ry <= P[2] * P[2]) ? P[3] : P[4];
      break;
    }
    case CVWENO_IC_QUADRANTS: {
      int qd = (x >= P[0] ? 1 : 0) + 2 * (y >= P[1] ? 1 : 0);
      const float* s = P + 2 + 4 * qd;
      prim_to_cons((float)a.gas_gamma, s[0], s[1], s[2], s[3], U);
      break;
    }
    case CVWENO_IC_FOURIER: {
      int M = (int)P[0];
      float acc = 0.0f;
      for (int j = 0; j < M && j < 15; ++j) {
        const float* md = P + 1 + 4 * j;
        acc += md[0] * sinf(twopi * (md[1] * (x - (float)a.x0) / (float)a.lx + md[2] * (y - (float)a.y0) / (float)a.ly) +
                            md[3]);
      }
      U[0] = acc;
      break;
    }
    case CVWENO_IC_POLY: {
      float acc = 0.0f, yp = 1.0f;
      for (int j = 0; j < 5; ++j) {
        float xp = 1.0f;
        for (int i = 0; i < 5; ++i) {
          acc += P[i + 5 * j] * xp * yp;
          xp *= x;
        }
        yp *= y;
      }
      U[0] = acc;
      break;
    }
    case CVWENO_IC_DENSITY_WAVE: {
      float rho = 1.0f + P[0] * sinf(twopi * (P[1] * (x - (float)a.x0) / (float)a.lx +
                                              P[2] * (y - (float)a.y0) / (float)a.ly));
      prim_to_cons((float)a.gas_gamma, rho, P[3], P[4], P[5], U);
      break;
    }
    default:
      U[0] = U[1] = U[2] = U[3] = 0.0f;
  }
}

// one thread per cell: c_m = (2mx+1)(2my+1)/4 sum_q w w P_mx P_my u0   (2D)
__global__ void project_kernel(const __grid_constant__ ProjArgs a, const __grid_constant__ ProjTables T) {
  const int64_t ncell = (int64_t)a.nx * a.ny;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ncell; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % a.nx), j = (int)(e / a.nx);
    const double xc = a.x0 + (i + 0.5) * a.dx, yc = a.dim == 2 ? a.y0 + (j + 0.5) * a.dy : 0.0;
    float acc[4][25];
    for (int v = 0; v < 4; ++v)
      for (int m = 0; m < 25; ++m) acc[v][m] = 0.0f;
    const int npy = a.dim == 2 ? kProjN : 1;
    for (int qb = 0; qb < npy; ++qb)
      for (int qa = 0; qa < kProjN; ++qa) {
        float x = (float)(xc + 0.5 * a.dx * T.x[qa]);
        float y = a.dim == 2 ? (float)(yc + 0.5 * a.dy * T.x[qb]) : 0.0f;
        float W = T.w[qa] * (a.dim == 2 ? T.w[qb] : 1.0f);
        float U[4];
        ic_eval(a, x, y, U);
        for (int m = 0; m < a.nd; ++m) {
          int mx = m % a.n, my = m / a.n;
          float ph = T.P[qa][mx] * (a.dim == 2 ? T.P[qb][my] : 1.0f);
          for (int v = 0; v < a.nvar; ++v) acc[v][m] = fmaf(W * ph, U[v], acc[v][m]);
        }
      }
    for (int v = 0; v < a.nvar; ++v)
      for (int m = 0; m < a.nd; ++m) {
        int mx = m % a.n, my = m / a.n;
        float s = a.dim == 2 ? 0.25f * (2 * mx + 1) * (2 * my + 1) : 0.5f * (2 * mx + 1);
        a.u[((size_t)v * ncell + e) * a.nd + m] = acc[v][m] * s;
      }
  }
}

// CG: interpolation at the GLL nodes of the periodic lattice (reading A25)
__global__ void project_cg_kernel(const __grid_constant__ ProjArgs a, const __grid_constant__ ProjTables T,
                                  int p, int nnx, int nny, const float* __restrict__ xg_dev) {
  (void)T;
  const int64_t nn = (int64_t)nnx * nny;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nn; j += (int64_t)gridDim.x * blockDim.x) {
    const int I = (int)(j % nnx), J = (int)(j / nnx);
    const int i = I / p, ai = I % p, jj = J / p, bj = J % p;
    const float x = (float)(a.x0 + (i + 0.5) * a.dx + 0.5 * a.dx * xg_dev[ai]);
    const float y = a.dim == 2 ? (float)(a.y0 + (jj + 0.5) * a.dy + 0.5 * a.dy * xg_dev[bj]) : 0.0f;
    float U[4];
    ic_eval(a, x, y, U);
    a.u[j] = U[0];
  }
}

// ---- FP64 reductions --------------------------------------------------------------------

// CG: partial sums of ML_j u_j (FP64) with the lumped mass of each lattice node
__global__ void sum_cg_partial(const float* __restrict__ u, int nnx, int nny, int p, const double* __restrict__ ml1x,
                               const double* __restrict__ ml1y, double* __restrict__ partial) {
  __shared__ double sh[kRedThreads];
  double acc = 0.0;
  const int64_t nn = (int64_t)nnx * nny;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nn; j += (int64_t)gridDim.x * blockDim.x) {
    const int I = (int)(j % nnx), J = (int)(j / nnx);
    acc += ml1x[I % p] * ml1y[J % p] * (double)u[j];
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

// partial[b] = sum over a grid-stride slice of x[i * stride] (FP64), fixed order per block
__global__ void sum_mode0_partial(const float* __restrict__ x, int64_t n, int stride, double* __restrict__ partial) {
  __shared__ double sh[kRedThreads];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc += (double)x[i * stride];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

__global__ void max_partial(const float* __restrict__ x, int64_t n, double* __restrict__ partial) {
  __shared__ double sh[kRedThreads];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc = fmax(acc, (double)x[i]);
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

// single block: out[0] = sum (or max) of partial[0..n) in a fixed order
__global__ void finish_reduce(const double* __restrict__ partial, int n, int is_max, double* __restrict__ out) {
  __shared__ double sh[kRedThreads];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc = is_max ? fmax(acc, partial[i]) : acc + partial[i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] = is_max ? fmax(sh[threadIdx.x], sh[threadIdx.x + s]) : sh[threadIdx.x] + sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

StageArgs base_args(const cvweno_mesh_s* m) {
  StageArgs a;
  memset(&a, 0, sizeof(a));
  const cvweno_params& p = m->desc.params;
  a.status = m->d_status;
  set_check_extents(a, m->chk_state >= 0 ? m->chk_state : m->nstate, m->chk_cell >= 0 ? m->chk_cell : m->ncell);
  a.nx = m->nx;
  a.ny = m->ny;
  a.perx = m->desc.bc[0] == CVWENO_PERIODIC;
  a.pery = m->dim == 2 && m->desc.bc[2] == CVWENO_PERIODIC;
  a.vx = m->vx;
  a.two_dx = (float)(2.0 / m->dx);
  a.two_dy = (float)(2.0 / m->dy);
  a.nu_scale = (float)(m->h / (2.0 * m->p));
  a.h_e = (float)m->h;
  a.tab_img = m->d_tabimg;
  a.mlp = m->surrogate;
  a.mlp_conf_min = m->surrogate_conf_min;
  a.mlp_fallbacks = m->surrogate_fallbacks;
  a.eps = (float)p.eps;
  a.r = (int)p.r;
  a.q = (float)p.q;
  a.gamma_vertex = (float)p.gamma_vertex;
  a.c_gamma = (float)p.c_gamma;
  a.lambda_const = (float)p.lambda_const;
  a.sc = p.sc_quadrature;
  a.sensor_mode = p.sensor_mode;
  a.limit_all = 0;
  a.adv_vx = (float)p.adv_vx;
  a.adv_vy = (float)p.adv_vy;
  a.gas_gamma = (float)p.gas_gamma;
  a.rk_b = 1.0f;
  a.nnx = m->nnx;
  a.nny = m->nny;
  a.rloc = m->d_rloc;
  a.rnode = m->d_r;
  a.du = m->d_du;
  a.du2 = m->d_du2;
  return a;
}

cudaError_t launch(const cvweno_mesh_s* m, const StageArgs& a, cudaStream_t s) {
  if (m->kind == CVWENO_CG) return launch_stage_cg(m, a, s);  // marks after each kernel itself
  cudaError_t e = m->desc.system == CVWENO_EULER ? launch_stage_euler(m, a, s) : launch_stage(m, a, s);
  kernel_mark(m, s);
  return e;
}

cvweno_status read_status(cvweno_mesh m, cudaStream_t s) {
  cudaError_t e = cudaMemcpyAsync(m->h_status, m->d_status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return CVWENO_ERR_CUDA;
  int st = *m->h_status;
  if (st) {
    e = cudaMemsetAsync(m->d_status, 0, sizeof(int), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return CVWENO_ERR_CUDA;
  }
  if (st & kStatCheck) return CVWENO_ERR_CHECK;
  if (st & kStatPositivity) return CVWENO_ERR_POSITIVITY;
  if (st & kStatNonfinite) return CVWENO_ERR_NONFINITE;
  if (st & kStatTimeout) return CVWENO_ERR_TIMEOUT;
  return CVWENO_OK;
}

cvweno_status rk_stage(cvweno_mesh m, const float* in, const float* un, float* out, float ra, float rb, float dt,
                       cudaStream_t s) {
  NvtxRange range("rk_stage");
  StageArgs a = base_args(m);
  a.u_in = in;
  a.u_n = un;
  a.u_out = out;
  a.rk_a = ra;
  a.rk_b = rb;
  a.dt = dt;
  a.mode = kModeRK;
  return cuda_status(launch(m, a, s));
}

cvweno_status limit_stage(cvweno_mesh m, const float* in, float* out, cudaStream_t s) {
  StageArgs a = base_args(m);
  a.u_in = in;
  a.u_out = out;
  a.mode = kModeLimit;
  return cuda_status(launch(m, a, s));
}

cvweno_status positivity_stage(cvweno_mesh m, float* x, cudaStream_t s) {
  StageArgs a = base_args(m);
  a.u_in = x;
  a.u_out = x;
  cudaError_t e = launch_positivity(m, a, nullptr, s);
  kernel_mark(m, s);
  return cuda_status(e);
}

// A 1D scalar DG mesh of one tile without a limiter runs its steps in one launch, unless
// kernel timing asks for the stages one by one.
bool steps_in_one_launch(cvweno_mesh m) {
  return m->dim == 1 && m->kind != CVWENO_CG && m->desc.system != CVWENO_EULER && !m->desc.params.positivity &&
         !m->desc.params.hweno_limiter && !m->timing && m->nx <= kTile1D;
}

cvweno_status enqueue_steps_one_launch(cvweno_mesh m, float* u, float dt, int nsteps, cudaStream_t s) {
  StepArgs sa;
  const float* in[3] = {u, m->d_u1, m->d_u2};
  float* out[3] = {m->d_u1, m->d_u2, u};
  const float ra[3] = {0.0f, 0.75f, 1.0f / 3.0f}, rb[3] = {1.0f, 0.25f, 2.0f / 3.0f};
  for (int k = 0; k < 3; ++k) {
    StageArgs& a = sa.st[k];
    a = base_args(m);
    a.u_in = in[k];
    a.u_n = u;
    a.u_out = out[k];
    a.rk_a = ra[k];
    a.rk_b = rb[k];
    a.dt = dt;
    a.mode = kModeRK;
  }
  sa.nsteps = nsteps;
  return cuda_status(launch_steps_1d_tile(m, sa, s));
}

cvweno_status enqueue_step(cvweno_mesh m, float* u, float dt, cudaStream_t s) {
  if (steps_in_one_launch(m)) return enqueue_steps_one_launch(m, u, dt, 1, s);
  if (m->desc.params.positivity) {
    // every stage result is limited in place (reading P3): the limiter is cell-local
    if (m->timing) {
      m->tcount = 0;
      kernel_mark(m, s);
    }
    cvweno_status st = rk_stage(m, u, u, m->d_u1, 0.0f, 1.0f, dt, s);
    if (st == CVWENO_OK) st = positivity_stage(m, m->d_u1, s);
    if (st == CVWENO_OK) st = rk_stage(m, m->d_u1, u, m->d_u2, 0.75f, 0.25f, dt, s);
    if (st == CVWENO_OK) st = positivity_stage(m, m->d_u2, s);
    if (st == CVWENO_OK) st = rk_stage(m, m->d_u2, u, u, 1.0f / 3.0f, 2.0f / 3.0f, dt, s);
    if (st == CVWENO_OK) st = positivity_stage(m, u, s);
    return st;
  }
  if (m->timing) {
    m->tcount = 0;
    kernel_mark(m, s);
  }
  if (m->desc.params.hweno_limiter) {
    // every stage result is limited (reading A27); the limiter reads neighbours, so it
    // runs out of place: stages write d_u1, the limiter writes d_u2 (the last one u)
    cvweno_status st = rk_stage(m, u, u, m->d_u1, 0.0f, 1.0f, dt, s);
    if (st == CVWENO_OK) st = limit_stage(m, m->d_u1, m->d_u2, s);
    if (st == CVWENO_OK) st = rk_stage(m, m->d_u2, u, m->d_u1, 0.75f, 0.25f, dt, s);
    if (st == CVWENO_OK) st = limit_stage(m, m->d_u1, m->d_u2, s);
    if (st == CVWENO_OK) st = rk_stage(m, m->d_u2, u, m->d_u1, 1.0f / 3.0f, 2.0f / 3.0f, dt, s);
    if (st == CVWENO_OK) st = limit_stage(m, m->d_u1, u, s);
    return st;
  }
  cvweno_status st = rk_stage(m, u, u, m->d_u1, 0.0f, 1.0f, dt, s);
  if (st == CVWENO_OK) st = rk_stage(m, m->d_u1, u, m->d_u2, 0.75f, 0.25f, dt, s);
  if (st == CVWENO_OK) st = rk_stage(m, m->d_u2, u, u, 1.0f / 3.0f, 2.0f / 3.0f, dt, s);
  return st;
}

}  // namespace

namespace cvw {
StageArgs stage_base_args(const cvweno_mesh_s* m) { return base_args(m); }

void kernel_mark(const cvweno_mesh_s* mc, cudaStream_t s) {
  cvweno_mesh_s* m = const_cast<cvweno_mesh_s*>(mc);
  if (!m->timing || m->tcount >= kMaxMarks) return;
  // inside stream capture the record becomes an event-record node of the graph, so the
  // events time every replay
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cs);
  cudaEventRecordWithFlags(m->tev[m->tcount++], s, cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : 0);
}
}  // namespace cvw

extern "C" {

void cvweno_default_params(cvweno_params* p) {
  if (!p) return;
  p->eps = 1e-6;
  p->r = 2.0;
  p->q = 1.0;
  p->gamma_vertex = 1e-3;
  p->c_gamma = 0.9;
  p->sc_quadrature = 1;
  p->sensor_mode = CVWENO_SENSOR_COMPUTED;
  p->lambda_const = 0.0;
  p->gas_gamma = 1.4;
  p->adv_vx = 1.0;
  p->adv_vy = 0.0;
}

const char* cvweno_status_string(cvweno_status s) {
  switch (s) {
    case CVWENO_OK: return "ok";
    case CVWENO_ERR_ARG: return "invalid argument";
    case CVWENO_ERR_CUDA: return "CUDA runtime error";
    case CVWENO_ERR_NONFINITE: return "non-finite value produced";
    case CVWENO_ERR_POSITIVITY: return "non-positive density or pressure";
    case CVWENO_ERR_TIMEOUT: return "bounded device wait timed out";
    case CVWENO_ERR_UNSUPPORTED: return "unsupported configuration";
    case CVWENO_ERR_NOMEM: return "out of memory";
    case CVWENO_ERR_CHECK: return "bounds check failed (checked build)";
  }
  return "unknown status";
}

cvweno_status cvweno_mesh_destroy(cvweno_mesh m) {
  if (!m) return CVWENO_OK;
  if (m->d_u1) cudaDeviceSynchronize();
  cudaFree(m->d_u1);
  cudaFree(m->d_u2);
  cudaFree(m->d_lambda);
  cudaFree(m->d_red);
  cudaFree(m->d_status);
  cudaFree(m->d_rloc);
  cudaFree(m->d_r);
  cudaFree(m->d_du);
  cudaFree(m->d_du2);
  cudaFree(m->d_cg_xg);
  cudaFree(m->d_cg_ml);
  cudaFree(m->d_tabimg);
  cudaFreeHost(m->h_status);
  cudaFreeHost(m->h_red);
  for (int i = 0; i < kMaxMarks; ++i)
    if (m->tev[i]) cudaEventDestroy(m->tev[i]);
  free(m->cell_vertices);
  free(m->vertex_cells);
  free(m->colour);
  free(m->tables);
  free(m->cg_tables);
  free(m);
  return CVWENO_OK;
}

cvweno_status cvweno_mesh_create(const cvweno_mesh_desc* d, cvweno_mesh* out) {
  if (!d || !out) return CVWENO_ERR_ARG;
  *out = nullptr;
  if (d->dim != 1 && d->dim != 2) return CVWENO_ERR_ARG;
  if (d->nx < 1 || (d->dim == 2 && d->ny < 1)) return CVWENO_ERR_ARG;
  if (d->nx > (1 << 24) || (d->dim == 2 && d->ny > (1 << 20))) return CVWENO_ERR_ARG;
  if (!(d->x1 > d->x0) || (d->dim == 2 && !(d->y1 > d->y0))) return CVWENO_ERR_ARG;
  for (int i = 0; i < 4; ++i)
    if (d->bc[i] != CVWENO_PERIODIC && d->bc[i] != CVWENO_TRANSMISSIVE) return CVWENO_ERR_ARG;
  if ((d->bc[0] == CVWENO_PERIODIC) != (d->bc[1] == CVWENO_PERIODIC)) return CVWENO_ERR_ARG;
  if (d->dim == 2 && (d->bc[2] == CVWENO_PERIODIC) != (d->bc[3] == CVWENO_PERIODIC)) return CVWENO_ERR_ARG;
  if (d->system < CVWENO_BURGERS || d->system > CVWENO_EULER) return CVWENO_ERR_ARG;
  const cvweno_params& p = d->params;
  if (!(p.eps > 0.0) || !(p.q >= 1.0) || !(p.gamma_vertex > 0.0) || (1 << d->dim) * p.gamma_vertex >= 1.0)
    return CVWENO_ERR_ARG;
  if (p.sensor_mode < 0 || p.sensor_mode > 2) return CVWENO_ERR_ARG;
  if (p.hweno_limiter != 0 && p.hweno_limiter != 1) return CVWENO_ERR_ARG;
  if (p.hweno_limiter && (d->kind != CVWENO_DG || d->system == CVWENO_EULER)) return CVWENO_ERR_UNSUPPORTED;
  if (p.positivity != 0 && p.positivity != 1) return CVWENO_ERR_ARG;
  if (p.positivity && (d->kind != CVWENO_DG || d->system != CVWENO_EULER)) return CVWENO_ERR_UNSUPPORTED;
  if (d->kind != CVWENO_DG && d->kind != CVWENO_CG) return CVWENO_ERR_ARG;
  // CG: scalar laws on periodic meshes (no boundary flux term is implemented)
  if (d->kind == CVWENO_CG && (d->system == CVWENO_EULER || d->bc[0] != CVWENO_PERIODIC ||
                               (d->dim == 2 && d->bc[2] != CVWENO_PERIODIC)))
    return CVWENO_ERR_UNSUPPORTED;
  if (d->degree < 1 || d->degree > kMaxP) return CVWENO_ERR_UNSUPPORTED;
  if (p.r != floor(p.r) || p.r < 1.0 || p.r > 8.0) return CVWENO_ERR_UNSUPPORTED;
  if ((d->system == CVWENO_KPP || d->system == CVWENO_EULER) && d->dim != 2) return CVWENO_ERR_UNSUPPORTED;

  cvweno_mesh m = (cvweno_mesh)calloc(1, sizeof(cvweno_mesh_s));
  if (!m) return CVWENO_ERR_NOMEM;
  m->desc = *d;
  m->chk_state = m->chk_cell = -1;
  cudaGetDevice(&m->device);
  m->dim = d->dim;
  m->p = d->degree;
  m->n = d->degree + 1;
  m->nd = d->dim == 2 ? m->n * m->n : m->n;
  m->nq = m->nd;
  m->nvar = d->system == CVWENO_EULER ? 4 : 1;
  m->ncorner = 1 << d->dim;
  m->nx = d->nx;
  m->ny = d->dim == 2 ? d->ny : 1;
  m->vx = d->bc[0] == CVWENO_PERIODIC ? m->nx : m->nx + 1;
  m->vy = d->dim == 2 ? (d->bc[2] == CVWENO_PERIODIC ? m->ny : m->ny + 1) : 1;
  m->ncell = (int64_t)m->nx * m->ny;
  m->nvert = (int64_t)m->vx * m->vy;
  m->kind = d->kind;
  m->nnx = d->kind == CVWENO_CG ? m->p * m->nx : 0;
  m->nny = d->kind == CVWENO_CG ? (d->dim == 2 ? m->p * m->ny : 1) : 0;
  m->nnode = (int64_t)m->nnx * m->nny;
  m->nstate = d->kind == CVWENO_CG ? m->nnode * m->nvar : m->ncell * m->nd * m->nvar;
  m->dx = (d->x1 - d->x0) / m->nx;
  m->dy = d->dim == 2 ? (d->y1 - d->y0) / m->ny : 1.0;
  m->h = d->dim == 2 ? sqrt(m->dx * m->dx + m->dy * m->dy) : m->dx;

  cvweno_status st = build_tables(m);
  if (st != CVWENO_OK) { cvweno_mesh_destroy(m); return st; }
  cudaError_t e = cudaSuccess;
  size_t sbytes = sizeof(float) * (size_t)m->nstate;
  if (e == cudaSuccess) e = cudaMalloc(&m->d_u1, sbytes);
  if (e == cudaSuccess) e = cudaMalloc(&m->d_u2, sbytes);
  if (e == cudaSuccess) e = cudaMalloc(&m->d_lambda, sizeof(float) * (size_t)m->ncell);
  if (e == cudaSuccess) e = cudaMalloc(&m->d_tabimg, sizeof(float) * (size_t)tab_image_floats(m->dim, m->p));
  if (e == cudaSuccess) e = launch_tab_image(m->dim, m->p, m->tables, m->d_tabimg, 0);
  if (e == cudaSuccess) e = cudaStreamSynchronize(0);
  if (m->kind == CVWENO_CG) {
    if (e == cudaSuccess) e = cudaMalloc(&m->d_rloc, sizeof(float) * (size_t)m->ncell * m->nd);
    if (m->dim == 1) {  // 2D meshes keep the node phase in one kernel's shared memory
      if (e == cudaSuccess) e = cudaMalloc(&m->d_du2, sizeof(float) * (size_t)m->nnode);
      if (e == cudaSuccess) e = cudaMalloc(&m->d_r, sizeof(float) * (size_t)m->nnode);
      if (e == cudaSuccess) e = cudaMalloc(&m->d_du, sizeof(float) * (size_t)m->nnode);
    }
    if (e == cudaSuccess) e = cudaMalloc(&m->d_cg_xg, sizeof(float) * (kMaxP + 1));
    if (e == cudaSuccess) e = cudaMalloc(&m->d_cg_ml, sizeof(double) * 2 * (kMaxP + 1));
    if (e == cudaSuccess) {
      float xg[kMaxP + 1];
      double ml[2 * (kMaxP + 1)];
      for (int i = 0; i <= kMaxP; ++i) {
        xg[i] = i <= m->p ? (float)m->cg_xg[i] : 0.0f;
        const double w = i <= m->p ? m->cg_wl[i] * (i == 0 ? 2.0 : 1.0) : 0.0;  // vertex nodes: two cells
        ml[i] = w * 0.5 * m->dx;
        ml[kMaxP + 1 + i] = m->dim == 2 ? w * 0.5 * m->dy : 1.0;
      }
      e = cudaMemcpy(m->d_cg_xg, xg, sizeof(xg), cudaMemcpyHostToDevice);
      if (e == cudaSuccess) e = cudaMemcpy(m->d_cg_ml, ml, sizeof(ml), cudaMemcpyHostToDevice);
    }
  }
  if (e == cudaSuccess) e = cudaMalloc(&m->d_red, sizeof(double) * (kRedBlocks + 8));
  if (e == cudaSuccess) e = cudaMalloc(&m->d_status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(m->d_status, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMallocHost(&m->h_status, sizeof(int));
  if (e == cudaSuccess) e = cudaMallocHost(&m->h_red, sizeof(double) * 8);
  if (e != cudaSuccess) {
    cvweno_mesh_destroy(m);
    return e == cudaErrorMemoryAllocation ? CVWENO_ERR_NOMEM : CVWENO_ERR_CUDA;
  }
  *out = m;
  return CVWENO_OK;
}

cvweno_status cvweno_mesh_info(cvweno_mesh m, int64_t* ncells, int64_t* ndof, int* nvars, int64_t* nverts,
                               int* nquad) {
  if (!m) return CVWENO_ERR_ARG;
  if (ncells) *ncells = m->ncell;
  if (ndof) *ndof = m->nd;
  if (nvars) *nvars = m->nvar;
  if (nverts) *nverts = m->nvert;
  if (nquad) *nquad = m->nq;
  return CVWENO_OK;
}

cvweno_status cvweno_state_size(cvweno_mesh m, int64_t* nstate) {
  if (!m || !nstate) return CVWENO_ERR_ARG;
  *nstate = m->nstate;
  return CVWENO_OK;
}

cvweno_status cvweno_mesh_tables(cvweno_mesh m, int32_t* cell_vertices, int32_t* vertex_cells, int32_t* colour) {
  if (!m) return CVWENO_ERR_ARG;
  if (cell_vertices) memcpy(cell_vertices, m->cell_vertices, sizeof(int32_t) * m->ncell * m->ncorner);
  if (vertex_cells) memcpy(vertex_cells, m->vertex_cells, sizeof(int32_t) * m->nvert * m->ncorner);
  if (colour) memcpy(colour, m->colour, sizeof(int32_t) * m->ncell);
  return CVWENO_OK;
}

cvweno_status cvweno_project(cvweno_mesh m, int ic_type, const double* ic_params, float* u, void* stream) {
  if (!m || !ic_params || !u) return CVWENO_ERR_ARG;
  if (ic_type < CVWENO_IC_CONST || ic_type > CVWENO_IC_DENSITY_WAVE) return CVWENO_ERR_ARG;
  if ((ic_type == CVWENO_IC_QUADRANTS || ic_type == CVWENO_IC_DENSITY_WAVE) != (m->nvar == 4) &&
      ic_type != CVWENO_IC_CONST)
    return CVWENO_ERR_ARG;
  ProjArgs a;
  memset(&a, 0, sizeof(a));
  a.u = u;
  a.nx = m->nx;
  a.ny = m->ny;
  a.dim = m->dim;
  a.nd = m->nd;
  a.n = m->n;
  a.nvar = m->nvar;
  a.type = ic_type;
  a.x0 = m->desc.x0;
  a.y0 = m->desc.y0;
  a.dx = m->dx;
  a.dy = m->dy;
  a.lx = m->desc.x1 - m->desc.x0;
  a.ly = m->dim == 2 ? m->desc.y1 - m->desc.y0 : 1.0;
  a.gas_gamma = m->desc.params.gas_gamma;
  for (int i = 0; i < 64; ++i) a.prm[i] = (float)ic_params[i];
  // Gauss nodes/weights of the 12-point projection rule and Legendre values there.
  ProjTables T;
  {
    static_assert(kProjN <= kMaxGaussRule, "projection rule larger than the Gauss rule builder");
    double x[kProjN], w[kProjN], pv[kMaxP + 1];
    if (!gauss_rule(kProjN, x, w)) return CVWENO_ERR_ARG;
    for (int q = 0; q < kProjN; ++q) {
      T.x[q] = (float)x[q];
      T.w[q] = (float)w[q];
      legendre_values(x[q], kMaxP, pv);
      for (int mm = 0; mm <= kMaxP; ++mm) T.P[q][mm] = (float)pv[mm];
    }
  }
  if (m->kind == CVWENO_CG) {
    int blocks = (int)((m->nnode + 255) / 256);
    if (blocks > 65535) blocks = 65535;
    project_cg_kernel<<<blocks, 256, 0, S(stream)>>>(a, T, m->p, m->nnx, m->nny, m->d_cg_xg);
    return cuda_status(cudaGetLastError());
  }
  int blocks = (int)((m->ncell + 127) / 128);
  if (blocks > 65535) blocks = 65535;
  project_kernel<<<blocks, 128, 0, S(stream)>>>(a, T);
  return cuda_status(cudaGetLastError());
}

cvweno_status cvweno_vertex_data(cvweno_mesh m, const float* u, float* tstar, void* stream) {
  if (!m || !u || !tstar) return CVWENO_ERR_ARG;
  NvtxRange range("cvweno_vertex_data");
  StageArgs a = base_args(m);
  a.u_in = u;
  a.tstar_out = tstar;
  a.mode = kModeSensorOnly;
  return cuda_status(launch(m, a, S(stream)));
}

cvweno_status cvweno_sensor(cvweno_mesh m, const float* u, float* gamma, float* nu, void* stream) {
  if (!m || !u) return CVWENO_ERR_ARG;
  NvtxRange range("cvweno_sensor");
  StageArgs a = base_args(m);
  a.u_in = u;
  a.gamma_out = gamma;
  a.nu_out = nu;
  a.mode = kModeSensorOnly;
  return cuda_status(launch(m, a, S(stream)));
}

cvweno_status cvweno_positivity(cvweno_mesh m, const float* u, float* out, float* theta, void* stream) {
  if (!m || !u || !out) return CVWENO_ERR_ARG;
  if (m->kind != CVWENO_DG || m->desc.system != CVWENO_EULER || m->dim != 2) return CVWENO_ERR_UNSUPPORTED;
  StageArgs a = base_args(m);
  a.u_in = u;
  a.u_out = out;
  return cuda_status(launch_positivity(m, a, theta, S(stream)));
}

cvweno_status cvweno_limit(cvweno_mesh m, const float* u, float* out, int all_cells, int32_t* troubled,
                           void* stream) {
  if (!m || !u || !out || u == out) return CVWENO_ERR_ARG;
  if (m->kind != CVWENO_DG || m->desc.system == CVWENO_EULER) return CVWENO_ERR_UNSUPPORTED;
  NvtxRange range("cvweno_limit");
  StageArgs a = base_args(m);
  a.u_in = u;
  a.u_out = out;
  a.troubled_out = troubled;
  a.limit_all = all_cells ? 1 : 0;
  a.mode = kModeLimit;
  return cuda_status(launch(m, a, S(stream)));
}

cvweno_status cvweno_residual_ex(cvweno_mesh m, const float* u, const int32_t* troubled_override, float* dudt,
                                 float* gamma, float* nu, float* alpha, int32_t* troubled, void* stream) {
  if (!m || !u || !dudt || u == dudt) return CVWENO_ERR_ARG;
  NvtxRange range("cvweno_residual");
  StageArgs a = base_args(m);
  a.u_in = u;
  a.u_n = u;
  a.u_out = dudt;
  a.gamma_out = gamma;
  a.nu_out = nu;
  a.alpha_out = alpha;
  a.troubled_out = troubled;
  a.troubled_override = troubled_override;
  a.mode = kModeResidual;
  return cuda_status(launch(m, a, S(stream)));
}

cvweno_status cvweno_residual(cvweno_mesh m, const float* u, float* dudt, void* stream) {
  return cvweno_residual_ex(m, u, nullptr, dudt, nullptr, nullptr, nullptr, nullptr, stream);
}

cvweno_status cvweno_max_wavespeed(cvweno_mesh m, const float* u, double* lam, void* stream) {
  if (!m || !u || !lam) return CVWENO_ERR_ARG;
  cudaStream_t s = S(stream);
  StageArgs a = base_args(m);
  a.u_in = u;
  a.lambda_out = m->d_lambda;
  a.mode = kModeSensorOnly;
  cudaError_t e = launch(m, a, s);
  if (e == cudaSuccess) {
    max_partial<<<kRedBlocks, kRedThreads, 0, s>>>(m->d_lambda, m->ncell, m->d_red);
    finish_reduce<<<1, kRedThreads, 0, s>>>(m->d_red, kRedBlocks, 1, m->d_red + kRedBlocks);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(m->h_red, m->d_red + kRedBlocks, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return CVWENO_ERR_CUDA;
  cvweno_status st = read_status(m, s);  // synchronises
  if (st != CVWENO_OK) return st;
  *lam = m->h_red[0];
  return CVWENO_OK;
}

cvweno_status cvweno_step(cvweno_mesh m, float* u, double dt, double cfl, double* dt_used, void* stream) {
  if (!m || !u) return CVWENO_ERR_ARG;
  NvtxRange range("cvweno_step");
  cudaStream_t s = S(stream);
  if (!(dt > 0.0)) {
    if (!(cfl > 0.0)) return CVWENO_ERR_ARG;
    double lam = 0.0;
    cvweno_status st = cvweno_max_wavespeed(m, u, &lam, stream);
    if (st != CVWENO_OK) return st;
    if (!(lam > 0.0)) return CVWENO_ERR_ARG;
    double hmin = m->dim == 2 ? fmin(m->dx, m->dy) : m->dx;
    dt = cfl * hmin / (m->dim * lam);
  }
  if (dt_used) *dt_used = dt;
  return enqueue_step(m, u, (float)dt, s);
}

cvweno_status cvweno_advance(cvweno_mesh m, float* u, double dt, int nsteps, void* stream) {
  if (!m || !u || !(dt > 0.0) || nsteps < 0) return CVWENO_ERR_ARG;
  NvtxRange range("cvweno_advance");
  if (nsteps > 0 && steps_in_one_launch(m)) return enqueue_steps_one_launch(m, u, (float)dt, nsteps, S(stream));
  for (int i = 0; i < nsteps; ++i) {
    cvweno_status st = enqueue_step(m, u, (float)dt, S(stream));
    if (st != CVWENO_OK) return st;
  }
  return CVWENO_OK;
}

cvweno_status cvweno_mass_total(cvweno_mesh m, const float* u, double* totals, void* stream) {
  if (!m || !u || !totals) return CVWENO_ERR_ARG;
  cudaStream_t s = S(stream);
  if (m->kind == CVWENO_CG) {
    // sum_j ML_j u_j with ML_j = ml1x(I mod p) ml1y(J mod p)
    sum_cg_partial<<<kRedBlocks, kRedThreads, 0, s>>>(u, m->nnx, m->nny, m->p, m->d_cg_ml, m->d_cg_ml + (kMaxP + 1),
                                                     m->d_red);
    finish_reduce<<<1, kRedThreads, 0, s>>>(m->d_red, kRedBlocks, 0, m->d_red + kRedBlocks);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(m->h_red, m->d_red + kRedBlocks, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return CVWENO_ERR_CUDA;
    totals[0] = m->h_red[0];
    return CVWENO_OK;
  }
  // int_{K_e} u_h = |K_e| * (Legendre mode 0)
  const double vol = m->dim == 2 ? m->dx * m->dy : m->dx;
  for (int v = 0; v < m->nvar; ++v) {
    const float* base = u + (size_t)v * m->ncell * m->nd;
    sum_mode0_partial<<<kRedBlocks, kRedThreads, 0, s>>>(base, m->ncell, m->nd, m->d_red);
    finish_reduce<<<1, kRedThreads, 0, s>>>(m->d_red, kRedBlocks, 0, m->d_red + kRedBlocks + v);
  }
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(m->h_red, m->d_red + kRedBlocks, sizeof(double) * m->nvar, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return CVWENO_ERR_CUDA;
  for (int v = 0; v < m->nvar; ++v) totals[v] = m->h_red[v] * vol;
  return CVWENO_OK;
}

cvweno_status cvweno_mesh_set_kernel_timing(cvweno_mesh m, int enable) {
  if (!m) return CVWENO_ERR_ARG;
  if (enable && !m->tev[0])
    for (int i = 0; i < kMaxMarks; ++i)
      if (cudaEventCreate(&m->tev[i]) != cudaSuccess) return CVWENO_ERR_CUDA;
  m->timing = enable ? 1 : 0;
  if (enable) m->tcount = 0;  // disabling keeps the last step's events readable
  return CVWENO_OK;
}

cvweno_status cvweno_mesh_set_tensor_cores(cvweno_mesh m, int enable) {
  if (!m || (enable != 0 && enable != 1)) return CVWENO_ERR_ARG;
  if (enable && !(m->dim == 2 && m->kind == CVWENO_DG && m->p == 3 && m->desc.system != CVWENO_EULER))
    return CVWENO_ERR_UNSUPPORTED;
  m->tensor_cores = enable;
  return CVWENO_OK;
}

cvweno_status cvweno_mesh_set_check_extents(cvweno_mesh m, int64_t state_floats, int64_t cells) {
  if (!m || state_floats > m->nstate || cells > m->ncell || ((state_floats < 0) != (cells < 0)))
    return CVWENO_ERR_ARG;
#ifdef CVWENO_CHECK
  m->chk_state = state_floats;
  m->chk_cell = cells;
  return CVWENO_OK;
#else
  return CVWENO_ERR_UNSUPPORTED;
#endif
}

cvweno_status cvweno_kernel_times(cvweno_mesh m, float* ms, int capacity, int* count) {
  if (!m || !count || capacity < 0 || (capacity > 0 && !ms)) return CVWENO_ERR_ARG;
  *count = 0;
  if (!m->tev[0] || m->tcount < 2) return CVWENO_OK;
  if (cudaEventSynchronize(m->tev[m->tcount - 1]) != cudaSuccess) return CVWENO_ERR_CUDA;
  const int n = m->tcount - 1 < capacity ? m->tcount - 1 : capacity;
  for (int i = 0; i < n; ++i)
    if (cudaEventElapsedTime(&ms[i], m->tev[i], m->tev[i + 1]) != cudaSuccess) return CVWENO_ERR_CUDA;
  *count = n;
  return CVWENO_OK;
}

cvweno_status cvweno_status_check(cvweno_mesh m, void* stream) {
  if (!m) return CVWENO_ERR_ARG;
  return read_status(m, S(stream));
}

}  // extern "C"
