// cvweno_step_static: one SSP-RK3 step that allocates nothing.
//
// Some callers cannot allocate: code that runs inside a memory pool or arena it does not
// own, an embedding that forbids cudaMalloc after start-up, or a process whose
// allocator must not be re-entered from a library.  For them this entry point advances a
// caller-owned state by one SSP-RK3 step without creating a mesh (mesh creation
// allocates).  Everything it needs lives elsewhere:
//   - the two RK stage buffers live in one file-scope __device__ array of fixed size
//     (kStaticStateFloats floats per buffer, 2 buffers, 32 MiB in total), which every
//     GPU that loads the library holds until the process exits;
//   - its device status word is a second file-scope __device__ variable;
//   - the reference-cell tabulations are built on the host stack.
// It calls no cudaMalloc, cudaFree, malloc or other allocating routine.
#include <math.h>
#include <string.h>

#include <mutex>

#include "cvweno_internal.cuh"

namespace {

constexpr size_t kStaticStateFloats = size_t(1) << 22;  // per stage buffer (16 MiB)
constexpr int kMaxDevices = 64;

static __device__ __align__(256) float g_stage_scratch[2 * kStaticStateFloats];
static __device__ __align__(256) int g_static_status;
static __device__ __align__(256) float g_static_tab_image[cvw::kMaxTabImage];

struct DeviceSlots {
  float* scratch;
  int* status;
  float* tab_image;
};
DeviceSlots g_slots[kMaxDevices];
bool g_ready[kMaxDevices];
std::mutex g_mutex;

// Device addresses of the static scratch, looked up once per device with that device
// current (host code must not pass the symbols themselves to a kernel).
cudaError_t static_slots(DeviceSlots* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_ready[dev]) {
    DeviceSlots s;
    e = cudaGetSymbolAddress((void**)&s.scratch, g_stage_scratch);
    if (e != cudaSuccess) return e;
    e = cudaGetSymbolAddress((void**)&s.status, g_static_status);
    if (e != cudaSuccess) return e;
    e = cudaGetSymbolAddress((void**)&s.tab_image, g_static_tab_image);
    if (e != cudaSuccess) return e;
    g_slots[dev] = s;
    g_ready[dev] = true;
  }
  *out = g_slots[dev];
  return cudaSuccess;
}

// ---- host tabulations on the stack (FP64, rounded once) ------------------------------------

constexpr int kMaxN = cvw::kMaxP + 1;

void sym_eigen(int n, double a[8][8], double lam[8], double v[8][8]) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) v[i][j] = i == j ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j) off += a[i][j] * a[i][j];
    if (off < 1e-300) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        if (fabs(a[p][q]) < 1e-300) continue;
        double th = (a[q][q] - a[p][p]) / (2.0 * a[p][q]);
        double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
        double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {
          double akp = a[k][p], akq = a[k][q];
          a[k][p] = c * akp - s * akq;
          a[k][q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {
          double apk = a[p][k], aqk = a[q][k];
          a[p][k] = c * apk - s * aqk;
          a[q][k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          double vkp = v[k][p], vkq = v[k][q];
          v[k][p] = c * vkp - s * vkq;
          v[k][q] = s * vkp + c * vkq;
        }
      }
  }
  for (int i = 0; i < n; ++i) lam[i] = a[i][i];
}

// Gauss-Legendre rule (n <= 8) from the Legendre Jacobi matrix, ascending nodes.
void gauss(int n, double* x, double* w) {
  double J[8][8] = {}, lam[8], V[8][8];
  for (int k = 1; k < n; ++k) J[k - 1][k] = J[k][k - 1] = k / sqrt(4.0 * k * k - 1.0);
  sym_eigen(n, J, lam, V);
  int idx[8];
  for (int i = 0; i < n; ++i) idx[i] = i;
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j)
      if (lam[idx[j]] < lam[idx[i]]) { int t = idx[i]; idx[i] = idx[j]; idx[j] = t; }
  for (int i = 0; i < n; ++i) {
    x[i] = lam[idx[i]];
    w[i] = 2.0 * V[0][idx[i]] * V[0][idx[i]];
  }
  for (int i = 0; i < n / 2; ++i) {
    double xm = 0.5 * (x[n - 1 - i] - x[i]), wm = 0.5 * (w[i] + w[n - 1 - i]);
    x[i] = -xm;
    x[n - 1 - i] = xm;
    w[i] = w[n - 1 - i] = wm;
  }
  if (n % 2) x[n / 2] = 0.0;
}

// out[k][m] = D^k P_m(x) for m, k < kMaxN
void leg(double x, double out[kMaxN][kMaxN]) {
  for (int k = 0; k < kMaxN; ++k)
    for (int m = 0; m < kMaxN; ++m) out[k][m] = 0.0;
  out[0][0] = 1.0;
  out[0][1] = x;
  for (int m = 1; m + 1 < kMaxN; ++m) out[0][m + 1] = ((2.0 * m + 1.0) * x * out[0][m] - m * out[0][m - 1]) / (m + 1.0);
  for (int k = 1; k < kMaxN; ++k) {
    out[k][1] = k == 1 ? 1.0 : 0.0;
    for (int m = 1; m + 1 < kMaxN; ++m) out[k][m + 1] = out[k][m - 1] + (2.0 * m + 1.0) * out[k - 1][m];
  }
}

template <int DIM, int P>
bool fill_tables(cvw::DgTables<DIM, P>& t, double dx, double dy, double h) {
  using T = cvw::DgTables<DIM, P>;
  constexpr int N = T::N, ND = T::ND, NS = T::NS, NC = T::NC;
  memset(&t, 0, sizeof(t));
  double gx[N], gw[N], L[kMaxN][kMaxN];
  gauss(N, gx, gw);
  leg(1.0, L);
  for (int k = 0; k < N; ++k)
    for (int m = 0; m < N; ++m) t.E[k][m] = (float)L[k][m];
  for (int q = 0; q < N; ++q) {
    leg(gx[q], L);
    for (int m = 0; m < N; ++m) {
      t.B[q][m] = (float)L[0][m];
      t.Bd[q][m] = (float)L[1][m];
      for (int k = 0; k < N; ++k) t.Bk[k][q][m] = (float)L[k][m];
    }
    t.w[q] = (float)gw[q];
  }
  // scalings as functions of h/dx and h/dy only (h = sqrt(dx^2 + dy^2) in 2D, dx in 1D)
  (void)h;
  const double ax = DIM == 2 ? sqrt(1.0 + (dy / dx) * (dy / dx)) : 1.0;
  const double ay = DIM == 2 ? sqrt((dx / dy) * (dx / dy) + 1.0) : 1.0;
  for (int k = 0; k < ND; ++k) {
    int kx = k % N, ky = DIM == 2 ? k / N : 0;
    t.sigma[k] = k == 0 ? 0.0f : (float)(pow(2.0 * ax, 2 * kx) * (DIM == 2 ? pow(2.0 * ay, 2 * ky) : 1.0));
    t.tscale[k] = (float)(pow(2.0 / dx, kx) * (DIM == 2 ? pow(2.0 / dy, ky) : 1.0));
  }
  const int NG = 8;
  double qx[NG], qw[NG];
  gauss(NG, qx, qw);
  double g[kMaxN][kMaxN][kMaxN] = {};
  for (int q = 0; q < NG; ++q) {
    leg(qx[q], L);
    for (int k = 0; k < N; ++k)
      for (int a = 0; a < N; ++a)
        for (int b = 0; b < N; ++b) g[k][a][b] += qw[q] * L[k][a] * L[k][b];
  }
  double G[ND][ND] = {};
  for (int k = 1; k < ND; ++k) {
    int kx = k % N, ky = DIM == 2 ? k / N : 0;
    // h^(2|k| - dim) (2/dx)^(2kx) (2/dy)^(2ky) |J|
    double rho = pow(2.0 * ax, 2 * kx) * (DIM == 2 ? pow(2.0 * ay, 2 * ky) : 1.0) /
                 (DIM == 2 ? 4.0 * ax * ay : 2.0 * ax);
    for (int a = 0; a < ND; ++a)
      for (int b = 0; b < ND; ++b) {
        double v = g[kx][a % N][b % N];
        if (DIM == 2) v *= g[ky][a / N][b / N];
        G[a][b] += rho * v;
      }
  }
  double R[NS][NS] = {};
  for (int j = 0; j < NS; ++j) {
    double s = G[j + 1][j + 1];
    for (int k = 0; k < j; ++k) s -= R[k][j] * R[k][j];
    if (!(s > 0.0)) return false;
    R[j][j] = sqrt(s);
    for (int i = j + 1; i < NS; ++i) {
      double v = G[j + 1][i + 1];
      for (int k = 0; k < j; ++k) v -= R[k][j] * R[k][i];
      R[j][i] = v / R[j][j];
    }
  }
  for (int i = 0; i < NS; ++i)
    for (int j = 0; j < NS; ++j) t.R[i][j] = (float)R[i][j];
  double Gs[2][kMaxN][kMaxN] = {};
  for (int si = 0; si < 2; ++si)
    for (int a = 0; a < N; ++a)
      for (int k = 0; k < N; ++k) {
        double acc = 0.0, fk = 1.0;
        for (int i = 2; i <= k; ++i) fk *= i;
        for (int q = 0; q < NG; ++q) {
          leg(qx[q], L);
          acc += qw[q] * L[0][a] * pow(qx[q] - (si ? 1.0 : -1.0), k) / fk;
        }
        Gs[si][a][k] = 0.5 * (2 * a + 1) * acc;
      }
  for (int l = 0; l < NC; ++l) {
    int sxi = l & 1, syi = (l >> 1) & 1;
    for (int i = 0; i < NS; ++i)
      for (int j = 0; j < NS; ++j) {
        double acc = 0.0;
        for (int k = i; k < NS; ++k) {
          int a = k + 1, b = j + 1;
          double c = Gs[sxi][a % N][b % N];
          if (DIM == 2) c *= Gs[syi][a / N][b / N];
          acc += R[i][k] * c;
        }
        t.A[l][i][j] = (float)acc;
      }
  }
  return true;
}

// Large enough for every DgTables<DIM, P> instance.
union AnyTables {
  cvw::DgTables<1, 1> t11;
  cvw::DgTables<1, 2> t12;
  cvw::DgTables<1, 3> t13;
  cvw::DgTables<1, 4> t14;
  cvw::DgTables<2, 1> t21;
  cvw::DgTables<2, 2> t22;
  cvw::DgTables<2, 3> t23;
  cvw::DgTables<2, 4> t24;
};

}  // namespace

extern "C" cvweno_status cvweno_step_static(const cvweno_mesh_desc* d, float* u, double dt, int32_t* status_out,
                                            void* stream) {
  using namespace cvw;
  if (!d || !u || !(dt > 0.0)) return CVWENO_ERR_ARG;
  if (d->dim != 1 && d->dim != 2) return CVWENO_ERR_ARG;
  if (d->nx < 1 || (d->dim == 2 && d->ny < 1)) return CVWENO_ERR_ARG;
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
  if (p.hweno_limiter || p.positivity) return CVWENO_ERR_UNSUPPORTED;  // limited steps are not in this variant
  if (d->kind != CVWENO_DG || d->degree < 1 || d->degree > kMaxP) return CVWENO_ERR_UNSUPPORTED;
  if (p.r != floor(p.r) || p.r < 1.0 || p.r > 8.0) return CVWENO_ERR_UNSUPPORTED;
  if ((d->system == CVWENO_KPP || d->system == CVWENO_EULER) && d->dim != 2) return CVWENO_ERR_UNSUPPORTED;

  // the mesh description this step needs, on the stack
  cvweno_mesh_s m;
  memset(&m, 0, sizeof(m));
  m.desc = *d;
  m.dim = d->dim;
  m.p = d->degree;
  m.n = d->degree + 1;
  m.nd = d->dim == 2 ? m.n * m.n : m.n;
  m.nq = m.nd;
  m.nvar = d->system == CVWENO_EULER ? 4 : 1;
  m.ncorner = 1 << d->dim;
  m.nx = d->nx;
  m.ny = d->dim == 2 ? d->ny : 1;
  m.vx = d->bc[0] == CVWENO_PERIODIC ? m.nx : m.nx + 1;
  m.vy = d->dim == 2 ? (d->bc[2] == CVWENO_PERIODIC ? m.ny : m.ny + 1) : 1;
  m.ncell = (int64_t)m.nx * m.ny;
  m.nvert = (int64_t)m.vx * m.vy;
  m.nstate = m.ncell * m.nd * m.nvar;
  if ((size_t)m.nstate > kStaticStateFloats) return CVWENO_ERR_ARG;  // beyond the static scratch
  m.dx = (d->x1 - d->x0) / m.nx;
  m.dy = d->dim == 2 ? (d->y1 - d->y0) / m.ny : 1.0;
  m.h = d->dim == 2 ? sqrt(m.dx * m.dx + m.dy * m.dy) : m.dx;

  AnyTables tabs;
  bool ok = false;
  switch (m.dim * 10 + m.p) {
    case 11: ok = fill_tables(tabs.t11, m.dx, m.dy, m.h); m.tables_bytes = sizeof(tabs.t11); break;
    case 12: ok = fill_tables(tabs.t12, m.dx, m.dy, m.h); m.tables_bytes = sizeof(tabs.t12); break;
    case 13: ok = fill_tables(tabs.t13, m.dx, m.dy, m.h); m.tables_bytes = sizeof(tabs.t13); break;
    case 14: ok = fill_tables(tabs.t14, m.dx, m.dy, m.h); m.tables_bytes = sizeof(tabs.t14); break;
    case 21: ok = fill_tables(tabs.t21, m.dx, m.dy, m.h); m.tables_bytes = sizeof(tabs.t21); break;
    case 22: ok = fill_tables(tabs.t22, m.dx, m.dy, m.h); m.tables_bytes = sizeof(tabs.t22); break;
    case 23: ok = fill_tables(tabs.t23, m.dx, m.dy, m.h); m.tables_bytes = sizeof(tabs.t23); break;
    case 24: ok = fill_tables(tabs.t24, m.dx, m.dy, m.h); m.tables_bytes = sizeof(tabs.t24); break;
    default: return CVWENO_ERR_UNSUPPORTED;
  }
  if (!ok) return CVWENO_ERR_ARG;
  m.tables = &tabs;

  DeviceSlots slots;
  if (static_slots(&slots) != cudaSuccess) return CVWENO_ERR_CUDA;
  float* u1 = slots.scratch;
  float* u2 = slots.scratch + kStaticStateFloats;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // the tabulation image first: the stage kernels read it before their dependent-launch
  // wait, so a stream operation that is not one of them (the status reset) separates them
  if (launch_tab_image(m.dim, m.p, m.tables, slots.tab_image, s) != cudaSuccess) return CVWENO_ERR_CUDA;
  // the status word must start at zero for this step; the stage buffers are fully
  // written before they are read
  if (cudaMemsetAsync(slots.status, 0, sizeof(int), s) != cudaSuccess) return CVWENO_ERR_CUDA;

  StageArgs a;
  memset(&a, 0, sizeof(a));
  a.status = slots.status;
  a.nx = m.nx;
  a.ny = m.ny;
  a.perx = d->bc[0] == CVWENO_PERIODIC;
  a.pery = m.dim == 2 && d->bc[2] == CVWENO_PERIODIC;
  a.vx = m.vx;
  a.two_dx = (float)(2.0 / m.dx);
  a.two_dy = (float)(2.0 / m.dy);
  a.nu_scale = (float)(m.h / (2.0 * m.p));
  a.h_e = (float)m.h;
  a.tab_img = slots.tab_image;
  a.eps = (float)p.eps;
  a.r = (int)p.r;
  a.q = (float)p.q;
  a.gamma_vertex = (float)p.gamma_vertex;
  a.c_gamma = (float)p.c_gamma;
  a.lambda_const = (float)p.lambda_const;
  a.sc = p.sc_quadrature;
  a.sensor_mode = p.sensor_mode;
  a.adv_vx = (float)p.adv_vx;
  a.adv_vy = (float)p.adv_vy;
  a.gas_gamma = (float)p.gas_gamma;
  a.mode = kModeRK;
  a.dt = (float)dt;
  const float* ins[3] = {u, u1, u2};
  float* outs[3] = {u1, u2, u};
  const float ra[3] = {0.0f, 0.75f, 1.0f / 3.0f}, rb[3] = {1.0f, 0.25f, 2.0f / 3.0f};
  for (int st = 0; st < 3; ++st) {
    a.u_in = ins[st];
    a.u_n = u;
    a.u_out = outs[st];
    a.rk_a = ra[st];
    a.rk_b = rb[st];
    cudaError_t e = d->system == CVWENO_EULER ? launch_stage_euler(&m, a, s) : launch_stage(&m, a, s);
    if (e != cudaSuccess) return CVWENO_ERR_CUDA;
  }
  if (status_out) {
    int st = 0;
    if (cudaMemcpyAsync(&st, slots.status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return CVWENO_ERR_CUDA;
    *status_out = st;
    if (st & kStatPositivity) return CVWENO_ERR_POSITIVITY;
    if (st & kStatNonfinite) return CVWENO_ERR_NONFINITE;
  }
  return CVWENO_OK;
}
