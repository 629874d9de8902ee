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
//   - the reference-cell tabulations are built on the host stack by the library's one
//     tabulation builder (fill_dg_tables, tables.cpp), the same that meshes use.
// It calls no cudaMalloc, cudaFree, malloc or other allocating routine.
//
// The device addresses of that storage are looked up once per device (static_slots), with
// the device current, by the first call on it.  Under CUDA's lazy module loading (the
// default) that lookup also loads this module, which is when the storage comes into
// existence on the device: make the first call at start-up, before reserving an arena
// of all free memory and before any stream capture.  The cached addresses belong to the
// device's current context: do not call it across a cudaDeviceReset of that device.
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
// current (in host code the symbols are host-side stand-ins: passed to a kernel they
// would fault or, where the GPU can reach host memory, silently use the wrong memory).
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
  NvtxRange range("cvweno_step_static");
  // the checks of cvweno_mesh_create, in its order and with its codes
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
  if (p.positivity != 0 && p.positivity != 1) return CVWENO_ERR_ARG;
  if (d->kind != CVWENO_DG && d->kind != CVWENO_CG) return CVWENO_ERR_ARG;
  if (d->degree < 1 || d->degree > kMaxP) return CVWENO_ERR_UNSUPPORTED;
  if (p.r != floor(p.r) || p.r < 1.0 || p.r > 8.0) return CVWENO_ERR_UNSUPPORTED;
  if ((d->system == CVWENO_KPP || d->system == CVWENO_EULER) && d->dim != 2) return CVWENO_ERR_UNSUPPORTED;
  // what this variant leaves out: CG meshes and the limited steps
  if (d->kind != CVWENO_DG || p.hweno_limiter || p.positivity) return CVWENO_ERR_UNSUPPORTED;

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
  const cvweno_status tst = fill_dg_tables(m.dim, m.p, m.dx, m.dy, &tabs, sizeof(tabs), &m.tables_bytes);
  if (tst != CVWENO_OK) return tst;
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
  set_check_extents(a, m.nstate, m.ncell);
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
    if (st & kStatCheck) return CVWENO_ERR_CHECK;
    if (st & kStatPositivity) return CVWENO_ERR_POSITIVITY;
    if (st & kStatNonfinite) return CVWENO_ERR_NONFINITE;
  }
  return CVWENO_OK;
}
