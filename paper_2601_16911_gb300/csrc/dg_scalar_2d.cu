// Instantiations of the fused scalar stage kernel for uniform quadrilateral meshes.
#include "dg_scalar_launch.cuh"

namespace cvw {

cudaError_t launch_stage_1d(const cvweno_mesh_s* m, const StageArgs& a, cudaStream_t s);
cudaError_t launch_stage_surrogate(const cvweno_mesh_s* m, const StageArgs& a, cudaStream_t s);

cudaError_t launch_stage(const cvweno_mesh_s* m, const StageArgs& a, cudaStream_t s) {
  if (m->dim == 1) return launch_stage_1d(m, a, s);
  if ((a.mlp && !(a.mode & kModeLimit)) || (a.mode & kModeFeatures)) return launch_stage_surrogate(m, a, s);
  constexpr int TX = 16, TY = 8;
  if (m->tensor_cores && m->p == 3) {
    switch (m->desc.system) {
      case CVWENO_BURGERS: return launch_scalar_tc<CVWENO_BURGERS>(m, a, s);
      case CVWENO_KPP: return launch_scalar_tc<CVWENO_KPP>(m, a, s);
      case CVWENO_LINADV: return launch_scalar_tc<CVWENO_LINADV>(m, a, s);
      default: return cudaErrorNotSupported;
    }
  }
  switch (m->p * 10 + m->desc.system) {
    case 10 + CVWENO_BURGERS: return launch_scalar<2, 1, CVWENO_BURGERS, TX, TY>(m, a, s);
    case 20 + CVWENO_BURGERS: return launch_scalar<2, 2, CVWENO_BURGERS, TX, TY>(m, a, s);
    case 30 + CVWENO_BURGERS: return launch_scalar<2, 3, CVWENO_BURGERS, TX, TY>(m, a, s);
    case 40 + CVWENO_BURGERS: return launch_scalar<2, 4, CVWENO_BURGERS, TX, TY>(m, a, s);
    case 10 + CVWENO_KPP: return launch_scalar<2, 1, CVWENO_KPP, TX, TY>(m, a, s);
    case 20 + CVWENO_KPP: return launch_scalar<2, 2, CVWENO_KPP, TX, TY>(m, a, s);
    case 30 + CVWENO_KPP: return launch_scalar<2, 3, CVWENO_KPP, TX, TY>(m, a, s);
    case 40 + CVWENO_KPP: return launch_scalar<2, 4, CVWENO_KPP, TX, TY>(m, a, s);
    case 10 + CVWENO_LINADV: return launch_scalar<2, 1, CVWENO_LINADV, TX, TY>(m, a, s);
    case 20 + CVWENO_LINADV: return launch_scalar<2, 2, CVWENO_LINADV, TX, TY>(m, a, s);
    case 30 + CVWENO_LINADV: return launch_scalar<2, 3, CVWENO_LINADV, TX, TY>(m, a, s);
    case 40 + CVWENO_LINADV: return launch_scalar<2, 4, CVWENO_LINADV, TX, TY>(m, a, s);
    default: return cudaErrorNotSupported;
  }
}

namespace {
template <int DIM, int P>
cudaError_t tab_image(const void* t, float* dst, cudaStream_t s) {
  tab_image_kernel<DIM, P><<<1, 256, 0, s>>>(*static_cast<const DgTables<DIM, P>*>(t), dst);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_tab_image(int dim, int p, const void* t, float* dst, cudaStream_t s) {
  if (!t || !dst) return cudaErrorInvalidValue;
  switch (dim * 10 + p) {
    case 11: return tab_image<1, 1>(t, dst, s);
    case 12: return tab_image<1, 2>(t, dst, s);
    case 13: return tab_image<1, 3>(t, dst, s);
    case 14: return tab_image<1, 4>(t, dst, s);
    case 21: return tab_image<2, 1>(t, dst, s);
    case 22: return tab_image<2, 2>(t, dst, s);
    case 23: return tab_image<2, 3>(t, dst, s);
    case 24: return tab_image<2, 4>(t, dst, s);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace cvw

namespace cvw {
namespace {
// sin d and cos d - 1 as the KPP flux forms them: the series up to |d| = 1, the reduced
// series beyond (ScalarLaw<KPP>::flux_dev).
__global__ void kpp_sincos_kernel(const float* __restrict__ d, float* __restrict__ out, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    float s, cm1;
    if (fabsf(d[i]) <= 1.0f)
      sin_cosm1_small(d[i], s, cm1);
    else
      sin_cosm1_reduced(d[i], s, cm1);
    out[i] = s;
    out[n + i] = cm1;
  }
}
}  // namespace
}  // namespace cvw

extern "C" cvweno_status cvweno_kpp_sincos(const float* d, float* out, int n, void* stream) {
  if (n < 0 || (n > 0 && (!d || !out))) return CVWENO_ERR_ARG;
  if (n == 0) return CVWENO_OK;
  const int threads = 256, blocks = (n + threads - 1) / threads < 1024 ? (n + threads - 1) / threads : 1024;
  cvw::kpp_sincos_kernel<<<blocks, threads, 0, static_cast<cudaStream_t>(stream)>>>(d, out, n);
  return cudaGetLastError() == cudaSuccess ? CVWENO_OK : CVWENO_ERR_CUDA;
}
