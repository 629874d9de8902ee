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
