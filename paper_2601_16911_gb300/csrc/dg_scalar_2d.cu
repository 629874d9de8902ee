// Instantiations of the fused scalar stage kernel for uniform quadrilateral meshes.
#include "dg_scalar_launch.cuh"

namespace cvw {

cudaError_t launch_stage_1d(const cvweno_mesh_s* m, const StageArgs& a, cudaStream_t s);
cudaError_t launch_stage_surrogate(const cvweno_mesh_s* m, const StageArgs& a, cudaStream_t s);

cudaError_t launch_stage(const cvweno_mesh_s* m, const StageArgs& a, cudaStream_t s) {
  if (m->dim == 1) return launch_stage_1d(m, a, s);
  if ((a.mlp && !(a.mode & kModeLimit)) || (a.mode & kModeFeatures)) return launch_stage_surrogate(m, a, s);
  constexpr int TX = 16, TY = 8;
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

}  // namespace cvw
