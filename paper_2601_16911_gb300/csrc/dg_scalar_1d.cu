// Instantiations of the fused scalar stage kernel for uniform 1D meshes.
#include "dg_scalar_launch.cuh"

namespace cvw {

cudaError_t launch_stage_1d(const cvweno_mesh_s* m, const StageArgs& a, cudaStream_t s) {
  constexpr int TX = 128;
  switch (m->p * 10 + m->desc.system) {
    case 10 + CVWENO_BURGERS: return launch_scalar<1, 1, CVWENO_BURGERS, TX, 1>(m, a, s);
    case 20 + CVWENO_BURGERS: return launch_scalar<1, 2, CVWENO_BURGERS, TX, 1>(m, a, s);
    case 30 + CVWENO_BURGERS: return launch_scalar<1, 3, CVWENO_BURGERS, TX, 1>(m, a, s);
    case 40 + CVWENO_BURGERS: return launch_scalar<1, 4, CVWENO_BURGERS, TX, 1>(m, a, s);
    case 10 + CVWENO_LINADV: return launch_scalar<1, 1, CVWENO_LINADV, TX, 1>(m, a, s);
    case 20 + CVWENO_LINADV: return launch_scalar<1, 2, CVWENO_LINADV, TX, 1>(m, a, s);
    case 30 + CVWENO_LINADV: return launch_scalar<1, 3, CVWENO_LINADV, TX, 1>(m, a, s);
    case 40 + CVWENO_LINADV: return launch_scalar<1, 4, CVWENO_LINADV, TX, 1>(m, a, s);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace cvw
