// Instantiations of the fused scalar stage kernel for uniform 1D meshes, and of the
// one-launch step kernel for a 1D mesh that is a single tile.
#include "dg_scalar_launch.cuh"

namespace cvw {

cudaError_t launch_stage_1d(const cvweno_mesh_s* m, const StageArgs& a, cudaStream_t s) {
  constexpr int TX = kTile1D;
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

template <int P, int SYS>
static cudaError_t launch_steps_tile(const cvweno_mesh_s* m, const StepArgs& a, cudaStream_t s) {
  constexpr int TX = kTile1D;
  using Lay = TileLayout<1, P, TX, 1>;
  static_assert(Lay::BYTES <= 48 * 1024, "a 1D tile fits the default shared memory");
  if (m->tables_bytes != sizeof(DgTables<1, P>)) return cudaErrorInvalidValue;
  return launch_pdl(dg_scalar_steps_tile<P, SYS, TX>, dim3(1), dim3(stage_block_threads<1, P, TX, 1>()), Lay::BYTES,
                    s, a, *static_cast<const DgTables<1, P>*>(m->tables));
}

cudaError_t launch_steps_1d_tile(const cvweno_mesh_s* m, const StepArgs& a, cudaStream_t s) {
  if (m->dim != 1 || a.st[0].nx > kTile1D || a.nsteps < 1) return cudaErrorNotSupported;
  switch (m->p * 10 + m->desc.system) {
    case 10 + CVWENO_BURGERS: return launch_steps_tile<1, CVWENO_BURGERS>(m, a, s);
    case 20 + CVWENO_BURGERS: return launch_steps_tile<2, CVWENO_BURGERS>(m, a, s);
    case 30 + CVWENO_BURGERS: return launch_steps_tile<3, CVWENO_BURGERS>(m, a, s);
    case 40 + CVWENO_BURGERS: return launch_steps_tile<4, CVWENO_BURGERS>(m, a, s);
    case 10 + CVWENO_LINADV: return launch_steps_tile<1, CVWENO_LINADV>(m, a, s);
    case 20 + CVWENO_LINADV: return launch_steps_tile<2, CVWENO_LINADV>(m, a, s);
    case 30 + CVWENO_LINADV: return launch_steps_tile<3, CVWENO_LINADV>(m, a, s);
    case 40 + CVWENO_LINADV: return launch_steps_tile<4, CVWENO_LINADV>(m, a, s);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace cvw
