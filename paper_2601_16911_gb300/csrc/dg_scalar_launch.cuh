// Host-side launcher of the fused scalar stage kernel.
#pragma once

#include "dg_scalar_kernel.cuh"

namespace cvw {

template <int DIM, int P, int SYS, int TX, int TY, bool SURR>
constexpr auto stage_kernel() {
  if constexpr (SURR)
    return dg_scalar_stage_surrogate<DIM, P, SYS, TX, TY>;
  else
    return dg_scalar_stage<DIM, P, SYS, TX, TY>;
}

template <int DIM, int P, int SYS, int TX, int TY, bool SURR = false>
cudaError_t launch_scalar(const cvweno_mesh_s* m, const StageArgs& a, cudaStream_t s) {
  using Tb = DgTables<DIM, P>;
  using Lay = TileLayout<DIM, P, TX, TY>;
  static_assert(Lay::BYTES_MLP <= 200 * 1024, "tile too large for shared memory");
  const size_t smem = (SURR && a.mlp) ? Lay::BYTES_MLP : Lay::BYTES;
  auto kern = stage_kernel<DIM, P, SYS, TX, TY, SURR>();
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  if (m->tables_bytes != sizeof(Tb)) return cudaErrorInvalidValue;
  dim3 grid((a.nx + TX - 1) / TX, DIM == 2 ? (a.ny + TY - 1) / TY : 1);
  const int threads = stage_block_threads<DIM, P, TX, TY>();
  return launch_pdl(kern, grid, dim3(threads), smem, s, a, *static_cast<const Tb*>(m->tables));
}

// The tensor-core form of the 2D Q3 stage kernel (8 x 16 tiles, TileLayout<..., true>).
template <int SYS>
cudaError_t launch_scalar_tc(const cvweno_mesh_s* m, const StageArgs& a, cudaStream_t s) {
  using Tb = DgTables<2, 3>;
  using Lay = TileLayout<2, 3, 8, 16, true>;
  static_assert(4 * (Lay::BYTES + 1024) <= 228 * 1024, "the tensor-core tile must leave 4 CTAs per SM");
  auto kern = dg_scalar_stage_tc<SYS>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Lay::BYTES);
  if (e != cudaSuccess) return e;
  if (m->tables_bytes != sizeof(Tb)) return cudaErrorInvalidValue;
  dim3 grid((a.nx + 7) / 8, (a.ny + 15) / 16);
  return launch_pdl(kern, grid, dim3(128), Lay::BYTES, s, a, *static_cast<const Tb*>(m->tables));
}

}  // namespace cvw
