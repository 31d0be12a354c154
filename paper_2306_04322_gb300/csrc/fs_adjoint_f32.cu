// float instantiations of the adjoint kernels.
#include "fs_adjoint_impl.cuh"

namespace fs {
cudaError_t adjoint_launch_f32(const KArgs& a, const CUtensorMap& tm, void* lam_out, cudaStream_t s) {
  return adjoint_launch_t<float>(a, tm, lam_out, s);
}
cudaError_t adjoint3_launch_f32(const KArgs& a, const CUtensorMap& tm_y, const CUtensorMap& tm_z, void* lam_out,
                               cudaStream_t s) {
  return adjoint3_launch_t<float>(a, tm_y, tm_z, lam_out, s);
}
}  // namespace fs
