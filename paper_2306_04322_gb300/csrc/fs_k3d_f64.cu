// double instantiations of the 3D y / z passes.
#include "fs_k2d_impl.cuh"
#include "fs_k3d_impl.cuh"

namespace fs {
cudaError_t ypass_launch_f64(const KArgs& a, const CUtensorMap& tm, int dir, int nslots, cudaStream_t s) {
  return ypass_launch_t<double>(a, tm, dir, nslots, s);
}
cudaError_t zstep_launch_f64(const KArgs& a, const CUtensorMap& tm, cudaStream_t s) {
  return zstep_launch_t<double>(a, tm, s);
}
cudaError_t energy_z_launch_f64(const KArgs& a, const CUtensorMap& tm, cudaStream_t s) {
  return energy_z_launch_t<double>(a, tm, s);
}
int line_tile_width_f64(int nx, int nl) { return line_tk_t<double>(nx, nl); }
}  // namespace fs
