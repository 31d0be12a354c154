// FP32 instantiations of the 2D row / column kernels.
#include "fs_k2d_impl.cuh"

namespace fs {
cudaError_t row_launch_f32(const KArgs& a, cudaStream_t s) { return row_launch_t<float>(a, s); }
cudaError_t col_launch_f32(const KArgs& a, const CUtensorMap& tm, cudaStream_t s) {
  return col_launch_t<float>(a, tm, s);
}
cudaError_t sum_launch_f32(const void* x, long long n, double* out, cudaStream_t s) {
  return sum_launch_t<float>(x, n, out, s);
}
int col_tile_width(bool f64, int nx, int ny) { return f64 ? col_tk_t<double>(nx, ny) : col_tk_t<float>(nx, ny); }
cudaError_t energy_col_launch_f32(const KArgs& a, const CUtensorMap& tm, cudaStream_t s) {
  return energy_col_launch_t<float>(a, tm, s);
}
}  // namespace fs
