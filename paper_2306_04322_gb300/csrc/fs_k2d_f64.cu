// FP64 instantiations of the 2D row / column kernels.
#include "fs_k2d_impl.cuh"

namespace fs {
cudaError_t row_launch_f64(const KArgs& a, cudaStream_t s) { return row_launch_t<double>(a, s); }
cudaError_t col_launch_f64(const KArgs& a, const CUtensorMap& tm, cudaStream_t s) {
  return col_launch_t<double>(a, tm, s);
}
cudaError_t sum_launch_f64(const void* x, long long n, double* out, cudaStream_t s) {
  return sum_launch_t<double>(x, n, out, s);
}
cudaError_t energy_col_launch_f64(const KArgs& a, const CUtensorMap& tm, cudaStream_t s) {
  return energy_col_launch_t<double>(a, tm, s);
}
}  // namespace fs
