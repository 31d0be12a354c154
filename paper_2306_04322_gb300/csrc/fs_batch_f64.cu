// double instantiations of the batched ensemble kernels.
#include "fs_batch_impl.cuh"

namespace fs {
cudaError_t row_batch_launch_f64(const BatchArgs& b, cudaStream_t s) { return row_batch_launch_t<double>(b, s); }
cudaError_t col_batch_launch_f64(const BatchArgs& b, cudaStream_t s) { return col_batch_launch_t<double>(b, s); }
size_t row_smem_f64(int nx, int nf) { return row_smem_t<double>(nx, nf); }
long long row_blocks_f64(int nx, long long lines) { return row_blocks_t<double>(nx, lines); }
int col_batch_tk_f64(int nx, int ny) { return col_batch_tk_t<double>(nx, ny); }
size_t col_smem_f64(int ny, int tk) { return col_smem_t<double>(ny, tk); }
}  // namespace fs
