// float instantiations of the batched ensemble kernels.
#include "fs_batch_impl.cuh"

namespace fs {
cudaError_t row_batch_launch_f32(const BatchArgs& b, cudaStream_t s) { return row_batch_launch_t<float>(b, s); }
cudaError_t col_batch_launch_f32(const BatchArgs& b, cudaStream_t s) { return col_batch_launch_t<float>(b, s); }
size_t row_smem_f32(int nx, int nf) { return row_smem_t<float>(nx, nf); }
long long row_blocks_f32(int nx, long long lines) { return row_blocks_t<float>(nx, lines); }
int col_batch_tk_f32(int nx, int ny) { return col_batch_tk_t<float>(nx, ny); }
size_t col_smem_f32(int ny, int tk) { return col_smem_t<float>(ny, tk); }
}  // namespace fs
