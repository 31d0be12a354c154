// FP32 instantiations of the warp-per-line row (pair form) and column passes.
#include "fs_k2d_v2.cuh"

namespace fs {
bool row2_supported(int nx, int nf) { return (nx == 256 || nx == 512 || nx == 1024) && nf >= 1 && nf <= 5; }
bool col2_supported(int ny, int nf) { return (ny == 256 || ny == 512 || ny == 1024) && nf >= 1 && nf <= 5; }
cudaError_t row2_launch_f32(const KArgs& a, cudaStream_t s) {
  if (!a.tw_row2 || a.mode > 2 || !row2_supported(a.nx, a.nf) || a.lines % 2) return cudaErrorNotSupported;
  switch (a.nx) {
    case 256: return row2_launch_n<256>(a, s);
    case 512: return row2_launch_n<512>(a, s);
    case 1024: return row2_launch_n<1024>(a, s);
    default: return cudaErrorNotSupported;
  }
}
cudaError_t col2_launch_f32(const KArgs& a, const CUtensorMap& tm, cudaStream_t s) {
  if (!a.tw_col2 || a.tc != 0 || a.nz != 1 || !col2_supported(a.ny, a.nf) || a.nx < 4) return cudaErrorNotSupported;
  switch (a.ny) {
    case 256: return col2_launch_n<256>(a, tm, s);
    case 512: return col2_launch_n<512>(a, tm, s);
    case 1024: return col2_launch_n<1024>(a, tm, s);
    default: return cudaErrorNotSupported;
  }
}
}  // namespace fs
