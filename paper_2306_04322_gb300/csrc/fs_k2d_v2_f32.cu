// FP32 instantiations of the warp-per-line row (pair form) and column passes:
// lines of 64 to 1024 points held by one warp (G = 1, tables tw_row2 /
// tw_col2) or, from 128 points, by two warps (G = 2, tables tw_row2w /
// tw_col2w; columns up to 2048 points).
#include "fs_k2d_v2.cuh"

namespace fs {
static bool v2_size(int n) { return n == 64 || n == 128 || n == 256 || n == 512 || n == 1024; }
bool row2_supported(int nx, int nf) { return v2_size(nx) && nf >= 1 && nf <= 5; }
bool col2_supported(int ny, int nf) { return (v2_size(ny) || ny == 2048) && nf >= 1 && nf <= 5; }

template <int G>
cudaError_t row2_launch_g(const KArgs& a, cudaStream_t s) {
  switch (a.nx) {
    case 64: if constexpr (G == 1) return row2_launch_n<64, G>(a, s); else return cudaErrorNotSupported;
    case 128: return row2_launch_n<128, G>(a, s);
    case 256: return row2_launch_n<256, G>(a, s);
    case 512: return row2_launch_n<512, G>(a, s);
    case 1024: return row2_launch_n<1024, G>(a, s);
    default: return cudaErrorNotSupported;
  }
}
template <int G>
cudaError_t col2_launch_g(const KArgs& a, const CUtensorMap& tm, cudaStream_t s) {
  switch (a.ny) {
    case 64: if constexpr (G == 1) return col2_launch_n<64, G>(a, tm, s); else return cudaErrorNotSupported;
    case 128: return col2_launch_n<128, G>(a, tm, s);
    case 256: return col2_launch_n<256, G>(a, tm, s);
    case 512: return col2_launch_n<512, G>(a, tm, s);
    case 1024: return col2_launch_n<1024, G>(a, tm, s);
    case 2048: if constexpr (G == 2) return col2_launch_n<2048, G>(a, tm, s); else return cudaErrorNotSupported;
    default: return cudaErrorNotSupported;
  }
}

cudaError_t row2_launch_f32(const KArgs& a, cudaStream_t s) {
  if (a.mode > 2 || !row2_supported(a.nx, a.nf) || a.lines % 2) return cudaErrorNotSupported;
  if (a.tw_row2w) return row2_launch_g<2>(a, s);
  if (a.tw_row2) return row2_launch_g<1>(a, s);
  return cudaErrorNotSupported;
}
cudaError_t col2_launch_f32(const KArgs& a, const CUtensorMap& tm, cudaStream_t s) {
  if (a.tc != 0 || a.nz != 1 || !col2_supported(a.ny, a.nf) || a.nx < 4) return cudaErrorNotSupported;
  if (a.tw_col2w) return col2_launch_g<2>(a, tm, s);
  if (a.tw_col2) return col2_launch_g<1>(a, tm, s);
  return cudaErrorNotSupported;
}
}  // namespace fs
