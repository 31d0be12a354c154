// Compile-time launch configuration shared by the kernels and the host-side
// table builders (the host builds twiddle tables for exactly the (L, E) pairs
// the kernels use).
#pragma once

namespace fs {

// Complex values per thread of a row (x) line FFT of length L = nx / 2:
// 16, or fewer for short rows; at most 32 threads per line.
constexpr int row_E(int L, bool f64) { return L < 16 ? L : (L / 16 > 32 ? L / 32 : 16); }
// Rows per row-pass CTA: one warp covers 32 / TPL rows of one field.
constexpr int row_R(int L, bool f64) { return 32 / (L / row_E(L, f64)); }
// Complex values per thread of a column (y or z) line FFT of length L.
constexpr int col_E(int L, bool f64) { return L < (f64 ? 8 : 16) ? L : (f64 ? 8 : 16); }
// Columns per column-pass CTA: about `threads` threads, at most 32 columns.
constexpr int col_tk(int L, bool f64, int threads = 256) {
  return (threads / (L / col_E(L, f64))) < 1 ? 1
         : ((threads / (L / col_E(L, f64))) > 32 ? 32 : (threads / (L / col_E(L, f64))));
}

}  // namespace fs
