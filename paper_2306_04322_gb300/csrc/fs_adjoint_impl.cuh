// Launch sequence of the adjoint of one 2D step (three kernels).
#pragma once

#include "fs_adjoint.cuh"
#include "fs_k2d_impl.cuh"

namespace fs {

template <typename T, int NX>
size_t adj_row_smem(int nf) {
  using RC = RowCfg<T, NX>;
  return RC::BAR_BYTES + RC::TW_BYTES + (size_t)3 * nf * RC::R * RC::PL * sizeof(cplx<T>);
}

template <typename T, int NX>
cudaError_t adj_row_n(const KArgs& a, bool inverse, cudaStream_t s) {
  using RC = RowCfg<T, NX>;
  const long long reff = a.lines < RC::R ? a.lines : RC::R;
  const size_t smem = adj_row_smem<T, NX>(a.nf);
  const unsigned threads = 32 * (a.nf + 1);
  static unsigned d1 = 0, d2 = 0;
  cudaError_t e;
  if (!inverse) {
    e = allow_big_smem(fs_adj_row_fwd_kernel<T, NX>, &d1);
    if (e != cudaSuccess) return e;
    fs_adj_row_fwd_kernel<T, NX><<<(unsigned)(a.lines / reff), threads, smem, s>>>(a);
  } else {
    e = allow_big_smem(fs_adj_row_inv_kernel<T, NX>, &d2);
    if (e != cudaSuccess) return e;
    fs_adj_row_inv_kernel<T, NX><<<(unsigned)(a.lines / reff), threads, smem, s>>>(a);
  }
  return cudaGetLastError();
}

template <typename T, int NY>
cudaError_t adj_col_n(const KArgs& a, const CUtensorMap& tm, cudaStream_t s) {
  using CC = ColCfg<T, NY>;
  const int tk = col_tk_n<T, NY>(a.nx);
  const size_t smem = CC::HEAD + (size_t)3 * CC::TROWS * tk * sizeof(cplx<T>);
  static unsigned d = 0;
  cudaError_t e = allow_big_smem(fs_adj_col_kernel<T, NY>, &d);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)(a.nx / 2 / tk), (unsigned)a.nf);
  fs_adj_col_kernel<T, NY><<<grid, (unsigned)(tk * CC::TPL), smem, s>>>(a, tm);
  return cudaGetLastError();
}

#define FS_ADJ_SIZES(X) X(8) X(16) X(32) X(64) X(128) X(256) X(512) X(1024)

template <typename T>
cudaError_t adjoint_launch_t(const KArgs& a0, const CUtensorMap& tm, void* lam_out, cudaStream_t s) {
  cudaError_t e = cudaErrorInvalidValue;
  switch (a0.nx) {
#define FS_CASE(n) \
  case n: e = adj_row_n<T, n>(a0, false, s); break;
    FS_ADJ_SIZES(FS_CASE)
#undef FS_CASE
    default: break;
  }
  if (e != cudaSuccess) return e;
  e = cudaErrorInvalidValue;
  switch (a0.ny) {
#define FS_CASE(n) \
  case n: e = adj_col_n<T, n>(a0, tm, s); break;
    FS_ADJ_SIZES(FS_CASE)
#undef FS_CASE
    default: break;
  }
  if (e != cudaSuccess) return e;
  KArgs a1 = a0;
  a1.real = lam_out;
  e = cudaErrorInvalidValue;
  switch (a0.nx) {
#define FS_CASE(n) \
  case n: e = adj_row_n<T, n>(a1, true, s); break;
    FS_ADJ_SIZES(FS_CASE)
#undef FS_CASE
    default: break;
  }
  return e;
}

}  // namespace fs
