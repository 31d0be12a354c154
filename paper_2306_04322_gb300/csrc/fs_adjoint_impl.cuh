// Launch sequence of the adjoint of one 2D step (three kernels).
#pragma once

#include "fs_adjoint.cuh"
#include "fs_adjoint3.cuh"
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

template <typename T, int NZ>
cudaError_t adj_z_n(const KArgs& a, const CUtensorMap& tm, cudaStream_t s) {
  using Cfg = LineCfg<T, NZ>;
  const int tk = line_tk<T, NZ>(a.nx);
  const size_t smem = Cfg::HEAD + (size_t)3 * Cfg::TROWS * tk * sizeof(cplx<T>);
  static unsigned d = 0;
  cudaError_t e = allow_big_smem(fs_adj_z_kernel<T, NZ>, &d);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)(a.nx / 2 / tk), (unsigned)a.ny, (unsigned)a.nf);
  fs_adj_z_kernel<T, NZ><<<grid, (unsigned)(tk * Cfg::TPL), smem, s>>>(a, tm);
  return cudaGetLastError();
}

// Adjoint of one 3D step (five launches): x forward of lam', u, f(u) (the
// 2D adjoint's row kernel over ny nz rows), y forward of the 3 nf slots (the
// step's y pass), the z part (fs_adj_z_kernel), y inverse of the 2 nf result
// slots, x inverse with the pointwise Hessian product.  tm_y: [slot nz + z][y]
// [kx] over the adjoint slots; tm_z: [slot][z][y][kx].
template <typename T>
cudaError_t adjoint3_launch_t(const KArgs& a0, const CUtensorMap& tm_y, const CUtensorMap& tm_z, void* lam_out,
                              cudaStream_t s) {
  cudaError_t e = cudaErrorInvalidValue;
  switch (a0.nx) {
#define FS_CASE(n) \
  case n: e = adj_row_n<T, n>(a0, false, s); break;
    FS_ADJ_SIZES(FS_CASE)
#undef FS_CASE
    default: break;
  }
  if (e != cudaSuccess) return e;
  KArgs b = a0;
  b.carry3 = 0;  // plain y transforms of every slot (no carried c)
  b.plane0 = 0;
  b.tc = 0;
  constexpr bool f64 = sizeof(T) == 8;
  e = f64 ? ypass_launch_f64(b, tm_y, -1, 3 * a0.nf, s) : ypass_launch_f32(b, tm_y, -1, 3 * a0.nf, s);
  if (e != cudaSuccess) return e;
  e = cudaErrorInvalidValue;
  switch (a0.nz) {
#define FS_CASE(n) \
  case n: e = adj_z_n<T, n>(b, tm_z, s); break;
    FS_LINE_SIZES(FS_CASE)
#undef FS_CASE
    default: break;
  }
  if (e != cudaSuccess) return e;
  e = f64 ? ypass_launch_f64(b, tm_y, 1, 2 * a0.nf, s) : ypass_launch_f32(b, tm_y, 1, 2 * a0.nf, s);
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
