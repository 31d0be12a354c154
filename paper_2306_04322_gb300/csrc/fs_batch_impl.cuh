// Batched ensemble: many independent 2D simulations of uneven grid sizes and
// parameters advanced by one launch per pass.  The launch is persistent: a
// grid of G CTAs (G picked by the plan's autotuner) walks a flat work list
// of (simulation, row block) or (simulation, column tile, field group) items;
// each item dispatches to the row / column body instantiated for that
// simulation's size.  Items of one simulation are contiguous; simulations
// are ordered largest first.
#pragma once

#include "fs_k2d_impl.cuh"

namespace fs {

// index of the simulation owning work item `item` (begin[] ascending, nm entries)
__device__ __forceinline__ int find_member(const long long* __restrict__ begin, int nm, long long item) {
  int lo = 0, hi = nm - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(&begin[mid]) <= item) lo = mid; else hi = mid - 1;
  }
  return lo;
}

#define FS_BATCH_SIZES(X) X(16) X(32) X(64) X(128) X(256) X(512) X(1024)

template <typename T>
__global__ void __launch_bounds__(128, RowCfg<T, 1024>::MIN_BLOCKS)
    fs_row_batch_kernel(const KArgs* __restrict__ mem, const long long* __restrict__ begin, int nm,
                        long long total) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t parity = 0;
  for (long long item = blockIdx.x; item < total; item += gridDim.x) {
    const int m = find_member(begin, nm, item);
    const KArgs& a = mem[m];
    const long long rb = item - begin[m];
    bool ok = false;
    switch (a.nx) {
#define FS_CASE(n) \
  case n: ok = row_body<T, n>(a, rb, smem_raw, bar, parity); break;
      FS_BATCH_SIZES(FS_CASE)
#undef FS_CASE
      default: break;
    }
    if (!ok) return;
    parity ^= 1u;
    __syncthreads();
  }
}

template <typename T>
__global__ void __launch_bounds__(256, 2)
    fs_col_batch_kernel(const KArgs* __restrict__ mem, const CUtensorMap* __restrict__ maps,
                        const long long* __restrict__ begin, const int* __restrict__ tiles, int nm,
                        long long total) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t parity = 0;
  for (long long item = blockIdx.x; item < total; item += gridDim.x) {
    const int m = find_member(begin, nm, item);
    const KArgs& a = mem[m];
    const int nt = tiles[m];
    const int rem = (int)(item - begin[m]);
    const int g = rem / nt, bx = rem % nt;
    bool ok = false;
    switch (a.ny) {
#define FS_CASE(n) \
  case n: ok = col_body<T, n>(a, &maps[m], bx, g, smem_raw, bar, parity); break;
      FS_BATCH_SIZES(FS_CASE)
#undef FS_CASE
      default: break;
    }
    if (!ok) return;
    parity ^= 1u;
    __syncthreads();
  }
}

// Host-side sizing helpers (per simulation).
template <typename T>
size_t row_smem_t(int nx, int nf) {
  switch (nx) {
#define FS_CASE(n) \
  case n: return row_smem_bytes<T, n>(nf);
    FS_BATCH_SIZES(FS_CASE)
#undef FS_CASE
    default: return 0;
  }
}
template <typename T>
long long row_blocks_t(int nx, long long lines) {
  switch (nx) {
#define FS_CASE(n) \
  case n: return lines / (lines < RowCfg<T, n>::R ? lines : RowCfg<T, n>::R);
    FS_BATCH_SIZES(FS_CASE)
#undef FS_CASE
    default: return 0;
  }
}
// column tile width when the batch column launch (256 threads) fits this
// size exactly, else 0
template <typename T>
int col_batch_tk_t(int nx, int ny) {
  switch (ny) {
#define FS_CASE(n)                                                              \
  case n: {                                                                     \
    using Cfg = ColCfg<T, n>;                                                   \
    return (Cfg::THREADS == 256 && Cfg::TK <= nx / 2) ? Cfg::TK : 0;            \
  }
    FS_BATCH_SIZES(FS_CASE)
#undef FS_CASE
    default: return 0;
  }
}
template <typename T>
size_t col_smem_t(int ny, int tk) {
  switch (ny) {
#define FS_CASE(n) \
  case n: return col_smem_bytes<T, n>(tk);
    FS_BATCH_SIZES(FS_CASE)
#undef FS_CASE
    default: return 0;
  }
}

template <typename T>
cudaError_t row_batch_launch_t(const BatchArgs& b, cudaStream_t s) {
  static unsigned done = 0;
  cudaError_t e = allow_big_smem(fs_row_batch_kernel<T>, &done);
  if (e != cudaSuccess) return e;
  fs_row_batch_kernel<T><<<(unsigned)b.row_grid, 128, b.row_smem, s>>>(
      b.mem, b.row_begin, b.nm, b.row_total);
  return cudaGetLastError();
}

template <typename T>
cudaError_t col_batch_launch_t(const BatchArgs& b, cudaStream_t s) {
  static unsigned done = 0;
  cudaError_t e = allow_big_smem(fs_col_batch_kernel<T>, &done);
  if (e != cudaSuccess) return e;
  fs_col_batch_kernel<T><<<(unsigned)b.col_grid, 256, b.col_smem, s>>>(b.mem_col, b.maps, b.col_begin,
                                                                         b.col_tiles, b.nm, b.col_total);
  return cudaGetLastError();
}

}  // namespace fs
