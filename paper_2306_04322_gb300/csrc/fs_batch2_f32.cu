// Ensemble (batched) launches of the warp-per-line forms, FP32: a persistent
// grid walks the work list of every member -- row pairs for the row pass,
// (column pair, field group) for the column pass -- members ordered largest
// first, each item running the body instantiated for its member's size.
// The plan's autotuner times these against the half-length / tile ensemble
// kernels and keeps the faster form and grid size per pass.
#include "fs_batch_impl.cuh"
#include "fs_k2d_v2.cuh"

namespace fs {

#define FS_V2_SIZES(X) X(64) X(128) X(256) X(512) X(1024)

__global__ void __launch_bounds__(Row2Cfg<1024>::MAX_THREADS, 3)
    fs_row2_batch_kernel(const KArgs* __restrict__ mem, const long long* __restrict__ begin, int nm,
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
    const long long rp = item - begin[m];
    bool ok = true;
    switch (a.nx) {
#define FS_CASE(n) \
  case n: ok = row2_body<n>(a, rp, smem_raw, bar, parity); break;
      FS_V2_SIZES(FS_CASE)
#undef FS_CASE
      default: break;
    }
    // a bounded wait that gave up ends the whole CTA (every thread sees it)
    if (__syncthreads_or(!ok)) return;
    parity ^= 1u;
  }
}

__global__ void __launch_bounds__(128, 4)
    fs_col2_batch_kernel(const KArgs* __restrict__ mem, const CUtensorMap* __restrict__ maps,
                         const long long* __restrict__ begin, const int* __restrict__ pairs, int nm,
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
    const int np = pairs[m];
    const int rem = (int)(item - begin[m]);
    const int group = rem / np, cp = rem % np;
    bool ok = true;
    switch (a.ny) {
#define FS_CASE(n) \
  case n: ok = col2_body<n>(a, &maps[m], cp, group, smem_raw, bar, parity); break;
      FS_V2_SIZES(FS_CASE)
#undef FS_CASE
      default: break;
    }
    if (__syncthreads_or(!ok)) return;
    parity ^= 1u;
  }
}

size_t row2_smem_f32(int nx, int nf) {
  switch (nx) {
#define FS_CASE(n) \
  case n: return row2_smem_bytes<n>(nf);
    FS_V2_SIZES(FS_CASE)
#undef FS_CASE
    default: return 0;
  }
}
size_t col2_smem_f32(int ny) {
  switch (ny) {
#define FS_CASE(n) \
  case n: return col2_smem_bytes<n>();
    FS_V2_SIZES(FS_CASE)
#undef FS_CASE
    default: return 0;
  }
}
int col2_groups(int nf) { return 1 + (nf - 1 + 1) / 2; }

cudaError_t row2_batch_launch_f32(const BatchArgs& b, cudaStream_t s) {
  static unsigned done = 0;
  cudaError_t e = allow_big_smem(fs_row2_batch_kernel, &done);
  if (e != cudaSuccess) return e;
  fs_row2_batch_kernel<<<(unsigned)b.row2_grid, (unsigned)(32 * (b.nf1 - 1)), b.row2_smem, s>>>(
      b.mem, b.row2_begin, b.nm, b.row2_total);
  return cudaGetLastError();
}

cudaError_t col2_batch_launch_f32(const BatchArgs& b, cudaStream_t s) {
  static unsigned done = 0;
  cudaError_t e = allow_big_smem(fs_col2_batch_kernel, &done);
  if (e != cudaSuccess) return e;
  fs_col2_batch_kernel<<<(unsigned)b.col2_grid, 128, b.col2_smem, s>>>(b.mem_col, b.maps2, b.col2_begin,
                                                                      b.col2_pairs, b.nm, b.col2_total);
  return cudaGetLastError();
}

}  // namespace fs
