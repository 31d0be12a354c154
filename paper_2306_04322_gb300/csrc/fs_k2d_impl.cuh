// Launch dispatch for the 2D row / column kernels of one precision.
#pragma once

#include <type_traits>

#include "fs_kernels.cuh"

namespace fs {

// Opt a kernel into the full dynamic shared-memory size once per device.
template <typename K>
cudaError_t allow_big_smem(K kernel, unsigned* done_mask) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  unsigned bit = 1u << (dev & 31);
  if (__atomic_load_n(done_mask, __ATOMIC_ACQUIRE) & bit) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  if (e == cudaSuccess) __atomic_fetch_or(done_mask, bit, __ATOMIC_RELEASE);
  return e;
}

// Launch with programmatic stream serialisation: the kernel may be scheduled
// while the previous kernel of the stream is still running.  Only kernels
// that call griddep_wait() before touching anything the previous kernel
// writes or reads are launched this way.
template <typename... KP, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KP...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <typename T, int NX, bool W>
cudaError_t row_launch_w(const KArgs& a, cudaStream_t s) {
  using Cfg = RowCfg<T, NX, W>;
  const long long reff = a.lines < Cfg::R ? a.lines : Cfg::R;
  const size_t smem = row_smem_bytes<T, NX, W>(a.nf);
  // five fields at 32 values per thread (rows of 2048, wide rows of 1024):
  // one warp per field (2048^2: 73.3 us against 76.8 us; with 16 values per
  // thread, whose CTAs pack more densely, the 3D 256^3 x pass lost 5 %)
  if constexpr (sizeof(T) == 4 && Cfg::E >= 32) {
    if (a.nf == 5) {
      static unsigned done5 = 0;
      cudaError_t e = allow_big_smem(fs_row_kernel<T, NX, W, 5>, &done5);
      if (e != cudaSuccess) return e;
      return launch_pdl(fs_row_kernel<T, NX, W, 5>, dim3((unsigned)(a.lines / reff)), dim3(160u), smem, s, a);
    }
  }
  static unsigned done = 0;
  cudaError_t e = allow_big_smem(fs_row_kernel<T, NX, W>, &done);
  if (e != cudaSuccess) return e;
  return launch_pdl(fs_row_kernel<T, NX, W>, dim3((unsigned)(a.lines / reff)), dim3((unsigned)Cfg::THREADS), smem, s,
                    a);
}

// FP32 rows of 1024 take the wide (radix 32, 16) variant when the plan
// provides its table.
template <typename T, int NX>
cudaError_t row_launch_n(const KArgs& a, cudaStream_t s) {
  if constexpr (sizeof(T) == 4 && NX == 1024) {
    if (a.tw_row_w) return row_launch_w<T, NX, true>(a, s);
  }
  return row_launch_w<T, NX, false>(a, s);
}

template <typename T, int NY>
int col_tk_n(int nx) {
  using Cfg = ColCfg<T, NY>;
  int Lh = nx / 2;
  return Cfg::TK < Lh ? Cfg::TK : Lh;
}

template <typename T, int NY, int TCM>
cudaError_t col_launch_tc(const KArgs& a, const CUtensorMap& tm, cudaStream_t s) {
  using Cfg = ColCfg<T, NY>;
  const int tk = col_tk_n<T, NY>(a.nx);
  size_t smem = col_smem_bytes<T, NY, TCM>(tk);
  static unsigned done = 0;
  cudaError_t e = allow_big_smem(fs_col_kernel<T, NY, TCM>, &done);
  if (e != cudaSuccess) return e;
  if (TCM == TC_TF32 && (tk * Cfg::TPL) % 128 != 0) return cudaErrorNotSupported;  // 128-row MMAs
  dim3 grid((unsigned)(a.nx / 2 / tk), (unsigned)a.nf);
  return launch_pdl(fs_col_kernel<T, NY, TCM>, grid, dim3((unsigned)(tk * Cfg::TPL)), smem, s, a, tm);
}

template <typename T, int NY>
cudaError_t col_launch_n(const KArgs& a, const CUtensorMap& tm, cudaStream_t s) {
  if constexpr (sizeof(T) == 4 && NY >= 64) {
    if (a.tc == TC_TF32) return col_launch_tc<T, NY, TC_TF32>(a, tm, s);
    if (a.tc == TC_BF16X3) return col_launch_tc<T, NY, TC_BF16X3>(a, tm, s);
  }
  if (a.tc != TC_NONE) return cudaErrorInvalidValue;
  return col_launch_tc<T, NY, TC_NONE>(a, tm, s);
}

template <typename T, int NY>
cudaError_t energy_col_launch_n(const KArgs& a, const CUtensorMap& tm, cudaStream_t s) {
  using Cfg = ColCfg<T, NY>;
  const int tk = col_tk_n<T, NY>(a.nx);
  size_t smem = Cfg::HEAD + (size_t)Cfg::TROWS * tk * sizeof(cplx<T>);
  static unsigned done = 0;
  cudaError_t e = allow_big_smem(fs_energy_col_kernel<T, NY>, &done);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)(a.nx / 2 / tk), (unsigned)a.nf);
  fs_energy_col_kernel<T, NY><<<grid, (unsigned)(tk * Cfg::TPL), smem, s>>>(a, tm);
  return cudaGetLastError();
}

template <typename T>
cudaError_t energy_col_launch_t(const KArgs& a, const CUtensorMap& tm, cudaStream_t s) {
  switch (a.ny) {
    case 8: return energy_col_launch_n<T, 8>(a, tm, s);
    case 16: return energy_col_launch_n<T, 16>(a, tm, s);
    case 32: return energy_col_launch_n<T, 32>(a, tm, s);
    case 64: return energy_col_launch_n<T, 64>(a, tm, s);
    case 128: return energy_col_launch_n<T, 128>(a, tm, s);
    case 256: return energy_col_launch_n<T, 256>(a, tm, s);
    case 512: return energy_col_launch_n<T, 512>(a, tm, s);
    case 1024: return energy_col_launch_n<T, 1024>(a, tm, s);
    case 2048: return energy_col_launch_n<T, 2048>(a, tm, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t row_launch_t(const KArgs& a, cudaStream_t s) {
  switch (a.nx) {
    case 8: return row_launch_n<T, 8>(a, s);
    case 16: return row_launch_n<T, 16>(a, s);
    case 32: return row_launch_n<T, 32>(a, s);
    case 64: return row_launch_n<T, 64>(a, s);
    case 128: return row_launch_n<T, 128>(a, s);
    case 256: return row_launch_n<T, 256>(a, s);
    case 512: return row_launch_n<T, 512>(a, s);
    case 1024: return row_launch_n<T, 1024>(a, s);
    case 2048: return row_launch_n<T, 2048>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t col_launch_t(const KArgs& a, const CUtensorMap& tm, cudaStream_t s) {
  switch (a.ny) {
    case 8: return col_launch_n<T, 8>(a, tm, s);
    case 16: return col_launch_n<T, 16>(a, tm, s);
    case 32: return col_launch_n<T, 32>(a, tm, s);
    case 64: return col_launch_n<T, 64>(a, tm, s);
    case 128: return col_launch_n<T, 128>(a, tm, s);
    case 256: return col_launch_n<T, 256>(a, tm, s);
    case 512: return col_launch_n<T, 512>(a, tm, s);
    case 1024: return col_launch_n<T, 1024>(a, tm, s);
    case 2048: return col_launch_n<T, 2048>(a, tm, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
int col_tk_t(int nx, int ny) {
  switch (ny) {
    case 8: return col_tk_n<T, 8>(nx);
    case 16: return col_tk_n<T, 16>(nx);
    case 32: return col_tk_n<T, 32>(nx);
    case 64: return col_tk_n<T, 64>(nx);
    case 128: return col_tk_n<T, 128>(nx);
    case 256: return col_tk_n<T, 256>(nx);
    case 512: return col_tk_n<T, 512>(nx);
    case 1024: return col_tk_n<T, 1024>(nx);
    case 2048: return col_tk_n<T, 2048>(nx);
    default: return 0;
  }
}

// FP64 sum reduction (grid-stride, warp shuffles, one atomic per CTA).
// VEC: 16-byte vector loads (x 16-byte aligned, n a multiple of 16 / sizeof(T)).
template <typename T, bool VEC>
__global__ void __launch_bounds__(256) fs_sum_kernel(const T* __restrict__ x, long long n, double* out) {
  double s = 0.0;
  if constexpr (VEC) {
    using V = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
    constexpr int W = 16 / sizeof(T);
    const V* __restrict__ xv = reinterpret_cast<const V*>(x);
    const long long nv = n / W;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nv;
         i += (long long)gridDim.x * blockDim.x) {
      const V v = __ldg(&xv[i]);
      if constexpr (W == 4)
        s += ((double)v.x + (double)v.y) + ((double)v.z + (double)v.w);
      else
        s += (double)v.x + (double)v.y;
    }
  } else {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
      s += (double)x[i];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  __shared__ double ws[8];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
    atomicAdd(out, t);
  }
}

template <typename T>
cudaError_t sum_launch_t(const void* x, long long n, double* out, cudaStream_t s) {
  const long long W = 16 / (long long)sizeof(T);
  const bool vec = ((uintptr_t)x % 16 == 0) && (n % W == 0);
  long long blocks = ((vec ? n / W : n) + 255) / 256;
  if (blocks > 608) blocks = 608;
  if (blocks < 1) blocks = 1;
  if (vec)
    fs_sum_kernel<T, true><<<(unsigned)blocks, 256, 0, s>>>(reinterpret_cast<const T*>(x), n, out);
  else
    fs_sum_kernel<T, false><<<(unsigned)blocks, 256, 0, s>>>(reinterpret_cast<const T*>(x), n, out);
  return cudaGetLastError();
}

}  // namespace fs
