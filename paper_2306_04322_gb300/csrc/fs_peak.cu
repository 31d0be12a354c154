// Measured FP64 arithmetic rate of the current GPU: the denominator of the
// FP64 step's arithmetic roofline.  A grid of CTAs runs long chains of
// independent DFMA (or DADD) instructions; the rate is thread-instructions
// per second from CUDA events around the launch (best of three after a
// warm-up launch).  Every FP64 add, multiply and fused multiply-add issues
// to the same FP64 pipe, so the DFMA rate bounds the FP64 instruction rate
// of any kernel (the DADD rate is measured beside it to check this).
#include <cuda_runtime.h>

#include "fs.h"

namespace {

constexpr int kChains = 8;    // independent dependency chains per thread
constexpr int kUnroll = 16;   // instructions per chain per loop iteration

template <bool FMA>
__global__ void __launch_bounds__(256) fs_fp64_rate_kernel(double* out, int iters, double b, double c) {
  double a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = 1.0 + 1e-3 * (threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = FMA ? fma(a[k], b, c) : a[k] + c;
    }
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  // never true for the arguments used (every chain stays positive); keeps
  // the chains live.  The index stays inside the 256-entry buffer.
  if (s == -1.0) out[threadIdx.x] = s;
}

template <bool FMA>
cudaError_t rate(cudaStream_t s, double* out, double* per_s) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int blocks = 8 * sms, threads = 256, iters = 256;
  cudaEvent_t e0, e1;
  e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) return e;
  float best = 1e30f;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
    e = cudaEventRecord(e0, s);
    fs_fp64_rate_kernel<FMA><<<blocks, threads, 0, s>>>(out, iters, 1.0000000001, 1e-12);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;  // the first launch warms up
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return e;
  const double inst = (double)blocks * threads * iters * kUnroll * kChains;
  *per_s = inst / (best * 1e-3);
  return cudaSuccess;
}

}  // namespace

extern "C" fs_status fs_measure_fp64_rate(void* stream, double* dfma_per_s, double* dadd_per_s) {
  if (!dfma_per_s) return FS_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  double* out = nullptr;  // never written (see the kernel); a valid pointer all the same
  if (cudaMalloc(&out, sizeof(double) * 256) != cudaSuccess) return FS_ERR_OOM;
  cudaError_t e = rate<true>(s, out, dfma_per_s);
  if (e == cudaSuccess && dadd_per_s) e = rate<false>(s, out, dadd_per_s);
  cudaFree(out);
  return e == cudaSuccess ? FS_OK : FS_ERR_CUDA;
}
