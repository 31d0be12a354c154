// Fused step (pass form 4, FP32, 2D): one cooperative launch runs several
// whole steps of Algorithm 1 -- every row pair of the pair-form row pass,
// a grid-wide barrier, every (column pair, field group) item of the
// warp-per-column pass, a grid-wide barrier, and again -- with the same
// bodies as the separate passes (fs_k2d_v2.cuh).  It removes the launch,
// ramp-up and drain between the passes and between steps.  Square grids of
// 256, 512 and 1024 points per axis, p <= 3 (four warps per CTA).
//
// Memory ordering across the barrier: every thread fences its generic
// global stores against the async proxy (the column pass reads by TMA what
// the row pass stored), thread 0 makes the CTA's writes visible at GPU scope
// before it arrives, and after the barrier the copy-issuing threads fence
// again before their bulk / TMA loads.  The column pass's TMA stores have
// completed (cp.async.bulk.wait_group 0) before its CTA arrives.
#include "fs_k2d_v2.cuh"

namespace fs {

namespace {

constexpr uint32_t kGridWaitPolls = 1u << 25;  // with a 32 ns back-off: about a second

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Grid-wide barrier of a cooperative launch (all CTAs resident), two
// levels so that no counter sees more than a few dozen atomics: CTA b
// arrives at group counter b % kGroups; the last arrival of a group arrives
// at the top counter; the last arrival there advances the generation the
// waiters watch.  Counters sit on their own 128-byte lines of `sync` (word
// 32 g for group g, 32 kGroups for the top, 32 (kGroups + 1) for the
// generation).  Returns false in every thread of the CTA if the wait gave up
// after `limit` polls (FS_FLAG_TIMEOUT is set); the host then zeroes the
// counters.
constexpr int kGroups = 16;
constexpr int kSyncWords = 32 * (kGroups + 2);

__device__ __forceinline__ bool grid_barrier(unsigned* sync, unsigned nblocks, uint32_t limit, int* flag) {
  fence_proxy_async_global();
  __syncthreads();
  bool ok = true;
  if (threadIdx.x == 0) {
    unsigned* gen_p = sync + 32 * (kGroups + 1);
    const unsigned gen = ld_acquire_gpu(gen_p);  // cannot advance before this CTA arrives
    const unsigned groups = nblocks < (unsigned)kGroups ? nblocks : (unsigned)kGroups;
    const unsigned g = blockIdx.x % groups;
    const unsigned in_group = nblocks / groups + (g < nblocks % groups ? 1u : 0u);
    __threadfence();
    bool last = false;
    if (atomicAdd(&sync[32 * g], 1u) == in_group - 1) {
      atomicExch(&sync[32 * g], 0u);
      __threadfence();
      if (atomicAdd(&sync[32 * kGroups], 1u) == groups - 1) {
        atomicExch(&sync[32 * kGroups], 0u);
        __threadfence();
        atomicAdd(gen_p, 1u);
        last = true;
      }
    }
    if (!last) {
      uint32_t i = 0;
      while (ld_acquire_gpu(gen_p) == gen) {
        if (i++ >= limit) {
          ok = false;
          atomicOr(flag, FS_FLAG_TIMEOUT);
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
    fence_proxy_async_global();
  }
  return __syncthreads_and(ok) != 0;
}

template <int N>
__global__ void __launch_bounds__(128, 4)
    fs_step2_kernel(KArgs a, const __grid_constant__ CUtensorMap tmap, unsigned* gsync, int nsteps) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t parity = 0;
  const long long row_items = a.lines / 2;
  const int pairs = N / 2 / Col2Cfg<N>::TK;
  const long long col_items = (long long)pairs * (1 + a.nf / 2);
  const uint32_t limit = (a.short_wait & 2) ? 0u : kGridWaitPolls;
  for (int step = 0; step < nsteps; ++step) {
    for (long long item = blockIdx.x; item < row_items; item += gridDim.x) {
      const bool ok = row2_body<N, 1>(a, item, smem_raw, bar, parity);
      if (__syncthreads_or(!ok)) return;
      parity ^= 1u;
    }
    if (!grid_barrier(gsync, gridDim.x, limit, a.flag)) return;
    for (long long item = blockIdx.x; item < col_items; item += gridDim.x) {
      const bool ok = col2_body<N, 1>(a, &tmap, (int)(item % pairs), (int)(item / pairs), smem_raw, bar, parity);
      if (__syncthreads_or(!ok)) return;
      parity ^= 1u;
    }
    if (step + 1 < nsteps && !grid_barrier(gsync, gridDim.x, limit, a.flag)) return;
  }
}

template <int N>
cudaError_t step2_launch_n(const KArgs& a, const CUtensorMap& tm, unsigned* gsync, int nsteps, cudaStream_t s) {
  static unsigned done = 0;
  cudaError_t e = allow_big_smem(fs_step2_kernel<N>, &done);
  if (e != cudaSuccess) return e;
  const size_t r = row2_smem_bytes<N, 1>(a.nf), c = col2_smem_bytes<N, 1>();
  const size_t smem = r > c ? r : c;
  int dev = 0, sms = 0, per_sm = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fs_step2_kernel<N>, 128, smem);
  if (e != cudaSuccess) return e;
  const long long items = a.lines / 2 > (long long)(N / 4) * (1 + a.nf / 2) ? a.lines / 2
                                                                              : (long long)(N / 4) * (1 + a.nf / 2);
  const long long resident = (long long)per_sm * sms;
  const unsigned grid = (unsigned)(items < resident ? items : resident);
  if (grid == 0) return cudaErrorNotSupported;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(128);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;  // every CTA resident: the grid barrier cannot wait forever
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, fs_step2_kernel<N>, a, tm, gsync, nsteps);
}

}  // namespace

bool step2_supported(int nx, int ny, int nf) { return nx == ny && (nx == 256 || nx == 512 || nx == 1024) && nf <= 4; }

cudaError_t step2_launch_f32(const KArgs& a, const CUtensorMap& tm, unsigned* gsync, int nsteps, cudaStream_t s) {
  if (a.mode != 0 || a.tc != 0 || a.nz != 1 || !step2_supported(a.nx, a.ny, a.nf) || !a.tw_row2 || !a.tw_col2 ||
      nsteps < 1)
    return cudaErrorNotSupported;
  switch (a.nx) {
    case 256: return step2_launch_n<256>(a, tm, gsync, nsteps, s);
    case 512: return step2_launch_n<512>(a, tm, gsync, nsteps, s);
    case 1024: return step2_launch_n<1024>(a, tm, gsync, nsteps, s);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace fs
