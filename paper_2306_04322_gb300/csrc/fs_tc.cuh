// Tensor-core DFT stage for the FP32 column transforms (precisions
// FS_F32_TC_TF32 and FS_F32_TC_BF16X3).  The first Stockham pass of a
// forward line transform (sub-length 1, radix 16) is one real GEMM per
// column tile:
//   [Yr | Yi] (M x 32) = [Xr | Xi] (M x 32) * B (32 x 32),
//   B = [[Wr, Wi], [-Wi, Wr]],  W[r][k] = exp(-2 pi i r k / 16),
// with one GEMM row per (butterfly b, column j): X[b][r] = x[b + (NL/16) r].
// Both run a three-product split, a = a_hi + a_lo, b = b_hi + b_lo:
//   a_hi b_hi + a_hi b_lo + a_lo b_hi, FP32 accumulation.
// The product a_lo b_lo (2^-22 relative for TF32 halves) is dropped and
// a_lo is itself rounded to the half's precision, so the stage keeps about
// 21 significant bits with TF32 halves (FP32 has 24) and about 15 with BF16
// halves; the parity tests state the resulting tolerances.
//   TF32 x 3 (FS_F32_TC_TF32): fifth-generation tensor cores, tcgen05.mma
//     kind::tf32 issued by one thread, M = 128 rows per MMA, N = 32, K = 8,
//     operands in shared memory in the canonical K-major layout (no
//     swizzle), accumulator in tensor memory (TMEM), read back with
//     tcgen05.ld; completion tracked by tcgen05.commit on an mbarrier.
//   BF16 x 3 (FS_F32_TC_BF16X3): the warp-level mma.sync m16n8k16 path.
// The outputs land at the positions the second Stockham pass reads
// (q' = 16 b + k, padded exchange layout), so the transform continues on
// CUDA cores from sub-length 16.
#pragma once

#include <cuda_bf16.h>

#include "fs_fft.cuh"
#include "fs_internal.h"

namespace fs {

enum : int { TC_NONE = 0, TC_TF32 = 1, TC_BF16X3 = 2 };

__device__ __forceinline__ uint32_t f32_to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// Copies the split DFT matrix B (2048 words, layout per precision, see the
// host's tc_table) into shared memory (all threads of the CTA, no barrier
// inside).
__device__ __forceinline__ void tc_load_b(float* bsm, const float* __restrict__ tab) {
  for (int idx = threadIdx.x; idx < 2048; idx += blockDim.x) bsm[idx] = __ldg(&tab[idx]);
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo_k, float hi_k) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo_k, hi_k);  // .x = lower k index
  return *reinterpret_cast<uint32_t*>(&v);
}

// First forward Stockham pass (radix 16) of the NL-point transforms of all
// tk columns of `tile` (natural layout [q][tk], complex float), results
// written to the padded exchange layout q' -> q' + (q' >> 4) of the same
// tile.  Every thread of the CTA calls it; blockDim.x * 16 == NL * tk
// (E = 16 values per thread), so each warp owns two 16-row M tiles.
// mma.sync form of the first radix-16 pass, BF16 x 3 (m16n8k16): every
// thread of the CTA calls it; blockDim.x * 16 == NL * tk (E = 16 values per
// thread), so each warp owns two 16-row M tiles.  Results written to the
// padded exchange layout q' -> q' + (q' >> 4) of the same tile.
template <int NL, int MODE>
__device__ __forceinline__ void tc_first_pass16_mma(float2* tile, int tk, const float* bsm) {
  static_assert(MODE == TC_BF16X3, "the mma.sync stage is the BF16 x 3 one");
  constexpr int NB = NL / 16;  // butterflies per column
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ltk = __ffs(tk) - 1;  // tk is a power of two
  const int g = lane >> 2, t4 = lane & 3;
  // the thread's A-fragment columns r (input index of the radix-16 DFT)
  auto rof = [t4](int sl) { return 2 * t4 + (sl & 1) + 8 * (sl >> 1); };
  float xr[2][2][4], xi[2][2][4];  // [M tile][row g / g + 8][slot]
#pragma unroll
  for (int tt = 0; tt < 2; ++tt) {
    const int mt = warp * 2 + tt;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int row = mt * 16 + g + 8 * h;
      const int b = row >> ltk, j = row & (tk - 1);
#pragma unroll
      for (int sl = 0; sl < 4; ++sl) {
        const float2 x = tile[(b + NB * rof(sl)) * tk + j];
        xr[tt][h][sl] = x.x;
        xi[tt][h][sl] = x.y;
      }
    }
  }
  __syncthreads();  // all inputs read before the outputs overwrite the tile
#pragma unroll
  for (int tt = 0; tt < 2; ++tt) {
    const int row0 = (warp * 2 + tt) * 16 + g;
    uint32_t ahi[2][4], alo[2][4];
    // K tile kk = columns kk*16 + c: kk 0 real, 1 imaginary;
    // reg e: rows g (+8 for odd e), columns 2 t4 (+8 for e >= 2) and the next
#pragma unroll
    for (int kk = 0; kk < 2; ++kk)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int h = e & 1, sl = 2 * (e >> 1);
        const float x0 = kk ? xi[tt][h][sl] : xr[tt][h][sl];
        const float x1 = kk ? xi[tt][h][sl + 1] : xr[tt][h][sl + 1];
        const float h0 = __bfloat162float(__float2bfloat16_rn(x0));
        const float h1 = __bfloat162float(__float2bfloat16_rn(x1));
        ahi[kk][e] = pack_bf16(h0, h1);
        alo[kk][e] = pack_bf16(x0 - h0, x1 - h1);
      }
    // four N tiles of 8 output columns: nn 0, 1 real parts (k in [0, 16)), nn 2, 3 imaginary
#pragma unroll
    for (int nn = 0; nn < 4; ++nn) {
      float d[4] = {0.f, 0.f, 0.f, 0.f};
      const uint4* bq = reinterpret_cast<const uint4*>(bsm);
#pragma unroll
      for (int kk = 0; kk < 2; ++kk) {
        const uint4 bf = bq[(nn * 2 + kk) * 32 + lane];
        mma_bf16(d, alo[kk], bf.x, bf.y);
        mma_bf16(d, ahi[kk], bf.z, bf.w);
        mma_bf16(d, ahi[kk], bf.x, bf.y);
      }
      // D fragment: (g, 2t4), (g, 2t4+1), (g+8, 2t4), (g+8, 2t4+1)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int row = row0 + 8 * (e >> 1);
        const int ncol = nn * 8 + 2 * t4 + (e & 1);
        const int k = ncol & 15;
        const int b = row >> ltk, j = row & (tk - 1);
        const int q = 16 * b + k;
        float* dst = reinterpret_cast<float*>(&tile[(q + (q >> 4)) * tk + j]);
        dst[ncol >> 4] = d[e];
      }
    }
  }
  __syncthreads();
}

// ---- tcgen05 (fifth-generation tensor cores, accumulator in TMEM) --------
template <int NL>
__device__ __forceinline__ void tc5_first_pass16(float2* tile, int tk, const float* bsm, int* flag);

// The stage of precision MODE: TF32 x 3 on tcgen05, BF16 x 3 on mma.sync.
template <int NL, int MODE>
__device__ __forceinline__ void tc_first_pass16(float2* tile, int tk, const float* bsm, int* flag) {
  if constexpr (MODE == TC_TF32) tc5_first_pass16<NL>(tile, tk, bsm, flag);
  else tc_first_pass16_mma<NL, MODE>(tile, tk, bsm);
}

// Shared-memory matrix descriptor of a K-major operand without swizzle:
// 8-row x 16-byte core matrices, `lbo` bytes between core matrices adjacent
// in K, `sbo` bytes between core matrices adjacent in M (N); bits 46-48 hold
// the fixed value 0b001 of the tcgen05 descriptor format.
__device__ __forceinline__ uint64_t umma_desc(const void* p, uint32_t lbo, uint32_t sbo) {
  const uint32_t a = smem_u32(p);
  uint64_t d = (uint64_t)((a & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo & 0x3FFFFu) >> 4) << 16;
  d |= (uint64_t)((sbo & 0x3FFFFu) >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;  // base offset 0, relative leading offset, no swizzle
}
// Instruction descriptor of kind::tf32: D FP32, A and B TF32, both K-major,
// no negation, N >> 3 at bit 17, M >> 4 at bit 24.
constexpr uint32_t umma_idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc5_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc5_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// D (TMEM) = A B (+ D when accumulate), one thread issues
__device__ __forceinline__ void umma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// the mbarrier completes one arrival once every MMA this thread issued is done
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
// 32 consecutive 32-bit TMEM columns of this thread's lane (warp w reads
// lanes 32 (w % 4) .. 32 (w % 4) + 31)
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
      "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared memory the tcgen05 stage needs after the B matrix (bsm, 8 KB):
// an mbarrier, the TMEM address slot, then A_hi and A_lo of `threads` rows
// x 32 TF32 values each in the canonical layout.
__host__ __device__ constexpr size_t tc5_extra_bytes(int threads) { return 128 + (size_t)threads * 32 * 4 * 2; }

// tcgen05 form of the first radix-16 pass (same inputs and output positions
// as tc_first_pass16).  blockDim.x = M rows (a multiple of 128), row =
// threadIdx.x = (b, j).  bsm holds B_hi then B_lo, 32 x 32 TF32 each, in
// the canonical K-major layout (see tc_table on the host); the bytes after
// it (tc5_extra_bytes) are the stage's own.  TMEM (64 columns) is allocated
// and freed inside the call, so no return path of the caller can hold it.
// `flag` receives FS_FLAG_TIMEOUT if the bounded wait for the MMAs gives up.
template <int NL>
__device__ __forceinline__ void tc5_first_pass16(float2* tile, int tk, const float* bsm, int* flag) {
  constexpr int NB = NL / 16;
  constexpr uint32_t kBlock = 128 * 32 * 4;  // bytes of A per 128-row block (16 x 8 core matrices)
  const int warp = threadIdx.x >> 5;
  const int M = blockDim.x;
  unsigned char* ex = reinterpret_cast<unsigned char*>(const_cast<float*>(bsm)) + 8192;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(ex);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(ex + 8);
  unsigned char* Ahi = ex + 128;
  unsigned char* Alo = Ahi + (size_t)M * 128;
  const unsigned char* Bhi = reinterpret_cast<const unsigned char*>(bsm);
  const unsigned char* Blo = Bhi + 4096;
  const int ltk = __ffs(tk) - 1;
  const int row = threadIdx.x;
  const int b = row >> ltk, j = row & (tk - 1);
  {
    // this row of A (Re x then Im x at r = 0..15), split into TF32 halves,
    // stored as the row's 8 16-byte pieces of the canonical layout
    const int mb = row >> 7, mr = row & 127;
    const size_t base = (size_t)mb * kBlock + (size_t)(mr >> 3) * 8 * 128 + (size_t)(mr & 7) * 16;
    float x[32];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const float2 v = tile[(b + NB * r) * tk + j];
      x[r] = v.x;
      x[16 + r] = v.y;
    }
#pragma unroll
    for (int ki = 0; ki < 8; ++ki) {
      uint4 hi, lo;
      uint32_t* h = &hi.x;
      uint32_t* l = &lo.x;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const uint32_t hb = f32_to_tf32(x[4 * ki + e]);
        h[e] = hb;
        l[e] = f32_to_tf32(x[4 * ki + e] - __uint_as_float(hb));
      }
      *reinterpret_cast<uint4*>(Ahi + base + ki * 128) = hi;
      *reinterpret_cast<uint4*>(Alo + base + ki * 128) = lo;
    }
  }
  fence_proxy_async_smem();  // the MMAs read A through the async proxy
  if (threadIdx.x == 0) {
    mbar_init(mbar, 1);
    fence_mbar_init();
  }
  if (warp == 0) tmem_alloc(tslot, 64);
  tc5_fence_before();
  __syncthreads();
  tc5_fence_after();
  const uint32_t tbase = *tslot;
  if (threadIdx.x == 0) {
    constexpr uint32_t idesc = umma_idesc_tf32(128, 32);
    for (int mb = 0; mb < M / 128; ++mb) {
      // products hi x hi, hi x lo, lo x hi; K = 32 in four steps of 8 (two core matrices)
#pragma unroll
      for (int prod = 0; prod < 3; ++prod) {
        const unsigned char* A = (prod == 2 ? Alo : Ahi) + (size_t)mb * kBlock;
        const unsigned char* B = (prod == 1 ? Blo : Bhi);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
          umma_tf32(tbase + 32 * mb, umma_desc(A + kk * 256, 128, 1024), umma_desc(B + kk * 256, 128, 1024), idesc,
                    (prod > 0 || kk > 0) ? 1u : 0u);
      }
    }
    umma_commit(mbar);
  }
  if (!mbar_wait_bounded(mbar, 0, kWaitPolls)) {
    if (threadIdx.x == 0) atomicOr(flag, 2 /* FS_FLAG_TIMEOUT */);
    mbar_wait_bounded(mbar, 0, kWaitPolls);
  }
  tc5_fence_after();
  uint32_t d[32];
  tmem_ld32(tbase + ((uint32_t)(32 * (warp & 3)) << 16) + 32u * (uint32_t)(warp >> 2), d);
  // D row = this thread's (b, j); column nc: Re Y[k] for nc < 16, Im Y[k - 16] above
#pragma unroll
  for (int nc = 0; nc < 32; ++nc) {
    const int k = nc & 15;
    const int q = 16 * b + k;
    float* dst = reinterpret_cast<float*>(&tile[(q + (q >> 4)) * tk + j]);
    dst[nc >> 4] = __uint_as_float(d[nc]);
  }
  tc5_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc5_fence_after();
    tmem_dealloc(tbase, 64);
  }
}

}  // namespace fs
