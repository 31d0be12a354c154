// Tensor-core DFT stage for the FP32 column transforms (precisions
// FS_F32_TC_TF32 and FS_F32_TC_BF16X3).  The first Stockham pass of a
// forward line transform (sub-length 1, radix 16) is one real GEMM per
// column tile:
//   [Yr | Yi] (M x 32) = [Xr | Xi] (M x 32) * B (32 x 32),
//   B = [[Wr, Wi], [-Wi, Wr]],  W[r][k] = exp(-2 pi i r k / 16),
// with one GEMM row per (butterfly b, column j): X[b][r] = x[b + (NL/16) r].
// It runs on warp-level tensor-core MMAs (mma.sync) with FP32 accumulation
// and a three-product split so the result keeps close to FP32 accuracy:
//   TF32 x 3:  a = a_hi + a_lo, b = b_hi + b_lo (each TF32), a_hi b_hi + a_hi b_lo + a_lo b_hi
//   BF16 x 3:  the same with BF16 halves.
// The outputs land at the positions the second Stockham pass reads
// (q' = 16 b + k, padded exchange layout), so the transform continues on
// CUDA cores from sub-length 16.
#pragma once

#include <cuda_bf16.h>

#include "fs_fft.cuh"

namespace fs {

enum : int { TC_NONE = 0, TC_TF32 = 1, TC_BF16X3 = 2 };

__device__ __forceinline__ uint32_t f32_to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// Copies the split DFT matrix B into shared memory (all threads of the CTA,
// no barrier inside).  The host stores it in fragment order: for every
// (N tile nn, K tile kk) and lane, the four 32-bit words the lane passes to
// its three MMAs (hi b0, hi b1, lo b0, lo b1; TF32 values, or pairs of BF16
// values packed lower-k first), so one 16-byte load per (nn, kk) feeds them.
__device__ __forceinline__ void tc_load_b(float* bsm, const float* __restrict__ tab) {
  for (int idx = threadIdx.x; idx < 2048; idx += blockDim.x) bsm[idx] = __ldg(&tab[idx]);
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
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
template <int NL, int MODE>
__device__ __forceinline__ void tc_first_pass16(float2* tile, int tk, const float* bsm) {
  constexpr int NB = NL / 16;  // butterflies per column
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ltk = __ffs(tk) - 1;  // tk is a power of two
  const int g = lane >> 2, t4 = lane & 3;
  // The thread's A-fragment columns r (input index of the radix-16 DFT):
  //   TF32 (m16n8k8):  r = t4 + 4 sl;             BF16 (m16n8k16): r = 2 t4 + (sl & 1) + 8 (sl >> 1)
  auto rof = [t4](int sl) { return MODE == TC_TF32 ? t4 + 4 * sl : 2 * t4 + (sl & 1) + 8 * (sl >> 1); };
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
    uint32_t ahi[4][4], alo[4][4];
    if (MODE == TC_TF32) {
      // K tile kk = columns kk*8 + c: kk 0, 1 real parts (r = c, 8 + c), kk 2, 3 imaginary;
      // a0 (g, t4), a1 (g+8, t4), a2 (g, t4+4), a3 (g+8, t4+4)
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int h = e & 1, sl = (e >> 1) + 2 * (kk & 1);
          const float x = (kk < 2) ? xr[tt][h][sl] : xi[tt][h][sl];
          const uint32_t hb = f32_to_tf32(x);
          ahi[kk][e] = hb;
          alo[kk][e] = f32_to_tf32(x - __uint_as_float(hb));
        }
    } else {
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
    }
    // four N tiles of 8 output columns: nn 0, 1 real parts (k in [0, 16)), nn 2, 3 imaginary
#pragma unroll
    for (int nn = 0; nn < 4; ++nn) {
      float d[4] = {0.f, 0.f, 0.f, 0.f};
      const uint4* bq = reinterpret_cast<const uint4*>(bsm);
      if (MODE == TC_TF32) {
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const uint4 bf = bq[(nn * 4 + kk) * 32 + lane];
          mma_tf32(d, alo[kk], bf.x, bf.y);
          mma_tf32(d, ahi[kk], bf.z, bf.w);
          mma_tf32(d, ahi[kk], bf.x, bf.y);
        }
      } else {
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
          const uint4 bf = bq[(nn * 2 + kk) * 32 + lane];
          mma_bf16(d, alo[kk], bf.x, bf.y);
          mma_bf16(d, ahi[kk], bf.z, bf.w);
          mma_bf16(d, ahi[kk], bf.x, bf.y);
        }
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

}  // namespace fs
