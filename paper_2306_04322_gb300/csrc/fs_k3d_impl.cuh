// 3D passes of the semi-implicit Fourier-spectral step (Eq. Gamma_fft_3d,
// Algorithm 1 for 3D domains).  A step is four passes over the packed
// x-spectra [slot][z][y][kx] (kx < nx/2, bin 0 = DC + i Nyquist):
//   x pass     the 2D row kernel with ny * nz rows;
//   y forward  fs_ypass_kernel<DIR = -1> on the slots g_i, df/dc (and c in
//              the first step after the fields are set);
//   z step     fs_zstep_kernel: forward z transform, k-space update with
//              K2 = |xi_x|^2 + |xi_y|^2 + |xi_z|^2, inverse z transform;
//   y inverse  fs_ypass_kernel<DIR = +1> on slots c, g_i.
// c is carried between steps as Algorithm 1 carries c^: the z step leaves
// c's (kx, ky, z) spectrum in slot 0 and the y inverse writes c's x spectrum
// to slot nf (df/dc is consumed by then) instead of over it, so the next
// step's x pass reads c from slot nf, its y forward skips slot 0, and its
// z step finds c's (kx, ky, z) spectrum in slot 0 (a factor ny smaller than
// the y forward would give: folded into the update).
// The packed kx = 0 / Nyquist column of every z plane is split in the
// y passes into the y-spectra A (x-DC) and B (x-Nyquist), each Hermitian in
// ky, and stored as
//   col[0] = A(0) + i A(ny/2),  col[ny/2] = B(0) + i B(ny/2)   (all real)
//   col[ky] = A(ky), col[ny - ky] = B(ky)                      (0 < ky < ny/2)
// so that every z line holds the z-dependence of one well-defined (kx, ky)
// mode (or of two real-to-complex packed ones for ky = 0 and ny/2), and the z
// pass never needs another CTA's column.
#pragma once

#include "fs_kernels.cuh"

namespace fs {

template <typename T, int NL>
struct LineCfg {
  static constexpr bool F64 = sizeof(T) == 8;
  static constexpr int E = col_E(NL, F64);
  static constexpr int TPL = NL / E;
  static constexpr int TK = col_tk(NL, F64, 128);  // 3D line passes: about 128 threads per CTA
  static constexpr int THREADS = TPL * TK;
  static constexpr int BH = NL < 256 ? NL : 256;  // TMA box extent along the line
  static constexpr int BAR_BYTES = 128;
  static constexpr int TWS = pass_table_size(NL, E);
  static constexpr int TW_BYTES = ((TWS * (int)sizeof(cplx<T>)) + 127) & ~127;
  static constexpr int K2_BYTES = ((NL * (int)sizeof(T)) + 127) & ~127;
  static constexpr int LOGE = ilog2(E);
  static constexpr int TROWS = (NL + NL / E + 1 + 15) & ~15;
  static constexpr int HEAD = BAR_BYTES + TW_BYTES + K2_BYTES;
};

// ---------------------------------------------------------------------------
// y pass: one CTA per (kx tile, z, slot); DIR = -1 forward (slots 0..nf),
// DIR = +1 inverse (slots 0..nf-1).  Tensor map: [slot * nz + z][y][kx].
// ---------------------------------------------------------------------------
template <typename T, int NY, int DIR, int TCM = TC_NONE>
__global__ void __launch_bounds__(LineCfg<T, NY>::THREADS, 4)
    fs_ypass_kernel(KArgs a, const __grid_constant__ CUtensorMap tmap) {
  using C = cplx<T>;
  using Cfg = LineCfg<T, NY>;
  constexpr int E = Cfg::E, TPL = Cfg::TPL, BH = Cfg::BH, LOGE = Cfg::LOGE;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  C* tw = reinterpret_cast<C*>(smem_raw + Cfg::BAR_BYTES);
  C* tile = reinterpret_cast<C*>(smem_raw + Cfg::HEAD);
  const int tk = blockDim.x / TPL;
  const int j = threadIdx.x % tk, t = threadIdx.x / tk;
  const int Lh = a.nx / 2;
  const int kx0 = blockIdx.x * tk;
  const int plane = blockIdx.y + a.plane0;  // slot * nz + z
  // y inverse of c with the 3D carry: c's x spectrum goes to slot nf
  const int oplane = (DIR > 0 && a.carry3 && plane < a.nz) ? plane + a.nf * a.nz : plane;
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_arrive_expect_tx(bar, (uint32_t)(NY * tk * sizeof(C)));
    const int cx = kx0 * (int)(sizeof(C) / 8);
    for (int y0 = 0; y0 < NY; y0 += BH) tma_load_3d(tile + y0 * tk, &tmap, cx, y0, plane, bar);
  }
  copy_to_smem(tw, reinterpret_cast<const C*>(a.tw_col), Cfg::TWS);
  __syncthreads();
  if (!mbar_wait_bounded(bar, 0, first_wait_polls(a))) {
    if (threadIdx.x == 0) atomicOr(a.flag, FS_FLAG_TIMEOUT);
    mbar_wait_bounded(bar, 0, kWaitPolls);
    return;
  }
  const bool special = (kx0 == 0);
  C v[E];
  if (DIR > 0 && special) {
    // unpack the kx = 0 / Nyquist column: Z(ky) = A(ky) + i B(ky)
    if (j == 0) {
#pragma unroll
      for (int m = 0; m < E; ++m) {
        const int ky = t + TPL * m;
        const C s0 = tile[0], sh = tile[(NY / 2) * tk];
        C A, B;
        if (ky == 0) {
          A = mk<C>(s0.x, T(0));
          B = mk<C>(sh.x, T(0));
        } else if (ky == NY / 2) {
          A = mk<C>(s0.y, T(0));
          B = mk<C>(sh.y, T(0));
        } else if (ky < NY / 2) {
          A = tile[ky * tk];
          B = tile[(NY - ky) * tk];
        } else {
          A = cconj(tile[(NY - ky) * tk]);
          B = cconj(tile[ky * tk]);
        }
        v[m] = cadd(A, mul_i<1>(B));
      }
    }
    __syncthreads();
    if (j != 0) {
#pragma unroll
      for (int m = 0; m < E; ++m) v[m] = tile[(t + TPL * m) * tk + j];
    }
  } else {
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = tile[(t + TPL * m) * tk + j];
  }
  {
    C* tl = tile + j;
    auto st = [tl, tk](int q, C x) { tl[(q + (q >> LOGE)) * tk] = x; };
    auto ld = [tl, tk](int q) { return tl[(q + (q >> LOGE)) * tk]; };
    auto sync = []() { __syncthreads(); };
    if constexpr (TCM != TC_NONE && DIR < 0) {
      // first radix-16 pass on tensor cores (input still in the tile), rest on CUDA cores
      static_assert(sizeof(T) == 4 && E == 16, "tensor-core stage: FP32, radix 16");
      float* bsm = reinterpret_cast<float*>(tile + Cfg::TROWS * tk);
      tc_load_b(bsm, reinterpret_cast<const float*>(a.tc_b));
      __syncthreads();
      tc_first_pass16<NY, TCM>(reinterpret_cast<float2*>(tile), tk, bsm, a.flag);
#pragma unroll
      for (int m = 0; m < E; ++m) v[m] = ld(t + TPL * m);
      stockham<NY, E, 16, DIR>(v, t, tw, st, ld, sync);
    } else {
      line_fft<NY, E, DIR>(v, t, tw, st, ld, sync);
    }
  }
  if (DIR < 0 && special) {
    // pack: A = (Z(ky) + conj Z(-ky)) / 2, B = (Z(ky) - conj Z(-ky)) / (2i)
    __syncthreads();
    if (j == 0) {
#pragma unroll
      for (int m = 0; m < E; ++m) tile[(t + TPL * m) * tk] = v[m];
    }
    __syncthreads();
    if (j == 0) {
#pragma unroll
      for (int m = 0; m < E; ++m) {
        const int ky = t + TPL * m;
        const C z = v[m], zq = cconj(tile[((NY - ky) & (NY - 1)) * tk]);
        const C A = cscale(cadd(z, zq), T(0.5)), B = cscale(mul_i<-1>(csub(z, zq)), T(0.5));
        if (ky == 0) {
          // col[0] = A(0) + i A(ny/2) = Re Z(0) + i Re Z(ny/2)
          v[m] = mk<C>(tile[0].x, tile[(NY / 2) * tk].x);
        } else if (ky == NY / 2) {
          // col[ny/2] = B(0) + i B(ny/2) = Im Z(0) + i Im Z(ny/2)
          v[m] = mk<C>(tile[0].y, tile[(NY / 2) * tk].y);
        } else if (ky < NY / 2) {
          v[m] = A;
        } else {
          v[m] = cconj(B);  // col[ky] = B(ny - ky) = conj B(ky)
        }
      }
    }
  }
  C* S = reinterpret_cast<C*>(a.spec) + (long long)oplane * NY * Lh + kx0 + j;
#pragma unroll
  for (int m = 0; m < E; ++m)
    if (spec_ok(a, &S[(long long)(t + TPL * m) * Lh], sizeof(C))) S[(long long)(t + TPL * m) * Lh] = v[m];
}

// ---------------------------------------------------------------------------
// z step: one CTA per (kx tile, ky storage row, field group).  Tensor map:
// [slot][z][y][kx] with a box of one y row and up to 256 z planes.
// ---------------------------------------------------------------------------
template <typename T, int NZ, int TCM = TC_NONE>
__global__ void __launch_bounds__(LineCfg<T, NZ>::THREADS, 4)
    fs_zstep_kernel(KArgs a, const __grid_constant__ CUtensorMap tmap) {
  using C = cplx<T>;
  using Cfg = LineCfg<T, NZ>;
  constexpr int E = Cfg::E, TPL = Cfg::TPL, BH = Cfg::BH, LOGE = Cfg::LOGE, TROWS = Cfg::TROWS;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  C* tw = reinterpret_cast<C*>(smem_raw + Cfg::BAR_BYTES);
  T* k2zt = reinterpret_cast<T*>(smem_raw + Cfg::BAR_BYTES + Cfg::TW_BYTES);
  C* tiles = reinterpret_cast<C*>(smem_raw + Cfg::HEAD);
  const int tk = blockDim.x / TPL;
  const int j = threadIdx.x % tk, t = threadIdx.x / tk;
  const int Lh = a.nx / 2, NY = a.ny;
  const int kx0 = blockIdx.x * tk, kx = kx0 + j;
  const int ky = blockIdx.y;  // storage row
  const int g = blockIdx.z;   // field group
  const int nf = a.nf;
  const int nin = (g == 0) ? 2 : 1;
  const long long zstride = (long long)NY * Lh;
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_arrive_expect_tx(bar, (uint32_t)(nin * NZ * tk * sizeof(C)));
    const int cx = kx0 * (int)(sizeof(C) / 8);
    for (int i = 0; i < nin; ++i) {
      const int slot = (g == 0) ? (i == 0 ? nf : 0) : g;
      for (int z0 = 0; z0 < NZ; z0 += BH)
        tma_load_4d(tiles + (i * TROWS + z0) * tk, &tmap, cx, ky, z0, slot, bar);
    }
  }
  copy_to_smem(tw, reinterpret_cast<const C*>(a.tw_z), Cfg::TWS);
  for (int i = threadIdx.x; i < NZ; i += blockDim.x) k2zt[i] = reinterpret_cast<const T*>(a.k2z)[i];
  __syncthreads();
  if (!mbar_wait_bounded(bar, 0, first_wait_polls(a))) {
    if (threadIdx.x == 0) atomicOr(a.flag, FS_FLAG_TIMEOUT);
    mbar_wait_bounded(bar, 0, kWaitPolls);
    return;
  }
  const KUpdate<T> up(a);
  const T* __restrict__ k2xt = reinterpret_cast<const T*>(a.k2x);
  const T* __restrict__ k2yt = reinterpret_cast<const T*>(a.k2y);
  // K2 of this line without the z part.  In the packed column (kx = 0 tile,
  // j = 0) rows below ny/2 are x-DC modes, rows above are x-Nyquist modes;
  // rows 0 and ny/2 hold two modes (handled in `pair` below).
  const bool col0 = (kx0 == 0 && j == 0);
  const T kx2 = k2xt[kx], kxn2 = k2xt[Lh];
  const T kxy2 = (col0 ? (ky <= NY / 2 ? k2xt[0] : kxn2) : kx2) + k2yt[ky];
  const bool pairCTA = (kx0 == 0) && (ky == 0 || ky == NY / 2);  // CTA-uniform
  const bool pair = pairCTA && j == 0;
  const T kxa = (ky == 0) ? k2xt[0] : kxn2;  // pair rows: x part of both modes
  const T kya = k2yt[0], kyb = k2yt[NY / 2];

  C* stash = tiles;
  C* xt = tiles + (nin - 1) * TROWS * tk;
  auto sync = []() { __syncthreads(); };
  float* bsm = reinterpret_cast<float*>(tiles + 2 * TROWS * tk);
  if constexpr (TCM != TC_NONE) {
    static_assert(sizeof(T) == 4 && E == 16, "tensor-core stage: FP32, radix 16");
    tc_load_b(bsm, reinterpret_cast<const float*>(a.tc_b));
    __syncthreads();
  }
  C v[E];
  for (int i = 0; i < nin; ++i) {
    C* tl = tiles + i * TROWS * tk + j;
    auto st = [tl, tk](int q, C x) { tl[(q + (q >> LOGE)) * tk] = x; };
    auto ld = [tl, tk](int q) { return tl[(q + (q >> LOGE)) * tk]; };
    if constexpr (TCM != TC_NONE) {
      tc_first_pass16<NZ, TCM>(reinterpret_cast<float2*>(tiles + i * TROWS * tk), tk, bsm, a.flag);
#pragma unroll
      for (int m = 0; m < E; ++m) v[m] = ld(t + TPL * m);
      stockham<NZ, E, 16, -1>(v, t, tw, st, ld, sync);
    } else {
#pragma unroll
      for (int m = 0; m < E; ++m) v[m] = tl[(t + TPL * m) * tk];
      line_fft<NZ, E, -1>(v, t, tw, st, ld, sync);
    }
    if (i == 0 && nin == 2) {
      sync();
#pragma unroll
      for (int m = 0; m < E; ++m) tl[(t + TPL * m) * tk] = v[m];
    }
  }
  if (pairCTA) {
    sync();
    if (j == 0) {
#pragma unroll
      for (int m = 0; m < E; ++m) xt[(t + TPL * m) * tk] = v[m];
    }
    sync();
  }
  if (pair) {
    // two real z-sequences packed as P = U + i V; U, V Hermitian in kz
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const int kz = t + TPL * m, kq = (NZ - kz) & (NZ - 1);
      const T kz2 = k2zt[kz];
      const C pz = cconj(xt[kq * tk]);
      const C U = cscale(cadd(v[m], pz), T(0.5)), V = cscale(mul_i<-1>(csub(v[m], pz)), T(0.5));
      C Un, Vn;
      if (g == 0) {
        const C zf = stash[kz * tk], pf = cconj(stash[kq * tk]);
        const C Uf = cscale(cadd(zf, pf), T(0.5)), Vf = cscale(mul_i<-1>(csub(zf, pf)), T(0.5));
        Un = up.c(U, Uf, kxa + kya + kz2);
        Vn = up.c(V, Vf, kxa + kyb + kz2);
        if (ky == 0 && kz == 0 && a.csum) Un = mk<C>((T)(*a.csum * a.inv_npts), T(0));
      } else {
        Un = up.eta(U, kxa + kya + kz2);
        Vn = up.eta(V, kxa + kyb + kz2);
      }
      v[m] = cadd(Un, mul_i<1>(Vn));
    }
  } else if (g == 0) {
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const int kz = t + TPL * m;
      v[m] = up.c(v[m], stash[kz * tk + j], kxy2 + k2zt[kz]);
    }
  } else {
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = up.eta(v[m], kxy2 + k2zt[t + TPL * m]);
  }
  {
    C* tl = xt + j;
    auto st = [tl, tk](int q, C x) { tl[(q + (q >> LOGE)) * tk] = x; };
    auto ld = [tl, tk](int q) { return tl[(q + (q >> LOGE)) * tk]; };
    line_fft<NZ, E, 1>(v, t, tw, st, ld, sync);
  }
  C* S = reinterpret_cast<C*>(a.spec) + (long long)(g == 0 ? 0 : g) * a.slot_stride + (long long)ky * Lh + kx;
#pragma unroll
  for (int m = 0; m < E; ++m)
    if (spec_ok(a, &S[(long long)(t + TPL * m) * zstride], sizeof(C))) S[(long long)(t + TPL * m) * zstride] = v[m];
}

// ---- launchers ---------------------------------------------------------------
template <typename T, int NL>
int line_tk(int nx) {
  int Lh = nx / 2;
  return LineCfg<T, NL>::TK < Lh ? LineCfg<T, NL>::TK : Lh;
}

// ---------------------------------------------------------------------------
// Free-energy diagnostic, 3D gradient terms (Eq. fe through Parseval with the
// scheme's |xi|^2 of Eq. Gamma_fft_3d, K2 = kx^2 + ky^2 + kz^2).  Input: the
// x pass in mode 3 (2 x^(phi) of every field in slots 0..nf-1) and the
// forward y pass over those slots (the kx = 0 / Nyquist column packed as
// described at the top of this file).  One CTA per (kx tile, ky storage row,
// field g): forward z transform of the z lines, then the sum of w K2 |.|^2
// over the line, each stored mode weighted by the modes of the full spectrum
// it stands for:
//   kx >= 1: weight 2 (the conjugate mode at -k is not stored);
//   packed column, rows 0 < ky < ny/2: x-DC modes (0, ky, kz), weight 2;
//   rows ky > ny/2: x-Nyquist modes (nx/2, ny - ky, kz), weight 2;
//   rows 0 and ny/2: P + i Q of two real z sequences (y-DC and y-Nyquist of
//   the x-DC resp. x-Nyquist column), separated through Z(kz) and
//   conj Z(-kz), each mode once (weight 1).
// FP64 atomics into acc[1 + g].
// ---------------------------------------------------------------------------
template <typename T, int NZ>
__global__ void __launch_bounds__(LineCfg<T, NZ>::THREADS, 4)
    fs_energy_z_kernel(KArgs a, const __grid_constant__ CUtensorMap tmap) {
  using C = cplx<T>;
  using Cfg = LineCfg<T, NZ>;
  constexpr int E = Cfg::E, TPL = Cfg::TPL, BH = Cfg::BH, LOGE = Cfg::LOGE;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  C* tw = reinterpret_cast<C*>(smem_raw + Cfg::BAR_BYTES);
  T* k2zt = reinterpret_cast<T*>(smem_raw + Cfg::BAR_BYTES + Cfg::TW_BYTES);
  C* tile = reinterpret_cast<C*>(smem_raw + Cfg::HEAD);
  const int tk = blockDim.x / TPL;
  const int j = threadIdx.x % tk, t = threadIdx.x / tk;
  const int Lh = a.nx / 2, NY = a.ny;
  const int kx0 = blockIdx.x * tk, kx = kx0 + j;
  const int ky = blockIdx.y;  // storage row
  const int g = blockIdx.z;   // field
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_arrive_expect_tx(bar, (uint32_t)(NZ * tk * sizeof(C)));
    const int cx = kx0 * (int)(sizeof(C) / 8);
    for (int z0 = 0; z0 < NZ; z0 += BH) tma_load_4d(tile + z0 * tk, &tmap, cx, ky, z0, g, bar);
  }
  copy_to_smem(tw, reinterpret_cast<const C*>(a.tw_z), Cfg::TWS);
  for (int i = threadIdx.x; i < NZ; i += blockDim.x) k2zt[i] = reinterpret_cast<const T*>(a.k2z)[i];
  __syncthreads();
  if (!mbar_wait_bounded(bar, 0, first_wait_polls(a))) {
    if (threadIdx.x == 0) atomicOr(a.flag, FS_FLAG_TIMEOUT);
    mbar_wait_bounded(bar, 0, kWaitPolls);
    return;
  }
  C v[E];
#pragma unroll
  for (int m = 0; m < E; ++m) v[m] = tile[(t + TPL * m) * tk + j];
  {
    C* tl = tile + j;
    auto st = [tl, tk](int q, C x) { tl[(q + (q >> LOGE)) * tk] = x; };
    auto ld = [tl, tk](int q) { return tl[(q + (q >> LOGE)) * tk]; };
    line_fft<NZ, E, -1>(v, t, tw, st, ld, []() { __syncthreads(); });
  }
  const T* __restrict__ k2xt = reinterpret_cast<const T*>(a.k2x);
  const T* __restrict__ k2yt = reinterpret_cast<const T*>(a.k2y);
  const bool col0 = (kx0 == 0 && j == 0);
  const bool pairCTA = (kx0 == 0) && (ky == 0 || ky == NY / 2);  // CTA-uniform
  const bool pair = pairCTA && j == 0;
  if (pairCTA) {
    // the pair rows need Z(-kz): the transformed line in natural order
    __syncthreads();
    if (j == 0) {
#pragma unroll
      for (int m = 0; m < E; ++m) tile[(t + TPL * m) * tk] = v[m];
    }
    __syncthreads();
  }
  // K2 without the z part, and the weight, of a line that holds one mode set
  const double kxy = (double)(col0 ? (ky <= NY / 2 ? k2xt[0] : k2xt[Lh]) : k2xt[kx]) + (double)k2yt[ky];
  const double kxa = (double)((ky == 0) ? k2xt[0] : k2xt[Lh]);  // pair rows: x part of both modes
  const double kya = (double)k2yt[0], kyb = (double)k2yt[NY / 2];
  double sum = 0.0;
#pragma unroll
  for (int m = 0; m < E; ++m) {
    const int kz = t + TPL * m;
    const double kz2 = (double)k2zt[kz];
    if (pair) {
      const C pz = cconj(tile[((NZ - kz) & (NZ - 1)) * tk]);
      const C P = cscale(cadd(v[m], pz), T(0.5)), Q = cscale(mul_i<-1>(csub(v[m], pz)), T(0.5));
      sum += (kxa + kya + kz2) * ((double)P.x * P.x + (double)P.y * P.y);
      sum += (kxa + kyb + kz2) * ((double)Q.x * Q.x + (double)Q.y * Q.y);
    } else {
      sum += 2.0 * (kxy + kz2) * ((double)v[m].x * v[m].x + (double)v[m].y * v[m].y);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(&a.acc[1 + g], sum);
}

template <typename T, int NZ>
cudaError_t energy_z_launch_n(const KArgs& a, const CUtensorMap& tm, cudaStream_t s) {
  using Cfg = LineCfg<T, NZ>;
  const int tk = line_tk<T, NZ>(a.nx);
  const size_t smem = Cfg::HEAD + (size_t)Cfg::TROWS * tk * sizeof(cplx<T>);
  static unsigned done = 0;
  cudaError_t e = allow_big_smem(fs_energy_z_kernel<T, NZ>, &done);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)(a.nx / 2 / tk), (unsigned)a.ny, (unsigned)a.nf);
  fs_energy_z_kernel<T, NZ><<<grid, (unsigned)(tk * Cfg::TPL), smem, s>>>(a, tm);
  return cudaGetLastError();
}

template <typename T, int NY, int DIR, int TCM>
cudaError_t ypass_launch_tc(const KArgs& a, const CUtensorMap& tm, int nslots, cudaStream_t s) {
  using Cfg = LineCfg<T, NY>;
  const int tk = line_tk<T, NY>(a.nx);
  size_t smem = Cfg::HEAD + (size_t)Cfg::TROWS * tk * sizeof(cplx<T>) + (TCM ? 8192 : 0) +
                (TCM == TC_TF32 ? tc5_extra_bytes(tk * Cfg::TPL) : 0);
  // the tcgen05 stage runs 128-row MMAs over the CTA's (butterfly, column) rows
  if (TCM == TC_TF32 && (tk * Cfg::TPL) % 128 != 0) return cudaErrorNotSupported;
  static unsigned done = 0;
  cudaError_t e = allow_big_smem(fs_ypass_kernel<T, NY, DIR, TCM>, &done);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)(a.nx / 2 / tk), (unsigned)(a.nz * nslots));
  fs_ypass_kernel<T, NY, DIR, TCM><<<grid, (unsigned)(tk * Cfg::TPL), smem, s>>>(a, tm);
  return cudaGetLastError();
}

template <typename T, int NY, int DIR>
cudaError_t ypass_launch_n(const KArgs& a, const CUtensorMap& tm, int nslots, cudaStream_t s) {
  if constexpr (sizeof(T) == 4 && NY >= 64 && DIR < 0) {
    if (a.tc == TC_TF32) return ypass_launch_tc<T, NY, DIR, TC_TF32>(a, tm, nslots, s);
    if (a.tc == TC_BF16X3) return ypass_launch_tc<T, NY, DIR, TC_BF16X3>(a, tm, nslots, s);
  }
  if (a.tc != TC_NONE && DIR < 0) return cudaErrorInvalidValue;
  return ypass_launch_tc<T, NY, DIR, TC_NONE>(a, tm, nslots, s);
}

template <typename T, int NZ, int TCM>
cudaError_t zstep_launch_tc(const KArgs& a, const CUtensorMap& tm, cudaStream_t s) {
  using Cfg = LineCfg<T, NZ>;
  const int tk = line_tk<T, NZ>(a.nx);
  size_t smem = Cfg::HEAD + 2 * (size_t)Cfg::TROWS * tk * sizeof(cplx<T>) + (TCM ? 8192 : 0) +
                (TCM == TC_TF32 ? tc5_extra_bytes(tk * Cfg::TPL) : 0);
  if (TCM == TC_TF32 && (tk * Cfg::TPL) % 128 != 0) return cudaErrorNotSupported;
  static unsigned done = 0;
  cudaError_t e = allow_big_smem(fs_zstep_kernel<T, NZ, TCM>, &done);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)(a.nx / 2 / tk), (unsigned)a.ny, (unsigned)a.nf);
  fs_zstep_kernel<T, NZ, TCM><<<grid, (unsigned)(tk * Cfg::TPL), smem, s>>>(a, tm);
  return cudaGetLastError();
}

template <typename T, int NZ>
cudaError_t zstep_launch_n(const KArgs& a, const CUtensorMap& tm, cudaStream_t s) {
  if constexpr (sizeof(T) == 4 && NZ >= 64) {
    if (a.tc == TC_TF32) return zstep_launch_tc<T, NZ, TC_TF32>(a, tm, s);
    if (a.tc == TC_BF16X3) return zstep_launch_tc<T, NZ, TC_BF16X3>(a, tm, s);
  }
  if (a.tc != TC_NONE) return cudaErrorInvalidValue;
  return zstep_launch_tc<T, NZ, TC_NONE>(a, tm, s);
}

#define FS_LINE_SIZES(X) X(8) X(16) X(32) X(64) X(128) X(256) X(512)

template <typename T>
cudaError_t ypass_launch_t(const KArgs& a, const CUtensorMap& tm, int dir, int nslots, cudaStream_t s) {
  switch (a.ny) {
#define FS_CASE(n)                                                            \
  case n:                                                                     \
    return dir < 0 ? ypass_launch_n<T, n, -1>(a, tm, nslots, s)               \
                   : ypass_launch_n<T, n, 1>(a, tm, nslots, s);
    FS_LINE_SIZES(FS_CASE)
#undef FS_CASE
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t zstep_launch_t(const KArgs& a, const CUtensorMap& tm, cudaStream_t s) {
  switch (a.nz) {
#define FS_CASE(n) \
  case n: return zstep_launch_n<T, n>(a, tm, s);
    FS_LINE_SIZES(FS_CASE)
#undef FS_CASE
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t energy_z_launch_t(const KArgs& a, const CUtensorMap& tm, cudaStream_t s) {
  switch (a.nz) {
#define FS_CASE(n) \
  case n: return energy_z_launch_n<T, n>(a, tm, s);
    FS_LINE_SIZES(FS_CASE)
#undef FS_CASE
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
int line_tk_t(int nx, int nl) {
  switch (nl) {
#define FS_CASE(n) \
  case n: return line_tk<T, n>(nx);
    FS_LINE_SIZES(FS_CASE)
#undef FS_CASE
    default: return 0;
  }
}

}  // namespace fs
