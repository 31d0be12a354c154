// Adjoint of one 3D semi-implicit Fourier-spectral step: the z part.
//
// The 3D step has the same form as the 2D one (fs_adjoint.cuh), with
// K2 = |xi_x|^2 + |xi_y|^2 + |xi_z|^2 (Eq. Gamma_fft_3d) in D1, D2.  Its
// adjoint runs the 2D adjoint's row kernels along x (ny nz rows) and the 3D
// y passes of the step (fs_ypass_kernel, with the packing of the kx = 0 /
// Nyquist column into (kx, ky) modes), around this kernel:
//   z forward of lam'_phi, u_phi, f_phi(u) (3 nf adjoint slots), the
//   multipliers D1 lam'^ and D2 lam'^ with the parameter sensitivities
//   (Parseval over the stored modes), z inverse of both, into slots phi and
//   nf + phi.
// One CTA per (kx tile, ky storage row, field phi), as the step's z kernel;
// a tensor map over the adjoint slots [slot][z][y][kx].
#pragma once

#include "fs_adjoint.cuh"
#include "fs_k3d_impl.cuh"

namespace fs {

template <typename T, int NZ>
__global__ void __launch_bounds__(LineCfg<T, NZ>::THREADS, 2)
    fs_adj_z_kernel(KArgs a, const __grid_constant__ CUtensorMap tmap) {
  using C = cplx<T>;
  using Cfg = LineCfg<T, NZ>;
  constexpr int E = Cfg::E, TPL = Cfg::TPL, BH = Cfg::BH, LOGE = Cfg::LOGE, TROWS = Cfg::TROWS;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  C* tw = reinterpret_cast<C*>(smem_raw + Cfg::BAR_BYTES);
  T* k2zt = reinterpret_cast<T*>(smem_raw + Cfg::BAR_BYTES + Cfg::TW_BYTES);
  C* tiles = reinterpret_cast<C*>(smem_raw + Cfg::HEAD);  // [3][TROWS][tk]: lam', u, f
  const int tk = blockDim.x / TPL;
  const int j = threadIdx.x % tk, t = threadIdx.x / tk;
  const int Lh = a.nx / 2, NY = a.ny, nf = a.nf;
  const int kx0 = blockIdx.x * tk, kx = kx0 + j;
  const int ky = blockIdx.y;  // storage row
  const int phi = blockIdx.z;
  const int fk = phi == 0 ? 0 : 1;
  const long long zstride = (long long)NY * Lh;
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_arrive_expect_tx(bar, (uint32_t)(3 * NZ * tk * sizeof(C)));
    const int cx = kx0 * (int)(sizeof(C) / 8);
    for (int i = 0; i < 3; ++i)
      for (int z0 = 0; z0 < NZ; z0 += BH)
        tma_load_4d(tiles + (i * TROWS + z0) * tk, &tmap, cx, ky, z0, i * nf + phi, bar);
  }
  copy_to_smem(tw, reinterpret_cast<const C*>(a.tw_z), Cfg::TWS);
  for (int i = threadIdx.x; i < NZ; i += blockDim.x) k2zt[i] = reinterpret_cast<const T*>(a.k2z)[i];
  __syncthreads();
  if (!mbar_wait_bounded(bar, 0, first_wait_polls(a))) {
    if (threadIdx.x == 0) atomicOr(a.flag, FS_FLAG_TIMEOUT);
    mbar_wait_bounded(bar, 0, kWaitPolls);
    return;
  }
  auto sync = []() { __syncthreads(); };
  // forward z of the three tiles, results back in natural layout
  for (int i = 0; i < 3; ++i) {
    C* tl = tiles + i * TROWS * tk + j;
    auto st = [tl, tk](int q, C x) { tl[(q + (q >> LOGE)) * tk] = x; };
    auto ld = [tl, tk](int q) { return tl[(q + (q >> LOGE)) * tk]; };
    C v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = tl[(t + TPL * m) * tk];
    line_fft<NZ, E, -1>(v, t, tw, st, ld, sync);
    sync();
#pragma unroll
    for (int m = 0; m < E; ++m) tl[(t + TPL * m) * tk] = v[m];
  }
  sync();
  const Coef<T>& co = coef<T>(a);
  AdjCoef<T> ac;
  ac.Mdt = co.Mdt;
  ac.Ldt = co.Ldt;
  ac.kc = co.kc;
  ac.ke = co.ke;
  ac.dt = co.dt;
  const T scale = co.scale;
  const T* __restrict__ k2xt = reinterpret_cast<const T*>(a.k2x);
  const T* __restrict__ k2yt = reinterpret_cast<const T*>(a.k2y);
  // K2 of this line without the z part, as in the step's z kernel: in the
  // packed column (kx = 0 tile, j = 0) rows below ny/2 are x-DC modes, rows
  // above x-Nyquist modes; rows 0 and ny/2 hold two modes each (`pair`).
  const bool col0 = (kx0 == 0 && j == 0);
  const T kxn2 = k2xt[Lh];
  const T kxy2 = (col0 ? (ky <= NY / 2 ? k2xt[0] : kxn2) : k2xt[kx]) + k2yt[ky];
  const bool pair = col0 && (ky == 0 || ky == NY / 2);
  const T kxa = (ky == 0) ? k2xt[0] : kxn2;
  const T kya = k2yt[0], kyb = k2yt[NY / 2];
  const C* TL = tiles;              // Lam'
  const C* TU = tiles + TROWS * tk;  // U
  const C* TF = tiles + 2 * TROWS * tk;  // Fu
  double g4[4] = {0.0, 0.0, 0.0, 0.0};
  C va[E], vb[E];
  // Parseval over the stored modes: a line that is not a pair row stands for
  // itself and its conjugate partner (weight 2); a pair row's two real-packed
  // z sequences are stored whole (weight 1 each)
#pragma unroll
  for (int m = 0; m < E; ++m) {
    const int kz = t + TPL * m;
    const T kz2 = k2zt[kz];
    const C l = TL[kz * tk + j], u = TU[kz * tk + j], f = TF[kz * tk + j];
    T d1, d2, dd1[4], dd2[4];
    if (pair) {
      const int kq = (NZ - kz) & (NZ - 1);
      const C lq = cconj(TL[kq * tk + j]), uq = cconj(TU[kq * tk + j]), fq = cconj(TF[kq * tk + j]);
      const C lP = cscale(cadd(l, lq), T(0.5)), lQ = cscale(mul_i<-1>(csub(l, lq)), T(0.5));
      const C uP = cscale(cadd(u, uq), T(0.5)), uQ = cscale(mul_i<-1>(csub(u, uq)), T(0.5));
      const C fP = cscale(cadd(f, fq), T(0.5)), fQ = cscale(mul_i<-1>(csub(f, fq)), T(0.5));
      ac.eval(fk, kxa + kya + kz2, d1, d2, dd1, dd2);
      const C aP = cscale(lP, d1 * scale), bP = cscale(lP, d2 * scale);
      for (int q = 0; q < 4; ++q)
        g4[q] += (double)lP.x * (dd1[q] * uP.x + dd2[q] * fP.x) + (double)lP.y * (dd1[q] * uP.y + dd2[q] * fP.y);
      ac.eval(fk, kxa + kyb + kz2, d1, d2, dd1, dd2);
      const C aQ = cscale(lQ, d1 * scale), bQ = cscale(lQ, d2 * scale);
      for (int q = 0; q < 4; ++q)
        g4[q] += (double)lQ.x * (dd1[q] * uQ.x + dd2[q] * fQ.x) + (double)lQ.y * (dd1[q] * uQ.y + dd2[q] * fQ.y);
      va[m] = cadd(aP, mul_i<1>(aQ));
      vb[m] = cadd(bP, mul_i<1>(bQ));
    } else {
      ac.eval(fk, kxy2 + kz2, d1, d2, dd1, dd2);
      va[m] = cscale(l, d1 * scale);
      vb[m] = cscale(l, d2 * scale);
      for (int q = 0; q < 4; ++q)
        g4[q] += 2.0 * ((double)l.x * (dd1[q] * u.x + dd2[q] * f.x) + (double)l.y * (dd1[q] * u.y + dd2[q] * f.y));
    }
  }
  for (int q = 0; q < 4; ++q) {
    double v = g4[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(&a.acc[q], v);
  }
  sync();  // every thread has read the three tiles: they become exchange buffers
  C* base = reinterpret_cast<C*>(a.spec) + (long long)ky * Lh + kx;
  // inverse z of D1 lam'^ (exchange in tile 0) into slot phi and of D2 lam'^
  // (tile 1) into slot nf + phi
  auto inverse_store = [&](C(&v)[E], int o) {
    C* tl = tiles + o * TROWS * tk + j;
    auto st = [tl, tk](int q, C x) { tl[(q + (q >> LOGE)) * tk] = x; };
    auto ld = [tl, tk](int q) { return tl[(q + (q >> LOGE)) * tk]; };
    line_fft<NZ, E, 1>(v, t, tw, st, ld, sync);
    C* S = base + (long long)(o * nf + phi) * a.slot_stride;
#pragma unroll
    for (int m = 0; m < E; ++m)
      if (spec_ok(a, &S[(long long)(t + TPL * m) * zstride], sizeof(C))) S[(long long)(t + TPL * m) * zstride] = v[m];
  };
  inverse_store(va, 0);
  inverse_store(vb, 1);
}

}  // namespace fs
