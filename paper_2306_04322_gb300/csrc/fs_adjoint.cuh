// Adjoint of one 2D semi-implicit Fourier-spectral step.  The step maps the
// real state u to u'_phi = F^-1[ D1_phi F u_phi + D2_phi F f_phi(u) ] with
//   c:     D1 = 1/(1 + M dt kc K2^2),  D2 = -M dt K2 / (1 + M dt kc K2^2)
//   eta_i: D1 = 1/(1 + L dt ke K2),    D2 = -L dt / (1 + L dt ke K2)
// (Eqs. C-H_discrete_fft .. A-C_discrete_fft_eta), f_phi = df_chem/dphi.
// D1, D2 are real and even in k, so G = F^-1 D F is real symmetric, and
//   lambda_phi = G1_phi lam'_phi + sum_psi H_phi,psi(u) G2_psi lam'_psi
// with H the pointwise Hessian of f_chem.  Parameter sensitivities of
// <lam', u'> for theta = (M, L, kappa_c, kappa_eta) follow from Parseval:
//   d/dtheta = (1/N) sum_k conj(Lam'(k)) (dD1/dtheta U(k) + dD2/dtheta Fu(k)).
// Three passes (adjoint workspace: 3 nf packed half-spectrum slots):
//   adj row forward  x transforms of lam'_phi, u_phi, f_phi(u)
//   adj column       y transforms, G1/G2 multipliers, sensitivities, inverse y
//   adj row inverse  inverse x transforms and the pointwise Hessian product
#pragma once

#include "fs_kernels.cuh"

namespace fs {

// Pointwise Hessian of f_chem in (c, eta_1..eta_p):
//   H_cc = 2 rho2, H_c,k = -2 rho2 (cb - ca) h'(eta_k),
//   H_k,k = rho2 (cb - ca)(cb + ca - 2c) h''(eta_k)
//           + w [2 - 12 eta_k + 12 eta_k^2 + 4 alpha sum_{j != k} eta_j^2],
//   H_k,l = 8 w alpha eta_k eta_l (k != l),  h''(e) = 60 e (1 - e)(1 - 2e).
template <typename T>
__device__ __forceinline__ void hessian_apply(const Pointwise<T>& pw, T c, const T* eta, int p, const T* mu,
                                              T* out) {
  T S2 = T(0);
  for (int i = 0; i < p; ++i) S2 += eta[i] * eta[i];
  out[0] = pw.two_rho2 * mu[0];
  const T alpha = pw.four_alpha * T(0.25);
  for (int k = 0; k < p; ++k) {
    const T e = eta[k];
    const T hck = -pw.two_rho2 * pw.dcab * pw.dh(e);
    out[0] += hck * mu[1 + k];
    const T d2h = T(60) * e * (T(1) - e) * (T(1) - T(2) * e);
    T hkk = pw.rho2dcab * (pw.cab - T(2) * c) * d2h +
            pw.w * (T(2) - T(12) * e + T(12) * e * e + T(4) * alpha * (S2 - e * e));
    T acc = hck * mu[0] + hkk * mu[1 + k];
    for (int l = 0; l < p; ++l)
      if (l != k) acc += T(8) * pw.w * alpha * e * eta[l] * mu[1 + l];
    out[1 + k] = acc;
  }
}

// ---------------------------------------------------------------------------
// Adjoint row forward: CTA of nf + 1 warps and R rows (as the step's row
// pass).  Inputs real: lam' (a.real), u (a.aux).  Outputs 2 x^ of lam'_phi,
// u_phi, f_phi(u) into adjoint slots [0, nf), [nf, 2nf), [2nf, 3nf).
// ---------------------------------------------------------------------------
template <typename T, int NX>
__global__ void __launch_bounds__(192) fs_adj_row_fwd_kernel(KArgs a) {
  using C = cplx<T>;
  using Cfg = RowCfg<T, NX>;
  constexpr int L = Cfg::L, E = Cfg::E, TPL = Cfg::TPL, R = Cfg::R, PL = Cfg::PL;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  C* twr = reinterpret_cast<C*>(smem_raw + Cfg::BAR_BYTES);
  C* slots = reinterpret_cast<C*>(smem_raw + Cfg::BAR_BYTES + Cfg::TW_BYTES);
  const int nf = a.nf, nw = blockDim.x >> 5;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane / TPL, t = lane % TPL;
  const int Reff = a.lines < R ? (int)a.lines : R;
  const bool active = g < Reff;
  const long long row0 = (long long)blockIdx.x * Reff, row = row0 + g;
  const C* __restrict__ twh = reinterpret_cast<const C*>(a.tw_half);
  const long long half_stride = a.npts / 2;
  auto slot = [slots](int f, int r) { return slots + (f * R + r) * PL; };
  auto wsync = []() { __syncwarp(); };
  copy_to_smem(twr, reinterpret_cast<const C*>(a.tw_row), Cfg::TWS);
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint32_t bytes = (uint32_t)(L * sizeof(C));
    mbar_arrive_expect_tx(bar, bytes * Reff * 2 * nf);
    for (int f = 0; f < nf; ++f)
      for (int r = 0; r < Reff; ++r) {
        bulk_g2s(slot(f, r), reinterpret_cast<const C*>(a.real) + f * half_stride + (row0 + r) * L, bytes, bar);
        bulk_g2s(slot(nf + f, r), reinterpret_cast<const C*>(a.aux) + f * half_stride + (row0 + r) * L, bytes,
                 bar);
      }
  }
  if (!mbar_wait_bounded(bar, 0, first_wait_polls(a))) {
    if (threadIdx.x == 0) atomicOr(a.flag, FS_FLAG_TIMEOUT);
    mbar_wait_bounded(bar, 0, kWaitPolls);
    return;
  }
  // f(u) into slots [2nf, 3nf)
  {
    const Pointwise<T> pw(a);
    const int p = nf - 1;
    for (int idx = threadIdx.x; idx < Reff * L; idx += blockDim.x) {
      const int r = idx / L, i0 = idx % L;
      const C c = slot(nf, r)[i0];
      C h = mk<C>(T(0), T(0)), S2 = mk<C>(T(0), T(0));
      for (int i = 0; i < p; ++i) {
        const C e = slot(nf + 1 + i, r)[i0];
        h.x += pw.hpoly(e.x);
        h.y += pw.hpoly(e.y);
        S2.x += e.x * e.x;
        S2.y += e.y * e.y;
      }
      slot(2 * nf, r)[i0] = mk<C>(pw.fc(c.x, h.x), pw.fc(c.y, h.y));
      for (int i = 0; i < p; ++i) {
        const C e = slot(nf + 1 + i, r)[i0];
        slot(2 * nf + 1 + i, r)[i0] = mk<C>(pw.feta(c.x, e.x, S2.x), pw.feta(c.y, e.y, S2.y));
      }
    }
  }
  __syncthreads();
  C* spec = reinterpret_cast<C*>(a.spec);
  for (int o = w; o < 3 * nf; o += nw) {
    C* s = slot(o, g);
    auto st = [s](int i, C v) { s[Cfg::P16 ? pad16(i) : pad32(i)] = v; };
    auto ld = [s](int i) { return s[Cfg::P16 ? pad16(i) : pad32(i)]; };
    C v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = s[t + TPL * m];
    line_fft<L, E, -1>(v, t, twr, st, ld, wsync);
    wsync();
#pragma unroll
    for (int m = 0; m < E; ++m) s[t + TPL * m] = v[m];
    wsync();
    C* P = spec + o * a.slot_stride + row * L;
    if (active) {
#pragma unroll
      for (int m = 0; m < E; ++m) {
        const int k = t + TPL * m;
        const C zk = s[k];
        C out;
        if (k == 0) {
          out = mk<C>(T(2) * (zk.x + zk.y), T(2) * (zk.x - zk.y));
        } else {
          const C zm = cconj(s[L - k]);
          const C A = cadd(zk, zm), B = csub(zk, zm);
          out = cadd(A, mul_i<-1>(cmul(B, __ldg(&twh[k]))));
        }
        P[k] = out;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Adjoint column pass: one CTA per (kx tile, field phi).  Loads the tiles of
// lam'_phi, u_phi, f_phi; forward y; sensitivities into acc[0..3]; writes
// D1 lam'^ (slot phi) and D2 lam'^ (slot nf + phi), inverse y, scaled 1/(2N).
// ---------------------------------------------------------------------------
template <typename T>
struct AdjCoef {
  T Mdt, Ldt, kc, ke, dt;
  // multipliers and their parameter derivatives at K2 for field kind f (0: c)
  __device__ __forceinline__ void eval(int f, T k2, T& d1, T& d2, T* dd1, T* dd2) const {
    if (f == 0) {
      const T den = T(1) + Mdt * kc * k2 * k2, i2 = T(1) / (den * den);
      d1 = T(1) / den;
      d2 = -Mdt * k2 / den;
      dd1[0] = -dt * kc * k2 * k2 * i2;          // d/dM
      dd1[1] = T(0);                             // d/dL
      dd1[2] = -Mdt * k2 * k2 * i2;              // d/dkappa_c
      dd1[3] = T(0);                             // d/dkappa_eta
      dd2[0] = -dt * k2 * i2;
      dd2[1] = T(0);
      dd2[2] = Mdt * Mdt * k2 * k2 * k2 * i2;
      dd2[3] = T(0);
    } else {
      const T den = T(1) + Ldt * ke * k2, i2 = T(1) / (den * den);
      d1 = T(1) / den;
      d2 = -Ldt / den;
      dd1[0] = T(0);
      dd1[1] = -dt * ke * k2 * i2;
      dd1[2] = T(0);
      dd1[3] = -Ldt * k2 * i2;
      dd2[0] = T(0);
      dd2[1] = -dt * i2;
      dd2[2] = T(0);
      dd2[3] = Ldt * Ldt * k2 * i2;
    }
  }
};

template <typename T, int NY>
__global__ void __launch_bounds__(ColCfg<T, NY>::THREADS) fs_adj_col_kernel(KArgs a, const __grid_constant__ CUtensorMap tmap) {
  using C = cplx<T>;
  using Cfg = ColCfg<T, NY>;
  constexpr int E = Cfg::E, TPL = Cfg::TPL, BH = Cfg::BH, TROWS = Cfg::TROWS, LOGE = Cfg::LOGE;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  C* twc = reinterpret_cast<C*>(smem_raw + Cfg::BAR_BYTES);
  T* k2yt = reinterpret_cast<T*>(smem_raw + Cfg::BAR_BYTES + Cfg::TW_BYTES);
  C* tiles = reinterpret_cast<C*>(smem_raw + Cfg::HEAD);  // [3][TROWS][tk]
  const int tk = blockDim.x / TPL;
  const int j = threadIdx.x % tk, t = threadIdx.x / tk;
  const int Lh = a.nx / 2, nf = a.nf;
  const int kx0 = blockIdx.x * tk, kx = kx0 + j, phi = blockIdx.y;
  const int fk = phi == 0 ? 0 : 1;
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_arrive_expect_tx(bar, (uint32_t)(3 * NY * tk * sizeof(C)));
    const int cx = kx0 * (int)(sizeof(C) / 8);
    for (int i = 0; i < 3; ++i)
      for (int y0 = 0; y0 < NY; y0 += BH) tma_load_3d(tiles + (i * TROWS + y0) * tk, &tmap, cx, y0, i * nf + phi, bar);
  }
  copy_to_smem(twc, reinterpret_cast<const C*>(a.tw_col), Cfg::TWS);
  for (int i = threadIdx.x; i < NY; i += blockDim.x) k2yt[i] = reinterpret_cast<const T*>(a.k2y)[i];
  __syncthreads();
  if (!mbar_wait_bounded(bar, 0, first_wait_polls(a))) {
    if (threadIdx.x == 0) atomicOr(a.flag, FS_FLAG_TIMEOUT);
    mbar_wait_bounded(bar, 0, kWaitPolls);
    return;
  }
  auto sync = []() { __syncthreads(); };
  // forward y of the three tiles, results back in natural layout
  for (int i = 0; i < 3; ++i) {
    C* tl = tiles + i * TROWS * tk + j;
    auto st = [tl, tk](int q, C x) { tl[(q + (q >> LOGE)) * tk] = x; };
    auto ld = [tl, tk](int q) { return tl[(q + (q >> LOGE)) * tk]; };
    C v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = tl[(t + TPL * m) * tk];
    line_fft<NY, E, -1>(v, t, twc, st, ld, sync);
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
  const T* k2xt = reinterpret_cast<const T*>(a.k2x);
  const T kx2 = k2xt[kx], kxn2 = k2xt[Lh], scale = co.scale;
  const C* TL = tiles + 0 * TROWS * tk;  // Lam'
  const C* TU = tiles + 1 * TROWS * tk;  // U
  const C* TF = tiles + 2 * TROWS * tk;  // Fu
  double g4[4] = {0.0, 0.0, 0.0, 0.0};
  C va[E], vb[E];
  const bool col0 = (kx0 == 0 && j == 0);
#pragma unroll
  for (int m = 0; m < E; ++m) {
    const int ky = t + TPL * m;
    const T ky2 = k2yt[ky];
    const C l = TL[ky * tk + j], u = TU[ky * tk + j], f = TF[ky * tk + j];
    T d1, d2, dd1[4], dd2[4];
    if (col0) {
      // split the packed column into its kx = 0 (P) and kx = nx/2 (Q) parts
      const int kq = (NY - ky) & (NY - 1);
      const C lq = cconj(TL[kq * tk]), uq = cconj(TU[kq * tk]), fq = cconj(TF[kq * tk]);
      const C lP = cscale(cadd(l, lq), T(0.5)), lQ = cscale(mul_i<-1>(csub(l, lq)), T(0.5));
      const C uP = cscale(cadd(u, uq), T(0.5)), uQ = cscale(mul_i<-1>(csub(u, uq)), T(0.5));
      const C fP = cscale(cadd(f, fq), T(0.5)), fQ = cscale(mul_i<-1>(csub(f, fq)), T(0.5));
      ac.eval(fk, kx2 + ky2, d1, d2, dd1, dd2);
      C aP = cscale(lP, d1 * scale), bP = cscale(lP, d2 * scale);
      for (int q = 0; q < 4; ++q)
        g4[q] += (double)lP.x * (dd1[q] * uP.x + dd2[q] * fP.x) + (double)lP.y * (dd1[q] * uP.y + dd2[q] * fP.y);
      ac.eval(fk, kxn2 + ky2, d1, d2, dd1, dd2);
      C aQ = cscale(lQ, d1 * scale), bQ = cscale(lQ, d2 * scale);
      for (int q = 0; q < 4; ++q)
        g4[q] += (double)lQ.x * (dd1[q] * uQ.x + dd2[q] * fQ.x) + (double)lQ.y * (dd1[q] * uQ.y + dd2[q] * fQ.y);
      va[m] = cadd(aP, mul_i<1>(aQ));
      vb[m] = cadd(bP, mul_i<1>(bQ));
    } else {
      ac.eval(fk, kx2 + ky2, d1, d2, dd1, dd2);
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
  sync();
  // inverse y of D1 lam'^ (exchange in tile 0) and D2 lam'^ (tile 1)
  C* base = reinterpret_cast<C*>(a.spec) + kx;
  {
    C* tl = tiles + 0 * TROWS * tk + j;
    auto st = [tl, tk](int q, C x) { tl[(q + (q >> LOGE)) * tk] = x; };
    auto ld = [tl, tk](int q) { return tl[(q + (q >> LOGE)) * tk]; };
    line_fft<NY, E, 1>(va, t, twc, st, ld, sync);
    C* S = base + (long long)phi * a.slot_stride;
#pragma unroll
    for (int m = 0; m < E; ++m) S[(long long)(t + TPL * m) * Lh] = va[m];
  }
  {
    C* tl = tiles + 1 * TROWS * tk + j;
    auto st = [tl, tk](int q, C x) { tl[(q + (q >> LOGE)) * tk] = x; };
    auto ld = [tl, tk](int q) { return tl[(q + (q >> LOGE)) * tk]; };
    line_fft<NY, E, 1>(vb, t, twc, st, ld, sync);
    C* S = base + (long long)(nf + phi) * a.slot_stride;
#pragma unroll
    for (int m = 0; m < E; ++m) S[(long long)(t + TPL * m) * Lh] = vb[m];
  }
}

// ---------------------------------------------------------------------------
// Adjoint row inverse: inverse x transforms of G1 lam' (slots [0, nf)) and
// G2 lam' (slots [nf, 2nf)); lambda_phi = G1 lam'_phi + sum H_phi,psi G2 lam'_psi
// with H at u (a.aux, real); result to a.real (lambda_out).
// ---------------------------------------------------------------------------
template <typename T, int NX>
__global__ void __launch_bounds__(192) fs_adj_row_inv_kernel(KArgs a) {
  using C = cplx<T>;
  using Cfg = RowCfg<T, NX>;
  constexpr int L = Cfg::L, E = Cfg::E, TPL = Cfg::TPL, R = Cfg::R, PL = Cfg::PL;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  C* twr = reinterpret_cast<C*>(smem_raw + Cfg::BAR_BYTES);
  C* slots = reinterpret_cast<C*>(smem_raw + Cfg::BAR_BYTES + Cfg::TW_BYTES);
  const int nf = a.nf, nw = blockDim.x >> 5;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane / TPL, t = lane % TPL;
  const int Reff = a.lines < R ? (int)a.lines : R;
  const long long row0 = (long long)blockIdx.x * Reff;
  const C* __restrict__ twh = reinterpret_cast<const C*>(a.tw_half);
  const long long half_stride = a.npts / 2;
  auto slot = [slots](int f, int r) { return slots + (f * R + r) * PL; };
  auto wsync = []() { __syncwarp(); };
  copy_to_smem(twr, reinterpret_cast<const C*>(a.tw_row), Cfg::TWS);
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint32_t bytes = (uint32_t)(L * sizeof(C));
    mbar_arrive_expect_tx(bar, bytes * Reff * 3 * nf);
    for (int f = 0; f < 2 * nf; ++f)
      for (int r = 0; r < Reff; ++r)
        bulk_g2s(slot(f, r), reinterpret_cast<const C*>(a.spec) + f * a.slot_stride + (row0 + r) * L, bytes, bar);
    for (int f = 0; f < nf; ++f)
      for (int r = 0; r < Reff; ++r)
        bulk_g2s(slot(2 * nf + f, r), reinterpret_cast<const C*>(a.aux) + f * half_stride + (row0 + r) * L, bytes,
                 bar);
  }
  if (!mbar_wait_bounded(bar, 0, first_wait_polls(a))) {
    if (threadIdx.x == 0) atomicOr(a.flag, FS_FLAG_TIMEOUT);
    mbar_wait_bounded(bar, 0, kWaitPolls);
    return;
  }
  for (int o = w; o < 2 * nf; o += nw) {
    C* s = slot(o, g);
    auto st = [s](int i, C v) { s[Cfg::P16 ? pad16(i) : pad32(i)] = v; };
    auto ld = [s](int i) { return s[Cfg::P16 ? pad16(i) : pad32(i)]; };
    C v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const int k = t + TPL * m;
      const C pk = s[k];
      if (k == 0) {
        v[m] = mk<C>(pk.x + pk.y, pk.x - pk.y);
      } else {
        const C pm = cconj(s[L - k]);
        const C A = cadd(pk, pm), B = csub(pk, pm);
        v[m] = cadd(A, mul_i<1>(mul_tw<1>(B, __ldg(&twh[k]))));
      }
    }
    line_fft<L, E, 1>(v, t, twr, st, ld, wsync);
    wsync();
#pragma unroll
    for (int m = 0; m < E; ++m) s[t + TPL * m] = v[m];
  }
  __syncthreads();
  const Pointwise<T> pw(a);
  const int p = nf - 1;
  C* out = reinterpret_cast<C*>(a.real);
  for (int idx = threadIdx.x; idx < Reff * L; idx += blockDim.x) {
    const int r = idx / L, i0 = idx % L;
#pragma unroll
    for (int h2 = 0; h2 < 2; ++h2) {
      T eta[4], mu[5], res[5];
      const C uc = slot(2 * nf, r)[i0];
      const T c = h2 ? uc.y : uc.x;
      for (int i = 0; i < p; ++i) {
        const C e = slot(2 * nf + 1 + i, r)[i0];
        eta[i] = h2 ? e.y : e.x;
      }
      for (int f = 0; f < nf; ++f) {
        const C m2 = slot(nf + f, r)[i0];
        mu[f] = h2 ? m2.y : m2.x;
      }
      hessian_apply(pw, c, eta, p, mu, res);
      for (int f = 0; f < nf; ++f) {
        C* sv = slot(f, r) + i0;
        if (h2) sv->y += res[f]; else sv->x += res[f];
      }
    }
    for (int f = 0; f < nf; ++f) out[f * half_stride + (row0 + r) * L + i0] = slot(f, r)[i0];
  }
}

}  // namespace fs
