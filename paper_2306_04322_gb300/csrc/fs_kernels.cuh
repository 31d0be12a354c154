// CUDA kernels of the semi-implicit Fourier-spectral phase-field step.
//
// Model (Boccardo et al., arXiv 2306.04322, Section 2.1): composition c and
// order parameters eta_1..eta_p, chemical free energy
//   f_chem = rho2 (c - c_a)^2 (1 - h) + rho2 (c_b - c)^2 h + w g,
//   h = sum_i eta_i^3 (6 eta_i^2 - 15 eta_i + 10),
//   g = sum_i eta_i^2 (1 - eta_i)^2 + alpha sum_i sum_{j != i} eta_i^2 eta_j^2.
// Time step (Section 2.2, Eqs. C-H_discrete_fft / A-C_discrete_fft, b terms
// C-H_fft_b / A-C_fft_b, per-mode solve A-C_discrete_fft_c / _eta, Algorithm 1):
//   c^'   = (c^ - M dt K2 (df/dc)^) / (1 + M dt kappa_c K2^2)
//   eta^' = (eta^ - L dt (df/deta)^) / (1 + L dt kappa_eta K2)
// with K2 = |xi|^2 (Eqs. Gamma_fft, Gamma_fft_3d or the FS-FD forms).
//
// Pass structure on the device (2D, nf = 1 + p fields, all spectra stored as
// packed half spectra along x: nx/2 complex per row, bin 0 holding the real
// DC value in .x and the real Nyquist value in .y):
//   row pass    (one CTA per group of rows): inverse x transform of the
//               previous step's spectra (or a load of the real fields), the
//               pointwise derivative stage, and forward x transforms of
//               c, g_i = eta_i - L dt df/deta_i and df/dc.  Linearity of the
//               DFT lets the eta update use one transform of g_i instead of
//               two (eta^ - L dt (df/deta)^ = (eta - L dt df/deta)^).
//   column pass (one CTA per tile of kx columns): forward y transforms, the
//               per-mode k-space update with the 1/N scale folded in, and
//               inverse y transforms, in place.
// The next step's row pass starts with the inverse x transform, so the real
// fields only reach global memory when they are asked for.
#pragma once

#include "fs_fft.cuh"
#include "fs_internal.h"

namespace fs {

// ---------------------------------------------------------------------------
// Pointwise derivative stage (Section 2.1 definitions, differentiated).
//   df/dc     = 2 rho2 (c - c_a - (c_b - c_a) h)
//   df/deta_i = rho2 (c_b - c_a)(c_b + c_a - 2c) h'(eta_i)
//               + w [2 eta_i (1 - eta_i)(1 - 2 eta_i) + 4 alpha eta_i sum_{j!=i} eta_j^2]
//   h'(e) = 30 e^2 (1 - e)^2.  The factor 4 alpha counts the ordered pairs of
//   the double sum in g.
// ---------------------------------------------------------------------------
template <typename T>
struct Pointwise {
  T two_rho2, ca, dcab, rho2dcab, cab, w, four_alpha, Ldt;
  __device__ explicit Pointwise(const KArgs& a)
      : two_rho2((T)(2.0 * a.rho2)), ca((T)a.c_alpha), dcab((T)(a.c_beta - a.c_alpha)),
        rho2dcab((T)(a.rho2 * (a.c_beta - a.c_alpha))), cab((T)(a.c_beta + a.c_alpha)), w((T)a.w),
        four_alpha((T)(4.0 * a.alpha)), Ldt((T)(a.L * a.dt)) {}
  __device__ __forceinline__ T hpoly(T e) const { return e * e * e * (e * (T(6) * e - T(15)) + T(10)); }
  __device__ __forceinline__ T dh(T e) const {
    T q = e * (T(1) - e);
    return T(30) * q * q;
  }
  __device__ __forceinline__ T fc(T c, T h) const { return two_rho2 * (c - ca - dcab * h); }
  __device__ __forceinline__ T feta(T c, T e, T S2) const {
    T chem = rho2dcab * (cab - T(2) * c) * dh(e);
    T well = T(2) * e * (T(1) - e) * (T(1) - T(2) * e) + four_alpha * e * (S2 - e * e);
    return chem + w * well;
  }
};

template <typename T>
__device__ __forceinline__ bool finite_val(T x) {
  return isfinite(x);
}

// ---------------------------------------------------------------------------
// Row pass.  Lines along x; one group of TPL threads per row.
// Shared memory per row: (nf + 1) slots of padded_len(L) complex values.
// mode 0: step, previous state in spec slots 0..nf-1 (y-inverted spectra)
// mode 1: step, previous state in the real fields
// mode 2: inverse only: spec slots 0..nf-1 -> real fields
// Outputs of a step: spec slot 0 = 2 x^(c), slots 1..p = 2 x^(g_i),
// slot nf = 2 x^(df/dc) (x-spectra scaled by 2; the factor is folded into
// the k-space scale).
// ---------------------------------------------------------------------------
template <typename T, int NX>
struct RowCfg {
  static constexpr int L = NX / 2;
  static constexpr int E = imin(L, sizeof(T) == 4 ? 16 : 8);
  static constexpr int TPL = L / E;
  static constexpr int PL = padded_len(L);
  static constexpr int THREADS = imax(TPL, 128);
};

template <typename T, int NX>
__global__ void __launch_bounds__(RowCfg<T, NX>::THREADS) fs_row_kernel(KArgs a) {
  using C = cplx<T>;
  using Cfg = RowCfg<T, NX>;
  constexpr int L = Cfg::L, E = Cfg::E, TPL = Cfg::TPL, PL = Cfg::PL;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sm = reinterpret_cast<C*>(smem_raw);
  const int nf = a.nf;
  const int rl = threadIdx.x / TPL, t = threadIdx.x % TPL;
  const int rpc = blockDim.x / TPL;
  const long long row = (long long)blockIdx.x * rpc + rl;
  C* slots = sm + (size_t)rl * (nf + 1) * PL;
  const C* __restrict__ tw = reinterpret_cast<const C*>(a.tw);
  C* spec = reinterpret_cast<C*>(a.spec);
  C* realc = reinterpret_cast<C*>(a.real);  // real row as complex pairs
  const long long half_stride = a.npts / 2;  // complex pairs per real field
  auto sync = []() { __syncthreads(); };

  bool bad = false;
  // 1. real-space row of every field into its slot (as pairs x[2j], x[2j+1])
  for (int f = 0; f < nf; ++f) {
    C* s = slots + f * PL;
    auto st = [s](int i, C v) { s[pad32(i)] = v; };
    auto ld = [s](int i) { return s[pad32(i)]; };
    C v[E];
    if (a.mode == 1) {
      const C* src = realc + f * half_stride + row * L;
#pragma unroll
      for (int m = 0; m < E; ++m) v[m] = src[t + TPL * m];
    } else {
      const C* P = spec + f * a.slot_stride + row * L;
#pragma unroll
      for (int m = 0; m < E; ++m) {
        int k = t + TPL * m;
        C pk = P[k];
        if (k == 0) {
          v[m] = mk<C>(pk.x + pk.y, pk.x - pk.y);
        } else {
          C pm = P[L - k];
          C A = cadd(pk, cconj(pm)), B = csub(pk, cconj(pm));
          v[m] = cadd(A, mul_i<1>(cmul(tw_root<1, NX>(tw, k), B)));
        }
      }
      line_fft<L, E, 1>(v, t, tw, st, ld, sync);
      sync();
    }
    if (a.mode == 2) {
      C* dst = realc + f * half_stride + row * L;
#pragma unroll
      for (int m = 0; m < E; ++m) dst[t + TPL * m] = v[m];
    } else {
#pragma unroll
      for (int m = 0; m < E; ++m) st(t + TPL * m, v[m]);
    }
  }
  if (a.mode == 2) return;

  // 2. pointwise derivative stage on the thread's own points
  {
    Pointwise<T> pw(a);
    const int p = nf - 1;
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const int ip = pad32(t + TPL * m);
      C c = slots[ip];
      C h = mk<C>(T(0), T(0)), S2 = mk<C>(T(0), T(0));
      for (int i = 0; i < p; ++i) {
        C e = slots[(1 + i) * PL + ip];
        h.x += pw.hpoly(e.x);
        h.y += pw.hpoly(e.y);
        S2.x += e.x * e.x;
        S2.y += e.y * e.y;
        bad |= !(finite_val(e.x) && finite_val(e.y));
      }
      bad |= !(finite_val(c.x) && finite_val(c.y));
      slots[nf * PL + ip] = mk<C>(pw.fc(c.x, h.x), pw.fc(c.y, h.y));
      for (int i = 0; i < p; ++i) {
        C e = slots[(1 + i) * PL + ip];
        C g = mk<C>(e.x - pw.Ldt * pw.feta(c.x, e.x, S2.x), e.y - pw.Ldt * pw.feta(c.y, e.y, S2.y));
        slots[(1 + i) * PL + ip] = g;
      }
    }
  }

  // 3. forward x transforms (packed half spectra, scaled by 2)
  for (int o = 0; o <= nf; ++o) {
    C* s = slots + o * PL;
    auto st = [s](int i, C v) { s[pad32(i)] = v; };
    auto ld = [s](int i) { return s[pad32(i)]; };
    C v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = ld(t + TPL * m);
    line_fft<L, E, -1>(v, t, tw, st, ld, sync);
    sync();
#pragma unroll
    for (int m = 0; m < E; ++m) st(t + TPL * m, v[m]);
    sync();
    C* P = spec + o * a.slot_stride + row * L;
#pragma unroll
    for (int m = 0; m < E; ++m) {
      int k = t + TPL * m;
      C zk = ld(k);
      C out;
      if (k == 0) {
        out = mk<C>(T(2) * (zk.x + zk.y), T(2) * (zk.x - zk.y));
      } else {
        C zm = ld(L - k);
        C A = cadd(zk, cconj(zm)), B = csub(zk, cconj(zm));
        out = cadd(A, mul_i<-1>(cmul(tw_root<-1, NX>(tw, k), B)));
      }
      P[k] = out;
    }
  }
  if (bad) atomicOr(a.flag, FS_FLAG_NONFINITE);
}

// ---------------------------------------------------------------------------
// Column pass (2D step).  Lines along y of the packed x-spectra; one CTA per
// tile of TK adjacent kx columns, TPL threads per column.  Forward y
// transforms, k-space update, inverse y transforms, in place.
// ---------------------------------------------------------------------------
template <typename T, int NY>
struct ColCfg {
  static constexpr int E = imin(NY, sizeof(T) == 4 ? 16 : 8);
  static constexpr int TPL = NY / E;
  static constexpr int TK = imin(sizeof(T) == 4 ? 16 : 8, imax(1, 512 / TPL));
  static constexpr int THREADS = TPL * TK;
};

template <typename T>
struct KUpdate {
  T Mdt, Mdtkc, Ldtke, scale;
  __device__ explicit KUpdate(const KArgs& a)
      : Mdt((T)(a.M * a.dt)), Mdtkc((T)(a.M * a.dt * a.kappa_c)), Ldtke((T)(a.L * a.dt * a.kappa_eta)),
        scale((T)a.scale) {}
  // c^' = (c^ - M dt K2 f^) / (1 + M dt kappa_c K2^2), times the 1/(2N) scale
  template <typename C>
  __device__ __forceinline__ C c(C zc, C zf, T k2) const {
    T d = scale / (T(1) + Mdtkc * k2 * k2);
    T b = Mdt * k2;
    return mk<C>((zc.x - b * zf.x) * d, (zc.y - b * zf.y) * d);
  }
  // eta^' = g^ / (1 + L dt kappa_eta K2), times the 1/(2N) scale
  template <typename C>
  __device__ __forceinline__ C eta(C zg, T k2) const {
    return cscale(zg, scale / (T(1) + Ldtke * k2));
  }
};

template <typename T, int NY>
__global__ void __launch_bounds__(ColCfg<T, NY>::THREADS) fs_col_kernel(KArgs a) {
  using C = cplx<T>;
  using Cfg = ColCfg<T, NY>;
  constexpr int E = Cfg::E, TPL = Cfg::TPL;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tile = reinterpret_cast<C*>(smem_raw);
  const int tk = blockDim.x / TPL;  // columns in this CTA (<= TK)
  const int j = threadIdx.x % tk, t = threadIdx.x / tk;
  const int Lh = a.nx / 2;
  const int kx0 = blockIdx.x * tk;
  const int kx = kx0 + j;
  const C* __restrict__ tw = reinterpret_cast<const C*>(a.tw);
  C* spec = reinterpret_cast<C*>(a.spec) + kx;
  auto st = [tile, tk, j](int i, C v) { tile[i * tk + j] = v; };
  auto ld = [tile, tk, j](int i) { return tile[i * tk + j]; };
  auto sync = []() { __syncthreads(); };
  const KUpdate<T> up(a);
  const int nf = a.nf;
  const bool special = (kx0 == 0);  // CTA holding the packed DC/Nyquist column
  const T kx2 = (T)__ldg(&a.k2x[kx]);
  const T kxn2 = (T)__ldg(&a.k2x[Lh]);  // Nyquist column

  // ---- c and df/dc
  C vc[E], vf[E];
  {
    const C* Sc = spec;
    const C* Sf = spec + (long long)nf * a.slot_stride;
#pragma unroll
    for (int m = 0; m < E; ++m) {
      vc[m] = Sc[(long long)(t + TPL * m) * Lh];
      vf[m] = Sf[(long long)(t + TPL * m) * Lh];
    }
  }
  line_fft<NY, E, -1>(vc, t, tw, st, ld, sync);
  line_fft<NY, E, -1>(vf, t, tw, st, ld, sync);
  if (special) {
    // Separate the packed column Z = A + i B (A: kx = 0, B: kx = nx/2, both
    // Hermitian in ky) through shared memory, update both, repack.
    sync();
    C* zc = tile;
    C* zf = tile + NY;
    if (j == 0) {
#pragma unroll
      for (int m = 0; m < E; ++m) {
        zc[t + TPL * m] = vc[m];
        zf[t + TPL * m] = vf[m];
      }
    }
    sync();
    if (j == 0) {
#pragma unroll
      for (int m = 0; m < E; ++m) {
        int ky = t + TPL * m, kq = (NY - ky) & (NY - 1);
        C pc = cconj(zc[kq]), pf = cconj(zf[kq]);
        C Ac = cscale(cadd(vc[m], pc), T(0.5)), Bc = cscale(mul_i<-1>(csub(vc[m], pc)), T(0.5));
        C Af = cscale(cadd(vf[m], pf), T(0.5)), Bf = cscale(mul_i<-1>(csub(vf[m], pf)), T(0.5));
        T ky2 = (T)__ldg(&a.k2y[ky]);
        C An = up.c(Ac, Af, kx2 + ky2);
        C Bn = up.c(Bc, Bf, kxn2 + ky2);
        if (ky == 0 && a.csum) An = mk<C>((T)(*a.csum * a.inv_npts), T(0));
        vc[m] = cadd(An, mul_i<1>(Bn));
      }
    } else {
#pragma unroll
      for (int m = 0; m < E; ++m) {
        int ky = t + TPL * m;
        vc[m] = up.c(vc[m], vf[m], kx2 + (T)__ldg(&a.k2y[ky]));
      }
    }
  } else {
#pragma unroll
    for (int m = 0; m < E; ++m) {
      int ky = t + TPL * m;
      vc[m] = up.c(vc[m], vf[m], kx2 + (T)__ldg(&a.k2y[ky]));
    }
  }
  line_fft<NY, E, 1>(vc, t, tw, st, ld, sync);
  {
    C* Sc = spec;
#pragma unroll
    for (int m = 0; m < E; ++m) Sc[(long long)(t + TPL * m) * Lh] = vc[m];
  }

  // ---- eta_i (slot i holds g_i = eta_i - L dt df/deta_i)
  for (int i = 1; i < nf; ++i) {
    C* S = spec + (long long)i * a.slot_stride;
    C v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = S[(long long)(t + TPL * m) * Lh];
    line_fft<NY, E, -1>(v, t, tw, st, ld, sync);
    if (special) {
      sync();
      C* z = tile;
      if (j == 0) {
#pragma unroll
        for (int m = 0; m < E; ++m) z[t + TPL * m] = v[m];
      }
      sync();
      if (j == 0) {
#pragma unroll
        for (int m = 0; m < E; ++m) {
          int ky = t + TPL * m, kq = (NY - ky) & (NY - 1);
          C pz = cconj(z[kq]);
          C A = cscale(cadd(v[m], pz), T(0.5)), B = cscale(mul_i<-1>(csub(v[m], pz)), T(0.5));
          T ky2 = (T)__ldg(&a.k2y[ky]);
          v[m] = cadd(up.eta(A, kx2 + ky2), mul_i<1>(up.eta(B, kxn2 + ky2)));
        }
      } else {
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = up.eta(v[m], kx2 + (T)__ldg(&a.k2y[t + TPL * m]));
      }
    } else {
#pragma unroll
      for (int m = 0; m < E; ++m) v[m] = up.eta(v[m], kx2 + (T)__ldg(&a.k2y[t + TPL * m]));
    }
    line_fft<NY, E, 1>(v, t, tw, st, ld, sync);
#pragma unroll
    for (int m = 0; m < E; ++m) S[(long long)(t + TPL * m) * Lh] = v[m];
  }
}

}  // namespace fs
