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
//   row pass    (one group of threads per row): bulk-async load of every
//               field's row into shared memory, inverse x transform of the
//               previous step's spectra (or the real fields as loaded), the
//               pointwise derivative stage, and forward x transforms of
//               c, g_i = eta_i - L dt df/deta_i and df/dc.  Linearity of the
//               DFT lets the eta update use one transform of g_i instead of
//               two (eta^ - L dt (df/deta)^ = (eta - L dt df/deta)^).
//   column pass (one CTA per tile of kx columns and per field group): forward
//               y transforms, the per-mode k-space update with the 1/N scale
//               folded in, and inverse y transforms, in place.
// The next step's row pass starts with the inverse x transform, so the real
// fields only reach global memory when they are asked for.
#pragma once

#include "fs_fft.cuh"
#include "fs_internal.h"
#include "fs_tc.cuh"

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
  __device__ explicit Pointwise(const KArgs& a) {
    const Coef<T>& k = coef<T>(a);
    two_rho2 = k.two_rho2;
    ca = k.ca;
    dcab = k.dcab;
    rho2dcab = k.rho2dcab;
    cab = k.cab;
    w = k.w;
    four_alpha = k.four_alpha;
    Ldt = k.Ldt;
  }
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
  // The same on two lanes (two grid points per pair, lane-wise arithmetic).
  template <typename V>
  __device__ __forceinline__ V hpoly2(V e) const {  // e^3 (e (6 e - 15) + 10)
    const V t = vfma(e, vfma(e, vsplat<V>(T(6)), vsplat<V>(T(-15))), vsplat<V>(T(10)));
    return vmul(vmul(vmul(e, e), e), t);
  }
  template <typename V>
  __device__ __forceinline__ V fc2(V c, V h) const {  // 2 rho2 (c - c_a - (c_b - c_a) h)
    return vmul(vsplat<V>(two_rho2), vfma(h, vsplat<V>(-dcab), csub(c, vsplat<V>(ca))));
  }
  // g = eta - L dt df/deta
  template <typename V>
  __device__ __forceinline__ V g2(V c, V e, V S2) const {
    const V q = vfma(e, mk<V>(-e.x, -e.y), e);                                     // e (1 - e)
    const V chem = vmul(vmul(vsplat<V>(T(30) * rho2dcab), vmul(q, q)),
                        vfma(c, vsplat<V>(T(-2)), vsplat<V>(cab)));                // h'(e) rho2 dcab (cab - 2c)
    const V dw = vmul(q, vfma(e, vsplat<V>(T(-2)), vsplat<V>(T(1))));            // e (1 - e)(1 - 2e)
    const V pair = vmul(e, vfma(e, mk<V>(-e.x, -e.y), S2));                      // e (S2 - e^2)
    const V well = vfma(dw, vsplat<V>(T(2)), vmul(vsplat<V>(four_alpha), pair));
    return vfma(vfma(well, vsplat<V>(w), chem), vsplat<V>(-Ldt), e);
  }
};

// Polls of the first bounded wait of a pass: kWaitPolls, or none when the
// plan's test hook asks every pass to report a timeout.  The wait that
// follows a timeout (letting the CTA's own copies land) keeps kWaitPolls.
__device__ __forceinline__ uint32_t first_wait_polls(const KArgs& a) { return (a.short_wait & 1) ? 0u : kWaitPolls; }

// Index checks of the bounds-checked build (compiled with FS_DEBUG_BOUNDS):
// an access of `bytes` at p outside [base, base + extent) sets
// FS_FLAG_BOUNDS and is skipped instead of reaching memory.  In the normal
// build this is `true` and costs nothing.
__device__ __forceinline__ bool in_bounds(const KArgs& a, const void* p, long long bytes, const void* base,
                                          long long extent) {
#ifdef FS_DEBUG_BOUNDS
  const long long off = (long long)((const char*)p - (const char*)base);
  if (off < 0 || off + bytes > extent) {
    atomicOr(a.flag, FS_FLAG_BOUNDS);
    return false;
  }
#endif
  return true;
}
__device__ __forceinline__ bool spec_ok(const KArgs& a, const void* p, long long bytes) {
  return in_bounds(a, p, bytes, a.spec, a.spec_bytes);
}
__device__ __forceinline__ bool real_ok(const KArgs& a, const void* p, long long bytes) {
  return in_bounds(a, p, bytes, a.real, a.real_bytes);
}

template <typename T>
__device__ __forceinline__ bool finite_val(T x) {
  return isfinite(x);
}

// ---------------------------------------------------------------------------
// Row pass.  Lines along x.  A CTA holds R rows and four warps; warp w
// works on fields w, w + 4, ... of all R rows (TPL = L / E threads per line,
// 32 / TPL lines per warp), so the independent transforms of the fields run
// in parallel:
//   load    one thread issues bulk-async copies of every field's R rows
//           (packed half spectra, or real pairs in mode 1) into the slots;
//   phase 1 warp f < nf: inverse x transform of field f (modes 0 and 2);
//   phase 2 all threads: pointwise stage, df/dc into slot nf, g_i over eta_i;
//   phase 3 warp o <= nf: forward x transform of slot o to global memory.
// Slot contents use the natural layout (element i at i) except during the
// FFT exchanges, which use a padded layout (element i at pad16(i) or pad32(i),
// see RowCfg).
// mode 0: step, previous state in spec slots 0..nf-1 (y-inverted spectra)
// mode 1: step, previous state in the real fields
// mode 2: inverse only: spec slots 0..nf-1 -> real fields
// mode 3: free-energy diagnostic: real fields in, sum of f_chem into acc[0],
//         2 x^(phi) of every field into spec slots 0..nf-1
// Outputs of a step: slots 1..p = 2 x^(g_i), slot nf = 2 x^(df/dc) (x-spectra
// scaled by 2; the factor is folded into the k-space scale); slot 0 = x^(c)
// / nx, the scaling in which the column pass leaves the updated c, so in
// mode 0 slot 0 is left as loaded (c^ is carried from step to step, as in
// Algorithm 1) and only mode 1 writes it.
// ---------------------------------------------------------------------------
// W: the wide variant, E = 32 values per thread (radix 32 then 16 for
// L = 512: two passes, one exchange), used by plans for FP32 rows of 1024
// with the plan's second pass table (KArgs::tw_row_w).
template <typename T, int NX, bool W = false>
struct RowCfg {
  static constexpr bool F64 = sizeof(T) == 8;
  static constexpr int L = NX / 2;
  static constexpr int E = W ? 32 : row_E(L, F64);
  static constexpr int TPL = L / E;
  static constexpr int R = 32 / TPL;                       // rows per CTA
  // Exchange layout: pad16 when a warp holds several lines (R > 1), which
  // with the pitch below makes the radix-16 writes and the stride-TPL
  // accesses of 8-byte elements bank-conflict free; a warp holding one line
  // keeps pad32 (fewer index instructions, conflicts already rare).
  static constexpr bool P16 = R > 1;
  // Slot pitch (complex): room for the layout, even so that every slot is
  // 16-byte aligned for the bulk copies, and with R > 1 = TPL (mod 16), so
  // the lines of a half-warp start on different banks.
  static constexpr int PL0 = ((P16 ? padded16_len(L) : padded_len(L)) + 1) & ~1;
  static constexpr int PL = (R > 1 && TPL >= 2) ? PL0 + ((TPL - PL0 % 16) + 16) % 16 : PL0;
  static constexpr int THREADS = 4 * 32;                // four warps; warp w takes fields w, w + 4, ...
  // 32 values per thread (wide rows, rows of 2048) need about twice the
  // registers of 16
  static constexpr int MIN_BLOCKS = F64 ? (E >= 32 ? 2 : 3) : (E >= 32 ? 4 : 7);
  static constexpr int BAR_BYTES = 128;
  static constexpr int TWS = pass_table_size(L, E);  // twiddle entries (complex)
  static constexpr int TW_BYTES = ((TWS * (int)sizeof(cplx<T>)) + 127) & ~127;
};

// Shared memory of one row-pass CTA (bytes).
template <typename T, int NX, bool W = false>
constexpr size_t row_smem_bytes(int nf) {
  using Cfg = RowCfg<T, NX, W>;
  return Cfg::BAR_BYTES + Cfg::TW_BYTES + (size_t)(nf + 1) * Cfg::R * Cfg::PL * sizeof(cplx<T>);
}

// Issues the bulk-async copies of row block rb (every field's rows) into
// the input slots `in` ([nf][R][PL]), completion on `bar`.  One thread only.
template <typename T, int NX, bool W = false>
__device__ __forceinline__ void row_issue(const KArgs& a, long long rb, cplx<T>* in, uint64_t* bar) {
  using C = cplx<T>;
  using Cfg = RowCfg<T, NX, W>;
  constexpr int L = Cfg::L, R = Cfg::R, PL = Cfg::PL;
  const int nf = a.nf;
  const int Reff = a.lines < R ? (int)a.lines : R;
  const long long row0 = rb * Reff;
  const uint32_t bytes = (uint32_t)(L * sizeof(C));
  const bool from_real = (a.mode == 1 || a.mode == 3);
  const C* realc = reinterpret_cast<const C*>(a.real);
  const C* spec = reinterpret_cast<const C*>(a.spec);
  mbar_arrive_expect_tx(bar, bytes * Reff * nf);
  for (int f = 0; f < nf; ++f) {
    // the R rows of field f are contiguous in global memory
    // 3D carry: c's x spectrum sits in slot nf (see the 3D passes)
    const int sl = (f == 0 && a.carry3) ? nf : f;
    const C* src = from_real ? realc + f * (a.npts / 2) + row0 * L : spec + sl * a.slot_stride + row0 * L;
    for (int r = 0; r < Reff; ++r) {
      // a skipped copy leaves the barrier short of bytes: the pass then
      // reports a timeout besides the index error
      if (from_real ? real_ok(a, src + r * L, bytes) : spec_ok(a, src + r * L, bytes))
        bulk_g2s(in + (f * R + r) * PL, src + r * L, bytes, bar);
    }
  }
}

// Pointwise stage of the half-length row pass with p = P known at compile
// time: U independent points per iteration -- all loads, then the
// arithmetic, then the stores (points past the end repeat idx).  in: the
// field slots [nf][R][PL] (eta_i replaced by g_i), scr: df/dc [R][PL].
template <typename T, int P, int U, int R, int PL, int L>
__device__ __forceinline__ void row_pointwise_fixed(const Pointwise<T>& pw, cplx<T>* in, cplx<T>* scr, int n,
                                                    bool& bad) {
  using C = cplx<T>;
  for (int idx = threadIdx.x; idx < n; idx += U * blockDim.x) {
    int off[U];
    C c[U], e[U][P], fc[U], gv[U][P];
    T chk = T(0);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int j = idx + u * (int)blockDim.x < n ? idx + u * (int)blockDim.x : idx;
      off[u] = (j / L) * PL + j % L;
      c[u] = in[off[u]];
#pragma unroll
      for (int i = 0; i < P; ++i) e[u][i] = in[(1 + i) * R * PL + off[u]];
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      C h = vsplat<C>(T(0)), S2 = vsplat<C>(T(0));
#pragma unroll
      for (int i = 0; i < P; ++i) {
        h = cadd(h, pw.hpoly2(e[u][i]));
        S2 = vfma(e[u][i], e[u][i], S2);
      }
      fc[u] = pw.fc2(c[u], h);
      chk += fc[u].x + fc[u].y;  // non-finite whenever any input is (see the runtime loop)
#pragma unroll
      for (int i = 0; i < P; ++i) gv[u][i] = pw.g2(c[u], e[u][i], S2);
    }
    bad |= !finite_val(chk);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      scr[off[u]] = fc[u];
#pragma unroll
      for (int i = 0; i < P; ++i) in[(1 + i) * R * PL + off[u]] = gv[u][i];
    }
  }
}

// Compute part of one row-pass work item (row block rb) once its rows have
// landed: input slots `in` ([nf][R][PL], fields in natural layout), scratch
// slot `scr` ([R][PL], df/dc), pass tables `twr` in shared memory.
template <typename T, int NX, bool W = false>
__device__ __forceinline__ void row_compute(const KArgs& a, long long rb, cplx<T>* in, cplx<T>* scr,
                                            const cplx<T>* twr) {
  using C = cplx<T>;
  using Cfg = RowCfg<T, NX, W>;
  constexpr int L = Cfg::L, E = Cfg::E, TPL = Cfg::TPL, R = Cfg::R, PL = Cfg::PL;
  const int nf = a.nf;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane / TPL, t = lane % TPL;  // row within the CTA, thread within the line
  const int Reff = a.lines < R ? (int)a.lines : R;  // rows this CTA really holds
  const bool active = g < Reff;
  const long long row0 = rb * Reff;
  const long long row = row0 + g;
  const C* __restrict__ twh = reinterpret_cast<const C*>(a.tw_half);
  C* spec = reinterpret_cast<C*>(a.spec);
  C* realc = reinterpret_cast<C*>(a.real);  // real row as complex pairs
  const long long half_stride = a.npts / 2;  // complex pairs per real field
  auto wsync = []() { __syncwarp(); };
  auto slot = [in, scr, nf](int f, int r) { return f < nf ? in + (f * R + r) * PL : scr + r * PL; };
  // Twiddles of the real <-> half-length complex step, W_k = exp(-2 pi i k / (2L))
  // for k = t + TPL m: W_t (one table entry) times the exact constant
  // exp(-2 pi i m / (2E)) when 2E <= 32, else the table entry of k.
  const C wt = __ldg(&twh[t]);
  auto wk = [wt, twh, t](int m) {
    if constexpr (2 * E <= 32) return twiddle_small<-1>(wt, m, 2 * E);
    else return __ldg(&twh[t + TPL * m]);
  };

  // Both transform phases share one FFT call site (small instruction
  // footprint); the inverse is computed as conj(FFT(conj(.))).
  //   phase 1 (ph = 0): warp f < nf, inverse x transform of field f (modes 0, 2)
  //   phase 2         : pointwise stage, all threads
  //   phase 3 (ph = 1): warp o <= nf, forward x transform of slot o
  bool bad = false;
  const int nw = blockDim.x >> 5;
  for (int ph = 0; ph < 2; ++ph) {
    const bool inv = (ph == 0);
    // transforms of this phase: inverse of the nf fields (modes 0, 2), forward
    // of c, g_1..g_p, df/dc (nf slots only for the diagnostic, mode 3); warp
    // w takes items w, w + nw, ...
    const int items = inv ? ((a.mode == 0 || a.mode == 2) ? nf : 0) : (a.mode == 3 ? nf : nf + 1);
    // c's x spectrum is carried (Algorithm 1 keeps c^ from the previous
    // step): in mode 0 the loaded slot 0 already holds it, so the forward
    // phase starts at slot 1
    const int f0 = (!inv && a.mode == 0) ? 1 : 0;
    for (int f = f0 + w; f < items; f += nw) {
      C* s = slot(f, g);
      auto st = [s](int i, C v) { s[Cfg::P16 ? pad16(i) : pad32(i)] = v; };
      auto ld = [s](int i) { return s[Cfg::P16 ? pad16(i) : pad32(i)]; };
      C v[E];
      if (inv) {
        // half-length complex sequence of the real row from its packed half
        // spectrum (conjugated for the conj-FFT-conj inverse)
#pragma unroll
        for (int m = 0; m < E; ++m) {
          const int k = t + TPL * m;
          const C pk = s[k];
          C z;
          if (k == 0) {
            z = mk<C>(pk.x + pk.y, pk.x - pk.y);
          } else {
            const C pm = cconj(s[L - k]);
            const C A = cadd(pk, pm), B = csub(pk, pm);
            z = cadd(A, mul_i<1>(mul_tw<1>(B, wk(m))));
          }
          v[m] = cconj(z);
        }
      } else {
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = s[t + TPL * m];
      }
      line_fft<L, E, -1>(v, t, twr, st, ld, wsync);
      if (inv) {
        if (a.mode == 2) {
          C* dst = realc + f * half_stride + row * L;
          if (active) {
#pragma unroll
            for (int m = 0; m < E; ++m)
              if (real_ok(a, &dst[t + TPL * m], sizeof(C))) dst[t + TPL * m] = cconj(v[m]);
          }
        } else {
          wsync();
#pragma unroll
          for (int m = 0; m < E; ++m) s[t + TPL * m] = cconj(v[m]);
        }
      } else {
        // packed half spectrum, scaled by 2, straight to global memory
        const bool c_carried = (f == 0 && a.mode == 1);
        const T c_scale = T(0.5) / T(a.nx);
        wsync();
#pragma unroll
        for (int m = 0; m < E; ++m) s[t + TPL * m] = v[m];
        wsync();
        C* P = spec + f * a.slot_stride + row * L;
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
              out = cadd(A, mul_i<-1>(cmul(B, wk(m))));
            }
            // mode 1, c: store in the carried scaling, x spectrum / nx (what
            // the column pass leaves behind), 2 x^ / (2 nx) (exact: power of 2)
            if (c_carried) out = cscale(out, c_scale);
            if (spec_ok(a, &P[k], sizeof(C))) P[k] = out;
          }
        }
      }
    }
    if (!inv) break;
    if (a.mode == 2) return;
    __syncthreads();

    // phase 2: pointwise derivative stage, all threads over all R * L pairs
    if (a.mode == 3) {
      // chemical free energy f_chem = rho2 (c-ca)^2 (1-h) + rho2 (cb-c)^2 h + w g
      const Coef<T>& k = coef<T>(a);
      const T rho2 = k.two_rho2 * T(0.5), cb = k.ca + k.dcab, alpha = k.four_alpha * T(0.25);
      const Pointwise<T> pw(a);
      const int p = nf - 1;
      double sum = 0.0;
      for (int idx = threadIdx.x; idx < Reff * L; idx += blockDim.x) {
        const int r = idx / L, i0 = idx % L;
        const C c = slot(0, r)[i0];
        T part[2];
        const T cc[2] = {c.x, c.y};
#pragma unroll
        for (int h2 = 0; h2 < 2; ++h2) {
          T h = T(0), g = T(0), s2 = T(0), s4 = T(0);
          for (int i = 0; i < p; ++i) {
            const C e2 = slot(1 + i, r)[i0];
            const T e = h2 ? e2.y : e2.x;
            h += pw.hpoly(e);
            g += e * e * (T(1) - e) * (T(1) - e);
            s2 += e * e;
            s4 += e * e * e * e;
          }
          g += alpha * (s2 * s2 - s4);
          const T da = cc[h2] - k.ca, db = cb - cc[h2];
          part[h2] = rho2 * da * da * (T(1) - h) + rho2 * db * db * h + k.w * g;
        }
        sum += (double)part[0] + (double)part[1];
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o);
      if (lane == 0) atomicAdd(&a.acc[0], sum);
    } else if (sizeof(T) == 4 && nf >= 2) {
      // FP32: p known at compile time for every supported field count (FP64
      // is bound by its arithmetic pipe and keeps the loop below)
      const Pointwise<T> pw(a);
      switch (nf) {
        case 2: row_pointwise_fixed<T, 1, 4, R, PL, L>(pw, in, scr, Reff * L, bad); break;
        case 3: row_pointwise_fixed<T, 2, 4, R, PL, L>(pw, in, scr, Reff * L, bad); break;
        case 4: row_pointwise_fixed<T, 3, 2, R, PL, L>(pw, in, scr, Reff * L, bad); break;
        default: row_pointwise_fixed<T, 4, 2, R, PL, L>(pw, in, scr, Reff * L, bad); break;
      }
    } else {
      const Pointwise<T> pw(a);
      const int p = nf - 1;
      for (int idx = threadIdx.x; idx < Reff * L; idx += blockDim.x) {
        const int r = idx / L, i0 = idx % L;
        // two grid points per pair, lane-wise
        const C c = slot(0, r)[i0];
        C h = vsplat<C>(T(0)), S2 = vsplat<C>(T(0));
        for (int i = 0; i < p; ++i) {
          const C e = slot(1 + i, r)[i0];
          h = cadd(h, pw.hpoly2(e));
          S2 = vfma(e, e, S2);
        }
        // df/dc is non-finite whenever c or any eta_i is: h is a polynomial
        // in the eta_i and enters with the factor c_beta - c_alpha, and
        // 0 * inf is NaN, so one test of its two lanes' sum covers all inputs
        const C fc = pw.fc2(c, h);
        bad |= !finite_val(fc.x + fc.y);
        slot(nf, r)[i0] = fc;
        for (int i = 0; i < p; ++i) {
          const C e = slot(1 + i, r)[i0];
          slot(1 + i, r)[i0] = pw.g2(c, e, S2);
        }
      }
    }
    __syncthreads();
  }
  if (bad) atomicOr(a.flag, FS_FLAG_NONFINITE);
}

// One row-pass work item with its own table copy and load (ensemble kernel):
// `bar` is an initialised mbarrier whose next phase has parity `parity`.
// Returns false if a bounded wait gave up (the caller must stop).
template <typename T, int NX, bool W = false>
__device__ __forceinline__ bool row_body(const KArgs& a, long long rb, unsigned char* smem_raw, uint64_t* bar,
                                         uint32_t parity) {
  using C = cplx<T>;
  using Cfg = RowCfg<T, NX, W>;
  C* twr = reinterpret_cast<C*>(smem_raw + Cfg::BAR_BYTES);
  C* slots = reinterpret_cast<C*>(smem_raw + Cfg::BAR_BYTES + Cfg::TW_BYTES);  // [(nf + 1) * R][PL]
  copy_to_smem(twr, reinterpret_cast<const C*>(W ? a.tw_row_w : a.tw_row), Cfg::TWS);
  __syncthreads();
  // everything above only touched constant tables; the spectra are the
  // previous pass's output
  griddep_wait();
  if (threadIdx.x == 0) {
    // the ensemble kernel reuses the slots: order the previous item's
    // generic accesses (ended by the CTA barrier above) before the copies
    fence_proxy_async_smem();
    row_issue<T, NX, W>(a, rb, slots, bar);
  }
  griddep_launch_dependents();
  if (!mbar_wait_bounded(bar, parity, first_wait_polls(a))) {
    if (threadIdx.x == 0) atomicOr(a.flag, FS_FLAG_TIMEOUT);
    mbar_wait_bounded(bar, parity, kWaitPolls);  // let the copies land before exiting
    return false;
  }
  row_compute<T, NX, W>(a, rb, slots, slots + a.nf * Cfg::R * Cfg::PL, twr);
  return true;
}


// NW warps per CTA: 4 (fields w, w + 4, ...), or 5 for five fields in FP32
// at 32 values per thread, one warp per field, so no warp carries two
// transforms per phase (register budget of three CTAs per SM).
template <typename T, int NX, bool W = false, int NW = 4>
__global__ void __launch_bounds__(32 * NW, NW == 4 ? RowCfg<T, NX, W>::MIN_BLOCKS
                                                   : (RowCfg<T, NX, W>::E >= 32 ? 3 : 5))
    fs_row_kernel(KArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  row_body<T, NX, W>(a, blockIdx.x, smem_raw, bar, 0);
}

// ---------------------------------------------------------------------------
// Column pass (2D step).  Lines along y of the packed x-spectra; one CTA per
// tile of tk adjacent kx columns (TPL threads per column) and per field group
// (blockIdx.y = 0: c with df/dc, g >= 1: eta_g).  The tiles [NY][tk] of the
// group's slots arrive by TMA (3D tensor map over [slot][y][kx]); then
// forward y transforms, k-space update and inverse y transforms, stored in
// place.  Each loaded tile is also the exchange buffer of its own transform;
// for the c group the transformed df/dc stays in tile 0 for the update.
// ---------------------------------------------------------------------------
template <typename T, int NY>
struct ColCfg {
  static constexpr bool F64 = sizeof(T) == 8;
  static constexpr int E = col_E(NY, F64);
  static constexpr int TPL = NY / E;
  static constexpr int TK = col_tk(NY, F64);
  static constexpr int THREADS = TPL * TK;
  static constexpr int BH = NY < 256 ? NY : 256;  // TMA box height (rows)
  static constexpr int BAR_BYTES = 128;
  static constexpr int TWS = pass_table_size(NY, E);  // twiddle entries (complex)
  static constexpr int TW_BYTES = ((TWS * (int)sizeof(cplx<T>)) + 127) & ~127;
  static constexpr int K2_BYTES = ((NY * (int)sizeof(T)) + 127) & ~127;
  static constexpr int LOGE = ilog2(E);
  // tile rows: NY natural rows plus room for the padded exchange layout
  static constexpr int TROWS = (NY + NY / E + 1 + 15) & ~15;
  static constexpr int HEAD = BAR_BYTES + TW_BYTES + K2_BYTES;
};

template <typename T>
struct KUpdate {
  T Mdt, Mdtkc, Ldtke, scale, Mdt_c, scale_c;
  __device__ explicit KUpdate(const KArgs& a) {
    const Coef<T>& k = coef<T>(a);
    Mdt = k.Mdt;
    Mdtkc = k.Mdtkc;
    Ldtke = k.Ldtke;
    scale = k.scale;
    // c arrives in the carried scaling (x spectrum / nx, see the row pass)
    // while df/dc arrives as 2 x^: fold the factor 2 nx into the
    // coefficients (powers of two, so exact).  3D steady state: c comes
    // straight from the previous z step, without the y inverse / forward
    // round trip that would multiply it by ny: fold that in too.
    const T q = (a.carry3 && a.mode == 0) ? T(2 * a.nx_full) * T(a.ny) : T(2 * a.nx_full);
    Mdt_c = Mdt / q;
    scale_c = scale * q;
  }
  // c^' = (c^ - M dt K2 f^) / (1 + M dt kappa_c K2^2), times the 1/(2N) scale;
  // zc = c^ / (2 nx) in the units of zf
  template <typename C>
  __device__ __forceinline__ C c(C zc, C zf, T k2) const {
    T d = quot(scale_c, T(1) + Mdtkc * k2 * k2);
    T b = Mdt_c * k2;
    return cscale(vfma(zf, vsplat<C>(-b), zc), d);
  }
  // eta^' = g^ / (1 + L dt kappa_eta K2), times the 1/(2N) scale
  template <typename C>
  __device__ __forceinline__ C eta(C zg, T k2) const {
    return cscale(zg, quot(scale, T(1) + Ldtke * k2));
  }
  // x / y for the denominators above (y >= 1): FP32 through the fast
  // reciprocal (2 ulp, as the warp-per-column pass), FP64 rounded
  __device__ __forceinline__ static T quot(T x, T y) {
    if constexpr (sizeof(T) == 4) return __fdividef(x, y);
    else return x / y;
  }
};

// Shared memory of one column-pass CTA (bytes) for a tile of tk columns
// (plus the split DFT matrix of the tensor-core stage).
template <typename T, int NY, int TCM = TC_NONE>
constexpr size_t col_smem_bytes(int tk) {
  return ColCfg<T, NY>::HEAD + 2 * (size_t)ColCfg<T, NY>::TROWS * tk * sizeof(cplx<T>) + (TCM ? 8192 : 0) +
         (TCM == TC_TF32 ? tc5_extra_bytes(ColCfg<T, NY>::TPL * tk) : 0);
}

// One column-pass work item: kx tile bx, field group g of the simulation
// described by `a`, tiles loaded through the tensor map `tmap`.  TCM != 0:
// the first radix-16 pass of each forward transform runs on tensor cores.
template <typename T, int NY, int TCM = TC_NONE>
__device__ __forceinline__ bool col_body(const KArgs& a, const CUtensorMap* tmap, int bx, int g,
                                         unsigned char* smem_raw, uint64_t* bar, uint32_t parity) {
  using C = cplx<T>;
  using Cfg = ColCfg<T, NY>;
  constexpr int E = Cfg::E, TPL = Cfg::TPL, BH = Cfg::BH;
  constexpr int TROWS = Cfg::TROWS, LOGE = Cfg::LOGE;
  C* twc = reinterpret_cast<C*>(smem_raw + Cfg::BAR_BYTES);
  T* k2yt = reinterpret_cast<T*>(smem_raw + Cfg::BAR_BYTES + Cfg::TW_BYTES);
  C* tiles = reinterpret_cast<C*>(smem_raw + Cfg::HEAD);
  const int tk = blockDim.x / TPL;  // columns in this CTA (<= TK)
  const int j = threadIdx.x % tk, t = threadIdx.x / tk;
  const int Lh = a.nx / 2;
  const int kx0 = bx * tk;
  const int kx = kx0 + j;
  const int nf = a.nf;
  const int nin = (g == 0) ? 2 : 1;
  const T* __restrict__ k2xt = reinterpret_cast<const T*>(a.k2x);

  if (threadIdx.x == 0) {
    griddep_wait();  // the tiles are the previous pass's output
    // the ensemble kernel reuses the tiles: order the previous item's generic
    // accesses (ended by the caller's CTA barrier) before the TMA writes
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(bar, (uint32_t)(nin * NY * tk * sizeof(C)));
    const int cx = kx0 * (int)(sizeof(C) / 8);  // innermost coordinate in 8-byte units
    for (int i = 0; i < nin; ++i) {
      const int slot = (g == 0) ? (i == 0 ? nf : 0) : g;
      for (int y0 = 0; y0 < NY; y0 += BH) tma_load_3d(tiles + (i * TROWS + y0) * tk, tmap, cx, y0, slot, bar);
    }
  }
  copy_to_smem(twc, reinterpret_cast<const C*>(a.tw_col), Cfg::TWS);
  for (int i = threadIdx.x; i < NY; i += blockDim.x) k2yt[i] = reinterpret_cast<const T*>(a.k2y)[i];
  griddep_wait();
  griddep_launch_dependents();
  __syncthreads();
  if (!mbar_wait_bounded(bar, parity, first_wait_polls(a))) {
    if (threadIdx.x == 0) atomicOr(a.flag, FS_FLAG_TIMEOUT);
    mbar_wait_bounded(bar, parity, kWaitPolls);
    return false;
  }

  const KUpdate<T> up(a);
  const bool special = (a.kx_base + kx0 == 0);  // CTA holding the packed DC/Nyquist column
  const T kx2 = k2xt[kx];
  const T kxn2 = k2xt[Lh];  // Nyquist column
  C* stash = tiles;  // c group: transformed df/dc, natural layout [ky][j]
  C* xt = tiles + (nin - 1) * TROWS * tk;  // exchange tile of the updated field
  auto sync = []() { __syncthreads(); };
  float* bsm = reinterpret_cast<float*>(tiles + 2 * TROWS * tk);
  if constexpr (TCM != TC_NONE) {
    static_assert(sizeof(T) == 4 && E == 16, "tensor-core stage: FP32, radix 16");
    tc_load_b(bsm, reinterpret_cast<const float*>(a.tc_b));
    __syncthreads();
  }

  // All transforms share one call site (small instruction footprint):
  // iterations 0..nin-1 are the forward transforms of the loaded tiles (the
  // c group takes df/dc, kept in tile 0, then c), the last iteration is the
  // inverse transform, computed as conj(FFT(conj(v))).
  C v[E];
  for (int it = 0; it <= nin; ++it) {
    const bool inv = (it == nin);
    C* tl = (inv ? xt : tiles + it * TROWS * tk) + j;
    auto st = [tl, tk](int q, C x) { tl[(q + (q >> LOGE)) * tk] = x; };
    auto ld = [tl, tk](int q) { return tl[(q + (q >> LOGE)) * tk]; };
    if constexpr (TCM != TC_NONE) {
      if (!inv) {
        // first radix-16 pass on tensor cores, the rest on CUDA cores
        tc_first_pass16<NY, TCM>(reinterpret_cast<float2*>(tiles + it * TROWS * tk), tk, bsm, a.flag);
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = ld(t + TPL * m);
        stockham<NY, E, 16, -1>(v, t, twc, st, ld, sync);
      } else {
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = cconj(v[m]);
        line_fft<NY, E, -1>(v, t, twc, st, ld, sync);
      }
    } else {
      if (!inv) {
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = tl[(t + TPL * m) * tk];
      } else {
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = cconj(v[m]);
      }
      line_fft<NY, E, -1>(v, t, twc, st, ld, sync);
    }
    if (inv) break;
    if (it + 1 < nin) {
      sync();
#pragma unroll
      for (int m = 0; m < E; ++m) tl[(t + TPL * m) * tk] = v[m];
      continue;
    }
    // k-space update of the last forward transform
    if (special) {
      // Separate the packed column Z = A + i B (A: kx = 0, B: kx = nx/2, both
      // Hermitian in ky) through shared memory, update both, repack.
      sync();
      if (j == 0) {
#pragma unroll
        for (int m = 0; m < E; ++m) xt[(t + TPL * m) * tk] = v[m];
      }
      sync();
    }
    if (special && j == 0) {
#pragma unroll
      for (int m = 0; m < E; ++m) {
        const int ky = t + TPL * m, kq = (NY - ky) & (NY - 1);
        const T ky2 = k2yt[ky];
        const C pz = cconj(xt[kq * tk]);
        const C A = cscale(cadd(v[m], pz), T(0.5)), B = cscale(mul_i<-1>(csub(v[m], pz)), T(0.5));
        C An, Bn;
        if (g == 0) {
          const C zf = stash[ky * tk], pf = cconj(stash[kq * tk]);
          const C Af = cscale(cadd(zf, pf), T(0.5)), Bf = cscale(mul_i<-1>(csub(zf, pf)), T(0.5));
          An = up.c(A, Af, kx2 + ky2);
          Bn = up.c(B, Bf, kxn2 + ky2);
          if (ky == 0 && a.csum) An = mk<C>((T)(*a.csum * a.inv_npts), T(0));
        } else {
          An = up.eta(A, kx2 + ky2);
          Bn = up.eta(B, kxn2 + ky2);
        }
        v[m] = cadd(An, mul_i<1>(Bn));
      }
    } else if (g == 0) {
#pragma unroll
      for (int m = 0; m < E; ++m) {
        const int ky = t + TPL * m;
        v[m] = up.c(v[m], stash[ky * tk + j], kx2 + k2yt[ky]);
      }
    } else {
#pragma unroll
      for (int m = 0; m < E; ++m) v[m] = up.eta(v[m], kx2 + k2yt[t + TPL * m]);
    }
  }
  C* S = reinterpret_cast<C*>(a.spec) + kx + (long long)(g == 0 ? 0 : g) * a.slot_stride;
#pragma unroll
  for (int m = 0; m < E; ++m)
    if (spec_ok(a, &S[(long long)(t + TPL * m) * Lh], sizeof(C))) S[(long long)(t + TPL * m) * Lh] = cconj(v[m]);
  return true;
}

// Free-energy diagnostic, gradient terms (Eq. fe through Parseval): forward
// y transform of slot g (= field g) and the sum of w(kx) K2 |phi^|^2 over the
// tile, w = 2 for 0 < kx < nx/2 (the conjugate half is not stored), 1 for
// the separated kx = 0 and kx = nx/2 columns; FP64 atomics into acc[1 + g].
template <typename T, int NY>
__global__ void __launch_bounds__(ColCfg<T, NY>::THREADS, 2)
    fs_energy_col_kernel(KArgs a, const __grid_constant__ CUtensorMap tmap) {
  using C = cplx<T>;
  using Cfg = ColCfg<T, NY>;
  constexpr int E = Cfg::E, TPL = Cfg::TPL, BH = Cfg::BH, LOGE = Cfg::LOGE;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  C* twc = reinterpret_cast<C*>(smem_raw + Cfg::BAR_BYTES);
  T* k2yt = reinterpret_cast<T*>(smem_raw + Cfg::BAR_BYTES + Cfg::TW_BYTES);
  C* tile = reinterpret_cast<C*>(smem_raw + Cfg::HEAD);
  const int tk = blockDim.x / TPL;
  const int j = threadIdx.x % tk, t = threadIdx.x / tk;
  const int Lh = a.nx / 2;
  const int kx0 = blockIdx.x * tk, kx = kx0 + j, g = blockIdx.y;
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_arrive_expect_tx(bar, (uint32_t)(NY * tk * sizeof(C)));
    const int cx = kx0 * (int)(sizeof(C) / 8);
    for (int y0 = 0; y0 < NY; y0 += BH) tma_load_3d(tile + y0 * tk, &tmap, cx, y0, g, bar);
  }
  copy_to_smem(twc, reinterpret_cast<const C*>(a.tw_col), Cfg::TWS);
  for (int i = threadIdx.x; i < NY; i += blockDim.x) k2yt[i] = reinterpret_cast<const T*>(a.k2y)[i];
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
    line_fft<NY, E, -1>(v, t, twc, st, ld, []() { __syncthreads(); });
  }
  const T* k2xt = reinterpret_cast<const T*>(a.k2x);
  const double kx2 = (double)k2xt[kx], kxn2 = (double)k2xt[Lh];
  double sum = 0.0;
  const bool special = (kx0 == 0);
  if (special) {
    __syncthreads();
    if (j == 0) {
#pragma unroll
      for (int m = 0; m < E; ++m) tile[(t + TPL * m) * tk] = v[m];
    }
    __syncthreads();
  }
#pragma unroll
  for (int m = 0; m < E; ++m) {
    const int ky = t + TPL * m;
    const double ky2 = (double)k2yt[ky];
    if (special && j == 0) {
      const C pz = cconj(tile[((NY - ky) & (NY - 1)) * tk]);
      const C A = cscale(cadd(v[m], pz), T(0.5)), B = cscale(mul_i<-1>(csub(v[m], pz)), T(0.5));
      sum += (kx2 + ky2) * ((double)A.x * A.x + (double)A.y * A.y);
      sum += (kxn2 + ky2) * ((double)B.x * B.x + (double)B.y * B.y);
    } else {
      sum += 2.0 * (kx2 + ky2) * ((double)v[m].x * v[m].x + (double)v[m].y * v[m].y);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(&a.acc[1 + g], sum);
}

template <typename T, int NY, int TCM = TC_NONE>
__global__ void __launch_bounds__(ColCfg<T, NY>::THREADS, 2)
    fs_col_kernel(KArgs a, const __grid_constant__ CUtensorMap tmap) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  col_body<T, NY, TCM>(a, &tmap, blockIdx.x, blockIdx.y, smem_raw, bar, 0);
}

}  // namespace fs
