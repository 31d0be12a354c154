// Shared-memory / register FFT engine for the semi-implicit Fourier-spectral
// step.  Everything here is generic over the real type T (float or double)
// and the line length L (a power of two).
//
// Distribution convention used by every kernel: a line of length L is held
// by TPL = L / E threads, each with E complex values in registers, thread t
// holding elements t + TPL * m for m = 0..E-1 ("stride-TPL" order).  The FFT
// is a Stockham autosort decomposition L = R_1 R_2 ... with every radix
// R <= E; each pass does E/R radix-R butterflies per thread in registers.
// Between passes the data goes through shared memory once; the last pass
// leaves its results in the same stride-TPL order, so a line FFT of P passes
// costs P - 1 shared-memory round trips and no global traffic.
//
// Twiddles come from one table tw[j] = exp(-2 pi i j / kTwN) built on the
// host in long double; a root w_M^e is tw[(e mod M) * kTwN / M].  No device
// trigonometry is used anywhere.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fs {

constexpr int kTwN = 4096;  // master twiddle table length (max axis 2048)

template <typename T> struct CplxOf;
template <> struct CplxOf<float> { using type = float2; };
template <> struct CplxOf<double> { using type = double2; };
template <typename T> using cplx = typename CplxOf<T>::type;

template <typename C> __device__ __forceinline__ C mk(decltype(C::x) a, decltype(C::x) b) {
  C r;
  r.x = a;
  r.y = b;
  return r;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return mk<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return mk<C>(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return mk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C> __device__ __forceinline__ C cconj(C a) { return mk<C>(a.x, -a.y); }
template <typename C> __device__ __forceinline__ C cscale(C a, decltype(C::x) s) { return mk<C>(a.x * s, a.y * s); }
// multiply by +i (DIR = +1) or -i (DIR = -1)
template <int DIR, typename C> __device__ __forceinline__ C mul_i(C a) {
  return DIR > 0 ? mk<C>(-a.y, a.x) : mk<C>(a.y, -a.x);
}

constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n / 2); }
constexpr int imin(int a, int b) { return a < b ? a : b; }
constexpr int imax(int a, int b) { return a > b ? a : b; }
__host__ __device__ constexpr int bitrev(int v, int bits) {
  int r = 0;
  for (int b = 0; b < bits; ++b) r = (r << 1) | ((v >> b) & 1);
  return r;
}

// cos / sin of 2 pi j / 32 for j = 0..8 (first octant and its end points),
// decimal expansions of the exact values.
__device__ __forceinline__ double cos32(int j) {
  switch (j) {
    case 0: return 1.0;
    case 1: return 0.98078528040323044912618223613424;
    case 2: return 0.92387953251128675612818318939679;
    case 3: return 0.83146961230254523707878837761791;
    case 4: return 0.70710678118654752440084436210485;
    case 5: return 0.55557023301960222474283081394853;
    case 6: return 0.38268343236508977172845998403040;
    case 7: return 0.19509032201612826784828486847702;
    default: return 0.0;
  }
}
__device__ __forceinline__ double sin32(int j) { return cos32(8 - j); }

// Multiply a by exp(DIR * 2 pi i * k / len) for a compile-time-known k/len
// (after unrolling), len <= 32.  Trivial roots avoid multiplies.
template <int DIR, typename C>
__device__ __forceinline__ C twiddle_small(C a, int k, int len) {
  using T = decltype(C::x);
  int j = (k * 32 / len) & 31;  // angle in units of 2 pi / 32
  if (j == 0) return a;
  if (j == 8) return mul_i<DIR>(a);
  if (j == 16) return mk<C>(-a.x, -a.y);
  if (j == 24) return mul_i<-DIR>(a);
  // reduce to first quadrant: exp(i theta), theta = 2 pi j / 32
  int q = j / 8, r = j % 8;
  T c = (T)cos32(r), s = (T)sin32(r);
  // rotate by q quarter turns
  T cr, sr;
  if (q == 0) { cr = c; sr = s; }
  else if (q == 1) { cr = -s; sr = c; }
  else if (q == 2) { cr = -c; sr = -s; }
  else { cr = s; sr = -c; }
  if (r == 4) {  // (+-1 +- i)/sqrt(2): 2 adds + 2 multiplies
    T h = (T)cos32(4);
    T sx = (cr > 0 ? 1 : -1), sy = (DIR * sr > 0 ? 1 : -1);
    // (a.x + i a.y)(sx + i sy) h
    return mk<C>((sx * a.x - sy * a.y) * h, (sy * a.x + sx * a.y) * h);
  }
  C w = mk<C>(cr, DIR * sr);
  return cmul(a, w);
}

// In-register DFT of length R (R <= 32) on a[0], a[S], ..., a[(R-1) S],
// natural order in and out, X[k] = sum_n x[n] exp(DIR 2 pi i n k / R).
// Radix-2 decimation in time with a compile-time bit reversal.
template <int R, int DIR, int S, typename C>
__device__ __forceinline__ void reg_dft(C* a) {
  if constexpr (R == 1) {
    return;
  } else if constexpr (R == 2) {
    C u = a[0], v = a[S];
    a[0] = cadd(u, v);
    a[S] = csub(u, v);
  } else if constexpr (R == 4) {
    C x0 = a[0], x1 = a[S], x2 = a[2 * S], x3 = a[3 * S];
    C s02 = cadd(x0, x2), d02 = csub(x0, x2), s13 = cadd(x1, x3), d13 = mul_i<DIR>(csub(x1, x3));
    a[0] = cadd(s02, s13);
    a[2 * S] = csub(s02, s13);
    a[S] = cadd(d02, d13);
    a[3 * S] = csub(d02, d13);
  } else {
    constexpr int B = ilog2(R);
    C t[R];
#pragma unroll
    for (int i = 0; i < R; ++i) t[i] = a[bitrev(i, B) * S];
    // first two levels as radix-4 butterflies on bit-reversed data
#pragma unroll
    for (int i = 0; i < R; i += 4) {
      C x0 = t[i], x1 = t[i + 1], x2 = t[i + 2], x3 = t[i + 3];
      // length-2 DFTs: (x0,x1), (x2,x3); then length-4 combine
      C a0 = cadd(x0, x1), a1 = csub(x0, x1), b0 = cadd(x2, x3), b1 = csub(x2, x3);
      b1 = mul_i<DIR>(b1);
      t[i] = cadd(a0, b0);
      t[i + 2] = csub(a0, b0);
      t[i + 1] = cadd(a1, b1);
      t[i + 3] = csub(a1, b1);
    }
#pragma unroll
    for (int len = 8; len <= R; len <<= 1) {
#pragma unroll
      for (int i = 0; i < R; i += len) {
#pragma unroll
        for (int k = 0; k < len / 2; ++k) {
          C u = t[i + k];
          C v = twiddle_small<DIR>(t[i + k + len / 2], k, len);
          t[i + k] = cadd(u, v);
          t[i + k + len / 2] = csub(u, v);
        }
      }
    }
#pragma unroll
    for (int i = 0; i < R; ++i) a[i * S] = t[i];
  }
}

// Twiddle exp(DIR * 2 pi i * e / M) from the master table.
template <int DIR, int M, typename C>
__device__ __forceinline__ C tw_root(const C* __restrict__ tw, int e) {
  C w = __ldg(&tw[(e & (M - 1)) * (kTwN / M)]);
  if (DIR > 0) w.y = -w.y;
  return w;
}

// Radix sequence: each pass uses R = min(E, remaining).
template <int L, int E, int NS>
struct PassRadix {
  static constexpr int R = imin(E, L / NS);
};

// One Stockham pass (and, recursively, the following ones).  On entry the
// thread holds pass inputs x[b + r L/R] for its butterflies b = t + TPL q in
// v[q + (E/R) r].  Not-last passes write outputs to shared memory through
// `st` and read the next pass's inputs back in stride-TPL order.
template <int L, int E, int NS, int DIR, typename C, class Store, class Load, class Sync>
__device__ __forceinline__ void stockham(C (&v)[E], int t, const C* __restrict__ tw, Store st, Load ld,
                                         Sync sync) {
  constexpr int TPL = L / E;
  constexpr int R = PassRadix<L, E, NS>::R;
  constexpr int Q = E / R;
  static_assert(E % R == 0, "radix must divide E");
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    int b = t + TPL * q;
    if constexpr (NS > 1) {
      int j = b & (NS - 1);
#pragma unroll
      for (int r = 1; r < R; ++r) v[q + Q * r] = cmul(v[q + Q * r], tw_root<DIR, NS * R>(tw, r * j));
    }
    reg_dft<R, DIR, Q>(&v[q]);
  }
  if constexpr (NS * R < L) {
    sync();
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      int b = t + TPL * q;
      int j = b & (NS - 1);
      int base = (b - j) * R + j;
#pragma unroll
      for (int r = 0; r < R; ++r) st(base + r * NS, v[q + Q * r]);
    }
    sync();
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = ld(t + TPL * m);
    stockham<L, E, NS * R, DIR>(v, t, tw, st, ld, sync);
  }
}

// Full line FFT, X[k] = sum_n x[n] exp(DIR 2 pi i n k / L), unnormalised.
template <int L, int E, int DIR, typename C, class Store, class Load, class Sync>
__device__ __forceinline__ void line_fft(C (&v)[E], int t, const C* __restrict__ tw, Store st, Load ld,
                                         Sync sync) {
  static_assert(L % E == 0, "E must divide L");
  stockham<L, E, 1, DIR>(v, t, tw, st, ld, sync);
}

// Padded shared-memory index: one spare slot every 32 elements keeps the
// stride-R butterfly writes and the stride-TPL reads free of bank conflicts.
__device__ __forceinline__ int pad32(int i) { return i + (i >> 5); }
constexpr int padded_len(int L) { return L + L / 32 + 1; }

}  // namespace fs
