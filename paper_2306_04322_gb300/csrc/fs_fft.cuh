// Shared-memory / register FFT engine for the semi-implicit Fourier-spectral
// step.  Everything here is generic over the real type T (float or double)
// and the line length L (a power of two).
//
// Distribution convention used by every kernel: a line of length L is held
// by TPL = L / E threads, each with E complex values in registers, thread t
// holding elements t + TPL * m for m = 0..E-1 ("stride-TPL" order).  The FFT
// is a Stockham autosort decomposition L = R_1 R_2 ... with every radix
// R = min(E, remaining); each pass does E/R radix-R butterflies per thread in
// registers.  Between passes the data goes through shared memory once; the
// last pass leaves its results in the same stride-TPL order, so a line FFT of
// P passes costs P - 1 shared-memory round trips and no global traffic.
//
// Twiddles: per-pass tables built on the host in long double, laid out
// [pass][r][j] (r = 0..R-1, j = 0..NS-1; entries r = 0 are 1), so the lanes
// of a warp, which hold consecutive j, read consecutive entries.  Kernels
// copy the tables to shared memory first.  No device trigonometry is used.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fs {

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
// a * conj(b)
template <typename C> __device__ __forceinline__ C cmulc(C a, C b) {
  return mk<C>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename C> __device__ __forceinline__ C cconj(C a) { return mk<C>(a.x, -a.y); }
template <typename C> __device__ __forceinline__ C cscale(C a, decltype(C::x) s) { return mk<C>(a.x * s, a.y * s); }
// FP32 complex add / subtract / scale as packed two-lane FP32 instructions
// (f32x2, sm_100 and later): one instruction per complex operation.
__device__ __forceinline__ uint64_t pk2(float2 a) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
  return r;
}
__device__ __forceinline__ float2 upk2(uint64_t r) {
  float2 a;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
  return a;
}
template <> __device__ __forceinline__ float2 cadd<float2>(float2 a, float2 b) {
  uint64_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk2(a)), "l"(pk2(b)));
  return upk2(d);
}
template <> __device__ __forceinline__ float2 csub<float2>(float2 a, float2 b) {
  uint64_t d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk2(a)), "l"(pk2(b)));
  return upk2(d);
}
template <> __device__ __forceinline__ float2 cscale<float2>(float2 a, float s) {
  uint64_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk2(a)), "l"(pk2(make_float2(s, s))));
  return upk2(d);
}

// Lane-wise arithmetic on two independent reals held in one complex-type
// pair (the row pass keeps two adjacent grid points per pair).  FP32: packed
// f32x2 instructions; FP64: two scalar lanes.
template <typename C> __device__ __forceinline__ C vsplat(decltype(C::x) s) { return mk<C>(s, s); }
template <typename C> __device__ __forceinline__ C vmul(C a, C b) { return mk<C>(a.x * b.x, a.y * b.y); }
template <typename C> __device__ __forceinline__ C vfma(C a, C b, C c) {
  return mk<C>(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}
template <> __device__ __forceinline__ float2 vmul<float2>(float2 a, float2 b) {
  uint64_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk2(a)), "l"(pk2(b)));
  return upk2(d);
}
template <> __device__ __forceinline__ float2 vfma<float2>(float2 a, float2 b, float2 c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(pk2(a)), "l"(pk2(b)), "l"(pk2(c)));
  return upk2(d);
}

// multiply by +i (DIR = +1) or -i (DIR = -1)
template <int DIR, typename C> __device__ __forceinline__ C mul_i(C a) {
  return DIR > 0 ? mk<C>(-a.y, a.x) : mk<C>(a.y, -a.x);
}
// multiply by exp(DIR i theta) given w = exp(-i theta) (forward tables)
template <int DIR, typename C> __device__ __forceinline__ C mul_tw(C a, C w) {
  return DIR < 0 ? cmul(a, w) : cmulc(a, w);
}

constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n / 2); }
constexpr int imin(int a, int b) { return a < b ? a : b; }
constexpr int imax(int a, int b) { return a > b ? a : b; }
__host__ __device__ constexpr int bitrev(int v, int bits) {
  int r = 0;
  for (int b = 0; b < bits; ++b) r = (r << 1) | ((v >> b) & 1);
  return r;
}

// cos(2 pi j / 32) for j = 0..8, decimal expansions of the exact values.
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

// Multiply a by exp(DIR * 2 pi i * k / len) for compile-time-known k / len
// (after unrolling), len <= 32.  Trivial roots avoid multiplies.
template <int DIR, typename C>
__device__ __forceinline__ C twiddle_small(C a, int k, int len) {
  using T = decltype(C::x);
  int j = (k * 32 / len) & 31;  // angle in units of 2 pi / 32
  if (j == 0) return a;
  if (j == 8) return mul_i<DIR>(a);
  if (j == 16) return mk<C>(-a.x, -a.y);
  if (j == 24) return mul_i<-DIR>(a);
  int q = j / 8, r = j % 8;
  T c = (T)cos32(r), s = (T)sin32(r);
  T cr, sr;
  if (q == 0) { cr = c; sr = s; }
  else if (q == 1) { cr = -s; sr = c; }
  else if (q == 2) { cr = -c; sr = -s; }
  else { cr = s; sr = -c; }
  if (r == 4) {  // (+-1 +- i)/sqrt(2): adds, then one scaling
    T h = (T)cos32(4);
    T sx = (cr > 0 ? 1 : -1), sy = (DIR * sr > 0 ? 1 : -1);
    return mk<C>((sx * a.x - sy * a.y) * h, (sy * a.x + sx * a.y) * h);
  }
  return cmul(a, mk<C>(cr, DIR * sr));
}

// In-register DFT of length R (R <= 32) on a[0], a[S], ..., a[(R-1) S],
// natural order in and out, X[k] = sum_n x[n] exp(DIR 2 pi i n k / R).
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
#pragma unroll
    for (int i = 0; i < R; i += 4) {
      C x0 = t[i], x1 = t[i + 1], x2 = t[i + 2], x3 = t[i + 3];
      C a0 = cadd(x0, x1), a1 = csub(x0, x1), b0 = cadd(x2, x3), b1 = mul_i<DIR>(csub(x2, x3));
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

// ---- pass structure (identical on host and device) -------------------------
template <int L, int E, int NS>
struct PassRadix {
  static constexpr int R = imin(E, L / NS);
};
// offset (in complex entries) of the table of the pass starting at NS
template <int L, int E, int NS>
constexpr int pass_table_offset() {
  int off = 0;
  for (int ns = 1; ns < NS;) {
    int r = imin(E, L / ns);
    if (ns > 1) off += ns * r;
    ns *= r;
  }
  return off;
}
// total table size of a line FFT of length L with E per thread
__host__ __device__ constexpr int pass_table_size(int L, int E) {
  int off = 0;
  for (int ns = 1; ns < L;) {
    int r = E < L / ns ? E : L / ns;
    if (ns > 1) off += ns * r;
    ns *= r;
  }
  return off;
}

// One Stockham pass (and, recursively, the following ones).  On entry the
// thread holds pass inputs x[b + r L/R] for its butterflies b = t + TPL q in
// v[q + (E/R) r].  Not-last passes write outputs to shared memory through
// `st` and read the next pass's inputs back in stride-TPL order.
template <int L, int E, int NS, int DIR, typename C, class Store, class Load, class Sync>
__device__ __forceinline__ void stockham(C (&v)[E], int t, const C* __restrict__ twp, Store st, Load ld,
                                         Sync sync) {
  constexpr int TPL = L / E;
  constexpr int R = PassRadix<L, E, NS>::R;
  constexpr int Q = E / R;
  static_assert(E % R == 0, "radix must divide E");
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int b = t + TPL * q;
    if constexpr (NS > 1) {
      const int j = b & (NS - 1);
      const C* w = twp + pass_table_offset<L, E, NS>() + j;
#pragma unroll
      for (int r = 1; r < R; ++r) v[q + Q * r] = mul_tw<DIR>(v[q + Q * r], w[r * NS]);
    }
    reg_dft<R, DIR, Q>(&v[q]);
  }
  if constexpr (NS * R < L) {
    sync();
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int b = t + TPL * q;
      const int j = b & (NS - 1);
      const int base = (b - j) * R + j;
#pragma unroll
      for (int r = 0; r < R; ++r) st(base + r * NS, v[q + Q * r]);
    }
    sync();
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = ld(t + TPL * m);
    stockham<L, E, NS * R, DIR>(v, t, twp, st, ld, sync);
  }
}

// Full line FFT, X[k] = sum_n x[n] exp(DIR 2 pi i n k / L), unnormalised.
// twp: the pass tables of (L, E) (forward roots; the inverse conjugates),
// usually a shared-memory copy.
template <int L, int E, int DIR, typename C, class Store, class Load, class Sync>
__device__ __forceinline__ void line_fft(C (&v)[E], int t, const C* __restrict__ twp, Store st, Load ld,
                                         Sync sync) {
  static_assert(L % E == 0, "E must divide L");
  stockham<L, E, 1, DIR>(v, t, twp, st, ld, sync);
}

// Line FFT of length L = E * E held by one warp-sized group of E threads
// with E values each (E = 32: 1024 points, one warp): two radix-E passes and
// one exchange, as line_fft, but both passes run the same loop body, so the
// radix-E butterfly code is emitted once (half the instruction footprint of
// the unrolled pass sequence; the instruction cache is what the warp-per-line
// kernels run short of).  twp: the pass table of (L, E), entries [r][j] of
// the second pass (sub-length E).
template <int E, int DIR, typename C, class Store, class Load, class Sync>
__device__ __forceinline__ void line_fft_sq(C (&v)[E], int t, const C* __restrict__ twp, Store st, Load ld,
                                            Sync sync) {
#pragma unroll 1
  for (int pass = 0; pass < 2; ++pass) {
    if (pass == 1) {
#pragma unroll
      for (int r = 1; r < E; ++r) v[r] = mul_tw<DIR>(v[r], twp[r * E + t]);
    }
    reg_dft<E, DIR, 1>(v);
    if (pass == 0) {
      sync();
#pragma unroll
      for (int r = 0; r < E; ++r) st(t * E + r, v[r]);
      sync();
#pragma unroll
      for (int m = 0; m < E; ++m) v[m] = ld(t + E * m);
    }
  }
}

// Padded shared-memory indices: one spare slot every 32 (pad32) or 16
// (pad16) elements.  pad16 keeps the radix-16 butterfly writes (16
// consecutive elements per thread) and the stride-TPL reads of the row
// exchanges free of bank conflicts for 8-byte elements (each half-warp is
// served separately).
__device__ __forceinline__ int pad32(int i) { return i + (i >> 5); }
__device__ __forceinline__ int pad16(int i) { return i + (i >> 4); }
constexpr int padded_len(int L) { return L + L / 32 + 1; }
constexpr int padded16_len(int L) { return L + L / 16 + 1; }

// Cooperative copy of n complex values global -> shared (all threads).
template <typename C>
__device__ __forceinline__ void copy_to_smem(C* dst, const C* __restrict__ src, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = __ldg(&src[i]);
}

// ---- asynchronous bulk copies and mbarriers (inline PTX, sm_90+) ----------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Programmatic dependent launch (PTX griddepcontrol).  griddep_wait blocks
// until the grids this one depends on have completed and their memory
// operations are visible (it returns at once for a launch without such a
// dependency); griddep_launch_dependents lets the next grid of the stream be
// scheduled, so its prologue overlaps this grid's tail.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Orders this thread's earlier generic-proxy shared-memory accesses before
// its later async-proxy (bulk copy / TMA) accesses to shared memory.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// Global -> shared bulk copy (bytes a multiple of 16, both addresses 16-byte
// aligned), completion signalled on `bar`.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// 3D tiled TMA load (box given by the tensor map), completion on `bar`.
// The innermost coordinate c0 times the element size must be a multiple of
// 16 bytes.
__device__ __forceinline__ void tma_load_3d(void* dst, const void* tmap, int c0, int c1, int c2, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_u32(dst)),
      "l"(tmap), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
      : "memory");
}
// 4D tiled TMA load, completion on `bar` (same alignment rule as 3D).
__device__ __forceinline__ void tma_load_4d(void* dst, const void* tmap, int c0, int c1, int c2, int c3,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
      "%5}], [%6];" ::"r"(smem_u32(dst)),
      "l"(tmap), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
      : "memory");
}
// Named CTA barriers (PTX bar.sync / bar.arrive with an id and a thread
// count, a multiple of 32): bar_sync waits until `count` threads have
// arrived at barrier `id`; bar_arrive counts this warp in without waiting
// (producer side).  Shared-memory writes before the arrive are visible to
// the threads that pass the matching bar_sync.  Id 0 is __syncthreads().
__device__ __forceinline__ void bar_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_arrive(int id, int count) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// 3D tiled TMA store shared -> global (bulk-group completion); the innermost
// coordinate times the element size must be a multiple of 16 bytes and no
// coordinate may be negative.  The writing threads order their generic
// shared-memory stores before it with fence_proxy_async_smem() and a barrier.
__device__ __forceinline__ void tma_store_3d(const void* tmap, int c0, int c1, int c2, const void* src) {
  asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(tmap),
               "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(src))
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// Waits until every committed bulk group of this thread has completed (its
// global writes performed).
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Bounded wait: true when the phase completed, false after `limit` polls.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t limit) {
  for (uint32_t i = 0; i < limit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

}  // namespace fs
