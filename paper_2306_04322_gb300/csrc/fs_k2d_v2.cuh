// Warp-per-line forms of the row and column passes (FP32, lines of 256, 512
// or 1024 points).  Every line transform is held by one warp, E = L / 32
// values per thread (radix 32 x 32 at L = 1024: one exchange), so the FFT
// exchanges synchronise the warp only; CTA-wide barriers remain only where
// fields meet (the pointwise stage of the row pass) and named 64-thread
// barriers where the column pass hands df/dc^ to the c update.
//
// Row pass, pair form.  Grid rows a and b of one field are transformed as
// the single complex line z = a + i b of length nx:
//   inverse: Z[k] = X_a[k] + i X_b[k] over all nx bins, built from the two
//            packed half spectra with X[nx - k] = conj X[k]; the inverse DFT
//            of Z gives a + i b at once;
//   forward: Z = DFT(g_a + i g_b), then 2 X_a[k] = Z[k] + conj Z[nx - k]
//            and 2 X_b[k] = -i (Z[k] - conj Z[nx - k]) (k <= nx/2), which is
//            the factor-2 scaling the column pass expects.
// The two rows' values sit in the two lanes of a float2 in real space, so the
// pointwise derivative stage (Section 2.1 definitions) runs lane-wise on the
// pair.  Modes as the row pass of fs_kernels.cuh: 0 step from spectra, 1 step
// from real fields, 2 inverse only (mode 3, the free-energy diagnostic, keeps
// the half-length kernel).
//
// Column pass, warp per column.  A CTA holds two adjacent kx columns (16-byte
// TMA rows) of one field group -- {df/dc, c} or a pair of eta -- one warp per
// (slot, column).  All warps transform forward; the df/dc warps publish their
// result for the c warps of the same column, and the c and eta warps apply
// the k-space update (Eqs. A-C_discrete_fft_c, A-C_discrete_fft_eta) and
// transform back.
#pragma once

#include "fs_k2d_impl.cuh"

namespace fs {

// Line FFT of the warp-per-line kernels: the looped two-pass form at 1024
// points (E = 32), the pass sequence of line_fft otherwise.
template <int L, int E, int DIR, typename C, class Store, class Load, class Sync>
__device__ __forceinline__ void warp_line_fft(C (&v)[E], int t, const C* __restrict__ twp, Store st, Load ld,
                                              Sync sync) {
  if constexpr (L == E * E) line_fft_sq<E, DIR>(v, t, twp, st, ld, sync);
  else line_fft<L, E, DIR>(v, t, twp, st, ld, sync);
}

// G warps per line (1, or 2 to double the warps in flight when lines are
// few); a line's TPL = 32 G threads hold E = NX / TPL values each.
template <int NX, int G = 1>
struct Row2Cfg {
  static constexpr int TPL = 32 * G;                          // threads per line
  static constexpr int E = NX / TPL;                          // values per thread
  static constexpr int H = NX / 2;                            // packed bins per row
  static constexpr int PL = (padded_len(NX) + 1) & ~1;        // complex per field area (16-byte multiple)
  static constexpr int TWS = pass_table_size(NX, E);
  static constexpr int TW_BYTES = ((TWS * 8) + 127) & ~127;
  static constexpr int BAR_BYTES = 128;
  static constexpr int MAX_THREADS = TPL * 5;                 // one line per field, nf <= 5
};

template <int NX, int G = 1>
constexpr size_t row2_smem_bytes(int nf) {
  return Row2Cfg<NX, G>::BAR_BYTES + Row2Cfg<NX, G>::TW_BYTES + (size_t)(nf + 1) * Row2Cfg<NX, G>::PL * 8;
}

// Synchronisation of the threads of one line: the warp itself, or the two
// warps of a line through named barrier 1 + line (64 threads).
template <int G>
struct LineSync {
  int id;
  __device__ __forceinline__ void operator()() const {
    if constexpr (G == 1) __syncwarp();
    else bar_sync(id, 32 * G);
  }
};

// Pointwise stage of the pair-form row pass (Section 2.1 derivatives, lane-
// wise on the two rows of a pair) with p = P known at compile time: four
// independent points per iteration -- all loads, then the arithmetic, then
// the stores (points past the row repeat point n).  areas: [nf + 1][PL],
// c, eta_i (replaced by g_i), df/dc in area nf.  df/dc is non-finite
// whenever c or any eta_i is (see the row pass of fs_kernels.cuh): one test
// of the sum of its lanes covers all inputs.
template <int P, int NX, int PL>
__device__ __forceinline__ void row2_pointwise_fixed(const Pointwise<float>& pw, float2* areas, bool& bad) {
  using C = float2;
  constexpr int PE = P > 0 ? P : 1, U = 4;
  for (int n = threadIdx.x; n < NX; n += U * blockDim.x) {
    int k[U];
    C c[U], e[U][PE], fc[U], g[U][PE];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      k[u] = n + u * (int)blockDim.x < NX ? n + u * (int)blockDim.x : n;
      c[u] = areas[k[u]];
#pragma unroll
      for (int i = 0; i < P; ++i) e[u][i] = areas[(1 + i) * PL + k[u]];
    }
    float chk = 0.f;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      C h = vsplat<C>(0.f), S2 = vsplat<C>(0.f);
#pragma unroll
      for (int i = 0; i < P; ++i) {
        h = cadd(h, pw.hpoly2(e[u][i]));
        S2 = vfma(e[u][i], e[u][i], S2);
      }
      fc[u] = pw.fc2(c[u], h);
      chk += fc[u].x + fc[u].y;
#pragma unroll
      for (int i = 0; i < P; ++i) g[u][i] = pw.g2(c[u], e[u][i], S2);
    }
    bad |= !finite_val(chk);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      areas[(P + 1) * PL + k[u]] = fc[u];
#pragma unroll
      for (int i = 0; i < P; ++i) areas[(1 + i) * PL + k[u]] = g[u][i];
    }
  }
}

// One row pair (rows 2 pair and 2 pair + 1) of the simulation `a`, one warp
// per field (blockDim = 32 nf).  Field areas [nf + 1][PL] (the last one holds
// df/dc): staging of the bulk copies, then the warp's exchange buffer (pad32
// layout), then the pair values in natural order for the pointwise stage.
// `bar` is an initialised mbarrier whose next phase has parity `parity`; the
// ensemble kernel calls this once per work item.  Returns false if a bounded
// wait gave up.  PC >= 0: the caller guarantees nf = PC + 1, and the
// pointwise stage is compiled for that p alone (the 96-thread kernel, whose
// nf is 3: a kernel holding the code for every p measured slower there).
template <int NX, int G = 1, int PC = -1>
__device__ __forceinline__ bool row2_body(const KArgs& a, long long pair, unsigned char* smem_raw, uint64_t* bar,
                                          uint32_t parity) {
  using C = float2;
  using Cfg = Row2Cfg<NX, G>;
  constexpr int E = Cfg::E, H = Cfg::H, PL = Cfg::PL, TPL = Cfg::TPL;
  C* tw = reinterpret_cast<C*>(smem_raw + Cfg::BAR_BYTES);
  C* areas = reinterpret_cast<C*>(smem_raw + Cfg::BAR_BYTES + Cfg::TW_BYTES);
  const int nf = a.nf;
  const int line = (threadIdx.x >> 5) / G, t = threadIdx.x % TPL;  // line of this thread, thread within it
  const int nw = blockDim.x / TPL;  // lines per CTA = nf
  const long long row0 = 2LL * pair;  // row a; row b = row0 + 1
  const LineSync<G> lsync{1 + line};
  const bool from_real = (a.mode == 1);

  if (threadIdx.x == 0) {
    // the ensemble kernel reuses the areas: order the previous item's generic
    // accesses (ended by the caller's CTA barrier) before the bulk writes
    fence_proxy_async_smem();
    // both rows of a field are contiguous: NX complex (packed) or 2 NX reals
    const uint32_t bytes = (uint32_t)(NX * sizeof(C));
    const uint32_t tbytes = (uint32_t)(Cfg::TWS * sizeof(C));
    mbar_arrive_expect_tx(bar, tbytes + bytes * nf);
    // the constant pass table first, overlapping the previous grid's tail
    bulk_g2s(tw, G == 1 ? a.tw_row2 : a.tw_row2w, tbytes, bar);
    griddep_wait();  // the spectra are the previous pass's output
    const C* spec = reinterpret_cast<const C*>(a.spec);
    const float* real = reinterpret_cast<const float*>(a.real);
    for (int f = 0; f < nf; ++f) {
      // 3D carry: c's x spectrum sits in slot nf
      const int sl = (f == 0 && a.carry3) ? nf : f;
      const void* src = from_real ? (const void*)(real + f * a.npts + row0 * NX)
                                  : (const void*)(spec + sl * a.slot_stride + row0 * H);
      if (from_real ? real_ok(a, src, bytes) : spec_ok(a, src, bytes)) bulk_g2s(areas + f * PL, src, bytes, bar);
    }
  }
  griddep_launch_dependents();
  if (!mbar_wait_bounded(bar, parity, first_wait_polls(a))) {
    if (threadIdx.x == 0) atomicOr(a.flag, FS_FLAG_TIMEOUT);
    mbar_wait_bounded(bar, parity, kWaitPolls);  // let the copies land before exiting
    return false;
  }

  C* spec = reinterpret_cast<C*>(a.spec);
  float* real = reinterpret_cast<float*>(a.real);
  bool bad = false;
  // Both transform phases share one FFT call site (the inverse is computed as
  // conj(FFT(conj(.)))): ph 0 inverse of the nf fields (modes 0, 2; mode 1
  // only interleaves the real rows), ph 1 forward of g_1..g_p and df/dc (and
  // of c in mode 1).
  for (int ph = 0; ph < 2; ++ph) {
    const bool inv = (ph == 0);
    const int f0 = inv ? 0 : (from_real ? 0 : 1);
    const int items = nf + 1 - f0 - (inv ? 1 : 0);  // inverse: fields 0..nf-1; forward: f0..nf
    for (int i = line; i < items; i += nw) {
      const int f = f0 + i;
      C* s = areas + f * PL;
      auto st = [s](int q, C x) { s[pad32(q)] = x; };
      auto ld = [s](int q) { return s[pad32(q)]; };
      C v[E];
      if (inv) {
        if (from_real) {
          // rows a and b (NX reals each) -> pairs (a[n], b[n]) in natural order
          const float* r = reinterpret_cast<const float*>(s);
          float xa[E], xb[E];
#pragma unroll
          for (int m = 0; m < E; ++m) {
            xa[m] = r[t + TPL * m];
            xb[m] = r[NX + t + TPL * m];
          }
          lsync();
#pragma unroll
          for (int m = 0; m < E; ++m) s[t + TPL * m] = make_float2(xa[m], xb[m]);
          continue;
        }
        // conj(Z), Z[k] = X_a[k] + i X_b[k]; staging: row a bins [0, H), row b [H, 2H);
        // bin 0 of a packed row holds (X[0], X[H]), both real
#pragma unroll
        for (int m = 0; m < E; ++m) {
          const int k = t + TPL * m;
          C z;
          if (k < H) {
            const C xa = s[k], xb = s[H + k];
            z = (k == 0) ? make_float2(xa.x, xb.x) : make_float2(xa.x - xb.y, xa.y + xb.x);
          } else if (k == H) {
            z = make_float2(s[0].y, s[H].y);
          } else {
            const C xa = s[NX - k], xb = s[H + NX - k];
            z = make_float2(xa.x + xb.y, xb.x - xa.y);
          }
          v[m] = cconj(z);
        }
        lsync();  // the staging area becomes the exchange buffer
      } else {
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = s[t + TPL * m];  // z = g_a + i g_b, natural order
      }
      warp_line_fft<NX, E, -1>(v, t, tw, st, ld, lsync);
      if (inv) {
        // a + i b = conj(v)
        if (a.mode == 2) {
          float* ra = real + f * a.npts + row0 * NX;
#pragma unroll
          for (int m = 0; m < E; ++m) {
            const int n = t + TPL * m;
            if (real_ok(a, &ra[n], 4)) ra[n] = v[m].x;
            if (real_ok(a, &ra[NX + n], 4)) ra[NX + n] = -v[m].y;
          }
        } else {
          lsync();
#pragma unroll
          for (int m = 0; m < E; ++m) s[t + TPL * m] = cconj(v[m]);
        }
      } else {
        // separate the two rows' spectra; Z[nx - k] through shared memory
        lsync();
#pragma unroll
        for (int m = 0; m < E; ++m) s[t + TPL * m] = v[m];
        lsync();
        const bool c_carried = (f == 0);  // mode 1: c stored as x spectrum / nx
        const float cs = c_carried ? 0.5f / (float)NX : 1.0f;
        C* Pa = spec + f * a.slot_stride + row0 * H;
        C* Pb = Pa + H;
#pragma unroll
        for (int m = 0; m < E / 2; ++m) {
          const int k = t + TPL * m;
          const C zk = v[m];
          C pa, pb;
          if (k == 0) {
            const C zh = s[H];
            pa = make_float2(2.f * zk.x, 2.f * zh.x);
            pb = make_float2(2.f * zk.y, 2.f * zh.y);
          } else {
            const C zm = s[NX - k];
            pa = make_float2(zk.x + zm.x, zk.y - zm.y);
            pb = make_float2(zk.y + zm.y, zm.x - zk.x);
          }
          if (c_carried) {
            pa = cscale(pa, cs);
            pb = cscale(pb, cs);
          }
          if (spec_ok(a, &Pa[k], sizeof(C))) Pa[k] = pa;
          if (spec_ok(a, &Pb[k], sizeof(C))) Pb[k] = pb;
        }
      }
    }
    if (!inv) break;
    if (a.mode == 2) return true;
    __syncthreads();

    // pointwise stage: pairs (row a, row b) of every field, lane-wise
    const Pointwise<float> pw(a);
    if constexpr (PC >= 0) {
      row2_pointwise_fixed<PC, NX, PL>(pw, areas, bad);
    } else {
      switch (nf) {  // p known at compile time for every supported field count
        case 1: row2_pointwise_fixed<0, NX, PL>(pw, areas, bad); break;
        case 2: row2_pointwise_fixed<1, NX, PL>(pw, areas, bad); break;
        case 3: row2_pointwise_fixed<2, NX, PL>(pw, areas, bad); break;
        case 4: row2_pointwise_fixed<3, NX, PL>(pw, areas, bad); break;
        case 5: row2_pointwise_fixed<4, NX, PL>(pw, areas, bad); break;
        default: break;
      }
    }
    __syncthreads();
  }
  if (bad) atomicOr(a.flag, FS_FLAG_NONFINITE);
  return true;
}

// NW: the most warps per line group the instantiation takes (nf <= NW).
// With one warp per line and nf = 3 the register budget is that of four
// 96-thread CTAs per SM (170 per thread; a pass of 1024 rows stays one
// wave), which leaves the compiler room to schedule the values of each
// thread; otherwise three 160-thread CTAs (136).  Measured (L2 flushed
// before each step, p = 2): 512^2 step 17.1 us against 19.1 us, 1024^2
// unchanged; with nf = 2 the 1024^2 step lost 4 %, so only nf = 3 takes it.
template <int NX, int G, int NW>
__global__ void __launch_bounds__(32 * G * NW, (G == 1 && NW <= 3) ? 4 : (G == 1 ? 3 : 2))
    fs_row2_kernel(KArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  row2_body<NX, G, (G == 1 && NW == 3) ? 2 : -1>(a, blockIdx.x, smem_raw, bar, 0);
}

template <int NY, int G = 1>
struct Col2Cfg {
  static constexpr int TPL = 32 * G;                          // threads per line
  static constexpr int E = NY / TPL;
  static constexpr int TK = 2;                                // kx columns per CTA
  static constexpr int BH = NY < 256 ? NY : 256;              // TMA box height (rows)
  static constexpr int PL = (padded_len(NY) + 1) & ~1;        // complex per compact column area
  // slot region: the [NY][TK] tile as loaded, then TK compact areas, then the
  // [NY][TK] tile again for the TMA store; a multiple of 16 complex so every
  // region starts on 128 bytes (TMA)
  static constexpr int SLOT = (((NY * TK > TK * PL) ? NY * TK : TK * PL) + 15) & ~15;
  static constexpr int TWS = pass_table_size(NY, E);
  static constexpr int TW_BYTES = ((TWS * 8) + 127) & ~127;
  static constexpr int K2_BYTES = ((NY * 4) + 127) & ~127;
  static constexpr int HEAD = 128 + TW_BYTES + K2_BYTES;
  // CTAs per SM the registers are budgeted for: 128 per thread at 32 values
  static constexpr int MIN_BLOCKS = E >= 32 ? 4 / G : (G == 1 ? 4 : 3);
};

// Shared memory of one CTA: the head and two slot regions.
template <int NY, int G = 1>
constexpr size_t col2_smem_bytes() {
  return Col2Cfg<NY, G>::HEAD + (size_t)2 * Col2Cfg<NY, G>::SLOT * 8;
}

// The packed kx = 0 / Nyquist column of the first CTA: y holds this warp's
// forward transform Z = A + i B (A the kx = 0 column, B the kx = nx/2 one,
// both Hermitian in ky), fz the same packing of df/dc^ (c only).  A and B are
// separated through Z(ky) and conj Z(ny - ky), updated with their own K2
// (Eqs. A-C_discrete_fft_c / _eta) and repacked, in place.  The update maps
// each pair {ky, ny - ky} onto itself (A(ny - ky) = conj A(ky), the same for
// B, and the update is real-linear with the same K2 at ky and ny - ky), so a
// thread owns both entries of its pairs and no other thread touches them.  A
// few warps of the grid run this, so it stays out of line and rolled.
template <int NY, int TPL>
__device__ __noinline__ void col2_packed_update(float2* __restrict__ y, const float2* __restrict__ fz, int t,
                                                bool isC, KUpdate<float> up, float kx2, float kxn2,
                                                const float* __restrict__ k2yt, const double* csum,
                                                double inv_npts) {
  using C = float2;
#pragma unroll 1
  for (int m = 0; m <= NY / (2 * TPL); ++m) {
    const int ky = t + TPL * m;  // pairs ky = 0 .. ny/2
    if (ky > NY / 2) break;
    const int kq = (NY - ky) & (NY - 1);
    const float ky2 = k2yt[ky];
    const C z = y[ky], pz = cconj(y[kq]);
    const C A = cscale(cadd(z, pz), 0.5f), B = cscale(mul_i<-1>(csub(z, pz)), 0.5f);
    C An, Bn;
    if (isC) {
      const C zf = fz[ky], pf = cconj(fz[kq]);
      const C Af = cscale(cadd(zf, pf), 0.5f), Bf = cscale(mul_i<-1>(csub(zf, pf)), 0.5f);
      An = up.c(A, Af, kx2 + ky2);
      Bn = up.c(B, Bf, kxn2 + ky2);
      if (ky == 0 && csum) An = make_float2((float)(*csum * inv_npts), 0.f);
    } else {
      An = up.eta(A, kx2 + ky2);
      Bn = up.eta(B, kxn2 + ky2);
    }
    y[ky] = cadd(An, mul_i<1>(Bn));
    if (kq != ky) y[kq] = cadd(cconj(An), mul_i<1>(cconj(Bn)));
  }
}

// CTA: two adjacent kx columns (kx0 = 2 blockIdx.x, kx0 + 1) of one field
// group (blockIdx.y): group 0 holds df/dc and c, group g >= 1 eta_{2g-1} and
// eta_{2g}; warp (region r, column j), r = 0, 1.  Four warps per CTA and
// 1 + ceil(p / 2) groups, so every CTA carries about two transforms per warp
// and several CTAs share an SM.  The tiles come in by TMA, every warp copies
// its column to registers, then its region becomes two compact per-column
// areas (exchange buffers, pad32 layout).  After the update and the inverse
// transform the results go back to the interleaved tile layout and out by
// TMA, so the global writes are whole 16-byte rows instead of one 8-byte
// value per lane and row.
// Column pair `cpair`, field group `group` of the simulation `a` (blockDim =
// 128); `bar` as for row2_body.  Returns false if a bounded wait gave up.
template <int NY, int G = 1>
__device__ __forceinline__ bool col2_body(const KArgs& a, const CUtensorMap* tmap, int cpair, int group,
                                          unsigned char* smem_raw, uint64_t* bar, uint32_t parity) {
  using C = float2;
  using Cfg = Col2Cfg<NY, G>;
  constexpr int E = Cfg::E, BH = Cfg::BH, PL = Cfg::PL, SLOT = Cfg::SLOT, TPL = Cfg::TPL;
  C* tw = reinterpret_cast<C*>(smem_raw + 128);
  float* k2yt = reinterpret_cast<float*>(smem_raw + 128 + Cfg::TW_BYTES);
  C* regions = reinterpret_cast<C*>(smem_raw + Cfg::HEAD);
  const int nf = a.nf, p = nf - 1;
  const int line = (threadIdx.x >> 5) / G, t = threadIdx.x % TPL;  // line (region, column), thread in it
  const int j = line & 1, r = line >> 1;
  const int nreg = group == 0 ? 2 : (p - 2 * (group - 1) >= 2 ? 2 : 1);
  // slot of region q of this group: group 0: df/dc (nf), c (0); else eta_{2g-1+q}
  auto slot_of = [nf, group](int q) { return group == 0 ? (q == 0 ? nf : 0) : 2 * group - 1 + q; };
  const bool isF = (group == 0 && r == 0), isC = (group == 0 && r == 1);
  const int kx0 = cpair * Cfg::TK, kx = kx0 + j;
  const int H = a.nx / 2;

  if (r >= nreg) return true;  // the second region of a last group with one eta
  if (threadIdx.x == 0) {
    // the ensemble kernel reuses the regions: order the previous item's
    // generic accesses (ended by the caller's CTA barrier) before the TMA writes
    fence_proxy_async_smem();
    const uint32_t tbytes = (uint32_t)(Cfg::TWS * sizeof(C)), kbytes = (uint32_t)(NY * sizeof(float));
    mbar_arrive_expect_tx(bar, tbytes + kbytes + (uint32_t)(nreg * NY * Cfg::TK * sizeof(C)));
    // the constant tables first, overlapping the previous grid's tail
    bulk_g2s(tw, G == 1 ? a.tw_col2 : a.tw_col2w, tbytes, bar);
    bulk_g2s(k2yt, a.k2y, kbytes, bar);
    griddep_wait();  // the tiles are the previous pass's output
    for (int q = 0; q < nreg; ++q)
      // innermost coordinate kx0 (8-byte units) is even: 16-byte aligned
      for (int y0 = 0; y0 < NY; y0 += BH)
        tma_load_3d(regions + q * SLOT + y0 * Cfg::TK, tmap, kx0, y0, slot_of(q), bar);
  }
  const float* __restrict__ k2xt = reinterpret_cast<const float*>(a.k2x);
  const float kx2 = k2xt[kx];
  griddep_launch_dependents();
  if (!mbar_wait_bounded(bar, parity, first_wait_polls(a))) {
    if (threadIdx.x == 0) atomicOr(a.flag, FS_FLAG_TIMEOUT);
    mbar_wait_bounded(bar, parity, kWaitPolls);
    return false;
  }

  C* reg = regions + r * SLOT;
  C v[E];
#pragma unroll
  for (int m = 0; m < E; ++m) v[m] = reg[(t + TPL * m) * Cfg::TK + j];
  // named barriers with compile-time ids: 1, 2 per region (its two column
  // lines), 3, 4 per column (df/dc^ handed to the c line), 5.. per line (its
  // G warps, G = 2)
  auto region_sync = [r]() { if (r == 0) bar_sync(1, 64 * G); else bar_sync(2, 64 * G); };
  const LineSync<G> lsync{5 + line};
  // both columns of this region have left the tile: it becomes two compact areas
  region_sync();
  C* xa = reg + j * PL;
  auto st = [xa](int q, C x) { xa[pad32(q)] = x; };
  auto ld = [xa](int q) { return xa[pad32(q)]; };
  const KUpdate<float> up(a);
  const bool special = (a.kx_base + kx0 == 0 && j == 0);  // the packed kx = 0 / Nyquist column
  const C* fz = regions + j * PL;             // df/dc^ of this column (region 0 of group 0)

  // One FFT call site: it 0 forward (all warps), it 1 inverse (c, eta) as
  // conj(FFT(conj(.))).
  for (int it = 0; it < 2; ++it) {
    warp_line_fft<NY, E, -1>(v, t, tw, st, ld, lsync);
    if (it == 1) break;
    if (isF) {
      // df/dc^: natural layout for the c warp of this column
      lsync();
#pragma unroll
      for (int m = 0; m < E; ++m) xa[t + TPL * m] = v[m];
      if (j == 0) bar_arrive(3, 64 * G); else bar_arrive(4, 64 * G);
      return true;
    }
    if (isC) {
      if (j == 0) bar_sync(3, 64 * G); else bar_sync(4, 64 * G);
    }
    if (special) {
      lsync();
#pragma unroll
      for (int m = 0; m < E; ++m) xa[t + TPL * m] = v[m];
      lsync();
      col2_packed_update<NY, TPL>(xa, fz, t, isC, up, kx2, k2xt[H], k2yt, a.csum, a.inv_npts);
      lsync();
#pragma unroll
      for (int m = 0; m < E; ++m) v[m] = cconj(xa[t + TPL * m]);
    } else {
      // c^' = (c^ - M dt K2 f^) / (1 + M dt kappa_c K2^2), eta^' = g^ / (1 + L dt kappa_eta K2)
      // (scales folded as in KUpdate); one code path for both, the quotient by
      // the fast reciprocal (the denominators are >= 1)
      const float num = isC ? up.scale_c : up.scale;
      const float qk = isC ? up.Mdtkc : up.Ldtke;
      const float bk = isC ? up.Mdt_c : 0.f;
#pragma unroll
      for (int m = 0; m < E; ++m) {
        const int ky = t + TPL * m;
        const float k2 = kx2 + k2yt[ky];
        const float d = __fdividef(num, fmaf(qk, isC ? k2 * k2 : k2, 1.f));
        const C zf = isC ? fz[ky] : make_float2(0.f, 0.f);
        v[m] = cconj(cscale(vfma(zf, vsplat<C>(-bk * k2), v[m]), d));
      }
    }
  }
  // results (conj of the last transform) back to the interleaved tile layout
  // of this region, then out by TMA: c -> slot 0, eta_i -> slot i
  region_sync();  // both columns are done with their compact areas
#pragma unroll
  for (int m = 0; m < E; ++m) reg[(t + TPL * m) * Cfg::TK + j] = cconj(v[m]);
  fence_proxy_async_smem();
  region_sync();
  if (j == 0 && t == 0) {  // one thread of the region's column-0 line
    for (int y0 = 0; y0 < NY; y0 += BH) tma_store_3d(tmap, kx0, y0, slot_of(r), reg + y0 * Cfg::TK);
    bulk_commit();
    bulk_wait_all();  // the tile is read (and written out) before the region is reused or the CTA exits
  }
  return true;
}

template <int NY, int G>
__global__ void __launch_bounds__(128 * G, Col2Cfg<NY, G>::MIN_BLOCKS)
    fs_col2_kernel(KArgs a, const __grid_constant__ CUtensorMap tmap) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  col2_body<NY, G>(a, &tmap, blockIdx.x, blockIdx.y, smem_raw, bar, 0);
}

// Launchers: cudaErrorNotSupported when this form does not cover the
// request (the caller falls back to the half-length / tile kernels).
template <int NX, int G, int NW>
cudaError_t row2_launch_nw(const KArgs& a, cudaStream_t s) {
  static unsigned done = 0;
  cudaError_t e = allow_big_smem(fs_row2_kernel<NX, G, NW>, &done);
  if (e != cudaSuccess) return e;
  return launch_pdl(fs_row2_kernel<NX, G, NW>, dim3((unsigned)(a.lines / 2)), dim3((unsigned)(32 * G * a.nf)),
                    row2_smem_bytes<NX, G>(a.nf), s, a);
}
template <int NX, int G>
cudaError_t row2_launch_n(const KArgs& a, cudaStream_t s) {
  if (G == 1 && a.nf == 3) return row2_launch_nw<NX, G, 3>(a, s);
  return row2_launch_nw<NX, G, 5>(a, s);
}

template <int NY, int G>
cudaError_t col2_launch_n(const KArgs& a, const CUtensorMap& tm, cudaStream_t s) {
  static unsigned done = 0;
  cudaError_t e = allow_big_smem(fs_col2_kernel<NY, G>, &done);
  if (e != cudaSuccess) return e;
  const unsigned groups = (unsigned)(1 + (a.nf - 1 + 1) / 2);  // {df/dc, c} and the eta pairs
  return launch_pdl(fs_col2_kernel<NY, G>, dim3((unsigned)(a.nx / 2 / Col2Cfg<NY, G>::TK), groups),
                    dim3((unsigned)(128 * G)), col2_smem_bytes<NY, G>(), s, a, tm);
}

}  // namespace fs
