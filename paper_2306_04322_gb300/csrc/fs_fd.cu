// Explicit finite-difference comparison scheme of Boccardo et al. (arXiv
// 2306.04322, Section 2.2): forward Euler in time, second-order centred
// 5-point Laplacian on a periodic 2D grid, three stages per step
//   (i)   mu    = df/dc - kappa_c lap(c)
//   (ii)  c'    = c + dt M lap(mu)
//   (iii) eta'_i = eta_i - dt L (df/deta_i - kappa_eta lap(eta_i))
// fused into one kernel: a CTA loads a tile with a two-point halo (periodic
// wrap instead of the paper's ghost layers), forms mu on the tile plus a
// one-point halo in shared memory, then updates its interior.
#include "fs_kernels.cuh"

namespace fs {

namespace {

constexpr int FD_TX = 32, FD_TY = 16;
constexpr int FD_WX = FD_TX + 4, FD_WY = FD_TY + 4;  // loaded tile (halo 2)
constexpr int FD_MX = FD_TX + 2, FD_MY = FD_TY + 2;  // mu region (halo 1)

template <typename T>
__global__ void __launch_bounds__(FD_TX* FD_TY) fs_fd_kernel(KArgs a, const T* __restrict__ in, T* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* tile = reinterpret_cast<T*>(smem_raw);  // [nf][FD_WY][FD_WX]
  const int nf = a.nf, nx = a.nx, ny = a.ny;
  T* mu = tile + nf * FD_WY * FD_WX;  // [FD_MY][FD_MX]
  const long long N = a.npts;
  const int x0 = blockIdx.x * FD_TX, y0 = blockIdx.y * FD_TY;
  const int tid = threadIdx.x;
  for (int f = 0; f < nf; ++f)
    for (int i = tid; i < FD_WX * FD_WY; i += blockDim.x) {
      const int lx = i % FD_WX, ly = i / FD_WX;
      const int gx = ((x0 + lx - 2) % nx + nx) % nx, gy = ((y0 + ly - 2) % ny + ny) % ny;
      tile[(f * FD_WY + ly) * FD_WX + lx] = in[f * N + (long long)gy * nx + gx];
    }
  __syncthreads();
  const Pointwise<T> pw(a);
  const Coef<T>& k = coef<T>(a);
  const T idx2 = k.idx2, idy2 = k.idy2, kc = k.kc, ke = k.ke, dtM = k.dtM, dtL = k.dtL;
  auto at = [tile](int f, int ly, int lx) { return tile[(f * FD_WY + ly) * FD_WX + lx]; };
  auto lap = [&](int f, int ly, int lx) {
    const T c0 = at(f, ly, lx);
    return (at(f, ly, lx - 1) - T(2) * c0 + at(f, ly, lx + 1)) * idx2 +
           (at(f, ly - 1, lx) - T(2) * c0 + at(f, ly + 1, lx)) * idy2;
  };
  // (i) mu on the tile plus a one-point halo
  for (int i = tid; i < FD_MX * FD_MY; i += blockDim.x) {
    const int mx = i % FD_MX, my = i / FD_MX;
    const int lx = mx + 1, ly = my + 1;
    T h = T(0);
    for (int f = 1; f < nf; ++f) h += pw.hpoly(at(f, ly, lx));
    mu[my * FD_MX + mx] = pw.fc(at(0, ly, lx), h) - kc * lap(0, ly, lx);
  }
  __syncthreads();
  // (ii), (iii) interior update
  const int tx = tid % FD_TX, ty = tid / FD_TX;
  const int gx = x0 + tx, gy = y0 + ty;
  if (gx >= nx || gy >= ny) return;
  const int lx = tx + 2, ly = ty + 2, mx = tx + 1, my = ty + 1;
  const T m0 = mu[my * FD_MX + mx];
  const T lmu = (mu[my * FD_MX + mx - 1] - T(2) * m0 + mu[my * FD_MX + mx + 1]) * idx2 +
                (mu[(my - 1) * FD_MX + mx] - T(2) * m0 + mu[(my + 1) * FD_MX + mx]) * idy2;
  const T c = at(0, ly, lx);
  const long long o = (long long)gy * nx + gx;
  const T cn = c + dtM * lmu;
  bool bad = !finite_val(cn);
  out[o] = cn;
  T S2 = T(0);
  for (int f = 1; f < nf; ++f) {
    const T e = at(f, ly, lx);
    S2 += e * e;
  }
  for (int f = 1; f < nf; ++f) {
    const T e = at(f, ly, lx);
    const T en = e - dtL * (pw.feta(c, e, S2) - ke * lap(f, ly, lx));
    bad |= !finite_val(en);
    out[f * N + o] = en;
  }
  if (bad) atomicOr(a.flag, FS_FLAG_NONFINITE);
}

template <typename T>
cudaError_t fd_launch_t(const KArgs& a, const void* in, void* out, cudaStream_t s) {
  dim3 grid((unsigned)((a.nx + FD_TX - 1) / FD_TX), (unsigned)((a.ny + FD_TY - 1) / FD_TY));
  size_t smem = sizeof(T) * ((size_t)a.nf * FD_WX * FD_WY + FD_MX * FD_MY);
  fs_fd_kernel<T><<<grid, FD_TX * FD_TY, smem, s>>>(a, reinterpret_cast<const T*>(in), reinterpret_cast<T*>(out));
  return cudaGetLastError();
}

}  // namespace

cudaError_t fd_launch(bool f64, const KArgs& a, const void* in, void* out, cudaStream_t s) {
  return f64 ? fd_launch_t<double>(a, in, out, s) : fd_launch_t<float>(a, in, out, s);
}

}  // namespace fs
