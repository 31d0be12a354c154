// Explicit finite-difference comparison scheme of Boccardo et al. (arXiv
// 2306.04322, Section 2.2): forward Euler in time, second-order centred
// 5-point (2D) / 7-point (3D) Laplacian on a periodic grid, three stages per
// step
//   (i)   mu    = df/dc - kappa_c lap(c)
//   (ii)  c'    = c + dt M lap(mu)
//   (iii) eta'_i = eta_i - dt L (df/deta_i - kappa_eta lap(eta_i))
// In 2D fused into one kernel: a CTA loads a tile with a two-point halo
// (periodic wrap instead of the paper's ghost layers), forms mu on the tile
// plus a one-point halo in shared memory, then updates its interior.
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
      const int gx = (x0 + lx - 2) & (nx - 1), gy = (y0 + ly - 2) & (ny - 1);  // periodic (powers of two)
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
  const long long out_bytes = (long long)nf * N * (long long)sizeof(T);
  if (in_bounds(a, &out[o], sizeof(T), out, out_bytes)) out[o] = cn;
  T S2 = T(0);
  for (int f = 1; f < nf; ++f) {
    const T e = at(f, ly, lx);
    S2 += e * e;
  }
  for (int f = 1; f < nf; ++f) {
    const T e = at(f, ly, lx);
    const T en = e - dtL * (pw.feta(c, e, S2) - ke * lap(f, ly, lx));
    bad |= !finite_val(en);
    if (in_bounds(a, &out[f * N + o], sizeof(T), out, out_bytes)) out[f * N + o] = en;
  }
  if (bad) atomicOr(a.flag, FS_FLAG_NONFINITE);
}

// 3D: the same three stages with the 7-point Laplacian, as two kernels (one
// thread per grid point, neighbours through the caches).  Kernel 1 forms mu
// (stage i) into a scratch field and writes the updated eta_i (stage iii);
// kernel 2 applies stage ii to c.  Axes are powers of two, so the periodic
// neighbours are masks.
template <typename T>
struct Grid3 {
  int nx, ny, nz;
  long long N;
  int lx, lxy;  // log2(nx), log2(nx ny)
  __device__ Grid3(const KArgs& a) : nx(a.nx), ny(a.ny), nz(a.nz), N(a.npts) {
    lx = __ffs(nx) - 1;
    lxy = lx + __ffs(ny) - 1;
  }
  __device__ __forceinline__ void coords(long long i, int& x, int& y, int& z) const {
    x = (int)i & (nx - 1);
    y = (int)(i >> lx) & (ny - 1);
    z = (int)(i >> lxy);
  }
  __device__ __forceinline__ long long at(int x, int y, int z) const {
    return ((long long)z * ny + y) * nx + x;
  }
  // 7-point Laplacian of field f at (x, y, z)
  __device__ __forceinline__ T lap(const T* __restrict__ f, int x, int y, int z, T ix2, T iy2, T iz2) const {
    const T c0 = f[at(x, y, z)];
    return (f[at((x - 1) & (nx - 1), y, z)] - T(2) * c0 + f[at((x + 1) & (nx - 1), y, z)]) * ix2 +
           (f[at(x, (y - 1) & (ny - 1), z)] - T(2) * c0 + f[at(x, (y + 1) & (ny - 1), z)]) * iy2 +
           (f[at(x, y, (z - 1) & (nz - 1))] - T(2) * c0 + f[at(x, y, (z + 1) & (nz - 1))]) * iz2;
  }
};

template <typename T>
__global__ void __launch_bounds__(256) fs_fd3_mu_eta_kernel(KArgs a, const T* __restrict__ in, T* __restrict__ out,
                                                            T* __restrict__ mu) {
  const Grid3<T> g(a);
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.N) return;
  int x, y, z;
  g.coords(i, x, y, z);
  const Pointwise<T> pw(a);
  const Coef<T>& k = coef<T>(a);
  const int nf = a.nf;
  const T c = in[i];
  T h = T(0), S2 = T(0);
  for (int f = 1; f < nf; ++f) {
    const T e = in[f * g.N + i];
    h += pw.hpoly(e);
    S2 += e * e;
  }
  mu[i] = pw.fc(c, h) - k.kc * g.lap(in, x, y, z, k.idx2, k.idy2, k.idz2);
  bool bad = false;
  for (int f = 1; f < nf; ++f) {
    const T* ef = in + f * g.N;
    const T e = ef[i];
    const T en = e - k.dtL * (pw.feta(c, e, S2) - k.ke * g.lap(ef, x, y, z, k.idx2, k.idy2, k.idz2));
    bad |= !finite_val(en);
    out[f * g.N + i] = en;
  }
  if (bad) atomicOr(a.flag, FS_FLAG_NONFINITE);
}

template <typename T>
__global__ void __launch_bounds__(256) fs_fd3_c_kernel(KArgs a, const T* __restrict__ in, T* __restrict__ out,
                                                       const T* __restrict__ mu) {
  const Grid3<T> g(a);
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.N) return;
  int x, y, z;
  g.coords(i, x, y, z);
  const Coef<T>& k = coef<T>(a);
  const T cn = in[i] + k.dtM * g.lap(mu, x, y, z, k.idx2, k.idy2, k.idz2);
  if (!finite_val(cn)) atomicOr(a.flag, FS_FLAG_NONFINITE);
  out[i] = cn;
}

template <typename T>
cudaError_t fd_launch_t(const KArgs& a, const void* in, void* out, void* scratch, cudaStream_t s) {
  if (a.nz > 1) {
    const unsigned blocks = (unsigned)((a.npts + 255) / 256);
    fs_fd3_mu_eta_kernel<T><<<blocks, 256, 0, s>>>(a, reinterpret_cast<const T*>(in), reinterpret_cast<T*>(out),
                                                   reinterpret_cast<T*>(scratch));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    fs_fd3_c_kernel<T><<<blocks, 256, 0, s>>>(a, reinterpret_cast<const T*>(in), reinterpret_cast<T*>(out),
                                              reinterpret_cast<const T*>(scratch));
    return cudaGetLastError();
  }
  dim3 grid((unsigned)((a.nx + FD_TX - 1) / FD_TX), (unsigned)((a.ny + FD_TY - 1) / FD_TY));
  size_t smem = sizeof(T) * ((size_t)a.nf * FD_WX * FD_WY + FD_MX * FD_MY);
  fs_fd_kernel<T><<<grid, FD_TX * FD_TY, smem, s>>>(a, reinterpret_cast<const T*>(in), reinterpret_cast<T*>(out));
  return cudaGetLastError();
}

}  // namespace

int fd_launches_per_step(const KArgs& a) { return a.nz > 1 ? 2 : 1; }

cudaError_t fd_launch(bool f64, const KArgs& a, const void* in, void* out, void* scratch, cudaStream_t s) {
  return f64 ? fd_launch_t<double>(a, in, out, scratch, s) : fd_launch_t<float>(a, in, out, scratch, s);
}

}  // namespace fs
