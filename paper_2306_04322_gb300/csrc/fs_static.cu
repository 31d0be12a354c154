// fs_step2d_static: the 2D semi-implicit Fourier-spectral step for callers
// that cannot allocate device memory -- for example a host application that
// hands every byte of device memory to its own pool allocator before loading
// this library, or code on a real-time or signal-handling path where a
// cudaMalloc (which may synchronise the device and take driver locks) is not
// allowed.  It runs the same row and column kernels as a plan, but every
// intermediate (the packed spectra, the twiddle and |xi|^2 tables, the
// status flag and the FP64 mean carry) lives in one file-scope device array
// of fixed size, so the call allocates nothing: no cudaMalloc, no cudaFree,
// no host heap.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

#include "fs.h"
#include "fs_fft.cuh"
#include "fs_internal.h"

namespace {

// Limits of the static scratch: up to 65536 grid points, p <= 2 (three
// fields), FP64 or FP32.  Layout (bytes): [0, 256) flag, mean carry and
// accumulators; [256, 256 + kTableBytes) constant tables; then the
// (nf + 1) packed half-spectrum slots.
constexpr long long kMaxPoints = 65536;
constexpr int kMaxFields = 3;
constexpr size_t kHeadBytes = 256;
constexpr size_t kTableBytes = 131072;
constexpr size_t kSpecOffset = kHeadBytes + kTableBytes;
constexpr size_t kScratchBytes = kSpecOffset + (size_t)(kMaxFields + 1) * (kMaxPoints / 2) * 16;  // 2,228,480

}  // namespace

// The scratch itself: every GPU that loads the library holds it until exit.
static __device__ __align__(256) unsigned char g_fs_static_scratch[kScratchBytes];

namespace {

constexpr int kMaxDevices = 64;
void* g_scratch_dev[kMaxDevices];               // device address of the scratch, per device
unsigned char g_host_tables[kTableBytes];       // host staging of the tables (static)
int g_host_flag;                                // status read back (static)

bool pow2_between(int n, int lo, int hi) { return n >= lo && n <= hi && (n & (n - 1)) == 0; }

double axis_k2_static(int lap, int k, int n, double dx) {
  const long double pi = 3.141592653589793238462643383279502884L;
  int nk = k <= n / 2 ? k : k - n;
  double xi = (double)(2.0L * pi * (long double)nk / ((long double)n * (long double)dx));
  if (lap == FS_LAP_FD2) return -2.0 * (std::cos(dx * xi) - 1.0) / (dx * dx);
  if (lap == FS_LAP_FD4) return -(16.0 * std::cos(dx * xi) - std::cos(2.0 * dx * xi) - 15.0) / (6.0 * dx * dx);
  return xi * xi;
}

size_t up16(size_t v) { return (v + 15) & ~(size_t)15; }

// Writes the Stockham pass tables of (L, E) as complex T at dst; entries
// [r][j] = exp(-2 pi i r j / (NS R)) for every pass after the first.
template <typename T>
size_t put_pass_table(T* dst, int L, int E) {
  const long double pi = 3.141592653589793238462643383279502884L;
  size_t n = 0;
  for (int ns = 1; ns < L;) {
    int r = E < L / ns ? E : L / ns;
    if (ns > 1)
      for (int q = 0; q < r; ++q)
        for (int j = 0; j < ns; ++j) {
          long long e = (long long)q * j % ((long long)ns * r);
          long double ang = 2.0L * pi * (long double)e / (long double)(ns * r);
          dst[2 * n] = (T)cosl(ang);
          dst[2 * n + 1] = (T)(-sinl(ang));
          ++n;
        }
    ns *= r;
  }
  return n;
}

template <typename T>
void fill_coef_static(fs::Coef<T>& k, const fs_params& q, double scale) {
  k.two_rho2 = (T)(2.0 * q.rho2);
  k.ca = (T)q.c_alpha;
  k.dcab = (T)(q.c_beta - q.c_alpha);
  k.rho2dcab = (T)(q.rho2 * (q.c_beta - q.c_alpha));
  k.cab = (T)(q.c_beta + q.c_alpha);
  k.w = (T)q.w;
  k.four_alpha = (T)(4.0 * q.alpha);
  k.Ldt = (T)(q.L * q.dt);
  k.Mdt = (T)(q.M * q.dt);
  k.Mdtkc = (T)(q.M * q.dt * q.kappa_c);
  k.Ldtke = (T)(q.L * q.dt * q.kappa_eta);
  k.scale = (T)scale;
  k.idx2 = (T)(1.0 / (q.dx[0] * q.dx[0]));
  k.idy2 = (T)(1.0 / (q.dx[1] * q.dx[1]));
  k.idz2 = (T)0;
  k.kc = (T)q.kappa_c;
  k.ke = (T)q.kappa_eta;
  k.dtM = (T)(q.dt * q.M);
  k.dtL = (T)(q.dt * q.L);
  k.dt = (T)q.dt;
}

// Byte size of the tables build_tables writes for grid (nx, ny).
template <typename T>
size_t tables_bytes(int nx, int ny) {
  const bool f64 = sizeof(T) == 8;
  size_t o = up16(sizeof(T) * (nx / 2 + 1));
  o = up16(o + sizeof(T) * ny);
  o = up16(o + 2 * sizeof(T) * (size_t)fs::pass_table_size(nx / 2, fs::row_E(nx / 2, f64)));
  o = up16(o + 2 * sizeof(T) * (size_t)fs::pass_table_size(ny, fs::col_E(ny, f64)));
  return up16(o + 2 * sizeof(T) * (nx / 2));
}

// Builds the tables in g_host_tables (the caller has checked that they fit:
// tables_bytes <= kTableBytes); returns their byte size and the offsets of
// each table (relative to the table region).
template <typename T>
size_t build_tables(const fs_params& q, size_t off[5]) {
  const int nx = q.n[0], ny = q.n[1];
  unsigned char* b = g_host_tables;
  size_t o = 0;
  off[0] = o;  // k2x
  T* kx = reinterpret_cast<T*>(b + o);
  for (int k = 0; k <= nx / 2; ++k) kx[k] = (T)axis_k2_static(q.lap, k, nx, q.dx[0]);
  o = up16(o + sizeof(T) * (nx / 2 + 1));
  off[1] = o;  // k2y
  T* ky = reinterpret_cast<T*>(b + o);
  for (int k = 0; k < ny; ++k) ky[k] = (T)axis_k2_static(q.lap, k, ny, q.dx[1]);
  o = up16(o + sizeof(T) * ny);
  off[2] = o;  // row pass tables
  const bool f64 = sizeof(T) == 8;
  o = up16(o + 2 * sizeof(T) * put_pass_table(reinterpret_cast<T*>(b + o), nx / 2, fs::row_E(nx / 2, f64)));
  off[3] = o;  // column pass tables
  o = up16(o + 2 * sizeof(T) * put_pass_table(reinterpret_cast<T*>(b + o), ny, fs::col_E(ny, f64)));
  off[4] = o;  // exp(-2 pi i k / nx), k < nx/2
  T* h = reinterpret_cast<T*>(b + o);
  const long double pi = 3.141592653589793238462643383279502884L;
  for (int k = 0; k < nx / 2; ++k) {
    long double ang = 2.0L * pi * (long double)k / (long double)nx;
    h[2 * k] = (T)cosl(ang);
    h[2 * k + 1] = (T)(-sinl(ang));
  }
  o = up16(o + 2 * sizeof(T) * (nx / 2));
  return o;
}

typedef CUresult (*EncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                             const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                             CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

template <typename T>
fs_status run_static(const fs_params& q, void* fields, int64_t nsteps, cudaStream_t s, unsigned char* scratch) {
  const bool f64 = sizeof(T) == 8;
  const int nx = q.n[0], ny = q.n[1], nf = 1 + q.p;
  const long long N = (long long)nx * ny;
  size_t off[5];
  if (tables_bytes<T>(nx, ny) > kTableBytes) return FS_ERR_UNSUPPORTED;
  const size_t tbytes = build_tables<T>(q, off);
  unsigned char* tables = scratch + kHeadBytes;
  unsigned char* spec = scratch + kSpecOffset;
  cudaError_t e = cudaMemsetAsync(scratch, 0, kHeadBytes, s);  // flag, mean carry, accumulators start at 0
  if (e == cudaSuccess) e = cudaMemcpyAsync(tables, g_host_tables, tbytes, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return FS_ERR_CUDA;

  fs::KArgs a;
  std::memset(&a, 0, sizeof(a));
  a.spec = spec;
  a.real = fields;
  a.k2x = tables + off[0];
  a.k2y = tables + off[1];
  a.tw_row = tables + off[2];
  a.tw_col = tables + off[3];
  a.tw_half = tables + off[4];
  a.slot_stride = N / 2;
  a.npts = N;
  a.nx = nx;
  a.nx_full = nx;
  a.ny = ny;
  a.nz = 1;
  a.nf = nf;
  a.lines = ny;
  a.M = q.M;
  a.L = q.L;
  a.kappa_c = q.kappa_c;
  a.kappa_eta = q.kappa_eta;
  a.rho2 = q.rho2;
  a.c_alpha = q.c_alpha;
  a.c_beta = q.c_beta;
  a.w = q.w;
  a.alpha = q.alpha;
  a.dt = q.dt;
  a.scale = 1.0 / (2.0 * (double)N);
  a.inv_npts = 1.0 / (double)N;
  a.flag = reinterpret_cast<int*>(scratch);
  a.spec_bytes = (long long)(nf + 1) * (N / 2) * 2 * (long long)sizeof(T);
  a.real_bytes = (long long)nf * N * (long long)sizeof(T);
  a.csum = f64 ? nullptr : reinterpret_cast<double*>(scratch + 8);
  a.acc = reinterpret_cast<double*>(scratch + 64);
  fill_coef_static(a.cd, q, a.scale);
  fill_coef_static(a.cf, q, a.scale);

  // tensor map over the spectrum slots [nf + 1][ny][kx], column-tile boxes
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult qr;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &qr) !=
          cudaSuccess ||
      qr != cudaDriverEntryPointSuccess || !fn)
    return FS_ERR_CUDA;
  const int units = f64 ? 2 : 1;
  const int tk = fs::col_tile_width(f64, nx, ny);
  const cuuint64_t W = (cuuint64_t)(nx / 2) * units;
  cuuint64_t dims[3] = {W, (cuuint64_t)ny, (cuuint64_t)(nf + 1)};
  cuuint64_t strides[2] = {W * 8, W * 8 * ny};
  cuuint32_t box[3] = {(cuuint32_t)(tk * units), (cuuint32_t)(ny < 256 ? ny : 256), 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUtensorMap tm;
  if (reinterpret_cast<EncodeFn>(fn)(&tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, spec, dims, strides, box, estr,
                                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                     CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return FS_ERR_CUDA;

  if (!f64) e = fs::sum_launch_f32(fields, N, const_cast<double*>(a.csum), s);
  for (int64_t step = 0; step < nsteps && e == cudaSuccess; ++step) {
    a.mode = step == 0 ? 1 : 0;
    e = f64 ? fs::row_launch_f64(a, s) : fs::row_launch_f32(a, s);
    if (e == cudaSuccess) e = f64 ? fs::col_launch_f64(a, tm, s) : fs::col_launch_f32(a, tm, s);
  }
  if (e == cudaSuccess) {
    a.mode = 2;  // inverse row pass back into the caller's fields
    e = f64 ? fs::row_launch_f64(a, s) : fs::row_launch_f32(a, s);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&g_host_flag, a.flag, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return FS_ERR_CUDA;
  if (g_host_flag & fs::FS_FLAG_TIMEOUT) return FS_ERR_TIMEOUT;
  if (g_host_flag & fs::FS_FLAG_NONFINITE) return FS_ERR_NONFINITE;
  return g_host_flag ? FS_ERR_CUDA : FS_OK;
}

}  // namespace

extern "C" fs_status fs_step2d_static(const fs_params* prm, void* fields, int64_t nsteps, void* stream) {
  // Malformed arguments: FS_ERR_INVALID_ARG.  The kernels read and write the
  // fields with 16-byte bulk copies and vector stores, so the array must
  // start on a 16-byte boundary (a tensor view with an odd storage offset
  // does not); rejecting it here keeps a misaligned access off the GPU.
  if (!prm || !fields || nsteps < 0 || ((uintptr_t)fields & 15) != 0) return FS_ERR_INVALID_ARG;
  const fs_params& q = *prm;
  if ((q.ndim != 2 && q.ndim != 3) || q.p < 0 || q.p > 4 || !(q.dt > 0.0) || !std::isfinite(q.dt) ||
      !(q.dx[0] > 0.0) || !(q.dx[1] > 0.0) || q.precision < FS_F64 || q.precision > FS_F32_TC_BF16X3 ||
      q.lap < FS_LAP_SPECTRAL || q.lap > FS_LAP_FD4 || q.scheme < FS_SCHEME_SEMI_IMPLICIT_FS ||
      q.scheme > FS_SCHEME_EXPLICIT_FD)
    return FS_ERR_INVALID_ARG;
  // Valid requests outside this entry point's limits: FS_ERR_UNSUPPORTED.
  if (q.ndim != 2 || (q.precision != FS_F64 && q.precision != FS_F32) || q.scheme != FS_SCHEME_SEMI_IMPLICIT_FS)
    return FS_ERR_UNSUPPORTED;
  if (!pow2_between(q.n[0], 8, 1024) || !pow2_between(q.n[1], 8, 1024)) return FS_ERR_UNSUPPORTED;
  if ((long long)q.n[0] * q.n[1] > kMaxPoints || 1 + q.p > kMaxFields) return FS_ERR_UNSUPPORTED;
  if (nsteps == 0) return FS_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // The call copies its tables from one static host array and waits for the
  // stream before it returns; neither may be recorded into a graph, so a
  // capturing stream is refused (nothing is enqueued on it).
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return FS_ERR_CUDA;
  if (cap != cudaStreamCaptureStatusNone) return FS_ERR_UNSUPPORTED;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return FS_ERR_CUDA;
  if (!g_scratch_dev[dev]) {
    // first call on this device: look up the device address of the scratch
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_fs_static_scratch) != cudaSuccess || !ptr) return FS_ERR_CUDA;
    g_scratch_dev[dev] = ptr;
  }
  unsigned char* scratch = static_cast<unsigned char*>(g_scratch_dev[dev]);
  return q.precision == FS_F64 ? run_static<double>(q, fields, nsteps, s, scratch)
                               : run_static<float>(q, fields, nsteps, s, scratch);
}
