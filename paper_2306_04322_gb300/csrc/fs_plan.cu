// C ABI of the semi-implicit Fourier-spectral phase-field library: plan
// creation and validation, workspace ownership, state tracking, launch
// sequencing and CUDA-graph replay of the time loop (Algorithm 1 of
// Boccardo et al., arXiv 2306.04322).  Kernels live in the fs_k*.cu units.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "fs.h"
#include "fs_fft.cuh"
#include "fs_internal.h"
#include "fs_slab_hooks.h"

namespace {

thread_local std::string g_thread_error;

// Which buffers hold the current state: the real fields, the spectra (the
// carried x spectra the next row pass starts from), or both (after
// fs_get_fields, so reading the fields does not change the trajectory).
enum StateKind { kStateNone = 0, kStateReal = 1, kStateSpec = 2, kStateBoth = 3 };

struct Member {
  fs_params prm;
  long long npts = 0;
  // device pointers into the plan's arena
  void* spec = nullptr;
  void* real = nullptr;
  void* k2x = nullptr;  // plan precision
  void* k2y = nullptr;
  void* k2z = nullptr;
  void* tw_row = nullptr;  // complex, plan precision
  void* tw_col = nullptr;
  void* tw_z = nullptr;
  void* tw_half = nullptr;
  void* tw_row_w = nullptr;  // x-pass tables with 32 values per thread (FP32 rows of 1024)
  void* tc_b = nullptr;  // split DFT matrix of the tensor-core stage (TC precisions)
  void* tw_row2 = nullptr;  // x-line tables of the pair-form row pass (FP32, nx in {256, 512, 1024})
  void* tw_col2 = nullptr;  // y-line tables of the warp-per-column pass (FP32 2D, ny in [64, 1024])
  void* tw_row2w = nullptr; // the same with two warps per line (lines of 128 points and more)
  void* tw_col2w = nullptr;
  double* csum = nullptr;
  long long slot_stride = 0;
  // column plan of a slab (fs_slab_*): its nx covers kx columns kx_base ..
  // kx_base + nx/2 - 1 of a grid of nx_full x points and npts_full points
  // (0: an ordinary plan)
  int kx_base = 0, nx_full = 0;
  long long npts_full = 0;
  CUtensorMap tmap_col;  // [slot * nz + z][y][kx] tiles of the 2D column pass / 3D y passes
  CUtensorMap tmap_z;    // [slot][z][y][kx] z lines of the 3D z step
  CUtensorMap tmap_col2; // [slot][y][kx] two-column tiles of the warp-per-column pass
  int fd_cur = 0;        // explicit FD: 0 state in `real`, 1 state in `spec` (as real fields)
  // adjoint workspace (allocated on first use)
  void* aspec = nullptr;  // 3 nf packed half-spectrum slots
  void* alam = nullptr;   // lam' in (nf real fields)
  void* au = nullptr;     // u (nf real fields)
  void* aout = nullptr;   // lambda out (nf real fields)
  CUtensorMap tmap_adj;    // adjoint slots: 2D column tiles / 3D y-pass tiles
  CUtensorMap tmap_adj_z;  // adjoint slots: 3D z lines
};

}  // namespace

struct fs_plan {
  std::vector<Member> members;
  bool f64 = true;
  bool fd = false;  // explicit FD comparison scheme
  bool batch = false;  // ensemble: one launch per pass for all members
  fs::BatchArgs bargs{};
  const fs::KArgs* bmem1 = nullptr;  // row arguments in mode 1 (from real fields)
  bool tuned = false;
  int nf = 1;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  fs_alloc_fn alloc = nullptr;
  fs_free_fn dealloc = nullptr;
  void* actx = nullptr;
  std::vector<void*> blocks;
  size_t ws_bytes = 0;
  int* flag = nullptr;
  unsigned* gsync = nullptr; // grid-barrier counters of the fused step (pass form 4)
  double* acc = nullptr;     // diagnostic accumulators (device)
  int* host_flag = nullptr;  // pinned
  int state = kStateNone;
  cudaGraphExec_t gexec = nullptr;
  int gsteps = 0;
  int64_t last_launches = 0;
  int short_wait = 0;  // test hook of fs_test_short_wait
  int row_form = 0;    // fs_set_pass_forms: 0 default, 1 half-length / tile kernels, 2 warp-per-line
                       // kernels, 3 the same with two warps per line, 4 (both passes) the fused step
  int col_form = 0;
  std::vector<cudaEvent_t> ev_pool;  // fs_step_profiled timing events
  std::vector<int> ev_kind;
  size_t ev_used = 0;
  std::string err;
};

namespace {

fs_status fail(fs_plan* p, fs_status s, const std::string& msg) {
  if (p)
    p->err = msg;
  else
    g_thread_error = msg;
  return s;
}

fs_status cuda_fail(fs_plan* p, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return fail(p, FS_ERR_CUDA, m);
}

bool pow2_in(int n, int lo, int hi) { return n >= lo && n <= hi && (n & (n - 1)) == 0; }
bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }
bool finite_nonneg(double v) { return std::isfinite(v) && v >= 0.0; }

fs_status validate(const fs_params* p, std::string* why) {
  if (!p) {
    *why = "params is NULL";
    return FS_ERR_INVALID_ARG;
  }
  if (p->ndim != 2 && p->ndim != 3) {
    *why = "ndim must be 2 or 3";
    return FS_ERR_INVALID_ARG;
  }
  for (int d = 0; d < p->ndim; ++d) {
    if (p->n[d] <= 0) {
      *why = "grid size must be positive";
      return FS_ERR_INVALID_ARG;
    }
    if (!finite_pos(p->dx[d])) {
      *why = "dx must be finite and > 0";
      return FS_ERR_INVALID_ARG;
    }
  }
  if (p->p < 0 || p->p > 4) {
    *why = "p must be in [0, 4]";
    return FS_ERR_INVALID_ARG;
  }
  if (!finite_pos(p->dt)) {
    *why = "dt must be finite and > 0";
    return FS_ERR_INVALID_ARG;
  }
  const double nn[] = {p->M, p->L, p->kappa_c, p->kappa_eta, p->rho2, p->w, p->alpha};
  for (double v : nn)
    if (!finite_nonneg(v)) {
      *why = "M, L, kappa_c, kappa_eta, rho2, w, alpha must be finite and >= 0";
      return FS_ERR_INVALID_ARG;
    }
  if (!std::isfinite(p->c_alpha) || !std::isfinite(p->c_beta)) {
    *why = "c_alpha, c_beta must be finite";
    return FS_ERR_INVALID_ARG;
  }
  if (p->precision < FS_F64 || p->precision > FS_F32_TC_BF16X3) {
    *why = "unknown precision";
    return FS_ERR_INVALID_ARG;
  }
  if (p->lap < FS_LAP_SPECTRAL || p->lap > FS_LAP_FD4) {
    *why = "unknown lap";
    return FS_ERR_INVALID_ARG;
  }
  if (p->scheme < FS_SCHEME_SEMI_IMPLICIT_FS || p->scheme > FS_SCHEME_EXPLICIT_FD) {
    *why = "unknown scheme";
    return FS_ERR_INVALID_ARG;
  }
  for (int d = 0; d < p->ndim; ++d)
    if (!pow2_in(p->n[d], 8, 2048)) {
      *why = "each grid axis must be a power of two in [8, 2048]";
      return FS_ERR_UNSUPPORTED;
    }
  if (p->ndim == 3 && (p->n[0] > 1024 || p->n[1] > 512 || p->n[2] > 512)) {
    *why = "3D grids support a power of two up to 1024 along x and up to 512 along y and z";
    return FS_ERR_UNSUPPORTED;
  }
  if (p->precision == FS_F32_TC_TF32 || p->precision == FS_F32_TC_BF16X3) {
    if (p->scheme != FS_SCHEME_SEMI_IMPLICIT_FS || p->n[0] < 64 || p->n[1] < 64 ||
        (p->ndim > 2 && p->n[2] < 64)) {
      *why = "the tensor-core DFT stage needs the FS scheme and every axis of at least 64 points";
      return FS_ERR_UNSUPPORTED;
    }
  }
  return FS_OK;
}

// Squared frequency norm contribution of bin k on an axis of n points and
// spacing dx: spectral (Eq. Gamma_fft), FS-FD O(dl^2) (Eq. Gamma_fft-fdO2),
// FS-FD O(dl^4) (Eq. Gamma_fft-fdO4); index vector [0..n/2, -(n/2-1)..-1].
double axis_k2(int lap, int k, int n, double dx) {
  const long double pi = 3.141592653589793238462643383279502884L;
  int nk = k <= n / 2 ? k : k - n;
  double xi = (double)(2.0L * pi * (long double)nk / ((long double)n * (long double)dx));
  if (lap == FS_LAP_FD2) return -2.0 * (std::cos(dx * xi) - 1.0) / (dx * dx);
  if (lap == FS_LAP_FD4) return -(16.0 * std::cos(dx * xi) - std::cos(2.0 * dx * xi) - 15.0) / (6.0 * dx * dx);
  return xi * xi;
}

void* plan_alloc(fs_plan* p, size_t bytes) {
  bytes = (bytes + 255) & ~(size_t)255;
  void* ptr = nullptr;
  if (p->alloc) {
    ptr = p->alloc(bytes, p->actx);
  } else if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
    cudaGetLastError();
    ptr = nullptr;
  }
  if (ptr) {
    p->blocks.push_back(ptr);
    p->ws_bytes += bytes;
  }
  return ptr;
}

void plan_free_all(fs_plan* p) {
  for (void* b : p->blocks) {
    if (p->dealloc)
      p->dealloc(b, p->actx);
    else if (!p->alloc)
      cudaFree(b);
  }
  p->blocks.clear();
  p->ws_bytes = 0;
}

template <typename T>
void fill_coef(fs::Coef<T>& k, const fs_params& q, double scale) {
  k.idx2 = (T)(1.0 / (q.dx[0] * q.dx[0]));
  k.idy2 = (T)(1.0 / (q.dx[1] * q.dx[1]));
  k.idz2 = (T)(q.ndim > 2 ? 1.0 / (q.dx[2] * q.dx[2]) : 0.0);
  k.kc = (T)q.kappa_c;
  k.ke = (T)q.kappa_eta;
  k.dtM = (T)(q.dt * q.M);
  k.dtL = (T)(q.dt * q.L);
  k.dt = (T)q.dt;
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
}

fs::KArgs make_args(const fs_plan* p, const Member& m, int mode) {
  fs::KArgs a;
  std::memset(&a, 0, sizeof(a));
  a.spec = m.spec;
  a.real = m.real;
  a.tw_row = m.tw_row;
  a.tw_col = m.tw_col;
  a.tw_z = m.tw_z;
  a.tw_half = m.tw_half;
  a.tw_row_w = m.tw_row_w;
  // single plans: the warp-per-line forms by default for lines of 256 points
  // and more (form 0) -- rows only in 2D: a 3D x pass has ny nz lines, and
  // one row pair per CTA (table fetch and set-up per pair) loses to the
  // several-row CTAs of the half-length kernel there -- always with form 2,
  // never with form 1; ensemble members keep both tables (the autotuner
  // picks the form per pass)
  const bool r2 = p->batch || p->row_form == 2 || p->row_form == 4 ||
                  (p->row_form == 0 && m.prm.n[0] >= 256 && m.prm.ndim == 2);
  const bool c2 = p->batch || p->col_form == 2 || p->col_form == 4 || (p->col_form == 0 && m.prm.n[1] >= 256);
  a.tw_row2 = r2 ? m.tw_row2 : nullptr;
  a.tw_col2 = c2 ? m.tw_col2 : nullptr;
  a.tw_row2w = (!p->batch && p->row_form == 3) ? m.tw_row2w : nullptr;
  // columns of 2048 points have only the two-warp form, the default there
  a.tw_col2w = (!p->batch && (p->col_form == 3 || (p->col_form == 0 && m.prm.n[1] == 2048))) ? m.tw_col2w : nullptr;
  a.tc_b = m.tc_b;
  a.k2x = m.k2x;
  a.k2y = m.k2y;
  a.k2z = m.k2z;
  a.slot_stride = m.slot_stride;
  a.npts = m.npts;
  a.nx = m.prm.n[0];
  a.nx_full = m.nx_full ? m.nx_full : m.prm.n[0];
  a.kx_base = m.kx_base;
  a.ny = m.prm.n[1];
  a.nz = m.prm.ndim > 2 ? m.prm.n[2] : 1;
  a.nf = p->nf;
  a.lines = (long long)a.ny * a.nz;
  a.mode = mode;
  a.tc = m.prm.precision == FS_F32_TC_TF32 ? 1 : (m.prm.precision == FS_F32_TC_BF16X3 ? 2 : 0);
  a.carry3 = (m.prm.ndim == 3 && m.prm.scheme == FS_SCHEME_SEMI_IMPLICIT_FS) ? 1 : 0;
  a.plane0 = 0;
  a.M = m.prm.M;
  a.L = m.prm.L;
  a.kappa_c = m.prm.kappa_c;
  a.kappa_eta = m.prm.kappa_eta;
  a.rho2 = m.prm.rho2;
  a.c_alpha = m.prm.c_alpha;
  a.c_beta = m.prm.c_beta;
  a.w = m.prm.w;
  a.alpha = m.prm.alpha;
  a.dt = m.prm.dt;
  const double ntot = (double)(m.npts_full ? m.npts_full : m.npts);
  a.scale = 1.0 / (2.0 * ntot);
  a.inv_npts = 1.0 / ntot;
  a.csum = p->f64 ? nullptr : m.csum;
  a.flag = p->flag;
  a.acc = p->acc;
  a.short_wait = p->short_wait;
  const long long rs = p->f64 ? 8 : 4;
  a.spec_bytes = (long long)(p->nf + 1) * m.slot_stride * 2 * rs;
  a.real_bytes = (long long)p->nf * m.npts * rs;
  fill_coef(a.cd, m.prm, a.scale);
  fill_coef(a.cf, m.prm, a.scale);
  return a;
}

// FP32 plans take the warp-per-line forms where they apply (KArgs::tw_row2 /
// tw_col2 set), else the half-length row / tile column kernels.
cudaError_t launch_row(const fs_plan* p, const fs::KArgs& a, cudaStream_t s) {
  if (!p->f64 && (a.tw_row2 || a.tw_row2w)) {
    cudaError_t e = fs::row2_launch_f32(a, s);
    if (e != cudaErrorNotSupported) return e;
  }
  return p->f64 ? fs::row_launch_f64(a, s) : fs::row_launch_f32(a, s);
}
cudaError_t launch_col(const fs_plan* p, const Member& m, const fs::KArgs& a, cudaStream_t s) {
  if (!p->f64 && (a.tw_col2 || a.tw_col2w)) {
    cudaError_t e = fs::col2_launch_f32(a, m.tmap_col2, s);
    if (e != cudaErrorNotSupported) return e;
  }
  return p->f64 ? fs::col_launch_f64(a, m.tmap_col, s) : fs::col_launch_f32(a, m.tmap_col, s);
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// dependency on libcuda).
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(ptr);
  }
  return fn;
}

// Where the warp-per-line forms apply: FP32 (plain, and the row pass also
// for the tensor-core precisions, whose stage is in the column transforms),
// semi-implicit FS; rows of 256, 512 or 1024 points (2D rows and 3D x
// lines); 2D columns of 256, 512 or 1024 points with no tensor-core stage.
bool row2_form(const fs_params& prm, bool f64) {
  return !f64 && prm.scheme == FS_SCHEME_SEMI_IMPLICIT_FS && fs::row2_supported(prm.n[0], 1 + prm.p);
}
// (columns of 2048 points: two warps per line only)
bool col2_form(const fs_params& prm, bool f64) {
  return !f64 && prm.scheme == FS_SCHEME_SEMI_IMPLICIT_FS && prm.ndim == 2 && prm.precision == FS_F32 &&
         fs::col2_supported(prm.n[1], 1 + prm.p);
}

// Tensor map over the spectrum slots viewed as [nf + 1][ny][W] 8-byte units
// (W = nx/2 for FP32 complex, nx for FP64 complex); box = one column tile of
// the column pass, up to 256 rows.
bool encode_col_map(Member& m, int nslots, bool f64) {
  EncodeTiledFn enc = encode_tiled();
  if (!enc) return false;
  const int units = f64 ? 2 : 1;
  const int nx = m.prm.n[0], ny = m.prm.n[1], nz = m.prm.ndim > 2 ? m.prm.n[2] : 1;
  const cuuint64_t W = (cuuint64_t)(nx / 2) * units;  // 8-byte units per row
  {
    // [slot * nz + z][y][kx]: column tiles of the 2D column pass / 3D y passes
    const int tk = nz > 1 ? (f64 ? fs::line_tile_width_f64(nx, ny) : fs::line_tile_width_f32(nx, ny))
                          : fs::col_tile_width(f64, nx, ny);
    cuuint64_t dims[3] = {W, (cuuint64_t)ny, (cuuint64_t)nz * nslots};
    cuuint64_t strides[2] = {W * 8, W * 8 * ny};
    cuuint32_t box[3] = {(cuuint32_t)(tk * units), (cuuint32_t)(ny < 256 ? ny : 256), 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(&m.tmap_col, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, m.spec, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return false;
  }
  if (col2_form(m.prm, f64)) {
    // [slot][y][kx]: two-column tiles (16-byte rows) of the warp-per-column pass
    cuuint64_t dims[3] = {W, (cuuint64_t)ny, (cuuint64_t)nslots};
    cuuint64_t strides[2] = {W * 8, W * 8 * ny};
    cuuint32_t box[3] = {2, (cuuint32_t)(ny < 256 ? ny : 256), 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(&m.tmap_col2, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, m.spec, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return false;
  }
  if (nz > 1) {
    // [slot][z][y][kx]: z lines of one (ky, kx tile), up to 256 planes per box
    const int tk = f64 ? fs::line_tile_width_f64(nx, nz) : fs::line_tile_width_f32(nx, nz);
    cuuint64_t dims[4] = {W, (cuuint64_t)ny, (cuuint64_t)nz, (cuuint64_t)nslots};
    cuuint64_t strides[3] = {W * 8, W * 8 * ny, W * 8 * ny * nz};
    cuuint32_t box[4] = {(cuuint32_t)(tk * units), 1, (cuuint32_t)(nz < 256 ? nz : 256), 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = enc(&m.tmap_z, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4, m.spec, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return false;
  }
  return true;
}

// The passes of one step: 2D row, column; 3D x, y forward, z, y inverse.
int pass_kinds(const Member& m) { return m.prm.ndim > 2 ? 4 : 2; }

cudaError_t launch_pass(const fs_plan* p, const Member& m, const fs::KArgs& a, int kind, cudaStream_t s);

void* fd_buf(const Member& m, int which) { return which == 0 ? m.real : m.spec; }
// mu scratch of the 3D explicit FD step: the spectrum buffer's last slot
// (holds (nf + 1) N reals; the state uses the first nf N when it lives there)
void* fd_scratch(const fs_plan* p, const Member& m) {
  return (char*)m.spec + (size_t)(1 + m.prm.p) * m.npts * (p->f64 ? 8 : 4);
}

// Batched ensemble: kind 0 row pass (mode 0 from spectra, 1 from real
// fields), kind 1 column pass, each one persistent launch for all members.
cudaError_t launch_batch_pass(const fs_plan* p, int mode, int kind, cudaStream_t s) {
  fs::BatchArgs b = p->bargs;
  if (mode == 1) b.mem = p->bmem1;
  if (kind == 0) {
    if (b.row_form == 2) return fs::row2_batch_launch_f32(b, s);
    return p->f64 ? fs::row_batch_launch_f64(b, s) : fs::row_batch_launch_f32(b, s);
  }
  if (b.col_form == 2) return fs::col2_batch_launch_f32(b, s);
  return p->f64 ? fs::col_batch_launch_f64(b, s) : fs::col_batch_launch_f32(b, s);
}

// One time step of every member: row pass then column pass (or one explicit
// FD step, ping-ponging between the two real-field buffers).
cudaError_t enqueue_step(fs_plan* p, int mode, cudaStream_t s, int64_t* launches) {
  if (p->fd) {
    for (Member& m : p->members) {
      fs::KArgs a = make_args(p, m, 0);
      cudaError_t e = fs::fd_launch(p->f64, a, fd_buf(m, m.fd_cur), fd_buf(m, 1 - m.fd_cur), fd_scratch(p, m), s);
      if (e != cudaSuccess) return e;
      m.fd_cur = 1 - m.fd_cur;
      *launches += fs::fd_launches_per_step(a);
    }
    return cudaSuccess;
  }
  if (p->batch) {
    for (int k = 0; k < 2; ++k) {
      cudaError_t e = launch_batch_pass(p, mode, k, s);
      if (e != cudaSuccess) return e;
      *launches += 1;
    }
    return cudaSuccess;
  }
  for (const Member& m : p->members) {
    fs::KArgs a = make_args(p, m, mode);
    for (int k = 0; k < pass_kinds(m); ++k) {
      cudaError_t e = launch_pass(p, m, a, k, s);
      if (e != cudaSuccess) return e;
      *launches += 1;
    }
  }
  return cudaSuccess;
}

// Pass form 4: `nsteps` steady-state steps of a single 2D FP32 plan in one
// cooperative launch (row pass, grid barrier, column pass per step).
bool fused(const fs_plan* p) { return p->row_form == 4; }
cudaError_t launch_fused(const fs_plan* p, int64_t nsteps, cudaStream_t s) {
  const Member& m = p->members[0];
  const fs::KArgs a = make_args(p, m, 0);
  for (int64_t left = nsteps; left > 0;) {
    const int n = left > (1 << 30) ? (1 << 30) : (int)left;
    cudaError_t e = fs::step2_launch_f32(a, m.tmap_col2, p->gsync, n, s);
    if (e != cudaSuccess) return e;
    left -= n;
  }
  return cudaSuccess;
}

cudaError_t launch_pass(const fs_plan* p, const Member& m, const fs::KArgs& a, int kind, cudaStream_t s) {
  if (kind == 0) return launch_row(p, a, s);
  if (m.prm.ndim == 2) return launch_col(p, m, a, s);
  const int nf = p->nf;
  if (kind == 1) {
    // with c carried (steady state) the y forward skips slot 0
    fs::KArgs b = a;
    const bool skip_c = a.carry3 && a.mode == 0;
    b.plane0 = skip_c ? a.nz : 0;
    const int nslots = skip_c ? nf : nf + 1;
    return p->f64 ? fs::ypass_launch_f64(b, m.tmap_col, -1, nslots, s)
                  : fs::ypass_launch_f32(b, m.tmap_col, -1, nslots, s);
  }
  if (kind == 2) return p->f64 ? fs::zstep_launch_f64(a, m.tmap_z, s) : fs::zstep_launch_f32(a, m.tmap_z, s);
  return p->f64 ? fs::ypass_launch_f64(a, m.tmap_col, 1, nf, s) : fs::ypass_launch_f32(a, m.tmap_col, 1, nf, s);
}

void drop_graph(fs_plan* p) {
  if (p->gexec) cudaGraphExecDestroy(p->gexec);
  p->gexec = nullptr;
  p->gsteps = 0;
}

constexpr int kGraphSteps = 32;

cudaError_t build_graph(fs_plan* p) {
  if (!p->cap_stream) {
    cudaError_t e = cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
  }
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  int64_t dummy = 0;
  cudaError_t el = cudaSuccess;
  for (int i = 0; i < kGraphSteps && el == cudaSuccess; ++i) el = enqueue_step(p, 0, p->cap_stream, &dummy);
  e = cudaStreamEndCapture(p->cap_stream, &g);
  if (el != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return el;
  }
  if (e != cudaSuccess) return e;
  e = cudaGraphInstantiate(&p->gexec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return e;
  p->gsteps = kGraphSteps;
  return cudaSuccess;
}

fs_status read_flag(fs_plan* p) {
  cudaError_t e = cudaMemcpyAsync(p->host_flag, p->flag, sizeof(int), cudaMemcpyDeviceToHost, p->stream);
  if (e != cudaSuccess) return cuda_fail(p, e, "flag read");
  e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) return cuda_fail(p, e, "stream synchronize");
  int f = *p->host_flag;
  if (f) {
    cudaMemsetAsync(p->flag, 0, sizeof(int), p->stream);
    if (f & fs::FS_FLAG_TIMEOUT) {
      cudaMemsetAsync(p->gsync, 0, fs::kStep2SyncBytes, p->stream);  // a fused step may have left a barrier open
      return fail(p, FS_ERR_TIMEOUT, "a bounded device wait timed out");
    }
    if (f & fs::FS_FLAG_NONFINITE) return fail(p, FS_ERR_NONFINITE, "non-finite value in the fields");
    return fail(p, FS_ERR_CUDA, "device reported an index out of bounds");
  }
  return FS_OK;
}

// ---- per-member constant tables --------------------------------------------
// Layout of one member's table block (plan precision T, complex = 2 T):
//   k2x[nx/2 + 1] | k2y[ny] | k2z[nz]        (real, padded to 16 bytes)
//   tw_row | tw_col | tw_z                  (Stockham pass tables, complex)
//   tw_half[nx/2]                           (exp(-2 pi i k / nx), complex)
//   tc_b[2048] (TC precisions only)         (split DFT matrix of the tensor-core stage, 32-bit words)
struct TableLayout {
  size_t k2x, k2y, k2z, tw_row, tw_row_w, tw_col, tw_z, tw_half, tc_b, tw_row2, tw_col2, tw_row2w, tw_col2w,
      total;  // offsets (bytes)
  int Lrow, Erow, Lcol, Ecol, Lz, Ez;
};

size_t align16(size_t v) { return (v + 15) & ~(size_t)15; }
size_t align128(size_t v) { return (v + 127) & ~(size_t)127; }

// Tensor-core DFT stage of a precision (the device's TC mode numbers):
// 0 none, 1 TF32 x 3, 2 BF16 x 3.
constexpr int kTcTf32 = 1, kTcBf16 = 2;
int tc_split(int precision) {
  return precision == FS_F32_TC_TF32 ? kTcTf32 : precision == FS_F32_TC_BF16X3 ? kTcBf16 : 0;
}

// High half of a float in the split the tensor-core stage uses: TF32 (10
// mantissa bits, round to nearest with ties away from zero, as the device's
// cvt.rna.tf32.f32) or BF16 (7 mantissa bits, round to nearest even).
float split_hi(float x, int mode) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  if (mode == kTcTf32) {
    u = (u + 0x1000u) & 0xFFFFE000u;
  } else {
    u += 0x7FFFu + ((u >> 16) & 1u);
    u &= 0xFFFF0000u;
  }
  float r;
  std::memcpy(&r, &u, 4);
  return r;
}

// B = [[Wr, Wi], [-Wi, Wr]] (32 x 32; row kc = input index r, +16 for the
// imaginary half; column nc = output index k, +16 for the imaginary half),
// W[r][k] = exp(-2 pi i r k / 16), split into hi and lo halves:
//   TF32 (tcgen05 kind::tf32): B_hi then B_lo, 1024 words each, in the
//     canonical K-major layout without swizzle that the shared-memory
//     descriptor describes: core matrices of 8 N-rows x 4 K-values (16
//     bytes per row), word offset ((nc / 8) * 8 + kc / 4) * 32 + (nc % 8) * 4
//     + kc % 4 (core matrices 128 bytes apart along K, 1024 along N);
//   BF16 (mma.sync m16n8k16): fragment order, one 16-byte load per lane:
//     [nn < 4][kk < 2][lane][hi pair(k0), hi pair(k0 + 8), lo pair(k0), lo pair(k0 + 8)],
//     k0 = 16 kk + 2 (lane % 4), pair(k) = bf16(B[k][nc]) | bf16(B[k + 1][nc]) << 16.
void tc_table(int mode, uint32_t* out) {
  const long double pi = 3.141592653589793238462643383279502884L;
  float hi[32][32], lo[32][32];
  for (int kc = 0; kc < 32; ++kc)
    for (int nc = 0; nc < 32; ++nc) {
      const int r = kc & 15, pin = kc >> 4, k = nc & 15, pout = nc >> 4;
      const long double ang = 2.0L * pi * (long double)((r * k) % 16) / 16.0L;
      const double wr = (double)cosl(ang), wi = (double)-sinl(ang);
      const double v = (pin == 0) ? (pout == 0 ? wr : wi) : (pout == 0 ? -wi : wr);
      hi[kc][nc] = split_hi((float)v, mode);
      lo[kc][nc] = split_hi((float)(v - (double)hi[kc][nc]), mode);
    }
  auto bits = [](float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    return u;
  };
  auto pair = [&](const float (&m)[32][32], int k, int nc) {
    return (bits(m[k][nc]) >> 16) | (bits(m[k + 1][nc]) & 0xFFFF0000u);
  };
  if (mode == kTcTf32) {
    for (int nc = 0; nc < 32; ++nc)
      for (int kc = 0; kc < 32; ++kc) {
        const int w = ((nc / 8) * 8 + kc / 4) * 32 + (nc % 8) * 4 + kc % 4;
        out[w] = bits(hi[kc][nc]);
        out[1024 + w] = bits(lo[kc][nc]);
      }
    return;
  }
  const int nkk = 2;
  for (int nn = 0; nn < 4; ++nn)
    for (int kk = 0; kk < nkk; ++kk)
      for (int lane = 0; lane < 32; ++lane) {
        const int nc = 8 * nn + lane / 4, t4 = lane % 4;
        uint32_t* w = out + (((nn * nkk + kk) * 32 + lane) * 4);
        const int k0 = 16 * kk + 2 * t4;
        w[0] = pair(hi, k0, nc);
        w[1] = pair(hi, k0 + 8, nc);
        w[2] = pair(lo, k0, nc);
        w[3] = pair(lo, k0 + 8, nc);
      }
}

// Rows of 1024 in FP32 run the x-pass variant with 32 values per thread.
bool wide_rows(const fs_params& prm, bool f64) { return !f64 && prm.n[0] == 1024; }

TableLayout table_layout(const fs_params& prm, bool f64) {
  TableLayout t{};
  const size_t rs = f64 ? 8 : 4, cs = 2 * rs;
  int nx = prm.n[0], ny = prm.n[1], nz = prm.ndim > 2 ? prm.n[2] : 1;
  t.Lrow = nx / 2;
  t.Erow = fs::row_E(t.Lrow, f64);
  t.Lcol = ny;
  t.Ecol = fs::col_E(ny, f64);
  t.Lz = nz;
  t.Ez = fs::col_E(nz, f64);
  size_t o = 0;
  t.k2x = o;
  o = align16(o + rs * (nx / 2 + 1));
  t.k2y = o;
  o = align16(o + rs * ny);
  t.k2z = o;
  o = align16(o + rs * nz);
  t.tw_row = o;
  o = align16(o + cs * fs::pass_table_size(t.Lrow, t.Erow));
  t.tw_row_w = o;  // wide x-pass variant (32 values per thread): FP32 rows of 1024
  o = align16(o + (wide_rows(prm, f64) ? cs * fs::pass_table_size(t.Lrow, 32) : 0));
  t.tw_col = o;
  o = align16(o + cs * fs::pass_table_size(t.Lcol, t.Ecol));
  t.tw_z = o;
  o = align16(o + cs * (nz > 1 ? fs::pass_table_size(t.Lz, t.Ez) : 0));
  t.tw_half = o;
  o = align16(o + cs * (nx / 2));
  t.tc_b = o;
  o = align16(o + (tc_split(prm.precision) ? 2048 * sizeof(float) : 0));
  t.tw_row2 = o;  // pair-form row pass: L = nx, E = nx / 32
  o = align16(o + (row2_form(prm, f64) ? cs * fs::pass_table_size(nx, nx / 32) : 0));
  t.tw_col2 = o;  // warp-per-column pass: L = ny, E = ny / 32 (up to 1024 points)
  o = align16(o + (col2_form(prm, f64) && ny <= 1024 ? cs * fs::pass_table_size(ny, ny / 32) : 0));
  t.tw_row2w = o;  // two warps per line: E = nx / 64, ny / 64
  o = align16(o + (row2_form(prm, f64) && nx >= 128 ? cs * fs::pass_table_size(nx, nx / 64) : 0));
  t.tw_col2w = o;
  o = align16(o + (col2_form(prm, f64) && ny >= 128 ? cs * fs::pass_table_size(ny, ny / 64) : 0));
  t.total = o;
  return t;
}

size_t member_table_bytes(const fs_params& prm, bool f64) { return table_layout(prm, f64).total; }

// Stockham pass tables of a line FFT of length L with E values per thread:
// for every pass after the first (sub-length NS, radix R = min(E, L/NS)),
// entries [r][j] = exp(-2 pi i r j / (NS R)), r < R, j < NS.
void pass_table(int L, int E, std::vector<long double>& re, std::vector<long double>& im) {
  const long double pi = 3.141592653589793238462643383279502884L;
  for (int ns = 1; ns < L;) {
    int r = E < L / ns ? E : L / ns;
    if (ns > 1)
      for (int q = 0; q < r; ++q)
        for (int j = 0; j < ns; ++j) {
          long long e = (long long)q * j % ((long long)ns * r);
          long double ang = 2.0L * pi * (long double)e / (long double)(ns * r);
          re.push_back(cosl(ang));
          im.push_back(-sinl(ang));
        }
    ns *= r;
  }
}

template <typename T>
void put_real(std::vector<char>& buf, size_t off, const std::vector<double>& v) {
  T* d = reinterpret_cast<T*>(buf.data() + off);
  for (size_t i = 0; i < v.size(); ++i) d[i] = (T)v[i];
}
template <typename T>
void put_cplx(std::vector<char>& buf, size_t off, const std::vector<long double>& re,
              const std::vector<long double>& im) {
  T* d = reinterpret_cast<T*>(buf.data() + off);
  for (size_t i = 0; i < re.size(); ++i) {
    d[2 * i] = (T)re[i];
    d[2 * i + 1] = (T)im[i];
  }
}

cudaError_t upload_tables(Member& m, bool f64, char* dev, size_t bytes) {
  const fs_params& prm = m.prm;
  TableLayout t = table_layout(prm, f64);
  std::vector<char> buf(bytes, 0);
  int nx = prm.n[0], ny = prm.n[1], nz = prm.ndim > 2 ? prm.n[2] : 1;
  std::vector<double> kx(nx / 2 + 1), ky(ny), kz(nz, 0.0);
  for (int k = 0; k <= nx / 2; ++k) kx[k] = axis_k2(prm.lap, k, nx, prm.dx[0]);
  for (int k = 0; k < ny; ++k) ky[k] = axis_k2(prm.lap, k, ny, prm.dx[1]);
  for (int k = 0; k < nz && prm.ndim > 2; ++k) kz[k] = axis_k2(prm.lap, k, nz, prm.dx[2]);
  std::vector<long double> rr, ii, wr, wi, cr, ci, zr, zi, hr, hi, r2r, r2i, c2r, c2i, r3r, r3i, c3r, c3i;
  if (row2_form(prm, f64)) pass_table(nx, nx / 32, r2r, r2i);
  if (col2_form(prm, f64) && ny <= 1024) pass_table(ny, ny / 32, c2r, c2i);
  if (row2_form(prm, f64) && nx >= 128) pass_table(nx, nx / 64, r3r, r3i);
  if (col2_form(prm, f64) && ny >= 128) pass_table(ny, ny / 64, c3r, c3i);
  pass_table(t.Lrow, t.Erow, rr, ii);
  if (wide_rows(prm, f64)) pass_table(t.Lrow, 32, wr, wi);
  pass_table(t.Lcol, t.Ecol, cr, ci);
  if (nz > 1) pass_table(t.Lz, t.Ez, zr, zi);
  const long double pi = 3.141592653589793238462643383279502884L;
  for (int k = 0; k < nx / 2; ++k) {
    long double ang = 2.0L * pi * (long double)k / (long double)nx;
    hr.push_back(cosl(ang));
    hi.push_back(-sinl(ang));
  }
  if (f64) {
    put_real<double>(buf, t.k2x, kx);
    put_real<double>(buf, t.k2y, ky);
    put_real<double>(buf, t.k2z, kz);
    put_cplx<double>(buf, t.tw_row, rr, ii);
    put_cplx<double>(buf, t.tw_col, cr, ci);
    put_cplx<double>(buf, t.tw_z, zr, zi);
    put_cplx<double>(buf, t.tw_half, hr, hi);
  } else {
    put_real<float>(buf, t.k2x, kx);
    put_real<float>(buf, t.k2y, ky);
    put_real<float>(buf, t.k2z, kz);
    put_cplx<float>(buf, t.tw_row, rr, ii);
    put_cplx<float>(buf, t.tw_row_w, wr, wi);
    put_cplx<float>(buf, t.tw_col, cr, ci);
    put_cplx<float>(buf, t.tw_z, zr, zi);
    put_cplx<float>(buf, t.tw_half, hr, hi);
    put_cplx<float>(buf, t.tw_row2, r2r, r2i);
    put_cplx<float>(buf, t.tw_col2, c2r, c2i);
    put_cplx<float>(buf, t.tw_row2w, r3r, r3i);
    put_cplx<float>(buf, t.tw_col2w, c3r, c3i);
  }
  m.k2x = dev + t.k2x;
  m.k2y = dev + t.k2y;
  m.k2z = dev + t.k2z;
  m.tw_row = dev + t.tw_row;
  m.tw_row_w = wide_rows(prm, f64) ? dev + t.tw_row_w : nullptr;
  m.tw_col = dev + t.tw_col;
  m.tw_z = dev + t.tw_z;
  m.tw_half = dev + t.tw_half;
  m.tw_row2 = row2_form(prm, f64) ? dev + t.tw_row2 : nullptr;
  m.tw_col2 = col2_form(prm, f64) && ny <= 1024 ? dev + t.tw_col2 : nullptr;
  m.tw_row2w = row2_form(prm, f64) && nx >= 128 ? dev + t.tw_row2w : nullptr;
  m.tw_col2w = col2_form(prm, f64) && ny >= 128 ? dev + t.tw_col2w : nullptr;
  if (const int mode = tc_split(prm.precision)) {
    tc_table(mode, reinterpret_cast<uint32_t*>(buf.data() + t.tc_b));
    m.tc_b = dev + t.tc_b;
  }
  return cudaMemcpy(dev, buf.data(), bytes, cudaMemcpyHostToDevice);
}

// ---- batched ensemble set-up ------------------------------------------------
// Work lists in execution order (largest simulation first), argument blocks
// for both row-pass modes, the column tensor maps, and the shared-memory size
// of the largest member.  Requires 2D spectral-FS members whose column pass
// fits the 256-thread batch CTA.
fs_status setup_batch(fs_plan* p) {
  const int nm = (int)p->members.size();
  for (const Member& m : p->members) {
    if (m.prm.ndim != 2 || m.prm.scheme != FS_SCHEME_SEMI_IMPLICIT_FS)
      return fail(nullptr, FS_ERR_UNSUPPORTED, "batched plans hold 2D semi-implicit FS members");
    const int nx = m.prm.n[0], ny = m.prm.n[1];
    const int tk = p->f64 ? fs::col_batch_tk_f64(nx, ny) : fs::col_batch_tk_f32(nx, ny);
    if (nx < 16 || nx > 1024 || ny > 1024 || tk == 0)
      return fail(nullptr, FS_ERR_UNSUPPORTED,
                  "batched members need 16 <= nx <= 1024 and ny in [128 (FP32) / 64 (FP64), 1024]");
    if (m.prm.precision == FS_F32_TC_TF32 || m.prm.precision == FS_F32_TC_BF16X3)
      return fail(nullptr, FS_ERR_UNSUPPORTED, "batched plans use the CUDA-core transforms (FS_F64 or FS_F32)");
  }
  std::vector<int> order(nm);
  for (int i = 0; i < nm; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(),
                   [p](int a, int b) { return p->members[a].npts > p->members[b].npts; });
  std::vector<fs::KArgs> k0(nm), k1(nm);
  std::vector<CUtensorMap> maps(nm);
  std::vector<long long> rb(nm + 1, 0), cb(nm + 1, 0);
  std::vector<int> tiles(nm);
  size_t rsm = 0, csm = 0;
  // warp-per-line form: every member FP32 with both axes in [64, 1024]
  bool v2 = !p->f64;
  for (const Member& m : p->members) v2 = v2 && m.tw_row2 && m.tw_col2;
  std::vector<CUtensorMap> maps2(nm);
  std::vector<long long> rb2(nm + 1, 0), cb2(nm + 1, 0);
  std::vector<int> pairs2(nm, 0);
  size_t rsm2 = 0, csm2 = 0;
  p->batch = true;  // make_args: ensemble members keep both forms' tables
  for (int e = 0; e < nm; ++e) {
    const Member& m = p->members[order[e]];
    const int nx = m.prm.n[0], ny = m.prm.n[1];
    k0[e] = make_args(p, m, 0);
    k1[e] = make_args(p, m, 1);
    maps[e] = m.tmap_col;
    const long long blocks = p->f64 ? fs::row_blocks_f64(nx, ny) : fs::row_blocks_f32(nx, ny);
    const int tk = p->f64 ? fs::col_batch_tk_f64(nx, ny) : fs::col_batch_tk_f32(nx, ny);
    tiles[e] = nx / 2 / tk;
    rb[e + 1] = rb[e] + blocks;
    cb[e + 1] = cb[e] + (long long)tiles[e] * p->nf;
    rsm = std::max(rsm, p->f64 ? fs::row_smem_f64(nx, p->nf) : fs::row_smem_f32(nx, p->nf));
    csm = std::max(csm, p->f64 ? fs::col_smem_f64(ny, tk) : fs::col_smem_f32(ny, tk));
    if (v2) {
      maps2[e] = m.tmap_col2;
      pairs2[e] = nx / 4;  // nx / 2 columns, two per item
      rb2[e + 1] = rb2[e] + ny / 2;
      cb2[e + 1] = cb2[e] + (long long)pairs2[e] * fs::col2_groups(p->nf);
      rsm2 = std::max(rsm2, fs::row2_smem_f32(nx, p->nf));
      csm2 = std::max(csm2, fs::col2_smem_f32(ny));
    }
  }
  const size_t o_maps = 0, o_k0 = align16(o_maps + sizeof(CUtensorMap) * nm);
  const size_t o_k1 = align16(o_k0 + sizeof(fs::KArgs) * nm), o_rb = align16(o_k1 + sizeof(fs::KArgs) * nm);
  const size_t o_cb = align16(o_rb + sizeof(long long) * (nm + 1));
  // tensor maps read by TMA from global memory must be 64-byte aligned: both
  // map arrays start on 128 bytes (the block itself is 256-byte aligned)
  const size_t o_t = align16(o_cb + sizeof(long long) * (nm + 1)), o_m2 = align128(o_t + sizeof(int) * nm);
  const size_t o_rb2 = align16(o_m2 + sizeof(CUtensorMap) * nm), o_cb2 = align16(o_rb2 + sizeof(long long) * (nm + 1));
  const size_t o_p2 = align16(o_cb2 + sizeof(long long) * (nm + 1)), total = align16(o_p2 + sizeof(int) * nm);
  char* dev = (char*)plan_alloc(p, total);
  if (!dev) return fail(nullptr, FS_ERR_OOM, "device workspace allocation failed");
  if (((uintptr_t)(dev + o_maps) % 64) || ((uintptr_t)(dev + o_m2) % 64))
    return fail(nullptr, FS_ERR_CUDA, "tensor maps of the ensemble are not 64-byte aligned");
  std::vector<char> host(total, 0);
  std::memcpy(host.data() + o_maps, maps.data(), sizeof(CUtensorMap) * nm);
  std::memcpy(host.data() + o_k0, k0.data(), sizeof(fs::KArgs) * nm);
  std::memcpy(host.data() + o_k1, k1.data(), sizeof(fs::KArgs) * nm);
  std::memcpy(host.data() + o_rb, rb.data(), sizeof(long long) * (nm + 1));
  std::memcpy(host.data() + o_cb, cb.data(), sizeof(long long) * (nm + 1));
  std::memcpy(host.data() + o_t, tiles.data(), sizeof(int) * nm);
  std::memcpy(host.data() + o_m2, maps2.data(), sizeof(CUtensorMap) * nm);
  std::memcpy(host.data() + o_rb2, rb2.data(), sizeof(long long) * (nm + 1));
  std::memcpy(host.data() + o_cb2, cb2.data(), sizeof(long long) * (nm + 1));
  std::memcpy(host.data() + o_p2, pairs2.data(), sizeof(int) * nm);
  cudaError_t e = cudaMemcpy(dev, host.data(), total, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "batch tables");
  fs::BatchArgs& b = p->bargs;
  b.maps = reinterpret_cast<const CUtensorMap*>(dev + o_maps);
  b.mem = reinterpret_cast<const fs::KArgs*>(dev + o_k0);
  b.mem_col = b.mem;
  p->bmem1 = reinterpret_cast<const fs::KArgs*>(dev + o_k1);
  b.row_begin = reinterpret_cast<const long long*>(dev + o_rb);
  b.col_begin = reinterpret_cast<const long long*>(dev + o_cb);
  b.col_tiles = reinterpret_cast<const int*>(dev + o_t);
  b.nm = nm;
  b.nf1 = p->nf + 1;
  b.row_total = rb[nm];
  b.col_total = cb[nm];
  b.row_grid = b.row_total;  // until tuned: one CTA per item
  b.col_grid = b.col_total;
  b.row_smem = rsm;
  b.col_smem = csm;
  b.row_form = b.col_form = 1;  // until tuned
  if (v2) {
    b.maps2 = reinterpret_cast<const CUtensorMap*>(dev + o_m2);
    b.row2_begin = reinterpret_cast<const long long*>(dev + o_rb2);
    b.col2_begin = reinterpret_cast<const long long*>(dev + o_cb2);
    b.col2_pairs = reinterpret_cast<const int*>(dev + o_p2);
    b.row2_total = rb2[nm];
    b.col2_total = cb2[nm];
    b.row2_grid = b.row2_total;
    b.col2_grid = b.col2_total;
    b.row2_smem = rsm2;
    b.col2_smem = csm2;
  }
  return FS_OK;
}

// Autotuner of the batched launches.  For each pass it times every form the
// ensemble supports -- the half-length row / column-tile kernels (radix-16
// line transforms, column tiles of col_tk columns) and, for FP32 members with
// both axes in [64, 1024], the warp-per-line kernels (radix-32 / 16 / 8 ...
// line transforms held by one warp, two-column tiles) -- at the persistent
// grid sizes {1, 2, 3, 4, 5, 6, 8, 16} x SMs and one CTA per work item, and
// keeps the fastest (form, grid) pair.  Runs on the state just set (row pass
// from the real fields, column pass on its output), which it leaves
// unchanged.
cudaError_t autotune_batch(fs_plan* p) {
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int mult[] = {1, 2, 3, 4, 5, 6, 8, 16};
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) return e;
  fs::BatchArgs& b = p->bargs;
  const bool v2 = b.maps2 != nullptr;
  // the column pass is timed on the output of a row pass in the current row form
  b.row_form = 1;
  for (int kind = 0; kind < 2 && e == cudaSuccess; ++kind) {
    float best = 1e30f;
    int best_form = 1;
    long long best_g = 0;
    const int pinned = kind == 0 ? p->row_form : p->col_form;  // fs_set_pass_forms, 0: free
    for (int form = 1; form <= (v2 ? 2 : 1) && e == cudaSuccess; ++form) {
      if (pinned && form != pinned) continue;
      const long long total = kind == 0 ? (form == 2 ? b.row2_total : b.row_total)
                                        : (form == 2 ? b.col2_total : b.col_total);
      std::vector<long long> cand;
      for (int mm : mult)
        if ((long long)mm * sms < total) cand.push_back((long long)mm * sms);
      cand.push_back(total);
      for (long long g : cand) {
        if (kind == 0) {
          b.row_form = form;
          (form == 2 ? b.row2_grid : b.row_grid) = g;
        } else {
          b.col_form = form;
          (form == 2 ? b.col2_grid : b.col_grid) = g;
        }
        float acc = 0.f;
        for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
          if (kind == 1) e = launch_batch_pass(p, 1, 0, p->stream);  // fresh column input
          if (e == cudaSuccess) e = cudaEventRecord(e0, p->stream);
          if (e == cudaSuccess) e = launch_batch_pass(p, 1, kind, p->stream);
          if (e == cudaSuccess) e = cudaEventRecord(e1, p->stream);
          if (e == cudaSuccess) e = cudaEventSynchronize(e1);
          float t = 0.f;
          if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
          if (rep > 0) acc += t;  // first repetition warms up
        }
        if (acc < best) {
          best = acc;
          best_form = form;
          best_g = g;
        }
      }
    }
    if (kind == 0) {
      b.row_form = best_form;
      (best_form == 2 ? b.row2_grid : b.row_grid) = best_g;
    } else {
      b.col_form = best_form;
      (best_form == 2 ? b.col2_grid : b.col_grid) = best_g;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e == cudaSuccess) p->tuned = true;
  return e;
}

fs_status create_common(const fs_params* each, int count, void* stream, fs_alloc_fn alloc, fs_free_fn dealloc,
                        void* ctx, fs_plan_t* out) {
  if (!out) return fail(nullptr, FS_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!each || count <= 0) return fail(nullptr, FS_ERR_INVALID_ARG, "no simulations given");
  for (int i = 0; i < count; ++i) {
    std::string why;
    fs_status s = validate(&each[i], &why);
    if (s != FS_OK) return fail(nullptr, s, count > 1 ? "member " + std::to_string(i) + ": " + why : why);
    if (each[i].precision != each[0].precision || each[i].p != each[0].p ||
        each[i].scheme != each[0].scheme)
      return fail(nullptr, FS_ERR_INVALID_ARG, "batch members must share precision, p and scheme");
  }
  if ((alloc == nullptr) != (dealloc == nullptr))
    return fail(nullptr, FS_ERR_INVALID_ARG, "alloc and dealloc must both be given or both NULL");

  fs_plan* p = new fs_plan();
  p->f64 = each[0].precision == FS_F64;
  p->fd = each[0].scheme == FS_SCHEME_EXPLICIT_FD;
  p->nf = 1 + each[0].p;
  p->stream = reinterpret_cast<cudaStream_t>(stream);
  p->alloc = alloc;
  p->dealloc = dealloc;
  p->actx = ctx;
  const size_t rs = p->f64 ? sizeof(double) : sizeof(float);
  const size_t cs = 2 * rs;

  // Workspace first (through the allocator hook), then tables.
  p->members.resize(count);
  std::vector<size_t> table_bytes(count);
  for (int i = 0; i < count; ++i) {
    Member& m = p->members[i];
    m.prm = each[i];
    m.npts = 1;
    for (int d = 0; d < m.prm.ndim; ++d) m.npts *= m.prm.n[d];
    m.slot_stride = m.npts / 2;
    m.spec = plan_alloc(p, (size_t)(p->nf + 1) * m.slot_stride * cs);
    m.real = plan_alloc(p, (size_t)p->nf * m.npts * rs);
    table_bytes[i] = member_table_bytes(m.prm, p->f64);
    char* tb = (char*)plan_alloc(p, table_bytes[i]);
    m.csum = (double*)plan_alloc(p, sizeof(double) * 8);
    if (!m.spec || !m.real || !tb || !m.csum) {
      plan_free_all(p);
      delete p;
      return fail(nullptr, FS_ERR_OOM, "device workspace allocation failed");
    }
    m.k2x = tb;  // the rest of the table pointers are set by upload_tables
  }
  p->flag = (int*)plan_alloc(p, 256);
  p->acc = (double*)plan_alloc(p, 256);
  p->gsync = (unsigned*)plan_alloc(p, fs::kStep2SyncBytes);
  if (!p->flag || !p->acc || !p->gsync) {
    plan_free_all(p);
    delete p;
    return fail(nullptr, FS_ERR_OOM, "device workspace allocation failed");
  }
  cudaError_t e = cudaMallocHost(&p->host_flag, sizeof(int));
  if (e != cudaSuccess) {
    plan_free_all(p);
    delete p;
    return cuda_fail(nullptr, e, "cudaMallocHost");
  }
  for (int i = 0; i < count && e == cudaSuccess; ++i) {
    e = upload_tables(p->members[i], p->f64, (char*)p->members[i].k2x, table_bytes[i]);
    if (e == cudaSuccess) e = cudaMemset(p->members[i].csum, 0, sizeof(double) * 8);
    if (e == cudaSuccess && !encode_col_map(p->members[i], p->nf + 1, p->f64)) e = cudaErrorInvalidValue;
  }
  if (e == cudaSuccess) e = cudaMemset(p->flag, 0, 256);
  if (e == cudaSuccess) e = cudaMemset(p->gsync, 0, fs::kStep2SyncBytes);
  if (e != cudaSuccess) {
    fs_status s = cuda_fail(nullptr, e, "plan tables");
    cudaFreeHost(p->host_flag);
    plan_free_all(p);
    delete p;
    return s;
  }
  if (count > 1) {
    fs_status s = setup_batch(p);
    if (s != FS_OK) {
      cudaFreeHost(p->host_flag);
      plan_free_all(p);
      delete p;
      return s;
    }
  }
  *out = p;
  return FS_OK;
}

}  // namespace

extern "C" {

fs_status fs_plan_create(const fs_params* prm, void* stream, fs_plan_t* out) {
  return create_common(prm, 1, stream, nullptr, nullptr, nullptr, out);
}

fs_status fs_plan_create_ex(const fs_params* prm, void* stream, fs_alloc_fn alloc, fs_free_fn dealloc, void* ctx,
                            fs_plan_t* out) {
  return create_common(prm, 1, stream, alloc, dealloc, ctx, out);
}

fs_status fs_batch_create(const fs_params* each, int count, void* stream, fs_plan_t* out) {
  return create_common(each, count, stream, nullptr, nullptr, nullptr, out);
}

// Copies nf fields of n bytes each between the plan's contiguous field block
// `dev` and the caller's nf pointers; runs of caller pointers that are
// themselves contiguous go in one copy.
cudaError_t copy_fields(char* dev, const void* const* ptrs, int nf, size_t n, bool to_dev, cudaStream_t s) {
  for (int f = 0; f < nf;) {
    int g = f + 1;
    while (g < nf && (const char*)ptrs[g] == (const char*)ptrs[g - 1] + n) ++g;
    cudaError_t e = to_dev ? cudaMemcpyAsync(dev + f * n, ptrs[f], (g - f) * n, cudaMemcpyDefault, s)
                           : cudaMemcpyAsync(const_cast<void*>(ptrs[f]), dev + f * n, (g - f) * n,
                                             cudaMemcpyDefault, s);
    if (e != cudaSuccess) return e;
    f = g;
  }
  return cudaSuccess;
}

fs_status fs_set_fields(fs_plan_t p, const void* const* fields) {
  if (!p) return fail(nullptr, FS_ERR_INVALID_ARG, "plan is NULL");
  if (!fields) return fail(p, FS_ERR_INVALID_ARG, "fields is NULL");
  const size_t rs = p->f64 ? sizeof(double) : sizeof(float);
  for (size_t i = 0; i < p->members.size() * p->nf; ++i)
    if (!fields[i]) return fail(p, FS_ERR_INVALID_ARG, "field pointer is NULL");
  int idx = 0;
  for (Member& m : p->members) {
    cudaError_t ec = copy_fields((char*)m.real, fields + idx, p->nf, m.npts * rs, true, p->stream);
    if (ec != cudaSuccess) return cuda_fail(p, ec, "fs_set_fields copy");
    idx += p->nf;
    m.fd_cur = 0;
    if (!p->f64 && !p->fd) {
      cudaError_t e = cudaMemsetAsync(m.csum, 0, sizeof(double), p->stream);
      if (e == cudaSuccess) e = fs::sum_launch_f32(m.real, m.npts, m.csum, p->stream);
      if (e != cudaSuccess) return cuda_fail(p, e, "fs_set_fields mean carry");
    }
  }
  p->state = kStateReal;
  if (p->batch && !p->tuned) {
    cudaError_t e = autotune_batch(p);
    if (e != cudaSuccess) return cuda_fail(p, e, "batch autotune");
    drop_graph(p);
  }
  return FS_OK;
}

fs_status fs_step_async(fs_plan_t p, int64_t nsteps) {
  if (!p) return fail(nullptr, FS_ERR_INVALID_ARG, "plan is NULL");
  if (nsteps < 0) return fail(p, FS_ERR_INVALID_ARG, "nsteps < 0");
  if (p->state == kStateNone) return fail(p, FS_ERR_STATE, "fs_step before fs_set_fields");
  int64_t launches = 0;
  int64_t done = 0;
  cudaError_t e = cudaSuccess;
  if (nsteps > 0 && p->state == kStateReal && !p->fd) {
    e = enqueue_step(p, 1, p->stream, &launches);
    if (e != cudaSuccess) return cuda_fail(p, e, "step launch");
    done = 1;
    p->state = kStateSpec;
  }
  int64_t left = nsteps - done;
  if (left > 0 && fused(p)) {
    e = launch_fused(p, left, p->stream);
    if (e != cudaSuccess) return cuda_fail(p, e, "fused step launch");
    launches += 1;
    left = 0;
  }
  if (left >= kGraphSteps && !p->fd) {
    if (!p->gexec) {
      e = build_graph(p);
      if (e != cudaSuccess) return cuda_fail(p, e, "graph capture");
    }
    while (left >= p->gsteps) {
      e = cudaGraphLaunch(p->gexec, p->stream);
      if (e != cudaSuccess) return cuda_fail(p, e, "graph launch");
      left -= p->gsteps;
      launches += (int64_t)p->gsteps * 2 * (int64_t)p->members.size();
    }
  }
  for (; left > 0; --left) {
    e = enqueue_step(p, 0, p->stream, &launches);
    if (e != cudaSuccess) return cuda_fail(p, e, "step launch");
  }
  if (nsteps > 0 && !p->fd) p->state = kStateSpec;
  p->last_launches = launches;
  return FS_OK;
}

fs_status fs_sync(fs_plan_t p) {
  if (!p) return fail(nullptr, FS_ERR_INVALID_ARG, "plan is NULL");
  return read_flag(p);
}

fs_status fs_step(fs_plan_t p, int64_t nsteps) {
  fs_status s = fs_step_async(p, nsteps);
  if (s != FS_OK) return s;
  return read_flag(p);
}

fs_status fs_get_fields(fs_plan_t p, void* const* out) {
  if (!p) return fail(nullptr, FS_ERR_INVALID_ARG, "plan is NULL");
  if (!out) return fail(p, FS_ERR_INVALID_ARG, "fields_out is NULL");
  if (p->state == kStateNone) return fail(p, FS_ERR_STATE, "fs_get_fields before fs_set_fields");
  if (p->state == kStateSpec && !p->fd) {
    for (const Member& m : p->members) {
      fs::KArgs a = make_args(p, m, 2);
      cudaError_t e = launch_row(p, a, p->stream);
      if (e != cudaSuccess) return cuda_fail(p, e, "inverse row pass");
    }
    p->state = kStateBoth;  // the spectra stay valid: the next step carries on from them
  }
  const size_t rs = p->f64 ? sizeof(double) : sizeof(float);
  for (size_t i = 0; i < p->members.size() * p->nf; ++i)
    if (!out[i]) return fail(p, FS_ERR_INVALID_ARG, "output pointer is NULL");
  int idx = 0;
  for (const Member& m : p->members) {
    char* src = (char*)(p->fd ? fd_buf(m, m.fd_cur) : m.real);
    cudaError_t e = copy_fields(src, out + idx, p->nf, m.npts * rs, false, p->stream);
    if (e != cudaSuccess) return cuda_fail(p, e, "fs_get_fields copy");
    idx += p->nf;
  }
  cudaError_t e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) return cuda_fail(p, e, "stream synchronize");
  return FS_OK;
}

fs_status fs_set_params(fs_plan_t p, const fs_params* prm) {
  if (!p) return fail(nullptr, FS_ERR_INVALID_ARG, "plan is NULL");
  if (p->members.size() != 1) return fail(p, FS_ERR_UNSUPPORTED, "fs_set_params on a batch plan");
  std::string why;
  fs_status s = validate(prm, &why);
  if (s != FS_OK) return fail(p, s, why);
  const fs_params& o = p->members[0].prm;
  bool same = prm->ndim == o.ndim && prm->p == o.p && prm->precision == o.precision && prm->lap == o.lap &&
              prm->scheme == o.scheme;
  for (int d = 0; d < o.ndim; ++d) same = same && prm->n[d] == o.n[d] && prm->dx[d] == o.dx[d];
  if (!same) return fail(p, FS_ERR_INVALID_ARG, "fs_set_params may change only physical parameters and dt");
  p->members[0].prm = *prm;
  drop_graph(p);
  return FS_OK;
}

fs_status fs_set_stream(fs_plan_t p, void* stream) {
  if (!p) return fail(nullptr, FS_ERR_INVALID_ARG, "plan is NULL");
  p->stream = reinterpret_cast<cudaStream_t>(stream);
  return FS_OK;
}

fs_status fs_free_energy(fs_plan_t p, double* F, double* parts) {
  if (!p) return fail(nullptr, FS_ERR_INVALID_ARG, "plan is NULL");
  if (!F) return fail(p, FS_ERR_INVALID_ARG, "F is NULL");
  if (p->state == kStateNone) return fail(p, FS_ERR_STATE, "fs_free_energy before fs_set_fields");
  const Member& m = p->members[0];
  if (p->members.size() != 1 || p->fd)
    return fail(p, FS_ERR_UNSUPPORTED, "fs_free_energy is built for single semi-implicit FS plans");
  cudaError_t e = cudaSuccess;
  if (p->state == kStateSpec) {
    e = launch_row(p, make_args(p, m, 2), p->stream);
    if (e != cudaSuccess) return cuda_fail(p, e, "inverse row pass");
  }
  p->state = kStateReal;  // the diagnostic overwrites the spectra
  const int nparts = 2 + m.prm.p;
  e = cudaMemsetAsync(p->acc, 0, sizeof(double) * nparts, p->stream);
  fs::KArgs a = make_args(p, m, 3);
  if (e == cudaSuccess) e = launch_row(p, a, p->stream);  // chemical sum, 2 x^(phi) of every field
  if (m.prm.ndim == 2) {
    if (e == cudaSuccess)
      e = p->f64 ? fs::energy_col_launch_f64(a, m.tmap_col, p->stream)
                 : fs::energy_col_launch_f32(a, m.tmap_col, p->stream);
  } else {
    // 3D: forward y of slots 0..nf-1 (column packing), then z and the weighted sums
    fs::KArgs b = a;
    b.plane0 = 0;
    if (e == cudaSuccess)
      e = p->f64 ? fs::ypass_launch_f64(b, m.tmap_col, -1, p->nf, p->stream)
                 : fs::ypass_launch_f32(b, m.tmap_col, -1, p->nf, p->stream);
    if (e == cudaSuccess)
      e = p->f64 ? fs::energy_z_launch_f64(a, m.tmap_z, p->stream) : fs::energy_z_launch_f32(a, m.tmap_z, p->stream);
  }
  double h[8] = {0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, p->acc, sizeof(double) * nparts, cudaMemcpyDeviceToHost, p->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) return cuda_fail(p, e, "fs_free_energy");
  double dV = 1.0;
  for (int d = 0; d < m.prm.ndim; ++d) dV *= m.prm.dx[d];
  const double N = (double)m.npts;
  double total = h[0] * dV;
  if (parts) parts[0] = h[0] * dV;
  for (int f = 0; f < 1 + m.prm.p; ++f) {
    const double kap = f == 0 ? m.prm.kappa_c : m.prm.kappa_eta;
    const double term = 0.5 * kap * (h[1 + f] / (4.0 * N)) * dV;  // Parseval; spectra carry a factor 2
    if (parts) parts[1 + f] = term;
    total += term;
  }
  *F = total;
  return read_flag(p);
}

fs_status fs_step_adjoint(fs_plan_t p, const void* const* u, const void* const* lam_in, void* const* lam_out,
                          double grad[4]) {
  if (!p) return fail(nullptr, FS_ERR_INVALID_ARG, "plan is NULL");
  if (!u || !lam_in || !lam_out) return fail(p, FS_ERR_INVALID_ARG, "field pointer array is NULL");
  Member& m = p->members[0];
  if (p->members.size() != 1 || p->fd)
    return fail(p, FS_ERR_UNSUPPORTED, "fs_step_adjoint is built for single semi-implicit FS plans");
  const bool three = m.prm.ndim == 3;
  if (!three && (m.prm.n[0] > 1024 || m.prm.n[1] > 1024))
    return fail(p, FS_ERR_UNSUPPORTED, "fs_step_adjoint supports 2D axes up to 1024");
  const size_t rs = p->f64 ? sizeof(double) : sizeof(float), cs = 2 * rs;
  const int nf = p->nf;
  if (!m.aspec) {
    m.aspec = plan_alloc(p, (size_t)3 * nf * m.slot_stride * cs);
    m.alam = plan_alloc(p, (size_t)nf * m.npts * rs);
    m.au = plan_alloc(p, (size_t)nf * m.npts * rs);
    m.aout = plan_alloc(p, (size_t)nf * m.npts * rs);
    if (!m.aspec || !m.alam || !m.au || !m.aout) return fail(p, FS_ERR_OOM, "adjoint workspace allocation failed");
    EncodeTiledFn enc = encode_tiled();
    const int units = p->f64 ? 2 : 1, nx = m.prm.n[0], ny = m.prm.n[1], nz = three ? m.prm.n[2] : 1;
    const cuuint64_t W = (cuuint64_t)(nx / 2) * units;
    auto encode = [&](CUtensorMap* map, cuuint32_t rank, const cuuint64_t* dims, const cuuint64_t* strides,
                      const cuuint32_t* box) {
      const cuuint32_t estr[4] = {1, 1, 1, 1};
      return enc && enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, rank, m.aspec, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    // 2D: [slot][y][kx] column tiles; 3D: [slot nz + z][y][kx] tiles of the
    // y passes and [slot][z][y][kx] z lines
    const int tk = three ? (p->f64 ? fs::line_tile_width_f64(nx, ny) : fs::line_tile_width_f32(nx, ny))
                         : fs::col_tile_width(p->f64, nx, ny);
    const cuuint64_t dims[3] = {W, (cuuint64_t)ny, (cuuint64_t)nz * 3 * nf};
    const cuuint64_t strides[2] = {W * 8, W * 8 * ny};
    const cuuint32_t box[3] = {(cuuint32_t)(tk * units), (cuuint32_t)(ny < 256 ? ny : 256), 1};
    bool ok = encode(&m.tmap_adj, 3, dims, strides, box);
    if (ok && three) {
      const int tkz = p->f64 ? fs::line_tile_width_f64(nx, nz) : fs::line_tile_width_f32(nx, nz);
      const cuuint64_t dz[4] = {W, (cuuint64_t)ny, (cuuint64_t)nz, (cuuint64_t)(3 * nf)};
      const cuuint64_t sz[3] = {W * 8, W * 8 * ny, W * 8 * ny * nz};
      const cuuint32_t bz[4] = {(cuuint32_t)(tkz * units), 1, (cuuint32_t)(nz < 256 ? nz : 256), 1};
      ok = encode(&m.tmap_adj_z, 4, dz, sz, bz);
    }
    if (!ok) return fail(p, FS_ERR_CUDA, "adjoint tensor map");
  }
  cudaError_t e = cudaSuccess;
  for (int f = 0; f < nf && e == cudaSuccess; ++f) {
    if (!u[f] || !lam_in[f] || !lam_out[f]) return fail(p, FS_ERR_INVALID_ARG, "field pointer is NULL");
    e = cudaMemcpyAsync((char*)m.au + f * m.npts * rs, u[f], m.npts * rs, cudaMemcpyDefault, p->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync((char*)m.alam + f * m.npts * rs, lam_in[f], m.npts * rs, cudaMemcpyDefault, p->stream);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(p->acc, 0, sizeof(double) * 4, p->stream);
  fs::KArgs a = make_args(p, m, 0);
  a.spec = m.aspec;
  a.slot_stride = m.slot_stride;
  a.real = m.alam;
  a.spec_bytes = (long long)3 * nf * m.slot_stride * (long long)cs;
  a.real_bytes = (long long)nf * m.npts * (long long)rs;
  a.aux = m.au;
  if (e == cudaSuccess && three)
    e = p->f64 ? fs::adjoint3_launch_f64(a, m.tmap_adj, m.tmap_adj_z, m.aout, p->stream)
               : fs::adjoint3_launch_f32(a, m.tmap_adj, m.tmap_adj_z, m.aout, p->stream);
  else if (e == cudaSuccess)
    e = p->f64 ? fs::adjoint_launch_f64(a, m.tmap_adj, m.aout, p->stream)
               : fs::adjoint_launch_f32(a, m.tmap_adj, m.aout, p->stream);
  for (int f = 0; f < nf && e == cudaSuccess; ++f)
    e = cudaMemcpyAsync(lam_out[f], (char*)m.aout + f * m.npts * rs, m.npts * rs, cudaMemcpyDefault, p->stream);
  if (e != cudaSuccess) return cuda_fail(p, e, "fs_step_adjoint");
  p->last_launches = three ? 5 : 3;
  if (grad) {
    double h[4];
    e = cudaMemcpyAsync(h, p->acc, sizeof(h), cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return cuda_fail(p, e, "fs_step_adjoint sensitivities");
    // Parseval 1/N, and both spectra carry the factor 2 of the packed x transform
    const double norm = 1.0 / (4.0 * (double)m.npts);
    for (int q = 0; q < 4; ++q) grad[q] += h[q] * norm;
    return read_flag(p);
  }
  return FS_OK;
}

fs_status fs_step_profiled(fs_plan_t p, int64_t nsteps) {
  if (!p) return fail(nullptr, FS_ERR_INVALID_ARG, "plan is NULL");
  if (nsteps < 0) return fail(p, FS_ERR_INVALID_ARG, "nsteps < 0");
  if (p->state == kStateNone) return fail(p, FS_ERR_STATE, "fs_step before fs_set_fields");
  cudaError_t e = cudaSuccess;
  auto rec = [&](int k) {
    if (e != cudaSuccess) return;
    if (p->ev_used == p->ev_pool.size()) {
      cudaEvent_t x;
      e = cudaEventCreate(&x);
      if (e != cudaSuccess) return;
      p->ev_pool.push_back(x);
      p->ev_kind.push_back(0);
    }
    p->ev_kind[p->ev_used] = k;
    e = cudaEventRecord(p->ev_pool[p->ev_used], p->stream);
    if (e == cudaSuccess) p->ev_used++;
  };
  int64_t launches = 0;
  if (p->fd) {
    for (int64_t s = 0; s < nsteps && e == cudaSuccess; ++s)
      for (Member& m : p->members) {
        fs::KArgs a = make_args(p, m, 0);
        rec(0);
        if (e == cudaSuccess)
          e = fs::fd_launch(p->f64, a, fd_buf(m, m.fd_cur), fd_buf(m, 1 - m.fd_cur), fd_scratch(p, m), p->stream);
        rec(0);
        m.fd_cur = 1 - m.fd_cur;
        launches += fs::fd_launches_per_step(a);
      }
    if (e != cudaSuccess) return cuda_fail(p, e, "fs_step_profiled");
    p->last_launches = launches;
    return FS_OK;
  }
  for (int64_t s = 0; s < nsteps && e == cudaSuccess && p->batch; ++s) {
    int mode = p->state == kStateReal ? 1 : 0;
    for (int k = 0; k < 2; ++k) {
      rec(k);
      if (e == cudaSuccess) e = launch_batch_pass(p, mode, k, p->stream);
      rec(k);
      launches++;
    }
    p->state = kStateSpec;
  }
  for (int64_t s = 0; s < nsteps && e == cudaSuccess && !p->batch; ++s) {
    int mode = p->state == kStateReal ? 1 : 0;
    if (mode == 0 && fused(p)) {  // one launch per step, timed as pass 0
      rec(0);
      if (e == cudaSuccess) e = launch_fused(p, 1, p->stream);
      rec(0);
      launches++;
      continue;
    }
    for (const Member& m : p->members) {
      fs::KArgs a = make_args(p, m, mode);
      for (int k = 0; k < pass_kinds(m); ++k) {
        rec(k);
        if (e == cudaSuccess) e = launch_pass(p, m, a, k, p->stream);
        rec(k);
        launches++;
      }
    }
    p->state = kStateSpec;
  }
  if (e != cudaSuccess) return cuda_fail(p, e, "fs_step_profiled");
  p->last_launches = launches;
  return FS_OK;
}

fs_status fs_profile_read(fs_plan_t p, double* ms_per_pass, int64_t* launches_per_pass, int npass_max,
                          int* npass) {
  if (!p) return fail(nullptr, FS_ERR_INVALID_ARG, "plan is NULL");
  if (!ms_per_pass || !npass || npass_max < 1) return fail(p, FS_ERR_INVALID_ARG, "bad arguments");
  const int kinds = 4;
  double ms[kinds] = {0.0, 0.0, 0.0, 0.0};
  int64_t cnt[kinds] = {0, 0, 0, 0};
  cudaError_t e = cudaStreamSynchronize(p->stream);
  for (size_t i = 0; e == cudaSuccess && i + 1 < p->ev_used; i += 2) {
    float t = 0.f;
    e = cudaEventElapsedTime(&t, p->ev_pool[i], p->ev_pool[i + 1]);
    ms[p->ev_kind[i]] += t;
    cnt[p->ev_kind[i]]++;
  }
  p->ev_used = 0;
  if (e != cudaSuccess) return cuda_fail(p, e, "fs_profile_read");
  int used = p->fd ? 1 : (p->batch ? 2 : pass_kinds(p->members[0]));
  int n = used < npass_max ? used : npass_max;
  for (int i = 0; i < n; ++i) {
    ms_per_pass[i] = ms[i];
    if (launches_per_pass) launches_per_pass[i] = cnt[i];
  }
  *npass = n;
  return read_flag(p);
}

fs_status fs_set_pass_forms(fs_plan_t p, int row_form, int col_form) {
  if (!p) return fail(nullptr, FS_ERR_INVALID_ARG, "plan is NULL");
  if (row_form < 0 || row_form > 4 || col_form < 0 || col_form > 4 || ((row_form == 4) != (col_form == 4)))
    return fail(p, FS_ERR_INVALID_ARG,
                "pass forms are 0 (default), 1 (half-length / tile), 2 (warp per line), 3 (two warps per line), "
                "4 for both passes (fused step)");
  const Member& m = p->members[0];
  if (row_form == 4 && (p->batch || p->f64 || m.prm.ndim != 2 || !m.tw_row2 || !m.tw_col2 ||
                        !fs::step2_supported(m.prm.n[0], m.prm.n[1], p->nf)))
    return fail(p, FS_ERR_UNSUPPORTED, "the fused step covers single 2D FP32 plans of 256^2, 512^2 or 1024^2, p <= 3");
  const bool r2ok = p->batch ? p->bargs.maps2 != nullptr : m.tw_row2 != nullptr;
  const bool c2ok = p->batch ? p->bargs.maps2 != nullptr : m.tw_col2 != nullptr;
  const bool r3ok = !p->batch && m.tw_row2w != nullptr, c3ok = !p->batch && m.tw_col2w != nullptr;
  if ((row_form == 2 && !r2ok) || (col_form == 2 && !c2ok) || (row_form == 3 && !r3ok) || (col_form == 3 && !c3ok))
    return fail(p, FS_ERR_UNSUPPORTED, "the warp-per-line form does not cover this plan's grid or precision");
  p->row_form = row_form;
  p->col_form = col_form;
  if (p->batch) p->tuned = false;  // the next fs_set_fields tunes again within the pinned forms
  drop_graph(p);  // the captured launches hold the arguments by value
  return FS_OK;
}

fs_status fs_test_short_wait(fs_plan_t p, int enable) {
  if (!p) return fail(nullptr, FS_ERR_INVALID_ARG, "plan is NULL");
  if (p->batch) return fail(p, FS_ERR_UNSUPPORTED, "fs_test_short_wait is built for plans of one simulation");
  if (enable < 0 || enable > 2) return fail(p, FS_ERR_INVALID_ARG, "enable must be 0, 1 or 2");
  p->short_wait = enable;
  drop_graph(p);  // the captured launches hold the arguments by value
  return FS_OK;
}

fs_status fs_batch_schedule(fs_plan_t p, int64_t* row_grid, int64_t* col_grid, int64_t* row_items,
                            int64_t* col_items, int* row_form, int* col_form) {
  if (!p) return fail(nullptr, FS_ERR_INVALID_ARG, "plan is NULL");
  if (!p->batch) return fail(p, FS_ERR_INVALID_ARG, "not a batched plan");
  const fs::BatchArgs& b = p->bargs;
  const bool r2 = b.row_form == 2, c2 = b.col_form == 2;
  if (row_grid) *row_grid = r2 ? b.row2_grid : b.row_grid;
  if (col_grid) *col_grid = c2 ? b.col2_grid : b.col_grid;
  if (row_items) *row_items = r2 ? b.row2_total : b.row_total;
  if (col_items) *col_items = c2 ? b.col2_total : b.col_total;
  if (row_form) *row_form = b.row_form;
  if (col_form) *col_form = b.col_form;
  return FS_OK;
}

fs_status fs_workspace_bytes(fs_plan_t p, size_t* bytes) {
  if (!p) return fail(nullptr, FS_ERR_INVALID_ARG, "plan is NULL");
  if (!bytes) return fail(p, FS_ERR_INVALID_ARG, "bytes is NULL");
  *bytes = p->ws_bytes;
  return FS_OK;
}

fs_status fs_last_launch_count(fs_plan_t p, int64_t* launches) {
  if (!p) return fail(nullptr, FS_ERR_INVALID_ARG, "plan is NULL");
  if (!launches) return fail(p, FS_ERR_INVALID_ARG, "launches is NULL");
  *launches = p->last_launches;
  return FS_OK;
}

fs_status fs_destroy(fs_plan_t p) {
  if (!p) return FS_OK;
  cudaStreamSynchronize(p->stream);
  drop_graph(p);
  for (cudaEvent_t x : p->ev_pool) cudaEventDestroy(x);
  if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
  if (p->host_flag) cudaFreeHost(p->host_flag);
  plan_free_all(p);
  delete p;
  return FS_OK;
}

const char* fs_last_error(fs_plan_t p) { return p ? p->err.c_str() : g_thread_error.c_str(); }

const char* fs_version(void) { return "fs-gb300 0.1 (sm_103a)"; }

}  // extern "C"

// ---- hooks of the slab decomposition (fs_slab.cu) ---------------------------
namespace fs {

// Turn a single plan over nx' = 2 cols x points into the column plan of a
// slab: its kx columns are kx_base .. kx_base + cols - 1 of the global grid
// g (the k2x table gets their global |xi_x|^2, entry cols the global Nyquist
// one), its update uses the global nx and N (scale 1/(2N), the carried c
// scaling 2 nx), and only the slab holding kx_base = 0 separates the packed
// kx = 0 / Nyquist column.
cudaError_t slab_adopt_columns(fs_plan* p, int kx_base, const fs_params& g) {
  Member& m = p->members[0];
  const int cols = m.prm.n[0] / 2, nx = g.n[0];
  m.kx_base = kx_base;
  m.nx_full = nx;
  m.npts_full = (long long)g.n[0] * g.n[1];
  std::vector<double> k2(cols + 1);
  for (int j = 0; j < cols; ++j) k2[j] = axis_k2(g.lap, kx_base + j, nx, g.dx[0]);
  k2[cols] = axis_k2(g.lap, nx / 2, nx, g.dx[0]);
  if (p->f64) return cudaMemcpy(m.k2x, k2.data(), sizeof(double) * k2.size(), cudaMemcpyHostToDevice);
  std::vector<float> f(k2.begin(), k2.end());
  return cudaMemcpy(m.k2x, f.data(), sizeof(float) * f.size(), cudaMemcpyHostToDevice);
}

// One pass of a single plan on its stream: kind 0 the row pass in `mode`
// (0 from spectra, 1 from real fields, 2 inverse only), kind 1 the column pass.
cudaError_t slab_pass(fs_plan* p, int kind, int mode) {
  const Member& m = p->members[0];
  const KArgs a = make_args(p, m, mode);
  return kind == 0 ? launch_row(p, a, p->stream) : launch_col(p, m, a, p->stream);
}

void* slab_spec(fs_plan* p) { return p->members[0].spec; }
void* slab_real(fs_plan* p) { return p->members[0].real; }
double* slab_csum(fs_plan* p) { return p->members[0].csum; }
fs_status slab_read_flag(fs_plan* p) { return read_flag(p); }

}  // namespace fs
