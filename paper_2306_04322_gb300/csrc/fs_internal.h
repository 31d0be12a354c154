// Internal declarations shared by the plan layer (fs_plan.cu) and the kernel
// translation units.  Not part of the public C ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "fs_config.h"

namespace fs {

enum : int { FS_FLAG_NONFINITE = 1, FS_FLAG_TIMEOUT = 2, FS_FLAG_BOUNDS = 4 };

// Polls of an mbarrier before a wait gives up and reports FS_FLAG_TIMEOUT.
constexpr uint32_t kWaitPolls = 1u << 20;

// Scalar coefficients of the pointwise stage and the k-space update,
// precomputed on the host in FP64 and stored in both precisions so the FP32
// kernels issue no FP64 arithmetic.
template <typename T>
struct Coef {
  T two_rho2, ca, dcab, rho2dcab, cab, w, four_alpha, Ldt;  // pointwise stage
  T Mdt, Mdtkc, Ldtke, scale;                               // k-space update
  T idx2, idy2, idz2, kc, ke, dtM, dtL;                     // explicit FD scheme
  T dt;                                                     // adjoint
};

// Arguments of one pass over one simulation (passed by value).  Array
// pointers are in the plan's precision T (float or double) unless noted.
struct KArgs {
  void* spec;              // packed half spectra: slots of slot_stride complex values
  void* real;              // real fields: nf arrays of npts values
  const void* aux;         // adjoint: the state u the step is linearised at (real, nf arrays)
  const void* tw_row;      // pass tables of the x line FFT (L = nx/2)
  const void* tw_col;      // pass tables of the y line FFT (L = ny)
  const void* tw_z;        // pass tables of the z line FFT (L = nz, 3D)
  const void* tw_row_w;    // pass tables of the x line FFT with 32 values per thread (FP32, nx = 1024; NULL: none)
  const void* tw_half;     // exp(-2 pi i k / nx), k = 0..nx/2-1 (real <-> half-length complex)
  const void* tw_row2;     // pass tables of the x line FFT of the pair form (L = nx, E = nx / 32; NULL: none)
  const void* tw_col2;     // pass tables of the y line FFT of the warp-per-column form (L = ny, E = ny / 32)
  const void* tw_row2w;    // the same two with two warps per line (E = nx / 64, ny / 64; NULL: not this form)
  const void* tw_col2w;
  const void* tc_b;        // tensor-core DFT stage: split 16-point DFT matrix, [hi | lo][32][32] float
  const void* k2x;         // |xi_x|^2 per x bin, nx/2 + 1 entries
  const void* k2y;         // |xi_y|^2 per y bin, ny entries
  const void* k2z;         // |xi_z|^2 per z bin, nz entries (3D)
  long long slot_stride;   // complex values per spectrum slot
  long long npts;          // real points per field
  int nx, ny, nz, nf;
  int nx_full;             // x points of the whole grid (nx, except for the column plan of a slab, whose
                           // nx covers only its kx columns)
  int kx_base;             // global kx of the plan's column 0 (0, except for a slab's column plan)
  long long lines;         // rows handled by a row pass (ny * nz)
  int mode;                // row pass: 0 step from spectra, 1 step from real, 2 inverse only
  int tc;                  // FP32 column transforms: 0 CUDA cores, 1 TF32 x 3, 2 BF16 x 3 tensor-core stage
  int carry3;              // 3D FS: c stays in slot 0 as (kx, ky, z) spectrum between steps; its x spectrum
                           // for the x pass goes to slot nf (see the 3D passes)
  int plane0;              // y pass: first plane (slot * nz + z) of the launch
  double M, L, kappa_c, kappa_eta, rho2, c_alpha, c_beta, w, alpha, dt;
  double scale;            // k-space scale 1 / (2 N)
  double inv_npts;         // 1 / N
  const double* csum;      // FP64 sum of c carried for the k = 0 mode (NULL: off)
  double* acc;             // FP64 accumulators of the free-energy diagnostic (2 + p)
  int* flag;               // sticky error bits (FS_FLAG_*)
  int short_wait;          // test hook: 1 makes the first bounded wait of every pass give up
                           // without polling (the pass reports FS_FLAG_TIMEOUT; the kernels still
                           // wait, bounded, for their own copies before exiting); 2 does the same
                           // to the grid barriers of the fused step; 0 = normal
  long long spec_bytes;    // bytes of the buffer `spec` points into (index checks of FS_DEBUG_BOUNDS builds)
  long long real_bytes;    // bytes of the buffer `real` points into (same)
  Coef<float> cf;          // coefficients, FP32 copy
  Coef<double> cd;         // coefficients, FP64 copy
};

template <typename T> __host__ __device__ inline const Coef<T>& coef(const KArgs& a);
template <> __host__ __device__ inline const Coef<float>& coef<float>(const KArgs& a) { return a.cf; }
template <> __host__ __device__ inline const Coef<double>& coef<double>(const KArgs& a) { return a.cd; }

// Kernel launchers, one per precision (fs_k2d_f32.cu / fs_k2d_f64.cu).
// Return cudaErrorInvalidValue for a size without an instantiation.
cudaError_t row_launch_f32(const KArgs& a, cudaStream_t s);
cudaError_t row_launch_f64(const KArgs& a, cudaStream_t s);
cudaError_t col_launch_f32(const KArgs& a, const CUtensorMap& tm, cudaStream_t s);
cudaError_t col_launch_f64(const KArgs& a, const CUtensorMap& tm, cudaStream_t s);
// Warp-per-line forms (FP32; fs_k2d_v2.cuh): the row pass in pair form for
// nx in {256, 512, 1024} (modes 0, 1, 2; needs KArgs::tw_row2) and the column
// pass with one warp per (column, slot) for ny in {256, 512, 1024} (needs
// KArgs::tw_col2 and a tensor map with 2-column boxes).  Return
// cudaErrorNotSupported for other requests.
cudaError_t row2_launch_f32(const KArgs& a, cudaStream_t s);
cudaError_t col2_launch_f32(const KArgs& a, const CUtensorMap& tm, cudaStream_t s);
bool row2_supported(int nx, int nf);
bool col2_supported(int ny, int nf);
// Fused step (pass form 4, fs_step2_f32.cu): `nsteps` steady-state steps
// (mode 0) of a 2D FP32 plan in one cooperative launch, the pair-form row
// pass and the warp-per-column pass separated by grid-wide barriers on the
// counters at gsync (kStep2SyncBytes, zero between launches).  Square grids
// of 256, 512 or 1024 points, nf <= 4; needs tw_row2, tw_col2 and the
// two-column tensor map.  cudaErrorNotSupported for other requests.
bool step2_supported(int nx, int ny, int nf);
constexpr size_t kStep2SyncBytes = 4096;  // counters of the fused step's grid barriers (zeroed)
cudaError_t step2_launch_f32(const KArgs& a, const CUtensorMap& tm, unsigned* gsync, int nsteps, cudaStream_t s);
// Free-energy diagnostic, 2D (row pass mode 3 does the chemical sum and the
// x transforms): y transforms and sums of w K2 |phi^|^2 per field.
cudaError_t energy_col_launch_f32(const KArgs& a, const CUtensorMap& tm, cudaStream_t s);
cudaError_t energy_col_launch_f64(const KArgs& a, const CUtensorMap& tm, cudaStream_t s);
// Adjoint of one 2D step (fs_adjoint_f32.cu / fs_adjoint_f64.cu): spec = the
// 3 nf adjoint slots, real = lam' in / lambda out, aux = u, acc[0..3] += the
// raw sensitivity sums; tm = tensor map over the adjoint slots.
cudaError_t adjoint_launch_f32(const KArgs& a, const CUtensorMap& tm, void* lam_out, cudaStream_t s);
cudaError_t adjoint_launch_f64(const KArgs& a, const CUtensorMap& tm, void* lam_out, cudaStream_t s);
// Adjoint of one 3D step: the same slots and outputs; tm_y: [slot nz + z][y][kx]
// and tm_z: [slot][z][y][kx] over the 3 nf adjoint slots.
cudaError_t adjoint3_launch_f32(const KArgs& a, const CUtensorMap& tm_y, const CUtensorMap& tm_z, void* lam_out,
                                cudaStream_t s);
cudaError_t adjoint3_launch_f64(const KArgs& a, const CUtensorMap& tm_y, const CUtensorMap& tm_z, void* lam_out,
                                cudaStream_t s);
// Columns per CTA of the 2D column pass for this grid (the TMA box width).
int col_tile_width(bool f64, int nx, int ny);
// 3D passes (fs_k3d_f32.cu / fs_k3d_f64.cu): y transform of nslots slots of
// every z plane (dir -1 forward with kx = 0 column packing, +1 inverse), and
// the z step (forward z, k-space update, inverse z).
cudaError_t ypass_launch_f32(const KArgs& a, const CUtensorMap& tm, int dir, int nslots, cudaStream_t s);
cudaError_t ypass_launch_f64(const KArgs& a, const CUtensorMap& tm, int dir, int nslots, cudaStream_t s);
cudaError_t zstep_launch_f32(const KArgs& a, const CUtensorMap& tm, cudaStream_t s);
cudaError_t zstep_launch_f64(const KArgs& a, const CUtensorMap& tm, cudaStream_t s);
// Free-energy diagnostic, 3D: z transforms and sums of w K2 |phi^|^2 after
// the x pass in mode 3 and the forward y pass over slots 0..nf-1.
cudaError_t energy_z_launch_f32(const KArgs& a, const CUtensorMap& tm, cudaStream_t s);
cudaError_t energy_z_launch_f64(const KArgs& a, const CUtensorMap& tm, cudaStream_t s);
int line_tile_width_f32(int nx, int nl);
int line_tile_width_f64(int nx, int nl);
// Batched ensemble launches (fs_batch_f32.cu / fs_batch_f64.cu).
struct BatchArgs {
  const KArgs* mem;             // per simulation, row-pass arguments (execution order)
  const KArgs* mem_col;         // per simulation, column-pass arguments
  const CUtensorMap* maps;      // per simulation, column tile tensor map
  const long long* row_begin;   // first row work item of each simulation
  const long long* col_begin;   // first column work item of each simulation
  const int* col_tiles;         // kx tiles of each simulation
  int nm;                       // simulations
  int nf1;                      // nf + 1 (warps of a row CTA)
  long long row_total, col_total;
  long long row_grid, col_grid; // persistent grid sizes
  size_t row_smem, col_smem;
  // warp-per-line forms (FP32 members with both axes in [64, 1024]; NULL / 0:
  // not available): row-pair and (column pair, field group) work lists,
  // two-column tensor maps
  const CUtensorMap* maps2;
  const long long* row2_begin;
  const long long* col2_begin;
  const int* col2_pairs;        // column pairs of each simulation
  long long row2_total, col2_total;
  long long row2_grid, col2_grid;
  size_t row2_smem, col2_smem;
  int row_form, col_form;       // chosen per pass: 1 half-length / tile kernels, 2 warp-per-line kernels
};
cudaError_t row_batch_launch_f32(const BatchArgs& b, cudaStream_t s);
cudaError_t row_batch_launch_f64(const BatchArgs& b, cudaStream_t s);
cudaError_t col_batch_launch_f32(const BatchArgs& b, cudaStream_t s);
cudaError_t col_batch_launch_f64(const BatchArgs& b, cudaStream_t s);
cudaError_t row2_batch_launch_f32(const BatchArgs& b, cudaStream_t s);
cudaError_t col2_batch_launch_f32(const BatchArgs& b, cudaStream_t s);
size_t row2_smem_f32(int nx, int nf);
size_t col2_smem_f32(int ny);
int col2_groups(int nf);
size_t row_smem_f32(int nx, int nf);
size_t row_smem_f64(int nx, int nf);
long long row_blocks_f32(int nx, long long lines);
long long row_blocks_f64(int nx, long long lines);
int col_batch_tk_f32(int nx, int ny);
int col_batch_tk_f64(int nx, int ny);
size_t col_smem_f32(int ny, int tk);
size_t col_smem_f64(int ny, int tk);
// One explicit finite-difference step (fs_fd.cu): in -> out, nf fields each.
// Explicit FD step from `in` to `out` (nf real fields each); 3D needs an
// N-real scratch field for mu that aliases neither.
cudaError_t fd_launch(bool f64, const KArgs& a, const void* in, void* out, void* scratch, cudaStream_t s);
int fd_launches_per_step(const KArgs& a);
// FP64 sum of n values of x (float or double) added into *out.
cudaError_t sum_launch_f32(const void* x, long long n, double* out, cudaStream_t s);
cudaError_t sum_launch_f64(const void* x, long long n, double* out, cudaStream_t s);

}  // namespace fs
