// Slab decomposition of one 2D FS grid over R ranks (include/fs_slab.h).
//
// A slab is two single plans on one stream: a row plan over the rank's
// rows (nx x ny/R, the global x axis) and a column plan over its packed kx
// columns (nx/R x ny: nx/(2R) complex columns, the global y axis) whose
// |xi_x|^2 table, scale and packed-column test are those of its place in the
// global grid.  Two transpose kernels move the spectra between them:
//   pack   row spectra [s][y][kx]          -> send[q][s][y][kx - q cols] for q != rank,
//                                             colspec[s][rank rows + y][kx - rank cols] for q = rank
//   unpack recv[q][s][y][.] / own colspec -> row spectra [s][y][q cols + .]
// The blocks between ranks go through the caller's exchange.  Both kernels
// copy 16-byte units (two FP32 or one FP64 complex value), consecutive
// threads on consecutive units of one row: reads and writes are coalesced.
#include <cuda_runtime.h>

#include <string>

#include "fs.h"
#include "fs_internal.h"
#include "fs_slab.h"
#include "fs_slab_hooks.h"

struct fs_slab {
  fs_plan_t rowp = nullptr;  // rows x nx
  fs_plan_t colp = nullptr;  // ny x (2 cols): the column pass
  int rank = 0, R = 1, nx = 0, ny = 0, rows = 0, cols = 0, nf = 1;
  bool f64 = true;
  size_t cs = 16;            // bytes per complex value
  void* send = nullptr;
  void* recv = nullptr;
  double* csum_local = nullptr;  // device scratch of fs_slab_set_fields
  cudaStream_t stream = nullptr;
  int grid = 0;              // blocks of the transpose kernels (a multiple of the SM count)
  bool have_real = false;    // the next row pass starts from the real fields
  bool have_spec = false;    // a step has run: the state is the spectra
  bool csum_set = false;
  std::string err;
};

namespace {

thread_local std::string g_slab_error;

fs_status sfail(fs_slab* s, fs_status st, const std::string& msg) {
  (s ? s->err : g_slab_error) = msg;
  return st;
}

fs_status scuda(fs_slab* s, cudaError_t e, const char* where) {
  cudaGetLastError();
  return sfail(s, FS_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

int log2i(long long v) {
  int l = 0;
  while ((1LL << l) < v) ++l;
  return l;
}

// Shapes of one transpose, in 16-byte units; every extent a power of two.
struct Xpose {
  uint4* rowspec;        // pack: source; unpack: destination
  uint4* send_or_recv;   // pack: send (destination); unpack: recv (source)
  uint4* colspec;        // own block
  long long total;       // units: slots x rows x Hu
  long long slot_u;      // row spectrum slot stride (units)
  long long col_slot_u;  // colspec slot stride (units): ny x Lu
  int lg_hu, lg_rows, lg_lu;  // log2 of units per row, rows, units per block row
  int slots, rank;
};

// pack (PACK = true) or unpack (false); unit index i -> (s, y, u), u -> (q, ul).
template <bool PACK>
__global__ void __launch_bounds__(256) fs_slab_xpose_kernel(Xpose x) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long hu = 1LL << x.lg_hu, lu = 1LL << x.lg_lu, rows = 1LL << x.lg_rows;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < x.total; i += stride) {
    const long long u = i & (hu - 1), rest = i >> x.lg_hu;
    const long long y = rest & (rows - 1), s = rest >> x.lg_rows;
    const long long q = u >> x.lg_lu, ul = u & (lu - 1);
    const long long r_off = s * x.slot_u + y * hu + u;
    const long long b_off = q == x.rank ? s * x.col_slot_u + ((long long)x.rank * rows + y) * lu + ul
                                        : ((q * x.slots + s) * rows + y) * lu + ul;
    uint4* block = q == x.rank ? x.colspec : x.send_or_recv;
    if (PACK)
      block[b_off] = x.rowspec[r_off];
    else
      x.rowspec[r_off] = block[b_off];
  }
}

Xpose make_xpose(const fs_slab* s, bool pack) {
  Xpose x;
  const long long H = s->nx / 2;
  const long long hu = H * (long long)s->cs / 16, lu = (long long)s->cols * (long long)s->cs / 16;
  x.rowspec = static_cast<uint4*>(fs::slab_spec(s->rowp));
  x.send_or_recv = static_cast<uint4*>(pack ? s->send : s->recv);
  x.colspec = static_cast<uint4*>(fs::slab_spec(s->colp));
  x.slots = pack ? s->nf + 1 : s->nf;
  x.slot_u = (long long)s->rows * hu;
  x.col_slot_u = (long long)s->ny * lu;
  x.total = (long long)x.slots * s->rows * hu;
  x.lg_hu = log2i(hu);
  x.lg_rows = log2i(s->rows);
  x.lg_lu = log2i(lu);
  x.rank = s->rank;
  return x;
}

cudaError_t xpose(fs_slab* s, bool pack) {
  const Xpose x = make_xpose(s, pack);
  long long want = (x.total + 255) / 256;
  const unsigned blocks = (unsigned)(want < s->grid ? want : s->grid);
  if (pack)
    fs_slab_xpose_kernel<true><<<blocks, 256, 0, s->stream>>>(x);
  else
    fs_slab_xpose_kernel<false><<<blocks, 256, 0, s->stream>>>(x);
  return cudaGetLastError();
}

bool pow2(long long v) { return v > 0 && (v & (v - 1)) == 0; }

void destroy(fs_slab* s) {
  if (s->rowp) fs_destroy(s->rowp);
  if (s->colp) fs_destroy(s->colp);
  if (s->send) cudaFree(s->send);
  if (s->recv) cudaFree(s->recv);
  if (s->csum_local) cudaFree(s->csum_local);
  delete s;
}

}  // namespace

extern "C" {

fs_status fs_slab_create(const fs_params* prm, int rank, int nranks, void* stream, fs_slab_t* out) {
  if (!out) return sfail(nullptr, FS_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!prm) return sfail(nullptr, FS_ERR_INVALID_ARG, "params is NULL");
  if (nranks < 1 || rank < 0 || rank >= nranks) return sfail(nullptr, FS_ERR_INVALID_ARG, "rank out of range");
  if (prm->ndim != 2 || prm->scheme != FS_SCHEME_SEMI_IMPLICIT_FS ||
      (prm->precision != FS_F64 && prm->precision != FS_F32))
    return sfail(nullptr, FS_ERR_UNSUPPORTED, "slabs take 2D semi-implicit FS problems in FS_F64 or FS_F32");
  const int nx = prm->n[0], ny = prm->n[1];
  if (!pow2(nranks) || nx <= 0 || ny <= 0 || ny % nranks || nx % nranks || ny / nranks < 8 || nx / nranks < 8)
    return sfail(nullptr, FS_ERR_UNSUPPORTED, "nranks must be a power of two with ny / nranks and nx / nranks >= 8");
  for (int d = 0; d < 2; ++d)
    if (!pow2(prm->n[d]) || prm->n[d] > 2048)
      return sfail(nullptr, FS_ERR_UNSUPPORTED, "each grid axis must be a power of two in [8, 2048]");
  // the row plan (rows x nx) and the column plan (ny x nx / R) validate the
  // remaining parameters before any CUDA call
  fs_params rp = *prm, cp = *prm;
  rp.n[1] = ny / nranks;
  cp.n[0] = nx / nranks;

  fs_slab* s = new fs_slab();
  s->rank = rank;
  s->R = nranks;
  s->nx = nx;
  s->ny = ny;
  s->rows = ny / nranks;
  s->cols = nx / (2 * nranks);
  s->nf = 1 + prm->p;
  s->f64 = prm->precision == FS_F64;
  s->cs = s->f64 ? 16 : 8;
  s->stream = reinterpret_cast<cudaStream_t>(stream);
  fs_status st = fs_plan_create(&rp, stream, &s->rowp);
  if (st == FS_OK) st = fs_plan_create(&cp, stream, &s->colp);
  if (st != FS_OK) {
    const std::string why = fs_last_error(nullptr);
    destroy(s);
    return sfail(nullptr, st, "slab plans: " + why);
  }
  cudaError_t e = fs::slab_adopt_columns(s->colp, rank * s->cols, *prm);
  const size_t block = (size_t)s->rows * s->cols * s->cs;
  if (e == cudaSuccess) e = cudaMalloc(&s->send, block * nranks * (s->nf + 1));
  if (e == cudaSuccess) e = cudaMalloc(&s->recv, block * nranks * s->nf);
  if (e == cudaSuccess) e = cudaMalloc(&s->csum_local, sizeof(double));
  int dev = 0, sms = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    const fs_status f = e == cudaErrorMemoryAllocation ? FS_ERR_OOM : FS_ERR_CUDA;
    destroy(s);
    cudaGetLastError();
    return sfail(nullptr, f, std::string("slab set-up: ") + cudaGetErrorString(e));
  }
  s->grid = 8 * sms;  // 8 resident 256-thread CTAs per SM
  *out = s;
  return FS_OK;
}

fs_status fs_slab_info_get(fs_slab_t s, fs_slab_info* info) {
  if (!s || !info) return sfail(s, FS_ERR_INVALID_ARG, "slab or info is NULL");
  info->rank = s->rank;
  info->nranks = s->R;
  info->rows = s->rows;
  info->cols = s->cols;
  info->slots_fwd = s->nf + 1;
  info->slots_back = s->nf;
  info->elem_bytes = s->cs;
  info->block_elems = (size_t)s->rows * s->cols;
  info->send = s->send;
  info->recv = s->recv;
  info->colspec = fs::slab_spec(s->colp);
  return FS_OK;
}

fs_status fs_slab_set_fields(fs_slab_t s, const void* const* fields, double* c_sum_local) {
  if (!s) return sfail(nullptr, FS_ERR_INVALID_ARG, "slab is NULL");
  fs_status st = fs_set_fields(s->rowp, fields);
  if (st != FS_OK) return sfail(s, st, fs_last_error(s->rowp));
  s->have_real = true;
  s->have_spec = false;
  s->csum_set = s->f64;
  if (c_sum_local) {
    const long long n = (long long)s->rows * s->nx;
    cudaError_t e = cudaMemsetAsync(s->csum_local, 0, sizeof(double), s->stream);
    if (e == cudaSuccess)
      e = s->f64 ? fs::sum_launch_f64(fs::slab_real(s->rowp), n, s->csum_local, s->stream)
                 : fs::sum_launch_f32(fs::slab_real(s->rowp), n, s->csum_local, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c_sum_local, s->csum_local, sizeof(double), cudaMemcpyDefault, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return scuda(s, e, "local c sum");
  }
  return FS_OK;
}

fs_status fs_slab_set_c_sum(fs_slab_t s, double total) {
  if (!s) return sfail(nullptr, FS_ERR_INVALID_ARG, "slab is NULL");
  if (s->f64) return FS_OK;
  cudaError_t e = cudaMemcpyAsync(fs::slab_csum(s->colp), &total, sizeof(double), cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);  // `total` lives on this frame
  if (e != cudaSuccess) return scuda(s, e, "fs_slab_set_c_sum");
  s->csum_set = true;
  return FS_OK;
}

fs_status fs_slab_row_pass(fs_slab_t s) {
  if (!s) return sfail(nullptr, FS_ERR_INVALID_ARG, "slab is NULL");
  if (!s->have_real && !s->have_spec) return sfail(s, FS_ERR_STATE, "fs_slab_row_pass before fs_slab_set_fields");
  cudaError_t e = cudaSuccess;
  int mode = 1;
  if (!s->have_real) {
    e = xpose(s, false);
    mode = 0;
  }
  if (e == cudaSuccess) e = fs::slab_pass(s->rowp, 0, mode);
  if (e == cudaSuccess) e = xpose(s, true);
  if (e != cudaSuccess) return scuda(s, e, "slab row pass");
  s->have_real = false;
  s->have_spec = true;
  return FS_OK;
}

fs_status fs_slab_col_pass(fs_slab_t s) {
  if (!s) return sfail(nullptr, FS_ERR_INVALID_ARG, "slab is NULL");
  if (!s->have_spec) return sfail(s, FS_ERR_STATE, "fs_slab_col_pass before fs_slab_row_pass");
  if (!s->csum_set) return sfail(s, FS_ERR_STATE, "FS_F32 slab: fs_slab_set_c_sum not called");
  cudaError_t e = fs::slab_pass(s->colp, 1, 0);
  if (e != cudaSuccess) return scuda(s, e, "slab column pass");
  return FS_OK;
}

fs_status fs_slab_get_fields(fs_slab_t s, void* const* out) {
  if (!s) return sfail(nullptr, FS_ERR_INVALID_ARG, "slab is NULL");
  if (!out) return sfail(s, FS_ERR_INVALID_ARG, "fields_out is NULL");
  for (int f = 0; f < s->nf; ++f)
    if (!out[f]) return sfail(s, FS_ERR_INVALID_ARG, "output pointer is NULL");
  if (!s->have_real && !s->have_spec) return sfail(s, FS_ERR_STATE, "fs_slab_get_fields before fs_slab_set_fields");
  cudaError_t e = cudaSuccess;
  if (s->have_spec) {
    e = xpose(s, false);
    if (e == cudaSuccess) e = fs::slab_pass(s->rowp, 0, 2);
  }
  const size_t n = (size_t)s->rows * s->nx * (s->f64 ? 8 : 4);
  const char* real = static_cast<const char*>(fs::slab_real(s->rowp));
  for (int f = 0; f < s->nf && e == cudaSuccess; ++f)
    e = cudaMemcpyAsync(out[f], real + f * n, n, cudaMemcpyDefault, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return scuda(s, e, "fs_slab_get_fields");
  return FS_OK;
}

fs_status fs_slab_sync(fs_slab_t s) {
  if (!s) return sfail(nullptr, FS_ERR_INVALID_ARG, "slab is NULL");
  fs_status st = fs::slab_read_flag(s->rowp);
  if (st != FS_OK) return sfail(s, st, fs_last_error(s->rowp));
  st = fs::slab_read_flag(s->colp);
  if (st != FS_OK) return sfail(s, st, fs_last_error(s->colp));
  return FS_OK;
}

fs_status fs_slab_destroy(fs_slab_t s) {
  if (!s) return FS_OK;
  cudaStreamSynchronize(s->stream);
  destroy(s);
  return FS_OK;
}

const char* fs_slab_last_error(fs_slab_t s) { return s ? s->err.c_str() : g_slab_error.c_str(); }

}  // extern "C"
