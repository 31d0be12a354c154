/*
 * fs_slab.h -- slab decomposition of one 2D Fourier-spectral grid over
 * several ranks (one process per GPU), which spreads one grid's memory and
 * work over several GPUs (the paper's conclusions name one GPU's memory as
 * the limit of the FS method; Section 4 compares the memory of FS and FD).
 *
 * The step is Algorithm 1, split as the library's single-GPU plans split it:
 *   - row pass: inverse x transforms of the carried spectra, the pointwise
 *     derivatives df_chem/dc, df_chem/deta_i (Section 2.1), the explicit
 *     parts g_i = eta_i - L dt df/deta_i, forward x transforms;
 *   - column pass: forward y transforms, the per-mode solve of Eqs.
 *     (A-C_discrete_fft_c) and (A-C_discrete_fft_eta) with |xi|^2 of Eq.
 *     (Gamma_fft) or the FS-FD forms, inverse y transforms.
 * Both are local to one axis, so the grid shards with no other exchange
 * than a transpose between them (one forward, one back per step).  Rank r
 * of R holds:
 *   - for the row pass, rows y in [r rows, (r + 1) rows), rows = ny / R,
 *     every x;
 *   - for the column pass, the packed half-spectrum columns kx in
 *     [r cols, (r + 1) cols), cols = nx / (2R), every y.  Column 0 packs the
 *     real kx = 0 and kx = nx/2 spectra (real part, imaginary part), so rank
 *     0 holds both.
 *
 * One step, on every rank, all on the slab's stream:
 *   1. fs_slab_row_pass
 *   2. forward exchange (the caller's, e.g. NCCL point-to-point): for every
 *      peer q != rank and slot s < slots_fwd, the block send[q][s] goes to q,
 *      which receives it at colspec[s][rank * rows ..] (rows x cols values);
 *   3. fs_slab_col_pass
 *   4. back exchange: for every peer q != rank and slot s < slots_back, the
 *      block colspec[s][q * rows ..] goes to q, which receives it at
 *      recv[rank][s].
 * Each block is one contiguous array of rows x cols complex values (y
 * major, kx fastest).  The rank's own blocks never leave the GPU: the row
 * pass writes them straight into colspec and the next row pass reads them
 * from there.  Steps 2 and 4 move (R - 1) / R of the spectra per rank and
 * direction: (nf + 1) and nf slots of ny nx / (2R) complex values.
 *
 * Conventions are those of fs.h: fields c, eta_1 .. eta_p (nf = 1 + p), the
 * element type double for FS_F64 and float for FS_F32; complex values are
 * (re, im) pairs of that type.  Slabs take 2D semi-implicit FS problems in
 * FS_F64 or FS_F32 (no tensor-core stage), R a power of two with ny / R and
 * nx / R at least 8; the global grid follows fs.h's 2D limits.  Other
 * requests return FS_ERR_UNSUPPORTED.  Calls on one slab must not run
 * concurrently from several host threads.
 */
#ifndef FS_SLAB_H_
#define FS_SLAB_H_

#include "fs.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fs_slab* fs_slab_t; /* opaque; owns its device workspace */

/* Layout of one rank's share and its exchange buffers (device memory owned
 * by the slab; valid until fs_slab_destroy). */
typedef struct {
  int rank, nranks;
  int rows;            /* ny / R rows of the row pass, starting at y = rank * rows */
  int cols;            /* nx / (2R) packed columns of the column pass, starting at kx = rank * cols */
  int slots_fwd;       /* nf + 1 slots sent after the row pass: c, g_1 .. g_p, df/dc */
  int slots_back;      /* nf slots sent back after the column pass: c, eta_1 .. eta_p */
  size_t elem_bytes;   /* bytes of one complex value: 16 (FS_F64) or 8 (FS_F32) */
  size_t block_elems;  /* rows * cols: complex values of one exchanged block */
  void* send;          /* [R][slots_fwd][rows][cols]: row-pass output by destination (own block unused) */
  void* recv;          /* [R][slots_back][rows][cols]: column-pass results by source (own block unused) */
  void* colspec;       /* [slots_fwd][ny][cols]: the column pass's spectra; source q's rows at y = q * rows */
} fs_slab_info;

/* Create rank `rank` of `nranks` for the global 2D problem prm (the
 * initialisation block of Algorithm 1 with the global grid; the |xi|^2
 * tables hold the global frequencies of this rank's columns).  `stream` is
 * a cudaStream_t (NULL: legacy default stream) on the current device.
 * Validates first (no CUDA call for an invalid request).  On failure *out
 * is NULL. */
FS_API fs_status fs_slab_create(const fs_params* prm, int rank, int nranks, void* stream, fs_slab_t* out);

/* Fill *info (see fs_slab_info). */
FS_API fs_status fs_slab_info_get(fs_slab_t slab, fs_slab_info* info);

/* Copy this rank's rows of the state in (the initial conditions of
 * Algorithm 1): fields[f] points to rows * nx values of field f (rows y =
 * rank * rows .. , x fastest), nf pointers, device or host memory.  If
 * c_sum_local is not NULL it receives the FP64 sum of this rank's c values
 * (the call then synchronises the stream).  The next fs_slab_row_pass starts
 * from these real fields. */
FS_API fs_status fs_slab_set_fields(fs_slab_t slab, const void* const* fields, double* c_sum_local);

/* The FP64 sum of c over the whole grid (the sum of every rank's
 * c_sum_local), which FS_F32 slabs carry for the k = 0 mode of c (the k = 0
 * row of Eq. (A-C_discrete_fft_c) is the identity: mean(c) is conserved).
 * Required on FS_F32 slabs after fs_slab_set_fields and before the first
 * fs_slab_col_pass; ignored by FS_F64 slabs.  Synchronises the stream. */
FS_API fs_status fs_slab_set_c_sum(fs_slab_t slab, double c_sum_total);

/* Step 1 of a step (see the preamble): the row pass over this rank's rows,
 * from the real fields after fs_slab_set_fields, else from the spectra of
 * the previous step (its own block in colspec and the received blocks in
 * recv), then the transposed blocks into send and colspec.  Asynchronous. */
FS_API fs_status fs_slab_row_pass(fs_slab_t slab);

/* Step 3: the column pass over this rank's columns (colspec, in place).
 * Asynchronous. */
FS_API fs_status fs_slab_col_pass(fs_slab_t slab);

/* Copy this rank's rows of the current real fields out (nf pointers of
 * rows * nx values), after the back exchange of the last step: the inverse
 * x transforms close the iteration of Algorithm 1.  Synchronises the stream;
 * the run continues from the same spectra. */
FS_API fs_status fs_slab_get_fields(fs_slab_t slab, void* const* fields_out);

/* Synchronise the slab's stream and return the sticky device status
 * (FS_ERR_NONFINITE, FS_ERR_TIMEOUT, ...) of its passes. */
FS_API fs_status fs_slab_sync(fs_slab_t slab);

/* Release the slab and its device memory.  NULL is a no-op. */
FS_API fs_status fs_slab_destroy(fs_slab_t slab);

/* Text of the last failure on this slab (or on this thread for NULL). */
FS_API const char* fs_slab_last_error(fs_slab_t slab);

#ifdef __cplusplus
}
#endif

#endif /* FS_SLAB_H_ */
