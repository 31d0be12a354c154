/*
 * fs.h -- C ABI of the GB300 (sm_103a) semi-implicit Fourier-spectral
 * phase-field library.
 *
 * The library advances the coupled Cahn-Hilliard / Allen-Cahn model of
 * Boccardo, Tong, Leen, Tourret and Segurado, "Efficiency and accuracy of
 * GPU-parallelized Fourier spectral methods for solving phase-field models"
 * (arXiv 2306.04322):
 *   - free energy and chemical free-energy density f_chem: Section 2.1,
 *     Eq. (fe) and the definitions of f_alpha, f_beta, h and g after it;
 *   - evolution equations: Eqs. (C-H) and (A-C), periodic boundaries;
 *   - semi-implicit time discretisation: Eqs. (C-H_discrete), (A-C_discrete);
 *   - Fourier-space solve: Eqs. (C-H_discrete_fft), (A-C_discrete_fft),
 *     independent terms (C-H_fft_b), (A-C_fft_b), per-mode inversion
 *     (A-C_discrete_fft_c), (A-C_discrete_fft_eta);
 *   - squared frequency norm: Eqs. (Gamma_fft), (Gamma_fft_3d); FS-FD forms
 *     (Gamma_fft-fdO2), (Gamma_fft-fdO4) and their 3D versions;
 *   - the time loop: Algorithm 1 ("FS solution algorithm");
 *   - the explicit finite-difference comparison scheme: Section 2.2
 *     (forward Euler, 5-point / 7-point Laplacian, periodic boundaries).
 *
 * Conventions shared by every call:
 *   - Fields: nf = 1 + p real arrays, order c, eta_1 .. eta_p.  Each field is
 *     one contiguous array of N = nx*ny*nz values, x fastest:
 *     idx = (z*ny + y)*nx + x.  The element type is double for FS_F64 and
 *     float for every FS_F32* precision.
 *   - Pointers passed in and out may be device memory or host memory
 *     (pinned or pageable); copies use cudaMemcpyDefault.  The caller owns
 *     them; a plan keeps no caller pointer after a call returns.
 *   - Every call is ordered on the plan's CUDA stream.  Calls on one plan
 *     must not run concurrently from several host threads.
 *   - Grid sizes: each axis a power of two, in [8, 2048] for 2D plans (the
 *     paper's finest grid is 2048^2, Table 1) and in [8, 1024] along x, [8,
 *     512] along y and z for 3D plans; batched members and the 2D adjoint
 *     step take axes up to 1024.  Other sizes return FS_ERR_UNSUPPORTED.  p in
 *     [0, 4].  dt > 0; M = 0 or L = 0 is allowed.
 *   - Status codes are returned by value; fs_last_error() gives the text of
 *     the last failure on that plan (or on this thread for a NULL plan).
 */
#ifndef FS_H_
#define FS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Exported entry points; the library is built with hidden visibility, so
 * nothing else (C++ templates, function-local statics) is shared with other
 * libraries loaded in the same process. */
#if defined(__GNUC__)
#define FS_API __attribute__((visibility("default")))
#else
#define FS_API
#endif

typedef struct fs_plan* fs_plan_t; /* opaque; owns all device workspace */

typedef enum {
  FS_OK = 0,
  FS_ERR_INVALID_ARG = 1, /* NULL pointer, bad value (dt <= 0, p out of range, ...) */
  FS_ERR_UNSUPPORTED = 2, /* valid request this build does not implement (size, combination) */
  FS_ERR_OOM = 3,         /* device workspace allocation failed */
  FS_ERR_CUDA = 4,        /* a CUDA runtime call failed; see fs_last_error */
  FS_ERR_NONFINITE = 5,   /* a NaN / Inf appeared in the fields during fs_step */
  FS_ERR_TIMEOUT = 6,     /* a bounded device-side wait gave up */
  FS_ERR_STATE = 7        /* call out of order (e.g. fs_step before fs_set_fields) */
} fs_status;

typedef enum {
  FS_F64 = 0,          /* FP64 fields, transforms and update */
  FS_F32 = 1,          /* FP32 fields and transforms; mean(c) carried in FP64 */
  FS_F32_TC_TF32 = 2,  /* FP32 with one DFT stage on tensor cores (TF32) */
  FS_F32_TC_BF16X3 = 3 /* FP32 with one DFT stage on tensor cores (split BF16, 3 products) */
} fs_precision;

typedef enum {
  FS_LAP_SPECTRAL = 0, /* |xi|^2, Eqs. (Gamma_fft), (Gamma_fft_3d) */
  FS_LAP_FD2 = 1,      /* |xi_c2|^2, Eqs. (Gamma_fft-fdO2) and 3D form */
  FS_LAP_FD4 = 2       /* |xi_c4|^2, Eqs. (Gamma_fft-fdO4) and 3D form */
} fs_laplacian;

typedef enum {
  FS_SCHEME_SEMI_IMPLICIT_FS = 0, /* Algorithm 1 */
  FS_SCHEME_EXPLICIT_FD = 1       /* Section 2.2 comparison scheme (2D and 3D) */
} fs_scheme;

/* Problem description.  Physical parameters follow Section 2.1 (benchmark
 * values: kappa_c = kappa_eta = 3, rho2 = 2, c_alpha = 0.3, c_beta = 0.7,
 * w = 1, alpha = 5, M = L = 5); grid and dt follow the initialisation block
 * of Algorithm 1.  n[d] and dx[d] for d >= ndim are ignored. */
typedef struct {
  int ndim;     /* 2 or 3 */
  int n[3];     /* points along x, y, z */
  double dx[3]; /* spacing along x, y, z (> 0); domain length l = n dx */
  int p;        /* number of order parameters, 0..4 */
  double M, L, kappa_c, kappa_eta, rho2, c_alpha, c_beta, w, alpha, dt;
  int precision; /* fs_precision */
  int lap;       /* fs_laplacian */
  int scheme;    /* fs_scheme */
} fs_params;

/* Optional device-memory allocator used for all plan workspace.  NULL
 * functions select cudaMalloc / cudaFree.  alloc returns NULL on failure. */
typedef void* (*fs_alloc_fn)(size_t bytes, void* ctx);
typedef void (*fs_free_fn)(void* ptr, void* ctx);

/* Create a plan for one simulation: the initialisation block of Algorithm 1
 * (parameters of Section 2.1, grid x = [0, l) per axis, dt, and |xi|^2 of
 * Eq. (Gamma_fft) / (Gamma_fft_3d) or the FS-FD forms, built once as
 * per-axis tables).  `stream` is a cudaStream_t (NULL: the
 * legacy default stream).  Validates prm first (no CUDA call is made for an
 * invalid request), then allocates the workspace: nf real fields plus
 * (nf + 1) packed half-spectrum slots of N/2 complex values, and small
 * per-axis tables.  On failure *out is NULL. */
FS_API fs_status fs_plan_create(const fs_params* prm, void* stream, fs_plan_t* out);
FS_API fs_status fs_plan_create_ex(const fs_params* prm, void* stream, fs_alloc_fn alloc, fs_free_fn dealloc,
                            void* ctx, fs_plan_t* out);

/* Batched ensemble: `count` independent 2D simulations with their own grid
 * sizes and parameters (each[i]), one plan, one launch per pass for all of
 * them.  All members share precision and p; lap and scheme must be
 * spectral FS, precision FS_F64 or FS_F32, 16 <= nx <= 1024 and ny in
 * [128 (FS_F32) or 64 (FS_F64), 1024]; other members return
 * FS_ERR_UNSUPPORTED.  Field pointer arrays for a batch plan are
 * member-major: fields[i * nf + f]. */
FS_API fs_status fs_batch_create(const fs_params* each, int count, void* stream, fs_plan_t* out);

/* Copy the state in: the conserved composition c and the order parameters
 * eta_1 .. eta_p of Section 2.1 (the "initial conditions" input of
 * Algorithm 1).  fields[f] points to field f (nf pointers, plan dtype).
 * Also computes sum(c) in FP64 for the mean-mode carry of FP32 plans (the
 * k = 0 row of Eq. (A-C_discrete_fft_c) is the identity, so mean(c) is
 * conserved). */
FS_API fs_status fs_set_fields(fs_plan_t plan, const void* const* fields);

/* Advance nsteps >= 0 time steps (Algorithm 1 iterations, or explicit FD
 * steps for FS_SCHEME_EXPLICIT_FD).  Launches asynchronously, then
 * synchronises the stream and returns FS_ERR_NONFINITE if a non-finite value
 * was met.  Long runs replay a captured CUDA graph of the step. */
FS_API fs_status fs_step(fs_plan_t plan, int64_t nsteps);

/* As fs_step -- nsteps iterations of the loop of Algorithm 1 (derivatives,
 * forward transforms, the per-mode solve of Eqs. (A-C_discrete_fft_c) and
 * (A-C_discrete_fft_eta), inverse transforms) -- without the final
 * synchronisation and status read. */
FS_API fs_status fs_step_async(fs_plan_t plan, int64_t nsteps);

/* Synchronise the plan's stream and return the sticky device status. */
FS_API fs_status fs_sync(fs_plan_t plan);

/* Copy the current real fields c, eta_1 .. eta_p out (nf pointers): the
 * inverse transforms that close each iteration of Algorithm 1 (its output
 * step).  Materialises them first when the state is held as spectra (one
 * inverse row pass); the run continues from the spectra unchanged. */
FS_API fs_status fs_get_fields(fs_plan_t plan, void* const* fields_out);

/* Replace the physical parameters and dt of an existing plan.  Grid, p,
 * precision, lap and scheme must match the plan; the state is kept. */
FS_API fs_status fs_set_params(fs_plan_t plan, const fs_params* prm);

/* Rebind the plan to another stream. */
FS_API fs_status fs_set_stream(fs_plan_t plan, void* stream);

/* Total free energy, Eq. (fe), of the current state (rectangle rule, dV =
 * prod dx, gradient terms through Parseval with the plan's |xi|^2 of Eq.
 * (Gamma_fft) / (Gamma_fft_3d) or the FS-FD forms).  parts (may be NULL)
 * receives 2 + p values: chemical, c-gradient and each eta_i-gradient
 * contribution.  Synchronises.  Built for semi-implicit FS plans of one
 * simulation, 2D and 3D; batched and explicit-FD plans return
 * FS_ERR_UNSUPPORTED.  The spectra are overwritten: the next step starts
 * again from the real fields (as after fs_set_fields). */
FS_API fs_status fs_free_energy(fs_plan_t plan, double* F, double* parts);

/* Adjoint of one step linearised at the state u (nf real field pointers, plan
 * dtype, device memory): lambda_out = J(u)^T lambda_in, and grad_theta[0..3]
 * += d<lambda_in, step(u)>/d(M, L, kappa_c, kappa_eta).  The paper has no
 * adjoint; this is the transpose of the Jacobian of the Algorithm-1 step.
 * Uses the plan's workspace (the plan's own state is not modified).
 * Synchronises when grad_theta is not NULL.  Built for 2D and 3D
 * semi-implicit FS plans of one simulation (2D axes up to 1024; the 3D limits
 * of the plans, with |xi|^2 of Eq. (Gamma_fft_3d) or its FS-FD forms); others
 * return FS_ERR_UNSUPPORTED. */
FS_API fs_status fs_step_adjoint(fs_plan_t plan, const void* const* u, const void* const* lambda_in,
                          void* const* lambda_out, double grad_theta[4]);

/* Diagnostic timing: as fs_step_async with eager launches (no graph) and a
 * CUDA event pair recorded around every pass launch on the plan's stream.
 * fs_profile_read synchronises, writes the summed milliseconds and the launch
 * count of each pass kind since the last read to ms_per_pass[] and
 * launches_per_pass[] (may be NULL), at most npass_max entries, sets *npass
 * (2D: 0 row pass, 1 column pass) and returns the sticky device status. */
FS_API fs_status fs_step_profiled(fs_plan_t plan, int64_t nsteps);
FS_API fs_status fs_profile_read(fs_plan_t plan, double* ms_per_pass, int64_t* launches_per_pass, int npass_max,
                          int* npass);

/* Batched plans: the schedule the autotuner chose (it runs inside the first
 * fs_set_fields and times candidates on that state): per pass the kernel
 * form (1: half-length row pass / column tiles with radix-16 line
 * transforms; 2: warp-per-line kernels, one warp per line with radix up to
 * 32, two-column tiles -- FP32 members with both axes in [64, 1024]), the
 * persistent grid size (CTAs) and the number of work items.  Any output
 * pointer may be NULL. */
FS_API fs_status fs_batch_schedule(fs_plan_t plan, int64_t* row_grid, int64_t* col_grid, int64_t* row_items,
                                   int64_t* col_items, int* row_form, int* col_form);

/* Allocation-free 2D step, for callers that cannot allocate device memory:
 * a host program whose pool allocator owns all device memory before this
 * library is loaded, or code on a real-time / signal-handling path where a
 * cudaMalloc (which can synchronise the device and takes driver locks) is
 * not allowed.  The paper has no counterpart; it is a deployment
 * convenience.  Advances `fields` -- one device array of (1 + p) * nx * ny
 * values in the plan layout (c, eta_1 .. eta_p, x fastest), 16-byte aligned
 * -- by nsteps semi-implicit FS steps in place, with the same kernels and
 * results as a plan.  All intermediates live in one fixed file-scope device
 * array of 2,228,480 bytes that every GPU loading the library holds until
 * the process exits; the call makes no cudaMalloc / cudaFree and no host
 * heap allocation.
 *   - Limits: 2D, each axis a power of two in [8, 1024], nx * ny <= 65536,
 *     p <= 2, precision FS_F64 or FS_F32, scheme FS_SCHEME_SEMI_IMPLICIT_FS.
 *     Valid requests beyond them (3D, larger grids, p = 3 or 4, the
 *     tensor-core precisions, the explicit FD scheme) return
 *     FS_ERR_UNSUPPORTED before any CUDA call.  Malformed arguments (NULL
 *     pointers, nsteps < 0, a `fields` address that is not 16-byte aligned,
 *     dt <= 0, p outside [0, 4], unknown enum values) return
 *     FS_ERR_INVALID_ARG, also before any CUDA call.  fs_last_error() is not
 *     set.
 *   - The first call on a device looks up the array's device address with
 *     cudaGetSymbolAddress (with that device current); make that first call
 *     before any stream capture.
 *   - The call copies its tables from a static host array and synchronises
 *     `stream` (a cudaStream_t) before returning the status, so it returns
 *     FS_ERR_UNSUPPORTED, enqueueing nothing, when `stream` is capturing.
 *   - Every call shares the array and overwrites it.  Calls whose work
 *     overlaps on the GPU (several streams or host threads at once) race;
 *     serialise them. */
FS_API fs_status fs_step2d_static(const fs_params* prm, void* fields, int64_t nsteps, void* stream);

/* Kernel forms of the passes (FP32 plans; the paper's method is the same
 * either way, the rounding order differs).  row_form / col_form:
 *   1 = the half-length row pass (one real row as a complex line of nx/2)
 *       and the column-tile pass (radix-16 line transforms);
 *   2 = the warp-per-line forms: the row pass transforms two grid rows as
 *       one complex line (x lines of 64 to 1024 points), the column pass
 *       gives each (column, field) its own warp (2D columns of 64 to 1024
 *       points);
 *   3 = form 2 with two warps per line (lines of 128 to 1024 points, and
 *       2D columns of 2048): half the values per thread, twice the warps;
 *   4 = (both arguments) the fused step: the form-2 passes of every steady
 *       step of an fs_step call in one cooperative launch, grid-wide
 *       barriers between the passes (single 2D FS_F32 plans, square grids
 *       of 256, 512 or 1024 points, p <= 3; the first step after
 *       fs_set_fields runs the separate passes);
 *   0 = the default: form 2 for 2D lines of 256 to 1024 points, form 3 for
 *       2D columns of 2048, form 1 otherwise (3D x passes, with their many
 *       lines, keep form 1).
 * A form on a plan it does not cover returns FS_ERR_UNSUPPORTED (form 4 for
 * one pass only: FS_ERR_INVALID_ARG); FP64 plans
 * always run form 1.  On a batched plan a nonzero form pins the ensemble
 * kernels' form for that pass (the autotuner then only picks the grid size,
 * at the next fs_set_fields); 0 lets the autotuner choose.  Used by the
 * tests (both forms against the oracle) and for A/B timing. */
FS_API fs_status fs_set_pass_forms(fs_plan_t plan, int row_form, int col_form);

/* Test hook of the failure-detection path (the paper has no counterpart).
 * With enable = 1, the first bounded device wait of every pass this plan
 * launches gives up without polling: each pass sets the timeout flag, waits
 * (bounded) for its own copies to land and returns early, so the next
 * fs_step / fs_sync returns FS_ERR_TIMEOUT and the fields are unspecified.
 * With enable = 2, only the grid-wide barriers of the fused step (pass form
 * 4) give up without polling, with the same outcome.  enable = 0 restores
 * the normal poll limits; set the fields again before stepping on.  Nothing
 * hangs or faults: no wait is removed, only cut short.  Other values return
 * FS_ERR_INVALID_ARG.  Plans of one simulation only (batched plans return
 * FS_ERR_UNSUPPORTED). */
FS_API fs_status fs_test_short_wait(fs_plan_t plan, int enable);

/* Measurement helper (not part of the method): the FP64 instruction rate of
 * the current device, from a project-written kernel of independent DFMA
 * chains (and, if dadd_per_s is not NULL, DADD chains) timed with CUDA
 * events on `stream` (best of three launches after a warm-up).  Rates are
 * thread-instructions per second; FP64 flop/s = 2 * dfma_per_s.  The FP64
 * step is bound by this rate, not by HBM.  Allocates and frees 2 KB of
 * device memory; synchronises the stream. */
FS_API fs_status fs_measure_fp64_rate(void* stream, double* dfma_per_s, double* dadd_per_s);

/* Device bytes owned by the plan. */
FS_API fs_status fs_workspace_bytes(fs_plan_t plan, size_t* bytes);

/* Number of kernel launches issued by the last fs_step / fs_step_async. */
FS_API fs_status fs_last_launch_count(fs_plan_t plan, int64_t* launches);

/* Free everything the plan owns.  NULL is accepted. */
FS_API fs_status fs_destroy(fs_plan_t plan);

/* Text of the last error on `plan` (thread-local text for a NULL plan). */
FS_API const char* fs_last_error(fs_plan_t plan);

/* Library version string. */
FS_API const char* fs_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FS_H_ */
