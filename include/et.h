/* et.h — C ABI of the GB300 exponential-integrator library for the
 * Fisher-Kolmogorov glioblastoma model (Pabisz, Munoz-Matute, Paszynski,
 * arXiv 2402.02273).
 *
 * The library advances a tumour cell density u on an nx * ny * nz voxel grid
 * of spacing h by the exponential integrator of Sec. 2.2,
 *
 *     u^{n+1} = u^n + tau * phi1(tau A_n) (A_n u^n + f(u^n)),
 *
 * where A_n is the finite-difference diffusion operator L of Sec. 2.1
 * (eq. Amatrix) plus, in the default scheme, the linear part rho (1 - 2 u^n)
 * of the logistic term (eq. F / newF), and f(u^n) = rho (u^n)^2.  The action
 * tau phi1(tau A) b is evaluated as the top block of exp(tau B) v_1 with the
 * augmented matrix B of Sec. 2.2, as s sub-steps of a degree-m Taylor
 * polynomial, matrix-free, in hand-written CUDA kernels for sm_103a.
 *
 * Conventions for every entry point:
 *  - Arrays are dense, x fastest: voxel (i, j, k), 0-based, is element
 *    p = i + nx * (j + ny * k) (reading of the numbering formula of Sec. 2.1).
 *  - "device" pointers are CUDA global-memory addresses on the grid's device,
 *    8-byte aligned; "host" pointers are ordinary CPU memory (page-locked
 *    memory makes the copies asynchronous).  The caller owns every buffer it
 *    passes; the library keeps borrowed pointers only to the workspace.
 *  - Work is enqueued on the grid's CUDA stream; calls return without waiting
 *    unless stated.  Errors detected on the device (non-finite values, an
 *    out-of-range density) are collected in a device flag word and reported
 *    by et_sync_info, et_run_host and et_set_coeffs, which synchronise.
 *  - Every function returns ET_OK (0) or an error status and, for a non-NULL
 *    grid, stores a message readable with et_last_error; nothing throws and
 *    no argument error leaves work half-enqueued.
 */
#ifndef ET_H
#define ET_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ET_VERSION 100 /* 1.0.0 */

#if defined(__GNUC__)
#define ET_API __attribute__((visibility("default")))
#else
#define ET_API
#endif

typedef struct et_grid et_grid; /* opaque handle */

typedef enum {
    ET_OK = 0,
    ET_ERR_ARG = 1,         /* bad size, pointer, alignment, tau, option */
    ET_ERR_STATE = 2,       /* call order (e.g. et_step before et_set_coeffs) */
    ET_ERR_CUDA = 3,        /* a CUDA runtime call failed; message has details */
    ET_ERR_NUMERIC = 4,     /* D < 0 or not finite; u out of range or non-finite */
    ET_ERR_TIMEOUT = 5,     /* a bounded device-side wait ran out */
    ET_ERR_UNSUPPORTED = 6  /* combination the library does not provide */
} et_status;

/* Arithmetic of the Taylor-term kernels.  The state u is always FP64, and the
 * residual, the norm bound, the (s, m) selection and the update u += y are
 * FP64 in every form.
 *  ET_F64:  stencil terms and their sum in FP64 (the plain form).
 *  ET_F32:  stencil terms and their sum in FP32 (error about 1e-7 relative).
 *  ET_DF64: stencil terms and their sum in double-float pairs (hi + lo of two
 *           FP32 numbers, unit roundoff about 2^-48) on the FP32 pipes;
 *           FP64-level accuracy where the FP64 pipe is slow. */
typedef enum { ET_F64 = 0, ET_F32 = 1, ET_DF64 = 2 } et_precision;

/* Spatial operator L (Sec. 2.1; the printed formula is not in divergence form
 * and the paper states no boundary stencil, so two readings are provided;
 * in both, neighbours outside the box take the centre value, i.e. zero flux):
 *  ET_OP_CONSERVATIVE: (L v)_p = sum over the six faces of
 *      hm(D_p, D_q) / h^2 * (v_q - v_p),  hm(a, b) = 2ab / (a + b), 0 if a or b is 0;
 *      symmetric, mass-conserving (default).
 *  ET_OP_LITERAL: the Sec. 2.1 formula, i.e. row p of eq. Amatrix / h^2:
 *      (D_p + D_{p+e}) / h^2 towards +e, 2 D_p / h^2 towards -e, and a
 *      diagonal making the row sum zero. */
typedef enum { ET_OP_CONSERVATIVE = 0, ET_OP_LITERAL = 1 } et_operator;

/* Treatment of the logistic term rho u (1 - u) (Sec. 2.1, eq. F / newF):
 *  ET_SCHEME_ROSENBROCK: A_n = L + diag(rho (1 - 2 u^n)), f = rho (u^n)^2
 *      (the paper's fold; second order in tau) (default).
 *  ET_SCHEME_EXPEULER:   A = L, f = rho u^n (1 - u^n) (exponential Euler,
 *      first order). */
typedef enum { ET_SCHEME_ROSENBROCK = 0, ET_SCHEME_EXPEULER = 1 } et_scheme;

/* Choice of s and m, which Sec. 2.2 leaves to "proper selection".  Zero
 * fields take the defaults. */
typedef struct {
    double tol;       /* bound on the truncation error of one step, relative to
                         max|u^n|; default 1e-13 (F64, DF64), 1e-7 (F32) */
    double theta_max; /* largest tau/s * ||A - mu I||_inf per sub-step; default
                         32 with the shift (the e^{mu h} factor of a sub-step
                         cancels the growth of its partial sums), 7 (F64, DF64)
                         or 1.5 (F32) without it */
    int shift;        /* 1: shift A by mu = -max_p(off-diagonal row sum) (exact,
                         halves the norm); 0: no shift; -1 or 0-initialised
                         struct: default = 1 */
    int force_s;      /* > 0: use this many sub-steps */
    int force_m;      /* > 0: use this many Taylor terms per sub-step (>= 2) */
    int use_graph;    /* 1 (default): replay et_run / et_step as CUDA graphs;
                         -1: launch kernels directly */
    int single_terms; /* Taylor terms per launch (same arithmetic per voxel in
                         every case).  1: one.  -1: two consecutive terms of a
                         sub-step wherever the two-term kernel can run (F32,
                         DF64; about half the memory traffic).  0 (default):
                         DF64 two, F32 one (its four-voxel one-term kernel is
                         the faster), F64 always one */
    int timeout_probe_us; /* test hook, 0 (default): off.  1 .. 1000000: every
                         two-term launch (F32, DF64) first waits this many
                         microseconds on a device barrier that nothing
                         completes, so its bounded wait runs out: the run
                         stops early and the next synchronising call returns
                         ET_ERR_TIMEOUT (the state u is then not valid) */
    int every_row;    /* 0 (default): the one-term F64 and DF64 kernels
                         evaluate only dt z + beta b in warp rows (32
                         x-consecutive voxels) whose operator rows have no
                         off-diagonal entry (D = 0 around them,
                         et_get_zero_rows), and the DF64 two-term kernel at
                         each voxel whose six face weights are zero, and the
                         residual of every form in such rows; this gives the
                         full stencil's values up to the sign of zeros.  The
                         F32 term kernels evaluate every row.  1: every
                         product in every row (for comparison and timing) */
} et_options;

/* Per-step record written by the device (40 bytes). */
typedef struct {
    double umin, umax, mass; /* min, max and sum of u^{n+1}; mass / (nx ny nz)
                                is the paper's tumour volume (Sec. 3.5) */
    int s, m;                /* sub-steps and terms per sub-step used */
    unsigned flags;          /* ET_FLAG_* accumulated since the last sync */
    unsigned step;           /* index of the step within its et_run call */
} et_step_info;

#define ET_FLAG_NONFINITE 1u /* NaN or Inf met in u */
#define ET_FLAG_RANGE_IN  2u /* u^n outside [-1e-3, 1 + 1e-3] in the folded scheme:
                                the a-priori bound behind (s, m) did not hold */
#define ET_FLAG_D_INVALID 4u /* D < 0 or not finite (et_set_coeffs) */
#define ET_FLAG_TIMEOUT   8u /* a bounded device-side wait ran out (a TMA load
                                that never completed); the step is not valid */
#define ET_FLAG_TRUNCATION 16u /* the a-posteriori truncation estimate of a step
                                exceeded options.tol (see et_get_truncation);
                                informational: synchronising calls report it in
                                the record's flags, not as an error status */
#define ET_FLAG_CG_CAP    32u /* a Crank-Nicolson solve stopped at its iteration
                                cap before reaching its tolerance */

/* Bytes of device workspace a grid of this size needs (256-byte aligned
 * start required).  Returns 0 for non-positive sizes. */
ET_API size_t et_workspace_bytes(int nx, int ny, int nz, et_precision precision);

/* Creates a grid on the current CUDA device.
 *  nx, ny, nz  > 0 voxels per axis (nx * ny * nz < 2^31); h > 0 voxel width.
 *  workspace   device, >= et_workspace_bytes(...), 256-byte aligned,
 *              caller-owned, must outlive the grid.
 *  cuda_stream cudaStream_t to enqueue on (NULL = legacy default stream).
 *  out         receives the handle (NULL on failure).
 * Enqueues nothing. */
ET_API et_status et_create_grid(int nx, int ny, int nz, double h, et_precision precision,
                         void* workspace, size_t workspace_bytes, void* cuda_stream,
                         et_grid** out);

/* Sets the diffusion field and model constants (Sec. 2, Table 1).
 *  D       device, n FP64 values >= 0 (mm^2/day); read during the call only.
 *  rho     proliferation rate >= 0 (1/day).
 *  options NULL for defaults.
 * Builds the face weights of L in the workspace and the bound
 * max_p sum_{q != p} |L_pq|, then synchronises the stream (one 8-byte read).
 * ET_ERR_NUMERIC if some D is negative or not finite. */
ET_API et_status et_set_coeffs(et_grid* g, const double* D, double rho, et_operator op,
                        et_scheme scheme, const et_options* options);
/* Same as et_set_coeffs with the diffusion field dscale * D (dscale >= 0;
 * each product rounded once, in the coefficient kernel: the same weights as
 * et_set_coeffs on a field scaled beforehand in FP64).  For a uniform D scale
 * as a model parameter (its gradient comes from et_vjp) without a scaled
 * copy of D. */
ET_API et_status et_set_coeffs_scaled(et_grid* g, const double* D, double dscale, double rho, et_operator op,
                                      et_scheme scheme, const et_options* options);
/* Same as et_set_coeffs with D in host memory (copied through the workspace). */
ET_API et_status et_set_coeffs_host(et_grid* g, const double* D_host, double rho, et_operator op,
                             et_scheme scheme, const et_options* options);

/* One step u <- u + tau phi1(tau A)(A u + f(u)), in place.
 *  u    device, n FP64 values (the density, expected in [0, 1]).
 *  tau  step size > 0 (days).
 *  info device pointer to one et_step_info, or NULL (kept internally; read
 *       it with et_sync_info).
 * Asynchronous. */
ET_API et_status et_step(et_grid* g, double* u, double tau, et_step_info* info);

/* nsteps >= 1 steps of size tau, in place.  info: device array of nsteps
 * records, or NULL.  Asynchronous; replayed as one CUDA graph per
 * (u, info, tau, nsteps) after the first call (up to 8 kept per grid).  A
 * later et_set_coeffs keeps the graphs; a run replays one only if the new
 * coefficients give the same scalars (bound, rho, operator, scheme, options),
 * since the weights themselves are read from the workspace when it runs. */
ET_API et_status et_run(et_grid* g, double* u, double tau, int nsteps, et_step_info* info);

/* et_run on host buffers: copies u_host to the device, runs, copies u back
 * and, if info_host is non-NULL, the nsteps records; synchronises and returns
 * ET_ERR_NUMERIC if a device flag was raised. */
ET_API et_status et_run_host(et_grid* g, double* u_host, double tau, int nsteps,
                      et_step_info* info_host);

/* Synchronises the stream, copies the record of the latest step (whatever
 * info pointer that step was given) to host_out (may be NULL), clears the
 * device flags and returns ET_ERR_NUMERIC if NONFINITE or RANGE_IN was raised
 * since the previous sync. */
ET_API et_status et_sync_info(et_grid* g, et_step_info* host_out);

/* The (s, m, mu) that et_step / et_run use for step size tau on this grid,
 * and theta = tau / s * ||A - mu I||_inf bound. */
ET_API et_status et_get_schedule(const et_grid* g, double tau, int* s, int* m, double* mu,
                          double* theta);

/* Pure host function behind et_get_schedule (no CUDA call).
 *  rmax  max_p sum_{q != p} |L_pq| (1/day); rho, scheme as in et_set_coeffs.
 *  Minimises the number of stencil applications s*m - 1 subject to
 *  kappa * theta^m / m! * (1 + tau nu / (m+1)) / (1 - theta/(m+1)) <= tol and
 *  theta <= theta_max, with nu = ||A - mu I||_inf bound, theta = tau nu / s,
 *  kappa = tau (2 rmax + rho') e^{2 tau rho'} and rho' = rho (1 + 2e-3)
 *  (folded scheme; 0 for exponential Euler).  Returns ET_ERR_ARG if no pair
 *  with s <= 4096, m <= 96 qualifies. */
ET_API et_status et_select_schedule(double tau, double rmax, double rho, et_scheme scheme,
                             et_precision precision, const et_options* options, int* s,
                             int* m, double* mu, double* theta);

/* Changes the stream later calls enqueue on. */
ET_API et_status et_set_stream(et_grid* g, void* cuda_stream);

/* Per-step CUDA-event timing of the Taylor-term kernels inside et_run
 * (event records on the grid's stream around each step's term chain).
 * et_get_timing synchronises and returns the summed chain time of the last
 * et_run and the number of term-kernel launches in it. */
ET_API et_status et_enable_timing(et_grid* g, int enable);
ET_API et_status et_get_timing(et_grid* g, double* term_ms, long long* term_launches,
                        long long* other_launches);

/* Crank-Nicolson steps (Sec. 2.3, the paper's comparison method), in place.
 * The printed scheme is read as the trapezoidal rule on the same linearised
 * system as the exponential step:
 *     (I - tau/2 A_n) u^{n+1} = (I + tau/2 A_n) u^n + tau f_n,
 * solved for delta = u^{n+1} - u^n from (I - tau/2 A_n) delta = tau b_n by
 * matrix-free conjugate gradients in FP64, every scalar on the device, from
 * delta = 0 until ||r||_2 <= rtol ||tau b_n||_2 or max_iter iterations
 * (0: the a-priori cap of et_cn_iteration_cap).  A step that stops at the cap
 * raises ET_FLAG_CG_CAP (ET_ERR_NUMERIC at the next synchronising call).  One
 * step is captured as a CUDA graph (unless options.use_graph is -1) and
 * replayed nsteps times; iterations past convergence are empty launches.
 *  g       an ET_F64 grid with the conservative operator (the system is then
 *          symmetric positive definite when tau rho < 2), else
 *          ET_ERR_UNSUPPORTED; tau rho >= 2 in the folded scheme is ET_ERR_ARG.
 *  u, info as for et_run; a step's record has s = 0 and m = its iterations.
 *  rtol    in (0, 1).  Asynchronous.  Uses the grid's workspace (the
 *          exponential step's vectors), so it does not run concurrently with
 *          et_run on the same grid. */
ET_API et_status et_cn_run(et_grid* g, double* u, double tau, int nsteps, double rtol, int max_iter,
                           et_step_info* info);
/* The iteration cap et_cn_run takes for max_iter = 0: from Gershgorin bounds
 * on the spectrum of I - tau/2 A_n and the classical conjugate-gradient bound
 * ||r_k|| <= 2 sqrt(kappa) ((sqrt(kappa) - 1)/(sqrt(kappa) + 1))^k ||r_0||, plus
 * two.  0 for invalid arguments or before et_set_coeffs. */
ET_API int et_cn_iteration_cap(const et_grid* g, double tau, double rtol);

/* A-posteriori truncation estimate of the latest step (Sec. 2.2: the Taylor
 * series of the step is cut after m terms in each of s sub-steps).  Every
 * warp of a step's residual launch writes max|b| and max|u^n| of its voxels
 * (warp shuffles); the stats launch that ends the step reduces them with its
 * pass over u and evaluates
 *     est = C(s, m) max|b| / max|u^n|,
 *     C = tau e^{2 tau rho'} theta^m / m! (1 + tau nu / (m + 1)) / (1 - theta / (m + 1))
 * (the remainder bound behind et_select_schedule with the measured max|b| in
 * place of its a-priori bound (2 rmax + rho') max|u|; infinite if
 * theta >= m + 1) and raises ET_FLAG_TRUNCATION in the step's record when est
 * exceeds options.tol.  With the library's own schedules est <= tol whenever
 * u^n lies in [0, 1]; forced (s, m) can exceed it.  Synchronises the stream
 * and copies the latest step's estimate (relative to max|u^n|) to *estimate. */
ET_API et_status et_get_truncation(et_grid* g, double* estimate);

/* Voxels of the grid that lie in warp rows (32 x-consecutive voxels of one
 * grid row) without off-diagonal entries of the operator: every face weight
 * of the row's voxels is zero (D = 0 there and, for the conservative operator,
 * on one side of each face).  A one-term launch evaluates dt z + beta b there
 * (FP64: two FP64 instructions and 32 bytes a voxel instead of eight and 56),
 * unless options.every_row is set; the results are those of the full
 * stencil, whose skipped products are exact zeros, up to the sign of zeros.
 * The F64 and DF64 one-term kernels and the residual of every form skip such
 * rows, the DF64 two-term kernel skips the arithmetic of each voxel with six
 * zero weights (its loads are whole tiles), the F32 term kernels evaluate
 * every row.  Counted by et_set_coeffs; synchronises the stream. */
ET_API et_status et_get_zero_rows(et_grid* g, long long* voxels);

/* Grid facts: n voxels, bytes of the workspace actually used, and the
 * diffusion bound rmax (0 before et_set_coeffs). */
ET_API et_status et_get_info(const et_grid* g, long long* nvoxels, size_t* ws_used, double* rmax);

/* Vector-Jacobian product of nsteps steps (reverse mode, the discrete adjoint
 * of the computed step with every step's (s, m, mu) frozen):  given
 * ubar_final = dJ/du^K for u^K = step^K(u0), returns dJ/du0 in ubar0, dJ/drho
 * in *grad_rho and d/ds J(s D)|_{s=1} (D scaled uniformly) in *grad_dscale.
 * Runs its own forward pass from u0 keeping u every checkpoint_every steps,
 * then runs each segment forward once more, recording every step (its b,
 * diagonal and Taylor terms), and reverses the segment's steps.  The workspace
 * holds the checkpoints and one segment's records (about checkpoint_every x
 * (s m + s + 3) vectors of the grid's precision).  ET_F64 and ET_F32 grids
 * (ET_ERR_UNSUPPORTED for ET_DF64).
 *  u0, ubar_final, ubar0: device, n FP64 values (ubar0 may alias neither).
 *  workspace: device, >= et_vjp_workspace_bytes(...), 256-byte aligned.
 * Synchronises the stream (the two gradients are read back). */
ET_API size_t et_vjp_workspace_bytes(const et_grid* g, double tau, int nsteps, int checkpoint_every);
ET_API et_status et_vjp(et_grid* g, const double* u0, double tau, int nsteps, int checkpoint_every,
                        const double* ubar_final, double* ubar0, double* grad_rho, double* grad_dscale,
                        void* workspace, size_t workspace_bytes);
/* The same adjoint split in two, so that a forward run and its reverse pass
 * share one pass: et_run_checkpointed advances u (device, in place) by nsteps
 * steps like et_run and keeps the checkpoints in the adjoint workspace;
 * et_vjp_checkpointed then runs the reverse pass from them (same tau, nsteps,
 * checkpoint_every and workspace; coefficients unchanged in between).  The
 * results equal et_vjp's from the same u0. */
ET_API et_status et_run_checkpointed(et_grid* g, double* u, double tau, int nsteps, int checkpoint_every,
                                     void* workspace, size_t workspace_bytes);
ET_API et_status et_vjp_checkpointed(et_grid* g, double tau, int nsteps, int checkpoint_every,
                                     const double* ubar_final, double* ubar0, double* grad_rho,
                                     double* grad_dscale, void* workspace, size_t workspace_bytes);

/* ---- Batched form: many grids (patients, scenarios) advanced together ----
 * Grids of different sizes, each with its own D, rho and (s, m) schedule, share
 * one workspace with their fields concatenated in grid order.  Each step is one
 * batched residual launch, one batched launch per Taylor-term index (covering
 * every grid whose chain has that term) and one batched stats launch; a run is
 * captured as one CUDA graph.  The term-launch kernel variant (planes per tile,
 * looping or one-tile-per-block grids) is picked by timing the candidates on
 * the batch (et_batch_autotune, or automatically on the first run).  As on a
 * single grid, the FP64 one-tile-per-block kernel and the DF64 kernels skip
 * the products of rows without off-diagonal entries unless options.every_row
 * is set (et_batch_set_coeffs marks those rows per grid).
 *  dims: host array of 3*count ints (nx, ny, nz of grid i at 3i); count <= 1024.
 *  D, u: device, the grids' fields concatenated in order (sum of n_i FP64).
 *  rho: host array of count rates.  info: device array of nsteps*count records
 *  (record of grid i after step t at t*count + i), or NULL. */
typedef struct et_batch et_batch;
ET_API size_t et_batch_workspace_bytes(int count, const int* dims, et_precision precision);
ET_API et_status et_batch_create(int count, const int* dims, double h, et_precision precision, void* workspace,
                                 size_t workspace_bytes, void* cuda_stream, et_batch** out);
ET_API et_status et_batch_set_coeffs(et_batch* b, const double* D, const double* rho, et_operator op,
                                     et_scheme scheme, const et_options* options);
ET_API et_status et_batch_run(et_batch* b, double* u, double tau, int nsteps, et_step_info* info);
/* Times every kernel variant on the first launch of every grid's chain and
 * keeps the fastest.  Variants: planes per tile and looping blocks of the
 * one-term kernel, and for ET_F32 / ET_DF64 each of these with two terms of a
 * sub-step per launch (the first half of the index range).  us_per_variant
 * (host, et_batch_variant_count entries, may be NULL) receives microseconds
 * per Taylor term of the whole batch. */
ET_API et_status et_batch_autotune(et_batch* b, double tau, int* variant, double* us_per_variant);
ET_API int et_batch_variant_count(et_precision precision);
/* Uses kernel variant `variant` (0 .. et_batch_variant_count - 1) instead of the
 * autotuner's choice until the next et_batch_set_coeffs or et_batch_autotune. */
ET_API et_status et_batch_set_variant(et_batch* b, int variant);
/* Synchronises; copies the latest record of every grid (count records). */
ET_API et_status et_batch_sync_info(et_batch* b, et_step_info* host_out);
ET_API et_status et_batch_get_schedule(const et_batch* b, double tau, int* s, int* m);
/* Voxels of all grids that lie in warp rows without off-diagonal entries (as
 * et_get_zero_rows, per grid, summed); voxels: host, count entries, the
 * per-grid figures (NULL: only the total); *total may be NULL.  Marked by
 * et_batch_set_coeffs; synchronises the stream. */
ET_API et_status et_batch_get_zero_rows(et_batch* b, long long* voxels, long long* total);
ET_API et_status et_batch_set_stream(et_batch* b, void* cuda_stream);
ET_API const char* et_batch_last_error(const et_batch* b);
ET_API void et_batch_destroy(et_batch* b);

/* One step that allocates nothing (the paper has no counterpart; it exists for
 * callers that cannot allocate device memory at call time, e.g. code inside a
 * framework whose pool owns all device memory, or code run while a memory
 * budget is locked).  Same arithmetic as et_set_coeffs + et_step in FP64, with
 * all scratch in one static device array of the library (22 MiB, held by
 * every GPU that loads it until exit) instead of a workspace.
 *  nx, ny, nz, h, rho, op, scheme, tau: as for et_create_grid / et_set_coeffs
 *      / et_step; at most 64^3 = 262144 voxels, nz <= 65535 and 65536 blocks
 *      of the 32 x 8 tile, else ET_ERR_ARG.
 *  D    device, n FP64 values (read); u device, n FP64 values (in/out).
 *  cuda_stream  stream to run on; msg/msg_len optional buffer for an error
 *      message (may be NULL).
 * The first call in each CUDA context of a device looks up the array's address
 * (cudaGetSymbolAddress) with that device current and caches it by the
 * context's id; make that first call before any stream capture.  Calls share the
 * array: calls that overlap on the GPU race.  Synchronises the stream and
 * returns ET_ERR_NUMERIC for bad D or a non-finite / out-of-range density. */
ET_API et_status et_step_static(int nx, int ny, int nz, double h, const double* D, double rho,
                                et_operator op, et_scheme scheme, double* u, double tau,
                                void* cuda_stream, char* msg, size_t msg_len);

/* Diagnostic, not part of the method: measured FMA throughput of the device
 * (FP64 and FP32, TFLOP/s counting an FMA as 2 flops), the ALU roofline of the
 * stencil kernels.  scratch: device buffer of >= et_probe_alu_scratch_bytes()
 * bytes.  Synchronises the stream; takes about 20 ms. */
ET_API size_t et_probe_alu_scratch_bytes(void);
ET_API et_status et_probe_alu(void* scratch, size_t scratch_bytes, void* cuda_stream,
                              double* fp64_tflops, double* fp32_tflops);
/* Diagnostic, not part of the method: best streaming bandwidth (bytes read
 * plus bytes written per second, GB/s) of a plain device kernel that writes
 * dst[i] = the sum of nin input buffers at i (16-byte vectors), over a few
 * launch shapes, each timed over `reps` back-to-back passes with CUDA events on
 * cuda_stream.  nin = 1 is a copy; nin = 6 has the read/write mix of a stencil
 * term.  With buffers inside the L2 this is the L2 roofline of an L2-resident
 * kernel; with buffers far beyond it, the HBM roofline.
 *  src: device, nin consecutive buffers of `bytes` each; dst: device, `bytes`,
 *  not overlapping src; both 16-byte aligned; bytes a positive multiple of 16;
 *  1 <= nin <= 8.  Synchronises the stream. */
ET_API et_status et_probe_stream(const void* src, void* dst, size_t bytes, int nin, int reps, void* cuda_stream,
                                 double* gbs);

ET_API const char* et_last_error(const et_grid* g); /* g may be NULL: last create error */
ET_API const char* et_status_string(et_status status);
ET_API int et_version(void);
ET_API void et_destroy(et_grid* g); /* frees graphs and events; not the workspace */

#ifdef __cplusplus
}
#endif
#endif /* ET_H */
