/*
 * pat.h — C ABI of the GB300 photoacoustic reconstruction library.
 *
 * The library solves the wavelet-Sobolev / Matern regularised PAT problem of
 * Kultima, Ramlau, Sahlstrom, Tarvainen (arXiv 2507.02401):
 *
 *     min_u  1/2 || K E_s u - y ||^2 + alpha/2 || u ||^2 ,     x = E_s u,
 *
 * i.e. the normal equations (E_s* K* K E_s + alpha I) u = E_s* K* y, which
 * are the paper's Eq. (linear_minimization) written in wavelet coefficients
 * (multiply by E_s to recover (E_s E_s* K* K + alpha I) x = E_s E_s* K* y).
 *
 *   K    photoacoustic forward map (Sec. 2.2): initial pressure p0 on an
 *        n^d grid -> pressure at Ns point sensors for nt time samples, from
 *        the wave IVP of Eq. (wave_equation) discretised as a staggered
 *        leapfrog of spatial order 2M (2, 4, 6, 8), pressure zero outside
 *        the grid, p_t(0) = 0.
 *   K*   its exact discrete adjoint (transpose, Euclidean inner products).
 *   E_s  wavelet form of the Sobolev embedding (Sec. 4, Prop. 4.2): periodic
 *        orthonormal Daubechies synthesis W^T after scaling the level-i detail
 *        block by 2^{-s(m-i+o)} (i = 1 finest, m levels, o = level offset);
 *        E_s* = S_s W is its adjoint, and E_s E_s* = W^T S_s^2 W is the
 *        paper's operator W^{-1}(D W .) of Sec. 4.
 *
 * Conventions for every call:
 *   - Grids are row-major with x fastest: cell (x, y[, z]) at
 *     (z*ny + y)*nx + x, cell centre at (x*h, y*h, z*h).
 *   - Sensor data y are sensor-major: y[s*nt + t], t = 0 .. nt-1, t = 0 being
 *     the initial pressure itself.
 *   - Coefficient vectors u have N = n^d entries laid out as
 *     [cA_m, bands_m, bands_{m-1}, ..., bands_1], every band row-major;
 *     2D bands in the paper's order (H = x low/y high, V = x high/y low,
 *     D = both high), 3D bands in binary (z,y,x) order 001 .. 111 (1 = high).
 *   - Array pointers may be device pointers (fast path) or host pointers
 *     (pageable or pinned); host arrays are staged through plan-owned device
 *     buffers inside the call, which then returns only after the result is
 *     back on the host.  The caller owns every array it passes.
 *   - Calls with device pointers are asynchronous on `stream` (a
 *     cudaStream_t, NULL = legacy default stream).  Argument errors are
 *     returned immediately; device-side conditions (a timed-out wait inside a
 *     persistent kernel, a CG breakdown) are recorded in the plan and
 *     returned by pat_plan_check().
 *   - Calls on one plan must not overlap in time (they share the plan's
 *     workspace); different plans are independent.
 *   - Nothing aborts the process: errors are status codes, with a message in
 *     pat_last_error().
 */
#ifndef PAT_H
#define PAT_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pat_plan pat_plan;

typedef enum {
  PAT_OK = 0,
  PAT_ERR_INVALID = 1,   /* bad argument (sizes, order, sensor outside grid, NaN, ...) */
  PAT_ERR_CFL = 2,       /* c_max dt / h above the stability limit of the chosen order */
  PAT_ERR_CUDA = 3,      /* a CUDA runtime call failed */
  PAT_ERR_OOM = 4,       /* device allocation failed */
  PAT_ERR_TIMEOUT = 5,   /* a bounded wait in a persistent kernel ran out */
  PAT_ERR_BREAKDOWN = 6  /* CG met p.q <= 0 or a non-finite scalar; last iterate kept */
} pat_status;

/* Grid: dim = 2 or 3; n = {nx, ny, nz} (nz ignored for dim 2); spacing h [m]. */
typedef struct {
  int dim;
  int n[3];
  double h;
} pat_grid;

/* Wavelet: family = number of vanishing moments (1 = Haar, 2 = db2, 4 = db4);
 * levels m >= 1 with every n[i] divisible by 2^m; level_offset o >= 0
 * (0 = the paper's inline weight 2^{-2s(m-i)} for E_s E_s*). */
typedef struct {
  int family;
  int levels;
  int level_offset;
} pat_wavelet;

/*
 * pat_plan_create — validate a problem and build its device constants.
 * Paper Sec. 2 (Eq. wave_equation, the sensor map K) and Sec. 4 (W, D).
 *   grid     grid description (host).
 *   c        host array of N speeds of sound [m/s] (double), or NULL to use
 *            the constant c0.  Must be finite and > 0.
 *   sensors  host array ns x dim of sensor coordinates (x, y[, z]) [m]; each
 *            must lie in [0, (n_i - 1) h] (bilinear/trilinear sampling).
 *   dt, nt   time step [s] and number of samples (nt >= 1).
 *   order    spatial order 2, 4, 6 or 8 of the staggered scheme.  The plan
 *            is rejected with PAT_ERR_CFL when c_max dt / h exceeds
 *            1 / (sqrt(dim) * sum_k |c_k|) for the order's staggered weights.
 *   wavelet  wavelet description (host).
 *   stream   stream for the set-up copies (the call synchronises it).
 *   out      receives the plan; owns all device memory it needs (device
 *            constants and the workspace of every call).
 */
pat_status pat_plan_create(const pat_grid* grid, const double* c, double c0, const double* sensors, int ns,
                           double dt, int nt, int order, const pat_wavelet* wavelet, void* stream,
                           pat_plan** out);

/* Frees a plan and all device memory it owns.  NULL is ignored. */
void pat_plan_destroy(pat_plan* plan);

/* Sizes of a plan: number of cells N (= coefficient count), sensors, samples. */
pat_status pat_plan_info(const pat_plan* plan, long long* n_cells, int* ns, int* nt);

/*
 * pat_forward — y = K x.  Paper Sec. 2.2 (K: p0 -> [p(r_i, t_j)]).
 *   x  N floats (initial pressure).   y  ns*nt floats (sensor-major).
 */
pat_status pat_forward(pat_plan* plan, const float* x, float* y, void* stream);

/*
 * pat_adjoint — x = K* y, the exact transpose of pat_forward (reverse-time
 * recurrence with transposed sensor injection).  Paper Sec. 4 (K* needed by
 * the matrix-free solver).   y  ns*nt floats.   x  N floats.
 * FP32 fields; in 2D the adjoint state (kappa Q, which integrates the data
 * over time) is carried as a compensated pair, so the result stays within
 * ~1e-6 relative of the exact transpose for data simulated from a phantom.
 */
pat_status pat_adjoint(pat_plan* plan, const float* y, float* x, void* stream);

/*
 * pat_Es — x = E_s u = W^T S_s u (coefficients -> image).  Paper Sec. 4,
 * Prop. 4.2 (diagonal scaling of the wavelet coefficients).
 *   s  smoothness index (any real; s = 0 gives W^T).   u, x  N floats.
 */
pat_status pat_Es(pat_plan* plan, double s, const float* u, float* x, void* stream);

/* pat_EsT — u = E_s* x = S_s W x (image -> coefficients).  Paper Sec. 4. */
pat_status pat_EsT(pat_plan* plan, double s, const float* x, float* u, void* stream);

/*
 * pat_solve — CG on (E_s* K* K E_s + alpha I) u = E_s* K* y for `iters`
 * iterations (paper Eq. linear_minimization, Sec. 4 "GMRES or CG"; each
 * iteration costs one K and one K*, plus one K* for the right-hand side).
 * Vectors are FP32; inner products, step lengths and the residual norm are
 * FP64 on the device; no host synchronisation inside.
 *   y      ns*nt floats (data).         alpha  absolute regularisation > 0.
 *   s      smoothness index.            iters  >= 0.
 *   u0     N floats initial coefficients, or NULL for u0 = 0.
 *   u      N floats, final coefficients (may be NULL).
 *   x      N floats, final image E_s u (may be NULL).
 *   log    NULL or a DEVICE array of iters*3 doubles receiving, per
 *          iteration k, (r_k.r_k, p_k.q_k, a_k).
 * A breakdown keeps the last iterate and is reported by pat_plan_check().
 */
pat_status pat_solve(pat_plan* plan, const float* y, double alpha, double s, int iters, const float* u0, float* u,
                     float* x, double* log, void* stream);

/*
 * pat_solve_gmres — the paper's solver (Sec. 4 and 5: GMRES, 15 iterations
 * = 31 wave evaluations in its experiments) on the image-space system of
 * Eq. linear_minimization with the covariance Gamma = E_s E_s*:
 *   (Gamma K* K + alpha I) x = Gamma K* y,   x_0 = 0.
 * Arnoldi with classical Gram-Schmidt applied twice (FP32 basis vectors, FP64
 * inner products reduced in a fixed order, all projections of a pass in one
 * launch), Givens rotations and the Hessenberg matrix on the host in FP64.  Converges to the same minimiser as pat_solve
 * (x = E_s u).  Synchronous; allocates the (iters+1) x N basis per call.
 *   x    N floats (output; device or host).
 *   res  NULL or HOST array of iters+1 doubles: ||f - A x_k|| for k = 0..iters.
 *   J    NULL or HOST array of iters+1 doubles: J(u_k) = 1/2 ||K x_k - y||^2
 *        + alpha/2 ||u_k||^2 with u_k = E_s^{-1} x_k (costs one extra K per
 *        iteration).
 * Errors: PAT_ERR_INVALID (arguments), PAT_ERR_OOM (basis), PAT_ERR_CUDA.
 */
pat_status pat_solve_gmres(pat_plan* plan, const float* y, double alpha, double s, int iters, float* x, double* res,
                           double* J, void* stream);

/*
 * pat_solve_landweber — the Landweber (gradient) iteration on the coefficient
 * system: u_{k+1} = u_k - omega ((E_s* K* K E_s + alpha I) u_k - E_s* K* y),
 * u_0 = 0; it converges for 0 < omega < 2 / lambda_max.  Synchronous.
 *   u, x  N floats (outputs, may be NULL): final coefficients and image E_s u.
 *   J     NULL or HOST array of iters+1 doubles: J(u_k) for k = 0..iters
 *         (the forward map of each iterate is computed anyway; the last value
 *         costs one extra K).
 */
pat_status pat_solve_landweber(pat_plan* plan, const float* y, double alpha, double s, int iters, double omega,
                               float* u, float* x, double* J, void* stream);

/*
 * pat_solve_multi — nrhs pat_solve problems on one plan (same grid, medium
 * and sensors; each with its own data ys[r], alphas[r], ss[r]; u0 = 0; a
 * common iteration count), advanced two at a time: on the persistent engine
 * (no absorbing layer) every K and every K* of a pair runs as one launch
 * carrying both fields, so the pair shares each time step's halo exchange
 * and barrier (the paper's CG of Sec. 4 applied to several regularisations
 * of one measurement, e.g. a sweep over alpha and s).  Each right-hand side
 * gets exactly the result pat_solve gives it.  Other engines run the
 * problems one after the other.
 *   ys, xs   host arrays of nrhs DEVICE pointers (Ns*nt floats in, N floats
 *            out: x = E_s u after `iters` CG iterations).
 *   alphas, ss  host arrays of nrhs doubles (alpha > 0, s finite).
 * Asynchronous on `stream`; device status through pat_plan_check.  The first
 * call with nrhs >= 2 allocates the second right-hand side's buffers.
 * Errors: PAT_ERR_INVALID (NULL or host arrays, nrhs < 1, bad alpha / s),
 * PAT_ERR_CUDA, PAT_ERR_OOM.
 */
pat_status pat_solve_multi(pat_plan* plan, int nrhs, const float* const* ys, const double* alphas,
                           const double* ss, int iters, float* const* xs, void* stream);

/*
 * pat_objective — the Tikhonov functional whose minimiser pat_solve computes
 * (paper Sec. 3, the variational problem behind Eq. (linear_minimization),
 * in wavelet coefficients):
 *     J(u) = 1/2 ||K E_s u - y||^2 + alpha/2 ||u||^2
 * and, optionally, its gradient E_s* K* (K E_s u - y) + alpha u.  Reductions
 * in FP64 in a fixed order (bit-reproducible).  Synchronous.
 *   y      Ns*nt floats, u  N coefficients (device or host arrays).
 *   alpha  >= 0 (absolute), s  finite.
 *   J      HOST pointer to one double (output).
 *   grad   NULL or N floats (device or host; output).
 * Uses the plan's image and data buffers (not concurrently with other calls on
 * the same plan).  PAT_ERR_INVALID for NULL y / u / J or a non-finite alpha or s.
 */
pat_status pat_objective(pat_plan* plan, const float* y, double alpha, double s, const float* u, double* J,
                         float* grad, void* stream);

/*
 * pat_solve_batched — B independent pat_solve problems (each with its own
 * plan, data, alpha and s; a common iteration count) advanced together.
 * When every plan qualifies for a batch (see pat_batch_create) and ys / xs
 * are device arrays, this is pat_batch_create + pat_batch_solve +
 * pat_batch_destroy (tuning included); otherwise the instances are solved
 * one after the other with pat_solve.
 *   plans, ys, xs   host arrays of B plan / device-array pointers (xs[i]
 *                   receives E_s u of instance i).
 *   alphas, ss      host arrays of B doubles.
 *   per_inst        NULL or host array of B statuses; filled after the call
 *                   synchronises `stream` (the call is synchronous).
 */
pat_status pat_solve_batched(pat_plan* const* plans, int B, const float* const* ys, const double* alphas,
                             const double* ss, int iters, float* const* xs, pat_status* per_inst, void* stream);

/*
 * Batched engine.  Not in the paper (it reconstructs one image); the paper's
 * CG (Sec. 4) is run for many independent problems at once.
 *
 * pat_batch_create — group B plans into one batch.  Every plan must be 2D,
 * with the same stencil order, nx % 4 == 0 and no absorbing layer, and
 * appear once (the batch uses each plan's device buffers; the plans must
 * outlive the batch and must not be used concurrently with it).  Grid size,
 * time samples, sensors, medium (constant or varying speed of sound),
 * wavelet, alpha and s may differ.  All instances' 64-column tiles form one
 * table; each time step of K or K* walks the tiles of the instances still
 * running (one launch per step, or all steps in one launch: see
 * pat_batch_launch).  The tile height (64 or 32
 * rows) is chosen by timing both on the first steps of a batched K and K*
 * (an autotuner; PAT_BATCH_TILE_Y=64|32 in the environment fixes it).  The
 * batched K* keeps its state Z = kappa Q as a compensated pair in the plans'
 * field buffers (it overwrites three of them).
 * Synchronises `stream`.  Errors: PAT_ERR_INVALID (NULL, duplicate or
 * ineligible plan), PAT_ERR_CUDA, PAT_ERR_OOM.
 */
typedef struct pat_batch pat_batch;
pat_status pat_batch_create(pat_plan* const* plans, int B, void* stream, pat_batch** out);
void pat_batch_destroy(pat_batch* batch);

/*
 * pat_batch_forward / pat_batch_adjoint — K (or K*) of every instance:
 * xs[i] (N_i floats) -> ys[i] (ns_i x nt_i floats), or back.  Device arrays;
 * asynchronous on `stream`.
 */
pat_status pat_batch_forward(pat_batch* batch, const float* const* xs, float* const* ys, void* stream);
pat_status pat_batch_adjoint(pat_batch* batch, const float* const* ys, float* const* xs, void* stream);

/*
 * pat_batch_solve — pat_solve (u0 = 0) for every instance with its own
 * alphas[i] and ss[i] and a common `iters`.  One CG iteration of all
 * instances (E_s, batched K and K*, E_s*, FP64 CG scalars) is captured once
 * as a CUDA graph (re-captured when alphas or ss change) and replayed
 * `iters` times.  ys, xs: host arrays of B device pointers.  per_inst: NULL
 * or B statuses (breakdown per instance, timeout of the batched kernel).
 * Synchronous.  Returns the first non-OK status.
 */
pat_status pat_batch_solve(pat_batch* batch, const float* const* ys, const double* alphas, const double* ss,
                           int iters, float* const* xs, pat_status* per_inst, void* stream);

/*
 * pat_batch_info — tile height in use, CTAs per step launch, nodes of the
 * captured CG-iteration graph (0 before the first solve) and the autotuner's
 * times (ms; the first steps of K plus K*) of the 64-row and 32-row tiles.
 * Any output may be NULL.
 */
pat_status pat_batch_info(pat_batch* batch, int* tile_rows, int* ctas, long long* graph_nodes, double* tune_ms);

/*
 * pat_batch_launch — launch form of the batched K and K*.  Form 1: one
 * launch per time step (each walks the tiles still running).  Form 2: one
 * cooperative launch per application: every CTA co-resident, a grid-wide
 * barrier between time steps (each wait bounded: a CTA that gives up records
 * PAT_ERR_TIMEOUT, which the others see at their next barrier, and all
 * leave).  At creation the autotuner times both on the first steps of a K
 * plus K* and keeps the faster.
 *   mode    -1: query only; 0: the autotuner's choice; 1: per step; 2: one
 *           launch per application.  Changing the form drops the captured
 *           CG-iteration graph (re-captured at the next solve).
 *   runall  NULL or out: 1 when form 2 is in use.
 *   ms      NULL or out, 2 doubles: the autotuner's times (ms) of forms 1, 2.
 * Not in the paper (its one reconstruction has no batch).
 */
pat_status pat_batch_launch(pat_batch* batch, int mode, int* runall, double* ms);

/*
 * pat_grad_kappa — g = d<r, K x>/d kappa per cell, kappa = (c dt / h)^2: the
 * sensitivity of the measurements to the medium, e.g. the gradient of
 * J = 1/2 ||K x - y||^2 with r = K x - y (chain rule for c: dkappa/dc =
 * 2 kappa / c).  Not in the paper (its medium is known); used to
 * differentiate K with respect to c.  With the three-level form
 * P^{n+1} = 2P^n - P^{n-1} + kappa .* L P^n and adjoint states Q^n of K*r:
 *   g = sum_{n=1}^{nt-2} Q^{n+1} .* L P^n + 1/2 Q^1 .* L P^0.
 * The forward fields are needed in reverse order: the forward run keeps its
 * restart state every `segment` steps (0 = ceil(sqrt(nt))) and each segment is
 * recomputed when the adjoint reaches it.  Runs on the per-step engine.
 *   x  N floats;  r  ns*nt floats;  g  N floats (output).
 * Memory: (2 ceil((nt-1)/segment) + segment + 3) N floats + N doubles,
 * allocated by the first call and kept by the plan (PAT_ERR_OOM if absent).
 */
pat_status pat_grad_kappa(pat_plan* plan, const float* x, const float* r, float* g, int segment, void* stream);

/*
 * pat_plan_check — synchronises `stream`, returns and clears the plan's
 * device-side status (PAT_OK, PAT_ERR_TIMEOUT or PAT_ERR_BREAKDOWN), or
 * PAT_ERR_CUDA if the stream reports an error.
 */
pat_status pat_plan_check(pat_plan* plan, void* stream);

/*
 * Wave engine of a plan (tuning and testing):
 *   PAT_PATH_AUTO        default choice (persistent when available)
 *   PAT_PATH_PERSISTENT  2D only: one cooperative launch per K / K* with the
 *                        wavefield kept on chip; available when every 64 x 32
 *                        tile of the grid can be resident at once
 *   PAT_PATH_STEP        one launch per time step (any grid; 3D always)
 * Both engines compute the same operators (to FP32 rounding).
 */
typedef enum { PAT_PATH_AUTO = 0, PAT_PATH_PERSISTENT = 1, PAT_PATH_STEP = 2 } pat_path;
pat_status pat_plan_set_path(pat_plan* plan, int path);
pat_status pat_plan_get_path(const pat_plan* plan, int* path);

/*
 * pat_plan_set_prior — choose the form of E_s.  kind 0: the periodic
 * Daubechies wavelet form (the default, Prop. 4.2).  kind 1: the Fourier
 * form of Sec. 4 (implementation), where the paper applies its adjoint
 * embedding as ifft(B . fft(X)) with the Bessel potential
 * B = (1 + 4 pi^2 |xi|^2)^{-s}; that operator is this library's covariance
 * E_s E_s*, so E_s (= E_s*) is the filter with (1 + 4 pi^2 |xi|^2)^{-s/2}.
 * Lengths are measured in units of `length_cells` cells: DFT index k of an
 * n-cell axis is xi = k' length_cells / n, k' = k (k < n/2) or k - n.
 * Coefficients then live on the grid (N values, no wavelet bands).  Requires
 * a 2D grid with power-of-two extents up to 4096 (PAT_ERR_INVALID
 * otherwise).  Allocates two complex N-buffers on first use.
 */
pat_status pat_plan_set_prior(pat_plan* plan, int kind, double length_cells, void* stream);

/*
 * pat_plan_set_sponge — absorbing layer of `width` cells along every face of
 * a 2D grid (width = 0 removes it).  The paper's simulations absorb outgoing
 * waves with a perfectly matched layer of 10 grid points (Sec. 5); this
 * library's reading is a damping term in the pressure equation,
 * p_t + sigma(x) p = -c^2 div v, with sigma p averaged over the two time
 * levels, which changes the eliminated update to
 *   D^{n+1} = a D^n + b kappa L P^n,   a = (1-q)/(1+q), b = 1/(1+q), q = sigma dt/2
 * (first step D^1 = (a-1) P^0 + b kappa/2 L P^0), with K* its exact transpose.
 * Profile: sigma = sigma_max ((width - d)/width)^2 within `width` cells of a
 * face (d = cells to that face), summed over the two axes.
 *   sigma_max  damping rate at the faces [1/s]; 0 selects
 *              3 c_max ln(1e3) / (2 width h) (nominal reflection 1e-3).
 * Both 2D engines (persistent and per-step) carry the layer; the medium
 * gradient and batches reject plans with one.
 * Errors: PAT_ERR_INVALID for 3D plans, width < 0, 2 width > nx or ny, or a
 * negative / non-finite sigma_max.  Synchronises `stream`.
 */
pat_status pat_plan_set_sponge(pat_plan* plan, int width, double sigma_max, void* stream);

/* Bound (nanoseconds, default 2e9) on any single inter-tile wait inside the
 * persistent engine; when it runs out the call ends early and
 * pat_plan_check() reports PAT_ERR_TIMEOUT. */
pat_status pat_plan_set_timeout(pat_plan* plan, long long timeout_ns);

/*
 * Measurement hooks.  While enabled, every wave-engine application (one K or
 * one K*) is bracketed by CUDA events recorded on the stream it runs on, and
 * every kernel the plan launches is counted.  pat_plan_profile(plan, 1)
 * clears the counters; pat_plan_profile_read synchronises on the recorded
 * events and returns: kernels launched, wave applications timed, their
 * summed device time [ms] and the point-updates they made (cells x steps).
 */
pat_status pat_plan_profile(pat_plan* plan, int enable);
pat_status pat_plan_profile_read(pat_plan* plan, long long* kernels, int* wave_calls, double* wave_ms,
                                 long long* point_updates);

/*
 * pat_EsT_noalloc — u = E_s* x for a 2D image, with no device allocation at
 * all.  The paper has no counterpart: this is a deployment form of pat_EsT
 * for callers that cannot allocate device memory (a real-time loop that must
 * not pay cudaMalloc's implicit synchronisation, a plug-in whose host
 * application owns the device memory, a fixed up-front memory budget), and
 * so cannot create a plan.
 *   nx, ny        grid extents; nx * ny <= 2^20 cells (e.g. 1024 x 1024),
 *                 both divisible by 2^levels.  Larger grids are rejected with
 *                 PAT_ERR_INVALID and a message naming the limit.
 *   family, levels, level_offset, s   as for pat_plan_create / pat_EsT.
 *   x             device array of nx*ny floats (row-major, x fastest) on the
 *                 current device.
 *   u             device array of nx*ny floats, coefficient layout of pat_EsT,
 *                 on the current device; x and u must not overlap (rejected
 *                 with PAT_ERR_INVALID).  The library cannot see the arrays'
 *                 lengths: arrays shorter than nx*ny floats are the caller's
 *                 error and corrupt memory.
 *   stream        cudaStream_t (asynchronous, like pat_EsT).
 * The transform's scratch (2 MiB) is a fixed array in device memory that
 * every device loading the library holds until the process exits.  The first
 * call on a device looks up that array's address (once per device, with the
 * device current); make that first call before starting any stream capture.
 * All calls share the one array: calls that overlap on the GPU (two streams,
 * two host threads) race and corrupt each other's results, so serialise them.
 * Nothing in the array needs to start at zero: every call writes each scratch
 * element before reading it.  The cached address is not refreshed after
 * cudaDeviceReset: calls after a reset of the device are not supported.
 */
pat_status pat_EsT_noalloc(int nx, int ny, int family, int levels, int level_offset, double s, const float* x,
                           float* u, void* stream);

/* Message of the last error raised on the calling thread ("" if none). */
const char* pat_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PAT_H */
