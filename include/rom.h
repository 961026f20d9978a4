/*
 * rom.h -- C ABI of librom, a single-GPU (GB300, sm_103a) implementation of the
 * online step of the history-aware adaptive reduced-order model with an
 * incremental-SVD basis update (arXiv 2605.28684).
 *
 * The method (paper, Sec. 4 and Algorithms 1-2): a Galerkin (or DEIM-Galerkin)
 * reduced model q ~ q_ref + D^-1 Phi a is advanced by backward Euler; every z
 * steps a coarse backward-Euler full-order step of size z*dt (Eq.
 * coarse_fom_backward_euler) yields a correction snapshot y, whose
 * preprocessed form D (y - q_ref) updates the basis by Brand's rank-one
 * incremental SVD with forgetting factor lambda (Algorithm 2); the sampling
 * points and the reduced state are then refreshed (the adaptation event of Algorithm 1).
 *
 * Conventions common to every entry point
 *  - Host pointers are read or written during the call only; the library never
 *    keeps a caller pointer. Device pointers (entry points named *_dev) must
 *    point to device memory of the current CUDA device and stay valid until the
 *    call returns.
 *  - Every call is ordered on the CUDA stream given at creation (or passed to
 *    the call) and synchronises that stream before it returns.
 *  - Errors are reported by the return code only; nothing throws across the
 *    ABI. After ROM_ECUDA or ROM_ETIMEOUT a context is poisoned: every later
 *    call except rom_destroy returns ROM_ESTATE.
 *  - The library has no CPU fallback: if no usable sm_103 device is present
 *    rom_init returns ROM_ECUDA.
 *  - Vectors of the full-order state have N = n_var * n_cells entries, blocked
 *    by variable ([rho_0..rho_{N-1}, m_0.., E_0..] for the Euler system). The
 *    basis Phi is stored column-major, N x r, leading dimension N.
 */
#ifndef ROM_H
#define ROM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rom_ctx rom_ctx;   /* opaque; owns all device memory of one ROM */

typedef enum {
    ROM_OK = 0,
    ROM_EINVAL = 1,      /* invalid argument (null pointer, bad size or parameter) */
    ROM_ENOMEM = 2,      /* device allocation failed */
    ROM_ECUDA = 3,       /* CUDA runtime error (context poisoned) */
    ROM_ENOCONV = 4,     /* a Newton iteration hit its iteration limit */
    ROM_ENONFINITE = 5,  /* NaN or Inf met in the state */
    ROM_ETIMEOUT = 6,    /* a device-side wait ran out of time (context poisoned) */
    ROM_ESTATE = 7       /* context poisoned by an earlier error */
} rom_status;

typedef enum { ROM_BURGERS = 0, ROM_EULER = 1 } rom_problem;
typedef enum { ROM_FP64 = 0, ROM_MIXED_FP32 = 1 } rom_precision;
typedef enum { ROM_GALERKIN = 0, ROM_LSPG = 1 } rom_projection;
typedef enum {
    ROM_UPDATE_ISVD = 0,
    ROM_UPDATE_WINDOWED_SVD = 1,
    ROM_UPDATE_DIRECT = 2,
    ROM_UPDATE_ONESTEP = 3,
    ROM_UPDATE_OJA = 4,
    ROM_UPDATE_GROUSE = 5
} rom_update_rule;
typedef enum { ROM_BACKWARD_EULER = 0, ROM_SSPRK43 = 1 } rom_time_scheme;

/*
 * Hyper-parameters of one adaptive ROM: the inputs of Algorithm 1 (r, n_s,
 * w_init, z, lambda) plus the full-order model (paper Sec. 2, Sec. 5.1, App. B).
 *  problem     ROM_BURGERS: u_t + (u^2/2)_x = nu u_xx, periodic, Godunov flux,
 *              centred diffusion. ROM_EULER: 1D Euler, ideal gas (gamma),
 *              Rusanov flux, zero-gradient ghost cells (App. B).
 *  precision   ROM_FP64, or ROM_MIXED_FP32 (FP32 basis storage; FP32 lift,
 *              projections and rotation with FP32 accumulation; FP64 core SVD,
 *              FP64 re-orthonormalisation of the basis after every update, FP64
 *              full-order model).
 *  n_cells     cells of the uniform grid on [0, 1]; n_var = 1 (Burgers) or 3.
 *  r           maximum reduced dimension (1 <= r <= 64, r <= w_init, r < N).
 *  n_s         0: plain Galerkin. > 0: DEIM-Galerkin with n_s sampled rows
 *              (r <= n_s <= 256): QDEIM points plus feature-guided points of
 *              largest squared forward difference of the feature of the
 *              correction snapshot (Eq. fgs_selection). Burgers: the feature
 *              is the state, periodic. Euler (time_scheme ROM_SSPRK43 only,
 *              the Galerkin-FGS form of Sec. 5.3): the feature is the cell
 *              pressure, the right end faces the zero-gradient ghost cell, and
 *              the three rows of a cell share its score; the nine mesh rows
 *              per sample must fit shared memory (about 72 n_s r bytes <=
 *              220 kB), else ROM_EINVAL.
 *  w_init      fine FOM steps of the offline training window (>= 1).
 *  z           adaptation interval (>= 1); the coarse FOM step is z*dt.
 *  dt, nu, gamma, lambda   time step, viscosity, ratio of specific heats,
 *              forgetting factor in [0, 1].
 *  newton_max, newton_tol  Newton stops once max|delta| <= tol (1 + max|x|);
 *              newton_max iterations without that -> ROM_ENOCONV.
 *  rank_tol    singular directions with sigma_j <= rank_tol * sigma_1 are
 *              numerically null and kept as zero columns; a new iSVD direction
 *              enters only if ||q|| > rank_tol * max(||y||, sigma_1). <= 0 selects
 *              the precision's default: 1e-10 (FP64), 1e-5 (mixed; FP32
 *              projections cannot resolve smaller residuals).
 *  projection  ROM_GALERKIN (0): the Galerkin step of Eq. galerkin_continuous_rom
 *              (or Eq. deim_galerkin_rom with n_s > 0). ROM_LSPG (1): the
 *              least-squares Petrov-Galerkin step of Eq. lspg_minimization with
 *              the backward-Euler test basis of Eq. lspg_test_basis_be, solved by
 *              Gauss-Newton in FP64 (Burgers, ROM_FP64 only). With n_s > 0 the
 *              hyper-reduced LSPG step (Eq. hyperreduced_lspg_stationarity, DEIM
 *              basis = Phi) has the DEIM-Galerkin root as its minimiser, because
 *              (P^T Phi)^+ P^T Phi = I makes its objective the norm of the
 *              DEIM-Galerkin residual; that step is used.
 *  update_rule ROM_UPDATE_ISVD (0): Algorithm 2. The comparison rules of App.
 *              A act on a window of the `window` latest preprocessed correction
 *              snapshots (initially the last `window` training snapshots; each
 *              event drops the oldest and appends the new one):
 *              ROM_UPDATE_WINDOWED_SVD (1): the leading r left singular vectors
 *              of the window (Eqs. wsvd_window_matrix, wsvd_update);
 *              ROM_UPDATE_DIRECT (2): an orthonormal basis of
 *              span(Y (Phi^+ Y)^+) (Eqs. direct_optimization, direct_update),
 *              its "singular values" those of Phi^+ Y. Both transfer the state
 *              as a = Phi_new^T D (q~ - q_ref), and both are FP64 only.
 *              The instantaneous rules of App. A act on the live basis columns
 *              and the correction snapshot already held, yhat = D (y - q_ref)
 *              (an adaptation event updates the basis first and advances the
 *              coarse FOM at its end, so the snapshot approximates the current
 *              time level); the rank and sigma are kept:
 *              ROM_UPDATE_ONESTEP (3): Phi <- orth(Phi + (yhat - Phi a) a^T / |a|^2)
 *              with a the reduced state (Eq. onestep_update);
 *              ROM_UPDATE_OJA (4): Phi <- orth(Phi + eta yhat (yhat^T Phi))
 *              (Eq. oja_update); orth is CholQR applied twice, FP64;
 *              ROM_UPDATE_GROUSE (5): the rank-one geodesic step of Eqs.
 *              grouse_projection, grouse_update with alpha = eta |p| |r| (the
 *              residual by Gram-Schmidt twice; orthonormal by construction).
 *              Rules 3-5: FP64, n_s = 0, backward Euler; they transfer the state
 *              as rules 1 and 2.
 *  window      1 <= window <= min(w_init, 64) for rules 1 and 2 (unused otherwise).
 *  time_scheme ROM_BACKWARD_EULER (0): fine FOM steps and reduced steps by
 *              backward Euler (Newton). ROM_SSPRK43 (1): the explicit form of
 *              the paper's RDE solver (App. D): the fine FOM steps of the
 *              training window and the Galerkin (or DEIM-Galerkin) reduced
 *              steps da/dt = Phi^T D f (or (P^T Phi)^+ P^T D f) advance by the
 *              four-stage, third-order SSP Runge-Kutta scheme (SSP coefficient
 *              2: three half steps of forward Euler, an average with the start
 *              value after the third, a last half step); the coarse correction
 *              step stays backward Euler over z*dt (Eq.
 *              coarse_fom_backward_euler). Galerkin, ROM_FP64 and
 *              ROM_UPDATE_ISVD only.
 *  learning_rate  eta >= 0 of rules 4 and 5 (unused otherwise).
 */
typedef struct {
    int32_t problem;
    int32_t precision;
    int64_t n_cells;
    int32_t n_var;
    int32_t r;
    int32_t n_s;
    int32_t w_init;
    int32_t z;
    int32_t newton_max;
    double dt;
    double nu;
    double gamma;
    double lambda;
    double newton_tol;
    double rank_tol;
    int32_t projection;
    int32_t update_rule;
    int32_t window;
    int32_t time_scheme;
    double learning_rate;
} rom_config;

/*
 * Offline stage of Algorithm 1: w_init fine backward-Euler FOM
 * steps from q0, preprocessing (q_ref = q0, D_v = 1/phi_v with phi_v the mean
 * square of the centred training field of variable v; Eqs.
 * scaling_matrix_local_block, variable_normalization), POD of
 * D (Q_train - q_ref 1^T) truncated to r, the initial reduced state, the first
 * coarse correction state and, if n_s > 0, the sampling points.
 *  cfg       configuration (copied).
 *  q0_host   host array of N doubles, the initial state.
 *  stream    cudaStream_t to order all work on (NULL: the legacy default stream).
 *  out       receives the new context on ROM_OK, NULL otherwise.
 * Errors: ROM_EINVAL, ROM_ENOMEM, ROM_ECUDA, ROM_ENOCONV, ROM_ENONFINITE (a
 * NaN or Inf in q0_host is refused on the host before any device work; later
 * the FOM Newton solves report a non-finite state).
 */
rom_status rom_init(const rom_config* cfg, const double* q0_host, void* stream,
                    rom_ctx** out);

/*
 * n_steps iterations of the online loop of Algorithm 1: one
 * backward-Euler reduced step each, and an adaptation event (coarse FOM step,
 * iSVD update, sampling refresh, state transfer) after every step with
 * mod(n + 1 - w_init, z) = 0. The state stays on the device.
 * Errors: ROM_EINVAL (n_steps < 0), ROM_ENOCONV, ROM_ENONFINITE, ROM_ECUDA,
 * ROM_ETIMEOUT, ROM_ESTATE.
 */
rom_status rom_step(rom_ctx* ctx, int64_t n_steps);

/*
 * One adaptation event now (the adaptation event of Algorithm 1 with Algorithm 2): the
 * correction snapshot is y_host (N doubles, a raw full-order state, which also
 * replaces the stored coarse state) or, if y_host is NULL, one coarse FOM step
 * of the stored coarse state. It is preprocessed as D (y - q_ref), the basis is
 * updated by the rank-one iSVD with forgetting, the sampling points are
 * refreshed and the reduced state is transferred to the new basis. With the
 * comparison rules (rom_config.update_rule != ROM_UPDATE_ISVD) the basis is
 * updated by that rule instead; the instantaneous rules (3-5) take the
 * snapshot held (y_host, or, if y_host is NULL, the stored coarse state) and,
 * with y_host NULL, advance the coarse FOM after the update.
 * Errors: as rom_step; a NaN or Inf in y_host returns ROM_ENONFINITE before
 * any device work and leaves the context unchanged (not poisoned).
 */
rom_status rom_update_basis(rom_ctx* ctx, const double* y_host);

/*
 * Copies the current state to host buffers; any pointer may be NULL.
 *  q_tilde  N doubles: q_ref + D^-1 Phi a (Eq. trial_approximation).
 *  a        r doubles;  sigma  r doubles (descending, zeros for null directions).
 *  phi      N*r doubles, column-major; each non-zero column is sign-normalised
 *           so that its largest-magnitude entry is positive (a is flipped with
 *           it, which leaves q_tilde unchanged).
 *  y_corr   N doubles: the stored coarse correction state.
 *  step     the time level n of the reduced state.
 * Errors: ROM_EINVAL (ctx NULL), ROM_ECUDA, ROM_ESTATE.
 */
rom_status rom_state(rom_ctx* ctx, double* q_tilde, double* a, double* sigma,
                     double* phi, double* y_corr, int64_t* step);

/*
 * Replaces the online state (checkpoint import; resume is bit-exact with the
 * state exported by rom_state). phi: N*r column-major with orthonormal
 * non-zero columns; sigma: r; a: r; y_corr: N; step: time level. If n_s > 0
 * the sampling points are rebuilt from phi and y_corr.
 * Errors: ROM_EINVAL, ROM_ECUDA, ROM_ESTATE, ROM_ENONFINITE (a NaN or Inf in
 * any input array; checked on the host, the context is unchanged).
 */
rom_status rom_load_state(rom_ctx* ctx, const double* phi, const double* sigma,
                          const double* a, const double* y_corr, int64_t step);

/* Sampling points (n_s int32 row indices of the state, QDEIM points first;
 * for Burgers a row is a cell) of a hyper-reduced context. Errors: ROM_EINVAL (NULL or n_s = 0), ROM_ECUDA. */
rom_status rom_samples(rom_ctx* ctx, int32_t* idx_host);

/* Numerical rank of the current basis (number of non-null columns) and the
 * Newton iteration counts of the last reduced step and last FOM step. */
rom_status rom_info(rom_ctx* ctx, int32_t* rank, int32_t* rom_newton_iters,
                    int32_t* fom_newton_iters);

/*
 * Per-phase device timing (CUDA events recorded around every launch of a
 * phase, on the stream it runs on, while enabled). Phases: 0 reduced steps,
 * 1 coarse FOM step, 2 iSVD update, 3 sampling refresh (QDEIM points, the
 * sampled operator and stencil mesh), 4 feature-guided candidate selection on
 * a new correction snapshot (hyper-reduced models; in an adaptation cycle it
 * runs after the coarse FOM step, beside the reduced steps).
 * rom_profile(ctx, 1) clears the totals and starts recording;
 * rom_profile(ctx, 0) stops. rom_profile_read synchronises and returns, per
 * phase, the summed milliseconds and the number of launches (arrays of 5).
 * Errors: ROM_EINVAL, ROM_ECUDA, ROM_ESTATE.
 */
rom_status rom_profile(rom_ctx* ctx, int32_t enable);
rom_status rom_profile_read(rom_ctx* ctx, double* ms_total, int64_t* launches);

/* Releases the context and all its device memory. NULL is ignored. */
void rom_destroy(rom_ctx* ctx);

/* Static, human-readable name of a status code. */
const char* rom_status_string(rom_status s);

/*
 * Low-level full-order entry points on caller-owned device buffers (no
 * context). problem/n_cells/nu/gamma as in rom_config.
 *
 * rom_fom_rhs_dev: f(q) of the semi-discrete operator (Sec. 5.1 problem
 *   setup; App. B, Eq. sod_fv_semidiscrete_appendix).  q_dev, f_dev: N doubles.
 * rom_fom_step_dev: one backward-Euler step q - q_prev - h f(q) = 0 solved by
 *   Newton from q_prev (Eq. be_residual_rom_section); writes q_dev (N doubles,
 *   may not alias q_prev_dev) and, if iters_host is not NULL, the Newton count.
 *   Limits: Burgers n_cells <= 131072; Euler 8 <= n_cells <= 32768.
 * Errors: ROM_EINVAL, ROM_ENOMEM, ROM_ECUDA, ROM_ENOCONV, ROM_ENONFINITE,
 * ROM_ETIMEOUT.
 */
rom_status rom_fom_rhs_dev(int32_t problem, int64_t n_cells, double nu, double gamma,
                           const double* q_dev, double* f_dev, void* stream);
rom_status rom_fom_step_dev(int32_t problem, int64_t n_cells, double nu, double gamma,
                            double h, double newton_tol, int32_t newton_max,
                            const double* q_prev_dev, double* q_dev,
                            int32_t* iters_host, void* stream);

/*
 * Allocation-free variant of rom_fom_step_dev (this entry point has no
 * counterpart in the paper; it is a service for callers that must not
 * allocate). Some callers cannot call cudaMalloc: a host application that owns
 * all device memory through its own pool allocator and forbids raw
 * allocations, or a time-critical loop that cannot afford cudaMalloc/cudaFree
 * (cudaFree waits for the whole device). For the Burgers problem this call
 * runs the same Newton solve with the same arguments, results and errors as
 * rom_fom_step_dev, but allocates nothing: its scratch is one fixed 8448-byte
 * device array inside the library, held by every GPU that loads it until the
 * process exits.
 *  Problems: ROM_BURGERS only; ROM_EULER (whose separator system needs more
 *  scratch than the array holds) returns ROM_EINVAL.
 *  Limit: n_cells <= 131072 (larger values return ROM_EINVAL).
 *  The first call on a device looks up that array's device address
 *  (cudaGetSymbolAddress) and caches it.
 *  Every call synchronises `stream` and reads the status word back to the
 *  host before it returns.
 *  All calls share the array, and each call clears what must start at zero;
 *  calls that overlap on the GPU (from several host threads or streams at once)
 *  race on it and must be serialised by the caller.
 */
rom_status rom_fom_step_noalloc_dev(int32_t problem, int64_t n_cells, double nu,
                                    double gamma, double h, double newton_tol,
                                    int32_t newton_max, const double* q_prev_dev,
                                    double* q_dev, int32_t* iters_host, void* stream);

/*
 * Test hook (no counterpart in the paper): sets the bound, in SM clock
 * cycles, of every device-side wait of the library's kernels (the software
 * grid barrier between the phases of a cooperative launch). A kernel whose
 * wait runs out records ROM_ETIMEOUT and returns; the call then reports
 * ROM_ETIMEOUT and poisons its context. cycles <= 0 restores the default
 * (4e9 cycles, about 2 s). The setting is process-wide and applies to the
 * current device; change it only while none of the library's kernels runs.
 * Errors: ROM_ECUDA.
 */
rom_status rom_debug_set_wait_limit(int64_t cycles);

/*
 * Low-level iSVD update (Algorithm 2) on caller-owned device buffers.
 *  phi_dev    N x r column-major, updated in place (orthonormal non-zero
 *             columns; null columns are zero).
 *  sigma_dev  r doubles, updated in place.
 *  y_dev      N doubles: the preprocessed snapshot (not modified).
 *  ubar_host  if not NULL, receives the (r+1) x (r+1) left singular vectors of
 *             the core matrix, column-major, columns in descending order of
 *             the singular values.
 * Errors: ROM_EINVAL, ROM_ENOMEM, ROM_ECUDA, ROM_ETIMEOUT.
 */
rom_status rom_isvd_update_dev(int64_t n, int32_t r, double lambda, double rank_tol,
                               double* phi_dev, double* sigma_dev, const double* y_dev,
                               double* ubar_host, void* stream);

/*
 * Gradient of a terminal misfit of the adaptive ROM (the paper states no
 * adjoint; this differentiates Algorithm 1 with the iSVD update of Algorithm
 * 2 as this library computes it). For the plain-Galerkin Burgers ROM
 * (problem ROM_BURGERS, precision ROM_FP64, projection ROM_GALERKIN, n_s = 0,
 * w_init <= 128):
 *   J(nu, q0) = 1/2 || q~^{n_T} - target ||^2,
 * q~^{n_T} the lifted state returned by the last of n_steps online steps
 * (before that step's adaptation event, if it has one), and its gradient with
 * respect to the viscosity nu and the initial state q0 (which also fixes
 * q_ref = q0 and, through the training window, D and the POD basis). The call
 * runs the offline stage and the forward pass itself, then the reverse sweep:
 * transposed reduced Jacobian solves of every Galerkin step, the adjoint of
 * every iSVD update (core SVD, rotation, projection, state transfer), the
 * transposed periodic tridiagonal solve of every coarse and training FOM
 * step, and the adjoint of the POD of the training matrix. Discrete
 * decisions (Godunov branch, numerical rank, empty residual) are held fixed;
 * Newton roots are differentiated at the computed root. All arithmetic is FP64.
 *  cfg          configuration (as rom_init, restricted as above).
 *  q0_host      N doubles, the initial state.
 *  target_host  N doubles, the target of the misfit.
 *  n_steps      online steps (>= 1).
 *  ckpt_every   >= 1. The forward pass records every step of a segment of
 *               ckpt_every steps (per event about 8 N (r + 4) bytes); with
 *               ckpt_every < n_steps it keeps only the online state at the
 *               start of each segment and the reverse sweep re-runs each
 *               segment from it, so the memory is that of one segment plus
 *               one state per segment. The gradient does not depend on it.
 *  stream       cudaStream_t (NULL: the legacy default stream); the call
 *               synchronises it before returning.
 *  J, dJ_dnu    host scalars (out).
 *  dJ_dq0       N doubles (out) or NULL.
 *  q_final      N doubles (out): q~^{n_T}, or NULL.
 * Errors: ROM_EINVAL (configuration or arguments outside the above),
 * ROM_ENONFINITE (NaN/Inf in q0 or target, checked on the host), ROM_ENOMEM,
 * and the errors of rom_init and rom_step.
 */
rom_status rom_adjoint(const rom_config* cfg, const double* q0_host, const double* target_host,
                       int64_t n_steps, int32_t ckpt_every, void* stream, double* J,
                       double* dJ_dnu, double* dJ_dq0, double* q_final);

/* ------------------------------------------------------------------------
 * Batched execution of many independent ROMs.
 *
 * A batch holds `count` independent Burgers ROMs (Algorithm 1 with the plain
 * Galerkin step and the iSVD of Algorithm 2), each with its own n_cells, r,
 * nu, dt, z, lambda and initial state. It runs the mixed form only: FP32
 * basis, FP32 lift, projections and rotation with FP32 accumulation; FP64
 * residual, coarse FOM step, core SVD, Cholesky re-orthonormalisation and
 * reduced state. The instances advance in lockstep: every call to
 * rom_batch_step advances each of them by n_steps steps (with its own
 * adaptation events), and all data of the batch stays in device memory.
 * ------------------------------------------------------------------------ */
typedef struct rom_batch rom_batch;

/*
 * Offline stage of every instance (as rom_init), then packs the instances
 * into one device layout: bases back to back (FP32, column-major per
 * instance), N-vectors back to back, row tiles and FOM chunks.
 *  cfgs     count configurations: problem ROM_BURGERS, precision
 *           ROM_MIXED_FP32, projection ROM_GALERKIN, n_var 1, n_s 0, 1 <= r <= 64,
 *           256 <= n_cells <= 131072, z >= 1 (others as rom_init).
 *  q0s      count host pointers, q0s[i] holding n_cells doubles (copied).
 *  count    1 .. 4096, with at most 256 coarse-FOM chunks per CTA of the FOM
 *           grid in all (an instance has max(4, 2^ceil(log2(n_cells/512)))
 *           chunks; the grid is two CTAs per SM): 77,824 on a 152-SM GPU.
 *  stream   cudaStream_t or NULL; every batch call is ordered on it.
 *  out      receives the batch, which owns all its device memory.
 * Errors: ROM_EINVAL (a configuration outside the above), ROM_ENOMEM,
 * ROM_ECUDA, and the errors of rom_init for an instance.
 */
rom_status rom_batch_init(const rom_config* cfgs, const double* const* q0s, int32_t count,
                          void* stream, rom_batch** out);

/*
 * n_steps online steps of every instance. An instance i adapts (coarse FOM
 * step, iSVD update, state transfer) after each of its steps n with
 * (n + 1 - w_init_i) mod z_i == 0. Errors: ROM_EINVAL (n_steps < 0),
 * ROM_ENOCONV / ROM_ENONFINITE (some instance's Newton solve), ROM_ETIMEOUT,
 * ROM_ECUDA; after any of these the batch is poisoned (ROM_ESTATE on further
 * calls except rom_batch_destroy).
 */
rom_status rom_batch_step(rom_batch* b, int64_t n_steps);
/*   On a stream other than the legacy default stream, and while the per-phase
 *   timer (rom_batch_profile) is off, the launches of one whole adaptation
 *   interval are captured once into a CUDA graph and replayed for every
 *   interval of the same length; otherwise they are launched one by one. */

/*
 * State of instance i, as rom_state: q_tilde (n_cells), a (r), sigma (r),
 * phi (n_cells x r column-major, sign convention applied, a adjusted to
 * match), y_corr (n_cells), step; each output may be NULL.
 * Errors: ROM_EINVAL (i out of range), ROM_ESTATE, ROM_ECUDA.
 */
rom_status rom_batch_state(rom_batch* b, int32_t i, double* q_tilde, double* a, double* sigma,
                           double* phi, double* y_corr, int64_t* step);

/* Rank of instance i and the Newton iterations of its last reduced step and
 * of its last coarse FOM step. */
rom_status rom_batch_info(rom_batch* b, int32_t i, int32_t* rank, int32_t* rom_iters,
                          int32_t* fom_iters);

/* Layout of the batch: total FP32 basis bytes (sum of n_cells * r * 4), total
 * rows (sum of n_cells), number of row tiles and their size in rows (chosen by
 * rom_batch_init: the fastest of 2048, 4096, 8192 and 16384 rows in a timed
 * residual sweep over the instances' bases), CTAs of the sweep kernels, and
 * whether whole adaptation intervals replay a captured graph (1), have not
 * been tried yet (0) or launch one by one (-1). Any output may be NULL. */
rom_status rom_batch_layout(rom_batch* b, int64_t* basis_bytes, int64_t* rows, int32_t* tiles,
                            int32_t* tile_rows, int32_t* grid, int32_t* graph);

/* Per-phase device timing (as rom_profile): phases 0 reduced steps, 1 coarse
 * FOM, 2 iSVD update; ms_total and launches hold 3 entries each. */
rom_status rom_batch_profile(rom_batch* b, int32_t enable);
rom_status rom_batch_profile_read(rom_batch* b, double* ms_total, int64_t* launches);

/* Work of the reduced steps since the last rom_batch_profile call (or init):
 * Newton iterations summed over the instances, and the algorithmic bytes
 * they stream (each iteration reads the k live columns of the instance's FP32
 * basis and three FP32 words of reference-state data per row: 4 n_cells k +
 * 12 n_cells bytes, k the rank at that step). Either output may be NULL. */
rom_status rom_batch_work(rom_batch* b, int64_t* newton_iters, double* sweep_bytes);

/* Work of the coarse FOM steps (Eq. coarse_fom_backward_euler) since the last
 * rom_batch_profile call (or init): Newton iterations times n_cells, summed
 * over the instances and their events, and the algorithmic bytes of those
 * iterations (each reads the iterate and the previous state and writes the
 * update: 24 bytes a row). Either output may be NULL. */
rom_status rom_batch_fom_work(rom_batch* b, int64_t* row_iterations, double* fom_bytes);

/* Releases the batch and all its device memory (NULL is ignored). */
void rom_batch_destroy(rom_batch* b);

#ifdef __cplusplus
}
#endif

#endif /* ROM_H */
