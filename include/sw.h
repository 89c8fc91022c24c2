/*
 * libsw -- Schwarzschild orbit-superposition hot path on one GB300 (sm_103a).
 *
 * For one trial potential: integrate an orbit library in a rotating
 * disc + bar + halo potential, project every sample to the sky with four-fold
 * mirror symmetrisation, bin it into 3-D density cells and IFU pixels x
 * line-of-sight-velocity bins (or Gauss-Hermite rows) to form the orbit
 * matrix U, then solve the regularised non-negative weight problem
 * (arxiv 2607.00117, Sec. 2: density/potential, orbit library, projection,
 * mapping to observables, weight optimisation, likelihood).
 *
 * Conventions for every entry point:
 *  - Units: kpc, km/s, Msun, G = 4.300917e-6 kpc (km/s)^2 / Msun; time in
 *    kpc/(km/s) (977.79 Myr); angles in radians; Omega_p in km/s/kpc.
 *  - Every call returns sw_status and never aborts or prints; the message of
 *    the last failure is returned by sw_last_error().
 *  - Host arrays are owned by the caller and only read (inputs) or written
 *    (outputs) during the call.  "_device" variants take device pointers
 *    (CUDA global memory on the context's device) instead of host pointers.
 *  - The context owns all library-allocated device memory except sw_matrix
 *    objects, which the caller owns once returned and frees with
 *    sw_matrix_free() before destroying their context.
 *  - All work is ordered on the context's CUDA stream.  Calls with host
 *    outputs return after the results are copied out; "_device" calls are
 *    asynchronous with respect to the host unless stated.
 *  - A context is not thread-safe; use one context per host thread.
 */
#ifndef SW_H
#define SW_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif
#if defined(__GNUC__)
#pragma GCC visibility push(default)
#endif

typedef struct sw_ctx sw_ctx;       /* opaque */
typedef struct sw_matrix sw_matrix; /* opaque, device-resident orbit matrix */

typedef enum {
    SW_OK = 0,
    SW_EINVAL = 1,    /* invalid argument (NULL, size, grid) */
    SW_ENOMEM = 2,    /* device allocation failed */
    SW_ECUDA = 3,     /* CUDA runtime error */
    SW_ETIMEOUT = 4,  /* a bounded device wait ran out */
    SW_ENONCONV = 5,  /* iteration cap reached; best iterate returned */
    SW_ESTATE = 6     /* call out of order (e.g. project before integrate) */
} sw_status;

typedef enum {
    SW_FP64_PLAIN = 0,  /* FP64 integration, binning and solve (plain baseline form) */
    SW_FP32_KAHAN = 1   /* FP32 integration with Kahan-compensated positions; BF16 tensor-core
                           Gram with FP32 accumulation; FP64 refinement and chi^2 */
} sw_precision;

/* Per-orbit status written by the integration passes. */
enum { SW_ORBIT_OK = 0, SW_ORBIT_DRIFT = 1, SW_ORBIT_NONFINITE = 2 };

/* Potential (Sec. 3.2).  Disc: Miyamoto-Nagai Phi = -G M_d / sqrt(R^2 + (R_d + sqrt(z^2 + H_d^2))^2)
 * with (disc_M, disc_a, disc_b) = (M_d, R_d, H_d).  Halo: NFW from (halo_M200, halo_c) with
 * Delta = 200 and rho_crit = 3 H0^2 / (8 pi G), H0 in km/s/Mpc (Sec. 3.2.1).  Bar (bar_M = 0
 * disables it; its major axis is the rotating x axis), by bar_kind:
 *   0: the n = 1, eta = 0 needle convolution of Eq. (Rn_to_In) (the Long-Murali bar) with
 *      half-length bar_L, parent MN radial scale bar_b and height bar_c;
 *   1: the paper's bar (Sec. 2.1.2, App. A): a Dehnen-Aly T3 long bar (eta = 1, a = bar_L / 5,
 *      b = disc_b, needle half-length bar_L) plus a V4 boxy/peanut bulge (eta = 0, a = b = 0.5 kpc,
 *      half-length 0.1 kpc), each of mass bar_M / 2, every R^-n of the parent potentials replaced
 *      by the needle integral I_n of Eq. (Rn_to_In); bar_b and bar_c are not used.
 * test_kind 1 adds a point mass test_M, 2 a Plummer sphere (test_M, test_a); 0 none.  Components
 * with zero mass are skipped.  Other bar_kind values return SW_EINVAL. */
typedef struct {
    double disc_M, disc_a, disc_b;
    double halo_M200, halo_c, H0;
    double bar_M, bar_L, bar_b, bar_c;
    int32_t test_kind;
    int32_t bar_kind;
    double test_M, test_a;
} sw_potential_params;

/* Sky pixels: half-open bins [x0 + i dx, x0 + (i+1) dx), i < nx (same for y). */
typedef struct { int32_t nx, ny; double x0, y0, dx, dy; } sw_pixel_grid;
/* Line-of-sight velocity bins [v0 + k dv, v0 + (k+1) dv), k < nv. */
typedef struct { int32_t nv, reserved; double v0, dv; } sw_vbins;
/* Cylindrical cells in the bar frame, uniform in R in [0, Rmax), phi in [0, 2 pi) measured
 * from the bar's major axis, z in [zmin, zmax) (Sec. 2.2.4). */
typedef struct { int32_t nR, nphi, nz, reserved; double Rmax, zmin, zmax; } sw_density_grid;

/* ---- context ------------------------------------------------------------ */

/* Create a context on CUDA device `device` computing in `prec`.  `cuda_stream` is a
 * cudaStream_t to order all work on (e.g. PyTorch's current stream), or NULL for a
 * stream the context creates and owns.  *out receives the context. */
sw_status sw_create(sw_ctx** out, int device, sw_precision prec, void* cuda_stream);
/* Free every device buffer the context owns and the context itself (NULL is a no-op). */
sw_status sw_destroy(sw_ctx* ctx);
/* Message of the most recent failure on this context ("" if none).  Valid until the next call. */
const char* sw_last_error(const sw_ctx* ctx);

/* ---- the four calls of the method (Sec. 2) --------------------------------- */

/* Set the trial potential (Sec. 3.2; the NFW re-parameterisation of Sec. 3.2.1 is done here).
 * Returns SW_EINVAL for non-finite or non-positive scales. */
sw_status sw_set_potential(sw_ctx* ctx, const sw_potential_params* p);

/* Load the orbit library's initial conditions (Sec. 2.2.1-2.2.2): ics is n_orb x 6 row-major
 * (x, y, z, vx, vy, vz) in the inertial frame at t = 0 (host memory), with pattern speed
 * omega_p, fixed step dt > 0 and nsteps >= 1 kick-drift-kick steps.  When drift_out or
 * status_out is non-NULL, the orbits are also integrated once to return each orbit's Jacobi
 * drift max_n |E_J(t_n) - E_J(0)| / |E_J(0)| (Sec. 2.2.2) and status (SW_ORBIT_*; drift > 0.1
 * is SW_ORBIT_DRIFT); otherwise integration is deferred to sw_project, which fuses it with
 * binning.  Arrays are host memory of n_orb elements. */
sw_status sw_integrate_library(sw_ctx* ctx, const double* ics, int64_t n_orb, double omega_p, double dt,
                               int64_t nsteps, double* drift_out, uint8_t* status_out);
/* As sw_integrate_library with ics, drift_out and status_out in device memory. */
sw_status sw_integrate_library_device(sw_ctx* ctx, const double* ics_dev, int64_t n_orb, double omega_p,
                                      double dt, int64_t nsteps, double* drift_dev, uint8_t* status_dev);

/* Build the orbit matrix U (Sec. 2.2.3-2.2.4, Eq. Euler, Table 1) for the loaded library:
 * Euler angles alpha = bar_angle, beta = incl, gamma = pa (z-x-z, image = (x', y'),
 * v_los = v'_z); samples at t_1..t_nsteps, each with its four mirror copies when mirror4 != 0,
 * weight 1/(copies * nsteps).  Rows (M total): density cells (iR*nphi + iphi)*nz + iz; then
 * pixel mass iy*nx + ix; then either the velocity histogram (pixel*nv + iv) or, when gh_v0_s
 * (host, npix x 2 reference (v0, s) per pixel) is non-NULL, four Gauss-Hermite rows per pixel
 * (pixel*4 + m-1, m = 1..4) holding sum 2 sqrt(pi) alpha(w) H_m(w), w = (v_los - v0)/s.
 * Orbits whose Jacobi drift exceeds 0.1 or turn non-finite get zero columns.  *U_out receives a
 * device-resident matrix stored orbit-major (column i contiguous).  vb may be NULL in GH mode.
 * With the option project_bundle = n > 1 the matrix has n_orb / n columns, column j the mean of
 * orbits j n .. j n + n - 1 (Sec. 2.2.1 orbit bundles), accumulated at bin time. */
sw_status sw_project(sw_ctx* ctx, double incl, double pa, double bar_angle, const sw_pixel_grid* pix,
                     const sw_vbins* vb, const sw_density_grid* dens, const double* gh_v0_s, int mirror4,
                     sw_matrix** U_out);
/* Reduce a velocity-histogram orbit matrix to Gauss-Hermite rows (the form of the paper's
 * objective, Sec. 2.3 Eq. objective_function, and of its App. B conversion of a gridded LOSVD to
 * GH coefficients): density and pixel-mass rows are copied; for each pixel p and m = 1..4 the row
 * (p, m) is sum_k U[(p, k)] 2 sqrt(pi) alpha(w_k) H_m(w_k) with w_k = (v_k - v0_p)/s_p and v_k the
 * centre of velocity bin k (midpoint quadrature of the orbit's LOSVD).  gh_v0_s: host npix x 2
 * (v0, s > 0).  *U_gh_out receives a new matrix (rows nd + 5 npix, GH layout as in sw_project);
 * U_hist is unchanged. */
sw_status sw_reduce_gh(sw_ctx* ctx, const sw_matrix* U_hist, const double* gh_v0_s, sw_matrix** U_gh_out);
/* Orbit bundles (Sec. 2.2.1: each initial condition is dithered into n nearby realisations that
 * enter the fit as one orbit).  For a matrix whose N columns hold N/n bundles of n consecutive
 * realisations, *U_out receives a new matrix of N/n columns, column j the mean of columns
 * j n .. j n + n - 1 (summed in the matrix precision in realisation order); rows and layout are
 * unchanged.  n must divide N (SW_EINVAL otherwise).  U is unchanged; free both with
 * sw_matrix_free. */
sw_status sw_bundle(sw_ctx* ctx, const sw_matrix* U, int64_t n, sw_matrix** U_out);
/* Drift and status per orbit from the last sw_project (host arrays of n_orb, nullable). */
sw_status sw_project_stats(sw_ctx* ctx, double* drift_out, uint8_t* status_out);

/* Solve min_w 1/2 ||(U w - data) / errors||^2 + (lambda / N) ||w||^2 subject to w >= 0
 * (Sec. 2.3, Eq. objective_function in its compact NNLS form) to its exact minimiser (KKT
 * conditions to the option kkt_tol).  Two solvers reach it (option "solver"):
 *  - the default (solver = 0) is an active-set method (block principal pivoting) whenever its
 *    reduced systems stay definite -- lambda > 0, no more orbits than rows, or libraries above
 *    orbit_direct_max orbits -- which covers every solve with the default lambda = 1: each
 *    reduced problem on the passive set is solved by conjugate gradients with FP64 products of
 *    the stored U, preconditioned by the Cholesky factor of the passive set's tensor-core Gram;
 *  - the paper's ADMM (Sec. 2.3) runs when lambda = 0 with more orbits than rows (up to
 *    orbit_direct_max) and on request (solver = 2): ADMM on the Gram of the whitened matrix,
 *    then refinement with FP64 residuals against the stored U and an exact active-set polish.
 * data, errors: M host values (errors > 0); weights_out: N host values;
 * chi2_out: host [chi2_total, chi2_obs, reg] with chi2_total = ||(U w - data)/errors||^2,
 * chi2_obs the same without the density rows (Sec. 2.4) and reg = (lambda/N)||w||^2.
 * Returns SW_ENONCONV (with the best iterate) when the iteration caps are reached. */
sw_status sw_solve_weights(sw_ctx* ctx, const sw_matrix* U, const double* data, const double* errors,
                           double lambda, double* weights_out, double* chi2_out);
/* As sw_solve_weights with data, errors, weights_out and chi2_out in device memory. */
sw_status sw_solve_weights_device(sw_ctx* ctx, const sw_matrix* U, const double* data_dev,
                                  const double* errors_dev, double lambda, double* weights_dev,
                                  double* chi2_dev);

/* Bootstrap solves and the marginalised chi^2 (Sec. 2.4 and the model-likelihood passage after it).
 * For b = 0 .. n_boot-1 the observed rows of the data (every row after the 3-D density cells) are
 * perturbed by their errors, y_b = data + errors * xi[b] (the density rows unchanged); the weight
 * problem of sw_solve_weights is solved for y_b with the same matrix and lambda; chi2_b_out[b] is the
 * observational chi^2 of those weights against the unperturbed data (density rows excluded), and
 * *chi2_model_out = min_b chi2_b - 2 ln[(1/n_boot) sum_b exp(-(chi2_b - min_b chi2_b) / 2)], -2 ln of
 * the bootstrap-averaged likelihood.  The solves run the active-set method warm-started from the
 * solve on the unperturbed data, sharing the factor of its passive set (plus the orbits nearest to
 * entering) for every realisation whose passive set stays inside it.  xi: host n_boot x M standard
 * normal draws (the caller's random numbers); weights_out: host n_boot x N or NULL; chi2_b_out: host
 * n_boot; chi2_model_out: host, one value.  Needs lambda > 0 or N <= M (SW_EINVAL otherwise);
 * SW_ENONCONV if a realisation stopped at an iteration cap (its best iterate is used). */
sw_status sw_solve_bootstrap(sw_ctx* ctx, const sw_matrix* U, const double* data, const double* errors, double lambda,
                             int64_t n_boot, const double* xi, double* weights_out, double* chi2_b_out,
                             double* chi2_model_out);

/* The preconditioner of the active-set solve's reduced systems (Sec. 2.3 solves them by
 * conjugate gradients here): the Cholesky factor L of a symmetric positive definite K x K matrix
 * and the explicit inverse X = L^{-1}, exactly as the solve forms them, exposed so that they can be
 * checked on their own.  gram: host, K x K row-major FP32, only the lower triangle read; L_out,
 * X_out: host K x K row-major (L in the lower triangle, the upper triangle as given; X lower
 * triangular).  mode 0: 128-wide blocked steps with tensor-core trailing and inverse updates
 * (BF16 hi + lo operands, ~1e-4 relative); mode 1: 64-wide blocked FP32 SIMT.  *info_out: 0, or
 * j + 1 if the j-th pivot was not positive (the factorisation then continues with a tiny pivot).
 * Allocates and frees its own device buffers.  Errors: SW_EINVAL (NULL, K outside 1 .. 65 536,
 * mode), SW_ECUDA (no tensor-map encoder for mode 0), SW_ETIMEOUT (a bounded device wait ran out). */
sw_status sw_factor_preconditioner(sw_ctx* ctx, const float* gram, int64_t K, int mode, float* L_out, float* X_out,
                                   int* info_out);

/* Solver diagnostics of the last solve: out[0] ADMM iterations, out[1] refinement rounds,
 * out[2] final KKT projected-gradient infinity norm (scaled by max |U~^T y~|), out[3] 1 if the
 * orbits outnumbered the constraints (working-set or constraint-space form), out[4] number of
 * exact active-set (polish) solves, out[5] 1 if the KKT tolerance was met (0: chi^2 stable),
 * out[6] working-set rounds, out[7] final working-set size (0 without a working set). */
sw_status sw_solve_info(sw_ctx* ctx, double* out8);

/* ---- orbit matrix --------------------------------------------------------- */

/* Shape (rows M, orbits N) and row blocks: blocks3 = {density rows, pixel rows, kinematic rows}. */
sw_status sw_matrix_shape(const sw_matrix* U, int64_t* M, int64_t* N, int64_t* blocks3);
/* Copy U to host as double, orbit-major: host_out[i * M + row] (N * M values). */
sw_status sw_matrix_copy(const sw_matrix* U, double* host_out);
/* Model observables for weights w: y_out = U w (host w of N values, host y_out of M values;
 * FP64 accumulation over the stored matrix), e.g. the best-fit maps of a solve. */
sw_status sw_matrix_apply(const sw_matrix* U, const double* w, double* y_out);
/* No counterpart in the paper: a variant of sw_matrix_apply for callers that cannot allocate
 * device memory when they call (e.g. a process whose device memory belongs to another allocator's
 * pool, or a pipeline that must not allocate once running).  Same arguments and result as
 * sw_matrix_apply, but its scratch (the staged w, the FP64 accumulator of U w and, for an FP32
 * matrix, the float hi + lo halves of w) lives in a fixed static device array of 2^21 doubles
 * (16 MiB), held by every device that loads the library until the process exits; a call needing
 * more than 2^21 doubles (N + M for an FP64 matrix, 2 N + M for an FP32 one) returns SW_EINVAL.
 * It calls no cudaMalloc/cudaFree and touches none of the context's workspace.  The
 * first call on a device looks up the array's device address (once per device, with that device
 * current); make that first call before any stream capture.  All calls share the array, so calls
 * that overlap on the GPU race: serialise them. */
sw_status sw_matrix_apply_static(const sw_matrix* U, const double* w, double* y_out);
/* Free a matrix returned by sw_project (NULL is a no-op).  May be called before or after
 * sw_destroy of its context: a destroyed context's bookkeeping lives until its last matrix
 * is freed. */
sw_status sw_matrix_free(sw_matrix* U);

/* ---- diagnostics and test hooks -------------------------------------------- */

/* Trajectories of n orbits (host ics, n x 6) under the context's potential and precision with
 * pattern speed omega_p and step dt: out is host n x (nsteps + 1) x 6 (inertial x, v at t_n). */
sw_status sw_trajectory(sw_ctx* ctx, const double* ics, int64_t n, double omega_p, double dt, int64_t nsteps,
                        double* out);
/* Static bar-frame potential and acceleration of the context's potential at n host points
 * (n x 3), in the context's precision: phi_out n, acc_out n x 3 (host). */
sw_status sw_potential_eval(sw_ctx* ctx, const double* xyz, int64_t n, double* phi_out, double* acc_out);

/* Per-kernel CUDA-event timing: when enabled every kernel launch of this context is bracketed by
 * events on the context's stream.  sw_kernel_stats synchronises the stream and returns, for
 * kernel index k (0 <= k < sw_kernel_count()), its name, launch count and total milliseconds
 * since the last reset; sw_reset_stats clears them.  sw_launch_count returns the number of
 * kernels this context has launched since its creation (timing on or off). */
sw_status sw_set_profiling(sw_ctx* ctx, int enable);
int sw_kernel_count(void);
sw_status sw_kernel_stats(sw_ctx* ctx, int k, const char** name, int64_t* launches, double* total_ms);
sw_status sw_reset_stats(sw_ctx* ctx);
/* Algorithmic work accumulated by kernel k while profiling is on (since the last reset): *kind 1 =
 * FLOPs on the SIMT pipes (dense factorisation, MLP), 2 = FLOPs on the tensor cores (Gram), 3 = HBM
 * bytes (streaming kernels: the bytes their algorithm must move), 4 = orbit-steps (orbit kernels),
 * 0 = not counted.  Either output may be NULL. */
sw_status sw_kernel_work(sw_ctx* ctx, int k, double* work, int* kind);
int64_t sw_launch_count(const sw_ctx* ctx);
/* Number of device allocations (cudaMalloc of a workspace buffer) the context has made since its
 * creation; -1 for a NULL context.  Lets a caller check that a call allocated nothing. */
int64_t sw_alloc_count(const sw_ctx* ctx);

/* Tunables (value semantics in parentheses); unknown keys return SW_EINVAL.  The ADMM keys apply to the
 * paper's solver (Sec. 2.3), the "as_" keys to the active-set solver; "solver" chooses between them.
 *  "ej_every" (>= 1)        steps between Jacobi-energy checks in sw_project (default 1 in FP64, 8 in FP32)
 *  "admm_max_iter" (>= 1)   ADMM iteration cap per run (default 400; a run also stops when its residual
 *                           has not halved over five checks)
 *  "admm_tol" (> 0)         ADMM stopping tolerance (default 1e-6)
 *  "refine_max" (>= 0)      refinement rounds with FP64 residuals (default 8)
 *  "kkt_tol" (> 0)          KKT tolerance relative to max |U~^T y~| (default 1e-9)
 *  "check_every" (>= 1)     ADMM iterations between convergence checks (default 20)
 *  "admm_rho" (> 0)         ADMM penalty of orbit i is admm_rho * ||column i of U~||^2 when the Gram is
 *                           in orbit space (default 0.01)
 *  "admm_rho_cspace" (> 0)  the same for the constraint-space (Woodbury) form (default 1)
 *  "admm_alpha" (0, 2)      ADMM over-relaxation (default 1.6)
 *  "chi2_tol" (>= 0)        refinement also stops when chi^2 changes by less than this, relative (1e-6)
 *  "polish_max" (>= 0)      largest support the exact active-set polish handles (default 2048; 0 = off)
 *  "polish_solves" (>= 0)   cap on reduced solves of one polish (default 400)
 *  "inner_refine" (0..8)    refinement steps of each ADMM linear solve against the Gram (default 1)
 *  "verbose" (0, 1, 2)      print solver progress to stderr (default 0; the only output the library makes)
 *  "working_set" (0/1)      ADMM path, N > M: orbit-space solves (default 1); 0 uses the constraint-space
 *                           (Woodbury) form of the ADMM step
 *  "orbit_direct_max" (>= 0) ADMM path, N > M up to this many orbits: orbit-space solve on all orbits
 *                           (default 8192); above it the large-library solver below
 *  "large_solver" (0/1)     above orbit_direct_max orbits: 0 active set (default), 1 ADMM on a working set
 *  "as_block" (>= 1)        active set: KKT violators entering per pivoting step (default 1024)
 *  "as_cg_max" (>= 0)       active set: preconditioned conjugate-gradient steps per reduced solve (default 200)
 *  "as_border" (0 .. 4096)  active set, FP32 tensor-core form: a passive set that adds at most this many orbits
 *                           to the factored set extends its factor by bordering (the new block row of the
 *                           factor's inverse from the kept one) instead of refactoring (default 256; 0: off)
 *  "as_mask" (0 .. 1)       active set: a factor serves the passive sets inside its factored set that leave at
 *                           most this fraction of it masked (default 0.02); more masked orbits refactor
 *  "as_cg_tol" (> 0)        active set: CG stops at max|r| <= as_cg_tol * kkt_tol * max|q| (default 0.05)
 *  "as_solves" (>= 1)       active set: cap on pivoting steps (default 400)
 *  "solver" (0/1/2)         0 (default): the active set when lambda > 0, when N <= M, or for libraries above
 *                           orbit_direct_max orbits, ADMM otherwise; 1: always the active set; 2: always ADMM
 *                           (the paper's solver, Sec. 2.3, with FP64 refinement and the exact polish)
 *  "chol_coop" (0/1)        active set: Cholesky and its inverse in one cooperative launch (default 0)
 *  "project_bundle" (>= 1)  orbits per column of sw_project's matrix (default 1): with n > 1 the n consecutive
 *                           orbits of a bundle (Sec. 2.2.1) accumulate into one column at bin time, which holds
 *                           their mean (counts / (copies nsteps n)); a realisation cut by the quality test adds a
 *                           zero column to the mean (its counts are removed exactly, GH sums to rounding), as
 *                           sw_bundle of the unbundled matrix; n must divide the orbit count; fixed-step KDK only
 *  "matrix_cache" (0/1)     sw_matrix_free keeps the freed matrix's device buffer in its context for the next
 *                           matrix of about the same size (at most four buffers; released by sw_destroy, on an
 *                           allocation failure, or by setting 0) instead of returning it to the driver (default 1)
 *  "chol_tc" (0/1)          active set, FP32 form: Cholesky and its inverse in 128-wide steps with the trailing and
 *                           inverse updates on the tensor cores (BF16 hi + lo split, default 1); 0: FP32 SIMT updates
 *  "boot_p0_extra" (0 .. 4) sw_solve_bootstrap: the factor kept for the realisations covers the plain solve's
 *                           support plus this fraction of it in near-active orbits (default 0: a wider factored set
 *                           serves more passive sets but preconditions the masked solves worse)
 *  "chol_pdl" (0/1)         tensor-core factorisation: each panel kernel launched programmatically behind its
 *                           diagonal-block kernel, staging its rows while that block is factored (default 1)
 *  "chol_panel_tc" (0/1)    tensor-core factorisation, 256-wide steps: each panel P = A D^T on the tensor cores from
 *                           the BF16 hi + lo split of A and D (1), or in FP32 SIMT (default 0: as fast, and the
 *                           FP32 panel keeps the preconditioner closer, fewer conjugate-gradient steps)
 *  "chol_super" (0/1)       tensor-core factorisation: two 128-wide diagonal blocks per step, their panels side by
 *                           side, so that the trailing matrix and the inverse take one rank-256 update per two
 *                           blocks (default 1); 0: a rank-128 update per block
 *  "chol_reserve_sms" (>= 0) tensor-core factorisation: SMs that the bulk trailing and inverse updates leave free
 *                           for the next steps' diagonal-block chain on the context's stream (default 8)
 *  "integrator" (0/1)       sw_project's integrator: 0 (default) kick-drift-kick at the fixed dt in the inertial
 *                           frame; 1 the paper's adaptive Bogacki-Shampine 3(2) pair (Sec. 2.2.2) in the frame
 *                           rotating with the bar, nsteps accepted steps from a first trial step dt, each sample
 *                           weighted by its step over the orbit's total time (Sec. 2.2.4)
 *  "bs3_rtol" (0, 1)        relative tolerance of the adaptive integrator on |x| and |v| per step (default 1e-4)
 *  "as_grow" (>= 0)         active set: at most max(as_block, as_grow |F|) orbits enter per step (default 0)
 *  "as_candidates" (>= 0)   active set: initial candidate-set size, 0 for 2 M (default 0)
 *  "ws_factor" (> 0)        initial working-set size in units of M (default 0.6; it grows to take in the
 *                           violators of each round, up to three times that)
 *  "ws_rounds" (>= 1)       working-set exchange rounds (default 6)
 *  "gram_tensor_cores" (0/1) tcgen05 BF16 Gram in the FP32 form (default 1; the operand is split into
 *                           BF16 hi + lo halves and three products are accumulated) */
sw_status sw_set_option(sw_ctx* ctx, const char* key, double value);

/* ---- Batched model construction.  The paper evaluates one trial potential at a time inside its
 * MCMC (Sec. 3.2); a batch builds the orbit matrices of many trial potentials at once: each model k
 * has its own potential, pattern speed, viewing angles and orbit count n_orb[k], and all share the
 * step count, dt and the observation grid.  One persistent launch integrates, projects and bins
 * every orbit of every model from a work queue of (model, orbit tile) items; the launch shape
 * (threads per CTA, CTAs) is chosen on the first run by timing short probe runs of the actual
 * models, and the run (zeroing, orbit kernel, quality cut, normalisation) is captured in a CUDA graph
 * that later runs replay.  Results are per-model matrices identical to those of sw_project with the
 * same inputs (Sec. 2.2.3-2.2.4). */
typedef struct sw_batch sw_batch;
/* Allocate a batch of n_models models (n_orb: host, n_models counts >= 1) with nsteps steps on the
 * given grid (vb NULL when gh != 0: Gauss-Hermite rows, as sw_project with gh_v0_s).  The batch
 * owns all its device memory; free it with sw_batch_destroy. */
sw_status sw_batch_create(sw_ctx* ctx, int n_models, const int64_t* n_orb, int64_t nsteps, const sw_pixel_grid* pix,
                          const sw_vbins* vb, const sw_density_grid* dens, int gh, int mirror4, sw_batch** out);
/* Load the models: pots[k], omega_p[k], angles[3 k .. 3 k + 2] = (incl, pa, bar_angle) of model k,
 * the common dt, ics (host, sum(n_orb) x 6 inertial initial conditions, model after model) and in GH
 * mode gh_v0_s (host, n_models x npix x 2 reference (v0, s) per pixel).  Host arrays are read during
 * the call only. */
sw_status sw_batch_set_models(sw_batch* b, const sw_potential_params* pots, const double* omega_p,
                              const double* angles, double dt, const double* ics, const double* gh_v0_s);
/* Build every model's matrix (autotunes and captures the graph on the first call). */
sw_status sw_batch_run(sw_batch* b);
/* A borrowed view of model k's matrix: valid until the batch is destroyed, overwritten by the next
 * sw_batch_run; usable wherever a matrix is read (sw_solve_weights, sw_matrix_copy, ...), but
 * sw_matrix_free refuses it (SW_EINVAL). */
sw_status sw_batch_matrix(sw_batch* b, int k, sw_matrix** view);
/* Per-orbit Jacobi drift and status of the last run (host arrays of sum(n_orb), either may be NULL). */
sw_status sw_batch_stats(sw_batch* b, double* drift_out, uint8_t* status_out);
/* info4 = (threads per CTA, CTAs, autotuned 0/1, graph 0/1); tune_ms12 (nullable) receives the probe
 * times of the 12 candidate shapes (threads 64, 128, 256 x 1, 2, 4, 8 CTAs per SM; -1 if not run). */
sw_status sw_batch_info(const sw_batch* b, int64_t* info4, double* tune_ms12);
sw_status sw_batch_destroy(sw_batch* b);

/* ---- Learned chi^2 emulator (no counterpart in the paper's method).  The paper samples the
 * potential parameters by MCMC on the exact chi^2, 1.3 s per evaluation (Sec. 3.2), and names
 * differentiable surrogates as the route to cheaper likelihoods (Sec. 5.3).  These calls train and
 * run a fully connected network n_in -> width (n_hidden SiLU layers) -> 1 that screens MCMC
 * proposals before the exact model judges them (delayed acceptance, Christen & Fox 2005).
 * Parameters: one FP32 device array; for each layer l, W_l (out x in, row-major) then b_l (out).
 * All arrays are device memory owned by the caller; activations live in the context's scratch.
 * Errors: SW_EINVAL for a bad shape or NULL pointer, SW_ECUDA / SW_ENOMEM from the runtime. */
/* Number of parameters of the network (-1 for an invalid shape). */
int64_t sw_mlp_param_count(int n_in, int width, int n_hidden);
/* out[b] = f(x[b, :]) for batch rows of x (batch x n_in, row-major FP32).  bf16 != 0 rounds weights
 * and layer inputs to BF16 as they enter each product (FP32 accumulation): the inference form. */
sw_status sw_mlp_forward(sw_ctx* ctx, int n_in, int width, int n_hidden, const float* params_dev,
                         const float* x_dev, int64_t batch, int bf16, float* out_dev);
/* Mean-squared error L = mean_b (f(x_b) - t_b)^2 (*loss_out, host) and its gradient dL/dparams
 * (grad_dev, same layout as params) by back-propagation, FP32. */
sw_status sw_mlp_loss_grad(sw_ctx* ctx, int n_in, int width, int n_hidden, const float* params_dev,
                           const float* x_dev, const float* t_dev, int64_t batch, float* grad_dev,
                           double* loss_out);
/* One Adam step (Kingma & Ba 2015, bias-corrected; step >= 1 counts from 1) on n_params values:
 * m, v are the caller's moment arrays (zero before the first step). */
sw_status sw_mlp_adam(sw_ctx* ctx, int64_t n_params, float* params_dev, const float* grad_dev, float* m_dev,
                      float* v_dev, int64_t step, double lr, double beta1, double beta2, double eps);

#if defined(__GNUC__)
#pragma GCC visibility pop
#endif
#ifdef __cplusplus
}
#endif
#endif /* SW_H */
