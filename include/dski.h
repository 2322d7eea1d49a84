/*
 * dski.h -- C ABI of the GB300 D-SKI library.
 *
 * D-SKI (Eriksson et al., "Scaling Gaussian Process Regression with
 * Derivatives", NeurIPS 2018, Sec. 3.1) approximates the kernel matrix of a
 * Gaussian process observed through values AND gradients at n points in d
 * dimensions (the n(d+1) x n(d+1) matrix K^grad of Sec. 2) by
 *
 *     K~ = [W; dW_1; ...; dW_d] K_UU [W; dW_1; ...; dW_d]^T + diag(noise)
 *
 * where W holds cubic-convolution interpolation weights (Keys, a = -1/2) on a
 * regular grid U, dW_p their derivatives in dimension p, and K_UU is the
 * squared-exponential (SE) kernel of App. A on the grid, a Kronecker product
 * of one m_k x m_k factor per dimension.  The library computes MVMs with K~
 * (Sec. 3.1), builds the truncated pivoted-Cholesky preconditioner of
 * Sec. 3.3, solves K~ x = b by preconditioned CG (Sec. 2), estimates
 * log|K~| by stochastic Lanczos quadrature (Sec. 2) and differentiates the
 * log marginal likelihood of Eq. 1 with respect to the hyperparameters.
 *
 * Conventions shared by every call
 * --------------------------------
 * - N = n (d + 1).  A length-N vector is in the block order of Sec. 3.1:
 *   [values (n); d/dx_1 (n); ...; d/dx_d (n)], each block in the caller's
 *   point order.  s right-hand sides are column-major N x s (column j starts
 *   at element j*N).
 * - Pointers named *_dev are device pointers owned by the caller; pointers
 *   named *_host are host pointers owned by the caller.  The library never
 *   frees caller memory and keeps no caller pointer after a call returns.
 * - All device work is issued on the stream given to dski_create.  Calls
 *   that return host results synchronise that stream before returning.
 * - A handle is not thread-safe; distinct handles may be used concurrently.
 * - Every int-returning call returns DSKI_OK (0) or a negative dski_status;
 *   dski_last_error() then gives a message (thread-local, valid until the
 *   next failing call on that thread).
 */
#ifndef DSKI_H
#define DSKI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dski_handle_* dski_handle;
typedef struct pivchol_* pivchol_handle;

typedef enum {
  DSKI_OK = 0,
  DSKI_ERR_ARG = -1,            /* bad size, pointer or hyperparameter      */
  DSKI_ERR_OUT_OF_GRID = -2,    /* a point lacks its full 4^d stencil       */
  DSKI_ERR_CUDA = -3,           /* a CUDA runtime call failed               */
  DSKI_ERR_NOT_CONVERGED = -4,  /* maxit reached; outputs hold best iterate */
  DSKI_ERR_BREAKDOWN = -5,      /* NaN/Inf, p^T A p <= 0, non-PD r x r      */
  DSKI_ERR_TIMEOUT = -6,        /* a device-side wait exceeded its budget   */
  DSKI_ERR_ALLOC = -7           /* device allocation failed                 */
} dski_status;

/* Arithmetic of the MVM.  FP64: every step in double.  MIXED_3XTF32: FP32
 * scatter/gather, Kronecker mode products on the tensor cores in TF32 with
 * the three-product split (hi*hi + hi*lo + lo*hi) and FP32 accumulation.
 * MIXED_TF32: as MIXED_3XTF32 with a single TF32 product.  In the mixed
 * modes CG scalars, dot products, x and r stay FP64 (see dski_pcg_solve).
 * FP64_TC: FP64 vectors, scatter and gather as in FP64, Kronecker mode
 * products (for m_k >= 64) on the BF16 tensor cores: each row of both
 * operands is scaled to a 62-bit integer and split into eight signed 8-bit
 * digits; the 36 leading digit-pair products accumulate exactly in FP32 and
 * combine exactly in integers (error ~2^-61 of the row maxima's product
 * per term); needs every m_k a multiple of 8 and <= 256.  Vectors are
 * double in FP64 and FP64_TC, float in the MIXED modes. */
typedef enum { DSKI_FP64 = 0, DSKI_MIXED_3XTF32 = 1, DSKI_MIXED_TF32 = 2,
               DSKI_FP64_TC = 3 } dski_precision;

/* Interpolation scheme of W and dW (Sec. 3.1): the rows of W hold the
 * tensor products of a 1-D convolution kernel phi at the grid nodes, dW its
 * derivatives.  CUBIC: Keys' cubic convolution (a = -1/2), 4 nodes per
 * dimension (4^d per row).  QUINTIC: the six-point quintic kernel the paper
 * uses (Meijering et al. 1999: even, piecewise quintic, interpolating, C^3,
 * reproducing quadratics), 6 nodes per dimension (6^d per row).  A
 * zero-initialised dski_params selects CUBIC. */
typedef enum { DSKI_INTERP_CUBIC = 0, DSKI_INTERP_QUINTIC = 1 } dski_interp;

/* How the products with K_UU are formed (Sec. 3.1).  DENSE: each Kronecker
 * factor K_k is applied as a dense m_k x m_k matrix (FP64 units, or the
 * tensor cores as the precision mode says).  FFT: each factor is a
 * symmetric Toeplitz matrix on the regular grid and is applied through its
 * embedding in an L x L circulant (L the smallest power of two >= 2 m_k - 1)
 * with FP64 FFTs, O(m_k log m_k) per grid line instead of O(m_k^2); FP64 and
 * FP64_TC modes only.  The FFT's rounding is normwise (~log2(L) u |Fc| |x|
 * per product), so dski_pcg_solve ends each pass at a 1e-4 reduction of the
 * residual (not while SLQ records Lanczos coefficients), forms its true
 * residuals with the dense factors, and its restarts refine x against the
 * dense operator.  The
 * gradient of Eq. 1 applies dK_k / dlog l_k densely in either case.  A
 * zero-initialised dski_params selects DENSE. */
typedef enum { DSKI_KUU_DENSE = 0, DSKI_KUU_FFT = 1 } dski_kuu;

/* Problem statement of Sec. 2 / Sec. 3.1 / App. A.
 *   n, d          points and dimensions, n >= 1, 1 <= d <= 3.
 *   grid_m[d]     grid nodes per dimension, S <= m_k <= 1027 (S = 4 for the
 *                 cubic, 6 for the quintic stencil); grid nodes are
 *                 u_a = lo_k + a (hi_k - lo_k)/(m_k - 1), a = 0..m_k-1 (both
 *                 end points included); the grid is flattened in C order.
 *   grid_lo/hi[d] grid extent, lo_k < hi_k.  With c = floor((x_k - lo_k)/h_k)
 *                 the stencil nodes are c - 1 .. c + 2 (cubic) or
 *                 c - 2 .. c + 3 (quintic), so every point needs
 *                 1 <= c <= m_k - 3 (cubic) or 2 <= c <= m_k - 4 (quintic) in
 *                 every dimension (else OUT_OF_GRID).
 *   lengthscale[d] SE length scales l_k > 0 (ARD form of App. A).
 *   outputscale   sigma_f > 0; K_UU = sigma_f^2 K_1 (x) ... (x) K_d with
 *                 K_k[a,b] = exp(-(u_a - u_b)^2 / (2 l_k^2)).
 *   noise_value   sigma^2 added on value rows (> 0).
 *   noise_grad    sigma^2 added on gradient rows (> 0).  Sec. 2 uses one
 *                 noise; the terrain experiment of Sec. 4 fits two.
 *   prec          arithmetic of the MVM (dski_precision).
 *   interp        interpolation scheme (dski_interp; 0 = CUBIC).
 *   kuu           K_UU product (dski_kuu; 0 = DENSE).
 * The arrays are read during dski_create only. */
typedef struct {
  int n, d;
  const int* grid_m;
  const double* grid_lo;
  const double* grid_hi;
  const double* lengthscale;
  double outputscale;
  double noise_value, noise_grad;
  dski_precision prec;
  dski_interp interp;
  dski_kuu kuu;
} dski_params;

/* Sec. 3.1: build the D-SKI operator for the points X_dev (device, n x d
 * row-major FP64).  Computes each point's grid cell and cell fractions in
 * FP64, sorts the points by cell (stable, deterministic), builds the cell
 * index and the Kronecker factors.  The handle owns all of it and a
 * workspace; X_dev is not referenced afterwards.  cuda_stream is a
 * cudaStream_t (NULL = legacy default stream).
 * Errors: ARG, OUT_OF_GRID, ALLOC, CUDA.  On error *out is NULL. */
int dski_create(dski_handle* out, const dski_params* params, const double* X_dev,
                void* cuda_stream);

/* Replace the hyperparameters (lengthscale[d], outputscale, both noises)
 * of an existing handle; rebuilds the Kronecker factors.  Preconditioners
 * built earlier keep the hyperparameters they were built with.
 * Errors: ARG, CUDA. */
int dski_set_hypers(dski_handle h, const double* lengthscale, double outputscale,
                    double noise_value, double noise_grad);

/* Sec. 3.1: out = K~ v for s >= 1 columns.  v_dev and out_dev are device
 * N x s column-major, FP64 (double) in the FP64 and FP64_TC modes and FP32
 * (float) in the MIXED modes; they must not overlap.  The product runs as
 * scatter (B^T v onto the grid) -> d Kronecker mode products -> gather
 * (B h) plus the noise diagonal.  Asynchronous on the handle's stream.
 * Errors: ARG, CUDA. */
int dski_mvm(dski_handle h, const void* v_dev, void* out_dev, int s);

/* Sec. 3.3: truncated pivoted Cholesky of the noise-free D-SKI matrix
 * K^grad_SKI = B K_UU B^T, computed from its diagonal and pivot rows only:
 * greedy pivot = largest residual diagonal (lowest block-order index on
 * ties); stops at `rank` steps or when the residual trace drops below
 * 1e-14 times the initial trace.  Then forms the preconditioner
 * M = D + L L^T (D = noise diagonal) in the QR-stable form of Sec. 3.3,
 * M^-1 b = D^-1/2 (y - Q1 (Q1^T y)), y = D^-1/2 b, with Q1 from two
 * CholeskyQR passes in FP64 (stored FP32 in the mixed modes with an FP64
 * r x r correction that keeps M^-1 symmetric positive definite).
 * 1 <= rank <= 128.  *rank_achieved (host) receives the steps taken.
 * The pivchol handle holds device memory until pivchol_destroy and is tied
 * to the hyperparameters current at build time.
 * Errors: ARG, BREAKDOWN, ALLOC, CUDA. */
int pivchol_build(dski_handle h, int rank, pivchol_handle* out, int* rank_achieved);

/* Sec. 3.3: copy the preconditioner's factor out.  L_dev (device, may be
 * NULL) receives L as N x rank_achieved column-major FP64 in the caller's
 * block order; pivots_host (host, may be NULL) receives the pivot rows in
 * the order chosen, as caller block-order row indices.  Synchronises.
 * Errors: ARG, CUDA. */
int pivchol_export(pivchol_handle pc, double* L_dev, int* pivots_host);

/* Sec. 3.3: log|M| = sum log D + log|I + L^T D^-1 L| (Sylvester's identity,
 * from the CholeskyQR factor R); NaN for a NULL handle. */
double pivchol_logdet(pivchol_handle pc);

/* Sec. 2 / Sec. 3.3: solve K~ x = b for s columns by preconditioned CG.
 *   pc       preconditioner from pivchol_build, or NULL for plain CG.
 *   b_dev    device N x s FP64 right-hand sides (block order).
 *   x_dev    device N x s FP64; on entry the initial guess, on exit the
 *            solution.
 *   rtol     stop when ||b - K~ x||_2 <= rtol ||b||_2 per column, the
 *            residual recomputed in FP64.
 *   maxit    iteration cap (MVMs of the inner loop).
 *   iters_host[s], relres_host[s]  iterations and final true relative
 *            residual per column (FP64 residual, even in the mixed modes).
 * FP64 mode runs PCG entirely in double.  In the mixed modes the MVM runs
 * in FP32 / (3x)TF32 while x, r, the dot products and the CG recurrences
 * are FP64, and the residual is periodically replaced by the FP64 residual
 * b - K~ x (reliable updates), so the FP64 tolerance is reachable.
 * Errors: ARG, NOT_CONVERGED (outputs filled), BREAKDOWN, CUDA. */
int dski_pcg_solve(dski_handle h, pivchol_handle pc, const double* b_dev, double* x_dev,
                   int s, double rtol, int maxit, int* iters_host, double* relres_host);

/* Sec. 2 / Sec. 3.3: solve K~_i x_i = b_i for `count` independent systems
 * (each its own handle: any n, d, grid and hyperparameters) in ONE
 * persistent launch of thread-block clusters.  A cluster of `cluster` CTAs
 * solves one system at a time, start to finish: its CTAs split the points,
 * rows and grid between them, each keeping the grid vector and Kronecker
 * factors in its shared memory and exchanging grid slices through
 * distributed shared memory; the cluster then takes the next system from a
 * device work queue ordered by estimated cost per iteration, largest first.
 * The PCG is dski_pcg_solve's in FP64: restarts from the FP64 true
 * residual, at most 64 passes, maxit MVMs.
 *   hs[count]     handles with FP64 vectors (FP64 or FP64_TC mode; here
 *                 the mode products always run the FP64 factors K_k on the
 *                 FP64 units); every m_k <= 64 and (M + sum_k m_k^2)
 *                 doubles must fit in one CTA's shared memory (~227 KB:
 *                 a 24^3 or 48^2 grid fits, 40^3 does not).
 *   pcs[count]    pivchol_build preconditioners of those handles (rank <=
 *                 32), applied in their QR form; pcs or an entry NULL: none.
 *   b[count]      device pointers, N_i FP64 each, block order (as dski_mvm).
 *   x[count]      device pointers, N_i FP64 each: initial guess in,
 *                 solution out.  b and x must be ready before the call.
 *   rtol, maxit   per system, as dski_pcg_solve.
 *   cluster       CTAs per system: 1, 2, 4 or 8; 0 picks the library's
 *                 default (4).  More CTAs finish a large system sooner;
 *                 fewer spend less on exchanges when systems are small.
 *   iters, relres, status, seconds  host arrays of count entries, each may
 *                 be NULL: MVMs, the final FP64 true relative residual, the
 *                 system's DSKI_OK / NOT_CONVERGED / BREAKDOWN, and the
 *                 system's solve time inside the launch (device clock).
 * The scatter adds with shared-memory atomics in no fixed order, so results
 * may differ between runs in their last bits.  Waits for every handle's
 * stream, runs on hs[0]'s stream, allocates its workspace (6 N_i doubles
 * per system) for the call and returns when done.
 * Errors: ARG (nothing runs), ALLOC, CUDA; NOT_CONVERGED or BREAKDOWN
 * (the status of the first failing system; every output is filled). */
int dski_pcg_solve_batch(int count, const dski_handle* hs, const pivchol_handle* pcs,
                         const double* const* b, double* const* x, double rtol, int maxit,
                         int cluster, int* iters, double* relres, int* status, double* seconds);

/* Sec. 2: stochastic Lanczos quadrature estimate of log|K~|.
 * Probe j (0-based) is z_j = D^1/2 (w1_j + L' w2_j), where w = [w1; w2] is a
 * Rademacher vector of length N + r and L' the preconditioner's low-rank
 * factor scaled by D^-1/2, so E[z z^T] = M.  Entry e of w (block-order row
 * for e < N, then the r extra rows) is +1 if the top bit of
 * SplitMix64(seed)[j (N + r) + e + 1] is 0 and -1 otherwise (the k-th
 * output of SplitMix64 is mix64(seed + k 0x9E3779B97F4A7C15)).  All probes
 * run in one batched PCG; the first `depth` CG coefficients of each give the
 * Lanczos tridiagonal T_j, and
 *   log|K~| ~ log|M| + mean_j (z_j^T M^-1 z_j) e1^T log(T_j) e1.
 * pc is required; 2 <= probes <= 256, 1 <= depth <= 128.
 * logdet_host and stderr_host (standard error over probes) are host
 * scalars.  Errors: ARG, BREAKDOWN, CUDA. */
int dski_logdet_slq(dski_handle h, pivchol_handle pc, int probes, int depth, uint64_t seed,
                    double* logdet_host, double* stderr_host);

/* Eq. 1: log marginal likelihood L = -1/2 [y^T a + log|K~| + N log 2 pi],
 * a = K~^-1 y, and its gradient with respect to
 * theta = (log l_1, ..., log l_d, log sigma_f, log sigma_n) (both noises
 * scale with sigma_n^2):
 *   dL/dtheta_i = 1/2 a^T (dK~/dtheta_i) a - 1/2 tr(K~^-1 dK~/dtheta_i),
 * the trace estimated with the probes of dski_logdet_slq
 * (mean_j (K~^-1 z_j)^T dK~ (M^-1 z_j)).  The solve uses rtol 1e-8 (FP64
 * residual).  y_dev: device length-N FP64.  mll_host: host scalar;
 * grad_host: host array of d + 2.  Errors: ARG, NOT_CONVERGED, BREAKDOWN,
 * CUDA. */
int dski_mll_grad(dski_handle h, pivchol_handle pc, const double* y_dev, int probes,
                  uint64_t seed, double* mll_host, double* grad_host);

/* Eq. 1, as dski_mll_grad with the batched PCG's stopping rule given:
 * every column (the solve K~ a = y and the P probe solves) stops when its
 * FP64 true relative residual is <= rtol (0 < rtol < 1), or after maxit
 * iterations (then NOT_CONVERGED).  dski_mll_grad is this call with
 * rtol = 1e-8, maxit = 100000.  Errors: as dski_mll_grad. */
int dski_mll_grad_tol(dski_handle h, pivchol_handle pc, const double* y_dev, int probes,
                      uint64_t seed, double rtol, int maxit, double* mll_host,
                      double* grad_host);

/* Prediction at n_star test points (Sec. 5: the mean, and the fast
 * predictive-variance estimate, that Bayesian optimisation evaluates at many
 * points).  The D-SKI cross-covariance of the test values / gradients with
 * the training data is [W*; dW*] K_UU [W; dW]^T (Sec. 3.1), so
 *   mean:      mu_star = [W*; dW*] K_UU [W; dW]^T alpha,
 *   variance:  v_hat(x) = s_f^2 - k_x^T M^-1 k_x,  k_x = [W; dW] K_UU w*(x)^T,
 * M = D + L L^T the pivoted-Cholesky preconditioner of `pc` (Sec. 5's first
 * approach: K~^-1 replaced by the preconditioner solve).  M <= K~, so v_hat
 * is at most the D-SKI variance s_f^2 - k_x^T K~^-1 k_x.
 *   alpha_dev: N = n (d+1) FP64, caller block order (K~^-1 y, e.g. the x of
 *              dski_pcg_solve with b = y); needed for the mean.
 *   Xs_dev:    n_star x d FP64, row-major; every test point needs a full
 *              stencil inside the grid (else DSKI_ERR_OUT_OF_GRID).
 *   with_grad: 0: mean_dev holds n_star values; 1: n_star (d + 1) values in
 *              block order [mean; its x_1 derivative; ...; its x_d derivative].
 *   mean_dev / var_dev: device outputs (n_star FP64 for the variance); either
 *              may be NULL (then that part is skipped).  var_dev needs pc.
 * All arithmetic is FP64 whatever the handle's mode.  Synchronises the
 * handle's stream.  Errors: ARG, OUT_OF_GRID, ALLOC, CUDA. */
int dski_predict(dski_handle h, pivchol_handle pc, const double* alpha_dev, const double* Xs_dev,
                 int n_star, int with_grad, double* mean_dev, double* var_dev);

/* Unbiased predictive variance at n_star test points by Sec. 5's second
 * approach: the randomized diagonal estimator (Bekas et al.) with the
 * preconditioner estimate v_hat as control variate,
 *   v = v_hat - diag(K_*X (K~^-1 - M^-1) K_X*),
 *   diag(A) ~ (1/P) sum_j z_j .* (A z_j),
 * z_j Rademacher over the test points: entry (i, j) is the sign of output
 * number j n_star + i + 1 of the SplitMix64 stream seeded with `seed`
 * (the convention of dski_logdet_slq).  The P probe solves K~ a = K_X* z_j
 * run as one batched PCG (rtol, maxit).  Xs_dev: n_star x d FP64 row-major;
 * var_dev: n_star FP64 (device).  The test-point scatter adds with FP64
 * atomics where test points share grid nodes, so results are reproducible
 * to rounding, not bitwise.  Errors: ARG, OUT_OF_GRID, NOT_CONVERGED (var_dev
 * still filled), ALLOC, CUDA. */
int dski_predict_var_cv(dski_handle h, pivchol_handle pc, const double* Xs_dev, int n_star,
                        int probes, uint64_t seed, double rtol, int maxit, double* var_dev);

/* Profiling aid (the paper has no counterpart): per-stage device timers.
 * Stages, in order: 0 permute (user block order <-> internal layout),
 * 1 scatter, 2 Kronecker mode products, 3 gather (+ noise), 4 preconditioner
 * apply, 5 CG vector work (dots, updates, residual refinement),
 * 6 pivoted Cholesky build, 7 Lanczos / quadrature.
 *   mode 1: reset and start recording.  Every stage launch issued on the
 *           handle's stream is bracketed by a pair of CUDA events.
 *   mode 0: stop; synchronise the stream; write, per stage, the summed
 *           device milliseconds to ms_host[DSKI_NSTAGES], the number of
 *           kernels launched to launches_host[DSKI_NSTAGES] and the number of
 *           those inside a timed event pair to timed_host[DSKI_NSTAGES] (any
 *           may be NULL).  At most 2^18 event pairs are kept; launches beyond
 *           that are counted but not timed (*truncated_host, may be NULL, = 1),
 *           so ms / timed is the mean time per launch.
 * Errors: ARG, CUDA. */
#define DSKI_NSTAGES 8
int dski_profile(dski_handle h, int mode, double* ms_host, long long* launches_host,
                 long long* timed_host, int* truncated_host);

/* Number of CUDA kernels this library has launched in this process (all
 * handles).  A host-side counter, incremented at every launch site. */
long long dski_launch_count(void);

/* Test aid for failure handling (the paper has no counterpart).  Every
 * CTA of the tensor-core mode products (FP64_TC, and the MIXED modes' split
 * contraction) waits on an mbarrier for its TMA loads with a bounded number
 * of polls; when the budget runs out the CTA records a device error word,
 * waits (with the full budget) for its loads to land, frees its tensor
 * memory and returns, so the context stays usable.  The next dski_pcg_solve
 * host check (at most 16 iterations later), dski_logdet_slq or
 * dski_mll_grad then returns DSKI_ERR_TIMEOUT and clears the word.
 *   polls >= 0  caps that first wait of every later product launched on
 *               this handle at `polls` polls (0: it gives up at once);
 *   polls < 0   restores the default budget (2^22 polls).
 * The products of a launch whose wait gave up are not valid.
 * Errors: ARG (NULL handle). */
int dski_set_wait_budget(dski_handle h, int polls);

/* The paper has no counterpart: this is dski_mvm for callers that cannot
 * allocate device memory -- applications whose device memory belongs to a
 * pool allocator that must see every allocation, real-time loops where
 * cudaMalloc's implicit device synchronisation is not allowed, plug-ins
 * whose host forbids device allocation after start-up.  Same arguments,
 * layouts and result as dski_mvm, but it calls no cudaMalloc, cudaFree or
 * allocating library routine: its temporaries live in one fixed device array
 * of DSKI_NOALLOC_SCRATCH_BYTES (32 MiB) that the library reserves on every
 * GPU that loads it, until the process exits.  They are:
 *   - the permuted input and output, N x s each, and two grids, M x s each,
 *     in the mode's element size;
 *   - the scatter's intermediate: with the cubic stencil, d = 2 and a MIXED
 *     mode, its per-cell stencil sums, 16 floats per cell of the grid and
 *     column; in FP64 mode with d >= 2 and s <= 4, its per-point
 *     sum-factorised coefficients, 2 S (d = 2) or 2 S^2 (d = 3) doubles per
 *     point and column, S the stencil width (4 cubic, 6 quintic);
 *   - in the MIXED modes, the tensor-core mode products' split-contraction
 *     partials (for m_k % 4 == 0, m_k <= 256): ceil(m_k/32) FP32 128 x 32
 *     tiles per 128 x 32 output tile and column, for the largest mode.
 *   - Sizes that do not fit (each part padded to 256 bytes) are rejected with
 *     DSKI_ERR_ARG and a message; nothing runs.
 *   - The first call on a device looks up the array's device address (with
 *     that device current); make that first call before any stream capture.
 *   - Every call on a device shares the one array, which keeps the last
 *     call's contents.  Calls whose work overlaps on the GPU (other streams,
 *     other handles, other host threads) race on it: serialise them.
 *   - The handle must live on the current device (else DSKI_ERR_ARG).
 *   - FP64 and MIXED handles only: an FP64_TC handle is rejected with
 *     DSKI_ERR_ARG (its mode products need a split-contraction workspace).
 * Errors: ARG, CUDA. */
#define DSKI_NOALLOC_SCRATCH_BYTES (32u << 20)
int dski_mvm_noalloc(dski_handle h, const void* v_dev, void* out_dev, int s);

/* Release a handle / preconditioner (NULL is ignored).  Synchronises the
 * handle's stream first. */
void dski_destroy(dski_handle h);
void pivchol_destroy(pivchol_handle pc);

/* Message of the last failing call on this thread ("" if none). */
const char* dski_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* DSKI_H */
