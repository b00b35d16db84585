/*
 * gp.h -- C ABI of the GB300 (sm_103a) preconditioned GP log-marginal-likelihood library.
 *
 * The library evaluates the stochastic estimator of Wenger et al., "Preconditioning
 * for Scalable Gaussian Process Hyperparameter Optimization" (ICML 2022):
 *   Alg. 1  log-marginal likelihood L(theta) = -1/2 (y^T K^-1 y + log det K + n log 2 pi)
 *   Alg. 2  its gradient dL/dtheta (eq. derivative_likelihood)
 * with K_hat = K + sigma^2 I (Sec. 2.1), a rank-k pivoted-Cholesky preconditioner
 * P_hat = sigma^2 I + L L^T applied through the matrix inversion lemma (Sec. 2.2),
 * preconditioned CG on [y, z_1..z_l] with Lanczos tridiagonals taken from the CG
 * coefficients (Sec. S1.2, footnote to Sec. 4.4), and the variance-reduced trace
 * estimators of eqs. (logdet-decomposition) and (logdet-decomposition_deriv).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Pointers are DEVICE pointers owned by the caller unless marked "host".  The
 *   library never allocates device memory: scratch comes from the caller's
 *   workspace `ws` of at least gp_workspace_size(...) bytes (256-byte aligned).
 * - Real arrays (X, y, V, W, L, B, ...) hold double when the problem's precision
 *   is GP_FP64 and float otherwise.  theta and all scalar outputs are double.
 * - X is n x d row-major.  Blocks of vectors (V, W, L, B, ...) are column-major
 *   with a leading dimension >= n.
 * - Arguments are validated on the host before anything is launched; an invalid
 *   call returns GP_ERR_INVALID_ARG (or GP_ERR_WORKSPACE) and launches nothing.
 *   gp_last_error_message() then describes the problem.
 * - Work is enqueued on `stream` (NULL = the legacy default stream).  Functions
 *   marked "asynchronous" return after enqueueing; device-side conditions are
 *   written to device status words.  gp_mbcg and gp_mll_and_grad poll the
 *   device for CG convergence and therefore synchronise with `stream`; they
 *   return the final status, including device-side conditions.
 * - Limits: 1 <= d <= 32, 0 <= k <= min(n, 2048), 1 <= t <= 1024, n < 2^31.
 * - Errors: negative gp_status values; positive values are warnings with full
 *   results written.
 */
#ifndef GP_H
#define GP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* gp_stream_t; /* identical to cudaStream_t */

typedef enum {
  GP_OK = 0,
  GP_WARN_NOT_CONVERGED = 1,   /* a CG column hit max_iter before the tolerance   */
  GP_WARN_RANK_DEFICIENT = 2,  /* pivoted Cholesky stopped below the requested k   */
  GP_ERR_INVALID_ARG = -1,
  GP_ERR_CUDA = -2,
  GP_ERR_NOT_SPD = -3,         /* Woodbury core or a tridiagonal lost definiteness */
  GP_ERR_WORKSPACE = -4,
  GP_ERR_DEVICE_TIMEOUT = -5,  /* an iteration cap in device code was reached      */
  GP_ERR_NUMERIC = -6          /* NaN/Inf or a CG breakdown (p^T K p <= 0)         */
} gp_status;

/* Sec. 5 "Experimental Setup": RBF and Matern kernels with output scale s = k(x,x),
 * lengthscales l_j and noise sigma^2; the rational quadratic kernel of the synthetic
 * study (Tab. S1).  r^2 = sum_j ((x_j - x'_j)/l_j)^2 and
 *   RBF       s exp(-r^2/2)
 *   MATERN32  s (1 + sqrt3 r) exp(-sqrt3 r)
 *   MATERN52  s (1 + sqrt5 r + 5r^2/3) exp(-sqrt5 r)
 *   RATQUAD   s (1 + r^2/(2 alpha))^-alpha with alpha = 1 (fixed): s / (1 + r^2/2)   */
typedef enum { GP_RBF = 0, GP_MATERN32 = 3, GP_MATERN52 = 5, GP_RATQUAD = 7 } gp_kernel_kind;

/* Storage and arithmetic of a problem.
 *   GP_FP64  everything in double (kernel MVMs on the FP64 pipe)
 *   GP_FP32  float vectors, kernel MVMs on CUDA-core FP32 FMAs
 *   GP_TF32  float vectors, kernel-MVM tiles on tcgen05 tensor cores in TF32
 *   GP_BF16  float vectors, kernel-MVM tiles on tcgen05 tensor cores in BF16
 * FP64 is always used for pivot selection, the k x k Woodbury core, the Lanczos
 * tridiagonal eigenproblems and the final sums.                                   */
typedef enum { GP_FP64 = 0, GP_FP32 = 1, GP_TF32 = 2, GP_BF16 = 3 } gp_precision;

typedef struct {
  int64_t n;            /* number of training points                           */
  int32_t d;            /* input dimension                                     */
  int32_t kind;         /* gp_kernel_kind                                      */
  int32_t ard;          /* 1: one lengthscale per dimension (D = d); 0: D = 1  */
  int32_t precision;    /* gp_precision: element type of every real array      */
  const void* X;        /* device, n x d row-major                             */
  const double* theta;  /* device, p = D + 2 values [l_1..l_D, s, sigma^2]     */
} gp_problem;

typedef struct {
  double cg_tol;           /* stop a column when ||r||_2 <= cg_tol ||b||_2        */
  int32_t max_iter;        /* CG iteration cap per column (>= 1)                  */
  int32_t recompute_every; /* r = b - K_hat x every R iterations (0 = never)      */
  uint64_t seed;           /* probe seed (counter-based SplitMix64 hash)          */
  double pivchol_tol;      /* stop pivoted Cholesky when tr(K - LL^T) <= tol tr K */
  int32_t check_every;     /* host polls CG convergence every this many steps (0 = 4) */
  int32_t flags;           /* GP_OPT_* bits (0: defaults)                          */
} gp_opts;

/* gp_opts.flags.  In GP_BF16 precision the kernel product rounds k(r)/s to FP16
 * (11 significant bits).  For smooth kernels with small noise (lambda_max(K) /
 * sigma^2 large) that rounding can make K + sigma^2 I indefinite and CG break down
 * (p^T K_hat p <= 0).  The product then has a split mode that carries k(r)/s as FP16
 * hi + lo (22 bits) at about twice the GEMM2 work.
 *   default           fast mode.  An eager call (stream not being captured) whose
 *                     CG breaks down reruns CG in split mode; otherwise, after the
 *                     evaluation, one product of the CG solutions in each mode gives
 *                     the first-order change of the MLL had the product been in split
 *                     mode (d quad = -u^T D u, d logdet ~ (1/l) sum_i (P^-1 z_i)^T D
 *                     (K^-1 z_i), D = K_split - K_fast); beyond 5e-3 |MLL| (the
 *                     mixed-precision bound; the estimate overstates large changes
 *                     about twofold) the evaluation is repeated in split mode.  The
 *                     estimates are returned in out[GP_OUT_DRIFT_QUAD / _LOGDET].
 *   GP_OPT_SPLIT_P    split mode from the start.
 *   GP_OPT_AUTO_SPLIT choose on the device before CG, from the Gershgorin bound
 *                     lambda_max(K_hat) <= max_i sum_j K_hat_ij (one extra product
 *                     with a vector of ones): split when 2^-11 * bound > 8 sigma^2.
 *                     For graph capture and batched calls, where the host cannot
 *                     rerun CG.  Conservative: some problems it splits would have
 *                     run in fast mode.
 *   GP_OPT_FAST_ONLY  fast mode with neither the rerun nor the check (exactly what
 *                     a graph-recorded evaluation does).                          */
#define GP_OPT_SPLIT_P 1
#define GP_OPT_AUTO_SPLIT 2
#define GP_OPT_FAST_ONLY 4
/* GP_OPT_SIMT_GRAD  in GP_BF16 precision, run the gradient contraction of Alg. 2 on
 *                   CUDA cores in FP32 instead of on the tensor cores (the default
 *                   for d <= 31 and t <= 64; see gp_mll_and_grad).                */
#define GP_OPT_SIMT_GRAD 8

/* Which entry point a workspace query is for. */
typedef enum {
  GP_FN_KERNEL_MVM = 0,
  GP_FN_KERNEL_GRAD_MVM = 1,
  GP_FN_PIVCHOL = 2,
  GP_FN_MBCG = 3,
  GP_FN_MLL_AND_GRAD = 4
} gp_fn;

/* Bytes of workspace entry point `fn` needs for a problem of n points in d
 * dimensions, preconditioner rank k, t right-hand-side columns (for
 * GP_FN_MLL_AND_GRAD: t = n_probes + 1), precision and CG cap max_iter.         */
size_t gp_workspace_size(int32_t fn, int64_t n, int32_t d, int32_t k, int32_t t,
                         int32_t precision, int32_t max_iter);

/* Kernel-matrix block product (the inner operation of CG, Sec. 2.2):
 *   W = (K + sigma^2 I) V,   V, W: n x t column-major (leading dims ldv, ldw).
 * K is never formed: each tile evaluates the kernel and multiplies it into V.
 * W must not alias V.  Asynchronous.                                              */
gp_status gp_kernel_mvm(const gp_problem* prob, const void* V, int64_t ldv, int32_t t,
                        void* W, int64_t ldw, void* ws, size_t ws_bytes,
                        gp_stream_t stream);

/* Derivative products for every hyperparameter (eq. derivative_likelihood needs
 * dK_hat/dtheta):  dW_q = dK_hat/dtheta_q V  for q = 0..p-1 in the order
 * [l_1..l_D, s, sigma^2]; block q starts at element q * ldw * t of dW and is
 * n x t column-major with leading dim ldw.  Asynchronous.                         */
gp_status gp_kernel_grad_mvm(const gp_problem* prob, const void* V, int64_t ldv, int32_t t,
                             void* dW, int64_t ldw, void* ws, size_t ws_bytes,
                             gp_stream_t stream);

/* Greedy rank-k partial pivoted Cholesky of the noise-free K (Prop. "Cholesky
 * approximation quality", after Harbrecht et al. 2012):
 *   pi_m = argmax of the residual diagonal (lowest index on ties, FP64),
 *   L[:, m] = (K[:, pi_m] - L[:, :m] L[pi_m, :m]^T) / sqrt(d_{pi_m}).
 * Stops early when the residual trace <= tol * tr K, or when the best residual
 * <= n u max_i K_ii (u = 2^-24 for FP32, 2^-53 for FP64: LAPACK xPSTRF's default
 * rank rule; below it the residual is rounding error of the earlier columns).
 * Outputs: L (n x k column-major, ld ldl; columns >= rank are zero), piv (k int32,
 * entries >= rank are -1), rank_out (1 int32).  piv_override (device, k int32, or
 * NULL) forces the pivot order; an entry outside [0, n) stops the factor there
 * (pad a shorter order with -1).  Asynchronous.                                   */
gp_status gp_pivchol(const gp_problem* prob, int32_t k, double tol,
                     const int32_t* piv_override, void* L, int64_t ldl, int32_t* piv,
                     int32_t* rank_out, void* ws, size_t ws_bytes, gp_stream_t stream);

/* Preconditioned CG on t right-hand sides at once (footnote to Sec. 4.4) with
 * P_hat = sigma^2 I + L L^T (L: n x k, ld ldl, the first k columns are used):
 *   per column: x_0 = 0, alpha_j = rho_j / p^T K_hat p, beta_j = rho_{j+1} / rho_j,
 *   stop when ||r|| <= cg_tol ||b|| or at max_iter (iters_override: device t int32
 *   caps, or NULL), true residual every recompute_every steps.
 * Outputs: Xsol (n x t, ld ldx) ~ K_hat^-1 B; PinvB (n x t, ld ldx, or NULL) =
 * P_hat^-1 B; the Lanczos tridiagonals from the CG coefficients (Sec. S1.2):
 * T_diag[c * max_iter + j] = 1/alpha_j + beta_{j-1}/alpha_{j-1},
 * T_off[c * max_iter + j] = sqrt(beta_j)/alpha_j; rho0[c] = b^T P^-1 b;
 * iters[c] = steps taken; status (1 int32).  Synchronises with `stream`.         */
gp_status gp_mbcg(const gp_problem* prob, const void* L, int64_t ldl, int32_t k,
                  const void* B, int64_t ldb, int32_t t, const int32_t* iters_override,
                  void* Xsol, int64_t ldx, void* PinvB, double* T_diag, double* T_off,
                  double* rho0, int32_t* iters, int32_t* status, const gp_opts* opts,
                  void* ws, size_t ws_bytes, gp_stream_t stream);

/* Output layout of gp_mll_and_grad (double, device).  p = D + 2, l = n_probes. */
#define GP_OUT_MLL 0      /* estimate of L(theta)                                   */
#define GP_OUT_QUAD 1     /* y^T u, u ~ K_hat^-1 y                                  */
#define GP_OUT_LOGDETP 2  /* log det P_hat (determinant lemma)                      */
#define GP_OUT_STOCH 3    /* (1/l) sum_i gamma_i ~ log det K_hat - log det P_hat    */
#define GP_OUT_LOGDET 4   /* GP_OUT_LOGDETP + GP_OUT_STOCH                          */
#define GP_OUT_DRIFT_QUAD 5   /* mixed fast mode: first-order change of y^T u had the */
#define GP_OUT_DRIFT_LOGDET 6 /* product been in split mode; of log det K_hat (0 if   */
                              /* not evaluated; see GP_OPT_*)                         */
#define GP_OUT_HEAD 8
#define GP_OUT_GRAD(p) (GP_OUT_HEAD)                 /* p entries: dL/dtheta      */
#define GP_OUT_GK(p) (GP_OUT_HEAD + (p))             /* p: 1/2 u^T dK u - (1/2l) sum_i (K^-1 z_i)^T dK (P^-1 z_i) */
#define GP_OUT_PROBEP(p) (GP_OUT_HEAD + 2 * (p))     /* p: (1/l) sum_i (P^-1 z_i)^T dP (P^-1 z_i) */
#define GP_OUT_TRP(p) (GP_OUT_HEAD + 3 * (p))        /* p: tr(P_hat^-1 dP_hat)    */
#define GP_OUT_GAMMA(p) (GP_OUT_HEAD + 4 * (p))      /* l: gamma_i                */
#define GP_OUT_LEN(p, l) (GP_OUT_HEAD + 4 * (p) + (l))
/* Integer output layout (int32, device). t = n_probes + 1.                        */
#define GP_IOUT_STATUS 0
#define GP_IOUT_RANK 1
#define GP_IOUT_ITERS 2                              /* t entries                 */
#define GP_IOUT_PIV(t) (2 + (t))                     /* k entries                 */
#define GP_IOUT_LEN(k, t) (2 + (t) + (k))

/* The whole estimator (Alg. 1 and Alg. 2 in one CG call):
 *   pivoted Cholesky -> Woodbury core and log det P_hat -> probes
 *   z_i = L eps1_i + sigma eps2_i (covariance P_hat) -> CG on [y, z_1..z_l]
 *   -> gamma_i = rho0_i e1^T log(T_i) e1 -> gradient contraction with dK_hat
 *   -> tr(P_hat^-1 dP_hat) (eq. preconditioner_trace) and the probe terms with
 *   dP_hat at frozen pivots -> assembly:
 *   mll = -1/2 (y^T u + log det P_hat + (1/l) sum gamma_i + n log 2 pi)
 *   grad = GK + 1/2 PROBEP - 1/2 TRP.
 * y: n reals.  eps_override (device, (k + n) x n_probes int8 +-1 column-major with
 * leading dim k + n: rows 0..k-1 eps1, rows k.. eps2; or NULL = SplitMix64 from
 * opts->seed), piv_override (k int32 or NULL; -1 entries stop the factor),
 * iters_override (t int32 or NULL) exist for parity testing.
 * out: GP_OUT_LEN(p, n_probes) doubles; iout: GP_IOUT_LEN(k, t) int32.
 * Synchronises with `stream`, except while `stream` is being captured into a CUDA
 * graph: then nothing is read back, mBCG's iteration
 * loop is recorded as a conditional WHILE node (the stopping rule is evaluated on
 * the device), the call returns GP_OK, and the status of the evaluation is
 * iout[GP_IOUT_STATUS] once the graph has run.                                   */
gp_status gp_mll_and_grad(const gp_problem* prob, const void* y, int32_t k,
                          int32_t n_probes, const int8_t* eps_override,
                          const int32_t* piv_override, const int32_t* iters_override,
                          double* out, int32_t* iout, const gp_opts* opts, void* ws,
                          size_t ws_bytes, gp_stream_t stream);

/* The same estimator with a random Fourier feature preconditioner in place of the
 * partial Cholesky factor (Tab. 2 "RFF"; Prop. "RFF approximation quality", after
 * Rahimi and Recht 2007): P_hat = sigma^2 I + Phi Phi^T with k = 2m features
 *   Phi[a, j] = sqrt(s/m) cos(u_j . x~_a),  Phi[a, m + j] = sqrt(s/m) sin(u_j . x~_a),
 * x~ = (x - mean x) / l (elementwise for ARD; the inputs' mean as the origin, which
 * leaves P_hat unchanged and fixes the probes), u_j = rho_j eps_j drawn from the
 * kernel's spectral density: RBF rho = 1; Matern-3/2 and -5/2 rho = sqrt(nu / g_j)
 * with g_j ~ Gamma(nu, 1);
 * rational quadratic (alpha = 1) rho = sqrt(g_j) with g_j ~ Gamma(1, 1).
 * eps: device, m x d doubles (row-major), standard-normal draws; g: device, m doubles
 * (may be NULL for the RBF).  The gradient's preconditioner terms take dP_hat at these
 * frozen draws.  Everything else (probes with k = 2m, mBCG, quadrature, contraction,
 * outputs, iout with rank = 2m and pivots -1, statuses, synchronisation) is as for
 * gp_mll_and_grad with k = 2m; the workspace is gp_workspace_size(GP_FN_MLL_AND_GRAD,
 * n, d, 2m, n_probes + 1, ...).  Requires 1 <= m and 2m <= min(n, the largest k).     */
gp_status gp_mll_and_grad_rff(const gp_problem* prob, const void* y, int32_t m,
                              int32_t n_probes, const double* eps, const double* g,
                              const int8_t* eps_override, const int32_t* iters_override,
                              double* out, int32_t* iout, const gp_opts* opts, void* ws,
                              size_t ws_bytes, gp_stream_t stream);

/* The same estimator with the quadrature Fourier feature preconditioner of Tab. 2
 * ("QFF"; Prop. "QFF approximation quality", after Mutny and Krause 2018), RBF kernel
 * only: E_w[cos(w . D)], w ~ N(0, I_d), by the tensor-product Gauss-Hermite rule of
 * mbar nodes per dimension (mbar even), each pair w, -w kept once with twice the weight:
 * m = mbar^d / 2 frequencies u_j (multi-indices in row-major order over ascending
 * nodes, the one with a positive first coordinate kept) with weights w_j, and k =
 * mbar^d features sqrt(s w_j) cos(u_j . x~), sqrt(s w_j) sin(u_j . x~), x~ = (x - mean
 * x) / l.  The rule is computed on the host and copied in; the call synchronises with
 * `stream` and cannot be captured into a graph.  Outputs, statuses and workspace as
 * for gp_mll_and_grad with k = mbar^d (<= min(n, the largest k)).                    */
gp_status gp_mll_and_grad_qff(const gp_problem* prob, const void* y, int32_t mbar,
                              int32_t n_probes, const int8_t* eps_override,
                              const int32_t* iters_override, double* out, int32_t* iout,
                              const gp_opts* opts, void* ws, size_t ws_bytes,
                              gp_stream_t stream);

/* The quadrature rule of gp_mll_and_grad_qff, on the host: writes the m = mbar^d / 2
 * frequencies (U, m x d doubles, row-major; NULL to skip) and their weights (W, m
 * doubles; NULL to skip) and returns m, or a negative gp_status (mbar odd or < 2, d out
 * of range, mbar^d > 4096).                                                          */
int32_t gp_qff_rule(int32_t mbar, int32_t d, double* U, double* W);

/* Batched estimator: n_problems independent problems (each its own n, d, X,
 * hyperparameters and precision; shared k, n_probes and opts; problem i draws its
 * probes from seed opts->seed + i).  The per-probe loops of Alg. 1 and Alg. 2 are
 * independent (the footnote to Sec. 4.4 batches them into one CG call); independent
 * problems are one more level of the same parallelism.  probs: host array; ys, outs,
 * iouts: host arrays of device pointers (per problem: n reals, GP_OUT_LEN(p_i,
 * n_probes) doubles, GP_IOUT_LEN(k, n_probes + 1) int32).  ws: device, at least
 * gp_workspace_size_batched(...) bytes, 256-byte aligned; problem i uses its own
 * slice, so results equal those of gp_mll_and_grad on that slice.
 * Execution: the problems run concurrently on up to 8 worker streams (largest
 * first, to the least-loaded worker), recorded as one CUDA graph with device-side
 * CG loops; the instantiated graph is cached per argument set (pointers, sizes,
 * options; up to 4 per host thread), so repeating a call with new values in the
 * same buffers is a single graph launch.  If `stream` is being captured, the batch
 * is recorded into the caller's graph instead.  Asynchronous: returns after the
 * launch; per-problem statuses are iouts[i][GP_IOUT_STATUS] once `stream` reaches
 * that point.  Host-side validation errors return before anything is launched.   */
size_t gp_workspace_size_batched(int32_t n_problems, const gp_problem* probs, int32_t k,
                                 int32_t n_probes, int32_t max_iter);
gp_status gp_mll_and_grad_batched(int32_t n_problems, const gp_problem* probs,
                                  const void* const* ys, int32_t k, int32_t n_probes,
                                  double* const* outs, int32_t* const* iouts,
                                  const gp_opts* opts, void* ws, size_t ws_bytes,
                                  gp_stream_t stream);

/* Autotuner of the tensor-core product's launch configuration (GP_BF16): times the
 * candidate column-chunk counts (work units per 128-row tile: 1..24, capped so every
 * chunk keeps >= 4 tiles and the units stay <= ~16 per SM) and B / V shared-memory
 * ring depths (4/4, 3/3, 2/2) on this problem with right-hand sides V (n x t,
 * column-major, ld ldv), one warm-up and three timed products each, and records the
 * fastest in a process-wide table keyed by (exponent operand width, t padded to 16,
 * kernel kind, ceil(log2(n / 128))).  Every later product of a matching shape uses it;
 * untuned shapes use the built-in heuristic.  W receives (K + sigma^2 I) V from the
 * chosen configuration.  Workspace: that of GP_FN_KERNEL_MVM.  best (host, 4 int32,
 * may be NULL): {chunks, B ring, V ring, candidates timed}.  Synchronises.  The
 * paper has no counterpart (its products are whatever the GPU library picks).      */
gp_status gp_autotune(const gp_problem* prob, const void* V, int64_t ldv, int32_t t,
                      void* W, int64_t ldw, void* ws, size_t ws_bytes, gp_stream_t stream,
                      int32_t* best);
/* The launch configuration the product uses for this shape (host, 4 int32):
 * {chunks, B ring, V ring, 1 if from the autotuner else 0}.  Host only.           */
gp_status gp_tc_config(const gp_problem* prob, int32_t t, int32_t* config);

/* Human-readable name of a status code (static storage). */
const char* gp_status_string(int32_t status);

/* Detail of the last host-side validation failure on this thread (static storage). */
const char* gp_last_error_message(void);

/* The kernel-matrix product of gp_kernel_mvm, W = (K + sigma^2 I) V, for callers that
 * cannot allocate device memory.  Such callers include:
 *   - real-time loops with a fixed memory budget, where a device allocation (or the
 *     synchronisation it can cause) is not allowed once the loop runs;
 *   - host frameworks that own the allocator and hand the library only its input and
 *     output buffers, with no room for a workspace of the library's own.
 * The paper has no counterpart: this repackages gp_kernel_mvm without a workspace.
 *
 * Scratch.  One static device array of 16 MiB + 80 KiB inside this library.  Every
 * GPU that loads the library holds it until the process exits.  Every call reuses
 * it and leaves its contents behind, so calls that overlap on the GPU (two streams,
 * or two host threads) race on it; the caller must serialise them.
 *
 * First call.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current.  Make that first call before
 * any stream capture.
 *
 * Limits.  Precision GP_FP32 or GP_FP64, and n * d * sizeof(real) <= 16 MiB (for
 * example n <= 131072 at d = 32 in FP32).  Larger problems are rejected with
 * GP_ERR_INVALID_ARG before anything runs.
 *
 * Calls no cudaMalloc, cudaFree or allocating library routine.  Otherwise behaves
 * like gp_kernel_mvm.  Asynchronous.                                               */
gp_status gp_kernel_mvm_noalloc(const gp_problem* prob, const void* V, int64_t ldv, int32_t t,
                                void* W, int64_t ldw, gp_stream_t stream);

/* Diagnostic for the tensor-core product (precision GP_BF16): computes W exactly
 * as gp_kernel_mvm does and also copies the FP32 exponent tile S of the first
 * 128 x 128 (row, column) tile pair to S_out (device, 128 x 128 row-major):
 * S_ij = log2(e) (-r_ij^2 / 2) + log2(s) for RBF, -r_ij^2 / 2 for Matern.  The
 * workspace is that of GP_FN_KERNEL_MVM.  Asynchronous.                          */
gp_status gp_tc_exponent_tile(const gp_problem* prob, const void* V, int64_t ldv, int32_t t,
                              void* W, int64_t ldw, float* S_out, void* ws, size_t ws_bytes,
                              gp_stream_t stream);

/* Instrumentation.  gp_launch_count: kernels this library has launched since it
 * was loaded (host-side count of launch sites).  gp_mvm_timing(1) makes the CG
 * loop of gp_mbcg / gp_mll_and_grad bracket every kernel-matrix product with CUDA
 * events on the caller's stream; gp_mvm_timing_read returns (and resets) their
 * summed duration in ms and the number of products timed.                        */
int64_t gp_launch_count(void);
void gp_mvm_timing(int32_t enable);
gp_status gp_mvm_timing_read(double* total_ms, int64_t* products);
/* The same timing for a phase of gp_mll_and_grad / gp_mbcg: phase 0 = the
 * kernel-matrix products (as gp_mvm_timing_read), phase 1 = the gradient contraction
 * of Alg. 2 (one bracket per evaluation), phase 2 = the work of a CG iteration outside
 * its products (two brackets per iteration: the alpha / update step, then the
 * preconditioner solve and the direction update; eager calls only).  Returns (and
 * resets) the summed duration in ms and the number of brackets.                    */
gp_status gp_phase_timing_read(int32_t phase, double* total_ms, int64_t* count);

/* Throughput microbenchmarks of the arithmetic units the path uses (roofline
 * denominators beside the measured copy bandwidth and BF16 GEMM rate):
 *   out[0] FP32 FMA FLOP/s, out[1] ex2.approx.f32 results/s (MUFU),
 *   out[2] ex2.approx.f16x2 results/s (two per instruction), out[3] FP64 FMA FLOP/s.
 * Each kernel runs independent dependency chains, 8 CTAs of 256 threads per SM,
 * timed with CUDA events on `stream` (best of three after a warm-up launch).
 * scratch: device, at least gp_peaks_scratch_elems() floats, overwritten.  out: host,
 * 4 doubles.  Synchronous: returns after the timings (about 0.2 s).               */
size_t gp_peaks_scratch_elems(void);
gp_status gp_measure_peaks(float* scratch, double* out, gp_stream_t stream);

/* Rademacher signs of the probe generator, for inspection:
 * out[c * rows + r] = +-1 for stream 1 (eps1) or 2 (eps2).  Asynchronous.         */
gp_status gp_rademacher(uint64_t seed, int32_t stream_id, int64_t rows, int32_t cols,
                        int8_t* out, gp_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* GP_H */
