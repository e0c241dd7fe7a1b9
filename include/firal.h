/*
 * firal.h -- C-ABI of the GB300 (sm_103a) Approx-FIRAL hot path.
 *
 * Approx-FIRAL (Chen, Wen, Biros, "A Scalable Algorithm for Active Learning",
 * SC24) selects b points of an unlabelled pool for labelling under a
 * multinomial logistic-regression model.  This library implements its
 * data-parallel hot path on one GPU:
 *
 *   Relax (Algorithm 2): entropic mirror descent on
 *        f(z) = Tr(Sigma_z^{-1} H_p),   Sigma_z = H_o + sum_i z_i H_i     (eqs. 4-7)
 *     with Hutchinson probes (eq. 11), the matrix-free Hessian apply of
 *     Lemma 1, and block-Jacobi preconditioned CG (Definition 1, eq. 13).
 *   Round (Algorithm 3): greedy block-diagonal FTRL selection with the
 *     Proposition 1 score (eq. 14), Lemma 2 updates and the eq. 10 root.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Pointers named "device" must point to device memory of the handle's
 *    device; "host" pointers to host memory.  The caller owns every buffer it
 *    passes; the library never frees caller memory.  The library allocates its
 *    own workspace (cudaMalloc) inside a handle or problem and frees it in the
 *    matching destroy call.
 *  - All device work is enqueued on the handle's stream.  Calls return after
 *    enqueueing unless they fill a host output (stats, histories, scalars), in
 *    which case they synchronise the stream first.
 *  - Matrices are row-major.  A vector of length dt = d*c is vec(V) of a d x c
 *    matrix (columns stacked, as in the paper's notation table): element
 *    k*d + e is V[e][k].  A block of s such vectors is stored probe-major:
 *    vector j occupies [j*dt, (j+1)*dt).
 *  - "vec type" is double for FIRAL_FP64 and float for FIRAL_FP32 and
 *    FIRAL_MIXED_BF16; z, probe blocks, CG iterates and gradients use it.
 *  - The status code is the only error channel; no exception crosses the ABI.
 *    After an error, firal_last_error() gives a one-line detail.  A CUDA
 *    error maps to FIRAL_ERR_CUDA; a non-positive Cholesky pivot to
 *    FIRAL_ERR_NOT_SPD (the outputs then hold the best values reached).
 *  - H_o = sum_{labelled} H_i + lambda I (full c-class softmax, d~ = dc);
 *    H_p = (1/n) sum_{pool} H_i (the pool average).
 */
#ifndef FIRAL_H
#define FIRAL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FIRAL_OK = 0,
  FIRAL_ERR_ARG = -1,              /* invalid argument (null pointer, bad size or dtype)      */
  FIRAL_ERR_CUDA = -2,             /* a CUDA runtime or driver call failed                    */
  FIRAL_ERR_NOT_SPD = -3,          /* a block Cholesky met a non-positive pivot              */
  FIRAL_ERR_CG_NOT_CONVERGED = -4, /* PCG hit its iteration limit above tolerance           */
  FIRAL_ERR_NONFINITE = -5,        /* NaN or Inf in the objective or gradient               */
  FIRAL_ERR_TIMEOUT = -6,          /* a bounded device-side wait gave up                      */
  FIRAL_ERR_NOMEM = -7,            /* workspace allocation failed                             */
  FIRAL_ERR_UNSUPPORTED = -8,      /* shape or precision the library does not support       */
  FIRAL_ERR_COMM = -9              /* the allreduce callback of a row-sharded problem failed */
} firal_status;

typedef enum {
  FIRAL_FP64 = 0,       /* every step in double (SIMT kernels)                                  */
  FIRAL_FP32 = 1,       /* contractions and vectors in float (SIMT); FP64 dots and factors       */
  FIRAL_MIXED_BF16 = 2, /* X, h contractions on bf16 tensor cores (tcgen05), FP32 accumulate;   */
                        /* float vectors, FP64 dots, FP64 block factorisations; the CG direction */
                        /* enters the contraction as bf16 hi + lo (about 2^-17 relative)         */
  FIRAL_MIXED_BF16_FAST = 3  /* as FIRAL_MIXED_BF16, but the CG direction enters the first      */
                        /* contraction of the Hessian apply as one bf16 operand (2^-9 relative   */
                        /* rounding of the low-rank term), which halves that contraction's       */
                        /* tensor work, and the diagonal-part block sums over the pool rows take */
                        /* their weights and the products x_e x_e' as one bf16 operand each      */
                        /* (per-element 2^-9 roundings that average over each class's points;   */
                        /* one product instead of three; labelled rows stay exact);              */
                        /* a problem whose rows' mean sum_k h_ik^2 exceeds 0.1 (confident or     */
                        /* few classes: the low-rank term is large) keeps hi + lo for both; with */
                        /* at most 32 classes per pool both modes run the same fused kernels     */
} firal_precision;

typedef enum { FIRAL_DT_F64 = 0, FIRAL_DT_F32 = 1, FIRAL_DT_BF16 = 2 } firal_dtype;

/* The unlabelled pool X_u: embeddings x_i (n x d) and class probabilities h_i (n x c),
 * device pointers, row-major, rows contiguous.  h rows are used as given (not renormalised). */
typedef struct {
  const void* X;     /* device, n*d elements of x_dtype                      */
  const void* h;     /* device, n*c elements of h_dtype (F32 or F64)         */
  int64_t n;         /* pool size, >= 1                                      */
  int32_t d;         /* feature dimension, 1..128                            */
  int32_t c;         /* classes, 2..4096                                     */
  int32_t x_dtype;   /* firal_dtype                                          */
  int32_t h_dtype;   /* firal_dtype (F32 or F64)                             */
} firal_pool;

/* The labelled set X_o that defines H_o (eq. 3) plus the ridge lambda (same dtypes as the pool). */
typedef struct {
  const void* Xo;    /* device, m*d, may be NULL when m == 0 */
  const void* ho;    /* device, m*c                          */
  int64_t m;         /* labelled points, >= 0                */
  double lambda;     /* ridge, > 0 unless the labelled Hessians alone are SPD */
} firal_hess0;

/* Preconditioned CG controls (Algorithm 2 lines 5-8).  x0 = 0; column j stops when its
 * recursive residual satisfies ||r_j|| <= tol ||b_j|| (unpreconditioned 2-norm) or when
 * p^T Sigma p <= 0.  fixed_iters > 0 runs exactly that many iterations on every column and
 * ignores tol (no host synchronisation inside the solve). */
typedef struct {
  double tol;           /* default 0.1 (Section 5 of the paper)  */
  int32_t maxit;        /* default 100                           */
  int32_t fixed_iters;  /* 0 = tolerance mode                    */
  int32_t block;        /* 0 (default): s independent PCG recurrences sharing each matvec;   */
                        /* 1: block PCG (O'Leary 1980), s x s step matrices in FP64 (s <= 32, */
                        /*    not for pooled problems); the solve stops when every column     */
                        /*    meets the tolerance, or early if the s x s system loses rank    */
  int32_t reserved;     /* 0                                                                  */
} firal_cg_opts;

/* Relax controls.  Defaults: s = 10, T = 20, beta0 = 1, seed = 1, cg = {0.1, 100, 0}. */
typedef struct {
  int32_t s;            /* Hutchinson probes per MD iteration (eq. 11)                        */
  int32_t T;            /* mirror-descent iterations                                          */
  firal_cg_opts cg;     /* both CG solves of an iteration                                     */
  double beta0;         /* step size beta_t = beta0 / ||g_t||_inf                              */
  uint64_t seed;        /* probe seed: v[t][j][q] from SplitMix64 (see firal_probes)          */
  int32_t precision;    /* firal_precision                                                    */
  int32_t estimator;    /* 0 = paper eq. 11 (W = S^-1 H_p S^-1 V); 1 = derivative of f^ (U,Y) */
  double md_tol;        /* > 0: stop when |f^_t - f^_{t-1}| <= md_tol |f^_{t-1}| (Section 5)  */
} firal_relax_opts;

/* Per-iteration record of a relax step (host). */
typedef struct {
  double fhat;          /* (1/s) sum_j <v_j, H_p Sigma_z^{-1} v_j> before the z update        */
  double gmax;          /* ||g||_inf                                                           */
  double zmax;          /* max_i z_i after the update (the box z <= 1 is not enforced)        */
  int32_t cg_iters[2];  /* iterations of the two solves (max over columns)                    */
  double cg_relres[2];  /* largest final relative residual over columns                        */
} firal_step_stats;

typedef struct {
  int32_t iters_done;   /* MD iterations run                                                   */
  double fhat_last;
  int32_t cg_iters_total;
} firal_relax_stats;

/* Round controls.  eta <= 0 selects eta = 8 sqrt(d c) (Theorem 1 with epsilon = 1). */
typedef struct {
  double eta;
  int32_t exclude_selected;  /* 1 (default): never select a point twice                       */
  int32_t precision;         /* firal_precision of the score contraction                      */
} firal_round_opts;

typedef struct {
  double nu_last;       /* nu_{b+1} of eq. 10                                                  */
  double score_last;    /* eq. 14 score of the last pick                                       */
} firal_round_stats;

typedef struct firal_handle firal_handle;
typedef struct firal_problem firal_problem;

/* ---------------------------------------------------------------- library and handles */

/* Human-readable name of a status code (static string). */
const char* firal_status_string(int32_t status);

/* Create a handle bound to the current CUDA device and to `stream` (a cudaStream_t passed
 * as void*; NULL = the legacy default stream).  *out receives the handle. */
int32_t firal_create(firal_handle** out, void* stream);

/* Destroy a handle (NULL is ignored).  Problems created from it must be destroyed first. */
int32_t firal_destroy(firal_handle* handle);

/* Rebind the handle (and its problems) to another stream of the same device. */
int32_t firal_set_stream(firal_handle* handle, void* stream);

/* Copy the last error detail of `handle` (NUL-terminated, truncated to len). */
int32_t firal_last_error(firal_handle* handle, char* buf, size_t len);

/* Bit-width and precision flags the library was compiled with: bit 0 = SIMT paths,
 * bit 1 = tcgen05 (sm_103a) tensor-core path. */
int32_t firal_build_info(void);

/* ---------------------------------------------------------------- instrumentation */

/* Number of kernels this library has launched in the process so far (all handles). */
int64_t firal_launch_count(void);

/* Enable (1) or disable (0) the kernel-class timers and reset their totals.  When enabled,
 * each group of launches records a CUDA event pair on the stream it is launched on; the
 * timers add that overhead and nothing else.  Not thread-safe across concurrent calls that
 * use different streams of different devices. */
int32_t firal_profile(int32_t enable);

/* Synchronise on the recorded events and copy, for each kernel class 0..count-1, the total
 * elapsed milliseconds (ms_out, host, may be NULL) and the number of timed groups
 * (calls_out, host, may be NULL).  Returns the number of kernel classes. */
int32_t firal_profile_read(double* ms_out, int64_t* calls_out, int32_t count);

/* Name of kernel class `id` (static string). */
const char* firal_profile_name(int32_t id);

/* ---------------------------------------------------------------- prepared problems */

/* Prepare one problem for repeated calls: copies the pool and labelled set into the
 * library's device layout for `precision` (labelled rows first, then pool rows; bf16 and
 * transposed copies for FIRAL_MIXED_BF16) and allocates the iteration workspace.  The
 * caller's X, h, Xo, ho may be freed after this call returns. */
int32_t firal_problem_create(firal_handle* handle, const firal_pool* pool,
                             const firal_hess0* hess0, int32_t precision,
                             firal_problem** out);
int32_t firal_problem_destroy(firal_problem* problem);

/* ---------------------------------------------------------------- Relax (Algorithm 2) */

/* Full Relax solve.  With opts->cg.fixed_iters > 0, no history or stats requested and
 * md_tol = 0, iterations 1..T-1 are replayed from a CUDA graph (captured on an internal
 * stream ordered after the handle's stream).
 * z0: device, n values of the vec type on the budget simplex
 * (z >= 0, sum z = budget) or NULL for z0 = budget/n.  z_out: device, n values; it holds
 * z_diamond on return (the iterates stay on the budget simplex, so no final rescale).
 * fhat_hist: host, opts->T doubles or NULL.  stats: host or NULL. */
int32_t firal_relax(firal_handle* handle, const firal_pool* pool, const firal_hess0* hess0,
                    double budget, const void* z0, const firal_relax_opts* opts, void* z_out,
                    double* fhat_hist, firal_relax_stats* stats);

/* Relax for many independent pools at once (the batched workload; one problem per pool, each
 * with its own budget).  pools, hess0s (may be NULL: no labelled set, lambda = 0), budgets and
 * z_outs have nproblems entries; z_outs[p] is a device buffer of pools[p].n values of the vec
 * type and receives that problem's z_diamond (iterates start at budget/n).  All problems use
 * *opts.  With opts->cg.fixed_iters > 0, iteration 0 runs
 * eagerly and one batched iteration is captured into a CUDA graph (problems spread over up
 * to 64 internal streams) and replayed T-1 times; otherwise the iterations run eagerly.
 * Synchronises before returning. */
int32_t firal_batched_relax(firal_handle* handle, int32_t nproblems, const firal_pool* pools,
                            const firal_hess0* hess0s, const double* budgets,
                            const firal_relax_opts* opts, void* const* z_outs);

/* One mirror-descent iteration t (0-based) of Algorithm 2 on a prepared problem:
 * probes V_t (line 4), preconditioner B(Sigma_z)^{-1} (line 5), U = Sigma_z^{-1} V (line 6),
 * H_p U and f^ (line 7), the second solve (line 8), the gradient (line 9) and the MD update
 * (lines 10-11).  z: device, n values, updated in place.  stats: host or NULL (NULL keeps
 * the call free of host synchronisation when opts->cg.fixed_iters > 0). */
int32_t firal_relax_step(firal_problem* problem, const firal_relax_opts* opts, int32_t t,
                         double budget, void* z, firal_step_stats* stats);

/* ---------------------------------------------------------------- Round (Algorithm 3) */

/* Diagonal Round step: selects `budget` pool indices (0-based) into selected_out (device,
 * int32, budget entries), in selection order.  z_relaxed: device, n values of the vec type
 * (z_diamond).  Ties in eq. 14 go to the lowest index. */
int32_t firal_round(firal_handle* handle, const firal_pool* pool, const firal_hess0* hess0,
                    const void* z_relaxed, int32_t budget, const firal_round_opts* opts,
                    int32_t* selected_out, firal_round_stats* stats);

/* Same on a prepared problem (its precision governs the score contraction). */
int32_t firal_round_problem(firal_problem* problem, const void* z_relaxed, int32_t budget,
                            const firal_round_opts* opts, int32_t* selected_out,
                            firal_round_stats* stats);

/* Choosing eta for Round (Section 5 of the paper): Algorithm 3 is run once per eta_e,
 * e < n_eta, from the same z_relaxed, and eta_e is scored by
 *   criterion_e = min_k lambda_min(H_k),  H_k = sum_{i selected} h_ik (1 - h_ik) x_i x_i^T
 * (the block-diagonal Hessian sum of the b selected points).  selected_out (device,
 * n_eta * budget int32, row e = the picks for eta_e), criteria (host, n_eta doubles) and
 * *best (host: the index maximising the criterion, first on ties) are written.
 * 1 <= n_eta <= 64; every eta_e must be > 0; opts->eta is ignored.  Errors as firal_round. */
int32_t firal_round_sweep(firal_problem* problem, const void* z_relaxed, int32_t budget,
                          const double* etas, int32_t n_eta, const firal_round_opts* opts,
                          int32_t* selected_out, double* criteria, int32_t* best);

/* ---------------------------------------------------------------- building blocks */

/* Rademacher probe block of MD iteration t (Algorithm 2 line 4): V_out (device, s*dt of
 * the vec type, probe-major) with v[t][j][q] = +1 if the top bit of
 * splitmix64(seed ^ splitmix64((t*s + j)*dt + q)) is 0, else -1, where splitmix64(x) is
 * the SplitMix64 output for state x (Steele, Lea, Flood 2014). */
int32_t firal_probes(firal_problem* problem, uint64_t seed, int32_t t, int32_t s,
                     void* V_out);

/* Hessian apply by Lemma 1 (Section 3.1) on s vectors: op 0 gives Sigma_z V
 * = H_o V + sum_pool z_i H_i V (z: device, n values); op 1 gives H_p V (z ignored).
 * V, out: device, s*dt of the vec type, probe-major; out must not alias V. */
int32_t firal_hessian_apply(firal_problem* problem, int32_t op, const void* z, const void* V,
                            int32_t s, void* out);

/* Preconditioner blocks B_k(Sigma_z) = B_k(H_o) + sum_pool z_i h_ik (1 - h_ik) x_i x_i^T
 * (Definition 1, eq. 13), k = 0..c-1: blocks_out (device, c*d*d doubles, block k row-major).
 * z == NULL gives B_k(H_o). */
int32_t firal_precond_blocks(firal_problem* problem, const void* z, double* blocks_out);

/* Block-Jacobi preconditioned CG on Sigma_z X = B (Algorithm 2 lines 5-8) for s columns.
 * B, X_out: device, s*dt of the vec type.  iters_out (host, s int32) and relres_out (host,
 * s doubles) may be NULL; when either is given the call synchronises.  Returns
 * FIRAL_ERR_CG_NOT_CONVERGED (with X_out filled) if a column stayed above tol in tolerance
 * mode. */
int32_t firal_pcg(firal_problem* problem, const void* z, const void* B, int32_t s,
                  const firal_cg_opts* cg, void* X_out, int32_t* iters_out,
                  double* relres_out);

/* Per-point quadratic forms g_i = -(scale/s) sum_j a_j^T H_i b_j for the n pool points
 * (eq. 11 with a = v, b = w; the autograd backward with a = u, b = y).  A, B: device,
 * s*dt of the vec type; g_out: device, n values of the vec type. */
int32_t firal_quad_forms(firal_problem* problem, const void* A, const void* B, int32_t s,
                         double scale, void* g_out);

/* Mirror-descent update (Algorithm 2 lines 10-11) on the budget simplex:
 * z <- z exp(-beta g), z <- budget z / sum(z), beta = beta0 / ||g||_inf.  z, g: device,
 * n values of the vec type; z updated in place. */
int32_t firal_md_step(firal_problem* problem, void* z, const void* g, double budget,
                      double beta0);

/* Allocation-free mirror-descent update (the paper has no counterpart; it exists for callers
 * that cannot allocate device memory: code running while a CUDA graph is captured, servers and
 * embedded runtimes that give all device memory to their own pool at start-up, and plug-in
 * hosts that forbid a library from growing its footprint).  Computes what firal_md_step does
 * -- z <- z exp(-beta g), z <- budget z / sum(z), beta = beta0/||g||_inf -- without a problem
 * handle and without calling cudaMalloc, cudaFree or any allocating routine.
 * z (in/out) and g: device, n values of dtype (FIRAL_DT_F32 or FIRAL_DT_F64).  stream: a
 * cudaStream_t as void* (NULL = legacy default stream).  Returns after enqueueing 5 kernels.
 * Scratch: a fixed array of 64 KiB + 64 bytes in the library, resident on every GPU that loads
 * it until the process exits; it limits n to 16,777,216 (larger n returns FIRAL_ERR_ARG).
 * Each call looks up that array's device address (cudaGetSymbolAddress, which allocates
 * nothing) with the current device; the first lookup on a device may load the library's device
 * code there, so make the first call on each device before any stream capture.  All calls share
 * the array and it keeps the last call's values (nothing in it needs clearing: every slot a
 * call reads is written by the same call), so calls whose kernels overlap on the GPU race and
 * must be ordered by the caller.  If ||g||_inf is NaN or infinite (or the updated z has no
 * positive finite sum) the kernels leave z unchanged; the status, returned before the kernels
 * run, cannot report that case, so check g where it may not be finite. */
int32_t firal_md_step_static(void* z, const void* g, int64_t n, int32_t dtype, double budget,
                             double beta0, void* stream);

/* Objective forward for the autograd Function: with probes V_t(seed, t), U = Sigma_z^{-1} V
 * and Y = Sigma_z^{-1} H_p V (one 2s-column PCG), f^ = (1/s) sum_j <H_p v_j, u_j>.
 * fhat_out: host double (the call synchronises).  U_out, Y_out: device, s*dt each (may be
 * NULL to discard; the backward can recompute them). */
int32_t firal_objective_fwd(firal_problem* problem, const void* z, uint64_t seed, int32_t t,
                            int32_t s, const firal_cg_opts* cg, double* fhat_out,
                            void* U_out, void* Y_out);

/* Objective backward: g_out = grad_out * d f^/d z_i = -(grad_out/s) sum_j u_j^T H_i y_j
 * (the exact derivative of f^ for fixed probes).  U, Y: device, from the forward; pass NULL
 * for both to recompute them with the forward's (z, seed, t, s, cg). */
int32_t firal_objective_bwd(firal_problem* problem, const void* z, uint64_t seed, int32_t t,
                            int32_t s, const firal_cg_opts* cg, const void* U, const void* Y,
                            double grad_out, void* g_out);

/* Eigenvalues of L_k^{-1} H_k L_k^{-T} for c blocks (Algorithm 3 line 9), FP64 Householder
 * tridiagonalisation and Sturm bisection.  Sig, H: device, c*d*d doubles (Sig_k SPD; L_k its
 * Cholesky factor); eig_out: device, c*d doubles, ascending per block. */
int32_t firal_block_eigvals(firal_handle* handle, int32_t c, int32_t d, const double* Sig,
                            const double* H, double* eig_out);

/* Root of sum_j (nu + mu_j)^{-2} = 1 (eq. 10, Algorithm 3 line 10) for count values
 * mu (device doubles); nu_out: host double (synchronises). */
int32_t firal_nu_bisect(firal_handle* handle, const double* mu, int64_t count, double* nu_out);

/* ---------------------------------------------------------------- Exact-FIRAL (Algorithm 1) */

/* Exact-FIRAL on dense d~ x d~ matrices (d~ = d c <= 16384), for pools small enough to form
 * Sigma_z.  Runs on a prepared, non-pooled problem in its vec type (FIRAL_FP64: double, every
 * other precision: float; the tile factorisations, the Round's c x c systems and all scalar
 * reductions use double).  Device workspace: up to 12 d~ x d~ matrices of the vec type,
 * allocated on first use and kept with the problem.  Errors: FIRAL_ERR_UNSUPPORTED for pooled
 * problems or d~ > 16384, FIRAL_ERR_NOT_SPD when Sigma_z (or a Round matrix) has no Cholesky
 * factor, FIRAL_ERR_NONFINITE for a non-finite objective or score. */

/* Objective and exact gradient (Section 2, eqs. 4-7; Algorithm 1 lines 5-6):
 * f = Tr(Sigma_z^{-1} H_p) with Sigma_z = H_o + sum_pool z_i H_i, and
 * g_i = -Tr(H_i Sigma_z^{-1} H_p Sigma_z^{-1}) for the n pool points.
 * z: device, n values of the vec type.  f_out: host double (the call synchronises), may be
 * NULL.  g_out: device, n values of the vec type, or NULL to skip the gradient. */
int32_t firal_exact_objective(firal_problem* problem, const void* z, double* f_out,
                              void* g_out);

/* Exact Relax (Algorithm 1 lines 2-10): T mirror-descent steps z <- z exp(-beta_t g),
 * z <- budget z / sum(z), beta_t = beta0 / ||g||_inf, with the exact gradient.
 * z0: device, n values on the budget simplex, or NULL for budget / n (may equal z_out).
 * z_out: device, n values; holds z_diamond on return.  f_hist: host, T doubles (f before each
 * step) or NULL.  Synchronises before returning. */
int32_t firal_exact_relax(firal_problem* problem, double budget, int32_t T, double beta0,
                          const void* z0, void* z_out, double* f_hist);

/* Exact Round (Algorithm 1 lines 11-20; eqs. 8-10) on the full Hessians: budget picks of
 *   i_t = argmin_i Tr[(A_t + (eta/b) H~_o + eta H~_i)^{-1}],  A_1 = sqrt(d~) I,
 *   A_{t+1} = nu_{t+1} I + eta H~_t,  H~_t = sum_{s <= t} (H~_o / b + H~_{i_s}),
 * with nu_{t+1} the root of sum_j (nu + lambda_j(eta H~_t))^{-2} = 1 and X~ = Sigma^{-1/2} X
 * Sigma^{-1/2}, Sigma = H_o + H_{z_relaxed}.  eta <= 0 selects 8 sqrt(d~).  c <= 112.
 * z_relaxed: device, n values of the vec type.  selected_out: device, budget int32 pool
 * indices in selection order (ties to the lowest index; exclude_selected != 0 never picks a
 * point twice).  r_out: host, budget doubles (the minimised trace of each pick) or NULL.
 * nu_out: host, budget doubles (nu_t used for pick t; nu_1 = sqrt(d~)) or NULL.
 * Synchronises before returning. */
int32_t firal_exact_round(firal_problem* problem, const void* z_relaxed, int32_t budget,
                          double eta, int32_t exclude_selected, int32_t* selected_out,
                          double* r_out, double* nu_out);

/* ---------------------------------------------------------------- device memory */

/* Destroyed problems park their device buffers in a process-wide cache (bounded by the
 * FIRAL_CACHE_BYTES environment variable, default 64 GiB; 0 disables it), from which later
 * problems on the same device take buffers of a similar size instead of calling cudaMalloc.
 * firal_cache_trim returns every parked buffer to the driver; firal_cache_bytes reports how
 * many bytes are parked. */
int32_t firal_cache_trim(void);
int64_t firal_cache_bytes(void);

/* ---------------------------------------------------------------- launch tuning */

/* Launch parameters an autotuner chooses for the tensor-core path (FIRAL_MIXED_BF16*); 0 keeps
 * the built-in shape rule for that field.  dterm_splits: point-range splits (the K extent of a
 * CTA's tile) of the Hessian apply's second GEMM; a value below what the accumulation-chain
 * bound of that GEMM needs is raised to it.  bsum_splits: point-range splits of the block sums
 * of eq. 13.  sm_budget: CTAs the problem's grids spread over (capped at the SM count).  The
 * FIRAL_SPLITS / FIRAL_SM_BUDGET environment overrides still take precedence. */
typedef struct {
  int32_t dterm_splits;
  int32_t bsum_splits;
  int32_t sm_budget;
  int32_t reserved;       /* 0 */
} firal_tuning;

/* Set a prepared problem's tuning (applies to its next launches). */
int32_t firal_problem_set_tuning(firal_problem* problem, const firal_tuning* tuning);

/* The values the problem's last launches used (0 for a kernel not launched yet). */
int32_t firal_problem_get_tuning(firal_problem* problem, firal_tuning* out);

/* Default tuning of every problem created on the handle afterwards, including the pooled
 * problems firal_batched_relax builds internally. */
int32_t firal_set_default_tuning(firal_handle* handle, const firal_tuning* tuning);

/* ---------------------------------------------------------------- row sharding (Section 3.3) */

/* The paper's data decomposition: each process (one GPU) holds a contiguous slice of the pool's
 * rows (x_i, h_i, z_i), every process holds the same labelled set, probes and dc x s vectors,
 * and the per-process partial sums are added across processes where the method sums over
 * points.  A problem joins such a group through firal_problem_set_comm; the library calls the
 * caller's allreduce at these points:
 *   - once per Hessian apply (Sigma_z V or H_p V): the d c x s partial, before the null-space
 *     projection and the CG dot products (vec type, sum);
 *   - once per MD iteration: the c preconditioner blocks (double) of eq. 13, before their
 *     Cholesky factorisation (sum);
 *   - the mirror-descent scalars: ||g||_inf (double, max) and sum_i z_i exp(-beta g_i)
 *     (double, sum), so that z stays on the budget simplex over all processes;
 *   - at set-up, the pool size (double, sum), so that H_p = (1/n) sum_pool H_i uses the total n.
 * The labelled rows and lambda count once, on rank 0.  Every process must make the same calls
 * in the same order.  Round, Exact-FIRAL and pooled problems do not take a communicator.
 *
 * allreduce(buf, count, dtype, op, stream, user): in-place allreduce of `count` elements of
 * `dtype` (FIRAL_DT_F32 or FIRAL_DT_F64) at device pointer buf, op 0 = sum, 1 = max; the data is
 * ready once the work enqueued on `stream` (the handle's cudaStream_t as void*) completes, and
 * the result must be in place for work enqueued on `stream` after the callback returns (an
 * NCCL allreduce on that stream, or a host-staged exchange after a stream synchronisation,
 * both qualify).  It returns 0 on success; anything else ends the library call with
 * FIRAL_ERR_COMM. */
typedef int32_t (*firal_allreduce_fn)(void* buf, int64_t count, int32_t dtype, int32_t op,
                                      void* stream, void* user);

typedef struct {
  int32_t rank;                 /* this process, 0 .. world - 1                     */
  int32_t world;                /* number of processes; 1 (or a NULL comm) = alone */
  firal_allreduce_fn allreduce; /* see above; may be NULL only when world == 1      */
  void* user;                   /* passed back to allreduce                         */
} firal_comm;

/* Join (comm->world > 1) or leave (NULL or world == 1) a row-sharded group.  Calls allreduce
 * once (the pool size) and synchronises.  FIRAL_ERR_UNSUPPORTED for pooled problems. */
int32_t firal_problem_set_comm(firal_problem* problem, const firal_comm* comm);

/* ---------------------------------------------------------------- active learning (Section 5) */

/* Class probabilities of the multinomial logistic-regression classifier (eq. 1):
 * h_i = softmax(W x_i) for the rows of X.  X: device, rows x d of x_dtype.  W: device, c x d
 * (row k = class k) of the vec type of `precision` (FIRAL_FP64: double, otherwise float).
 * h_out: device, rows x c of that type.  Synchronises. */
int32_t firal_lr_probs(firal_handle* handle, const void* X, int32_t x_dtype, const void* W,
                       int64_t rows, int32_t d, int32_t c, int32_t precision, void* h_out);

/* Classifier refit: W minimising sum_i -log softmax(W x_i)_{y_i} + (gamma / 2) ||W||_F^2 over
 * m labelled rows, by damped Newton steps (Armijo backtracking) whose systems
 * (sum_i H_i + gamma I) dW = grad, H_i of eq. 2, are solved with the block-Jacobi PCG of
 * Algorithm 2 (FP64 for FIRAL_FP64, FP32 otherwise).  X: device, m x d of x_dtype.  y: device,
 * m int32 labels in [0, c) (checked; FIRAL_ERR_ARG otherwise).  W: device, c x d of the vec type;
 * in: starting point, out: the fit.  Stops when ||grad|| <= tol max(1, ||grad(W_start)||)
 * (tol <= 0: 1e-8; in FP32 tol is raised to at least 2e-5, the float noise floor of the
 * gradient), when no Armijo step lowers the loss, or after max_newton steps.  iters_out,
 * gnorm_out: host or NULL. */
int32_t firal_lr_fit(firal_handle* handle, const void* X, int32_t x_dtype, const int32_t* y,
                     int64_t m, int32_t d, int32_t c, double gamma, int32_t precision,
                     int32_t max_newton, double tol, void* W, int32_t* iters_out,
                     double* gnorm_out);

/* Controls of the active-learning loop. */
typedef struct {
  int32_t rounds;          /* AL rounds (>= 1)                                              */
  int32_t budget;          /* points selected per round (>= 1; rounds * budget < n)         */
  double lambda;           /* ridge of H_o in Relax and Round (eq. 3)                       */
  double lr_gamma;         /* ridge of the classifier refit (> 0)                           */
  int32_t lr_max_newton;   /* Newton steps per refit (<= 0: 30)                             */
  int32_t reserved;        /* 0                                                             */
  double lr_tol;           /* refit gradient tolerance (<= 0: 1e-8)                         */
  firal_relax_opts relax;  /* Relax of every round; round r draws its probes with seed       */
                           /* relax.seed + r; relax.precision also sets Round's precision  */
  double eta;              /* Round eta (<= 0: 8 sqrt(d c))                                 */
} firal_al_opts;

/* Multi-round active learning (the outer loop of Section 5).  Round r = 0 .. rounds-1: refit W
 * on the labelled set (the m initial rows, then the pool rows picked so far, in selection
 * order; warm start from the previous round, W = 0 at first), set h = softmax(W x) on the
 * labelled set and on the remaining pool (pool rows not picked yet, in index order), run Relax
 * (Algorithm 2) with budget = opts->budget and Round (Algorithm 3) on that pool, and move the
 * picks to the labelled set.  X_pool: device, n x d of x_dtype; y_pool: device, n int32 labels
 * (a pool label enters only once its point is picked).  X_lab, y_lab: device, m rows / labels
 * (m >= 0).  selected_out: device, rounds * budget int32 pool indices, round-major in
 * selection order.  W_out: device, c x d of the vec type: the classifier refit on the final
 * labelled set, or NULL.  fhat_out: host, rounds doubles (last f^ of each Relax) or NULL.
 * Synchronises before returning. */
int32_t firal_active_learning(firal_handle* handle, const void* X_pool, const int32_t* y_pool,
                              int64_t n, const void* X_lab, const int32_t* y_lab, int64_t m,
                              int32_t d, int32_t c, int32_t x_dtype, const firal_al_opts* opts,
                              int32_t* selected_out, void* W_out, double* fhat_out);

#ifdef __cplusplus
}
#endif

#endif /* FIRAL_H */
