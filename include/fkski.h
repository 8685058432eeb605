/*
 * fkski -- faster kernel interpolation for Gaussian processes (GSGP / factorized SKI) on GB300.
 *
 * C ABI of libfkski.so.  Yadav, Sheldon & Musco, "Faster Kernel Interpolation for Gaussian
 * Processes" (arXiv 2101.11751).  Notation follows the paper: n training points x_i with targets
 * y_i, a regular grid G of m nodes, interpolation matrix W (n x m, cubic convolution, 4^d nonzeros
 * per row), grid kernel matrix K_G (= K_UU), noise variance sigma^2.
 *
 * Conventions for every entry point
 *  - Return value: FKSKI_OK (0) or a negative FKSKI_E_* code.  No call aborts or prints.
 *  - Pointers documented "device" are CUDA device pointers owned by the caller; the library never
 *    frees them.  Pointers documented "host" are ordinary host memory.
 *  - Every call takes a CUDA stream (cudaStream_t passed as void*; NULL = legacy default stream)
 *    and is ordered on it.  A call that synchronizes the stream says so.
 *  - fkski_stats owns its device memory (sufficient statistics, spectra, solver workspace); it is
 *    released only by fkski_destroy.  Calls on one fkski_stats must not run concurrently.
 *  - Determinism: identical inputs on the same GPU give bit-identical outputs.
 *  - Layouts: points X are d x n, structure of arrays (X[k*n + i] = coordinate k of point i).
 *    Grid vectors of length m are in C order over (M_1, ..., M_d), last axis fastest; node
 *    (j_1..j_d) sits at lo_k + j_k h_k.  Several right-hand sides are stored rhs-major.
 */
#ifndef FKSKI_H
#define FKSKI_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define FKSKI_API __attribute__((visibility("default")))
#else
#define FKSKI_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status codes */
#define FKSKI_OK 0
#define FKSKI_E_INVALID_ARG (-1)   /* d not in {1,2,3}, M_k < 4, h <= 0, sigma^2 <= 0, n < 1, NULL */
#define FKSKI_E_OUT_OF_GRID (-2)   /* some point has s_k = (x_k - lo_k)/h_k outside [1, M_k - 2]   */
#define FKSKI_E_NONFINITE (-3)     /* NaN or Inf in X, y or the probes                             */
#define FKSKI_E_NOT_CONVERGED (-4) /* maxiter reached; outputs are still written, info filled      */
#define FKSKI_E_BREAKDOWN (-5)     /* CG breakdown: p^T A p <= 0 or a non-finite inner product      */
#define FKSKI_E_TIMEOUT (-6)       /* a bounded device wait gave up (reserved: no kernel of this
                                      build waits on another; reductions use last-block counters) */
#define FKSKI_E_OOM (-7)           /* device allocation failed                                      */
#define FKSKI_E_CUDA (-8)          /* another CUDA runtime error                                    */
#define FKSKI_E_UNSUPPORTED (-9)   /* a size beyond what this build supports (see each call)        */
#define FKSKI_E_IO (-10)           /* file error in save/load                                       */

#define FKSKI_F32 0
#define FKSKI_F64 1
#define FKSKI_F32X2 2 /* double-float vectors, the MIXED solver's format: each value is a pair of
                         FP32 numbers (hi, lo), 8 bytes, value = hi + lo with |lo| <= ulp(hi)/2
                         (fkski_band_mvm only)                                               */

#define FKSKI_RBF 0      /* s * exp(-1/2 sum_k (r_k / l_k)^2), separable: K_G = s T_1 (x) ... (x) T_d */
#define FKSKI_MATERN52 1 /* s (1 + sqrt5 r + 5/3 r^2) exp(-sqrt5 r), r = ||r / l||: multilevel Toeplitz */

#define FKSKI_X0_ZERO 0      /* Alg. 3 (EFCG, x0 = 0, r0 = y), compressed on b' = y - W y_hat,
                                y_hat from a few CG steps on W^T W (see fkski_solve)            */
#define FKSKI_X0_Y_OVER_S2 1 /* Alg. 5 (simplified EFCG, x0 = y / sigma^2, r0 in span(W))            */

#define FKSKI_MIXED 0  /* FP32 band (the bulk of the bytes), every other vector and all operator
                          arithmetic in double-float form (pairs of FP32 numbers combined by
                          error-free transformations, about 46-bit accuracy) on the FP32 pipes;
                          FP64 solution, scalars and cross-warp inner-product sums.  The
                          products carry rounding near 1e-14 instead of FP32's 1e-7, so the CG
                          iteration counts follow those of FP64 CG.  Outputs are FP32.       */
#define FKSKI_DOUBLE 1 /* FP64 throughout (GB300's FP64 pipe is far slower than its FP32 pipe)  */
#define FKSKI_FP32 2   /* FP32 band, FFT and Krylov vectors; FP64 solution, scalars, cross-warp
                          inner-product sums, and the periodic true-residual replacement with
                          an FP64 SpMV and K_G ("reliable updates").  The fastest iteration, but
                          every FP32 K_G / band product carries a normwise rounding error near
                          1e-7..1e-6 that a CG step on A = W K W^T + sigma^2 I amplifies by up to
                          ||A|| / sigma^2: iteration counts grow well beyond FP64 CG's, and on
                          ill-conditioned systems rtol much below 1e-5 can end in
                          FKSKI_E_NOT_CONVERGED or FKSKI_E_BREAKDOWN.  Outputs are FP32.      */

/* ------------------------------------------------------------------ configuration structs */

/* Regular grid G (Sec. 2.2, "m points on a dense d-dimensional grid"): node j on axis k is at
 * lo[k] + j*h[k], j = 0..M[k]-1.  Cubic interpolation needs nodes c-1..c+2 around a point, so a
 * point must satisfy 1 <= (x_k - lo_k)/h_k <= M_k - 2 on every axis. */
typedef struct {
    int d;
    int64_t M[3];
    double lo[3];
    double h[3];
} fkski_grid;

/* Stationary kernel k(x, x') with hyperparameters theta = (l_1..l_d, s) and noise sigma^2
 * (App. C.1: squared exponential in a scale kernel; Matern-5/2 as a non-separable alternative). */
typedef struct {
    int type;
    double lengthscale[3];
    double outputscale;
    double noise_var;
} fkski_kernel;

typedef struct {
    double rtol;          /* stop when ||r_k||_2 <= rtol * ||b||_2, b = y or the probe z_p      */
    int maxiter;          /* CG iteration cap                                                  */
    int x0_mode;          /* FKSKI_X0_ZERO or FKSKI_X0_Y_OVER_S2 (fkski_solve only)             */
    int precision;        /* FKSKI_MIXED, FKSKI_DOUBLE or FKSKI_FP32                           */
    int check_every;      /* iterations per captured CUDA graph between host convergence checks */
    int n_probes;         /* Rademacher probes accumulated by fkski_precompute (<= 64)         */
    uint64_t probe_seed;  /* probe z_p(i) = sign of SplitMix64(seed) output k = p*2^40 + i + 1 */
    size_t iterate_budget_bytes; /* fkski_loglik_forward keeps its solutions if they fit     */
    int keep_sort;        /* fkski_precompute keeps cell keys and the permutation for export   */
    int reliable_updates; /* true-residual replacement when the residual has dropped 10x since
                             the last one: 0 default (on for MIXED, off for DOUBLE), 1 on, 2 off */
    int keep_points;      /* fkski_precompute keeps the points (local coordinates, y, cell keys) in
                             cell order, as fkski_ski_solve needs                                */
    int reserved[5];
} fkski_opts;

typedef struct {
    int iters;            /* CG iterations (max over right-hand sides)                          */
    int status;           /* FKSKI_OK, FKSKI_E_NOT_CONVERGED or FKSKI_E_BREAKDOWN               */
    double rel_residual;  /* final ||r||/||r_0|| (max over right-hand sides)                    */
    double t_ms[8];       /* stage times when measured (0 otherwise)                            */
    int iters_rhs[65];    /* per right-hand side iteration counts (grad: [y, z_1..z_T])         */
} fkski_info;

typedef struct fkski_stats fkski_stats;

/* Fill opts with defaults: rtol 1e-6, maxiter 1000, x0 Alg. 5, mixed precision, check_every 16,
 * no probes, seed 0, budget 1 GiB, keep_sort 0. */
FKSKI_API void fkski_default_opts(fkski_opts *opts);

/* Human-readable name of a status code (static string). */
FKSKI_API const char *fkski_strerror(int status);

/* The CUDA error behind the calling thread's last FKSKI_E_CUDA / FKSKI_E_OOM (runtime error
 * string, code and source location; empty if none).  Valid until the thread's next failing call. */
FKSKI_API const char *fkski_last_error_detail(void);

/* The launch configurations the K_G autotuner has chosen so far in this process, one line per
 * pass shape ("f32 L=256 M=128 S=32 lines=4096 -> radix 4, 4 lines/CTA, 256 threads, 0.0123 ms").
 * The paper has no counterpart: the tuner picks, per Kronecker pass shape, the lines per CTA and
 * threads per CTA (and, for the shared-memory transform used above L = 256 in FP32 / L = 64 in
 * FP64, the FFT stage radix 2 or 4; radix 0 denotes the register transform) by timing each
 * candidate once (before the solver captures its graphs); the choices give bit-identical results.  Writes at most len bytes
 * (NUL-terminated) to buf (may be NULL) and returns the size needed. */
FKSKI_API size_t fkski_tuning_table(char *buf, size_t len);

/* Stream-ordered temporaries (precompute scratch, covariance blocks, tuner buffers) and the
 * statistics' band, W^T y and W^T z come from a library memory pool per device that keeps freed
 * blocks cached, so repeated calls map no new memory.  This returns the cached blocks to the
 * device (the paper has no counterpart).  Call it with no library call in flight.  Returns OK or
 * CUDA. */
FKSKI_API int fkski_trim_memory(void);

/* Number of kernel launches this library has issued in the process so far (a replayed CUDA graph
 * counts each of its kernel nodes).  Host-only; for instrumentation. */
FKSKI_API long long fkski_kernel_launches(void);

/* ------------------------------------------------------------------ precompute (Sec. 3.1)
 * One O(n) pass computing the sufficient statistics of the Bayesian linear regression of Def. 2:
 *   W^T W  stored as its 7^d diagonals (Claim 2: at most (4r-1)^d = 7^d nonzeros per row, r = 2),
 *   W^T y, y^T y, and for opts->n_probes Rademacher probes z_p (or the caller's probes Z) W^T z_p
 *   and z_p^T z_p.
 * Points are sorted by grid cell with a stable sort (ties by input index) and reduced per cell
 * in that order, so the result is deterministic.
 *   grid   host; X d x n (dtype); y n (dtype); Z n_probes x n (dtype) or NULL.  X, y and Z are
 *          read once, by the first kernel: they may be device memory or page-locked host memory
 *          mapped into the device address space (e.g. cudaHostAlloc), which the kernel then reads
 *          over the host link without a separate copy; memory the CUDA runtime reports without a
 *          device mapping (pageable host memory on most systems) is INVALID_ARG.
 *   dtype  FKSKI_F32 or FKSKI_F64 (points and targets).  F32: per-cell sums in FP32 (runs of
 *          32 points per lane, then a second FP32 level) and FP32 statistics; F64: FP64 throughout.
 *   out    receives a new fkski_stats on success (NULL on failure).
 * Errors: INVALID_ARG, OUT_OF_GRID, NONFINITE, OOM, CUDA, UNSUPPORTED (n >= 2^31, cells >= 2^31,
 * n_probes > 64).  Synchronizes the stream once, at the end, to report point errors. */
FKSKI_API int fkski_precompute(const fkski_grid *grid, const void *X, const void *y, const void *Z, int64_t n,
                     int dtype, const fkski_opts *opts, fkski_stats **out, void *stream);

/* Sizes of a stats object (host outputs; any pointer may be NULL). */
FKSKI_API int fkski_stats_info(const fkski_stats *st, fkski_grid *grid, int64_t *n, int64_t *m,
                     int64_t *ncells, int *n_probes, double *yty, int *dtype);

/* Copy statistics to host memory in FP64 (any pointer may be NULL):
 * band 7^d x m with band[o*m + j] = (W^T W)[j, j + delta(o)], o = sum_k (delta_k + 3) 7^(d-1-k);
 * wty m; wtz n_probes x m; ztz n_probes.  Synchronizes the stream. */
FKSKI_API int fkski_stats_export(const fkski_stats *st, double *band, double *wty, double *wtz, double *ztz,
                       void *stream);

/* Copy the cell sort to host memory: keys[i] = linear cell index of point i (C order over
 * cells c_k - 1 in [0, M_k - 4]); perm = stable sort of points by key; offsets[c]..offsets[c+1]
 * is cell c's segment (ncells + 1 entries).  Needs opts.keep_sort at precompute time
 * (else UNSUPPORTED).  Synchronizes the stream. */
FKSKI_API int fkski_stats_export_sort(const fkski_stats *st, uint32_t *keys, int64_t *perm, int64_t *offsets,
                            void *stream);

/* Save / load the statistics (the paper's "computed once and saved to disk", Sec. 5). */
FKSKI_API int fkski_stats_save(const fkski_stats *st, const char *path, void *stream);
FKSKI_API int fkski_stats_load(const char *path, fkski_stats **out, void *stream);

/* Release a stats object and all its device memory (NULL is a no-op).  Synchronizes the device;
 * the pool-backed buffers go back to the library pool (see fkski_trim_memory). */
FKSKI_API void fkski_destroy(fkski_stats *st);

/* ------------------------------------------------------------------ operators (Sec. 2.2, 3.2)
 * K_G V for nrhs grid vectors (device, rhs-major, dtype FKSKI_F32, FKSKI_F64 or FKSKI_F32X2:
 * the MIXED solver's double-float vectors, (hi, lo) FP32 pairs, 8 bytes per value), or its
 * derivative w.r.t. one hyperparameter: param = -1 for K_G, k in [0, d) for dK_G/dl_k, d for
 * dK_G/ds.
 * RBF: Kronecker product of symmetric Toeplitz factors, one batched circulant-embedding FFT pass
 * per axis (Sec. 2.2; Lee 1986).  Matern-5/2: d-level circulant embedding (multilevel Toeplitz).
 * The spectra are recomputed on every call; in and out must not alias.  UNSUPPORTED if the
 * embedding of some axis exceeds 4096 points.  Synchronizes the stream (temporaries are freed). */
FKSKI_API int fkski_kg_mvm(const fkski_grid *grid, const fkski_kernel *kern, int param, const void *v,
                 void *out, int nrhs, int dtype, void *stream);

/* Allocation-free variant of fkski_kg_mvm (the paper has no counterpart: this serves callers that
 * may not allocate device memory during the call, e.g. under an allocator or memory budget owned
 * by someone else).  Same arguments, result and dtype rules as fkski_kg_mvm, RBF kernel only
 * (value or derivative, param as there).  All working memory -- the d axis spectra and one
 * intermediate of nrhs*m values -- is one fixed device array of FKSKI_NOALLOC_SCRATCH_BYTES per
 * device inside this library; nothing is allocated or freed and the stream is not synchronized.
 * Limits: every M_k <= 2048; for d > 1, nrhs * m * (4 or 8 bytes) <= FKSKI_NOALLOC_SCRATCH_BYTES
 * - 96 KiB (about 4.17 million FP32 values).  Beyond them, or for a Matern kernel, it returns
 * FKSKI_E_UNSUPPORTED.  The first call on a device looks the array up and may load this
 * library's device code, so make it before capturing a stream into a CUDA graph.  The array is
 * shared: calls that overlap on one device (other streams, other threads) corrupt each other's
 * results; order them.  Returns OK, INVALID_ARG, UNSUPPORTED, CUDA. */
#define FKSKI_NOALLOC_SCRATCH_BYTES ((size_t)16 << 20)
FKSKI_API int fkski_kg_mvm_noalloc(const fkski_grid *grid, const fkski_kernel *kern, int param, const void *v,
                                   void *out, int nrhs, int dtype, void *stream);

/* u = (W^T W) x for nrhs grid vectors (device, rhs-major, dtype) from the stored band
 * (Claim 2: O(m 7^d)).  dtype FKSKI_F32, FKSKI_F64, or FKSKI_F32X2 (the FP32 band applied to
 * double-float vectors, as in the MIXED iterations). */
FKSKI_API int fkski_band_mvm(const fkski_stats *st, const void *x, void *u, int nrhs, int dtype, void *stream);

/* ------------------------------------------------------------------ posterior mean (Sec. 4, App. B)
 * Solves the SKI system (W K_G W^T + sigma^2 I) z = y by factorized CG using only the sufficient
 * statistics: Alg. 5 (x0 = y/sigma^2) or Alg. 3 (x0 = 0), one B(x) = [(K_G W^T W + sigma^2 I)x,
 * W^T W x] per iteration.  Outputs (device, m entries, FP32 for MIXED and FP32, FP64 for DOUBLE):
 *   a_out = W^T z   and   v_out = K_G W^T z  (= z_bar, the GSGP posterior mean of theta, Fact 2).
 * With x0 = 0 the paper's Alg. 3 represents iterates as W v_hat + c y; here y is first split as
 * y = W y_hat + y' (y_hat: 8 CG steps on W^T W y_hat = W^T y) and iterates as W v_hat + c y'.
 * Both are exact; the split keeps y's out-of-range(W) part (an eigenvector of A) from cancelling
 * against in-range terms in the inner products of Claim 4, which otherwise costs ~30% more
 * iterations in FP64 and breaks down in FP32.
 * FP32: at the end of a chunk of opts->check_every iterations, a right-hand side whose residual
 * fell 10x since its last replacement (or below the tolerance) gets the true residual of its FP64
 * solution (FP64 SpMV and FP64 K_G) in place of the recursive one; convergence is declared only
 * on that true residual.  MIXED and DOUBLE test the recursive residual, as the paper's EFCG does.
 * Stops when ||r_k|| <= rtol ||y||.  info (host, may be NULL) receives iterations and residual.
 * Returns OK, NOT_CONVERGED (outputs written), BREAKDOWN, INVALID_ARG, OOM, CUDA.
 * Synchronizes the stream every opts->check_every iterations to test convergence. */
FKSKI_API int fkski_solve(fkski_stats *st, const fkski_kernel *kern, const fkski_opts *opts, void *a_out,
                void *v_out, fkski_info *info, void *stream);

/* Posterior mean at test points: mu(x*) = w_{x*}^T v (Def. 1 mean with v = K_G W^T z; Fact 2).
 * v device m (vdtype); Xstar device d x nstar (xdtype); mu_out device nstar (vdtype).
 * Errors: OUT_OF_GRID / NONFINITE for a test point (mu for other points still written). */
FKSKI_API int fkski_predict(const fkski_stats *st, const void *v, int vdtype, const void *Xstar, int xdtype,
                  int64_t nstar, void *mu_out, void *stream);

/* log det (W K_G W^T + sigma^2 I) by stochastic Lanczos quadrature with the efficiently factorized
 * Lanczos method (App. B, EFLA; refs [ScalableLD], [GPyTorchBM]): for each of the precompute's
 * probes z_p, k steps of EFLA started at z_p (FP64, full reorthogonalisation) give T_p, and
 * logdet ~ mean_p ||z_p||^2 e_1^T log(T_p) e_1 (Ritz values clamped at sigma^2).  The alternative
 * to the CG-coefficient quadrature inside fkski_loglik_forward, with reorthogonalised Lanczos
 * vectors.  Needs n_probes >= 1 at precompute time.  logdet_out (host); terms (host, n_probes,
 * may be NULL) receives each probe's term.  info->iters: the most Lanczos steps taken.  Returns
 * OK, BREAKDOWN (QL did not converge), INVALID_ARG, OOM, CUDA.  Synchronizes the stream. */
FKSKI_API int fkski_logdet_lanczos(fkski_stats *st, const fkski_kernel *kern, int k, double *logdet_out,
                                   double *terms, fkski_info *info, void *stream);

/* Plain SKI posterior mean (Def. 1) by n-space CG (Alg. 1) on W K_G W^T + sigma^2 I from x0 = 0:
 * the O(n + m log m)-per-iteration method the paper's factorized solvers replace (Sec. 5,
 * Fig. 2, Table 1), for comparison.  Needs the points kept by the precompute (opts.keep_points);
 * otherwise UNSUPPORTED.  n-space vectors per opts->precision for FP32 points (MIXED
 * double-float, FP32, or DOUBLE), FP64 for FP64 points; FP64 cross-block inner products.  W's
 * entries are the per-point weight products rounded once in the points' precision, and W^T is
 * their exact transpose.  Stops when ||r_k|| <= rtol ||y||; opts->maxiter, check_every as for
 * fkski_solve.  Outputs as fkski_solve: a_out = W^T z, v_out = K_G W^T z (device, m; FP64 for
 * FP64 points or DOUBLE, else FP32).  Returns OK, NOT_CONVERGED, BREAKDOWN, INVALID_ARG,
 * UNSUPPORTED, OOM, CUDA. */
FKSKI_API int fkski_ski_solve(fkski_stats *st, const fkski_kernel *kern, const fkski_opts *opts, void *a_out,
                              void *v_out, fkski_info *info, void *stream);

/* Posterior covariance at test points (Def. 1 / Fact 2, equal by Theorem 1):
 *   cov(x_i, x_j) = w_i^T K_G w_j - (W K_G w_i)^T (W K_G W^T + sigma^2 I)^{-1} (W K_G w_j).
 * The right-hand sides W K_G w_j lie in span(W): each is solved by the simplified EFCG from
 * x0 = 0 with r_hat_0 = K_G w_j (App. B), blocks of 32 test points sharing one band read per
 * iteration; opts as for fkski_solve (rtol relative to ||W K_G w_j||, precision, maxiter).
 * Xstar device d x nstar (xdtype); cov_out device nstar x nstar FP64, row-major (cov_out[i*nstar+j]).
 * info (host, may be NULL): max iterations and residual over the solves.  Returns OK,
 * NOT_CONVERGED, BREAKDOWN, OUT_OF_GRID / NONFINITE (a test point; its row and column are 0),
 * INVALID_ARG, OOM, CUDA.  Synchronizes the stream. */
FKSKI_API int fkski_posterior_cov(fkski_stats *st, const fkski_kernel *kern, const fkski_opts *opts,
                                  const void *Xstar, int xdtype, int64_t nstar, double *cov_out, fkski_info *info,
                                  void *stream);

/* Rank-k approximation of the same covariance (the paper's predictive-covariance task with
 * ref. [ConstantTimePD]): k steps of the efficiently factorized Lanczos method (App. B, EFLA) on
 * W K_G W^T + sigma^2 I started at y / ||y||, in FP64 with full reorthogonalisation, give
 * A^{-1} ~ Q T^{-1} Q^T with Q = W Q_hat + b d^T; then
 *   cov(x, x') ~ w_x^T K_G w_x' - (R^T w_x)^T (R^T w_x'),   R = K_G (W^T W Q_hat + W^T b d^T) L^{-T},
 * T = L L^T.  R (m x k FP64) is kept in the statistics object: later calls with the same kernel
 * and k evaluate new test points in O(4^d k) each plus the prior term (one K_G product per 32
 * test points).  Fewer than k steps are taken if the Krylov space closes (info->iters).  With k
 * large enough the result equals fkski_posterior_cov.  Xstar / cov_out as there (nstar may be 0:
 * build only).  Returns OK, BREAKDOWN (T not positive definite), OUT_OF_GRID / NONFINITE,
 * INVALID_ARG, OOM, CUDA.  Synchronizes the stream. */
FKSKI_API int fkski_posterior_cov_lowrank(fkski_stats *st, const fkski_kernel *kern, const fkski_opts *opts, int k,
                                          const void *Xstar, int xdtype, int64_t nstar, double *cov_out,
                                          fkski_info *info, void *stream);

/* ------------------------------------------------------------------ batches of independent problems
 * Many unrelated GP problems of uneven sizes (serving-style batch), each with its own grid, data,
 * kernel and noise; the arrays below have nprob entries, one per problem.  Per problem the
 * results equal those of the single-problem call.
 *
 * fkski_precompute_batched: fkski_precompute for every problem in turn on `stream` (grids[p],
 * X[p] (d_p x n[p] SoA), y[p], all in `dtype`; opts as for fkski_precompute, shared).  out[p]
 * receives each statistics object; on an error every object already made is destroyed, out[]
 * is set to NULL and the first error is returned.
 *
 * fkski_solve_batched: the posterior mean of every problem (Sec. 4, Alg. 5 or Alg. 3 per
 * opts->x0_mode, shared opts).  st[] must be distinct objects.  All problems are set up, then
 * their captured iteration chunks run as independent child graphs of one CUDA graph, launched
 * once per check_every iterations until every problem has finished; finished problems skip
 * their kernels.  a_out[p], v_out[p] as for fkski_solve (m_p entries); info (host, nprob
 * entries, may be NULL) per problem.  Returns OK, or the first error / NOT_CONVERGED /
 * BREAKDOWN met (BREAKDOWN first); outputs of every problem are written.
 *
 * fkski_predict_batched: mu_p(x*) = w_{x*}^T v_p for every problem in one kernel launch per
 * distinct d (Def. 1, Fact 2).  v[p] device m_p (vdtype), Xstar[p] device d_p x nstar[p]
 * (xdtype), mu_out[p] device nstar[p] (vdtype); status (host, nprob entries, may be NULL)
 * receives each problem's OUT_OF_GRID / NONFINITE / OK.  Returns OK or the first error. */
FKSKI_API int fkski_precompute_batched(int nprob, const fkski_grid *grids, const void *const *X, const void *const *y,
                                       const int64_t *n, int dtype, const fkski_opts *opts, fkski_stats **out,
                                       void *stream);
FKSKI_API int fkski_solve_batched(int nprob, fkski_stats *const *st, const fkski_kernel *kernels,
                                  const fkski_opts *opts, void *const *a_out, void *const *v_out, fkski_info *info,
                                  void *stream);
FKSKI_API int fkski_predict_batched(int nprob, const fkski_stats *const *st, const void *const *v, int vdtype,
                                    const void *const *Xstar, int xdtype, const int64_t *nstar, void *const *mu_out,
                                    int *status, void *stream);

/* ------------------------------------------------------------------ log-likelihood and gradient
 * Log marginal likelihood of Def. 1, L = -1/2 [logdet(A) + y^T A^{-1} y + n log 2pi] with
 * A = W K_G W^T + sigma^2 I, from sufficient statistics only:
 *   - batched factorized CG (Alg. 3, x0 = 0) on [y, z_1..z_T] sharing each B(x) application;
 *   - logdet(A) by stochastic Lanczos quadrature over the probes, with the Lanczos tridiagonal
 *     formed from the CG coefficients (Sec. 2.1 "Inference via iterative methods");
 *   - y^T A^{-1} y = (W^T y)^T x_hat + c^x y^T y from the compressed solution.
 * Gradient w.r.t. theta = (l_1..l_d, s, sigma^2) (the paper's "further trace computation",
 * Sec. 2.1):
 *   dL/dtheta   = 1/2 a^T dK a - 1/2 mean_p (W^T x_p)^T dK (W^T z_p),   a = W^T A^{-1} y
 *   dL/dsigma^2 = 1/2 ||A^{-1} y||^2 - 1/2 mean_p z_p^T x_p,              x_p = A^{-1} z_p
 * with dK applied by derivative-Toeplitz circulant-embedding MVMs.  Requires n_probes >= 1 at
 * precompute time.  loglik_out: host double; grad_out: host double[d + 2].
 * fkski_loglik_forward keeps the solutions in the stats workspace when
 * (T + 1) * m * sizeof(vector) * 2 <= opts->iterate_budget_bytes; fkski_loglik_backward reuses
 * them, or reruns the (deterministic) forward solves when they were not kept.
 * All three synchronize the stream.  info (host, may be NULL) gets per-rhs iteration counts. */
FKSKI_API int fkski_loglik_forward(fkski_stats *st, const fkski_kernel *kern, const fkski_opts *opts,
                         double *loglik_out, fkski_info *info, void *stream);
FKSKI_API int fkski_loglik_backward(fkski_stats *st, const fkski_kernel *kern, const fkski_opts *opts,
                          double *grad_out, fkski_info *info, void *stream);
FKSKI_API int fkski_grad(fkski_stats *st, const fkski_kernel *kern, const fkski_opts *opts,
               double *loglik_out, double *grad_out, fkski_info *info, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* FKSKI_H */
