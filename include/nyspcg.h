/*
 * nyspcg.h -- C ABI of the GB300 (sm_103a) Nystrom-preconditioned CG library.
 *
 * Solves regularized psd systems (A + mu I) x = b (Sec. 1.1, Eq. (1.1)) with
 * the randomized Nystrom preconditioner of Frangella, Tropp & Udell,
 * "Randomized Nystrom Preconditioning" (arXiv 2110.02820):
 *   - nys_sketch           Algorithm 1 (randomized Nystrom approximation)
 *   - nys_sketch_adaptive  Algorithm 5 with Algorithm 4 (adaptive rank)
 *   - nys_precond_apply    Eq. (5.3), the inverse preconditioner P^{-1}
 *   - nys_sketch_solve     Algorithm 2 (Nystrom sketch-and-solve), the accuracy contrast
 *   - nys_block_pcg        block Nystrom PCG (Sec. 5.2) for many right-hand sides of one mu
 *   - nys_reg_path         regularization path with warm starts and factor reuse (Sec. 6.2)
 *   - pcg_solve            Algorithm 3 (Nystrom PCG), batched over systems,
 *                          in FP64 or mixed precision with FP64-residual
 *                          iterative refinement
 *
 * Conventions for every entry point:
 *   - Matrices are ROW-MAJOR (C order).  An n x ell matrix M has element
 *     (i, j) at M[i * ell + j].  Batches of vectors are stored system-major:
 *     system s of a batch of n-vectors starts at V + s * n.
 *   - Array arguments are DEVICE pointers unless the comment says "host".
 *     The caller owns them; the library never frees or keeps them after the
 *     call returns (a factor keeps its own copies).
 *   - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *     stream.  Work is enqueued on it; entry points that must return a
 *     scalar result synchronise that stream before returning.
 *   - Errors are reported only through nys_status.  No entry point aborts,
 *     throws or traps the GPU.  Arguments are checked on the host before
 *     any launch; a bad argument returns NYS_ERR_ARG and enqueues nothing.
 *   - Every reduction runs in a fixed order: results are bitwise
 *     reproducible run to run on the same GPU and launch configuration.
 */
#ifndef NYSPCG_H
#define NYSPCG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum nys_status {
  NYS_OK = 0,
  NYS_ERR_ARG = 1,        /* invalid argument (shape, pointer, mu < 0, ell > n, ...) */
  NYS_ERR_NOT_PSD = 2,    /* Cholesky of Omega^T Y_nu failed after 6 shift escalations */
  NYS_ERR_BREAKDOWN = 3,  /* PCG: p^T (A+mu I) p <= 0 or a non-finite scalar */
  NYS_ERR_MAXIT = 4,      /* PCG: iteration cap reached; x holds the last iterate */
  NYS_ERR_TIMEOUT = 5,    /* a bounded device-side wait expired */
  NYS_ERR_CUDA = 6,       /* a CUDA runtime call failed */
  NYS_ERR_OOM = 7         /* device allocation failed */
} nys_status;

/* Operator kinds: how x -> A x is computed (Sec. 1.1 accesses A only through
 * matvecs). */
typedef enum nys_op_kind {
  NYS_OP_DENSE = 0, /* data: A, n x n symmetric psd, leading dimension ld (>= n) */
  NYS_OP_GRAM = 1,  /* data: X, m x n; A = X^T X (ridge normal operator, Eq. (1.7)),
                       applied matrix-free as X^T (X v) */
  NYS_OP_RBF = 2    /* data: points, n x d; A = K, K_ij = exp(-||x_i-x_j||^2/(2 sigma^2))
                       (Gaussian kernel of Sec. 6.5), never formed */
} nys_op_kind;

typedef enum nys_dtype { NYS_F64 = 0, NYS_F32 = 1 } nys_dtype;

/* NYS_PREC_F64: every step in FP64.
 * NYS_PREC_MIXED: sketch and tall-skinny products in FP32/TF32 (Gaussian
 *   kernel: FP16 hi/lo splits, 22 significant bits per operand) with FP32
 *   accumulation, U stored FP32, inner PCG on FP32 vectors with FP64
 *   scalars; the shift and the outer residual r = b - (A + mu I) x stay
 *   FP64-accurate, and the ell x ell factorisations run in FP64 or in
 *   double-FP32 arithmetic (~2^-48 relative, on the FP32 pipes). */
typedef enum nys_precision { NYS_PREC_F64 = 0, NYS_PREC_MIXED = 1 } nys_precision;

typedef struct nys_operator {
  int32_t kind;      /* nys_op_kind */
  int32_t dtype;     /* nys_dtype of `data`: DENSE needs F64; GRAM and RBF need F32 */
  int64_t n;         /* system dimension */
  int64_t m;         /* GRAM: number of rows of X; otherwise ignored */
  int64_t d;         /* RBF: point dimension (1..64); otherwise ignored */
  int64_t ld;        /* row stride of `data` in elements (>= its row length) */
  const void* data;  /* device pointer, row-major, 16-byte aligned */
  double sigma;      /* RBF bandwidth (> 0); otherwise ignored */
} nys_operator;

/* Opaque factor: U (n x ell, orthonormal columns), lambda_hat (ell,
 * descending, >= 0), the shift nu, ell.  Owned by the library. */
typedef struct nys_factor nys_factor;

/* Algorithm 1.  Draws Omega (n x ell) with the library's Philox4x32-10 +
 * Box-Muller generator from `seed` (elements [0, n ell) of stream
 * (seed, NYS_STREAM_OMEGA), see nys_random_stream), unless `omega` (device, n x ell FP64,
 * row-major, raw Gaussian before the thin QR) is given; orthonormalises it
 * (thin QR of step 2, computed by CholeskyQR2); forms Y = A Omega; shifts by
 * nu = eps(||Y||_F) (FP64) or the FP32 spacing (mixed); factors
 * Omega^T Y_nu = C^T C; B = Y_nu C^{-1}; thin SVD B = U Sigma W^T;
 * lambda_hat = max(0, Sigma^2 - nu).  If the Cholesky factorisation fails, nu
 * is multiplied by 10 and the shift redone, at most 6 times, then
 * NYS_ERR_NOT_PSD.  1 <= ell <= min(n, 4096).  On success *out receives a new
 * factor (free it with nys_factor_free).  Synchronises `stream`. */
int32_t nys_sketch(const nys_operator* op, int64_t ell, uint64_t seed, const double* omega,
                   int32_t precision, nys_factor** out, void* stream);

/* Column-sampling Nystrom sketch (Sec. 2.2, random projection versus column
 * sampling; the construction the paper uses for kernel ridge regression):
 * Algorithm 1 with Omega = I[:, S] for ell distinct column indices S, so that
 * the thin QR is trivial and Y = A[:, S].  The Gaussian kernel evaluates those
 * ell columns directly (n ell entries, against n^2 ell for a random
 * projection); dense A gathers them; the ridge operator forms X^T (X Omega).
 * `cols` (device, int64 [ell], distinct, in [0, n)) gives S; if NULL, S is
 * drawn uniformly without replacement from `seed`.  Indices are not checked on
 * the device: out-of-range or repeated entries are a caller error.  Gaussian
 * operators need d <= 64.  Otherwise as nys_sketch (factor, statuses,
 * precision).  Synchronises `stream`. */
int32_t nys_sketch_columns(const nys_operator* op, int64_t ell, uint64_t seed, const int64_t* cols,
                           int32_t precision, nys_factor** out, void* stream);

typedef enum nys_adapt_rule {
  NYS_RULE_ERR = 0,   /* Strategy 1 (Sec. 5.4.1): stop when the Algorithm 4 estimate <= tol */
  NYS_RULE_RATIO = 1  /* Strategy 2 (Sec. 5.4.2): stop when lambda_hat_ell / mu <= tol */
} nys_adapt_rule;

typedef struct nys_adapt_info {
  int64_t ell;          /* final sketch size */
  int32_t doublings;    /* number of times the sketch grew */
  int32_t estimates;    /* number of Algorithm 4 runs */
  double err_est;       /* last Algorithm 4 estimate of ||A - A_nys|| (NaN if none) */
  double lambda_ell;    /* lambda_hat_ell of the final factor */
  double kappa_est;     /* (lambda_hat_ell + mu + err_est) / mu, Eq. (5.6) (NaN if no estimate) */
} nys_adapt_info;

/* Algorithm 5 (adaptive rank doubling, reusing Omega and Y) with
 * nu = sqrt(n) eps(||Y||_2).  Blocks of Omega are drawn from `seed` unless
 * `omega` (device, n x ell_max FP64 raw Gaussian) is given: block k uses the
 * next columns of it in order.  The k-th Algorithm 4 estimate (q power steps
 * on E = A - U Lam U^T) starts from `g` + k*n (device, [kmax][n] FP64) if
 * given, where kmax = ceil(log2(ell_max/ell0)) + 1, else from a Philox
 * draw.  After each estimate the loop stops if the rule holds; otherwise the
 * sketch doubles; the last block is capped so that the sketch reaches
 * exactly ell_max, after which the factor is returned without a further
 * estimate.  `mu` is used by NYS_RULE_RATIO and for info->kappa_est.
 * `info` (host) may be NULL.  Synchronises `stream`. */
int32_t nys_sketch_adaptive(const nys_operator* op, int64_t ell0, int64_t ell_max, int32_t rule,
                            double tol, int32_t q, double mu, uint64_t seed, const double* omega,
                            const double* g, int32_t precision, nys_factor** out,
                            nys_adapt_info* info, void* stream);

/* Eq. (5.3): z_s = P_s^{-1} v_s = (lambda_hat_ell + mu_s) U (Lam + mu_s I)^{-1} U^T v_s
 * + (I - U U^T) v_s for s = 0..nrhs-1.  `mu` is a HOST array of nrhs shifts
 * (each >= 0, and > 0 when lambda_hat_ell = 0).  v and z are device arrays
 * of nrhs n-vectors of type `dtype` (may not alias).  Asynchronous. */
int32_t nys_precond_apply(const nys_factor* f, const double* mu, int64_t nrhs, const void* v,
                          void* z, int32_t dtype, void* stream);

/* Algorithm 2 (Nystrom sketch-and-solve, Sec. 4, Eq. (4.1)): solves the
 * approximated system (U Lam U^T + mu_s I) x_s = b_s directly,
 *   x_s = U (Lam + mu_s I)^{-1} U^T b_s + (b_s - U U^T b_s) / mu_s,
 * for s < nrhs.  This is the paper's accuracy contrast to PCG: x_s solves the
 * Nystrom approximation, not (A + mu_s I) x = b_s.  `mu` is a HOST array of nrhs
 * shifts, each > 0; b and x are device arrays [nrhs][n] of `dtype` (may not
 * alias).  An FP32 factor is applied through its orthonormalised basis, as in
 * nys_precond_apply.  Synchronises `stream`. */
int32_t nys_sketch_solve(const nys_factor* f, const double* mu, int64_t nrhs, const void* b,
                         void* x, int32_t dtype, void* stream);

typedef struct nys_pcg_opts {
  double tol;                 /* stop when ||r||_2 <= tol ||b||_2 (default 1e-8) */
  int32_t maxit;              /* iteration cap per system (default 500); in mixed precision
                                 the cap on a system's FP32 inner iterations summed over all
                                 refinement steps.  A mixed-precision system whose true
                                 residual (FP64-accurate) fails to halve over one FP32 inner
                                 solve, or that spends this budget, is escalated: its later
                                 inner solves run on FP64 vectors with FP64-accurate
                                 products (the FP32 products' error is then comparable to
                                 mu), under a second budget of maxit iterations.  An
                                 escalated system whose true residual fails to halve over
                                 two consecutive inner solves ends with NYS_ERR_MAXIT */
  int32_t precision;          /* nys_precision */
  double inner_tol;           /* mixed: relative tolerance of each inner solve (default 1e-4) */
  int32_t max_refine;         /* mixed: cap on outer refinement steps (default 20) */
  int32_t use_x0;             /* nonzero: x holds the initial guess; zero: start from x = 0 */
  double* residual_history;   /* optional device buffer [nsys][maxit+1] FP64: recurrence
                                 ||r_t|| of the (last inner) solve, NaN-padded; may be NULL */
} nys_pcg_opts;

typedef struct nys_pcg_result {
  int32_t status;             /* per system: NYS_OK, NYS_ERR_MAXIT or NYS_ERR_BREAKDOWN */
  int32_t iterations;         /* A-matvecs inside the PCG loop (summed over inner solves) */
  int32_t refinements;        /* mixed: outer steps taken; FP64: 0 */
  int32_t escalated;          /* mixed: 1 when the system's later inner solves ran on FP64
                                 vectors with FP64-accurate products (see nys_pcg_opts.maxit);
                                 otherwise 0 */
  double rel_residual;        /* FP64: recurrence ||r||/||b||; mixed: true FP64 ||b - A_mu x||/||b|| */
} nys_pcg_result;

/* Algorithm 3 for nsys independent systems (A + mu_s I) x_s = b_s sharing the
 * operator and the factor (f == NULL gives plain CG).  `mu` is a HOST array
 * [nsys]; b and x are device FP64 arrays [nsys][n]; `results` is a HOST array
 * [nsys].  `opts` may be NULL (defaults).  Returns the worst per-system
 * status.  Synchronises `stream`. */
int32_t pcg_solve(const nys_operator* op, const nys_factor* f, const double* mu, int64_t nsys,
                  const double* b, double* x, const nys_pcg_opts* opts,
                  nys_pcg_result* results, void* stream);

/* Block Nystrom PCG (Sec. 5.2, "Block Nystrom PCG"): O'Leary's block CG for
 * nrhs right-hand sides of ONE shifted system (A + mu I) X = B, preconditioned
 * by Eq. (5.3) (f == NULL gives unpreconditioned block CG), after the initial
 * residual block is orthonormalised, R_0 = Q S (Feng, Owen & Peric's
 * pre-processing; Gram-Schmidt with one reorthogonalisation, a column with no
 * new direction contributing through S only).  The block iterates share one
 * Krylov space, so a column can converge in fewer products than its single
 * solve.  Column j stops being a target when ||(R S) e_j|| <= tol ||b_j||;
 * the loop runs until every column meets it.
 *   mu      the shift (host scalar, >= 0; > 0 when lambda_hat_ell = 0);
 *   nrhs    1..32 columns;
 *   b, x    device FP64 [nrhs][n] (system-major); x is the initial guess when
 *           opts->use_x0, else overwritten;
 *   opts    as for pcg_solve (residual_history is ignored); NYS_PREC_MIXED
 *           runs the FP32 block solve inside the FP64-residual refinement;
 *   results HOST [nrhs]: status per column; iterations = block products
 *           (A + mu I) P summed over refinement steps, the same for every
 *           column; rel_residual as for pcg_solve.
 * Returns the worst column status (NYS_ERR_BREAKDOWN when P^T (A + mu I) P or
 * Z^T R stops being positive definite), or NYS_ERR_ARG / NYS_ERR_OOM /
 * NYS_ERR_CUDA / NYS_ERR_TIMEOUT.  Synchronises `stream`. */
int32_t nys_block_pcg(const nys_operator* op, const nys_factor* f, double mu, int64_t nrhs,
                      const double* b, double* x, const nys_pcg_opts* opts,
                      nys_pcg_result* results, void* stream);

typedef struct nys_path_result {
  int32_t status;       /* PCG status at this shift (NYS_OK, NYS_ERR_MAXIT, NYS_ERR_BREAKDOWN) */
  int32_t iterations;   /* PCG iterations at this shift (inner, summed, in mixed precision) */
  int32_t resketched;   /* 1 when a new factor was built for this shift */
  int32_t refinements;  /* mixed: outer refinement steps; FP64: 0 */
  int64_t ell;          /* sketch size of the factor used */
  double err_est;       /* Algorithm 4 estimate in force (NaN once the sketch reached ell_max) */
  double rel_residual;  /* as pcg_result.rel_residual */
} nys_path_result;

/* Regularization path with warm starts and factor reuse (the procedure of
 * the paper's path experiments, Sec. 6.2): (A + mu_i I) x_i = b for `count`
 * shifts, processed in DECREASING order of mu whatever the order of `mus`.
 * The first solve starts from zero, each later one from the previous shift's
 * solution.  A factor is built (Algorithm 5, Strategy 1, tolerance
 * err_factor * mu, q power steps, nu as nys_sketch_adaptive) for the first
 * shift, and rebuilt for a later shift only when the estimate in force
 * exceeds err_factor * mu and the sketch is still below ell_max; a rebuild
 * starts from twice the previous sketch size (capped at ell_max) with a fresh
 * test matrix.  The experiments use err_factor = 30, q = 5.
 *   mus      HOST [count], each > 0;
 *   b        device FP64 [n];  x  device FP64 [count][n], row i the solution for mus[i];
 *   omegas   device FP64 [count][n][ell_max] or NULL: the r-th factor build uses
 *            omegas + r n ell_max as its raw Gaussian test matrix (else drawn
 *            from seed + r);
 *   gs       device FP64 [count][kmax][n] or NULL, kmax = ceil(log2(ell_max / ell0)) + 1:
 *            the power-step starts of the r-th build (else drawn);
 *   opts     as for pcg_solve (precision applies to the sketches and the solves;
 *            use_x0 and residual_history are ignored);
 *   results  HOST [count], in the order of mus.
 * Returns the worst per-shift status or an error of the sketch or the
 * solver.  Synchronises `stream`. */
int32_t nys_reg_path(const nys_operator* op, int64_t count, const double* mus, const double* b,
                     double* x, int64_t ell0, int64_t ell_max, double err_factor, int32_t q,
                     uint64_t seed, const double* omegas, const double* gs,
                     const nys_pcg_opts* opts, nys_path_result* results, void* stream);

/* Read-only views of a factor's device arrays (valid until nys_factor_free):
 * U (n x ell row-major, FP64 when *u_dtype == NYS_F64 else FP32) and
 * lambda_hat (ell FP64, descending).  Any output pointer may be NULL. */
int32_t nys_factor_get(const nys_factor* f, const void** U, int32_t* u_dtype,
                       const double** lambda_hat, int64_t* n, int64_t* ell, double* nu);

/* Diagnostics of a factor (host outputs, each may be NULL): how many times
 * the shift nu was multiplied by 10 before the Cholesky factorisation of
 * Omega^T Y_nu succeeded (Algorithm 1), the number of FP32 block-Jacobi
 * sweeps of the thin SVD of the small factor, the number of FP64
 * eigen-refinement steps that followed them, and lambda_hat_ell. */
int32_t nys_factor_stats(const nys_factor* f, int32_t* shift_escalations, int32_t* svd_sweeps,
                         int32_t* svd_refinements, double* lambda_ell);

void nys_factor_free(nys_factor* f);

const char* nys_status_str(int32_t status);

/* Number of GPU kernels this library has launched in this process (all
 * devices, all threads).  A diagnostic: the difference across a call is the
 * number of kernels that call launched.  No paper counterpart. */
uint64_t nys_kernel_launch_count(void);

/* PCG launch mode (no counterpart in the paper).  With `on` = 1 (the
 * default, unless the environment sets NYS_PCG_GRAPH=0 before the first
 * solve) pcg_solve, the inner solves of the mixed path and the batched
 * solves capture four PCG iterations (Algorithm 3's loop body, every kernel
 * of it) once per solve as a CUDA graph and replay it between the host's
 * convergence checks; 0 launches the same kernels one by one on the stream.
 * Both modes run the same kernels in the same order and give bit-identical
 * results.  Where a capture is refused the solve falls back to plain
 * launches.  Returns the previous mode; any other `on` only queries it.
 * Process-wide; set it between solves, not during one. */
int32_t nys_pcg_graphs(int32_t on);

/* Device-side PCG loop (no counterpart in the paper).  With `on` = 1 (the
 * default, unless the environment sets NYS_PCG_LOOP=0 before the first
 * solve) and graph mode on, a PCG solve whose products allocate nothing
 * (FP32 products of every operator, FP64 products of the dense and ridge
 * operators) and whose products are not being timed runs its whole
 * iteration loop as ONE launch of a CUDA graph: a conditional WHILE node
 * repeats one iteration and a one-block kernel that ends the loop once every
 * system's done word is set or maxit iterations have run.  The host reads
 * the systems' states once per solve (in mixed precision: once per inner
 * solve).  Results are bit-identical to the replayed-chunk and plain modes.
 * Returns the previous mode; any other `on` only queries it.  Process-wide. */
int32_t nys_pcg_loop(int32_t on);

/* Mixed-precision solves of ONE system with a dense or ridge operator (no
 * counterpart in the paper; Gaussian-kernel systems always take the
 * refinement loop).  With `on` = 1 (the default, unless the environment sets
 * NYS_PCG_RELIABLE=0 before the first solve) pcg_solve runs a single FP32
 * recurrence of
 * Algorithm 3 with reliable updates: the iterate is kept in FP64, and each
 * time the recurrence residual has fallen by a factor 1e-3 (or met the
 * tolerance) the FP32 correction is folded into it, the true residual
 * b - (A + mu I) x is formed with FP64-accurate products and replaces the
 * recurrence residual, while the search direction is kept (residual
 * replacement).  Unlike restarted refinement this keeps the Krylov space, so
 * the solve takes about as many products as an FP64 one.  A replacement
 * that differs from the recurrence residual by more than a factor of two
 * restarts the search direction.  If the true residual stops halving between
 * replacements, or maxit iterations are spent, the system continues in the
 * escalating refinement loop described under nys_pcg_opts.maxit.
 * nys_pcg_result.refinements then counts the true-residual evaluations.
 * With 0, single systems take the refinement loop like batches do.  Returns
 * the previous mode; any other `on` only queries it.  Process-wide; set it
 * between solves. */
int32_t nys_pcg_reliable(int32_t on);

/* Launch-shape autotuner (no counterpart in the paper).  Where a kernel has
 * several correct launch shapes for one problem size (today: the number of
 * slices the points of a Gaussian kernel-matrix product are split into, for
 * one vector and for a batch of vectors), the first product of that size
 * times each shape with CUDA events and the fastest is used from then on.
 * Choices are kept per process and, when the environment names a file in
 * NYS_TUNE_CACHE, saved there as a JSON object {"key": choice, ...} and read
 * back by later processes.  Shapes that split a sum round its last bits
 * differently; every shape meets the same accuracy.
 *
 * nys_autotune: `on` = 1 times unseen sizes (the default unless NYS_TUNE=0),
 * 0 uses each launcher's own rule for them (cached choices still apply);
 * returns the previous mode, any other `on` only queries it.
 * nys_autotune_dump: writes the current choices as a NUL-terminated JSON
 * object into buf (at most cap bytes, truncated) and returns the full
 * length; buf may be NULL to query the length.
 * nys_autotune_clear: forgets every choice (the file is left alone and not
 * read again by this process).
 * nys_autotune_set: pins `choice` for `key` (a key as nys_autotune_dump
 * prints it); a choice that is not a candidate of the key is ignored at
 * launch and the sizes are timed again.  NYS_ERR_ARG for a NULL or empty
 * key. */
int32_t nys_autotune(int32_t on);
int64_t nys_autotune_dump(char* buf, int64_t cap);
void nys_autotune_clear(void);
int32_t nys_autotune_set(const char* key, int32_t choice);

/* Number of PCG iteration graphs replayed in this process (a diagnostic:
 * zero growth across a solve in graph mode means its capture was refused and
 * it ran on plain launches). */
uint64_t nys_pcg_graph_replays(void);

/* Diagnostics (no counterpart in the paper): CUDA-event timing of the FP32
 * operator products that mixed-precision PCG runs (the ridge or Gaussian
 * matvec) and of the dense products in FP64 and FP32, recorded on the stream
 * each product is launched on (inside a PCG iteration graph as event nodes
 * that every replay points at fresh events).
 * nys_timing_start allocates events for up to max_products products
 * (NYS_ERR_ARG if < 1; later products are not timed) and enables the
 * recording; nys_timing_stop waits for the recorded events, returns the
 * summed duration in ms and the number of products timed, and disables it.
 * Products shorter than a quarter of the median are left out of both: they
 * are launches for systems that had already converged (a replayed PCG
 * iteration past convergence), which return at once on the done word.
 * Not for concurrent use from several host threads. */
int32_t nys_timing_start(int32_t max_products);
int32_t nys_timing_stop(double* total_ms, int64_t* products);

/* y_s = (A + mu I) x_s for s = 0..nvec-1 (device FP64 [nvec][n]).  mode 0:
 * FP64 arithmetic (the product inside FP64 PCG); mode 1: the FP32 product
 * used inside mixed-precision PCG; mode 2: the FP64-accurate product of the
 * mixed path's refinement residual (double-FP32 arithmetic for the ridge
 * operator and the Gaussian kernel, ~2^-44 relative; FP64 for dense).
 * For the Gaussian kernel with d <= 32, mode 1 runs on the tensor cores
 * (FP16 hi/lo splits of points, kernel entries and vectors, three passes,
 * FP32 accuracy; 3xTF32 when the environment sets NYS_RBF_TF32=1 before the
 * first product), all nvec vectors in one pass over the kernel matrix.  Exposed so that each operator kernel can be checked on
 * its own.  Synchronises `stream`. */
int32_t nys_op_matvec(const nys_operator* op, double mu, int64_t nvec, const double* x, double* y,
                      int32_t mode, void* stream);

/* Algorithm 4: q power steps on E = A - U Lam U^T from the start vector g
 * (device FP64 [n]); *est (host) receives the estimate.  Synchronises. */
int32_t nys_power_err_est(const nys_operator* op, const nys_factor* f, const double* g, int32_t q,
                          double* est, void* stream);

/* Gaussian cross-kernel products for the kernel-ridge predictions and their
 * gradient (Sec. 6.5 uses k(x, y) = exp(-||x - y||^2 / (2 sigma^2))):
 *   kind 0: out_q[i] = sum_j k(t_i, x_j) v_q[j]
 *   kind 1: out_q[i] = sum_j k(t_i, x_j) ||t_i - x_j||^2 / sigma^3 v_q[j]
 *           (the derivative of kind 0 in sigma).
 * targets: nt x d FP32 (row stride ldt), points: n x d FP32 (row stride ldp),
 * v: device FP64 [nvec][n], out: device FP64 [nvec][nt], FP64 arithmetic.
 * K_v^T g is the same call with the roles of targets and points swapped (the
 * kernel is symmetric in its arguments).  1 <= d <= 64.  Synchronises. */
int32_t nys_rbf_cross_matvec(const float* targets, int64_t nt, int64_t ldt, const float* points,
                             int64_t n, int64_t ldp, int64_t d, double sigma, int64_t nvec,
                             const double* v, double* out, int32_t kind, void* stream);

/* Kernel ridge regression objective (Sec. 6.5, Eq. (6.3): KRR with the
 * Gaussian kernel, here with the validation mean squared error as the
 * objective) for alpha = (K + mu I)^{-1} b on the training points:
 *   pred = K_v alpha,   (K_v)_ij = exp(-||v_i - x_j||^2 / (2 sigma^2)),
 *   *loss (host) = mean_i (pred_i - yv_i)^2,
 *   g   = (2/m)(pred - yv)            (device FP64 [m], dL/dpred),
 *   ktg = K_v^T g                     (device FP64 [n], dL/dalpha: the
 *                                      right-hand side of the adjoint solve).
 * points: n x d FP32 (row stride ldp), vpoints: m x d FP32 (row stride ldv),
 * 1 <= d <= 64; alpha, yv: device FP64 [n], [m].  Products in double-FP32
 * arithmetic (~2^-44 relative), sums in FP64 in a fixed order.  g and ktg
 * must not alias each other or alpha.  Synchronises `stream`. */
int32_t nys_krr_validation(const float* points, int64_t n, int64_t ldp, const float* vpoints,
                           int64_t m, int64_t ldv, int64_t d, double sigma, const double* alpha,
                           const double* yv, double* loss, double* g, double* ktg, void* stream);

/* Gradient scalars of the KRR objective by implicit differentiation of the
 * training solve (the paper does not differentiate it): with
 * lam = (K + mu I)^{-1} dL/dalpha (the adjoint solve, which reuses the
 * training solve's Nystrom factor),
 *   out[0] = dL/dmu    = -lam^T alpha,
 *   out[1] = dL/dsigma = g^T (dK_v/dsigma) alpha - lam^T (dK/dsigma) alpha,
 *            dK_ij/dsigma = K_ij ||x_i - x_j||^2 / sigma^3,
 * (dL/db = lam itself).  vpoints may be NULL (g ignored): the objective then
 * depends on sigma only through alpha and out[1] = -lam^T (dK/dsigma) alpha.
 * Arrays as in nys_krr_validation; lam, alpha: device FP64 [n], g: device
 * FP64 [m]; out: HOST [2].  Synchronises `stream`. */
int32_t nys_krr_gradients(const float* points, int64_t n, int64_t ldp, const float* vpoints,
                          int64_t m, int64_t ldv, int64_t d, double sigma, const double* alpha,
                          const double* lam, const double* g, double* out, void* stream);

/* D = A B^T on the 5th-generation tensor cores: TF32 products (the low 13
 * mantissa bits of each FP32 operand are ignored), FP32 accumulation.  A is
 * M x K, B is N x K, D is M x N, all device FP32 row-major with leading
 * dimensions lda, ldb >= K and ldd >= N (lda, ldb multiples of 4; A and B
 * 16-byte aligned).  This is the kernel behind the mixed-precision sketch
 * Y = X^T (X Omega) of the ridge operator (Algorithm 1, step 3), exposed so
 * that it can be checked on its own.  NYS_ERR_ARG for unsupported shapes or
 * alignment.  Synchronises `stream`. */
int32_t nys_gemm_tf32_tn(int64_t M, int64_t N, int64_t K, const float* A, int64_t lda,
                         const float* B, int64_t ldb, float* D, int64_t ldd, void* stream);

/* Stream identifiers of the library's own random draws (see
 * nys_random_stream): Algorithm 1's Omega in nys_sketch; block k of
 * Algorithm 5 uses NYS_STREAM_ADAPTIVE + (the sketch size reached before
 * the block); the k-th start vector of Algorithm 4 inside
 * nys_sketch_adaptive uses NYS_STREAM_ESTIMATE + k. */
#define NYS_STREAM_OMEGA 0x4f6d656761ull
#define NYS_STREAM_ADAPTIVE 0x4164610000ull
#define NYS_STREAM_ESTIMATE 0x4573740000ull

/* Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11), the counter-based
 * generator behind Algorithm 1's Gaussian test matrix (step 1), applied to
 * caller-given blocks: out[4i..4i+3] = Philox4x32-10 of the counter
 * ctr[4i..4i+3] under the key key[2i..2i+1], for i < count.  ctr, key and
 * out are device uint32 arrays ([count][4], [count][2], [count][4]).
 * Exposed so that the bijection can be checked against the authors'
 * known-answer vectors.  NYS_ERR_ARG for count < 0 or a NULL array.
 * Synchronises `stream`. */
int32_t nys_philox4x32_10(const uint32_t* ctr, const uint32_t* key, int64_t count, uint32_t* out,
                          void* stream);

/* Elements [first, first + count) of the library's random stream
 * (seed, stream_id), the draw behind Algorithm 1 step 1 (Omega with i.i.d.
 * N(0, 1) entries) and the other NYS_STREAM_* draws.  Element e is word
 * e mod 4 of the Philox4x32-10 block of counter
 * (g mod 2^32, (g >> 32) ^ (stream_id mod 2^32), stream_id >> 32, 0x6e79)
 * under key (seed mod 2^32, seed >> 32), g = e / 4.  words (device uint32
 * [count]) receives those raw words; gauss (device FP64 [count]) receives
 * the Box-Muller values: with u(w) = ((w >> 9) + 1/2) 2^-23 (exact in FP32)
 * and a block's words w0..w3, element 0 is sqrt(-2 ln u(w0)) cos(2 pi u(w1)),
 * element 1 the same radius times sin(2 pi u(w1)), elements 2 and 3 likewise
 * from w2, w3; computed in FP32 (logf, sqrtf, sincospif) and widened, within
 * 4e-6 of the exact transform of the same words.  Either output may be
 * NULL, not both.  nys_sketch(seed) uses elements [0, n ell) of stream
 * (seed, NYS_STREAM_OMEGA) as its row-major n x ell Omega.
 * NYS_ERR_ARG for first < 0 or count < 0.  Synchronises `stream`. */
int32_t nys_random_stream(uint64_t seed, uint64_t stream_id, int64_t first, int64_t count,
                          uint32_t* words, double* gauss, void* stream);

/* Measured throughput of one execution unit on the current device (no
 * counterpart in the paper; the denominator of the roofline fractions of the
 * ALU-bound kernels): unit 0 = FP64 FMA pipe, 1 = FP32 FMA pipe (both in
 * FLOP/s, an FMA counting 2), 2 = MUFU ex2.approx (operations/s).  Runs
 * independent register-resident dependency chains on every SM, one untimed
 * launch then one timed with CUDA events on `stream` (tens of ms).
 * *ops_per_s (host) receives the rate.  NYS_ERR_ARG for another unit.
 * Synchronises `stream`. */
int32_t nys_unit_peak(int32_t unit, double* ops_per_s, void* stream);

/* Allocation-free ridge matvec: y = (X^T X + mu I) x in FP32 for an
 * NYS_OP_GRAM operator, computed by the same fused single-pass kernel as the
 * mixed-precision PCG matvec.  The paper has no counterpart; this exists for
 * callers that cannot allocate device memory during the call -- for example
 * code whose device memory is entirely reserved up front by another
 * framework's pool, or latency-bound loops that cannot afford the implicit
 * device synchronisation an allocation may cause.  Those callers still pass
 * x and y (device FP32 [n], 16-byte aligned, distinct); everything else the
 * kernel needs lives in one file-scope device array of 4 MiB + 256 bytes,
 * which every GPU that loads this library holds until the process exits.
 * Limit: n <= 6400 with n a multiple of 4 (the kernel's two-stage
 * shared-memory pipeline holds 2 x 4 rows of X in 200 KiB); X must be
 * row-contiguous (ld == n) and 16-byte aligned.  The partials also need
 * (number of SMs) x n <= 2^20 floats, which n <= 6400 implies on GPUs of up
 * to 163 SMs (the check stays for larger ones).
 * Larger or unsupported shapes return NYS_ERR_ARG without touching the GPU.
 * The first call on a device looks up the array's device address (with that
 * device current) and caches it; make that first call before any stream
 * capture.  cudaDeviceReset destroys the array with the device's context:
 * do not call this entry point after it in the same process.  Every call
 * shares the array and leaves its contents behind: the timeout word is
 * cleared at the start of each call and the partials are fully overwritten,
 * but calls that overlap on the GPU (several streams or threads at once)
 * race on the array and give wrong results.  Calls no cudaMalloc, cudaFree
 * or allocating library routine.  Synchronises `stream`; NYS_ERR_TIMEOUT if
 * a bounded device wait expired, in which case y is left unchanged. */
int32_t nys_gram_matvec_f32_noalloc(const nys_operator* op, double mu, const float* x, float* y,
                                    void* stream);

#ifdef __cplusplus
}
#endif

#endif /* NYSPCG_H */
