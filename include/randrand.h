/*
 * randrand.h -- C ABI of the GB300 RandRAND-PCG library.
 *
 * RandRAND (Randomized RANge Deflation; arXiv 2509.19747) preconditions a
 * Krylov solver for the shifted system
 *
 *     (A + mu I) x = b,   A symmetric positive semidefinite, mu >= 0
 *                                              (Sec. 1, eq:initsys)
 *
 * by orthogonal projection onto range(A_mu Omega), A_mu = A + mu I, where
 * Omega is a random n x k test matrix (Sec. 1.1 eq:testmatrix, q = 0).
 * The library builds the preconditioner once per (A, mu, k, seed) and then
 * solves for any number of right-hand sides.  Every floating-point step
 * runs in this library's own CUDA kernels on the GPU; there is no host
 * fallback.
 *
 * Conventions for every entry point:
 *   - Pointers named "device" must point to GPU global memory of the
 *     current device; the caller allocates and owns that memory.  The
 *     library allocates no device memory: all scratch lives in the
 *     caller-provided workspace (randrand_workspace_bytes).
 *   - All GPU work is enqueued on the stream given to randrand_build
 *     (a cudaStream_t passed as void*; NULL = the legacy default stream).
 *   - Every function returns an rr_status and never aborts.  Arguments are
 *     validated on the host before any launch; on an error return nothing
 *     has been written to caller buffers unless stated otherwise.
 *   - Matrices are row-major unless stated otherwise; right-hand sides and
 *     solutions are column-major (column j starts at ptr + j * ld).
 */
#ifndef RANDRAND_H
#define RANDRAND_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t rr_status;
enum {
  RR_OK = 0,
  RR_ERR_INVALID_ARG = 1,   /* a size, pointer, option or value is invalid */
  RR_ERR_WORKSPACE = 2,     /* workspace smaller than randrand_workspace_bytes */
  RR_ERR_NOT_SPD = 3,       /* a k x k Gram / core matrix is not positive definite */
  RR_ERR_BREAKDOWN = 4,     /* p^T A_mu p <= 0 or a non-finite Krylov scalar */
  RR_ERR_MAXIT = 5,         /* iteration budget reached before rtol; x holds the last iterate */
  RR_ERR_TIMEOUT = 6,       /* a bounded device-side wait gave up */
  RR_ERR_CUDA = 7,          /* a CUDA runtime call failed */
  RR_ERR_UNSUPPORTED = 8,   /* the combination of options is not implemented */
  RR_PENDING = 9            /* server request queued or running (rr_server_poll) */
};

/* Operator kinds: A is only accessed through u -> A u (Sec. 1) */
enum {
  RR_OP_DENSE = 0,          /* explicit n x n symmetric matrix */
  RR_OP_CSR = 1,            /* sparse symmetric matrix, CSR, int32 indices */
  RR_OP_GAUSS_KERNEL = 2    /* K_ij = exp(-|x_i - x_j|^2 / (2 h^2)), generated on the fly */
};

/* Test matrices Omega = X^T (Sec. 2) */
enum {
  RR_SKETCH_GAUSSIAN = 0,    /* entries N(0, 1/k) */
  RR_SKETCH_SPARSE_SIGN = 1, /* gamma entries +-1/sqrt(gamma) per row of Omega */
  RR_SKETCH_SRHT = 2,        /* subsampled randomized Hadamard transform (Sec. 2):
                                Omega = X^T, X = k^-1/2 S H D, the first n of
                                s = 2^ceil(log2 n) columns; entries +-1/sqrt(k) */
  RR_SKETCH_MULTILEVEL = 3   /* multi-level embedding X = X2 X1 (Sec. 2
                                eq:multilevelose): X1 a sparse random operator
                                (opts.ml_l1 x n, opts.ml_gamma entries
                                +-1/sqrt(ml_gamma) per column), X2 Gaussian
                                (k x ml_l1, entries N(0, 1/k)); Omega = X1^T X2^T.
                                Needs opts.ml_gamma >= 1 (see
                                rr_multilevel_defaults).  In the basis-less CSR
                                form Omega is applied as the two factors */
};

/* Arithmetic of the path */
enum {
  RR_PREC_FP64 = 0,         /* everything in float64 */
  RR_PREC_FP32 = 1,         /* float32 sketch, iterations and restart residual ("plain form") */
  RR_PREC_MIXED = 2         /* bf16 sketch with fp32 accumulation, fp32 iterations,
                               float64-accurate restart residual (iterative refinement) */
};

/* Preconditioner variants */
enum {
  RR_VARIANT_C = 0,         /* C-RandRAND PCG (Sec. 3.2, Alg. 7) */
  RR_VARIANT_R = 1,         /* R-RandRAND CG on B y = b, x = P y (Sec. 3.1, Alg. 4) */
  RR_VARIANT_G = 2          /* G-RandRAND MINRES (Sec. 3.3 eq:g_randrand, Sec. 6.3):
                               P = (I - Pi) + tau Q G Q^T, G = (R^-T Omega^T Omega
                               R^-1)^(1/2), for symmetric A_mu that may be
                               indefinite (mu < 0 allowed); explicit basis only
                               (orth CHOLQR2) */
};

/* Orthogonalisation of Y_mu = A_mu Omega */
enum {
  RR_ORTH_CHOLQR2 = 0,      /* Cholesky QR applied twice (Sec. 4.2 Alg. 2 as first pass) */
  RR_ORTH_RAND_CHOLQR = 1   /* Alg. 3, randomized Q-less QR: S = Theta Y_mu (Theta a
                               sparse-sign l_sk x n embedding), R_sk from a float64
                               Cholesky QR of S, W = Y_mu R_sk^-1, R = chol(W^T W) R_sk.
                               With a CSR operator no basis is kept (Sec. 4.2
                               basis-less form: Q^T v = R^-T Omega^T A_mu v and
                               Q s = A_mu Omega R^-1 s; variant C with three
                               products with A_mu per iteration, variant R with
                               five and four for the recovery; variant G:
                               RR_ERR_UNSUPPORTED); other operators form
                               Q = W chol(W^T W)^-1. */
};

/*
 * Operator description.  Borrowed: every pointer must stay valid and
 * unchanged until randrand_free of each handle built from it.
 *   kind = RR_OP_DENSE:   dense (device) n x n row-major with leading
 *                         dimension ld >= n, element type dtype
 *                         (0 = float64, 1 = float32); must be symmetric.
 *   kind = RR_OP_CSR:     rowptr (device, n+1 int32), colidx (device, nnz
 *                         int32, sorted per row), vals (device, nnz, dtype);
 *                         the matrix must be symmetric.
 *   kind = RR_OP_GAUSS_KERNEL: points (device, n x dim float32 row-major),
 *                         bandwidth h > 0; A = K is never stored.
 */
typedef struct {
  int32_t kind;
  int32_t dtype;
  int64_t n;
  const void* dense;
  int64_t ld;
  const int32_t* rowptr;
  const int32_t* colidx;
  const void* vals;
  int64_t nnz;
  const float* points;
  int32_t dim;
  int32_t pad_;
  double bandwidth;
} rr_operator;

typedef struct {
  int32_t variant;       /* RR_VARIANT_*                          default C      */
  int32_t precision;     /* RR_PREC_*                             default FP64   */
  int32_t orth;          /* RR_ORTH_*                             default CHOLQR2 */
  int32_t gamma;         /* nonzeros per row of a sparse-sign Omega, default 8  */
  int32_t l_sk;          /* rows of Theta for RAND_CHOLQR (0 -> 4k)             */
  int32_t gamma_sk;      /* nonzeros per column of Theta, default 8             */
  int32_t power_iters;   /* power iterations per estimate, default 20           */
  int32_t max_rhs;       /* right-hand sides a solve may pass (1..8), default 1 */
  int32_t profile;       /* 1: time the hot kernels with CUDA events (rr_profile) */
  int32_t kernel_impl;   /* Gaussian-kernel sketch (RR_PREC_MIXED) and float32
                            products (FP32 / MIXED), dim == 8: 0 auto (tensor
                            cores), 1 float32 cores only, 2 tensor cores required
                            (exponent arguments on the tensor cores, K v on the
                            float32 cores), 3 tensor cores for both (K split into
                            two bf16 parts, K v by a second tcgen05 product);
                            other values: RR_ERR_INVALID_ARG */
  int32_t iter_impl;     /* variant C with a basis: 0 auto (one persistent
                            cooperative launch per iteration for everything
                            after the operator product), 1 separate kernels;
                            basis-less CSR form: 0 one persistent launch per
                            chunk of iterations, in its shared-memory window
                            form (four grid barriers per iteration) when each
                            CTA's rows and the rows they read fit, 1 separate
                            kernels, 2 the persistent launch without windows
                            (seven grid barriers); elsewhere 2 acts as 0;
                            other values: RR_ERR_INVALID_ARG */
  int32_t q;             /* power of the test matrix Omega = A^q X^T
                            (eq:testmatrix), 0..4, default 0; q >= 1 costs q
                            more sketch products and is not available with the
                            basis-less CSR form */
  double rho;            /* C variant: <= 0 -> eq:optimal_rho with F = 1/mu     */
  double restart_eta;    /* restart after this residual reduction, default 1e-2 */
  int32_t keep_sketch;   /* 1: keep A Omega and the shift-free projections
                            Omega^T A^T A Omega, Omega^T A Omega, Omega^T Omega
                            (Sec. 5.1) so that randrand_set_mu can rebuild the
                            preconditioner for another shift without a new
                            sketch product; costs one more n x k array.
                            2: the joint basis instead (Sec. 5.1): Q_joint
                            with range(Q_joint) = range([Omega, A Omega]), C1 =
                            Q_joint^T A Omega and C2 = Q_joint^T Omega; a shift
                            then takes R from a float64 Cholesky QR of the 2k x k
                            C1 + mu C2 (never the Gram of an n-row matrix) and
                            Q = Q_joint Q_red; costs 3 more n x k arrays and
                            fails with RR_ERR_NOT_SPD when A Omega adds no
                            direction to Omega.  Variant C with an explicit
                            basis (orth CHOLQR2) and q = 0 only (else
                            RR_ERR_UNSUPPORTED).  Default 0 */
  int32_t ml_l1;         /* RR_SKETCH_MULTILEVEL: rows l1 of X1, k <= l1 <= 2^24 */
  int32_t ml_gamma;      /* RR_SKETCH_MULTILEVEL: nonzeros per column of X1,
                            1..16, <= ml_l1.  0 (the default) reserves no
                            workspace for the multi-level factors, and a
                            multi-level build then fails with
                            RR_ERR_INVALID_ARG */
  int32_t refine;        /* 1: refined projector (Sec. 4.3 eq:accurate_proj):
                            Pi ~ Q T Q^T and Pi A_mu^-1 Pi ~ Q T G T Q^T with
                            the Neumann T = 2 I - Q^T Q of the stored basis,
                            so P = I + Q (tau T G T - T) Q^T; one k x k Gram
                            at build, no cost per iteration.  s = 2..8: the
                            refinement recurrence of eq:accurate_proj_2 with
                            s steps beyond the first (v_1 = Q^T u, v_{i+1} =
                            v_i + Q^T (u - Q v_i)), whose result is the
                            polynomial T = sum_{j <= s} (I - Q^T Q)^j applied
                            to Q^T u: T is formed once at build (s - 1 more
                            k x k products).  Variants C and G with an
                            explicit basis (else RR_ERR_UNSUPPORTED); other
                            values RR_ERR_INVALID_ARG.  0 (default): plain
                            Q Q^T */
} rr_build_opts;

typedef struct {
  int32_t inner_iters;   /* Krylov iterations, summed over restarts           */
  int32_t outer_iters;   /* restarts (= refinement steps)                     */
  int32_t matvecs;       /* products with A_mu in the solve                    */
  rr_status status;      /* RR_OK, RR_ERR_MAXIT or RR_ERR_BREAKDOWN            */
  double rel_residual;   /* |b - A_mu x| / |b|, evaluated by the restart residual */
  double tau;            /* preconditioner coefficient                         */
  double normE;          /* power-iteration estimate of |(I-Pi) A_mu (I-Pi)|   */
  double lam_max;        /* estimate of lambda_max(Pi A_mu Pi~) (C variant)    */
} rr_solve_info;

/* Per-kernel device time of a profiled handle (opts.profile = 1), summed
 * over its build and solves: launches and milliseconds measured with CUDA
 * events recorded on the handle stream around each launch. */
enum {
  RR_PROF_SKETCH = 0,     /* Y_mu = A_mu Omega                                   */
  RR_PROF_MATVEC = 1,     /* A_mu p in the Krylov iterations (working precision) */
  RR_PROF_RESIDUAL = 2,   /* A_mu x of the restart residual                      */
  RR_PROF_POWER = 3,      /* A_mu u in the power iterations                      */
  RR_PROF_COUNT = 8
};
typedef struct {
  int32_t launches[RR_PROF_COUNT];
  double ms[RR_PROF_COUNT];
} rr_profile;

typedef struct rr_handle rr_handle;

/* Fill *o with the defaults listed in rr_build_opts. */
void rr_build_opts_default(rr_build_opts* o);

/* Set o->ml_gamma and o->ml_l1 to the multi-level embedding of the paper's
 * sparse + Gaussian experiment (Sec. 7): gamma1 = ceil(ln n) (at most 16)
 * nonzeros per column of X1 and l1 = gamma1 k rows.  Other fields are left
 * as they are.  No-op when o is NULL, n < 1 or k < 1. */
void rr_multilevel_defaults(int64_t n, int32_t k, rr_build_opts* o);

/* Human-readable name of a status code (static string, never NULL). */
const char* randrand_status_str(rr_status s);

/*
 * Device bytes the handle needs for (A, k, opts): the test matrix, the basis
 * Q (and Y_mu while building), the k x k factors, the power-iteration and
 * Krylov state for opts->max_rhs columns and all reduction scratch.
 * Host only; touches no device memory.  Errors: RR_ERR_INVALID_ARG.
 */
rr_status randrand_workspace_bytes(const rr_operator* A, int32_t k,
                                   const rr_build_opts* opts, size_t* bytes);

/*
 * Build the RandRAND preconditioner: Alg. 7 steps 1-4 (variant C) or Alg. 4
 * steps 1-2 (variant R), with the basis-explicit representation of Sec. 4.1.
 *   A          operator (see rr_operator); borrowed.
 *   mu         shift, >= 0 and finite.
 *   k          sketch dimension l of the paper, 1 <= k <= n.
 *   sketch     RR_SKETCH_GAUSSIAN, RR_SKETCH_SPARSE_SIGN, RR_SKETCH_SRHT or
 *              RR_SKETCH_MULTILEVEL.
 *   seed       64-bit key of the counter-based generator that draws Omega,
 *              Theta and the power-iteration start vectors.
 *   opts       NULL for defaults.
 *   workspace  device buffer of ws_bytes >= randrand_workspace_bytes(),
 *              256-byte aligned; owned by the caller, used exclusively by
 *              the handle until randrand_free.
 *   stream     cudaStream_t (as void*) for all work of this handle.
 *   out        receives a host-allocated handle (free with randrand_free).
 * Synchronises the stream once at the end (to read the tau estimates).
 * Errors: RR_ERR_INVALID_ARG, RR_ERR_WORKSPACE, RR_ERR_NOT_SPD (Y_mu
 * numerically rank deficient even after a shifted Cholesky retry),
 * RR_ERR_UNSUPPORTED, RR_ERR_CUDA.  On error *out is NULL.
 */
rr_status randrand_build(const rr_operator* A, double mu, int32_t k, int32_t sketch,
                         uint64_t seed, const rr_build_opts* opts, void* workspace,
                         size_t ws_bytes, void* stream, rr_handle** out);

/*
 * Solve A_mu X = B with the handle's preconditioner: PCG (variant C,
 * Alg. 7 steps 5-11) or CG on B y = r with recovery x = P y (variant R,
 * Alg. 4 steps 3-9), restarted after each residual reduction by
 * restart_eta (Sec. 7 setup).  Each restart recomputes r = b - A_mu x
 * (float64-accurate for RR_PREC_FP64 and RR_PREC_MIXED).
 *   b       device, n x nrhs float64, column-major, leading dimension ldb >= n.
 *   x       device, n x nrhs float64, column-major, ldx >= n.  On entry the
 *           initial guess if x_is_guess != 0 (else ignored); on exit the
 *           solution, also for RR_ERR_MAXIT.
 *   nrhs    1 <= nrhs <= opts.max_rhs of the build.
 *   rtol    stop when |b - A_mu x| <= rtol |b| for every column.
 *   maxit   budget of Krylov iterations per column (summed over restarts).
 *   info    host array of nrhs entries (may be NULL).
 * A zero column of b gets x = 0 (RR_OK); a column of b holding a NaN or an
 * Inf ends at once with RR_ERR_BREAKDOWN (0 iterations) while the other
 * columns solve.
 * Synchronises the stream.  Returns RR_OK when every column met rtol,
 * otherwise the worst per-column status.  Errors: RR_ERR_INVALID_ARG,
 * RR_ERR_CUDA.
 */
rr_status randrand_solve(rr_handle* h, const double* b, int32_t nrhs, int64_t ldb,
                         double* x, int64_t ldx, int32_t x_is_guess, double rtol,
                         int32_t maxit, rr_solve_info* info);

/*
 * Same as randrand_solve with host buffers (pageable or pinned): b is
 * copied to the device and x back inside the call.  b, x column-major
 * n x nrhs float64 with leading dimensions ldb, ldx.
 */
rr_status randrand_solve_host(rr_handle* h, const double* b_host, int32_t nrhs,
                              int64_t ldb, double* x_host, int64_t ldx, double rtol,
                              int32_t maxit, rr_solve_info* info);

/* Release a handle (host memory only; the workspace stays the caller's).
 * NULL is accepted.  Never fails.  Synchronises the handle's stream. */
void randrand_free(rr_handle* h);

/*
 * Rebuild the preconditioner of h for the shift mu (Sec. 5.1, multiple
 * shifting parameters): Y_mu = A Omega + mu Omega from the kept A Omega; the
 * first Cholesky QR pass takes its Gram from the shift-free projections,
 * (A Omega + mu Omega)^T (A Omega + mu Omega) = Omega^T A^T A Omega +
 * 2 mu Omega^T A Omega + mu^2 Omega^T Omega, the second pass orthogonalizes
 * the result as in the build; then Omega^T A_mu Omega = Omega^T A Omega + mu
 * Omega^T Omega for G, the power iterations for tau, and Q H.  With
 * keep_sketch = 2 the factors come from the joint basis instead: R = R(C1 +
 * mu C2) and Q = Q_joint (C1 + mu C2) R^-1.  Later solves use mu.
 * Synchronous on the handle stream.
 *   h   a handle built with opts.keep_sketch = 1 or 2.
 *   mu  new shift, >= 0 and finite.
 * Errors: RR_ERR_INVALID_ARG (h NULL, mu < 0 or not finite),
 * RR_ERR_UNSUPPORTED (handle built without keep_sketch), RR_ERR_NOT_SPD,
 * RR_ERR_TIMEOUT, RR_ERR_CUDA.  On an error the handle must not be used
 * for solves until a successful randrand_set_mu.
 */
rr_status randrand_set_mu(rr_handle* h, double mu);

/*
 * Test and inspection hooks (used by the parity tests): copy device-resident
 * build products into caller device buffers, enqueued on the handle stream.
 *   what = 0: Omega  (n x k row-major, float64)
 *          1: Q      (n x k row-major, float64; RR_ERR_UNSUPPORTED for a
 *                     basis-less build, which keeps no Q)
 *          2: R      (k x k row-major, float64, upper triangular)
 *          3: G      (k x k row-major, float64; C variant core matrix)
 *   dst   device buffer of float64 of the stated size.
 * Errors: RR_ERR_INVALID_ARG, RR_ERR_UNSUPPORTED, RR_ERR_CUDA.
 */
rr_status randrand_export(rr_handle* h, int32_t what, double* dst);

/* Profile of a handle built with opts.profile = 1 (zeros otherwise).
 * Synchronises the handle stream.  Errors: RR_ERR_INVALID_ARG, RR_ERR_CUDA. */
rr_status randrand_profile(rr_handle* h, rr_profile* out);

/* Scalars of a handle: tau, |E| estimate, lambda_max estimate. */
rr_status randrand_scalars(const rr_handle* h, double* tau, double* normE, double* lam_max);

/*
 * Jitter of the last core-matrix factorization (variant C, remark after
 * Alg. 7; App. C): 0 when M = sym(Omega^T A_mu Omega) factored as it is,
 * else the alpha of the ladder, the smallest of 10^-14 |M|, ..., 10^-1 |M|
 * for which M + alpha I factors, |M| the spectral norm of M (estimated by
 * 30 power iterations on the k x k M).  Host only; *alpha is written.
 * Errors: RR_ERR_INVALID_ARG (h or alpha NULL).
 */
rr_status randrand_core_jitter(const rr_handle* h, double* alpha);

/*
 * Apply the preconditioner (variants C and G: z = P r, P = I + Q H Q^T with
 * H = tau G - I, the footnote form of Sec. 7.3, or H = tau T G T - T with
 * opts.refine) or the operator B of variant R
 * (z = (I-Pi) A_mu (I-Pi) r + tau Pi r, eq:APdef2) to m <= max_rhs columns.
 *   r, z  device, n x m float64 column-major with leading dimension ld.
 * Enqueued on the handle stream; does not synchronise.
 */
rr_status randrand_apply(rr_handle* h, const double* r, double* z, int32_t m, int64_t ld);

/*
 * Product with the shifted operator in the handle's working precision
 * (float32 for RR_PREC_FP32 / RR_PREC_MIXED, the arithmetic of the Krylov
 * iterations), w = (A + mu I) v.  v, w device n x m float64 column-major
 * (converted at the boundary), ld >= n, m <= max_rhs.  Test hook.
 */
rr_status randrand_apply_operator(rr_handle* h, const double* v, double* w, int32_t m, int64_t ld);

/*
 * Product with the shifted operator, w = (A + mu I) v, float64 accurate
 * (the restart residual's arithmetic).  v, w device n x m float64
 * column-major, leading dimension ld; m <= max_rhs.
 */
rr_status randrand_matvec(rr_handle* h, const double* v, double* w, int32_t m, int64_t ld);

/*
 * Several built systems solved together in shared rounds.  Each round
 * advances every system's Krylov iteration once.  The round is one
 * persistent launch of the tensor-core kernel product over all systems'
 * (row pair, point tile) work items, plus one cooperative launch of the
 * persistent PCG step, in which each system gets a share of the SMs and
 * its own grid barrier.  A CUDA graph captures R rounds once.  Its kernels
 * read the group's system tables from device memory, so the same graph
 * serves the group while systems finish.  Between replays the host reads
 * every system's column states in one copy.  It runs the restarts
 * (float64-accurate residual, Alg. 7 step 10) of the systems whose inner
 * solves ended, and drops the systems that are done.  R, the rounds per
 * replay, is tuned on the first replays of each (columns, log2 mean n,
 * log2 mean k) class and then cached for the process.  Results equal
 * randrand_solve's up to the summation order of the split sums.  The paper
 * solves one system; this is a scheduling of its iterations for many.
 *   hs          nsys (1..152) distinct built handles that iterate in float32
 *               with the tensor-core product and the persistent step:
 *               RR_OP_GAUSS_KERNEL in d = 8, RR_PREC_FP32 or RR_PREC_MIXED,
 *               variant C, explicit basis, iter_impl 0, kernel_impl 0 or 2,
 *               profile 0, all with the same column count (max_rhs rounded
 *               up to a power of two); else RR_ERR_UNSUPPORTED.
 *   rhs         per system: b, x (device, column-major, as randrand_solve),
 *               nrhs <= opts.max_rhs, rtol, maxit.
 *   workspace   device, >= randrand_group_workspace_bytes(hs, nsys), 256-byte
 *               aligned, caller-owned: the handles' augmented point arrays
 *               stacked, the system tables, each system's partial sums.
 *   stream      cudaStream_t of all group work, not the legacy default
 *               stream (NULL: RR_ERR_INVALID_ARG).  While it runs each handle
 *               is moved to this stream, then back to its own.
 *   info        host, 8 entries per system (info[8 i + c]), may be NULL.
 * Synchronous.  Returns RR_OK when every system converged, else the first
 * non-OK status in input order.  Errors: RR_ERR_INVALID_ARG,
 * RR_ERR_UNSUPPORTED, RR_ERR_WORKSPACE, RR_ERR_CUDA, RR_ERR_TIMEOUT.
 */
typedef struct {
  const double* b;
  int64_t ldb;
  double* x;
  int64_t ldx;
  int32_t nrhs;
  int32_t maxit;
  double rtol;
} rr_group_rhs;
rr_status randrand_group_workspace_bytes(rr_handle* const* hs, int32_t nsys, size_t* bytes);
rr_status randrand_solve_group(rr_handle* const* hs, int32_t nsys, const rr_group_rhs* rhs,
                               void* workspace, size_t ws_bytes, void* stream, rr_solve_info* info);

/*
 * Allocation-free float64-accurate Gaussian-kernel product
 *     w = (K + mu I) v,   K_ij = exp(-|p_i - p_j|^2 / (2 h^2)),
 * the same double-float arithmetic as the restart residual of
 * RR_PREC_MIXED (randrand_matvec on such a handle), for callers that cannot
 * allocate device memory at the point of use: a plugin inside a framework
 * that owns all device memory through its own pool, a serving loop that
 * bans allocator calls on its hot path, a process whose memory is fully
 * committed.  The paper has no counterpart of this entry point; it exists
 * for those callers only.
 *   points  device, n x dim float32 row-major (dim <= 16); bandwidth h > 0.
 *   v, w    device, n x m float64 column-major, leading dimension ld >= n;
 *           1 <= m <= 8.  Caller-owned.
 *   stream  cudaStream_t (as void*) of the current device (a stream of
 *           another device: RR_ERR_INVALID_ARG).  Enqueued only; does not
 *           synchronise.
 * Scratch: a fixed 32 MiB static device array inside the library (held on
 * every GPU that loads it until the library is unloaded), nothing else; no
 * cudaMalloc, cudaFree or allocating library call.  Limit: with mp the
 * smallest power of two >= m, 16 * n * mp + 8 * n + 8 * n * mp bytes
 * (rounded up to 256-byte blocks) must fit in 32 MiB, else RR_ERR_WORKSPACE
 * and nothing is launched.  All calls share the array: calls that overlap
 * on the GPU race; serialise them.  Nothing in it needs to start at zero.
 * Each call outside stream capture looks up the array's device address on
 * the current device (and the first such call loads the library's module
 * there); a call on a capturing stream reuses the address of the last
 * uncaptured call on that device, so make the first call on each device
 * before any stream capture.  An error already pending in the CUDA runtime
 * when the call starts is left in place and reported as RR_ERR_CUDA with
 * nothing launched.  Errors: RR_ERR_INVALID_ARG, RR_ERR_WORKSPACE,
 * RR_ERR_CUDA.
 */
rr_status randrand_kernel_matvec_noalloc(const float* points, int64_t n, int32_t dim,
                                         double bandwidth, double mu, const double* v, double* w,
                                         int32_t m, int64_t ld, void* stream);

/* ======================================================================
 * Many systems on one GPU: batched execution and a serving loop.
 * Neither is in the paper; they run its solver (randrand_build +
 * randrand_solve + randrand_free per system) for many independent systems
 * at once.  Worker threads of the library each own a CUDA stream and run
 * one system at a time in a slice of a caller-provided device arena; the
 * kernels of the systems resident at the same time overlap on the GPU.
 * ====================================================================== */

/* One system to solve.  Everything the pointers reference is borrowed until
 * the request has completed (its result is no longer RR_PENDING). */
typedef struct {
  rr_operator op;
  double mu;
  int32_t k;
  int32_t sketch;          /* RR_SKETCH_*                                     */
  uint64_t seed;
  rr_build_opts opts;      /* opts.max_rhs >= nrhs                            */
  const double* b;         /* device, n x nrhs column-major, leading dim ldb */
  double* x;               /* device, n x nrhs column-major, leading dim ldx:
                              the solution, written before completion        */
  int64_t ldb;
  int64_t ldx;
  int32_t nrhs;            /* 1..8                                            */
  int32_t maxit;
  double rtol;
} rr_request;

/* Outcome of one request.  Times are host wall-clock milliseconds since the
 * server (or batch) was created: submit, admission (start) and completion
 * (end); queue = start - submit, build and solve are the two phases. */
typedef struct {
  rr_status status;        /* RR_PENDING until done, then the solve's status
                              (or the build's, if the build failed)          */
  int32_t nrhs;
  size_t ws_bytes;         /* arena bytes the request held                    */
  double submit_ms, start_ms, end_ms;
  double queue_ms, build_ms, solve_ms;
  rr_solve_info info[8];   /* per right-hand side                             */
  int32_t rounds;          /* 1: its iterations ran in the shared rounds      */
  int32_t pad_;
} rr_result;

/* First-fit allocator of the serving loop over byte offsets [0, bytes),
 * 256-byte granularity, neighbouring free blocks coalesced.  Host only (no
 * CUDA call); exposed for inspection and tests.  alloc returns
 * RR_ERR_WORKSPACE when no free block is large enough; free returns
 * RR_ERR_INVALID_ARG for an offset that is not allocated. */
typedef struct rr_arena rr_arena;
rr_status rr_arena_create(size_t bytes, rr_arena** out);
rr_status rr_arena_alloc(rr_arena* a, size_t bytes, size_t* offset);
rr_status rr_arena_free(rr_arena* a, size_t offset);
rr_status rr_arena_stats(const rr_arena* a, size_t* in_use, size_t* largest_free);
void rr_arena_destroy(rr_arena* a);

/*
 * Serving loop.  rr_server_create: `arena` (device, 256-byte aligned,
 * caller-owned, arena_bytes >= 256) is the HBM budget shared by all resident
 * requests; `workers` (1..256) threads on the current device.  Requests are
 * admitted in arrival order: the oldest waiting request starts as soon as a
 * worker is idle and randrand_workspace_bytes of it fits in the arena.
 * rr_server_submit copies the request and returns a ticket at once
 * (RR_ERR_WORKSPACE if the request could never fit, RR_ERR_INVALID_ARG on
 * bad arguments).  rr_server_poll fills *out for a ticket (wait != 0: block
 * until it is done).  rr_server_drain waits until every submitted request is
 * done.  rr_server_destroy drains, then stops the workers.
 */
typedef struct rr_server rr_server;
rr_status rr_server_create(void* arena, size_t arena_bytes, int32_t workers, rr_server** out);
rr_status rr_server_submit(rr_server* s, const rr_request* req, uint64_t* ticket);
rr_status rr_server_poll(rr_server* s, uint64_t ticket, int32_t wait, rr_result* out);
rr_status rr_server_drain(rr_server* s);
rr_status rr_server_stats(rr_server* s, int32_t* queued, int32_t* running, size_t* bytes_in_use,
                          size_t* peak_bytes);
void rr_server_destroy(rr_server* s);

/*
 * Shared rounds in the serving loop and the batch (see randrand_solve_group):
 * systems whose handles qualify for the rounds (and have mp columns and
 * k <= kmax) are handed, once built, to one executor thread that joins them
 * into its running group at the next replay boundary and completes each
 * request when its system is done; the others are solved by their worker as
 * before.  Continuous batching: requests that arrive while others iterate
 * join the same rounds as soon as they are built and the group has room.
 *   mp           columns of the group: max_rhs rounded up to a power of two,
 *                at least 2 (2, 4 or 8)
 *   kmax         largest sketch dimension k of a system in the rounds
 *   max_systems  systems resident in the rounds at once (1..152)
 *   max_rows     stacked rows: sum over resident systems of n rounded up to
 *                a multiple of 256
 * The group's workspace (rr_rounds_workspace_bytes) is taken from the front
 * of the arena given to rr_server_create_rounds / randrand_solve_batch_rounds;
 * the rest is the HBM budget of the handles.  A built system that does not
 * fit the group now waits for others to leave (or, when the group is empty,
 * is solved on its own).
 */
typedef struct {
  int32_t mp;
  int32_t kmax;
  int32_t max_systems;
  int32_t pad_;
  int64_t max_rows;
} rr_rounds_opts;
rr_status rr_rounds_workspace_bytes(const rr_rounds_opts* o, size_t* bytes);
/* Host wall-clock split of the rounds' executor: replays of the round graph
 * (launch to the read of every column state), restarts (bookkeeping and
 * polling between replays) and joins; replays and rounds run; the rounds per
 * replay the tuner settled on (0 while it is still trying candidates). */
typedef struct {
  double replay_s, restart_s, join_s;
  int64_t replays, rounds;
  int32_t rounds_per_replay;
  int32_t pad_;
} rr_rounds_stats;
rr_status rr_server_rounds_stats(rr_server* s, rr_rounds_stats* out);
rr_status rr_server_create_rounds(void* arena, size_t arena_bytes, int32_t workers,
                                  const rr_rounds_opts* rounds, rr_server** out);
/* Most requests resident at once (admitted and not completed) so far. */
rr_status rr_server_peak_running(rr_server* s, int32_t* peak);

/*
 * Batched execution of nsys independent systems: a server over `arena` with
 * min(workers, nsys) workers, the systems submitted largest workspace first,
 * drained; results[i] belongs to reqs[i].  Returns RR_OK when every system
 * converged, else the first non-OK status in input order.
 */
rr_status randrand_solve_batch(const rr_request* reqs, int32_t nsys, void* arena,
                               size_t arena_bytes, int32_t workers, rr_result* results);
/* The same with shared rounds (rounds != NULL; see rr_rounds_opts). */
rr_status randrand_solve_batch_rounds(const rr_request* reqs, int32_t nsys, void* arena,
                                      size_t arena_bytes, int32_t workers,
                                      const rr_rounds_opts* rounds, rr_result* results,
                                      rr_rounds_stats* stats /* may be NULL */);

#ifdef __cplusplus
}
#endif

#endif /* RANDRAND_H */
