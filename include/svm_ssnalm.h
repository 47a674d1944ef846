/*
 * svm_ssnalm.h -- C ABI of the GB300 (sm_103a) SSsNAL solver for the
 * linear-kernel C-SVC dual of arXiv 1910.01312.
 *
 * The problem (Sec. 1, eq. (1.2)):
 *     min_alpha  1/2 alpha' Q alpha - e' alpha
 *     s.t.       y' alpha = 0,   0 <= alpha_i <= C,
 * with Q = A A', A = Diag(y) X, X the n x q data matrix (linear kernel).
 * The paper calls the variable x; this header calls it alpha.
 *
 * Method: the augmented Lagrangian method on the restricted dual (Algorithm 1,
 * multiplier update of eq. (3.5)), whose subproblems are solved by the
 * semismooth Newton method with Armijo line search (Algorithm 3), using the
 * projection onto {y'x = 0, 0 <= x <= C} (Sec. 3.2.1), its HS-Jacobian
 * (Theorem 3.2) and the reduced Newton system of Proposition 3.5.  The stopping
 * test is the relative KKT residual of eq. (4.1).
 *
 * Conventions for every call below:
 *  - All entry points are extern "C"; no C++ exception crosses them.
 *  - Pointers marked "device" are CUDA device pointers (for example a torch
 *    tensor's data_ptr()); "host" pointers are ordinary CPU memory.
 *  - Work is issued on the stream given in svm_params.stream (NULL = legacy
 *    default stream).  Calls that return scalars synchronise that stream
 *    before returning.
 *  - Errors: every call returns an svm_status; svm_ssnalm_last_error() gives a
 *    one-line reason for the last failure on a handle.  On error the contents
 *    of output buffers are unspecified unless stated.
 *  - Threads: a handle is used by one host thread at a time.  Do not run
 *    solves of different handles concurrently on one GPU (different streams
 *    or threads): the projection and the Newton step for q > 128 are
 *    cooperative launches sized to the whole GPU, whose blocks wait on one
 *    another.  For many problems over one X use svm_ssnalm_solve_batch.
 */
#ifndef SVM_SSNALM_H
#define SVM_SSNALM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct svm_ssnalm svm_ssnalm_t; /* opaque solver handle */

typedef enum {
    SVM_OK = 0,
    SVM_ERR_INVALID_ARG = 1,   /* bad size, pointer, C, tol or label        */
    SVM_ERR_CUDA = 2,          /* a CUDA runtime call failed                */
    SVM_ERR_OOM = 3,           /* device or host allocation failed          */
    SVM_ERR_NOT_CONVERGED = 4, /* iteration cap reached; results are filled */
    SVM_ERR_NUMERIC = 5,       /* non-finite value or failed factorisation  */
    SVM_ERR_DEGENERATE = 6,    /* labels of one class only: alpha = 0       */
    SVM_ERR_TIMEOUT = 7,       /* a bounded device-side wait gave up        */
    SVM_ERR_UNSUPPORTED = 8    /* size or layout outside this build's range */
} svm_status;

typedef enum { SVM_DENSE_ROWMAJOR = 0, SVM_CSR = 1 } svm_layout;
typedef enum { SVM_F32 = 0, SVM_F64 = 1 } svm_dtype;

/* Arithmetic of the solve (requested in svm_params.precision).
 * PLAIN_FP64: every vector, product and reduction in IEEE FP64 (X is read in
 *   its storage type and widened exactly); dense X: direct Cholesky solve of
 *   the reduced Newton system.
 * MIXED: FP32 products; FP64 accuracy recovered where the method needs it by
 *   FP32 error-free transformations (compensated sums and products); FP64
 *   kept for the multiplier/sigma updates, the KKT/gap reductions and the
 *   small Newton factorisation.  The full mixed form needs dense FP32 X with
 *   q % 4 == 0.  MIXED on other problems is accepted and runs the form below
 *   that fits; the form that actually ran is reported in svm_result.form. */
typedef enum { SVM_PREC_PLAIN_FP64 = 0, SVM_PREC_MIXED = 1 } svm_precision;

/* The arithmetic a solve actually ran (svm_result.form).
 * FP64_DIRECT: IEEE FP64 vectors and products, direct reduced Newton solve
 *   (PLAIN_FP64 on dense X).
 * MIXED: the mixed form (MIXED on dense FP32 X with q % 4 == 0): FP32
 *   compensated products, double-float n-vectors, CG Newton solve
 *   preconditioned by an FP32 Cholesky factor.
 * COMPENSATED: FP64 n-vectors; products with FP32 X in compensated FP32
 *   arithmetic; CG Newton solve (MIXED on dense FP32 X with q % 4 != 0, or on
 *   CSR FP32 X).
 * FP64_CG: FP64 vectors and products; CG Newton solve (MIXED on FP64 X, and
 *   every CSR solve with FP64 values or PLAIN_FP64). */
typedef enum { SVM_FORM_FP64_DIRECT = 0, SVM_FORM_MIXED = 1, SVM_FORM_COMPENSATED = 2, SVM_FORM_FP64_CG = 3 } svm_form;

/* Where the problem arrays and the result arrays live. */
typedef enum { SVM_MEM_DEVICE = 0, SVM_MEM_HOST = 1 } svm_memory;

typedef struct {
    int64_t n;              /* number of samples (rows of X), >= 1             */
    int64_t q;              /* number of features (columns of X), >= 1         */
    int32_t layout;         /* svm_layout                                      */
    int32_t dtype;          /* svm_dtype of X                                  */
    int32_t memory;         /* svm_memory of X and y                           */
    int32_t reserved0;
    const void *X;          /* dense: n*q elements, row-major, 16-byte aligned */
    const int64_t *indptr;  /* CSR: n+1 row pointers, indptr[0] = 0, [n] = nnz */
    const int32_t *indices; /* CSR: nnz column indices, strictly increasing
                               within each row, each in [0, q)               */
    const void *values;     /* CSR: nnz values of type dtype                  */
    int64_t nnz;            /* CSR: number of stored entries (>= 0)            */
    const int8_t *y;        /* n labels, each +1 or -1                         */
} svm_problem;

typedef struct {
    double C;            /* box bound, finite and > 0                         */
    double tol;          /* R_KKT tolerance of eq. (4.1); default 1e-6         */
    int32_t max_outer;   /* ALM iterations; default 200 (Sec. 4.1)            */
    int32_t max_inner;   /* SsN iterations per subproblem; default 50          */
    int32_t max_ls;      /* Armijo trials per Newton step; default 40          */
    int32_t precision;   /* svm_precision; default SVM_PREC_MIXED              */
    double sigma0;       /* initial sigma of Algorithm 1; default 1            */
    double sigma_growth; /* sigma *= growth when R_KKT fell by < 1/2; 5        */
    double sigma_max;    /* cap on sigma; default 1e6                          */
    double mu;           /* Armijo constant of Algorithm 3; default 1e-4       */
    double delta;        /* step reduction of Algorithm 3; default 0.5         */
    double tau;          /* inexact-Newton exponent of Algorithm 3; 0.5        */
    double eta;          /* inexact-Newton cap of Algorithm 3; 0.1             */
    int32_t newton_mode; /* 0 auto (reserved for other solvers)                */
    int32_t deterministic; /* 1: fixed-order reductions (always, this build)   */
    void *stream;        /* cudaStream_t, NULL for the default stream          */
} svm_params;

typedef struct {
    double *alpha;  /* n, caller-owned, FP64; device pointer (memory=DEVICE) or
                       host pointer (memory=HOST).  Receives the solution.    */
    double *w;      /* q, caller-owned, FP64, same memory kind: w = A' alpha  */
    double b;       /* bias: the multiplier of y'alpha = 0 at the solution    */
    double kkt;     /* R_KKT(alpha), eq. (4.1), computed in FP64              */
    double objective;        /* 1/2 |A'alpha|^2 - e'alpha                     */
    double primal_objective; /* 1/2 |w|^2 + C sum hinge(1 - y_i(<w,x_i> + b)) */
    double gap;              /* primal_objective + objective (>= 0)           */
    double sigma;            /* final sigma                                   */
    int32_t outer_iters;
    int32_t inner_iters_total;
    int32_t status;          /* same as the return value of the solve         */
    int32_t form;            /* svm_form: the arithmetic this solve ran       */
    int64_t n_free;          /* 0 < alpha_i < C                               */
    int64_t n_upper;         /* alpha_i = C                                   */
    int64_t n_sv;            /* alpha_i > 0                                   */
} svm_result;

/* Fill *p with the defaults listed above (C = 1). */
void svm_default_params(svm_params *p);

/* Create a solver for one problem (Sec. 1, eq. (1.2)).
 * Validates n, q, C, tol, pointers and (device-side) the labels.  With
 * memory = SVM_MEM_DEVICE the handle BORROWS X and y: they must stay valid
 * and unchanged until svm_ssnalm_destroy.  With SVM_MEM_HOST it copies them
 * to the device (the copy is timed as part of create).  The handle owns all
 * device workspace (O(n) vectors, O(q^2) Newton matrix).
 * CSR (layout = SVM_CSR, any q < 2^31, Sec. 4's sparse datasets): create also
 * checks the row structure and builds a CSC copy of X (O(nnz) device memory,
 * borrowed arrays stay borrowed); the solve keeps its vectors in FP64 (with
 * FP32 values and SVM_PREC_MIXED the products run in compensated FP32
 * arithmetic), with z = A v over the rows, A'c over the CSC columns and the
 * Newton system (Prop. 3.5) by matrix-free Jacobi-preconditioned CG
 * (Algorithm 3) instead of a q x q factorisation.
 * Returns SVM_ERR_INVALID_ARG, SVM_ERR_OOM, SVM_ERR_CUDA, SVM_ERR_UNSUPPORTED.
 * *out is NULL on failure. */
svm_status svm_ssnalm_create(svm_ssnalm_t **out, const svm_problem *prob,
                             const svm_params *params);

/* Solve (Algorithm 1 with Algorithm 3 inside) until R_KKT <= tol or
 * max_outer.  alpha0 (nullable; same memory kind as the problem) is a warm
 * start: it is projected onto {y'x = 0, 0 <= x <= C} and the ALM dual starts
 * at v = A'alpha0; NULL starts from zero (Sec. 4.1).  res->alpha and res->w
 * must be non-NULL.  Synchronises the stream.  Returns SVM_OK,
 * SVM_ERR_NOT_CONVERGED (results filled), SVM_ERR_DEGENERATE (one class:
 * alpha = 0, b = NaN), SVM_ERR_NUMERIC, SVM_ERR_TIMEOUT, SVM_ERR_CUDA. */
svm_status svm_ssnalm_solve(svm_ssnalm_t *h, const double *alpha0, svm_result *res);

/* Solve B problems that share the handle's X (dense layout): problem b has
 * labels Y[b*n .. b*n+n-1] (+1/-1) and bound C[b], with every other setting
 * of the handle (precision, tolerance, iteration caps, sigma schedule).  This
 * is the one-vs-rest / regularisation-path use of the method: Algorithm 1 with
 * Algorithm 3 inside, run for all problems in lockstep -- each problem
 * advances one phase (start of a subproblem, Newton step with its first
 * Armijo trial, further trial, end of an outer iteration) per stream
 * synchronisation, problems that have converged drop out, and the forward
 * products A v of all problems in a phase share passes over X (1, 2, 4 or 8
 * vectors per pass, split by an autotuner that times the pass widths on this
 * X at the first call); the Newton steps of a phase also run together (for
 * q <= 128 in three launches over all problems; for 128 < q <= 1024 the
 * preconditioner set-ups in one cooperative launch and the CGs in another, a
 * group of blocks per problem, all problems sharing one FP16 copy of X).
 * Each problem's iterates, and so its results, are bit-identical to
 * svm_ssnalm_solve of the same problem (cold start).
 * Memory kind as the handle's: Y (B*n int8), alpha (B*n FP64, row b = problem
 * b) and w (B*q FP64) are device pointers for SVM_MEM_DEVICE, host pointers
 * for SVM_MEM_HOST; C (B doubles) and results (B entries) are host memory.
 * results[b] is filled as by svm_ssnalm_solve, with results[b].alpha/.w set to
 * the problem's rows of alpha and w and results[b].status its own status.
 * The first call with a given B creates B internal sub-handles (each owns an
 * O(n) workspace like a handle of its own; they are kept for later calls and
 * freed by svm_ssnalm_destroy).  Synchronises the stream.  Returns SVM_OK
 * when every problem converged, else the most severe per-problem status
 * (errors, then SVM_ERR_NOT_CONVERGED, then SVM_ERR_DEGENERATE);
 * SVM_ERR_INVALID_ARG for B < 1, null pointers, C <= 0 or non-finite, or a
 * label other than +1/-1; SVM_ERR_UNSUPPORTED for CSR handles or B > 65535. */
svm_status svm_ssnalm_solve_batch(svm_ssnalm_t *h, int32_t B, const int8_t *Y, const double *C, double *alpha,
                                  double *w, svm_result *results);

/* Release the handle and its workspace.  NULL-safe. */
void svm_ssnalm_destroy(svm_ssnalm_t *h);

/* One-line description of the last error on h (or of the last failed
 * create when h is NULL).  Never NULL. */
const char *svm_ssnalm_last_error(const svm_ssnalm_t *h);

/* ---------------------------------------------------------------------
 * Step-level entry points.  Each runs one step of the hot path with the
 * handle's problem, precision and workspace, so that each step can be checked
 * on its own.  All vector arguments are device pointers (FP64 unless stated);
 * they are valid for problems created with either memory kind.
 * ------------------------------------------------------------------- */

/* z = A v  (z_i = y_i <x_i, v>): v has q entries, z has n. */
svm_status svm_op_matvec(svm_ssnalm_t *h, const double *v, double *z);

/* out = A' c = sum_i c_i y_i x_i over the rows with c_i != 0 (q entries).
 * c has n entries; rows with c_i == 0 are skipped. */
svm_status svm_op_rmatvec(svm_ssnalm_t *h, const double *c, double *out);

/* pi = Pi_{K cap L}(u), K = [0,C]^n, L = {y'x = 0} (Sec. 3.2.1).
 * lambda (host, out): the multiplier lambda-hat with pi = clip(u - lambda y).
 * J (device int32, n, nullable): ascending indices with 0 < u_i - lambda y_i < C
 *   (the free set, complement of the active set of eq. (3.8)); *p_out its size.
 * S (device int32, n, nullable): ascending indices with pi_i > 0; *s_out.
 * Returns SVM_ERR_NUMERIC if the root search did not terminate. */
svm_status svm_op_project(svm_ssnalm_t *h, const double *u, double *pi, double *lambda,
                          int32_t *J, int64_t *p_out, int32_t *S, int64_t *s_out);

/* Newton direction of Algorithm 3, Step 1, through Proposition 3.5 in the
 * coordinates v = A'w:  (I_q + sigma A'PA) dv = -g, with P the HS-Jacobian of
 * Theorem 3.2 on the free set J (device int32, p ascending indices).
 * g, dv: q entries. */
svm_status svm_op_newton(svm_ssnalm_t *h, const int32_t *J, int64_t p, double sigma,
                         const double *g, double *dv);

/* Gram of the free rows as the large-free-set Newton step builds its
 * preconditioner (Proposition 3.5: the reduced matrix I + sigma (G - h h'/p)):
 * G = X_J' X_J (q x q, row-major FP64, device) and hsum = X_J' 1 (q, FP64,
 * device), J device int32 with p row indices (any order; p = 0 gives zeros).
 * G is formed on the tcgen05 tensor cores with FP32 sums within a block,
 * blocks added in FP64; hsum is exact to double-float accuracy.  q <= 128:
 * TF32 products (10-bit mantissa), one 128 x q accumulator per block;
 * 128 < q <= 1024: FP16 products of an FP16 copy of X scaled per feature by
 * a power of two (11-bit significand; the copy, n x 64 ceil(q / 64) x 2
 * bytes, is made on the first call and kept with the handle), (128-feature x 256-feature)
 * tiles of the lower triangle, G symmetrised from it.  Dense FP32 X with
 * q % 16 == 0 and q <= 1024 only (else SVM_ERR_UNSUPPORTED).  Synchronises
 * the stream. */
svm_status svm_op_gram(svm_ssnalm_t *h, const int32_t *J, int64_t p, double *G, double *hsum);

/* Relative KKT residual of eq. (4.1) at alpha (n, device).  *kkt and *lambda
 * (multiplier of the projection in the residual) are host outputs. */
svm_status svm_op_kkt(svm_ssnalm_t *h, const double *alpha, double *kkt, double *lambda);

/* ---------------------------------------------------------------------
 * Instrumentation (no counterpart in the paper: measurement support).
 * ------------------------------------------------------------------- */
typedef struct {
    int64_t launches;          /* kernels launched by this handle since reset  */
    int64_t matvec_calls;      /* one-vector products z = A v (one kernel each) */
    double matvec_ms;          /* their summed CUDA-event time (timing on)     */
    int64_t rmatvec_calls;     /* A' c products (two kernels each)             */
    double rmatvec_ms;
    int64_t proj_calls;        /* projections (one cooperative kernel each)    */
    double proj_ms;
    int64_t newton_calls;      /* Newton-system solves                          */
    double newton_ms;
    int64_t host_syncs;        /* stream synchronisations for scalar read-back */
    int64_t matvec2_calls;     /* two-vector passes [A v0, A v1] over X          */
    double matvec2_ms;
} svm_stats;

/* Enable (1) or disable (0) CUDA-event timing of the step kinds above.  When
 * enabled, each timed launch is bracketed by two events recorded on the
 * handle's stream; times are accumulated when the solve (or op) returns. */
svm_status svm_ssnalm_set_timing(svm_ssnalm_t *h, int enable);

/* Copy the counters into *out (host); reset them when reset != 0. */
svm_status svm_ssnalm_get_stats(svm_ssnalm_t *h, svm_stats *out, int reset);

/* ---------------------------------------------------------------------
 * Random Fourier features front-end (Sec. 4.3): the RBF-kernel C-SVC with
 * k(x, y) = exp(-|x - y|^2 / (2 alpha)) becomes the linear C-SVC on Z.
 * ------------------------------------------------------------------- */

/* Z (n x 2N, row-major FP32, device) from X (n x q, row-major FP32, device)
 * and the frequencies Omega (q x N, row-major FP32, device; column j is
 * omega_j, drawn by the caller from N(0, I/alpha)):
 *     Z[i][2j] = cos(<x_i, omega_j>) / sqrt(N),  Z[i][2j+1] = sin(<x_i, omega_j>) / sqrt(N),
 * so that Z Z' is the sample average (1/N) sum_j cos(omega_j'(x_i - x_k)) of
 * the paper's Bochner estimate.  The phases <x_i, omega_j> are FP32 sums in k
 * order.  Pass Z as the X of svm_ssnalm_create (q = 2N) to solve the
 * approximated problem.  Allocates nothing; stream-ordered (stream may be
 * NULL), returns without synchronising.  SVM_ERR_INVALID_ARG for null
 * pointers or n, q, N < 1; SVM_ERR_UNSUPPORTED when Z is not 8-byte aligned
 * or N > 2^28; SVM_ERR_CUDA when the launch fails. */
svm_status svm_rff_features(const float *X, int64_t n, int64_t q, const float *Omega, int64_t N, float *Z,
                            void *stream);

/* ---------------------------------------------------------------------
 * Allocation-free transposed product.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate memory.
 * ------------------------------------------------------------------- */

/* out = A'c = sum_i c_i y_i x_i (q entries) for dense row-major FP32 X
 * (n x q), labels y (n, +1/-1) and weights c (n, FP64), computed like the
 * mixed-form product of svm_op_rmatvec, WITHOUT allocating anything.
 *
 * For callers that cannot allocate: code inside a framework that owns all
 * device memory through its own pool, latency-critical loops that cannot
 * afford the synchronisation or the failure of an allocation, callers with a
 * fixed memory budget.  They cannot create a handle (a handle owns its
 * workspace), so this call needs only the caller's device buffers X, y, c,
 * out and a stream (NULL = default stream).
 *
 * Scratch: one fixed array in device global memory (1.25 MiB + 256 bytes:
 * block partials for up to 160 blocks x 1024 columns and a counter), present
 * on every GPU that loads the library until the process exits.  Limits:
 * 1 <= q <= 1024 and 1 <= n < 2^31; larger sizes return SVM_ERR_UNSUPPORTED,
 * null pointers or n, q < 1 return SVM_ERR_INVALID_ARG.  It calls no
 * allocation routine: it only looks up the array's device address, clears
 * the counter (cudaMemsetAsync) and launches one kernel.
 *
 * The call runs on the current device: X, y, c and out must be that device's
 * memory, and a non-NULL stream must belong to it (a stream of another device
 * returns SVM_ERR_INVALID_ARG).  The first call on a device (with that device
 * current) performs that device's one-time set-up (address look-up, kernel
 * attribute); make that first call before any stream capture.  The call is
 * stream-ordered and returns without synchronising.  All calls on a device share the one
 * scratch array: calls whose kernels could overlap on the GPU (different
 * streams or host threads) race and give wrong results -- serialise them. */
svm_status svm_rmatvec_noalloc(const float *X, const int8_t *y, int64_t n, int64_t q,
                               const double *c, double *out, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* SVM_SSNALM_H */
