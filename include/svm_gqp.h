/*
 * svm_gqp.h -- C ABI of the GB300 (sm_103a) SSsNAL solver for the paper's
 * unified QP (arXiv 1910.01312, Sec. 1, eq. (1.5)) and, as a case of it, the
 * linear-kernel SVR dual (eqs. (1.3)-(1.4)).
 *
 * The problem:
 *     min_x  1/2 x'Qx + c'x   s.t.  a'x = d,  l <= x <= u,     Q = B B',
 * B an n x q matrix (the method runs in the coordinates v = B'w of q-space as
 * the C-SVC solver of svm_ssnalm.h does), c, a, l, u n-vectors with any signs
 * and magnitudes (a_i = 0 allowed; l_i <= u_i), d any value for which the
 * set {a'x = d, l <= x <= u} is non-empty.  The C-SVC dual is the case
 * B = Diag(y) X, c = -e, a = y, d = 0, l = 0, u = C.
 *
 * Method: the same SSsNAL as svm_ssnalm_solve (Algorithm 1, multiplier update
 * of eq. (3.5); Algorithm 3 with Armijo line search; stop on R_KKT of eq.
 * (4.1); the sigma schedule, inner tolerances and Armijo constants of the
 * same params), with the projection onto {a'x = d, l <= x <= u} for a general
 * a (Sec. 3.2.1: x = clip(w - lambda a, l, u)), the HS-Jacobian of Theorem
 * 3.2 and the reduced Newton system of Proposition 3.5 in q-space:
 *     (I + sigma (B_J'B_J - h h'/s)) dv = -g,  h = B_J'a_J,  s = a_J'a_J
 * (no rank-one term when s = 0).  Arithmetic: IEEE FP64 throughout (B may be
 * stored FP32: its entries are widened exactly); the Newton system is solved
 * by a direct FP64 Cholesky factorisation.
 *
 * Conventions (pointers, streams, errors, threads) are those of svm_ssnalm.h;
 * svm_params supplies tol, max_outer, max_inner, max_ls, sigma0,
 * sigma_growth, sigma_max, mu, delta and stream (C and precision are unused,
 * except by svm_svr_create, which reads C).
 */
#ifndef SVM_GQP_H
#define SVM_GQP_H

#include <stdint.h>

#include "svm_ssnalm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct svm_gqp svm_gqp_t; /* opaque solver handle */

/* How B is stored. */
typedef enum {
    SVM_GQP_DENSE = 0,   /* B itself: n x q, row-major                           */
    SVM_GQP_STACKED = 1  /* B = [X; -X] for X m x q (n = 2m): the SVR dual's
                            matrix, whose 2m rows are never stored              */
} svm_gqp_layout;

typedef struct {
    int64_t n;          /* variables (rows of B), >= 1; even for STACKED         */
    int64_t q;          /* columns of B, 1 <= q <= 1024                          */
    int32_t layout;     /* svm_gqp_layout                                        */
    int32_t dtype;      /* svm_dtype of the stored matrix                        */
    int32_t memory;     /* svm_memory of every array below                       */
    int32_t reserved0;
    const void *B;      /* DENSE: n x q; STACKED: X, (n/2) x q; row-major,
                           16-byte aligned                                       */
    const double *c;    /* n: linear term                                        */
    const double *a;    /* n: the equality constraint's coefficients             */
    const double *l;    /* n: lower bounds (finite)                              */
    const double *u;    /* n: upper bounds (finite, >= l)                        */
    double d;           /* right-hand side of a'x = d                            */
} svm_gqp_problem;

typedef struct {
    double *x;          /* n, caller-owned FP64, same memory kind as the problem:
                           receives the solution                                 */
    double *w;          /* q, caller-owned FP64: w = B'x                         */
    double lambda;      /* multiplier of a'x = d in the KKT projection of eq.
                           (4.1) at the solution (x = clip(x - Qx - c - lambda a)
                           on the free components)                              */
    double kkt;         /* R_KKT(x) of eq. (4.1)                                 */
    double objective;   /* 1/2 |B'x|^2 + c'x                                     */
    double feasibility; /* a'x - d                                               */
    double sigma;       /* final sigma                                           */
    int32_t outer_iters;
    int32_t inner_iters_total;
    int32_t status;     /* same as the return value of the solve                 */
    int32_t reserved0;
    int64_t n_free;     /* l_i < x_i < u_i                                       */
} svm_gqp_result;

/* Create a solver for one problem.  Validates sizes, pointers, finiteness
 * (B, c, a, l, u, d), l <= u and, by one projection, that the feasible set is
 * non-empty.  SVM_MEM_DEVICE: the handle BORROWS B, c, a, l and u (keep them
 * valid and unchanged until svm_gqp_destroy); SVM_MEM_HOST: it copies them.
 * The handle owns its workspace (O(n) vectors, O(q^2) Newton matrix).
 * Returns SVM_ERR_INVALID_ARG (bad sizes, pointers, values, empty set),
 * SVM_ERR_UNSUPPORTED (q > 1024, n >= 2^31), SVM_ERR_OOM, SVM_ERR_CUDA.
 * *out is NULL on failure. */
svm_status svm_gqp_create(svm_gqp_t **out, const svm_gqp_problem *prob, const svm_params *params);

/* The SVR dual (eq. (1.4)) with the linear kernel K = X X' as a unified QP
 * in the 2m variables [x; z] (x multiplies eps + y, z multiplies eps - y):
 * layout STACKED over X (m x q, dtype, row-major, 16-byte aligned),
 * c = [eps + y; eps - y], a = [e; -e], d = 0, l = 0, u = params->C.  The
 * handle builds and owns c, a, l and u; X (and y, until this call returns)
 * follow `memory` as in svm_gqp_create.  After svm_gqp_solve the regression
 * function is f(t) = <w_svr, t> + b with w_svr = X'(z - x) = -res.w and
 * b = -res.lambda, and beta = z - x are the coefficients of eq. (1.3).
 * Returns as svm_gqp_create; SVM_ERR_INVALID_ARG also for eps < 0 or a
 * non-finite y. */
svm_status svm_svr_create(svm_gqp_t **out, const void *X, int64_t m, int64_t q, int32_t dtype, int32_t memory,
                          const double *y, double eps, const svm_params *params);

/* Solve from x^0 = 0, w^0 = 0 (Sec. 4.1) until R_KKT <= tol or max_outer.
 * res->x and res->w must be non-NULL (memory kind of the problem).
 * Synchronises the stream.  Returns SVM_OK, SVM_ERR_NOT_CONVERGED (results
 * filled), SVM_ERR_NUMERIC (failed factorisation or root search),
 * SVM_ERR_TIMEOUT, SVM_ERR_CUDA. */
svm_status svm_gqp_solve(svm_gqp_t *h, svm_gqp_result *res);

/* Release the handle and its workspace.  NULL-safe. */
void svm_gqp_destroy(svm_gqp_t *h);

/* One-line description of the last error on h (of the last failed create
 * when h is NULL).  Never NULL. */
const char *svm_gqp_last_error(const svm_gqp_t *h);

/* Step-level entry points (device FP64 buffers), so that each step can be
 * checked on its own:
 * svm_gqp_op_project: x = Pi(w) onto {a'x = d, l <= x <= u} (Sec. 3.2.1) with
 *   lambda (host out), the free set J (device int32, n, nullable; ascending
 *   indices with l_i < w_i - lambda a_i < u_i) and its size *p_out.
 * svm_gqp_op_newton: dv from (I + sigma (B_J'B_J - h h'/s)) dv = -g
 *   (Proposition 3.5 with Theorem 3.2's HS-Jacobian; J device int32, p of them).
 * svm_gqp_op_matvec: z = B v (q -> n);  svm_gqp_op_rmatvec: out = B'y (n -> q). */
svm_status svm_gqp_op_project(svm_gqp_t *h, const double *w, double *x, double *lambda, int32_t *J, int64_t *p_out);
svm_status svm_gqp_op_newton(svm_gqp_t *h, const int32_t *J, int64_t p, double sigma, const double *g, double *dv);
svm_status svm_gqp_op_matvec(svm_gqp_t *h, const double *v, double *z);
svm_status svm_gqp_op_rmatvec(svm_gqp_t *h, const double *y, double *out);

#ifdef __cplusplus
}
#endif
#endif /* SVM_GQP_H */
