/*
 * svm_oracle.c -- plain, slow, obviously-correct FP64 CPU oracle for the
 * sparse semismooth-Newton augmented Lagrangian method (SSsNAL) of
 * arXiv 1910.01312 on the linear-kernel C-SVC dual.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg load this library.  It shares no code, header,
 * table or helper with the GPU library; the two meet only on the seeded
 * synthetic inputs.
 *
 * Problem (Sec. 1, eq. (1.2)):  min 1/2 x'Qx - e'x  s.t. y'x = 0, 0 <= x <= C,
 * Q = A A', A = Diag(y) X.  The paper calls the SVM dual variable x; the code
 * calls it alpha.  The paper's ALM dual variable w lives in Ran(Q) subset R^n;
 * with Q = A A' we carry it as v = A'w in R^q (so Qw = A v, <w,Qw> = |v|^2,
 * grad psi = A g with g = v - A' Pi(u)).  Everything else follows the paper's
 * order:
 *   - outer loop      : Algorithm 1 with the multiplier update of eq. (3.5)
 *                       (alpha^{k+1} = Pi_{K cap L}(u(w^{k+1}))),
 *   - inner loop      : Algorithm 3 (semismooth Newton + Armijo line search),
 *   - projection      : Algorithm 2 (sorted breakpoint binary search), then the
 *                       componentwise clip that follows it,
 *   - generalized Jacobian : Theorem 3.2 (HS-Jacobian P = S(I - aa'/a'Sa)S),
 *   - reduced Newton system: Proposition 3.5, solved exactly either in q-space
 *                       or in |J|-space (both forms are exact solves of the
 *                       same system; see orc_newton_direction),
 *   - stopping test   : relative KKT residual of eq. (4.1) (Sec. 4.1).
 * Readings where the paper is silent (sigma schedule, inner tolerances, line
 * search constants, bias b) are marked "reading" below.
 *
 * Reductions over n use pairwise (recursive halving) summation in FP64.
 *
 * Threads.  The default build (oracle.build()) is single-threaded.  The same
 * source compiled with -fopenmp (oracle.build(omp=True)) runs on all host
 * cores for the timed CPU baseline and computes the same numbers bit for
 * bit: only loops whose iterations are independent are split across threads,
 * every sum keeps its order (the pairwise trees are evaluated as tasks, the
 * Gram and the column sums let each thread own whole output entries), and the
 * breakpoint sort is a merge of sorted chunks (a sorted array is the same
 * whatever algorithm produced it).  Without -fopenmp the pragmas are ignored
 * and the _OPENMP blocks are compiled out.
 *
 * Parity status: every exported function is pinned by the CPU test-suite
 * (brute-force active-set enumeration, closed forms, finite differences,
 * invariants); see tests/test_oracle_*.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* loops and sums shorter than this stay on one thread in the OpenMP build */
#define ORC_PAR_MIN 16384

/* Inside a parallel region: this thread's index and the team size (0 and 1
 * in the single-threaded build). */
#ifdef _OPENMP
#define ORC_TEAM(id, nt) int id = omp_get_thread_num(), nt = omp_get_num_threads()
#else
#define ORC_TEAM(id, nt) int id = 0, nt = 1
#endif

#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_OOM 3
#define ORC_ERR_NOT_CONVERGED 4
#define ORC_ERR_NUMERIC 5
#define ORC_ERR_DEGENERATE 6

/* ------------------------------------------------------------------ data */

/* Element (i,j) of the data matrix X (n x q, row-major), FP32 or FP64. */
static double x_at(const void *X, int x_f32, int64_t q, int64_t i, int64_t j)
{
    if (x_f32) return (double)((const float *)X)[i * q + j];
    return ((const double *)X)[i * q + j];
}

/* Pairwise summation of a[0..n). */
static double pair_sum_rec(const double *a, int64_t n)
{
    if (n <= 16) {
        double s = 0.0;
        for (int64_t i = 0; i < n; ++i) s += a[i];
        return s;
    }
    int64_t h = n / 2;
#ifdef _OPENMP
    if (n > ORC_PAR_MIN) {   /* the same tree: the two halves as tasks */
        double l = 0.0, r = 0.0;
#pragma omp task shared(l)
        l = pair_sum_rec(a, h);
        r = pair_sum_rec(a + h, n - h);
#pragma omp taskwait
        return l + r;
    }
#endif
    return pair_sum_rec(a, h) + pair_sum_rec(a + h, n - h);
}

static double pair_sum(const double *a, int64_t n)
{
#ifdef _OPENMP
    if (n > ORC_PAR_MIN && !omp_in_parallel()) {
        double s = 0.0;
#pragma omp parallel
#pragma omp single
        s = pair_sum_rec(a, n);
        return s;
    }
#endif
    return pair_sum_rec(a, n);
}

static double dot_q(const double *a, const double *b, int64_t q)
{
    double s = 0.0;
    for (int64_t j = 0; j < q; ++j) s += a[j] * b[j];
    return s;
}

/* ------------------------------------------------------ A v and A' pi */

/* z = A v, z_i = y_i <x_i, v>  (A = Diag(y) X, Sec. 1). */
int orc_matvec(const void *X, int x_f32, const int8_t *y, int64_t n, int64_t q,
               const double *v, double *z)
{
    if (!X || !y || !v || !z || n < 0 || q < 0) return ORC_ERR_ARG;
#pragma omp parallel for schedule(static) if (n > ORC_PAR_MIN)
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t j = 0; j < q; ++j) s += x_at(X, x_f32, q, i, j) * v[j];
        z[i] = (double)y[i] * s;
    }
    return ORC_OK;
}

/* out += sum_{i in [lo,hi)} p_i y_i x_i, pairwise over rows.
 * absout (optional) accumulates sum |p_i x_ij| for a roundoff scale. */
static void rmatvec_rec(const void *X, int x_f32, const int8_t *y, int64_t q,
                        const double *p, int64_t lo, int64_t hi, double *out,
                        double *absout, double *tmp_pool)
{
    if (hi - lo <= 32) {
        for (int64_t i = lo; i < hi; ++i) {
            double c = p[i] * (double)y[i];
            if (c == 0.0) continue;
            for (int64_t j = 0; j < q; ++j) {
                double t = c * x_at(X, x_f32, q, i, j);
                out[j] += t;
                if (absout) absout[j] += fabs(t);
            }
        }
        return;
    }
    int64_t mid = lo + (hi - lo) / 2;
    double *right = tmp_pool;            /* q doubles for the right half */
    double *pool2 = tmp_pool + q;        /* deeper levels */
    memset(right, 0, (size_t)q * sizeof(double));
#ifdef _OPENMP
    if (!absout && hi - lo > ORC_PAR_MIN) {
        /* the same tree: the right half as a task with scratch of its own */
        int levels = 2;
        for (int64_t m = hi - mid; m > 32; m /= 2) ++levels;
        double *pool_r = (double *)calloc((size_t)levels * (size_t)q, sizeof(double));
        if (pool_r) {
#pragma omp task
            rmatvec_rec(X, x_f32, y, q, p, mid, hi, right, NULL, pool_r);
            rmatvec_rec(X, x_f32, y, q, p, lo, mid, out, NULL, pool2);
#pragma omp taskwait
            free(pool_r);
            for (int64_t j = 0; j < q; ++j) out[j] += right[j];
            return;
        }
    }
#endif
    rmatvec_rec(X, x_f32, y, q, p, lo, mid, out, absout, pool2);
    rmatvec_rec(X, x_f32, y, q, p, mid, hi, right, absout, pool2);
    for (int64_t j = 0; j < q; ++j) out[j] += right[j];
}

/* out = A' p = sum_i p_i y_i x_i  (q-vector).  absscale (optional, q) gets
 * sum_i |p_i x_ij|, the magnitude that bounds the roundoff of out. */
int orc_rmatvec(const void *X, int x_f32, const int8_t *y, int64_t n, int64_t q,
                const double *p, double *out, double *absscale)
{
    if (!X || !y || !p || !out || n < 0 || q < 0) return ORC_ERR_ARG;
    int depth = 2;
    for (int64_t m = n; m > 32; m /= 2) ++depth;
    double *pool = (double *)calloc((size_t)(depth + 1) * (size_t)(q > 0 ? q : 1), sizeof(double));
    if (!pool) return ORC_ERR_OOM;
    memset(out, 0, (size_t)q * sizeof(double));
    if (absscale) memset(absscale, 0, (size_t)q * sizeof(double));
#ifdef _OPENMP
    if (n > ORC_PAR_MIN && !omp_in_parallel()) {
#pragma omp parallel
#pragma omp single
        rmatvec_rec(X, x_f32, y, q, p, 0, n, out, NULL, pool);
        free(pool);
        if (absscale) {
            /* sum_i |p_i y_i x_ij| in row order, as the leaves above add it:
             * each thread owns a block of the columns and walks all rows */
#pragma omp parallel
            {
                ORC_TEAM(id, nt);
                int64_t j0 = q * id / nt, j1 = q * (id + 1) / nt;
                double *acc = (double *)calloc((size_t)(j1 - j0 + 1), sizeof(double));   /* own cache lines */
                for (int64_t i = 0; acc && i < n; ++i) {
                    double c = p[i] * (double)y[i];
                    if (c == 0.0) continue;
                    for (int64_t j = j0; j < j1; ++j) acc[j - j0] += fabs(c * x_at(X, x_f32, q, i, j));
                }
                for (int64_t j = j0; acc && j < j1; ++j) absscale[j] = acc[j - j0];
                if (!acc && j0 < j1) absscale[j0] = NAN;
                free(acc);
            }
        }
        return ORC_OK;
    }
#endif
    rmatvec_rec(X, x_f32, y, q, p, 0, n, out, absscale, pool);
    free(pool);
    return ORC_OK;
}

/* ------------------------------------------------ the same products, CSR X */

/* Element k of a CSR value array, FP32 or FP64. */
static double csr_val(const void *vals, int v_f32, int64_t k)
{
    if (v_f32) return (double)((const float *)vals)[k];
    return ((const double *)vals)[k];
}

/* z = A v for X in CSR form (row i: columns ix[ip[i]..ip[i+1]), values
 * vals, ascending columns); the stored entries are summed in column order,
 * which is the dense loop of orc_matvec with its zero terms left out. */
int orc_matvec_csr(const int64_t *ip, const int32_t *ix, const void *vals, int v_f32,
                   const int8_t *y, int64_t n, int64_t q, const double *v, double *z)
{
    if (!ip || !y || !v || !z || n < 0 || q < 0) return ORC_ERR_ARG;
#pragma omp parallel for schedule(static) if (n > ORC_PAR_MIN)
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t k = ip[i]; k < ip[i + 1]; ++k) s += csr_val(vals, v_f32, k) * v[ix[k]];
        z[i] = (double)y[i] * s;
    }
    return ORC_OK;
}

/* out += sum_{i in [lo,hi)} p_i y_i x_i over CSR rows, pairwise over rows
 * exactly as rmatvec_rec (the zero entries it adds change nothing). */
static void rmatvec_csr_rec(const int64_t *ip, const int32_t *ix, const void *vals, int v_f32,
                            const int8_t *y, int64_t q, const double *p, int64_t lo, int64_t hi,
                            double *out, double *tmp_pool)
{
    if (hi - lo <= 32) {
        for (int64_t i = lo; i < hi; ++i) {
            double c = p[i] * (double)y[i];
            if (c == 0.0) continue;
            for (int64_t k = ip[i]; k < ip[i + 1]; ++k) out[ix[k]] += c * csr_val(vals, v_f32, k);
        }
        return;
    }
    int64_t mid = lo + (hi - lo) / 2;
    double *right = tmp_pool, *pool2 = tmp_pool + q;
    memset(right, 0, (size_t)q * sizeof(double));
    rmatvec_csr_rec(ip, ix, vals, v_f32, y, q, p, lo, mid, out, pool2);
    rmatvec_csr_rec(ip, ix, vals, v_f32, y, q, p, mid, hi, right, pool2);
    for (int64_t j = 0; j < q; ++j) out[j] += right[j];
}

/* out = A' p for CSR X (q-vector). */
int orc_rmatvec_csr(const int64_t *ip, const int32_t *ix, const void *vals, int v_f32,
                    const int8_t *y, int64_t n, int64_t q, const double *p, double *out)
{
    if (!ip || !y || !p || !out || n < 0 || q < 0) return ORC_ERR_ARG;
    int depth = 2;
    for (int64_t m = n; m > 32; m /= 2) ++depth;
    double *pool = (double *)calloc((size_t)(depth + 1) * (size_t)(q > 0 ? q : 1), sizeof(double));
    if (!pool) return ORC_ERR_OOM;
    memset(out, 0, (size_t)q * sizeof(double));
    rmatvec_csr_rec(ip, ix, vals, v_f32, y, q, p, 0, n, out, pool);
    free(pool);
    return ORC_OK;
}

/* ---------------------------------------------------- projection Pi_{K cap L} */

/* Pi_[0,C](t) with the tie rule of Sec. 3.2.1: t >= C -> C, t <= 0 -> 0. */
static double clip0C(double t, double C)
{
    if (t >= C) return C;
    if (t <= 0.0) return 0.0;
    return t;
}

/* grad phi(lambda) = -a' Pi_K(v - lambda a) + d  (Sec. 3.2.1), here with
 * a = y, d = 0, K = [0,C]^n and v = u.  tmp: n doubles. */
static double grad_phi(const double *u, const int8_t *y, int64_t n, double C,
                       double lam, double *tmp)
{
#pragma omp parallel for schedule(static) if (n > ORC_PAR_MIN)
    for (int64_t i = 0; i < n; ++i) {
        double yi = (double)y[i];
        tmp[i] = yi * clip0C(u[i] - lam * yi, C);
    }
    return -pair_sum(tmp, n);
}

static int cmp_double(const void *a, const void *b)
{
    double x = *(const double *)a, z = *(const double *)b;
    return (x > z) - (x < z);
}

/* Sort t[0..m) ascending.  The OpenMP build sorts one chunk per thread and
 * merges the sorted chunks pairwise; the sorted array is the same. */
static void sort_doubles(double *t, int64_t m)
{
#ifdef _OPENMP
    int P = omp_get_max_threads();
    double *buf = (P > 1 && m > ORC_PAR_MIN) ? (double *)malloc((size_t)m * sizeof(double)) : NULL;
    int64_t *bnd = buf ? (int64_t *)malloc((size_t)(P + 1) * sizeof(int64_t)) : NULL;
    if (bnd) {
        for (int k = 0; k <= P; ++k) bnd[k] = m * k / P;
#pragma omp parallel for schedule(static, 1)
        for (int k = 0; k < P; ++k) qsort(t + bnd[k], (size_t)(bnd[k + 1] - bnd[k]), sizeof(double), cmp_double);
        double *src = t, *dst = buf;
        for (int w = 1; w < P; w *= 2) {
#pragma omp parallel for schedule(static, 1)
            for (int k = 0; k < P; k += 2 * w) {
                int64_t lo = bnd[k], mid = bnd[k + w < P ? k + w : P], hi = bnd[k + 2 * w < P ? k + 2 * w : P];
                int64_t a = lo, b = mid, o = lo;
                while (a < mid && b < hi) dst[o++] = (src[a] <= src[b]) ? src[a++] : src[b++];
                while (a < mid) dst[o++] = src[a++];
                while (b < hi) dst[o++] = src[b++];
            }
            double *x = src; src = dst; dst = x;
        }
        if (src != t) memcpy(t, src, (size_t)m * sizeof(double));
        free(bnd);
        free(buf);
        return;
    }
    free(buf);
#endif
    qsort(t, (size_t)m, sizeof(double), cmp_double);
}

/* Pi_{K cap L}(u) by Algorithm 2 (breakpoint search of Helgason et al.),
 * followed by the componentwise clip.  Writes pi (n) and returns lambda-hat
 * through *lam_out.  The breakpoints (v_i - u_i)/a_i, (v_i - l_i)/a_i of the
 * paper become y_i (u_i - C), y_i u_i because 1/y_i = y_i. */
int orc_project(const double *u, const int8_t *y, int64_t n, double C,
                double *pi, double *lam_out)
{
    if (!u || !y || !pi || !lam_out || n < 1 || !(C > 0.0)) return ORC_ERR_ARG;
    double *t = (double *)malloc((size_t)(2 * n) * sizeof(double));
    double *tmp = (double *)malloc((size_t)n * sizeof(double));
    if (!t || !tmp) { free(t); free(tmp); return ORC_ERR_OOM; }
#pragma omp parallel for schedule(static) if (n > ORC_PAR_MIN)
    for (int64_t i = 0; i < n; ++i) {
        double yi = (double)y[i];
        t[2 * i] = yi * (u[i] - C);
        t[2 * i + 1] = yi * u[i];
    }
    /* Initialization: sort ascending t(1) <= ... <= t(2n). */
    sort_doubles(t, 2 * n);
    int64_t Il = 0, Iu = 2 * n - 1;         /* 0-based I_l = 1, I_u = 2n */
    double fl = grad_phi(u, y, n, C, t[Il], tmp);
    double fu = grad_phi(u, y, n, C, t[Iu], tmp);
    while (Iu - Il > 1 && t[Iu] > t[Il]) {
        int64_t Im = (Il + Iu) / 2;          /* floor((I_l + I_u)/2) */
        double fm = grad_phi(u, y, n, C, t[Im], tmp);
        if (fm >= 0.0) { Iu = Im; fu = fm; }
        else           { Il = Im; fl = fm; }
    }
    double lam;
    if (fu == 0.0 && fl == 0.0) lam = t[Il];
    else lam = t[Il] - fl / (fu - fl) * (t[Iu] - t[Il]);
#pragma omp parallel for schedule(static) if (n > ORC_PAR_MIN)
    for (int64_t i = 0; i < n; ++i) pi[i] = clip0C(u[i] - lam * (double)y[i], C);
    *lam_out = lam;
    free(t);
    free(tmp);
    return ORC_OK;
}

/* Free index set J = complement of the active set I(u) of eq. (3.8): the
 * components whose clipped value is strictly inside (0, C) at lambda-hat.
 * Writes the ascending index list to J (n ints) and returns p = |J|. */
int64_t orc_free_set(const double *u, const int8_t *y, int64_t n, double C,
                     double lam, int64_t *J)
{
    int64_t p = 0;
    for (int64_t i = 0; i < n; ++i) {
        double t = u[i] - lam * (double)y[i];
        if (t > 0.0 && t < C) J[p++] = i;
    }
    return p;
}

/* ------------------------------------------------------------- psi(w) */

/* psi^k of eq. (3.3), written with v = A'w and pi = Pi(u(w)):
 *   psi = 1/2 |v|^2 + (|u|^2 - |u - pi|^2)/(2 sigma) - |alpha^k|^2/(2 sigma)
 * and |u|^2 - |u - pi|^2 = sum_i pi_i (2 u_i - pi_i). */
double orc_psi(const double *v, int64_t q, const double *u, const double *pi,
               const double *alpha, int64_t n, double sigma)
{
    double *tmp = (double *)malloc((size_t)n * sizeof(double));
    double *tmp2 = (double *)malloc((size_t)n * sizeof(double));
    if (!tmp || !tmp2) { free(tmp); free(tmp2); return NAN; }
#pragma omp parallel for schedule(static) if (n > ORC_PAR_MIN)
    for (int64_t i = 0; i < n; ++i) {
        tmp[i] = pi[i] * (2.0 * u[i] - pi[i]);
        tmp2[i] = alpha[i] * alpha[i];
    }
    double s = 0.5 * dot_q(v, v, q) + pair_sum(tmp, n) / (2.0 * sigma)
               - pair_sum(tmp2, n) / (2.0 * sigma);
    free(tmp);
    free(tmp2);
    return s;
}

/* ------------------------------------------------------- dense Cholesky */

/* In-place lower Cholesky of the m x m SPD matrix M (row-major). */
static int cholesky(double *M, int64_t m)
{
    for (int64_t j = 0; j < m; ++j) {
        double d = M[j * m + j];
        for (int64_t k = 0; k < j; ++k) d -= M[j * m + k] * M[j * m + k];
        if (!(d > 0.0)) return ORC_ERR_NUMERIC;
        d = sqrt(d);
        M[j * m + j] = d;
        for (int64_t i = j + 1; i < m; ++i) {
            double s = M[i * m + j];
            for (int64_t k = 0; k < j; ++k) s -= M[i * m + k] * M[j * m + k];
            M[i * m + j] = s / d;
        }
    }
    return ORC_OK;
}

/* Solve L L' x = b in place (b -> x). */
static void chol_solve(const double *L, int64_t m, double *b)
{
    for (int64_t i = 0; i < m; ++i) {
        double s = b[i];
        for (int64_t k = 0; k < i; ++k) s -= L[i * m + k] * b[k];
        b[i] = s / L[i * m + i];
    }
    for (int64_t i = m - 1; i >= 0; --i) {
        double s = b[i];
        for (int64_t k = i + 1; k < m; ++k) s -= L[k * m + i] * b[k];
        b[i] = s / L[i * m + i];
    }
}

/* ------------------------------------------------- reduced Newton system */

/* Newton direction of Algorithm 3, Step 1, solved exactly.
 *
 * The n-space system (Q + sigma Q P Q) d = -grad psi, d in Ran(Q) (eq. (3.11))
 * with Q = A A', P the HS-Jacobian of Theorem 3.2 (a = y, Sigma = Diag(1_J)),
 * is, after the substitution L = A of the proof of Proposition 3.5 and
 * dv = A'd, the q x q system
 *     (I_q + sigma A'P A) dv = -g,
 *     A'P A = A_J'A_J - (A_J'a_J)(a_J'A_J)/(a_J'a_J)     (a_J'a_J = p),
 * and, when a'Sigma a = 0 (p = 0), case (b) with P = Sigma = 0: dv = -g.
 * form 1 (q-form): Cholesky of the q x q matrix above.
 * form 2 (p-form): Proposition 3.5's reduction to a p x p system, with the
 *   rank-one term taken out last (Woodbury on I + sigma A_J'A_J through the
 *   p x p matrix sigma^{-1} I + Q_JJ, then Sherman-Morrison for the rank-one
 *   term).  Both forms solve the same linear system exactly; the p-form is
 *   ordered so that its one scalar denominator is positive whenever the
 *   system is SPD (reading of the remark after Proposition 3.5).
 * form 0: the smaller of the two.
 * J: ascending free indices (p of them). */
int orc_newton_direction(const void *X, int x_f32, const int8_t *y, int64_t n,
                         int64_t q, const int64_t *J, int64_t p, double sigma,
                         const double *g, double *dv, int form)
{
    (void)n;
    if (p == 0) {
        for (int64_t j = 0; j < q; ++j) dv[j] = -g[j];
        return ORC_OK;
    }
    if (form == 0) form = (q <= p) ? 1 : 2;
    /* h = A_J' a_J = sum_{i in J} (y_i x_i) y_i */
    double *h = (double *)calloc((size_t)q, sizeof(double));
    if (!h) return ORC_ERR_OOM;
    /* (OpenMP build: each thread owns a block of the columns, rows in order) */
#pragma omp parallel if (p > 1024)
    {
        ORC_TEAM(id, nt);
        int64_t j0 = q * id / nt, j1 = q * (id + 1) / nt;
        double *acc = (double *)calloc((size_t)(j1 - j0 + 1), sizeof(double));   /* own cache lines */
        for (int64_t r = 0; acc && r < p; ++r) {
            int64_t i = J[r];
            double yy = (double)y[i] * (double)y[i];
            for (int64_t j = j0; j < j1; ++j) acc[j - j0] += yy * x_at(X, x_f32, q, i, j);
        }
        for (int64_t j = j0; acc && j < j1; ++j) h[j] = acc[j - j0];
        if (!acc && j0 < j1) h[j0] = NAN;
        free(acc);
    }
    double pp = (double)p;
    int rc = ORC_OK;
    if (form == 1) {
        double *M = (double *)calloc((size_t)(q * q), sizeof(double));
        if (!M) { free(h); return ORC_ERR_OOM; }
        /* A_J'A_J (OpenMP build: each thread owns every nt-th row of M and
         * adds the free rows in order) */
#pragma omp parallel if (p > 1024)
        {
            ORC_TEAM(id, nt);
            for (int64_t r = 0; r < p; ++r) {
                int64_t i = J[r];
                for (int64_t a = id; a < q; a += nt) {
                    double xa = (double)y[i] * x_at(X, x_f32, q, i, a);
                    for (int64_t b = 0; b <= a; ++b)
                        M[a * q + b] += xa * ((double)y[i] * x_at(X, x_f32, q, i, b));
                }
            }
        }
        for (int64_t a = 0; a < q; ++a)
            for (int64_t b = 0; b <= a; ++b) {
                double m = sigma * (M[a * q + b] - h[a] * h[b] / pp);
                if (a == b) m += 1.0;
                M[a * q + b] = m;
                M[b * q + a] = m;
            }
        rc = cholesky(M, q);
        if (rc == ORC_OK) {
            for (int64_t j = 0; j < q; ++j) dv[j] = -g[j];
            chol_solve(M, q, dv);
        }
        free(M);
    } else {
        /* K = sigma^{-1} I_p + Q_JJ,  Q_JJ = A_J A_J' */
        double *K = (double *)malloc((size_t)(p * p) * sizeof(double));
        double *t1 = (double *)malloc((size_t)p * sizeof(double));
        double *bg = (double *)malloc((size_t)q * sizeof(double));
        double *bh = (double *)malloc((size_t)q * sizeof(double));
        if (!K || !t1 || !bg || !bh) { free(K); free(t1); free(bg); free(bh); free(h); return ORC_ERR_OOM; }
        for (int64_t r = 0; r < p; ++r)
            for (int64_t s = 0; s <= r; ++s) {
                int64_t i = J[r], k = J[s];
                double acc = 0.0;
                for (int64_t j = 0; j < q; ++j)
                    acc += x_at(X, x_f32, q, i, j) * x_at(X, x_f32, q, k, j);
                acc *= (double)y[i] * (double)y[k];
                if (r == s) acc += 1.0 / sigma;
                K[r * p + s] = acc;
                K[s * p + r] = acc;
            }
        rc = cholesky(K, p);
        if (rc == ORC_OK) {
            /* B^{-1} x = x - A_J' K^{-1} A_J x,  B = I + sigma A_J'A_J (Woodbury) */
            const double *src[2] = { g, h };
            double *dst[2] = { bg, bh };
            for (int s = 0; s < 2; ++s) {
                for (int64_t r = 0; r < p; ++r) {
                    int64_t i = J[r];
                    double acc = 0.0;
                    for (int64_t j = 0; j < q; ++j) acc += x_at(X, x_f32, q, i, j) * src[s][j];
                    t1[r] = (double)y[i] * acc;
                }
                chol_solve(K, p, t1);
                for (int64_t j = 0; j < q; ++j) dst[s][j] = src[s][j];
                for (int64_t r = 0; r < p; ++r) {
                    int64_t i = J[r];
                    double c = t1[r] * (double)y[i];
                    for (int64_t j = 0; j < q; ++j) dst[s][j] -= c * x_at(X, x_f32, q, i, j);
                }
            }
            /* M = B - (sigma/p) h h'  ->  Sherman-Morrison */
            double hbh = dot_q(h, bh, q), hbg = dot_q(h, bg, q);
            double den = 1.0 - (sigma / pp) * hbh;
            if (!(den > 0.0)) rc = ORC_ERR_NUMERIC;
            else {
                double c = (sigma / pp) * hbg / den;
                for (int64_t j = 0; j < q; ++j) dv[j] = -(bg[j] + c * bh[j]);
            }
        }
        free(K); free(t1); free(bg); free(bh);
    }
    free(h);
    return rc;
}

/* ------------------------------------------------------------ KKT, b, gap */

/* Relative KKT residual of eq. (4.1):
 *   R_KKT(x) = |x - Pi_{K cap L}(x - Qx - c)| / (1 + |x|),  c = -e.
 * Qx = A (A'x).  Optionally returns the projection multiplier (which equals
 * the SVM bias at an exact optimum) and A'x. */
double orc_kkt(const void *X, int x_f32, const int8_t *y, int64_t n, int64_t q,
               double C, const double *alpha, double *lam_out, double *w_out)
{
    double *w = (double *)malloc((size_t)(q > 0 ? q : 1) * sizeof(double));
    double *Qa = (double *)malloc((size_t)n * sizeof(double));
    double *r = (double *)malloc((size_t)n * sizeof(double));
    double *pr = (double *)malloc((size_t)n * sizeof(double));
    if (!w || !Qa || !r || !pr) { free(w); free(Qa); free(r); free(pr); return NAN; }
    orc_rmatvec(X, x_f32, y, n, q, alpha, w, NULL);
    orc_matvec(X, x_f32, y, n, q, w, Qa);
#pragma omp parallel for schedule(static) if (n > ORC_PAR_MIN)
    for (int64_t i = 0; i < n; ++i) r[i] = alpha[i] - Qa[i] + 1.0;
    double lam = 0.0;
    orc_project(r, y, n, C, pr, &lam);
#pragma omp parallel for schedule(static) if (n > ORC_PAR_MIN)
    for (int64_t i = 0; i < n; ++i) { double d = alpha[i] - pr[i]; r[i] = d * d; pr[i] = alpha[i] * alpha[i]; }
    double num = sqrt(pair_sum(r, n)), na = sqrt(pair_sum(pr, n));
    if (lam_out) *lam_out = lam;
    if (w_out) memcpy(w_out, w, (size_t)q * sizeof(double));
    free(w); free(Qa); free(r); free(pr);
    return num / (1.0 + na);
}

/* R_KKT of eq. (4.1) for CSR X: the steps of orc_kkt with the CSR products. */
double orc_kkt_csr(const int64_t *ip, const int32_t *ix, const void *vals, int v_f32,
                   const int8_t *y, int64_t n, int64_t q, double C, const double *alpha,
                   double *lam_out, double *w_out)
{
    double *w = (double *)malloc((size_t)(q > 0 ? q : 1) * sizeof(double));
    double *Qa = (double *)malloc((size_t)n * sizeof(double));
    double *r = (double *)malloc((size_t)n * sizeof(double));
    double *pr = (double *)malloc((size_t)n * sizeof(double));
    if (!w || !Qa || !r || !pr) { free(w); free(Qa); free(r); free(pr); return NAN; }
    double res = NAN, lam = 0.0;
    if (orc_rmatvec_csr(ip, ix, vals, v_f32, y, n, q, alpha, w) == ORC_OK &&
        orc_matvec_csr(ip, ix, vals, v_f32, y, n, q, w, Qa) == ORC_OK) {
#pragma omp parallel for schedule(static) if (n > ORC_PAR_MIN)
        for (int64_t i = 0; i < n; ++i) r[i] = alpha[i] - Qa[i] + 1.0;
        if (orc_project(r, y, n, C, pr, &lam) == ORC_OK) {
#pragma omp parallel for schedule(static) if (n > ORC_PAR_MIN)
            for (int64_t i = 0; i < n; ++i) { double d = alpha[i] - pr[i]; r[i] = d * d; pr[i] = alpha[i] * alpha[i]; }
            res = sqrt(pair_sum(r, n)) / (1.0 + sqrt(pair_sum(pr, n)));
        }
    }
    if (lam_out) *lam_out = lam;
    if (w_out) memcpy(w_out, w, (size_t)q * sizeof(double));
    free(w); free(Qa); free(r); free(pr);
    return res;
}

/* Bias b (reading: the paper never defines b for the C-SVC).  b is a
 * minimiser of the primal hinge term sum_i max(0, 1 - y_i(<w,x_i> + b)) of
 * eq. (1.1) for the given w.  Its slope in b is -n_+ + #{kinks < b} with kinks
 * k_i = y_i - <w,x_i>, so the minimisers are the interval between the n_+-th
 * and (n_+ + 1)-th smallest kinks; the midpoint is returned. */
double orc_bias(const void *X, int x_f32, const int8_t *y, int64_t n, int64_t q,
                const double *w, double *lo_out, double *hi_out)
{
    double *k = (double *)malloc((size_t)n * sizeof(double));
    if (!k) return NAN;
    int64_t npos = 0;
    for (int64_t i = 0; i < n; ++i)
        if (y[i] > 0) ++npos;
#pragma omp parallel for schedule(static) if (n > ORC_PAR_MIN)
    for (int64_t i = 0; i < n; ++i) {
        double m = 0.0;
        for (int64_t j = 0; j < q; ++j) m += x_at(X, x_f32, q, i, j) * w[j];
        k[i] = (double)y[i] - m;
    }
    sort_doubles(k, n);
    double lo, hi;
    if (npos == 0) { lo = -INFINITY; hi = k[0]; }
    else if (npos == n) { lo = k[n - 1]; hi = INFINITY; }
    else { lo = k[npos - 1]; hi = k[npos]; }
    if (lo_out) *lo_out = lo;
    if (hi_out) *hi_out = hi;
    free(k);
    return 0.5 * (lo + hi);
}

/* Primal objective of eq. (1.1) with the linear kernel. */
double orc_primal(const void *X, int x_f32, const int8_t *y, int64_t n, int64_t q,
                  double C, const double *w, double b)
{
    double *h = (double *)malloc((size_t)n * sizeof(double));
    if (!h) return NAN;
#pragma omp parallel for schedule(static) if (n > ORC_PAR_MIN)
    for (int64_t i = 0; i < n; ++i) {
        double m = 0.0;
        for (int64_t j = 0; j < q; ++j) m += x_at(X, x_f32, q, i, j) * w[j];
        double t = 1.0 - (double)y[i] * (m + b);
        h[i] = t > 0.0 ? t : 0.0;
    }
    double s = 0.5 * dot_q(w, w, q) + C * pair_sum(h, n);
    free(h);
    return s;
}

/* ------------------------------------------------------------ the solver */

typedef struct {
    double tol;            /* R_KKT tolerance (eq. (4.1)) */
    int max_outer;         /* 200 (Sec. 4.1) */
    int max_inner;         /* reading: 50 */
    int max_ls;            /* reading: 40 trials */
    double sigma0;         /* reading: 1 */
    double sigma_growth;   /* reading: 5 */
    double sigma_max;      /* reading: 1e6 */
    double mu;             /* Algorithm 3: mu in (0, 1/2); reading 1e-4 */
    double delta;          /* Algorithm 3: delta in (0,1); reading 0.5 */
    double tau;            /* Algorithm 3: tau in (0,1]; reading 0.5 (unused by the exact solve) */
    double eta;            /* Algorithm 3: eta in (0,1); reading 0.1 (unused by the exact solve) */
    int newton_form;       /* 0 auto, 1 q-form, 2 p-form */
} orc_params;

typedef struct {
    double objective;      /* 1/2 |A'alpha|^2 - e'alpha */
    double kkt;            /* R_KKT(alpha) */
    double b;              /* bias (orc_bias) */
    double lam_kkt;        /* projection multiplier of the final KKT check */
    double primal;         /* eq. (1.1) at (w, b) */
    double gap;            /* primal - dual, dual = -objective */
    double sigma;          /* final sigma */
    int outer;             /* outer iterations taken */
    int inner_total;       /* Newton iterations, summed */
    int status;
    int pad;
    int64_t n_free, n_upper, n_sv;
} orc_result;

typedef struct {
    int k, inner, ls_fail, pad;
    double sigma, kkt, ytalpha, amin, amax, gnorm;
    int64_t p;
} orc_trace;

void orc_default_params(orc_params *P)
{
    P->tol = 1e-6; P->max_outer = 200; P->max_inner = 50; P->max_ls = 40;
    P->sigma0 = 1.0; P->sigma_growth = 5.0; P->sigma_max = 1e6;
    P->mu = 1e-4; P->delta = 0.5; P->tau = 0.5; P->eta = 0.1; P->newton_form = 0;
}

static double norm2(const double *a, int64_t n, double *tmp)
{
#pragma omp parallel for schedule(static) if (n > ORC_PAR_MIN)
    for (int64_t i = 0; i < n; ++i) tmp[i] = a[i] * a[i];
    return sqrt(pair_sum(tmp, n));
}

/* SSsNAL (Algorithm 1 with Algorithm 3 inside) on the C-SVC dual.
 * alpha (n) in/out: on entry the start point if warm != 0 (else zeros are
 * used, Sec. 4.1); on exit the solution.  w (q) out: A'alpha.
 * trace: optional, max_outer records. */
int orc_solve(const void *X, int x_f32, const int8_t *y, int64_t n, int64_t q,
              double C, const orc_params *P, double *alpha, int warm, double *w,
              orc_result *res, orc_trace *trace)
{
    if (!X || !y || !alpha || !w || !res || n < 1 || q < 1 || !(C > 0.0) || !P)
        return ORC_ERR_ARG;
    memset(res, 0, sizeof(*res));
    int64_t npos = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (y[i] != 1 && y[i] != -1) return ORC_ERR_ARG;
        if (y[i] > 0) ++npos;
    }
    if (npos == 0 || npos == n) {
        for (int64_t i = 0; i < n; ++i) alpha[i] = 0.0;
        for (int64_t j = 0; j < q; ++j) w[j] = 0.0;
        res->b = NAN; res->status = ORC_ERR_DEGENERATE;
        return ORC_ERR_DEGENERATE;
    }
    size_t nb = (size_t)n * sizeof(double), qb = (size_t)q * sizeof(double);
    double *z = malloc(nb), *u = malloc(nb), *pi = malloc(nb), *dz = malloc(nb);
    double *ut = malloc(nb), *pit = malloc(nb), *tmp = malloc(nb), *tmp2 = malloc(nb);
    double *v = malloc(qb), *g = malloc(qb), *dv = malloc(qb), *atp = malloc(qb), *gsc = malloc(qb);
    int64_t *J = malloc((size_t)n * sizeof(int64_t));
    if (!z || !u || !pi || !dz || !ut || !pit || !tmp || !tmp2 || !v || !g || !dv || !atp || !gsc || !J) {
        free(z); free(u); free(pi); free(dz); free(ut); free(pit); free(tmp); free(tmp2);
        free(v); free(g); free(dv); free(atp); free(gsc); free(J);
        return ORC_ERR_OOM;
    }
    if (!warm) for (int64_t i = 0; i < n; ++i) alpha[i] = 0.0;
    /* w^0 = 0 (Sec. 4.1); with a warm alpha the ALM dual still starts at
     * v = A'alpha, the natural warm start in Ran(A'). */
    if (warm) orc_rmatvec(X, x_f32, y, n, q, alpha, v, NULL);
    else memset(v, 0, qb);

    double sigma = P->sigma0;
    double lam = 0.0, lam_t = 0.0;
    double R = orc_kkt(X, x_f32, y, n, q, C, alpha, NULL, NULL), Rprev = R;
    int status = ORC_ERR_NOT_CONVERGED;
    int inner_total = 0, k;
    if (R <= P->tol) status = ORC_OK;
    for (k = 0; k < P->max_outer && status != ORC_OK; ++k) {
        /* reading: inner tolerances eps_k = delta_k = 0.1 * 0.5^k */
        double epsk = 0.1 * pow(0.5, (double)k);
        double asq = 0.0;
#pragma omp parallel for schedule(static) if (n > ORC_PAR_MIN)
        for (int64_t i = 0; i < n; ++i) tmp[i] = alpha[i] * alpha[i];
        asq = pair_sum(tmp, n);
        orc_matvec(X, x_f32, y, n, q, v, z);            /* z = A v = Q w */
        int j, ls_fail = 0;
        double gn = 0.0;
        int64_t p = 0;
        for (j = 0; ; ++j) {
            /* u(w) = x^k - sigma (Q w + c), c = -e  (eq. (3.3)) */
#pragma omp parallel for schedule(static) if (n > ORC_PAR_MIN)
            for (int64_t i = 0; i < n; ++i) u[i] = alpha[i] - sigma * (z[i] - 1.0);
            orc_project(u, y, n, C, pi, &lam);
            /* grad psi = Q w - Q Pi(u) = A g,  g = v - A'pi  (eq. (3.10)) */
            orc_rmatvec(X, x_f32, y, n, q, pi, atp, gsc);
            for (int64_t c = 0; c < q; ++c) g[c] = v[c] - atp[c];
            gn = sqrt(dot_q(g, g, q));
            /* stopping tests (A') and (B') in q-space, with a roundoff floor */
#pragma omp parallel for schedule(static) if (n > ORC_PAR_MIN)
            for (int64_t i = 0; i < n; ++i) { double d = pi[i] - alpha[i]; tmp[i] = d * d; }
            double dx = sqrt(pair_sum(tmp, n));
            double tol_in = fmin(epsk, epsk * dx) / sqrt(sigma);
            double floor_g = 1e-15 * sqrt(dot_q(gsc, gsc, q));
            if (gn <= fmax(tol_in, floor_g) || j >= P->max_inner || ls_fail) break;
            /* Step 1: Newton direction on the free set J */
            p = orc_free_set(u, y, n, C, lam, J);
            int rc = orc_newton_direction(X, x_f32, y, n, q, J, p, sigma, g, dv, P->newton_form);
            if (rc != ORC_OK) { status = rc; goto done; }
            /* Step 2: Armijo line search on psi (differences taken term by term) */
            orc_matvec(X, x_f32, y, n, q, dv, dz);       /* A dv = Q d */
            double slope = dot_q(g, dv, q);              /* <grad psi, d> */
            double vdv = dot_q(v, dv, q), dvdv = dot_q(dv, dv, q);
            double t = 1.0;
            int m, accepted = 0;
            for (m = 0; m < P->max_ls; ++m) {
#pragma omp parallel for schedule(static) if (n > ORC_PAR_MIN)
                for (int64_t i = 0; i < n; ++i) ut[i] = u[i] - t * sigma * dz[i];
                orc_project(ut, y, n, C, pit, &lam_t);
#pragma omp parallel for schedule(static) if (n > ORC_PAR_MIN)
                for (int64_t i = 0; i < n; ++i)
                    tmp[i] = pit[i] * (2.0 * ut[i] - pit[i]) - pi[i] * (2.0 * u[i] - pi[i]);
                double dpsi = t * vdv + 0.5 * t * t * dvdv + pair_sum(tmp, n) / (2.0 * sigma);
                if (dpsi <= P->mu * t * slope) { accepted = 1; break; }
                t *= P->delta;
            }
            if (!accepted) { ls_fail = 1; continue; }
            /* Step 3 */
            for (int64_t c = 0; c < q; ++c) v[c] += t * dv[c];
#pragma omp parallel for schedule(static) if (n > ORC_PAR_MIN)
            for (int64_t i = 0; i < n; ++i) z[i] += t * dz[i];
        }
        inner_total += j;
        (void)asq;
        /* Step 2 of Algorithm 1 in the simplified form of eq. (3.5) */
#pragma omp parallel for schedule(static) if (n > ORC_PAR_MIN)
        for (int64_t i = 0; i < n; ++i) alpha[i] = pi[i];
        R = orc_kkt(X, x_f32, y, n, q, C, alpha, NULL, NULL);
        if (trace) {
            orc_trace *T = &trace[k];
            T->k = k; T->inner = j; T->ls_fail = ls_fail; T->sigma = sigma; T->kkt = R;
            T->ytalpha = 0.0; T->amin = INFINITY; T->amax = -INFINITY;
            for (int64_t i = 0; i < n; ++i) {
                tmp[i] = (double)y[i] * alpha[i];
                if (alpha[i] < T->amin) T->amin = alpha[i];
                if (alpha[i] > T->amax) T->amax = alpha[i];
            }
            T->ytalpha = pair_sum(tmp, n); T->gnorm = gn; T->p = p;
        }
        if (!isfinite(R)) { status = ORC_ERR_NUMERIC; break; }
        if (R <= P->tol) { status = ORC_OK; ++k; break; }
        /* reading: sigma grows when R_KKT fell by less than one half */
        if (R > 0.5 * Rprev) sigma = fmin(P->sigma_max, P->sigma_growth * sigma);
        Rprev = R;
    }
done:
    res->outer = k;
    res->inner_total = inner_total;
    res->sigma = sigma;
    res->status = status;
    {
        double lamk = 0.0;
        res->kkt = orc_kkt(X, x_f32, y, n, q, C, alpha, &lamk, w);
        res->lam_kkt = lamk;
        double wsq = dot_q(w, w, q);
#pragma omp parallel for schedule(static) if (n > ORC_PAR_MIN)
        for (int64_t i = 0; i < n; ++i) tmp[i] = alpha[i];
        double sa = pair_sum(tmp, n);
        res->objective = 0.5 * wsq - sa;
        res->b = orc_bias(X, x_f32, y, n, q, w, NULL, NULL);
        res->primal = orc_primal(X, x_f32, y, n, q, C, w, res->b);
        res->gap = res->primal + res->objective;
        int64_t nf = 0, nu = 0, ns = 0;
        for (int64_t i = 0; i < n; ++i) {
            if (alpha[i] > 0.0) ++ns;
            if (alpha[i] >= C) ++nu;
            else if (alpha[i] > 0.0) ++nf;
        }
        res->n_free = nf; res->n_upper = nu; res->n_sv = ns;
    }
    free(z); free(u); free(pi); free(dz); free(ut); free(pit); free(tmp); free(tmp2);
    free(v); free(g); free(dv); free(atp); free(gsc); free(J);
    return status;
}
