// gqp.cuh -- workspace and kernel launchers of the unified-QP solver
// (gqp.cu, k_gqp.cu).  Not part of the public ABI.
//
// The problem (Sec. 1, eq. (1.5)): min 1/2 x'Qx + c'x  s.t.  a'x = d,
// l <= x <= u, with Q = B B' and B an n x q matrix held either densely
// (layout DENSE) or, for the SVR dual of eq. (1.4), as B = [X; -X] over an
// m x q matrix X (layout STACKED, n = 2m), so that the 2m rows are never
// stored.  Everything is FP64 (X may be stored FP32 and is widened exactly).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace svm {
namespace gqp {

enum Layout : int { DENSE = 0, STACKED = 1 };

// What the device reports after a projection (read back by the host).
struct ProjRec {
    double lam;        // lambda-hat: pi = clip(u - lambda a, l, u)
    double dpx;        // |pi - x|^2                     (x = the base point)
    double psi;        // sum pi (2w - pi) - [base] sum pib (2wb - pib)   (w = the projected point)
    double xx;         // |x|^2
    double cx;         // c'x
    double sJ;         // a_J'a_J over the free set J
    double feas;       // a'x - d of the base point x
    long long p;       // |J|
    long long nfree_x; // #{l_i < x_i < u_i}
    int passes;
    int status;        // 0 ok; 1 pass cap; 2 infeasible (a'x = d unreachable in the box)
};

// Inputs of one projection: the point w_i = x_i - sigma (z_i + t dz_i + c_i)
// (dz may be null), projected onto {a'y = d, l <= y <= u}.
struct ProjReq {
    const double *x = nullptr, *z = nullptr, *dz = nullptr;
    double sigma = 1.0, t = 0.0;
    const double *lam0 = nullptr;        // warm start (device, nullable)
    double *lam_out = nullptr;           // lambda-hat (device, nullable; may equal lam0)
    double *w_out = nullptr;             // the projected point
    double *pi_out = nullptr;
    int32_t *J = nullptr;                // free set, ascending (nullable)
    const double *pib = nullptr, *wb = nullptr;   // base of the psi difference (nullable)
};

struct Ws {
    // problem
    long long n = 0, m = 0;   // variables; rows of the stored matrix (m = n or n/2)
    int q = 0, layout = DENSE;
    bool xf32 = false;
    const void *X = nullptr;
    const double *c = nullptr, *a = nullptr, *lo = nullptr, *hi = nullptr;
    double d = 0.0;
    double *ainv = nullptr;   // 1/a_i (0 where a_i = 0): breakpoint offsets
    cudaStream_t st = nullptr;
    int dev = 0, nsm = 0;
    int proj_grid = 0, rm_grid = 0;
    // scratch
    double *part = nullptr;   // block partials (projection, products, Gram)
    size_t part_len = 0;
    long long *cnt = nullptr; // per-block free counts of the compaction
    unsigned *bar = nullptr;
    int *err = nullptr;
    ProjRec *rec = nullptr;   // device record of the last projection
};

cudaError_t setup(Ws &W);                                   // grid sizes, ainv, scratch
cudaError_t matvec(Ws &W, const double *v, double *z);      // z = B v
// out = B'y; scale (nullable) = | |B|'|y| |^2 into *scale_dev
cudaError_t rmatvec(Ws &W, const double *y, double *out, double *scale_dev);
cudaError_t project(Ws &W, const ProjReq &r);               // record in W.rec
// dv from (I + sigma (G - h h'/s)) dv = -g, G = B_J'B_J, h = B_J'a_J, s = a_J'a_J
// (s = 0: no rank-one term), by the FP64 Cholesky of k_newton.cu; M: q*q scratch.
cudaError_t newton(Ws &W, const int32_t *J, long long p, double sJ, double sigma, const double *g, double *dv,
                   double *M);
// red[0] = g'dv, red[1] = v'dv, red[2] = dv'dv, red[3] = |g|^2 for g = v - btp (written)
cudaError_t qvec(Ws &W, const double *v, const double *btp, double *g, const double *dv, double *red);
cudaError_t axpy_q(Ws &W, double *v, double t, const double *dv);            // v += t dv (q)
cudaError_t axpy_n(Ws &W, double *z, double t, const double *dz);            // z += t dz (n)
// checks at create: flags[0] non-finite X, [1] non-finite c/a/l/u, [2] l > u
cudaError_t validate(Ws &W, int *flags);
// the SVR dual's vectors: c = [eps + y; eps - y], a = [e; -e], l = 0, u = C (n = 2m)
cudaError_t svr_vectors(Ws &W, const double *y, double eps, double C, double *c, double *a, double *lo,
                        double *hi);

}  // namespace gqp

// FP64 Cholesky solve of k_newton.cu: dv = -M^{-1} g (M q x q, factored in place).
cudaError_t launch_chol_solve(int q, double *M, const double *g, double *dv, int *err, cudaStream_t st);

}  // namespace svm
