// k_newton.cu -- the reduced Newton system of Algorithm 3 / Proposition 3.5.
//
// With Q = A A' and the HS-Jacobian P = S (I - a a'/(a'S a)) S of Theorem 3.2
// (a = y, S = Diag(1_J)), the n-space Newton system (Q + sigma Q P Q) d =
// -grad psi, d in Ran(Q), is, in the coordinates dv = A'd (the substitution
// L = A in the proof of Proposition 3.5),
//     (I_q + sigma (G - h h'/p)) dv = -g,   G = X_J'X_J,  h = X_J'1,  p = |J|
// (y_i^2 = 1, so A_J'A_J = X_J'X_J and A_J'a_J = X_J'1).  The matrix is SPD
// (I - y_J y_J'/p is an orthogonal projector), so it is factored by Cholesky.
// p = 0 is case (b) of Proposition 3.5 with P = 0: dv = -g.
//
// PLAIN_FP64: the Gram over the gathered rows J is accumulated in FP64 in
// 32x32 lower-triangle tiles, split over row chunks; the q x q factorisation
// and the two triangular solves run in one block (shared memory when q <= 144).
#include <math.h>

#include "internal.cuh"

namespace svm {

constexpr int kGT = 32;   // Gram tile
constexpr int kGR = 16;   // rows staged per step

// part[ks][q][q] (lower tiles) and hpart[ks][q]
template <typename TX>
__global__ void __launch_bounds__(256) gram_kernel(const TX *__restrict__ X, int q, const int32_t *__restrict__ J,
                                                   long long p, int KS, double *__restrict__ part,
                                                   double *__restrict__ hpart)
{
    const int nt = (q + kGT - 1) / kGT;
    int t = blockIdx.x;          // lower-triangle tile index
    int ti = 0;
    while (t > ti) { t -= ti + 1; ++ti; }
    const int tj = t;
    const int ks = blockIdx.y;
    const long long per = (p + KS - 1) / KS;
    const long long r0 = (long long)ks * per;
    const long long r1 = r0 + per < p ? r0 + per : p;
    __shared__ double sA[kGR][kGT], sB[kGR][kGT];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
    double acc[4] = {0, 0, 0, 0};
    double hacc = 0.0;
    const int ca = ti * kGT, cb = tj * kGT;
    (void)nt;
    for (long long rb = r0; rb < r1; rb += kGR) {
        for (int e = threadIdx.x; e < kGR * kGT; e += blockDim.x) {
            int rr = e / kGT, cc = e % kGT;
            long long r = rb + rr;
            double va = 0.0, vb = 0.0;
            if (r < r1) {
                const TX *row = X + (long long)J[r] * q;
                if (ca + cc < q) va = (double)row[ca + cc];
                if (cb + cc < q) vb = (double)row[cb + cc];
            }
            sA[rr][cc] = va;
            sB[rr][cc] = vb;
        }
        __syncthreads();
#pragma unroll 4
        for (int rr = 0; rr < kGR; ++rr) {
            double b = sB[rr][tx];
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[k] = fma(sA[rr][ty + 8 * k], b, acc[k]);
            if (ti == tj && ty == 0) hacc += b;
        }
        __syncthreads();
    }
    double *P = part + (size_t)ks * q * q;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        int a = ca + ty + 8 * k, b = cb + tx;
        if (a < q && b < q) P[(size_t)a * q + b] = acc[k];
    }
    if (ti == tj && ty == 0 && cb + tx < q) hpart[(size_t)ks * q + cb + tx] = hacc;
}

// M = I + sigma (G - h h'/p), both triangles, from the KS partials.
__global__ void build_m_kernel(int q, int KS, const double *__restrict__ part, const double *__restrict__ hpart,
                               double p, double sigma, double *__restrict__ M, double *__restrict__ h)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)q * q;
         e += (long long)gridDim.x * blockDim.x) {
        int a = (int)(e / q), b = (int)(e % q);
        if (b > a) continue;
        // lower-tile element (a, b) lives in tile (a/32, b/32) with a/32 >= b/32
        if (a / kGT < b / kGT) continue;
        double gsum = 0.0, ha = 0.0, hb = 0.0;
        for (int ks = 0; ks < KS; ++ks) {
            gsum += part[(size_t)ks * q * q + (size_t)a * q + b];
            ha += hpart[(size_t)ks * q + a];
            hb += hpart[(size_t)ks * q + b];
        }
        double m = sigma * (gsum - ha * hb / p);
        if (a == b) { m += 1.0; h[a] = ha; }
        M[(size_t)a * q + b] = m;
        M[(size_t)b * q + a] = m;
    }
}

// One block: Cholesky of M (q x q, FP64) in place and dv = -M^{-1} g.
// SMEM: factor in shared memory (q <= 144), else in global memory.
template <bool SMEM>
__global__ void __launch_bounds__(1024) chol_solve_kernel(int q, double *__restrict__ Mg, const double *__restrict__ g,
                                                          double *__restrict__ dv, int *err)
{
    extern __shared__ double dsm[];
    double *M = SMEM ? dsm : Mg;
    double *b = SMEM ? dsm + (size_t)q * q : dv;
    __shared__ int bad;
    const int tid = threadIdx.x;
    if (SMEM)
        for (int e = tid; e < q * q; e += blockDim.x) M[e] = Mg[e];
    for (int j = tid; j < q; j += blockDim.x) b[j] = -g[j];
    if (tid == 0) bad = 0;
    __syncthreads();
    for (int j = 0; j < q; ++j) {
        if (tid == 0) {
            double d = M[(size_t)j * q + j];
            if (!(d > 0.0) || !isfinite(d)) { bad = 1; d = 1.0; }
            M[(size_t)j * q + j] = sqrt(d);
        }
        __syncthreads();
        double djj = M[(size_t)j * q + j];
        for (int i = j + 1 + tid; i < q; i += blockDim.x) M[(size_t)i * q + j] /= djj;
        __syncthreads();
        const int wy = tid >> 5, wx = tid & 31, ny = blockDim.x >> 5;
        for (int i = j + 1 + wy; i < q; i += ny) {
            double lij = M[(size_t)i * q + j];
            for (int k = j + 1 + wx; k <= i; k += 32) M[(size_t)i * q + k] -= lij * M[(size_t)k * q + j];
        }
        __syncthreads();
    }
    // forward: L x = b
    for (int k = 0; k < q; ++k) {
        if (tid == 0) b[k] /= M[(size_t)k * q + k];
        __syncthreads();
        double xk = b[k];
        for (int i = k + 1 + tid; i < q; i += blockDim.x) b[i] -= M[(size_t)i * q + k] * xk;
        __syncthreads();
    }
    // backward: L' x = b
    for (int k = q - 1; k >= 0; --k) {
        if (tid == 0) b[k] /= M[(size_t)k * q + k];
        __syncthreads();
        double xk = b[k];
        for (int i = tid; i < k; i += blockDim.x) b[i] -= M[(size_t)k * q + i] * xk;
        __syncthreads();
    }
    if (SMEM)
        for (int j = tid; j < q; j += blockDim.x) dv[j] = b[j];
    if (tid == 0 && bad) set_err(err, DEV_CHOL);
}

static int g_chol_smem_set = 0;

cudaError_t launch_newton(Work &W, const int32_t *J, long long p_host, const long long *p_dev, double sigma,
                          const double *g, double *dv)
{
    (void)p_dev;
    const int q = (int)W.q;
    if (p_host <= 0) return launch_negcopy(W, g, dv);
    const int nt = (q + kGT - 1) / kGT;
    const int ntiles = nt * (nt + 1) / 2;
    long long ks = (p_host + 255) / 256;
    int KSmax = (int)(W.part_len / ((size_t)q * q + q));
    if (KSmax > 4 * W.nsm) KSmax = 4 * W.nsm;
    if (ks > KSmax) ks = KSmax;
    if (ks < 1) ks = 1;
    double *part = W.part;
    double *hpart = W.part + (size_t)ks * q * q;
    dim3 grid(ntiles, (unsigned)ks);
    if (W.xf32)
        gram_kernel<float><<<grid, 256, 0, W.st>>>((const float *)W.X, q, J, p_host, (int)ks, part, hpart);
    else
        gram_kernel<double><<<grid, 256, 0, W.st>>>((const double *)W.X, q, J, p_host, (int)ks, part, hpart);
    build_m_kernel<<<W.nsm * 2, 256, 0, W.st>>>(q, (int)ks, part, hpart, (double)p_host, sigma, W.M, W.h);
    W.nlaunch += 3;   // gram, build_m, chol_solve
    size_t smem = ((size_t)q * q + q) * sizeof(double);
    if (q <= 144) {
        if (!g_chol_smem_set) {
            cudaFuncSetAttribute(chol_solve_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
            g_chol_smem_set = 1;
        }
        chol_solve_kernel<true><<<1, 1024, smem, W.st>>>(q, W.M, g, dv, W.err);
    } else {
        chol_solve_kernel<false><<<1, 1024, 0, W.st>>>(q, W.M, g, dv, W.err);
    }
    return cudaGetLastError();
}

}  // namespace svm
