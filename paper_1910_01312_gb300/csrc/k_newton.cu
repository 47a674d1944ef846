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

// M = I + sigma (G - h h'/p), both triangles, from the KS partials (and,
// when Mf != nullptr, its FP32 (hi, lo) split for the double-float operator).
__global__ void build_m_kernel(int q, int KS, const double *__restrict__ part, const double *__restrict__ hpart,
                               double p, double sigma, double *__restrict__ M, double *__restrict__ h,
                               float2 *__restrict__ Mf)
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
        if (Mf) {
            const float hi = (float)m;
            const float2 v = make_float2(hi, (float)(m - (double)hi));
            Mf[(size_t)a * q + b] = v;
            Mf[(size_t)b * q + a] = v;
        }
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

// ------------------------------------------------------------ mixed form

// Gram of FP32 rows with exact products (TwoProd) and double-float sums
// (TwoSum) on the FP32 pipes; same tiling and outputs as gram_kernel.
__global__ void __launch_bounds__(256) gram_df_kernel(const float *__restrict__ X, int q, const int32_t *__restrict__ J,
                                                      long long p, int KS, double *__restrict__ part,
                                                      double *__restrict__ hpart)
{
    int t = blockIdx.x;
    int ti = 0;
    while (t > ti) { t -= ti + 1; ++ti; }
    const int tj = t;
    const int ks = blockIdx.y;
    const long long per = (p + KS - 1) / KS;
    const long long r0 = (long long)ks * per;
    const long long r1 = r0 + per < p ? r0 + per : p;
    __shared__ float sA[kGR][kGT + 1], sB[kGR][kGT + 1];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
    float hs[4] = {0.f, 0.f, 0.f, 0.f}, hc[4] = {0.f, 0.f, 0.f, 0.f};
    float as[4] = {0.f, 0.f, 0.f, 0.f}, ac[4] = {0.f, 0.f, 0.f, 0.f};
    const int ca = ti * kGT, cb = tj * kGT;
    (void)hs; (void)hc;
    float hsum = 0.f, hcmp = 0.f;
    for (long long rb = r0; rb < r1; rb += kGR) {
        for (int e = threadIdx.x; e < kGR * kGT; e += blockDim.x) {
            const int rr = e / kGT, cc = e % kGT;
            const long long r = rb + rr;
            float va = 0.f, vb = 0.f;
            if (r < r1) {
                const float *row = X + (long long)J[r] * q;
                if (ca + cc < q) va = row[ca + cc];
                if (cb + cc < q) vb = row[cb + cc];
            }
            sA[rr][cc] = va;
            sB[rr][cc] = vb;
        }
        __syncthreads();
#pragma unroll 4
        for (int rr = 0; rr < kGR; ++rr) {
            const float b = sB[rr][tx];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                float pr, e, sn, tt;
                two_prod(sA[rr][ty + 8 * k], b, pr, e);
                two_sum(as[k], pr, sn, tt);
                as[k] = sn;
                ac[k] += tt + e;
            }
            if (ti == tj && ty == 0) {
                float sn, tt;
                two_sum(hsum, b, sn, tt);
                hsum = sn;
                hcmp += tt;
            }
        }
        __syncthreads();
    }
    double *P = part + (size_t)ks * q * q;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int a = ca + ty + 8 * k, b = cb + tx;
        if (a < q && b < q) P[(size_t)a * q + b] = (double)as[k] + (double)ac[k];
    }
    if (ti == tj && ty == 0 && cb + tx < q) hpart[(size_t)ks * q + cb + tx] = (double)hsum + (double)hcmp;
}

__device__ __forceinline__ double block_dot(const double *a, const double *b, int q, double *red)
{
    double s = 0.0;
    for (int j = threadIdx.x; j < q; j += blockDim.x) s = fma(a[j], b[j], s);
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    __syncthreads();
    return t;
}

// z = (L L')^{-1} r with the FP32 factor L (row stride ld), by warp 0:
// lane l owns rows l, l+32, ...  (q <= 32 * kMaxRows)
template <int kMaxRows>
__device__ void chol_apply_warp(const float *L, const float *rdiag, int ld, int q, const double *r, double *z)
{
    const int lane = threadIdx.x & 31;
    float b[kMaxRows];
    const int nr = (q + 31) / 32;
#pragma unroll
    for (int m = 0; m < kMaxRows; ++m) b[m] = (m < nr && lane + 32 * m < q) ? (float)r[lane + 32 * m] : 0.f;
    // forward: L y = b
    for (int k = 0; k < q; ++k) {
        const int own = k & 31, km = k >> 5;
        float yk = 0.f;
#pragma unroll
        for (int m = 0; m < kMaxRows; ++m)
            if (m == km) yk = b[m];
        yk = __shfl_sync(0xffffffffu, yk, own) * rdiag[k];
#pragma unroll
        for (int m = 0; m < kMaxRows; ++m) {
            const int i = lane + 32 * m;
            if (m < nr && i > k && i < q) b[m] -= L[(size_t)i * ld + k] * yk;
            if (m == km && lane == own) b[m] = yk;
        }
    }
    // backward: L' x = y
    for (int k = q - 1; k >= 0; --k) {
        const int own = k & 31, km = k >> 5;
        float xk = 0.f;
#pragma unroll
        for (int m = 0; m < kMaxRows; ++m)
            if (m == km) xk = b[m];
        xk = __shfl_sync(0xffffffffu, xk, own) * rdiag[k];
#pragma unroll
        for (int m = 0; m < kMaxRows; ++m) {
            const int i = lane + 32 * m;
            if (m < nr && i < k) b[m] -= L[(size_t)k * ld + i] * xk;
            if (m == km && lane == own) b[m] = xk;
        }
    }
#pragma unroll
    for (int m = 0; m < kMaxRows; ++m)
        if (m < nr && lane + 32 * m < q) z[lane + 32 * m] = (double)b[m];
}

// One block: FP32 Cholesky of fl32(M) (diagonal shift on breakdown) as the
// preconditioner of a conjugate-gradient solve of M dv = -g -- the CG of
// Algorithm 3, Step 1 -- stopped at |M dv + g| <= max(min(eta, |g|^{1+tau},
// 1e-10 |g|), 1e-14 |g|) or after maxit steps.  The paper's bound min(eta,
// |g|^{1+tau}) caps the residual; the 1e-10 |g| cap makes the step as exact as
// a direct solve (the next gradient is this residual when J does not change),
// at about one extra step, since each step gains ~6 digits with this
// preconditioner.  The operator is applied in double-float
// from the (hi, lo) FP32 split of M (relative accuracy ~2^-44, like FP64)
// so that the one SM doing the solve never waits on the FP64 pipe.
// Factorisation: right-looking, 32-wide panels: warp 0 factors the diagonal
// block, one thread per row solves the panel, all threads update the
// trailing matrix; three block barriers per panel.
// SMEM: the factor lives in shared memory, else in Lg (row stride q + 1).
// info[0] = CG steps, info[1] = final residual norm, info[2] = shift used.
template <bool SMEM, int NR>
__global__ void __launch_bounds__(1024) newton_pcg_kernel(int q, const double *__restrict__ M,
                                                          const float2 *__restrict__ Mf, float *__restrict__ Lg,
                                                          const double *__restrict__ g, double *__restrict__ dv,
                                                          double eta, double tau, int maxit, double *__restrict__ info,
                                                          int *err)
{
    extern __shared__ double dsm2[];
    double *x = dsm2, *r = x + q, *z = r + q, *pp = z + q, *Ap = pp + q, *rold = Ap + q;
    float2 *pf = reinterpret_cast<float2 *>(rold + q);   // df copy of pp
    const int ld = q + 1;
    float *L = SMEM ? reinterpret_cast<float *>(pf + q) : Lg;
    __shared__ double red[32];
    __shared__ int bad;
    __shared__ float rdiag[1024];   // 1 / L_jj of the final factor (q <= 1024)
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    // largest diagonal entry (block reduction), scale of the breakdown shift
    double md = 0.0;
    for (int j = tid; j < q; j += nt) md = fmax(md, (double)Mf[(size_t)j * q + j].x);
    md = warp_max(md);
    if (lane == 0) red[warp] = md;
    __syncthreads();
    double maxdiag = 0.0;
    for (int w = 0; w < nw; ++w) maxdiag = fmax(maxdiag, red[w]);
    __syncthreads();
    float shift = 0.f;
    for (int attempt = 0; attempt < 6; ++attempt) {
        for (int i = warp; i < q; i += nw)
            for (int j = lane; j <= i; j += 32) L[(size_t)i * ld + j] = Mf[(size_t)i * q + j].x + (i == j ? shift : 0.f);
        if (tid == 0) bad = 0;
        __syncthreads();
        for (int kb = 0; kb < q; kb += 32) {
            const int nb = (q - kb) < 32 ? (q - kb) : 32;
            // (1) diagonal block, warp 0, lane i owns row kb + i
            if (warp == 0) {
                for (int j = 0; j < nb; ++j) {
                    const float d = L[(size_t)(kb + j) * ld + kb + j];
                    const bool okp = (d > 0.f) && isfinite(d);
                    const float rs = okp ? rsqrtf(d) : 1.f;
                    if (!okp && lane == 0) bad = 1;
                    __syncwarp();
                    if (lane > j && lane < nb) L[(size_t)(kb + lane) * ld + kb + j] *= rs;
                    if (lane == j) { L[(size_t)(kb + j) * ld + kb + j] = okp ? d * rs : 1.f; rdiag[kb + j] = rs; }
                    __syncwarp();
                    if (lane > j && lane < nb) {
                        const float lij = L[(size_t)(kb + lane) * ld + kb + j];
                        for (int k = j + 1; k <= lane; ++k)
                            L[(size_t)(kb + lane) * ld + kb + k] -= lij * L[(size_t)(kb + k) * ld + kb + j];
                    }
                    __syncwarp();
                }
            }
            __syncthreads();
            if (bad) break;
            // (2) panel rows below the block: x L_b' = a, one thread per row
            for (int i = kb + nb + tid; i < q; i += nt) {
                float *row = L + (size_t)i * ld + kb;
                for (int j = 0; j < nb; ++j) {
                    float v = row[j];
                    const float *lj = L + (size_t)(kb + j) * ld + kb;
                    for (int m = 0; m < j; ++m) v -= row[m] * lj[m];
                    row[j] = v * rdiag[kb + j];
                }
            }
            __syncthreads();
            // (3) trailing update, rows i = base + wy + 32a, columns k = base + wx + 32b, k <= i
            const int base = kb + nb;
            for (int i = base + warp; i < q; i += nw) {
                const float *li = L + (size_t)i * ld + kb;
                for (int k = base + lane; k <= i; k += 32) {
                    const float *lk = L + (size_t)k * ld + kb;
                    float acc = 0.f;
#pragma unroll 8
                    for (int m = 0; m < nb; ++m) acc = fmaf(li[m], lk[m], acc);
                    L[(size_t)i * ld + k] -= acc;
                }
            }
            __syncthreads();
        }
        __syncthreads();
        if (!bad) break;
        shift = (shift == 0.f) ? (float)(1e-7 * maxdiag) : shift * 100.f;
        __syncthreads();
    }
    if (bad) {
        if (tid == 0) set_err(err, DEV_CHOL);
        return;
    }
    // CG on M dv = -g
    for (int j = tid; j < q; j += nt) { x[j] = 0.0; r[j] = -g[j]; }
    __syncthreads();
    const double gn = sqrt(block_dot(r, r, q, red));
    const double tol = fmax(fmin(fmin(eta, pow(gn, 1.0 + tau)), 1e-10 * gn), 1e-14 * gn);
    if (tid < 32) chol_apply_warp<NR>(L, rdiag, ld, q, r, z);
    __syncthreads();
    for (int j = tid; j < q; j += nt) pp[j] = z[j];
    __syncthreads();
    double rz = block_dot(r, z, q, red);
    double rn = gn;
    int it = 0;
    for (it = 0; it < maxit && rn > tol; ++it) {
        for (int j = tid; j < q; j += nt) {
            const float hi = (float)pp[j];
            pf[j] = make_float2(hi, (float)(pp[j] - (double)hi));
        }
        __syncthreads();
        // Ap = M p in double-float, warp per row
        for (int i = warp; i < q; i += nw) {
            float sh = 0.f, sc = 0.f;
            const float2 *mrow = Mf + (size_t)i * q;
            for (int j = lane; j < q; j += 32) {
                const float2 a = mrow[j], b = pf[j];
                float p0, e0, sn, t0;
                two_prod(a.x, b.x, p0, e0);
                e0 = fmaf(a.x, b.y, fmaf(a.y, b.x, e0));
                two_sum(sh, p0, sn, t0);
                sh = sn;
                sc += t0 + e0;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float s2 = __shfl_xor_sync(0xffffffffu, sh, o), c2 = __shfl_xor_sync(0xffffffffu, sc, o);
                float sn, e;
                two_sum(sh, s2, sn, e);
                e += sc + c2;
                sh = sn + e;
                sc = e - (sh - sn);
            }
            if (lane == 0) Ap[i] = (double)sh + (double)sc;
        }
        __syncthreads();
        const double pAp = block_dot(pp, Ap, q, red);
        if (!(pAp > 0.0)) break;
        const double al = rz / pAp;
        for (int j = tid; j < q; j += nt) {
            x[j] = fma(al, pp[j], x[j]);
            rold[j] = r[j];
            r[j] = fma(-al, Ap[j], r[j]);
        }
        __syncthreads();
        rn = sqrt(block_dot(r, r, q, red));
        if (rn <= tol) { ++it; break; }
        if (tid < 32) chol_apply_warp<NR>(L, rdiag, ld, q, r, z);
        __syncthreads();
        // flexible (Polak-Ribiere) beta: robust to the FP32 preconditioner
        const double rz_new = block_dot(r, z, q, red);
        const double rz_old = block_dot(rold, z, q, red);
        const double beta = fmax(0.0, (rz_new - rz_old) / rz);
        rz = rz_new;
        for (int j = tid; j < q; j += nt) pp[j] = fma(beta, pp[j], z[j]);
        __syncthreads();
    }
    for (int j = tid; j < q; j += nt) dv[j] = x[j];
    if (tid == 0 && info) { info[0] = it; info[1] = rn; info[2] = shift; }
    (void)M;
}

// ---- one-block dense SPD solver for q <= 200 (factor in shared memory) ----
// L (FP32, row stride ld = q + 1, lower triangle) and rdiag = 1 / diag(L).

// Blocked right-looking Cholesky of the matrix already in L; returns false
// (block-uniformly) when a pivot is not positive.
__device__ bool chol_blocked(float *L, float *rdiag, int q, int ld, int *bad_sh)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    for (int kb = 0; kb < q; kb += 32) {
        const int nb = (q - kb) < 32 ? (q - kb) : 32;
        // (1) diagonal block by warp 0, row kb + lane in registers
        if (warp == 0) {
            float a[32];
#pragma unroll
            for (int k = 0; k < 32; ++k) a[k] = (lane < nb && k <= lane) ? L[(size_t)(kb + lane) * ld + kb + k] : 0.f;
            bool ok = true;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                if (j < nb) {
                    const float d = __shfl_sync(0xffffffffu, a[j], j);
                    const bool okj = (d > 0.f) && isfinite(d);
                    ok = ok && okj;
                    const float rs = okj ? rsqrtf(d) : 1.f;
                    if (lane == j) a[j] = okj ? d * rs : 1.f;
                    else if (lane > j) a[j] *= rs;
#pragma unroll
                    for (int k = j + 1; k < 32; ++k) {
                        const float lkj = __shfl_sync(0xffffffffu, a[j], k);
                        if (lane >= k) a[k] -= a[j] * lkj;
                    }
                }
            }
            if (lane < nb) {
#pragma unroll
                for (int k = 0; k < 32; ++k)
                    if (k <= lane) L[(size_t)(kb + lane) * ld + kb + k] = a[k];
                float dl = 1.f;
#pragma unroll
                for (int k = 0; k < 32; ++k)
                    if (k == lane) dl = a[k];
                rdiag[kb + lane] = 1.f / dl;
            }
            if (!ok && lane == 0) *bad_sh = 1;
        }
        __syncthreads();
        if (*bad_sh) return false;
        // (2) panel rows below the block: x L_bb' = a, a warp per row, lane j holds x_j
        for (int i = kb + nb + warp; i < q; i += nw) {
            float v = (lane < nb) ? L[(size_t)i * ld + kb + lane] : 0.f;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                if (j < nb) {
                    const float xj = __shfl_sync(0xffffffffu, v, j) * rdiag[kb + j];
                    if (lane == j) v = xj;
                    else if (lane > j && lane < nb) v -= xj * L[(size_t)(kb + lane) * ld + kb + j];
                }
            }
            if (lane < nb) L[(size_t)i * ld + kb + lane] = v;
        }
        __syncthreads();
        // (3) trailing update with 4x4 register tiles: L_ik -= sum_m L_i,kb+m L_k,kb+m
        const int base = kb + nb, m = q - base;
        if (m > 0) {
            const int nbt = (m + 3) / 4;
            const int ntile = nbt * (nbt + 1) / 2;
            for (int t = tid; t < ntile; t += blockDim.x) {
                int ti = 0, tt = t;
                while (tt > ti) { tt -= ti + 1; ++ti; }
                const int i0 = base + 4 * ti, k0 = base + 4 * tt;
                float acc[4][4];
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
                for (int mm = 0; mm < nb; ++mm) {
                    float li[4], lk[4];
#pragma unroll
                    for (int a = 0; a < 4; ++a) {
                        li[a] = (i0 + a < q) ? L[(size_t)(i0 + a) * ld + kb + mm] : 0.f;
                        lk[a] = (k0 + a < q) ? L[(size_t)(k0 + a) * ld + kb + mm] : 0.f;
                    }
#pragma unroll
                    for (int a = 0; a < 4; ++a)
#pragma unroll
                        for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(li[a], lk[b], acc[a][b]);
                }
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const int i = i0 + a, k = k0 + b;
                        if (i < q && k <= i) L[(size_t)i * ld + k] -= acc[a][b];
                    }
            }
        }
        __syncthreads();
    }
    return true;
}

// b <- (L L')^{-1} b (FP32, in shared memory), blocked: warp 0 solves each
// 32-wide diagonal block with shuffles, all warps update the rest.
__device__ void chol_solve_blocked(const float *L, const float *rdiag, int q, int ld, float *b)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    // forward: L y = b
    for (int kb = 0; kb < q; kb += 32) {
        const int nb = (q - kb) < 32 ? (q - kb) : 32;
        if (warp == 0) {
            float v = (lane < nb) ? b[kb + lane] : 0.f;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                if (j < nb) {
                    const float yj = __shfl_sync(0xffffffffu, v, j) * rdiag[kb + j];
                    if (lane == j) v = yj;
                    else if (lane > j && lane < nb) v -= yj * L[(size_t)(kb + lane) * ld + kb + j];
                }
            }
            if (lane < nb) b[kb + lane] = v;
        }
        __syncthreads();
        for (int i = kb + nb + warp; i < q; i += nw) {
            float s = (lane < nb) ? L[(size_t)i * ld + kb + lane] * b[kb + lane] : 0.f;
            s = warp_sumf(s);
            if (lane == 0) b[i] -= s;
        }
        __syncthreads();
    }
    // backward: L' x = y
    const int last = ((q - 1) / 32) * 32;
    for (int kb = last; kb >= 0; kb -= 32) {
        const int nb = (q - kb) < 32 ? (q - kb) : 32;
        if (warp == 0) {
            float v = (lane < nb) ? b[kb + lane] : 0.f;
#pragma unroll
            for (int j = 31; j >= 0; --j) {
                if (j < nb) {
                    const float xj = __shfl_sync(0xffffffffu, v, j) * rdiag[kb + j];
                    if (lane == j) v = xj;
                    else if (lane < j) v -= xj * L[(size_t)(kb + j) * ld + kb + lane];
                }
            }
            if (lane < nb) b[kb + lane] = v;
        }
        __syncthreads();
        for (int i = warp; i < kb; i += nw) {
            float s = (lane < nb) ? L[(size_t)(kb + lane) * ld + i] * b[kb + lane] : 0.f;
            s = warp_sumf(s);
            if (lane == 0) b[i] -= s;
        }
        __syncthreads();
    }
}

// One block: FP32 Cholesky of fl32(M) (diagonal shift on breakdown) as the
// preconditioner of CG on M dv = -g (operator in double-float from the
// (hi, lo) split of M), stopped at |M dv + g| <= max(min(eta, |g|^{1+tau},
// 1e-10 |g|), 1e-14 |g|) -- the CG of Algorithm 3, Step 1, capped as in
// newton_pcg_kernel.  Every phase is parallel or a
// 32-step shuffle chain: no thread walks a q-long chain.
__global__ void __launch_bounds__(1024) newton_cg_smem_kernel(int q, const float2 *__restrict__ Mf,
                                                              const double *__restrict__ g, double *__restrict__ dv,
                                                              double eta, double tau, int maxit,
                                                              double *__restrict__ info, int *err)
{
    // Scalar FP64 work (norms, step sizes, the stopping test) is done by
    // thread 0 and broadcast through shared memory: replicated across 32 warps
    // it would occupy the SM's FP64 pipe for tens of microseconds.
    extern __shared__ double dsm3[];
    double *x = dsm3, *r = x + q, *pp = r + q, *Ap = pp + q, *rold = Ap + q, *z = rold + q;
    float2 *pf = reinterpret_cast<float2 *>(z + q);
    float *bz = reinterpret_cast<float *>(pf + q);
    float *rdiag = bz + q;
    const int ld = q + 1;
    float *L = rdiag + q + ((4 - (q & 3)) & 3);
    __shared__ double red[3][32];
    __shared__ double sc_tol, sc_al, sc_beta, sc_rn;
    __shared__ int sc_go;
    __shared__ float sc_shift;
    __shared__ int bad;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    // block partial sums of up to three dot products over q: warp totals to red[*][warp]
    auto dots = [&](const double *a0, const double *b0, const double *a1, const double *b1, const double *a2,
                    const double *b2, int nd) {
        double s0 = 0.0, s1 = 0.0, s2 = 0.0;
        for (int j = tid; j < q; j += nt) {
            s0 = fma(a0[j], b0[j], s0);
            if (nd > 1) s1 = fma(a1[j], b1[j], s1);
            if (nd > 2) s2 = fma(a2[j], b2[j], s2);
        }
        if (warp < (q + 31) / 32) {   // only warps holding entries reduce (q <= 200: at most 7 warps)
            s0 = warp_sum(s0);
            if (nd > 1) s1 = warp_sum(s1);
            if (nd > 2) s2 = warp_sum(s2);
        }
        if (lane == 0) { red[0][warp] = s0; red[1][warp] = s1; red[2][warp] = s2; }
        __syncthreads();
    };
    const int nwq = (q + 31) / 32;   // warps that hold vector entries (q <= nt)
    if (warp == 0) {
        float md = 0.f;
        for (int j = lane; j < q; j += 32) md = fmaxf(md, Mf[(size_t)j * q + j].x);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) md = fmaxf(md, __shfl_xor_sync(0xffffffffu, md, o));
        if (lane == 0) {
            sc_shift = 0.f;
            sc_tol = (double)md;   // reused below as the shift scale
        }
    }
    __syncthreads();
    const float maxdiag = (float)sc_tol;
    bool okf = false;
    for (int attempt = 0; attempt < 6 && !okf; ++attempt) {
        const float shift = sc_shift;
        for (int i = warp; i < q; i += nw)
            for (int j = lane; j <= i; j += 32) L[(size_t)i * ld + j] = Mf[(size_t)i * q + j].x + (i == j ? shift : 0.f);
        if (tid == 0) bad = 0;
        __syncthreads();
        okf = chol_blocked(L, rdiag, q, ld, &bad);
        __syncthreads();
        if (!okf && tid == 0) sc_shift = (shift == 0.f) ? 1e-7f * maxdiag : shift * 100.f;
        __syncthreads();
    }
    if (!okf) {
        if (tid == 0) set_err(err, DEV_CHOL);
        return;
    }
    for (int j = tid; j < q; j += nt) { x[j] = 0.0; r[j] = -g[j]; bz[j] = (float)(-g[j]); }
    __syncthreads();
    chol_solve_blocked(L, rdiag, q, ld, bz);   // z = P r
    for (int j = tid; j < q; j += nt) { z[j] = (double)bz[j]; pp[j] = z[j]; }
    __syncthreads();
    dots(r, r, r, z, r, r, 2);
    double rz = 0.0;
    if (tid == 0) {
        double rr = 0.0, t = 0.0;
        for (int w = 0; w < nwq; ++w) { rr += red[0][w]; t += red[1][w]; }
        const double gn = sqrt(rr);
        sc_tol = fmax(fmin(fmin(eta, pow(gn, 1.0 + tau)), 1e-10 * gn), 1e-14 * gn);
        sc_rn = gn;
        sc_al = t;   // rz
        sc_go = gn > sc_tol;
    }
    __syncthreads();
    rz = sc_al;
    int it = 0;
    while (sc_go && it < maxit) {
        for (int j = tid; j < q; j += nt) {
            const float hi = (float)pp[j];
            pf[j] = make_float2(hi, (float)(pp[j] - (double)hi));
        }
        __syncthreads();
        for (int i = warp; i < q; i += nw) {
            float sh = 0.f, sc = 0.f;
            const float2 *mrow = Mf + (size_t)i * q;
            for (int j = lane; j < q; j += 32) {
                const float2 a = mrow[j], bb = pf[j];
                float p0, e0, sn, t0;
                two_prod(a.x, bb.x, p0, e0);
                e0 = fmaf(a.x, bb.y, fmaf(a.y, bb.x, e0));
                two_sum(sh, p0, sn, t0);
                sh = sn;
                sc += t0 + e0;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float s2 = __shfl_xor_sync(0xffffffffu, sh, o), c2 = __shfl_xor_sync(0xffffffffu, sc, o);
                float sn, e;
                two_sum(sh, s2, sn, e);
                e += sc + c2;
                sh = sn + e;
                sc = e - (sh - sn);
            }
            if (lane == 0) Ap[i] = (double)sh + (double)sc;
        }
        __syncthreads();
        dots(pp, Ap, pp, pp, pp, pp, 1);
        if (tid == 0) {
            double pAp = 0.0;
            for (int w = 0; w < nwq; ++w) pAp += red[0][w];
            sc_go = pAp > 0.0;
            sc_al = sc_go ? rz / pAp : 0.0;
        }
        __syncthreads();
        if (!sc_go) break;
        const double al = sc_al;
        for (int j = tid; j < q; j += nt) {
            x[j] = fma(al, pp[j], x[j]);
            rold[j] = r[j];
            r[j] = fma(-al, Ap[j], r[j]);
            bz[j] = (float)r[j];
        }
        __syncthreads();
        ++it;
        dots(r, r, r, r, r, r, 1);
        if (tid == 0) {
            double rr = 0.0;
            for (int w = 0; w < nwq; ++w) rr += red[0][w];
            sc_rn = sqrt(rr);
            sc_go = sc_rn > sc_tol;
        }
        __syncthreads();
        if (!sc_go) break;
        chol_solve_blocked(L, rdiag, q, ld, bz);
        for (int j = tid; j < q; j += nt) z[j] = (double)bz[j];
        __syncthreads();
        // flexible (Polak-Ribiere) beta: robust to the FP32 preconditioner
        dots(r, z, rold, z, r, r, 2);
        if (tid == 0) {
            double rzn = 0.0, rzo = 0.0;
            for (int w = 0; w < nwq; ++w) { rzn += red[0][w]; rzo += red[1][w]; }
            sc_beta = fmax(0.0, (rzn - rzo) / rz);
            sc_al = rzn;
        }
        __syncthreads();
        const double beta = sc_beta;
        rz = sc_al;
        for (int j = tid; j < q; j += nt) pp[j] = fma(beta, pp[j], z[j]);
        __syncthreads();
    }
    for (int j = tid; j < q; j += nt) dv[j] = x[j];
    if (tid == 0 && info) { info[0] = it; info[1] = sc_rn; info[2] = sc_shift; }
}

static int g_cgs_attr = 0;

static int g_chol_smem_set = 0;
static int g_pcg_smem_set = 0;

cudaError_t launch_newton(Work &W, const int32_t *J, long long p_host, const long long *p_dev, double sigma,
                          const double *g, double *dv)
{
    (void)p_dev;
    const int q = (int)W.q;
    if (p_host <= 0) return launch_negcopy(W, g, dv);
    const int nt = (q + kGT - 1) / kGT;
    const int ntiles = nt * (nt + 1) / 2;
    long long ks = (p_host + 31) / 32;   // split-K: ~32 gathered rows per block
    int KSmax = (int)(W.part_len / ((size_t)q * q + q));
    if (KSmax > 4 * W.nsm) KSmax = 4 * W.nsm;
    if (ks > KSmax) ks = KSmax;
    if (ks < 1) ks = 1;
    double *part = W.part;
    double *hpart = W.part + (size_t)ks * q * q;
    dim3 grid(ntiles, (unsigned)ks);
    const bool mixed = W.precision == 1 && W.xf32;
    if (mixed)
        gram_df_kernel<<<grid, 256, 0, W.st>>>((const float *)W.X, q, J, p_host, (int)ks, part, hpart);
    else if (W.xf32)
        gram_kernel<float><<<grid, 256, 0, W.st>>>((const float *)W.X, q, J, p_host, (int)ks, part, hpart);
    else
        gram_kernel<double><<<grid, 256, 0, W.st>>>((const double *)W.X, q, J, p_host, (int)ks, part, hpart);
    const bool cg = W.precision == 1;
    build_m_kernel<<<W.nsm * 2, 256, 0, W.st>>>(q, (int)ks, part, hpart, (double)p_host, sigma, W.M, W.h,
                                                cg ? W.Mf : nullptr);
    W.nlaunch += 3;   // gram, build_m, and the solve below
    if (cg) {
        // FP32-Cholesky-preconditioned CG on the FP64 matrix (Algorithm 3's inexact solve)
        double *info = W.red + 12;
        const size_t smem_new = (size_t)6 * q * sizeof(double) + (size_t)q * sizeof(float2) + (size_t)2 * q * sizeof(float) +
                                16 + (size_t)q * (q + 1) * sizeof(float);
        if (smem_new <= (size_t)200 * 1024) {
            if (!g_cgs_attr) {
                const cudaError_t ea = cudaFuncSetAttribute(newton_cg_smem_kernel,
                                                            cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
                if (ea != cudaSuccess) return ea;
                g_cgs_attr = 1;
            }
            newton_cg_smem_kernel<<<1, 1024, smem_new, W.st>>>(q, W.Mf, g, dv, W.eta, W.tau, W.cg_maxit, info, W.err);
        } else {
            const size_t vec = (size_t)6 * q * sizeof(double) + (size_t)q * sizeof(float2);
            newton_pcg_kernel<false, 32><<<1, 1024, vec, W.st>>>(q, W.M, W.Mf, W.Lf, g, dv, W.eta, W.tau, W.cg_maxit,
                                                                 info, W.err);
        }
        return cudaGetLastError();
    }
    size_t smem = ((size_t)q * q + q) * sizeof(double);
    if (q <= 144) {
        if (!g_chol_smem_set) {
            const cudaError_t ea =
                cudaFuncSetAttribute(chol_solve_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
            if (ea != cudaSuccess) return ea;
            g_chol_smem_set = 1;
        }
        chol_solve_kernel<true><<<1, 1024, smem, W.st>>>(q, W.M, g, dv, W.err);
    } else {
        chol_solve_kernel<false><<<1, 1024, 0, W.st>>>(q, W.M, g, dv, W.err);
    }
    return cudaGetLastError();
}

}  // namespace svm
