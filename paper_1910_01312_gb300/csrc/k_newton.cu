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
#include "newton_dev.cuh"

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
__device__ __forceinline__ void gram_df_body(const float *__restrict__ X, int q, const int32_t *__restrict__ J,
                                             long long p, int KS, float2 *__restrict__ part,
                                             float2 *__restrict__ hpart, long long stride)
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
    float as[4] = {0.f, 0.f, 0.f, 0.f}, ac[4] = {0.f, 0.f, 0.f, 0.f};
    const int ca = ti * kGT, cb = tj * kGT;
    float hsum = 0.f, hcmp = 0.f;
    for (long long rb = r0; rb < r1; rb += kGR) {
        for (int e = threadIdx.x; e < kGR * kGT; e += blockDim.x) {
            const int rr = e / kGT, cc = e % kGT;
            const long long r = rb + rr;
            float va = 0.f, vb = 0.f;
            if (r < r1) {
                const float *row = X + (long long)J[r * stride] * q;   // row r of the (subsampled) list
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
    // double-float partials (normalised hi/lo), no FP64
    float2 *P = part + (size_t)ks * q * q;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int a = ca + ty + 8 * k, b = cb + tx;
        if (a < q && b < q) {
            float hi, lo;
            two_sum(as[k], ac[k], hi, lo);
            P[(size_t)a * q + b] = make_float2(hi, lo);
        }
    }
    if (ti == tj && ty == 0 && cb + tx < q) {
        float hi, lo;
        two_sum(hsum, hcmp, hi, lo);
        hpart[(size_t)ks * q + cb + tx] = make_float2(hi, lo);
    }
}

__global__ void __launch_bounds__(256) gram_df_kernel(const float *__restrict__ X, int q, const int32_t *__restrict__ J,
                                                      long long p, int KS, float2 *__restrict__ part,
                                                      float2 *__restrict__ hpart, long long stride)
{
    gram_df_body(X, q, J, p, KS, part, hpart, stride);
}

// The same for a batch of Newton steps (one per problem, blockIdx.z); blocks
// beyond a problem's own split count return at once.
__global__ void __launch_bounds__(256) gram_df_batch_kernel(const float *__restrict__ X, int q,
                                                            const NewtonTask *__restrict__ T)
{
    const NewtonTask &t = T[blockIdx.z];
    if ((int)blockIdx.y >= t.ks) return;
    gram_df_body(X, q, t.J, t.p, t.ks, t.part, t.hpart, 1);
}

// M = I + sigma (G - h h' / p) from the double-float split-K partials of
// gram_df_kernel, summed in a fixed order in double-float; written as the
// (hi, lo) pair Mf of the CG operator (and the factor's input).
__device__ __forceinline__ void build_m_df_body(int q, int KS, const float2 *__restrict__ part,
                                                const float2 *__restrict__ hpart, float2 pinv, float2 sig,
                                                float2 *__restrict__ Mf)
{
    // eight lanes per entry sum interleaved eighths of the KS partials, then
    // combine them by shuffles in a fixed order; four entries per warp step
    // (a warp-uniform trip count, so every lane takes part in the shuffles)
    const int lane = threadIdx.x & 31, sub = lane & 7;
    const long long wg = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwg = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long qq = (long long)q * q;
    for (long long base = wg * 4; base < qq; base += nwg * 4) {
        const long long e = base + (lane >> 3);
        const bool valid = e < qq;
        const int a = valid ? (int)(e / q) : 0, b = valid ? (int)(e - (long long)a * q) : 1;
        const bool act = valid && b <= a;
        float2 gsum = make_float2(0.f, 0.f), ha = gsum, hb = gsum;
        if (act) {
            for (int ks = sub; ks < KS; ks += 8) {
                gsum = dfx_add(gsum, __ldcg(&part[(size_t)ks * qq + e]));
                ha = dfx_add(ha, __ldcg(&hpart[(size_t)ks * q + a]));
                hb = dfx_add(hb, __ldcg(&hpart[(size_t)ks * q + b]));
            }
        }
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            gsum = dfx_add(gsum, shfl_xor_f2(gsum, o));
            ha = dfx_add(ha, shfl_xor_f2(ha, o));
            hb = dfx_add(hb, shfl_xor_f2(hb, o));
        }
        if (sub == 0 && act) {
            float2 m = dfx_mul(sig, dfx_sub(gsum, dfx_mul(dfx_mul(ha, hb), pinv)));
            if (a == b) m = dfx_addf(m, 1.f);
            Mf[(size_t)a * q + b] = m;
            Mf[(size_t)b * q + a] = m;
        }
    }
}

__global__ void build_m_df_kernel(int q, int KS, const float2 *__restrict__ part, const float2 *__restrict__ hpart,
                                  float2 pinv, float2 sig, float2 *__restrict__ Mf)
{
    build_m_df_body(q, KS, part, hpart, pinv, sig, Mf);
}

__global__ void build_m_df_batch_kernel(int q, const NewtonTask *__restrict__ T)
{
    const NewtonTask &t = T[blockIdx.z];
    build_m_df_body(q, t.ks, t.part, t.hpart, t.pinv, t.sig, t.Mf);
}

// ---- one-block dense SPD solver for q <= 200 (factor in shared memory) ----
// L (FP32, row stride ld = q + 1, lower triangle) and rdiag = 1 / diag(L).
// ---------------------------------------------------------------------------
// Newton solve for q <= 128 in one block of 512 threads: FP32 Cholesky of
// fl32(M) as the preconditioner of CG on M dv = -g with the operator applied
// in double-float from the (hi, lo) split of M -- the CG of Algorithm 3,
// Step 1.  No FP64 arithmetic except the final conversion of dv: on this part
// an FP64 operation costs ~64 cycles of latency, so a q = 128 solve with FP64
// vectors and scalars spends most of its time waiting on it.
//
// q is padded to qp = 32 ceil(q/32) with identity rows.  Shared memory holds
// the double-float M (qp x qp, the CG operator; one bulk asynchronous copy
// when q = qp) and the factor as a packed lower triangle.  The factor is
// right-looking by 8-column panels: the critical path of a Cholesky is one
// pivot after another, and an 8-wide diagonal block keeps each pivot step
// short (7 shuffles) and its unrolled code small -- wider blocks factored by
// one warp cost several times more per column.  Warp 0 factors the diagonal
// block and forms its inverse Dinv_b, the rows below become A_rb Dinv_b'
// (8-lane shuffle groups), and the trailing triangle is updated a warp per
// row.  The preconditioner is applied as blocked triangular solves through
// the Dinv_b.  CG stops at |M dv + g| <= max(min(eta, |g|^{1+tau}, 1e-10
// |g|), 1e-14 |g|) (the tolerance itself in FP32) or after maxit steps; beta
// is the flexible (Polak-Ribiere) form, robust to the FP32 preconditioner.

// t <- (L L')^{-1} t (blocked triangular solves through the Dinv_b)
__device__ __forceinline__ void cg_precond(const CgSmem &S, int qp)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nb = qp / kPb;
    for (int b = 0; b < nb; ++b) {   // forward: L y = t
        const int kb = b * kPb;
        if (warp == 0) {
            const float tv = lane < kPb ? S.t[kb + lane] : 0.f;
            const float *Db = S.D + b * kPb * kPb;
            float acc = 0.f;
#pragma unroll
            for (int k = 0; k < kPb; ++k)
                acc = fmaf(lane < kPb ? Db[lane * kPb + k] : 0.f, __shfl_sync(0xffffffffu, tv, k), acc);
            if (lane < kPb) S.t[kb + lane] = acc;
        }
        __syncthreads();
        if (b + 1 < nb) {
            const int r = kb + kPb + tid;
            if (r < qp) {
                float s = S.t[r];
#pragma unroll
                for (int k = 0; k < kPb; ++k) s = fmaf(-S.L[lpos(r, kb + k)], S.t[kb + k], s);
                S.t[r] = s;
            }
            __syncthreads();
        }
    }
    for (int b = nb - 1; b >= 0; --b) {   // backward: L' x = y
        const int kb = b * kPb;
        if (warp == 0) {
            const float tv = lane < kPb ? S.t[kb + lane] : 0.f;
            const float *Db = S.D + b * kPb * kPb;
            float acc = 0.f;
#pragma unroll
            for (int k = 0; k < kPb; ++k)
                acc = fmaf(lane < kPb ? Db[k * kPb + lane] : 0.f, __shfl_sync(0xffffffffu, tv, k), acc);
            if (lane < kPb) S.t[kb + lane] = acc;
        }
        __syncthreads();
        if (b > 0) {
            if (tid < kb) {
                float s = S.t[tid];
#pragma unroll
                for (int k = 0; k < kPb; ++k) s = fmaf(-S.L[lpos(kb + k, tid)], S.t[kb + k], s);
                S.t[tid] = s;
            }
            __syncthreads();
        }
    }
}

// sum_j a_j b_j over j < qp in double-float; every thread returns the same value
__device__ __forceinline__ float2 cg_dot(const float2 *a, const float2 *b, int qp, float2 *red)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float2 s = make_float2(0.f, 0.f);
    if (tid < qp) s = dfx_mul(a[tid], b[tid]);
    if (warp < (qp >> 5)) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s = dfx_add(s, shfl_xor_f2(s, o));
        if (lane == 0) red[warp] = s;
    }
    __syncthreads();
    float2 t = red[0];
    for (int w = 1; w < (qp >> 5); ++w) t = dfx_add(t, red[w]);
    __syncthreads();   // red is reused by the next call
    return t;
}


// M (q x q double-float pairs) into S.M, zero padded to qp (one bulk copy when
// q = qp), and the FP32 Cholesky factor of fl32(M) + shift into S.L / S.D (a
// diagonal shift is added and the factor retried when a pivot is not
// positive).  Block-uniform result; false (err set) when the copy or the
// factor failed.  *sc_shift (shared) receives the shift used.
__device__ bool cg_load_factor(CgSmem &S, int q, const float2 *__restrict__ Mf, int *err, float *sc_shift, int ld = -1)
{
    if (ld < 0) ld = q;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int qp = (q + 31) & ~31;
    __shared__ float sc_maxdiag;
    __shared__ int copy_ok;
    __shared__ __align__(8) unsigned long long mbar;
    // M into shared memory: one bulk copy when its rows need no padding
    if (q == qp && ld == q) {
        if (tid == 0) {
            mbar_init(&mbar, 1);
            mbar_fence_init();
            mbar_arrive_expect_tx(&mbar, (unsigned)(qp * qp * sizeof(float2)));
            bulk_g2s(S.M, Mf, (unsigned)(qp * qp * sizeof(float2)), &mbar);
            bool okc = mbar_wait_bounded(&mbar, 0, err);
            if (!okc) okc = mbar_wait_bounded(&mbar, 0, err);   // wait again for the copy in flight
            copy_ok = okc;
        }
    } else {
        for (int i = warp; i < qp; i += nw)
            for (int j = lane; j < qp; j += 32)
                S.M[i * qp + j] = (i < q && j < q) ? Mf[(size_t)i * ld + j] : make_float2(0.f, 0.f);
        if (tid == 0) copy_ok = 1;
    }
    if (tid == 0) *sc_shift = 0.f;
    __syncthreads();
    if (!copy_ok) return false;
    if (warp == 0) {
        float md = 0.f;
        for (int j = lane; j < q; j += 32) md = fmaxf(md, S.M[j * qp + j].x);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) md = fmaxf(md, __shfl_xor_sync(0xffffffffu, md, o));
        if (lane == 0) sc_maxdiag = md;
    }
    __syncthreads();
    bool okf = false;
    for (int attempt = 0; attempt < 6 && !okf; ++attempt) {
        const float shift = *sc_shift;
        for (int i = warp; i < qp; i += nw)
            for (int j = lane; j <= i; j += 32)
                S.L[lpos(i, j)] = (i < q) ? S.M[i * qp + j].x + (i == j ? shift : 0.f) : (i == j ? 1.f : 0.f);
        __syncthreads();
        okf = cg_factor_packed(S, qp);
        if (!okf && tid == 0) *sc_shift = (shift == 0.f) ? 1e-7f * sc_maxdiag : shift * 100.f;
        __syncthreads();
    }
    if (!okf) {
        if (tid == 0) set_err(err, DEV_CHOL);
        return false;
    }
    return true;
}

__device__ __forceinline__ void newton_cg_fast_body(int q, const float2 *__restrict__ Mf,
                                                    const double *__restrict__ g, double *__restrict__ dv,
                                                    float eta, float tau, float floor, int maxit,
                                                    double *__restrict__ info, int *err,
                                                    const double *__restrict__ vdot, double *__restrict__ rdots)
{
    extern __shared__ float4 cg_sm4[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int qp = (q + 31) & ~31, nb = qp / kPb;
    CgSmem S;
    S.M = reinterpret_cast<float2 *>(cg_sm4);
    S.L = reinterpret_cast<float *>(S.M + qp * qp);
    S.D = S.L + ((qp * (qp + 1)) >> 1);
    S.t = S.D + nb * kPb * kPb;
    S.X = reinterpret_cast<float2 *>(S.t + qp);
    S.R = S.X + qp; S.P = S.R + qp; S.AP = S.P + qp; S.Z = S.AP + qp; S.RO = S.Z + qp;
    __shared__ float2 red[8];
    __shared__ float sc_shift;
    if (!cg_load_factor(S, q, Mf, err, &sc_shift)) return;
    // CG on M dv = -g in double-float
    if (tid < qp) {
        float2 r0 = make_float2(0.f, 0.f);
        if (tid < q) {
            const double v = -g[tid];
            const float hi = (float)v;
            r0 = make_float2(hi, (float)(v - (double)hi));
        }
        S.X[tid] = make_float2(0.f, 0.f);
        S.R[tid] = r0;
        S.t[tid] = r0.x + r0.y;
    }
    __syncthreads();
    float2 rr = cg_dot(S.R, S.R, qp, red);
    const float gn = sqrtf(fmaxf(rr.x, 0.f));
    const float tol = cg_tol(gn, eta, tau, floor);
    const float tol2 = tol * tol;
    cg_precond(S, qp);
    if (tid < qp) { S.Z[tid] = make_float2(S.t[tid], 0.f); S.P[tid] = S.Z[tid]; }
    __syncthreads();
    float2 rz = cg_dot(S.R, S.Z, qp, red);
    int it = 0;
    bool go = rr.x > tol2;
    while (go && it < maxit) {
        // AP = M P: a warp per row, Dot2-style (s, c) sums of double-float products
        float2 pl[kCgMaxQ / 32];
#pragma unroll
        for (int c = 0; c < kCgMaxQ / 32; ++c) pl[c] = (lane + 32 * c < qp) ? S.P[lane + 32 * c] : make_float2(0.f, 0.f);
        for (int i = warp; i < qp; i += nw) {
            float s = 0.f, c = 0.f;
#pragma unroll
            for (int cc = 0; cc < kCgMaxQ / 32; ++cc) {
                const int j = lane + 32 * cc;
                if (j < qp) {
                    const float2 a = S.M[i * qp + j], b2 = pl[cc];
                    float p0, e0, sn, t0;
                    two_prod(a.x, b2.x, p0, e0);
                    e0 = fmaf(a.x, b2.y, fmaf(a.y, b2.x, e0));
                    two_sum(s, p0, sn, t0);
                    s = sn;
                    c += t0 + e0;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float s2 = __shfl_xor_sync(0xffffffffu, s, o), c2 = __shfl_xor_sync(0xffffffffu, c, o);
                float sn, e;
                two_sum(s, s2, sn, e);
                s = sn;
                c += e + c2;
            }
            if (lane == 0) { float hi, lo; two_sum(s, c, hi, lo); S.AP[i] = make_float2(hi, lo); }
        }
        __syncthreads();
        const float2 pap = cg_dot(S.P, S.AP, qp, red);
        if (!(pap.x > 0.f)) break;
        const float2 al = dfx_div(rz, pap);
        if (tid < qp) {
            S.X[tid] = dfx_add(S.X[tid], dfx_mul(al, S.P[tid]));
            S.RO[tid] = S.R[tid];
            const float2 rn = dfx_sub(S.R[tid], dfx_mul(al, S.AP[tid]));
            S.R[tid] = rn;
            S.t[tid] = rn.x + rn.y;
        }
        __syncthreads();
        ++it;
        rr = cg_dot(S.R, S.R, qp, red);
        go = rr.x > tol2;
        if (!go) break;
        cg_precond(S, qp);
        if (tid < qp) S.Z[tid] = make_float2(S.t[tid], 0.f);
        __syncthreads();
        const float2 rzn = cg_dot(S.R, S.Z, qp, red);
        const float2 rzo = cg_dot(S.RO, S.Z, qp, red);
        float2 beta = dfx_div(dfx_sub(rzn, rzo), rz);
        if (!(beta.x > 0.f)) beta = make_float2(0.f, 0.f);
        rz = rzn;
        if (tid < qp) S.P[tid] = dfx_add(S.Z[tid], dfx_mul(beta, S.P[tid]));
        __syncthreads();
    }
    if (tid < q) dv[tid] = (double)S.X[tid].x + (double)S.X[tid].y;
    if (tid == 0 && info) {
        info[0] = it;
        info[1] = sqrt((double)fmaxf(rr.x, 0.f));
        info[2] = sc_shift;
    }
    if (vdot) {
        // Algorithm 3, Step 2 quantities: rdots[2] = g'dv, rdots[3] = v'dv, rdots[4] = dv'dv
        __syncthreads();
        if (tid < qp) {
            float2 gv = make_float2(0.f, 0.f), vv = gv;
            if (tid < q) {
                const double a = g[tid], b = vdot[tid];
                const float ah = (float)a, bh = (float)b;
                gv = make_float2(ah, (float)(a - (double)ah));
                vv = make_float2(bh, (float)(b - (double)bh));
            }
            S.R[tid] = gv;
            S.P[tid] = vv;
        }
        __syncthreads();
        const float2 d0 = cg_dot(S.R, S.X, qp, red);
        const float2 d1 = cg_dot(S.P, S.X, qp, red);
        const float2 d2 = cg_dot(S.X, S.X, qp, red);
        if (tid == 0) {
            rdots[2] = (double)d0.x + (double)d0.y;
            rdots[3] = (double)d1.x + (double)d1.y;
            rdots[4] = (double)d2.x + (double)d2.y;
        }
    }
}

__global__ void __launch_bounds__(kCgThreads) newton_cg_fast_kernel(int q, const float2 *__restrict__ Mf,
                                                                    const double *__restrict__ g,
                                                                    double *__restrict__ dv, float eta, float tau,
                                                                    float floor, int maxit, double *__restrict__ info,
                                                                    int *err, const double *__restrict__ vdot,
                                                                    double *__restrict__ rdots)
{
    newton_cg_fast_body(q, Mf, g, dv, eta, tau, floor, maxit, info, err, vdot, rdots);
}

// One block per problem of a batch (blockIdx.x).
__global__ void __launch_bounds__(kCgThreads) newton_cg_fast_batch_kernel(int q, const NewtonTask *__restrict__ T)
{
    const NewtonTask &t = T[blockIdx.x];
    newton_cg_fast_body(q, t.Mf, t.g, t.dv, t.eta, t.tau, t.floor, t.maxit, t.info, t.err, t.vdot, t.rdots);
}

// ---------------------------------------------------------------------------
// Newton solve for 128 < q <= 1024 (Algorithm 3, Step 1, on the reduced system
// of Proposition 3.5): conjugate gradients on M dv = -g with the operator in
// double-float from the (hi, lo) split of M, preconditioned by the FP32
// Cholesky factor of fl32(M) -- as the q <= 128 kernel, but factored by many
// blocks at once.  One cooperative launch of G blocks:
//  * factor, right-looking by 128-wide panels, three grid barriers a panel:
//    block 0 factors the diagonal block in shared memory (the 8-wide panel
//    code of the q <= 128 kernel; the inverses of its 8 x 8 diagonal blocks go
//    to global memory for the triangular solves), every block then solves a
//    share of the panel's rows (x L_kk' = a, a warp per row), and every block
//    updates a share of the 64 x 64 tiles of the trailing lower triangle.  A
//    pivot that is not positive restarts the factor with a diagonal shift
//    (1e-7 max diag, then x100, at most six attempts; err = DEV_CHOL after).
//  * CG: every block holds the q-vectors in shared memory and updates them
//    identically (same dot products in the same order); the rows of M p are
//    shared out and exchanged through global memory (one grid barrier), and
//    block 0 applies (L L')^{-1} by 8-wide blocked triangular solves against
//    the factor in global memory (one grid barrier to publish z).
// Stop rule as the q <= 128 kernel (Algorithm 3's bound, tightened to 1e-10
// |g|), at most maxit steps.  Every block takes the same barriers; on a
// barrier that timed out (err = DEV_TIMEOUT) every block leaves.

// t <- (L L')^{-1} t with the row-major factor Lg (row stride q) and the
// inverses Dg of its 8 x 8 diagonal blocks; t in shared memory, zero beyond
// q up to a multiple of 8.  One block.
__device__ void bc_chol_solve(const float *__restrict__ Lg, const float *__restrict__ Dg, int q, float *t)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nb8 = (q + kPb - 1) / kPb;
    for (int b = 0; b < nb8; ++b) {   // forward: L y = t
        const int kb = b * kPb;
        if (warp == 0) {
            const float tv = lane < kPb ? t[kb + lane] : 0.f;
            const float *Db = Dg + (size_t)b * kPb * kPb;
            float acc = 0.f;
#pragma unroll
            for (int k = 0; k < kPb; ++k)
                acc = fmaf(lane < kPb ? __ldcg(&Db[lane * kPb + k]) : 0.f, __shfl_sync(0xffffffffu, tv, k), acc);
            if (lane < kPb) t[kb + lane] = acc;
        }
        __syncthreads();
        for (int r = kb + kPb + tid; r < q; r += blockDim.x) {
            const float *lr = Lg + (size_t)r * q + kb;
            float s = t[r];
#pragma unroll
            for (int k = 0; k < kPb; ++k)
                if (kb + k < q) s = fmaf(-__ldcg(&lr[k]), t[kb + k], s);
            t[r] = s;
        }
        __syncthreads();
    }
    for (int b = nb8 - 1; b >= 0; --b) {   // backward: L' x = y
        const int kb = b * kPb;
        if (warp == 0) {
            const float tv = lane < kPb ? t[kb + lane] : 0.f;
            const float *Db = Dg + (size_t)b * kPb * kPb;
            float acc = 0.f;
#pragma unroll
            for (int k = 0; k < kPb; ++k)
                acc = fmaf(lane < kPb ? __ldcg(&Db[k * kPb + lane]) : 0.f, __shfl_sync(0xffffffffu, tv, k), acc);
            if (lane < kPb) t[kb + lane] = acc;
        }
        __syncthreads();
        for (int r = tid; r < kb; r += blockDim.x) {
            float s = t[r];
#pragma unroll
            for (int k = 0; k < kPb; ++k)
                if (kb + k < q) s = fmaf(-__ldcg(&Lg[(size_t)(kb + k) * q + r]), t[kb + k], s);
            t[r] = s;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kCgThreads, 1) newton_bchol_kernel(int q, const float2 *__restrict__ Mf,
                                                                  const double *__restrict__ g, double *__restrict__ dv,
                                                                  float eta, float tau, float floor, int maxit,
                                                                  double *__restrict__ info, int *err,
                                                                  const double *__restrict__ vdot,
                                                                  double *__restrict__ rdots, float *__restrict__ Lg,
                                                                  float *__restrict__ Dg, float2 *__restrict__ xch,
                                                                  int *fflag, unsigned *bar)
{
    extern __shared__ float4 cg_sm4[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int b = blockIdx.x, G = gridDim.x;
    const int gw = b * nw + warp, ngw = G * nw;
    CgSmem S;   // a 128 x 128 panel's factor; the region of M holds tiles and vectors
    S.M = reinterpret_cast<float2 *>(cg_sm4);
    S.L = reinterpret_cast<float *>(S.M + kBcNb * kBcNb);
    S.D = S.L + ((kBcNb * (kBcNb + 1)) >> 1);
    S.t = S.D + (kBcNb / kPb) * kPb * kPb;
    __shared__ float2 red[kCgThreads / 32];
    float2 *apg = xch, *zg = xch + kBcMaxQ;
    float shift = 0.f;
    const int fr = bc_factor(q, Mf, Lg, Dg, fflag, bar, err, S, red, &shift, (int)blockIdx.x, (int)gridDim.x);
    if (fr <= 0) {
        if (fr == 0 && b == 0 && tid == 0) set_err(err, DEV_CHOL);
        return;
    }
    // CG: replicated vectors where the tiles were
    float2 *X = S.M, *R = X + kBcMaxQ, *P = R + kBcMaxQ, *RO = P + kBcMaxQ, *Z = RO + kBcMaxQ, *AP = Z + kBcMaxQ;
    float *tz = reinterpret_cast<float *>(AP + kBcMaxQ);
    const int q8 = (q + kPb - 1) / kPb * kPb;
    for (int j = tid; j < q; j += blockDim.x) {
        const double v = -g[j];
        const float hi = (float)v;
        R[j] = make_float2(hi, (float)(v - (double)hi));
        X[j] = make_float2(0.f, 0.f);
    }
    __syncthreads();
    float2 rr = bc_dot(R, R, q, red);
    const float gn = sqrtf(fmaxf(rr.x, 0.f));
    const float tol = cg_tol(gn, eta, tau, floor);
    const float tol2 = tol * tol;
    auto precond = [&]() -> bool {
        if (b == 0) {
            for (int j = tid; j < q8; j += blockDim.x) tz[j] = j < q ? R[j].x + R[j].y : 0.f;
            __syncthreads();
            bc_chol_solve(Lg, Dg, q, tz);
            for (int j = tid; j < q; j += blockDim.x) zg[j] = make_float2(tz[j], 0.f);
        }
        if (!grid_barrier(bar, err)) return false;
        for (int j = tid; j < q; j += blockDim.x) Z[j] = __ldcg(&zg[j]);
        __syncthreads();
        return true;
    };
    if (!precond()) return;
    for (int j = tid; j < q; j += blockDim.x) P[j] = Z[j];
    __syncthreads();
    float2 rz = bc_dot(R, Z, q, red);
    int it = 0;
    bool go = rr.x > tol2;
    while (go && it < maxit) {
        // AP = M P: a warp per row, Dot2-style sums of double-float products
        for (int i = gw; i < q; i += ngw) {
            const float2 *mrow = Mf + (size_t)i * q;
            float sh = 0.f, sc = 0.f;
            for (int j = lane; j < q; j += 32) {
                const float2 a = __ldg(&mrow[j]), b2 = P[j];
                float p0, e0, sn, t0;
                two_prod(a.x, b2.x, p0, e0);
                e0 = fmaf(a.x, b2.y, fmaf(a.y, b2.x, e0));
                two_sum(sh, p0, sn, t0);
                sh = sn;
                sc += t0 + e0;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float s2 = __shfl_xor_sync(0xffffffffu, sh, o), c2 = __shfl_xor_sync(0xffffffffu, sc, o);
                float sn, e;
                two_sum(sh, s2, sn, e);
                sh = sn;
                sc += e + c2;
            }
            if (lane == 0) { float hi, lo; two_sum(sh, sc, hi, lo); apg[i] = make_float2(hi, lo); }
        }
        if (!grid_barrier(bar, err)) return;
        for (int j = tid; j < q; j += blockDim.x) AP[j] = __ldcg(&apg[j]);
        __syncthreads();
        const float2 pap = bc_dot(P, AP, q, red);
        if (!(pap.x > 0.f)) break;
        const float2 al = dfx_div(rz, pap);
        for (int j = tid; j < q; j += blockDim.x) {
            X[j] = dfx_add(X[j], dfx_mul(al, P[j]));
            RO[j] = R[j];
            R[j] = dfx_sub(R[j], dfx_mul(al, AP[j]));
        }
        __syncthreads();
        ++it;
        rr = bc_dot(R, R, q, red);
        go = rr.x > tol2;
        if (!go) break;
        if (!precond()) return;
        const float2 rzn = bc_dot(R, Z, q, red);
        const float2 rzo = bc_dot(RO, Z, q, red);
        float2 beta = dfx_div(dfx_sub(rzn, rzo), rz);
        if (!(beta.x > 0.f)) beta = make_float2(0.f, 0.f);
        rz = rzn;
        for (int j = tid; j < q; j += blockDim.x) P[j] = dfx_add(Z[j], dfx_mul(beta, P[j]));
        __syncthreads();
    }
    if (b != 0) return;
    for (int j = tid; j < q; j += blockDim.x) dv[j] = (double)X[j].x + (double)X[j].y;
    if (tid == 0 && info) {
        info[0] = it;
        info[1] = sqrt((double)fmaxf(rr.x, 0.f));
        info[2] = shift;
    }
    if (vdot) {
        // Algorithm 3, Step 2 quantities: rdots[2] = g'dv, rdots[3] = v'dv, rdots[4] = dv'dv
        for (int j = tid; j < q; j += blockDim.x) {
            const double a = g[j], c = vdot[j];
            const float ah = (float)a, ch = (float)c;
            R[j] = make_float2(ah, (float)(a - (double)ah));
            P[j] = make_float2(ch, (float)(c - (double)ch));
        }
        __syncthreads();
        const float2 d0 = bc_dot(R, X, q, red);
        const float2 d1 = bc_dot(P, X, q, red);
        const float2 d2 = bc_dot(X, X, q, red);
        if (tid == 0) {
            rdots[2] = (double)d0.x + (double)d0.y;
            rdots[3] = (double)d1.x + (double)d1.y;
            rdots[4] = (double)d2.x + (double)d2.y;
        }
    }
}

// ---------------------------------------------------------------------------
// Newton step for a large free set (p > kMfMinP, FP32 X, q <= 128).  The exact
// double-float Gram costs p q^2 / 2 double-float terms on the FP32 pipes
// (2.4 ms at p = 5e5); instead CG runs on the exact operator
//     M d = d + sigma (X_J'(X_J d) - h (h'd) / p),   h = X_J'1,
// applied matrix-free in double-float: one pass over the rows of J per CG
// step, each row read once (its dot with d, then its share of X_J't).  The
// preconditioner is the explicit inverse of the FP32 Cholesky factor of the
// same matrix built from a stride subsample of s rows of J, the Gram scaled by
// p / s (a ~1/sqrt(s) relative approximation, so CG gains ~2 digits a step).
// The last block of each pass does the CG update; passes are launched back to
// back and return at once when the state says the solve is done, so the host
// never waits.  Same stopping rule as newton_cg_fast_kernel.
// Measured on gauss1m (q = 128, TF32 tensor-core preconditioner, CG in 2-3
// passes): p = 1.6e4: 207 us exact Gram vs 379 us matrix-free; p = 1e5: 587 vs
// 535 us; p = 5e5: 2437 vs 1260 us.  The matrix-free solve carries a fixed
// ~300 us (setup kernel, unused pass launches).  It starts above 5e4 rows: on
// the one-vs-rest problems (n = 1e5, q = 128, free sets of 5e4-1e5 rows) eight
// whole solves took 59 ms with that threshold against 94 ms at 1e5 (and 59 ms
// at 2e4 or 5e3: no step falls between), gauss1m unchanged.
constexpr long long kMfMinP = 50000;
// the threshold in use (SVM_MF_MIN_P overrides it, for measurements)
static long long mf_min_p()
{
    static long long v = -1;
    if (v < 0) {
        const char *e = getenv("SVM_MF_MIN_P");
        v = (e && atoll(e) > 0) ? atoll(e) : kMfMinP;
    }
    return v;
}
// The same at 128 < q <= 1024 (k_newton_wide.cu) for every free set: at q = 784
// (opbench newton, n = 2e5) p = 1514: 0.42 ms against 1.50 ms for the exact
// Gram and newton_bchol_kernel (whose CG applies the factor by triangular
// solves in one block, ~0.1 ms a CG step); p = 5e3: 0.50 vs 2.01; p = 2e4:
// 0.52 vs 4.23; p = 1e5: 3.1 vs 16.0.  newton_bchol_kernel remains for q % 16
// != 0.  SVM_MFW_MIN_P sets a lower bound on p for measurements.
constexpr long long kMfwMinP = 0;
static long long mfw_min_p()
{
    static long long v = -1;
    if (v < 0) {
        const char *e = getenv("SVM_MFW_MIN_P");
        v = (e && atoll(e) >= 0) ? atoll(e) : kMfwMinP;
    }
    return v;
}
// launch_newton takes the wide path of k_newton_wide.cu
bool newton_is_wide(const Work &W, long long p)
{
    const int q = (int)W.q;
    return !W.csr && W.precision == 1 && W.xf32 && W.mfw_st && q > kCgMaxQ && q <= kBcMaxQ && q % 16 == 0 &&
           p > mfw_min_p();
}

constexpr int kMfSample = 2048;
constexpr int kMfMaxPass = 6;
constexpr int kMfThreads = 512;

struct MfState {   // CG state carried between passes (global memory)
    float2 X[kCgMaxQ], R[kCgMaxQ], RO[kCgMaxQ], D[kCgMaxQ], H[kCgMaxQ];
    float2 rz;
    float tol2;
    float shift;
    int it;
    int done;
};

// Armijo quantities and the output of a finished solve (threads < q write dv)
__device__ __forceinline__ void mf_finish(const float2 *X, int q, int qp, double *dv, const double *g,
                                          const double *vdot, double *rdots, float2 *tmpa, float2 *tmpb, float2 *red)
{
    const int tid = threadIdx.x;
    if (tid < q) dv[tid] = (double)X[tid].x + (double)X[tid].y;
    if (!vdot) return;
    if (tid < qp) {
        float2 gv = make_float2(0.f, 0.f), vv = gv;
        if (tid < q) {
            const double a = g[tid], b = vdot[tid];
            const float ah = (float)a, bh = (float)b;
            gv = make_float2(ah, (float)(a - (double)ah));
            vv = make_float2(bh, (float)(b - (double)bh));
        }
        tmpa[tid] = gv;
        tmpb[tid] = vv;
    }
    __syncthreads();
    const float2 d0 = cg_dot(tmpa, X, qp, red);
    const float2 d1 = cg_dot(tmpb, X, qp, red);
    const float2 d2 = cg_dot(X, X, qp, red);
    if (tid == 0) {
        rdots[2] = (double)d0.x + (double)d0.y;
        rdots[3] = (double)d1.x + (double)d1.y;
        rdots[4] = (double)d2.x + (double)d2.y;
    }
}

// One block: factor the subsample matrix (in Mf), form Pinv = (L L')^{-1}
// explicitly, and start CG on M dv = -g: X = 0, R = -g, D = Pinv R.
__global__ void __launch_bounds__(kCgThreads) newton_mf_setup_kernel(int q, const float2 *__restrict__ Mf,
                                                                     const double *__restrict__ g,
                                                                     double *__restrict__ dv, float eta, float tau,
                                                                     float floor, MfState *__restrict__ st,
                                                                     float *__restrict__ Pinv, int *err,
                                                                     const double *__restrict__ vdot,
                                                                     double *__restrict__ rdots)
{
    extern __shared__ float4 cg_sm4[];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int qp = (q + 31) & ~31, nb = qp / kPb;
    CgSmem S;
    S.M = reinterpret_cast<float2 *>(cg_sm4);
    S.L = reinterpret_cast<float *>(S.M + qp * qp);
    S.D = S.L + ((qp * (qp + 1)) >> 1);
    S.t = S.D + nb * kPb * kPb;
    S.X = reinterpret_cast<float2 *>(S.t + qp);
    S.R = S.X + qp; S.P = S.R + qp; S.AP = S.P + qp; S.Z = S.AP + qp; S.RO = S.Z + qp;
    __shared__ float2 red[8];
    __shared__ float sc_shift;
    if (!cg_load_factor(S, q, Mf, err, &sc_shift)) {
        if (tid == 0) st->done = 1;
        return;
    }
    // Y = L^{-1} in the (now free) M area, row-major, ld = qp + 1
    float *Y = reinterpret_cast<float *>(S.M);
    const int ld = qp + 1;
    tri_inverse_packed(S, qp, Y, ld);
    // Pinv = Y'Y (symmetric; Y lower triangular)
    for (int e = tid; e < qp * qp; e += nt) {
        const int i = e / qp, j = e - i * qp;
        if (j < i) continue;
        float a = 0.f;
        for (int k = j; k < qp; ++k) a = fmaf(Y[k * ld + i], Y[k * ld + j], a);
        Pinv[i * qp + j] = a;
        Pinv[j * qp + i] = a;
    }
    __syncthreads();
    // CG start
    if (tid < qp) {
        float2 r0 = make_float2(0.f, 0.f);
        if (tid < q) {
            const double v = -g[tid];
            const float hi = (float)v;
            r0 = make_float2(hi, (float)(v - (double)hi));
        }
        S.R[tid] = r0;
        S.X[tid] = make_float2(0.f, 0.f);
        S.t[tid] = r0.x + r0.y;
    }
    __syncthreads();
    // z = Pinv t = Y'(Y t), from Y in shared memory (Y lower triangular)
    float *yt = reinterpret_cast<float *>(S.AP);
    if (tid < qp) {
        float a = 0.f;
        for (int k = 0; k <= tid; ++k) a = fmaf(Y[tid * ld + k], S.t[k], a);
        yt[tid] = a;
    }
    __syncthreads();
    if (tid < qp) {
        float z = 0.f;
        for (int k = tid; k < qp; ++k) z = fmaf(Y[k * ld + tid], yt[k], z);
        S.Z[tid] = make_float2(z, 0.f);
    }
    __syncthreads();
    const float2 rr = cg_dot(S.R, S.R, qp, red);
    const float2 rz = cg_dot(S.R, S.Z, qp, red);
    const float gn = sqrtf(fmaxf(rr.x, 0.f));
    const float tol = cg_tol(gn, eta, tau, floor);
    const bool done = !(rr.x > tol * tol);
    if (tid < qp) {
        st->X[tid] = S.X[tid];
        st->R[tid] = S.R[tid];
        st->D[tid] = S.Z[tid];
    }
    if (tid == 0) {
        st->rz = rz;
        st->tol2 = tol * tol;
        st->shift = sc_shift;
        st->it = 0;
        st->done = done ? 1 : 0;
    }
    if (done) mf_finish(S.X, q, qp, dv, g, vdot, rdots, S.AP, S.P, red);
}

// One CG step: y = X_J'(X_J D) over this block's rows of J (and, on the first
// pass, h = X_J'1), double-float block partials, and in the last block to
// finish the CG update.  VW = 4 columns per lane (q % 4 == 0, q <= 128).
template <bool FIRST>
__global__ void __launch_bounds__(kMfThreads) newton_mf_pass_kernel(
    const float *__restrict__ X, const int32_t *__restrict__ J, long long p, int q, float2 sig, float2 rp,
    MfState *__restrict__ st, const float *__restrict__ Pinv, float2 *__restrict__ part, unsigned *__restrict__ counter,
    int last, int maxit, double *__restrict__ dv, const double *__restrict__ g, const double *__restrict__ vdot,
    double *__restrict__ rdots, double *__restrict__ info)
{
    __shared__ int sh_flag;
    if (threadIdx.x == 0) sh_flag = __ldcg(&st->done);
    __syncthreads();
    if (sh_flag) return;
    const int G = gridDim.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int qp = (q + 31) & ~31;
    const bool has = 4 * lane < q;
    float2 dl[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) dl[k] = has ? __ldcg(&st->D[4 * lane + k]) : make_float2(0.f, 0.f);
    float as[4] = {0.f, 0.f, 0.f, 0.f}, ac[4] = {0.f, 0.f, 0.f, 0.f};
    float hs[4] = {0.f, 0.f, 0.f, 0.f}, hc[4] = {0.f, 0.f, 0.f, 0.f};
    const long long per = (p + G - 1) / G;
    const long long r_beg = (long long)blockIdx.x * per;
    const long long r_end = r_beg + per < p ? r_beg + per : p;
    constexpr int R = 4;
    for (long long c0 = r_beg + (long long)warp * 32; c0 < r_end; c0 += (long long)nw * 32) {
        const long long rl = c0 + lane;
        const int myi = (rl < r_end) ? J[rl] : -1;
        const int here = (int)((r_end - c0) < 32 ? (r_end - c0) : 32);
        for (int u0 = 0; u0 < here; u0 += R) {
            float4 xv[R];
#pragma unroll
            for (int u = 0; u < R; ++u) {
                const int ii = __shfl_sync(0xffffffffu, myi, (u0 + u) & 31);
                xv[u] = (u0 + u < here && has) ? __ldcs(reinterpret_cast<const float4 *>(X + (long long)ii * q) + lane)
                                               : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < R; ++u) {
                // t = x . d (Dot2, then an all-lane butterfly on (s, c))
                float s = 0.f, c = 0.f;
                dot2_step(xv[u].x, dl[0], s, c);
                dot2_step(xv[u].y, dl[1], s, c);
                dot2_step(xv[u].z, dl[2], s, c);
                dot2_step(xv[u].w, dl[3], s, c);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const float s2 = __shfl_xor_sync(0xffffffffu, s, o), c2 = __shfl_xor_sync(0xffffffffu, c, o);
                    float sn, e;
                    two_sum(s, s2, sn, e);
                    s = sn;
                    c += c2 + e;
                }
                float th, tl;
                two_sum(s, c, th, tl);
                const float2 t = make_float2(th, tl);
                dot2_step(xv[u].x, t, as[0], ac[0]);
                dot2_step(xv[u].y, t, as[1], ac[1]);
                dot2_step(xv[u].z, t, as[2], ac[2]);
                dot2_step(xv[u].w, t, as[3], ac[3]);
                if (FIRST) {
                    const float xs[4] = {xv[u].x, xv[u].y, xv[u].z, xv[u].w};
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        float sn, e;
                        two_sum(hs[k], xs[k], sn, e);
                        hs[k] = sn;
                        hc[k] += e;
                    }
                }
            }
        }
    }
    // warps in order -> block partial (double-float) -> part[list][blk][j].
    // One shared pool: the per-warp sums first, the last block's vectors after.
    __shared__ float2 pool[2 * (kMfThreads / 32) * kCgMaxQ];
    float2 *wy = pool, *wh = pool + (kMfThreads / 32) * kCgMaxQ;
    if (has) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            wy[warp * kCgMaxQ + 4 * lane + k] = make_float2(as[k], ac[k]);
            if (FIRST) wh[warp * kCgMaxQ + 4 * lane + k] = make_float2(hs[k], hc[k]);
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < q; j += blockDim.x) {
        float s = 0.f, c = 0.f, s2 = 0.f, c2 = 0.f;
        for (int w = 0; w < nw; ++w) {
            df_acc(s, c, wy[w * kCgMaxQ + j].x, wy[w * kCgMaxQ + j].y);
            if (FIRST) df_acc(s2, c2, wh[w * kCgMaxQ + j].x, wh[w * kCgMaxQ + j].y);
        }
        float hi, lo;
        two_sum(s, c, hi, lo);
        part[(size_t)blockIdx.x * q + j] = make_float2(hi, lo);
        if (FIRST) {
            two_sum(s2, c2, hi, lo);
            part[((size_t)G + blockIdx.x) * q + j] = make_float2(hi, lo);
        }
    }
    __threadfence();
    __syncthreads();
    __shared__ int is_last;
    if (threadIdx.x == 0) is_last = (atomicAdd(counter, 1u) == (unsigned)(G - 1));
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    // ---- last block: y (and h) in block order, then the CG update ----
    __syncthreads();   // the pool's per-warp sums are no longer read
    float2 *sy = pool, *sh = sy + kCgMaxQ, *sd = sh + kCgMaxQ, *sap = sd + kCgMaxQ, *sz = sap + kCgMaxQ,
           *sro = sz + kCgMaxQ, *sx = sro + kCgMaxQ, *sr = sx + kCgMaxQ;
    float2 *sub = sr + kCgMaxQ;                                  // [subs][kCgMaxQ]
    float2 *subh = sub + (kMfThreads / kCgMaxQ) * kCgMaxQ;       // [subs][kCgMaxQ]
    __shared__ float2 red[8];
    __shared__ float sw[kCgMaxQ];
    const int subs = blockDim.x / kCgMaxQ;   // 4 interleaved sub-sums per column
    {
        const int col = threadIdx.x % kCgMaxQ, sb = threadIdx.x / kCgMaxQ;
        float2 a = make_float2(0.f, 0.f), hh = a;
        if (col < q) {
            // eight loads in flight per step, added in block order
            int b = sb;
            for (; b + 7 * subs < G; b += 8 * subs) {
                float2 v[8], w[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    v[u] = __ldcg(&part[(size_t)(b + u * subs) * q + col]);
                    if (FIRST) w[u] = __ldcg(&part[((size_t)G + b + u * subs) * q + col]);
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    a = dfx_add(a, v[u]);
                    if (FIRST) hh = dfx_add(hh, w[u]);
                }
            }
            for (; b < G; b += subs) {
                a = dfx_add(a, __ldcg(&part[(size_t)b * q + col]));
                if (FIRST) hh = dfx_add(hh, __ldcg(&part[((size_t)G + b) * q + col]));
            }
        }
        sub[sb * kCgMaxQ + col] = a;
        subh[sb * kCgMaxQ + col] = hh;
        __syncthreads();
        if (sb == 0 && col < qp) {
            float2 t = make_float2(0.f, 0.f), th = t;
            if (col < q)
                for (int k = 0; k < subs; ++k) {
                    t = dfx_add(t, sub[k * kCgMaxQ + col]);
                    th = dfx_add(th, subh[k * kCgMaxQ + col]);
                }
            sy[col] = t;
            if (FIRST) { sh[col] = th; st->H[col] = th; }
            else sh[col] = (col < q) ? st->H[col] : make_float2(0.f, 0.f);
            sd[col] = (col < q) ? st->D[col] : make_float2(0.f, 0.f);
            sx[col] = (col < q) ? st->X[col] : make_float2(0.f, 0.f);
            sr[col] = (col < q) ? st->R[col] : make_float2(0.f, 0.f);
        }
        __syncthreads();
    }
    const int tid = threadIdx.x;
    const float2 hd = cg_dot(sh, sd, qp, red);
    if (tid < qp) {   // Ap = d + sigma (y - h (h'd) / p)
        const float2 corr = dfx_mul(sh[tid], dfx_mul(hd, rp));
        sap[tid] = dfx_add(sd[tid], dfx_mul(sig, dfx_sub(sy[tid], corr)));
    }
    __syncthreads();
    const float2 pap = cg_dot(sd, sap, qp, red);
    const float2 rz = st->rz;
    int it = st->it;
    bool done;
    float2 rr = make_float2(0.f, 0.f);
    if (!(pap.x > 0.f)) {
        done = true;   // breakdown: keep the current iterate
        rr = cg_dot(sr, sr, qp, red);
    } else {
        const float2 al = dfx_div(rz, pap);
        if (tid < qp) {
            sx[tid] = dfx_add(sx[tid], dfx_mul(al, sd[tid]));
            sro[tid] = sr[tid];
            sr[tid] = dfx_sub(sr[tid], dfx_mul(al, sap[tid]));
            sw[tid] = sr[tid].x + sr[tid].y;
        }
        __syncthreads();
        ++it;
        rr = cg_dot(sr, sr, qp, red);
        done = !(rr.x > st->tol2) || it >= maxit;
    }
    if (!done) {
        {   // z = Pinv r: all threads, a quarter of the k range each, loads batched
            float *zq = reinterpret_cast<float *>(sub);   // [subs][kCgMaxQ]
            const int col = tid % kCgMaxQ, qt = tid / kCgMaxQ;
            const int k0 = qt * (qp / subs), k1 = k0 + qp / subs;
            float z = 0.f;
            if (col < qp) {
#pragma unroll 8
                for (int k = k0; k < k1; ++k) z = fmaf(__ldcg(&Pinv[k * qp + col]), sw[k], z);
            }
            zq[qt * kCgMaxQ + col] = z;
            __syncthreads();
            if (tid < qp) {
                float t = 0.f;
                for (int k = 0; k < subs; ++k) t += zq[k * kCgMaxQ + tid];
                sz[tid] = make_float2(t, 0.f);
            }
        }
        __syncthreads();
        const float2 rzn = cg_dot(sr, sz, qp, red);
        const float2 rzo = cg_dot(sro, sz, qp, red);
        float2 beta = dfx_div(dfx_sub(rzn, rzo), rz);
        if (!(beta.x > 0.f)) beta = make_float2(0.f, 0.f);
        if (tid < q) st->D[tid] = dfx_add(sz[tid], dfx_mul(beta, sd[tid]));
        if (tid == 0) st->rz = rzn;
    }
    if (tid < q) { st->X[tid] = sx[tid]; st->R[tid] = sr[tid]; }
    if (tid == 0) {
        st->it = it;
        st->done = done ? 1 : 0;
        *counter = 0u;
    }
    if (done || last) {
        mf_finish(sx, q, qp, dv, g, vdot, rdots, sap, sz, red);
        if (tid == 0 && info) {
            info[0] = it;
            info[1] = sqrt((double)fmaxf(rr.x, 0.f));
            info[2] = st->shift;
        }
    }
}

// M_pre = I + sigma (G - h h' / p) from the TF32 Gram partials (FP32 sums in
// block order) and the exact column sums h; written as (value, 0) pairs for
// the factor (and h itself, double-float, to H when H != nullptr).
// Eight lanes per entry sum interleaved eighths of the partials, combined by
// shuffles in a fixed order.
__global__ void build_m_tc_kernel(int q, int G, const float *__restrict__ cpart, int Gh,
                                  const float2 *__restrict__ hpart, float2 rp, float2 sig, float2 *__restrict__ Mf,
                                  float2 *__restrict__ H, const int *skip)
{
    if (skip && __ldcg(skip)) return;
    const int lane = threadIdx.x & 31, sub = lane & 7;
    const int wg = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwg = (gridDim.x * blockDim.x) >> 5;
    // the trip count is uniform per warp (four entries per warp and step), so
    // every lane takes part in the shuffles below
    for (int base = wg * 4; base < q * q; base += nwg * 4) {
        const int t = base + (lane >> 3);
        const bool valid = t < q * q;
        const int a = valid ? t / q : 0, b = valid ? t - a * q : 1;
        float gs = 0.f;
        float2 ha = make_float2(0.f, 0.f), hb = ha;
        if (valid && b <= a) {
#pragma unroll 4
            for (int k = sub; k < G; k += 8) gs += __ldcg(&cpart[(size_t)k * q * q + t]);
#pragma unroll 4
            for (int k = sub; k < Gh; k += 8) {
                ha = dfx_add(ha, __ldcg(&hpart[(size_t)k * q + a]));
                hb = dfx_add(hb, __ldcg(&hpart[(size_t)k * q + b]));
            }
        }
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            gs += __shfl_xor_sync(0xffffffffu, gs, o);
            ha = dfx_add(ha, shfl_xor_f2(ha, o));
            hb = dfx_add(hb, shfl_xor_f2(hb, o));
        }
        if (sub == 0 && valid && b <= a) {
            float2 m = dfx_mul(sig, dfx_sub(make_float2(gs, 0.f), dfx_mul(dfx_mul(ha, hb), rp)));
            if (a == b) m = dfx_addf(m, 1.f);
            Mf[(size_t)a * q + b] = m;
            Mf[(size_t)b * q + a] = m;
            if (a == b && H) H[a] = ha;
        }
    }
}


static int g_cgs_attr = 0;

static int g_chol_smem_set = 0;

static int g_mf_attr = 0;

cudaError_t newton_mf_alloc(Work &W)
{
    if (cudaMalloc((void **)&W.mf_st, sizeof(MfState)) != cudaSuccess) return cudaErrorMemoryAllocation;
    if (cudaMalloc((void **)&W.mf_pinv, sizeof(float) * kCgMaxQ * kCgMaxQ) != cudaSuccess) return cudaErrorMemoryAllocation;
    if (cudaMalloc((void **)&W.mf_counter, sizeof(unsigned)) != cudaSuccess) return cudaErrorMemoryAllocation;
    return cudaMemsetAsync(W.mf_counter, 0, sizeof(unsigned), W.st);
}

static float2 split2(double v)
{
    const float hi = (float)v;
    return make_float2(hi, (float)(v - (double)hi));
}

cudaError_t launch_build_m_tc(Work &W, int G, const float *cpart, int Gh, const float2 *hpart, long long p,
                              double sigma, float2 *H, const int *skip)
{
    build_m_tc_kernel<<<W.nsm * 2, 256, 0, W.st>>>((int)W.q, G, cpart, Gh, hpart, split2(1.0 / (double)p),
                                                   split2(sigma), W.Mf, H, skip);
    ++W.nlaunch;
    return cudaGetLastError();
}

// Large free set: subsample Gram -> preconditioner -> matrix-free CG passes.
static cudaError_t launch_newton_mf(Work &W, const int32_t *J, long long p, double sigma, const double *g, double *dv,
                                    bool dots)
{
    const int q = (int)W.q;
    if (q % 16 == 0) {
        // preconditioner from the TF32 tensor-core Gram of all p rows and the exact h
        // (tcgen05 tensor cores, k_umma.cu)
        const int G = gram_umma_blocks(W);
        if (gram_umma_part_floats(W) > 2 * W.part_len) return cudaErrorInvalidValue;
        float *cpart = reinterpret_cast<float *>(W.part);
        float2 *hpart = reinterpret_cast<float2 *>(cpart + (size_t)G * q * q);
        const cudaError_t eg = launch_gram_umma(W, J, p, cpart, hpart);
        if (eg != cudaSuccess) return eg;
        build_m_tc_kernel<<<W.nsm, 256, 0, W.st>>>(q, G, cpart, G, hpart, split2(1.0 / (double)p), split2(sigma),
                                                   W.Mf, nullptr, nullptr);
    } else {
        // preconditioner from a stride subsample of s rows: M_s = I + sigma (p / s) (G_s - h_s h_s' / s)
        const int s = kMfSample;
        const long long stride = p / s;
        const int nt = (q + kGT - 1) / kGT, ntiles = nt * (nt + 1) / 2;
        const int ks = (s + 31) / 32 < W.nsm ? (s + 31) / 32 : W.nsm;
        double *part = W.part;
        double *hpart = W.part + (size_t)ks * q * q;
        gram_df_kernel<<<dim3(ntiles, ks), 256, 0, W.st>>>((const float *)W.X, q, J, s, ks,
                                                           reinterpret_cast<float2 *>(part),
                                                           reinterpret_cast<float2 *>(hpart), stride);
        build_m_df_kernel<<<W.nsm * 2, 256, 0, W.st>>>(q, ks, reinterpret_cast<const float2 *>(part),
                                                       reinterpret_cast<const float2 *>(hpart), split2(1.0 / s),
                                                       split2(sigma * (double)p / s), W.Mf);
        ++W.nlaunch;
    }
    if (!g_mf_attr) {
        const cudaError_t ea = cudaFuncSetAttribute(newton_mf_setup_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                    (int)cg_fast_smem(kCgMaxQ));
        if (ea != cudaSuccess) return ea;
        g_mf_attr = 1;
    }
    const double *vdot = dots ? W.v : nullptr;
    newton_mf_setup_kernel<<<1, kCgThreads, cg_fast_smem(q), W.st>>>(q, W.Mf, g, dv, (float)W.eta, (float)W.tau,
                                                                     (float)W.cg_floor, W.mf_st, W.mf_pinv, W.err,
                                                                     vdot, W.red);
    const float2 sig = split2(sigma), rp = split2(1.0 / (double)p);
    float2 *pp = reinterpret_cast<float2 *>(W.part);
    const int G = W.nsm;
    for (int k = 0; k < kMfMaxPass; ++k) {
        const int last = k == kMfMaxPass - 1;
        if (k == 0)
            newton_mf_pass_kernel<true><<<G, kMfThreads, 0, W.st>>>((const float *)W.X, J, p, q, sig, rp, W.mf_st,
                                                                    W.mf_pinv, pp, W.mf_counter, last, W.cg_maxit,
                                                                    dv, g, vdot, W.red, W.red + 12);
        else
            newton_mf_pass_kernel<false><<<G, kMfThreads, 0, W.st>>>((const float *)W.X, J, p, q, sig, rp, W.mf_st,
                                                                     W.mf_pinv, pp, W.mf_counter, last, W.cg_maxit,
                                                                     dv, g, vdot, W.red, W.red + 12);
    }
    W.nlaunch += 2 + kMfMaxPass;   // + the Gram, counted by its launcher
    return cudaGetLastError();
}

// Split-K count of the Gram of p gathered rows (~32 rows per block, bounded
// by the partials' workspace; one split per SM for double-float partials).
static long long gram_splits(const Work &W, long long p, bool mixed)
{
    const int q = (int)W.q;
    long long ks = (p + 31) / 32;
    int KSmax = (int)(W.part_len / ((size_t)q * q + q));
    if (KSmax > 4 * W.nsm) KSmax = 4 * W.nsm;
    if (ks > KSmax) ks = KSmax;
    if (mixed && ks > W.nsm) ks = W.nsm;
    if (ks < 1) ks = 1;
    return ks;
}

bool newton_task(const Work &W, const int32_t *J, long long p, double sigma, const double *g, double *dv, bool dots,
                 NewtonTask *t)
{
    const int q = (int)W.q;
    const bool mixed = W.precision == 1 && W.xf32;
    if (W.csr || !mixed || q > kCgMaxQ || p <= 0) return false;
    if (W.mf_st && q % 4 == 0 && p > mf_min_p()) return false;
    const long long ks = gram_splits(W, p, true);
    t->J = J;
    t->p = p;
    t->ks = (int)ks;
    t->maxit = W.cg_maxit;
    t->part = reinterpret_cast<float2 *>(W.part);
    t->hpart = reinterpret_cast<float2 *>(W.part + (size_t)ks * q * q);
    t->Mf = W.Mf;
    t->pinv = split2(1.0 / (double)p);
    t->sig = split2(sigma);
    t->eta = (float)W.eta;
    t->floor = (float)W.cg_floor;
    t->tau = (float)W.tau;
    t->g = g;
    t->dv = dv;
    t->info = W.red + 12;
    t->rdots = W.red;
    t->err = W.err;
    t->vdot = dots ? W.v : nullptr;
    return true;
}

static cudaError_t cg_fast_attr()
{
    if (!g_cgs_attr) {
        cudaError_t ea = cudaFuncSetAttribute(newton_cg_fast_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)cg_fast_smem(kCgMaxQ));
        if (ea == cudaSuccess)
            ea = cudaFuncSetAttribute(newton_cg_fast_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)cg_fast_smem(kCgMaxQ));
        if (ea != cudaSuccess) return ea;
        g_cgs_attr = 1;
    }
    return cudaSuccess;
}

cudaError_t launch_newton_batch(Work &W, const NewtonTask *T_dev, int ntask, int ks_max)
{
    const int q = (int)W.q;
    if (ntask < 1) return cudaSuccess;
    const int nt = (q + kGT - 1) / kGT;
    const int ntiles = nt * (nt + 1) / 2;
    const cudaError_t ea = cg_fast_attr();
    if (ea != cudaSuccess) return ea;
    gram_df_batch_kernel<<<dim3(ntiles, (unsigned)ks_max, (unsigned)ntask), 256, 0, W.st>>>((const float *)W.X, q,
                                                                                             T_dev);
    build_m_df_batch_kernel<<<dim3(W.nsm * 2, 1, (unsigned)ntask), 256, 0, W.st>>>(q, T_dev);
    newton_cg_fast_batch_kernel<<<ntask, kCgThreads, cg_fast_smem(q), W.st>>>(q, T_dev);
    W.nlaunch += 3;
    return cudaGetLastError();
}

static int g_bc_attr = 0;

// 128 < q <= 1024: the blocked-Cholesky CG above, one cooperative launch.  The
// factor lives in W.Lf (q x q row-major); the exchange vectors of M p and z,
// the 8 x 8 diagonal inverses and the restart flag use the Gram partials'
// workspace (consumed by build_m before this launch).
static cudaError_t launch_newton_bchol(Work &W, const double *g, double *dv, double *info, bool dots)
{
    const int q = (int)W.q;
    const size_t dg_floats = (size_t)((q + kPb - 1) / kPb) * kPb * kPb;
    const size_t need = 2 * kBcMaxQ * sizeof(float2) + dg_floats * sizeof(float) + 16;
    if (q > kBcMaxQ || W.part_len * sizeof(double) < need) return cudaErrorInvalidValue;
    const size_t smem = cg_fast_smem(kCgMaxQ);
    if (!g_bc_attr) {
        const cudaError_t ea =
            cudaFuncSetAttribute(newton_bchol_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (ea != cudaSuccess) return ea;
        g_bc_attr = 1;
    }
    int occ = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, newton_bchol_kernel, kCgThreads, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    // enough blocks for one row of M p per warp and one trailing tile per block
    const int nt = (q + kBcTile - 1) / kBcTile;
    int G = nt * (nt + 1) / 2;
    const int rows = (q + (kCgThreads / 32) - 1) / (kCgThreads / 32);
    if (G < rows) G = rows;
    if (G > occ * W.nsm) G = occ * W.nsm;
    int qq = q, maxit = W.cg_maxit;
    const float2 *Mf = W.Mf;
    float eta = (float)W.eta, tau = (float)W.tau;
    int *err = W.err;
    const double *vd = dots ? W.v : nullptr;
    double *rd = W.red;
    float *Lg = W.Lf;
    float2 *xch = reinterpret_cast<float2 *>(W.part);
    float *Dg = reinterpret_cast<float *>(xch + 2 * kBcMaxQ);
    int *fflag = reinterpret_cast<int *>(Dg + dg_floats);
    unsigned *bar = W.bar;
    float floor = (float)W.cg_floor;
    void *args[] = {&qq, &Mf, &g, &dv, &eta, &tau, &floor, &maxit, &info, &err, &vd, &rd, &Lg, &Dg, &xch, &fflag, &bar};
    return cudaLaunchCooperativeKernel((const void *)newton_bchol_kernel, dim3(G), dim3(kCgThreads), args, smem, W.st);
}

cudaError_t launch_newton(Work &W, const int32_t *J, long long p_host, const long long *p_dev, double sigma,
                          const double *g, double *dv, bool dots)
{
    (void)p_dev;
    if (W.csr) return launch_newton_csr(W, J, p_host, sigma, g, dv, dots);
    const int q = (int)W.q;
    if (p_host <= 0) {
        const cudaError_t e = launch_negcopy(W, g, dv);
        return (e == cudaSuccess && dots) ? launch_dots(W) : e;
    }
    {
        // mixed form, small free set: the three kernels of a NewtonTask
        NewtonTask t;
        if (newton_task(W, J, p_host, sigma, g, dv, dots, &t)) {
            const int nt = (q + kGT - 1) / kGT;
            const int ntiles = nt * (nt + 1) / 2;
            const cudaError_t ea = cg_fast_attr();
            if (ea != cudaSuccess) return ea;
            gram_df_kernel<<<dim3(ntiles, (unsigned)t.ks), 256, 0, W.st>>>((const float *)W.X, q, J, p_host, t.ks,
                                                                            t.part, t.hpart, 1);
            build_m_df_kernel<<<W.nsm * 2, 256, 0, W.st>>>(q, t.ks, t.part, t.hpart, t.pinv, t.sig, t.Mf);
            newton_cg_fast_kernel<<<1, kCgThreads, cg_fast_smem(q), W.st>>>(q, t.Mf, t.g, t.dv, t.eta, t.tau, t.floor,
                                                                            t.maxit, t.info, t.err, t.vdot, t.rdots);
            W.nlaunch += 3;
            return cudaGetLastError();
        }
    }
    const int nt = (q + kGT - 1) / kGT;
    const int ntiles = nt * (nt + 1) / 2;
    long long ks = (p_host + 31) / 32;   // split-K: ~32 gathered rows per block
    int KSmax = (int)(W.part_len / ((size_t)q * q + q));
    if (KSmax > 4 * W.nsm) KSmax = 4 * W.nsm;
    if (ks > KSmax) ks = KSmax;
    const bool mixed = W.precision == 1 && W.xf32;
    if (mixed && W.mf_st && q <= kCgMaxQ && q % 4 == 0 && p_host > mf_min_p())
        return launch_newton_mf(W, J, p_host, sigma, g, dv, dots);
    if (mixed && W.mfw_st && q > kCgMaxQ && q <= kBcMaxQ && q % 16 == 0 && p_host > mfw_min_p())
        return launch_newton_mfw(W, J, p_host, sigma, g, dv, dots);   // the same condition as newton_is_wide
    // double-float partials are summed in one chain per element: one split per SM
    if (mixed && ks > W.nsm) ks = W.nsm;
    if (ks < 1) ks = 1;
    double *part = W.part;
    double *hpart = W.part + (size_t)ks * q * q;
    dim3 grid(ntiles, (unsigned)ks);
    if (mixed)
        gram_df_kernel<<<grid, 256, 0, W.st>>>((const float *)W.X, q, J, p_host, (int)ks,
                                               reinterpret_cast<float2 *>(part), reinterpret_cast<float2 *>(hpart), 1);
    else if (W.xf32)
        gram_kernel<float><<<grid, 256, 0, W.st>>>((const float *)W.X, q, J, p_host, (int)ks, part, hpart);
    else
        gram_kernel<double><<<grid, 256, 0, W.st>>>((const double *)W.X, q, J, p_host, (int)ks, part, hpart);
    const bool cg = W.precision == 1;
    if (mixed) {
        const double pi = 1.0 / (double)p_host;
        const float pih = (float)pi, sh = (float)sigma;
        build_m_df_kernel<<<W.nsm * 2, 256, 0, W.st>>>(q, (int)ks, reinterpret_cast<const float2 *>(part),
                                                       reinterpret_cast<const float2 *>(hpart),
                                                       make_float2(pih, (float)(pi - (double)pih)),
                                                       make_float2(sh, (float)(sigma - (double)sh)), W.Mf);
    } else {
        build_m_kernel<<<W.nsm * 2, 256, 0, W.st>>>(q, (int)ks, part, hpart, (double)p_host, sigma, W.M, W.h,
                                                    cg ? W.Mf : nullptr);
    }
    W.nlaunch += 3;   // gram, build_m, and the solve below
    if (cg) {
        // FP32-Cholesky-preconditioned CG on the FP64 matrix (Algorithm 3's inexact solve)
        double *info = W.red + 12;
        if (q <= kCgMaxQ) {
            const size_t smem_new = cg_fast_smem(q);
            if (!g_cgs_attr) {
                const cudaError_t ea = cudaFuncSetAttribute(newton_cg_fast_kernel,
                                                            cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                            (int)cg_fast_smem(kCgMaxQ));
                if (ea != cudaSuccess) return ea;
                g_cgs_attr = 1;
            }
            newton_cg_fast_kernel<<<1, kCgThreads, smem_new, W.st>>>(q, W.Mf, g, dv, (float)W.eta, (float)W.tau,
                                                                    (float)W.cg_floor, W.cg_maxit, info, W.err,
                                                                    dots ? W.v : nullptr, W.red);
            return cudaGetLastError();
        }
        return launch_newton_bchol(W, g, dv, info, dots);
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
    const cudaError_t e = cudaGetLastError();
    return (e == cudaSuccess && dots) ? launch_dots(W) : e;
}

// The FP64 Cholesky solve above for another caller (the unified-QP solver).
cudaError_t launch_chol_solve(int q, double *M, const double *g, double *dv, int *err, cudaStream_t st)
{
    if (q <= 144) {
        if (!g_chol_smem_set) {
            const cudaError_t ea =
                cudaFuncSetAttribute(chol_solve_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
            if (ea != cudaSuccess) return ea;
            g_chol_smem_set = 1;
        }
        chol_solve_kernel<true><<<1, 1024, ((size_t)q * q + q) * sizeof(double), st>>>(q, M, g, dv, err);
    } else {
        chol_solve_kernel<false><<<1, 1024, 0, st>>>(q, M, g, dv, err);
    }
    return cudaGetLastError();
}

}  // namespace svm
