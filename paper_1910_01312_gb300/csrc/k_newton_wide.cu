// k_newton_wide.cu -- the reduced Newton system of Proposition 3.5,
//     (I_q + sigma (G - h h'/p)) dv = -g,   G = X_J'X_J,  h = X_J'1,  p = |J|,
// for a large free set at 128 < q <= 1024 (mixed form: FP32 X, q % 16 == 0).
//
// The exact double-float Gram costs p q^2 / 2 double-float terms on the FP32
// pipes (16 ms at p = 1e5, q = 784).  Instead, as for q <= 128 (k_newton.cu),
// CG runs on the exact operator applied matrix-free,
//     M d = d + sigma (X_J'(X_J d) - h (h'd) / p),
// one pass over the rows of J per CG step in double-float (Dot2), and the
// preconditioner comes from the Gram on the tensor cores:
//  1. colsum_kernel (k_umma.cu): the exact column sums h (double-float), then
//     gram_f16_wide_kernel (k_umma.cu): G_16 from FP16 products of X16 (X
//     scaled per feature by a power of two; TF32's precision), FP32 sums;
//  2. build_m_tc_kernel (k_newton.cu): M_pre = I + sigma (G_16 - h h'/p);
//  3. newton_mfw_setup_kernel (cooperative): the FP32 Cholesky factor L of
//     M_pre by the grid (bc_factor), the inverses of its 128 x 128 diagonal
//     tiles, then Pinv = (L L')^{-1} column by column -- two block triangular
//     solves per column, eight columns per block at once, the column stored
//     as a row (Pinv is symmetric up to rounding);
//  4. newton_mfw_cg_kernel (cooperative): the whole CG of Algorithm 3, Step 1.
//     Every block holds the q-vectors in shared memory and updates them
//     identically (the same dot products in the same order).  A step is one
//     pass (each block a contiguous share of J, a warp per row: t = x.d by
//     Dot2 and a butterfly, then its share of X_J't), the block partials
//     summed by column slices in block order, and z = Pinv r by rows across
//     the grid: three grid barriers.
// Stop rule as the other Newton solvers (Algorithm 3's bound, tightened to
// 1e-10 |g|), at most maxit steps; beta in the flexible (Polak-Ribiere) form.
// Every wait is bounded (grid_barrier records DEV_TIMEOUT and every block
// leaves).
//
// Reuse: consecutive Newton steps of a subproblem often share almost all of
// J, and only the preconditioner depends on it.  A first kernel counts the
// rows of J missing from the set the current preconditioner was built for (a
// bitmap) and those that left it; when together they are at most 1 % of p,
// sigma is unchanged and the last CG took at most 8 steps, the Gram and
// steps 2-3 are skipped (their kernels return at once); h is summed afresh.
// CG still runs on the exact operator of the current J, so only its step
// count depends on this.
#include <math.h>

#include "internal.cuh"
#include "newton_dev.cuh"

namespace svm {

namespace {

constexpr int kWdBlk = 128;   // diagonal tile of the inverse factor
constexpr int kMfwThreads = 256;   // CG kernel: 8 warps, up to 255 registers (two rows in flight per warp)
constexpr int kWdCols = 8;    // columns of Pinv one block solves together


// The set-up of one problem by G blocks (b = this block's rank): a whole
// cooperative launch, or one group of a launch over several problems.  Every
// step's arithmetic is the same whatever G is (tiles, rows and columns are
// computed by whichever block takes them, in the same order).
__device__ void mfw_setup_body(const MfwSetupArgs &A, const int b, const int G)
{
    const int q = A.q;
    const float2 *__restrict__ Mf = A.Mf;
    float *__restrict__ Lg = A.Lg;
    float *__restrict__ Dg = A.Dg;
    float *__restrict__ Linv = A.Linv;
    float *__restrict__ Pinv = A.Pinv;
    unsigned *bar = A.bar;
    int *err = A.err;
    if (__ldcg(A.skip)) return;   // the same value in every block of the group: no barrier is taken
    extern __shared__ float4 cg_sm4[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    CgSmem S;   // one 128 x 128 tile's packed factor; the region of M holds the work arrays
    S.M = reinterpret_cast<float2 *>(cg_sm4);
    S.L = reinterpret_cast<float *>(S.M + kBcNb * kBcNb);
    S.D = S.L + ((kBcNb * (kBcNb + 1)) >> 1);
    S.t = S.D + (kBcNb / kPb) * kPb * kPb;
    __shared__ float2 red[kCgThreads / 32];
    float shift = 0.f;
    const int fr = bc_factor(q, Mf, Lg, Dg, A.fflag, bar, err, S, red, &shift, b, G);
    if (fr <= 0) {
        if (fr == 0 && b == 0 && tid == 0) set_err(err, DEV_CHOL);
        return;
    }
    if (b == 0 && tid == 0 && A.info) A.info[2] = shift;
    const int nblk = (q + kWdBlk - 1) / kWdBlk;

    // (1) Y_tt = L_tt^{-1} for the diagonal tiles (zero above the diagonal)
    for (int tb = b; tb < nblk; tb += G) {
        const int kb = tb * kWdBlk;
        const int nbk = q - kb < kWdBlk ? q - kb : kWdBlk;
        const int qpk = (nbk + 31) & ~31;
        load_lower(S.L, LayPacked(), Lg + (size_t)kb * q + kb, (size_t)q, nbk, qpk);
        for (int e = tid; e < (qpk / kPb) * kPb * kPb; e += blockDim.x) {
            const int b8 = e / (kPb * kPb), w = e - b8 * kPb * kPb;
            S.D[e] = (b8 * kPb < nbk) ? __ldcg(&Dg[(size_t)kb * kPb + e]) : ((w / kPb == w % kPb) ? 1.f : 0.f);
        }
        __syncthreads();
        float *Y = reinterpret_cast<float *>(S.M);
        const int ld = qpk + 1;
        tri_inverse_packed(S, qpk, Y, ld);
        float *Lt = Linv + (size_t)tb * kWdBlk * kWdBlk;
        for (int e = tid; e < kWdBlk * kWdBlk; e += blockDim.x) {
            const int i = e / kWdBlk, j = e - i * kWdBlk;
            Lt[e] = (i < nbk && j <= i) ? Y[i * ld + j] : 0.f;
        }
        __syncthreads();
    }
    if (!group_barrier(bar, err, b, G)) return;

    // (2) columns c of Pinv: L y = e_c by block rows (T = E_i - L_i,<i Y_<i,
    // Y_i = Y_ii T), then L' z = y backwards (T = Y_i - L_>i,i' Z_>i, Z_i = Y_ii' T)
    const int ldv = nblk * kWdBlk;
    float *V = reinterpret_cast<float *>(S.M);   // [kWdCols][ldv]: y, then z
    float *T = V + kWdCols * ldv;                // [kWdCols][kWdBlk]
    float *P4 = T + kWdCols * kWdBlk;            // [slices][kWdCols][kWdBlk] partial sums
    const int nsl = blockDim.x / kWdBlk;         // column-parallel layout: jj fast, slice sl
    const int jj = tid % kWdBlk, sl = tid / kWdBlk;
    for (long long base = b; base < q; base += (long long)kWdCols * G) {
        int cm[kWdCols];
#pragma unroll
        for (int m = 0; m < kWdCols; ++m) cm[m] = (base + (long long)m * G < q) ? (int)(base + (long long)m * G) : -1;
        for (int e = tid; e < kWdCols * ldv; e += blockDim.x) V[e] = 0.f;
        __syncthreads();
        for (int i = 0; i < nblk; ++i) {
            const int r0 = i * kWdBlk, nbi = q - r0 < kWdBlk ? q - r0 : kWdBlk;
            for (int j = warp; j < nbi; j += nw) {   // a warp per row of the block row
                float acc[kWdCols];
#pragma unroll
                for (int m = 0; m < kWdCols; ++m) acc[m] = 0.f;
                const float *Lr = Lg + (size_t)(r0 + j) * q;
#pragma unroll 4
                for (int k = lane; k < r0; k += 32) {
                    const float l = __ldcg(Lr + k);
#pragma unroll
                    for (int m = 0; m < kWdCols; ++m) acc[m] = fmaf(l, V[m * ldv + k], acc[m]);
                }
#pragma unroll
                for (int m = 0; m < kWdCols; ++m) acc[m] = warp_sumf(acc[m]);
                if (lane == 0) {
#pragma unroll
                    for (int m = 0; m < kWdCols; ++m) T[m * kWdBlk + j] = ((r0 + j) == cm[m] ? 1.f : 0.f) - acc[m];
                }
            }
            __syncthreads();
            const float *Lt = Linv + (size_t)i * kWdBlk * kWdBlk;
            for (int j = warp; j < nbi; j += nw) {
                float acc[kWdCols];
#pragma unroll
                for (int m = 0; m < kWdCols; ++m) acc[m] = 0.f;
                for (int l = lane; l <= j; l += 32) {
                    const float v = __ldcg(Lt + j * kWdBlk + l);
#pragma unroll
                    for (int m = 0; m < kWdCols; ++m) acc[m] = fmaf(v, T[m * kWdBlk + l], acc[m]);
                }
#pragma unroll
                for (int m = 0; m < kWdCols; ++m) acc[m] = warp_sumf(acc[m]);
                if (lane == 0) {
#pragma unroll
                    for (int m = 0; m < kWdCols; ++m) V[m * ldv + r0 + j] = acc[m];
                }
            }
            __syncthreads();
        }
        for (int i = nblk - 1; i >= 0; --i) {
            const int r0 = i * kWdBlk, nbi = q - r0 < kWdBlk ? q - r0 : kWdBlk;
            float acc[kWdCols];
#pragma unroll
            for (int m = 0; m < kWdCols; ++m) acc[m] = 0.f;
            if (jj < nbi) {
#pragma unroll 4
                for (int k = r0 + kWdBlk + sl; k < q; k += nsl) {
                    const float l = __ldcg(&Lg[(size_t)k * q + r0 + jj]);
#pragma unroll
                    for (int m = 0; m < kWdCols; ++m) acc[m] = fmaf(l, V[m * ldv + k], acc[m]);
                }
            }
#pragma unroll
            for (int m = 0; m < kWdCols; ++m) P4[(sl * kWdCols + m) * kWdBlk + jj] = acc[m];
            __syncthreads();
            if (sl == 0 && jj < nbi) {
#pragma unroll
                for (int m = 0; m < kWdCols; ++m) {
                    float s = P4[m * kWdBlk + jj];
                    for (int t = 1; t < nsl; ++t) s += P4[(t * kWdCols + m) * kWdBlk + jj];
                    T[m * kWdBlk + jj] = V[m * ldv + r0 + jj] - s;
                }
            }
            __syncthreads();
            const float *Lt = Linv + (size_t)i * kWdBlk * kWdBlk;
#pragma unroll
            for (int m = 0; m < kWdCols; ++m) acc[m] = 0.f;
            if (jj < nbi) {
                for (int l = jj + sl; l < nbi; l += nsl) {
                    const float v = __ldcg(Lt + l * kWdBlk + jj);
#pragma unroll
                    for (int m = 0; m < kWdCols; ++m) acc[m] = fmaf(v, T[m * kWdBlk + l], acc[m]);
                }
            }
#pragma unroll
            for (int m = 0; m < kWdCols; ++m) P4[(sl * kWdCols + m) * kWdBlk + jj] = acc[m];
            __syncthreads();
            if (sl == 0 && jj < nbi) {
#pragma unroll
                for (int m = 0; m < kWdCols; ++m) {
                    float s = P4[m * kWdBlk + jj];
                    for (int t = 1; t < nsl; ++t) s += P4[(t * kWdCols + m) * kWdBlk + jj];
                    V[m * ldv + r0 + jj] = s;
                }
            }
            __syncthreads();
        }
#pragma unroll
        for (int m = 0; m < kWdCols; ++m) {
            if (cm[m] < 0) continue;
            for (int r = tid; r < q; r += blockDim.x) Pinv[(size_t)cm[m] * q + r] = V[m * ldv + r];
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kCgThreads, 1) newton_mfw_setup_kernel(const __grid_constant__ MfwSetupArgs A)
{
    mfw_setup_body(A, (int)blockIdx.x, (int)gridDim.x);
}

// several problems: groups of Gp consecutive blocks, group g sets up problem g
__global__ void __launch_bounds__(kCgThreads, 1) newton_mfw_setup_group_kernel(const MfwSetupArgs *__restrict__ T,
                                                                            int ntask, int Gp)
{
    const int g = (int)blockIdx.x / Gp;
    if (g >= ntask) return;
    mfw_setup_body(T[g], (int)blockIdx.x - g * Gp, Gp);
}

constexpr double kMfwReuseFrac = 0.01;   // changed rows of J, relative to p, that keep the preconditioner
constexpr int kMfwStaleIt = 8;           // CG steps above which it is rebuilt at the next step

}  // namespace

struct MfwState {
    double sigma;      // sigma the preconditioner was built for
    long long p;       // |J| it was built for (the bitmap holds that J)
    unsigned added;    // this step: rows of J not in the bitmap (summed by the blocks)
    unsigned done;     // finished blocks (last-block reductions)
    int valid;         // a preconditioner exists
    int skip;          // this step reuses it
};

namespace {

// skip = 1 when J differs from the bitmap's set in at most frac p rows, sigma
// is the same and the last CG took at most stale_it steps; else 0 and the
// state records this J's size and sigma (the bitmap is rewritten next).
__global__ void __launch_bounds__(256) mfw_decide_kernel(const int32_t *__restrict__ J, long long p, double sigma,
                                                         const unsigned *__restrict__ mask, MfwState *st,
                                                         const double *info, double frac, int stale_it)
{
    unsigned c = 0;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < p; r += (long long)gridDim.x * blockDim.x) {
        const int i = J[r];
        c += ((mask[i >> 5] >> (i & 31)) & 1u) ? 0u : 1u;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    __shared__ unsigned ws[8];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x != 0) return;
    unsigned t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
    atomicAdd(&st->added, t);
    __threadfence();
    if (atomicAdd(&st->done, 1u) != gridDim.x - 1) return;
    __threadfence();
    const long long added = (long long)atomicAdd(&st->added, 0u);
    const long long removed = st->p - (p - added);
    const bool stale = st->valid == 0 || st->sigma != sigma || !(frac > 0.0) ||
                       (double)(added + removed) > frac * (double)p || !(info[0] <= (double)stale_it);
    st->skip = stale ? 0 : 1;
    if (stale) {
        st->valid = 1;
        st->sigma = sigma;
        st->p = p;
    }
    st->added = 0u;
    st->done = 0u;
}

// the bitmap := J, on a rebuild (two launches: clear, then set)
__global__ void mfw_mask_clear_kernel(unsigned *__restrict__ mask, long long nwords, const MfwState *st)
{
    if (__ldcg(&st->skip)) return;
    for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < nwords; w += (long long)gridDim.x * blockDim.x)
        mask[w] = 0u;
}

__global__ void mfw_mask_set_kernel(const int32_t *__restrict__ J, long long p, unsigned *__restrict__ mask,
                                    const MfwState *st)
{
    if (__ldcg(&st->skip)) return;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < p; r += (long long)gridDim.x * blockDim.x) {
        const int i = J[r];
        atomicOr(&mask[i >> 5], 1u << (i & 31));
    }
}

// h = X_J'1 (double-float) when the Gram is skipped: each block a contiguous
// share of J, a thread per 4 columns, rows in order (TwoSum); the last block
// adds the block partials in block order.
// M_pre = I + sigma (G - h h'/p), lower triangle (the factor reads no more),
// one thread per entry: G_ab summed over the KS row-split partials in split
// order (FP32), the rest in double-float from the exact h
__global__ void __launch_bounds__(256) mfw_build_m_kernel(int q, int KS, const float *__restrict__ cpart,
                                                          const float2 *__restrict__ H, float2 rp, float2 sig,
                                                          float2 *__restrict__ Mf, const int *skip)
{
    if (__ldcg(skip)) return;
    const long long qq = (long long)q * q;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < qq; t += (long long)gridDim.x * blockDim.x) {
        const int a = (int)(t / q), b = (int)(t - (long long)a * q);
        if (b > a) continue;
        float gs = 0.f;
        for (int k = 0; k < KS; ++k) gs += __ldcg(&cpart[(size_t)k * qq + t]);
        const float2 ha = __ldcg(&H[a]), hb = __ldcg(&H[b]);
        float2 m = dfx_mul(sig, dfx_sub(make_float2(gs, 0.f), dfx_mul(dfx_mul(ha, hb), rp)));
        if (a == b) m = dfx_addf(m, 1.f);
        Mf[t] = m;
    }
}

// dynamic shared memory of newton_mfw_cg_kernel<NF4>
constexpr size_t mfw_smem(int nf4)
{
    return (size_t)nf4 * 128 * (4 * sizeof(float2) + 3 * sizeof(float) + (kMfwThreads / 32) * sizeof(float2));
}

// The CG of one problem by G blocks (b = this block's rank).  The rows of J
// are cut into A.vc chunks whatever G is: a block takes chunks b, b + G, ...
// and each chunk's partial, and the sum of the partials in chunk order, are the
// same for any G -- so the result is too.
template <int NF4>
__device__ void mfw_cg_body(const MfwArgs &A, const int b, const int G)
{
    extern __shared__ float4 mw_sm4[];
    constexpr int QW = NF4 * 128;   // padded width: NF4 float4 per lane
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int q = A.q;
    float2 *Xv = reinterpret_cast<float2 *>(mw_sm4);
    float2 *Rv = Xv + QW, *Dv = Rv + QW, *Hv = Dv + QW;
    float *Dh = reinterpret_cast<float *>(Hv + QW), *Dl = Dh + QW, *Rf = Dl + QW;
    float2 *wb = reinterpret_cast<float2 *>(Rf + QW);                  // [nw][QW] per-warp sums of a pass
    float2 *APv = wb, *Yv = wb + QW, *Zv = Yv + QW, *ROv = Zv + QW;    // the same memory between passes
    __shared__ float2 red[kMfwThreads / 32];

    for (int j = tid; j < QW; j += blockDim.x) {
        float2 r = make_float2(0.f, 0.f);
        if (j < q) {
            const double v = -A.g[j];
            const float hi = (float)v;
            r = make_float2(hi, (float)(v - (double)hi));
        }
        Rv[j] = r;
        Rf[j] = r.x + r.y;
        Xv[j] = make_float2(0.f, 0.f);
        Dv[j] = make_float2(0.f, 0.f);
        Hv[j] = j < q ? __ldcg(&A.H[j]) : make_float2(0.f, 0.f);
    }
    __syncthreads();
    float2 rr = bc_dot(Rv, Rv, q, red);
    const float gn = sqrtf(fmaxf(rr.x, 0.f));
    const float tol = cg_tol(gn, A.eta, A.tau, A.floor);
    const float tol2 = tol * tol;

    // z = Pinv r, rows shared out over the grid's warps; Zv = (z, 0)
    auto precond = [&]() -> bool {
        const int gw = b * nw + warp, ngw = G * nw;
        for (int i = gw; i < q; i += ngw) {
            const float4 *pr = reinterpret_cast<const float4 *>(A.Pinv + (size_t)i * q);
            float s = 0.f;
            for (int c = lane; 4 * c < q; c += 32) {
                const float4 pv = __ldcg(pr + c);
                const float4 rv = *reinterpret_cast<const float4 *>(Rf + 4 * c);
                s = fmaf(pv.x, rv.x, s);
                s = fmaf(pv.y, rv.y, s);
                s = fmaf(pv.z, rv.z, s);
                s = fmaf(pv.w, rv.w, s);
            }
            s = warp_sumf(s);
            if (lane == 0) A.zg[i] = s;
        }
        if (!group_barrier(A.bar, A.err, b, G)) return false;
        for (int j = tid; j < QW; j += blockDim.x) Zv[j] = make_float2(j < q ? __ldcg(&A.zg[j]) : 0.f, 0.f);
        __syncthreads();
        return true;
    };
    auto set_d = [&](float2 beta) {
        for (int j = tid; j < QW; j += blockDim.x) {
            const float2 d = dfx_add(Zv[j], dfx_mul(beta, Dv[j]));
            Dv[j] = d;
            Dh[j] = d.x;
            Dl[j] = d.y;
        }
        __syncthreads();
    };

    int it = 0;
    bool go = rr.x > tol2;
    float2 rz = make_float2(0.f, 0.f);
    if (go) {
        if (!precond()) return;
        set_d(make_float2(0.f, 0.f));
        rz = bc_dot(Rv, Zv, q, red);
    }
    const float4 *Dh4 = reinterpret_cast<const float4 *>(Dh), *Dl4 = reinterpret_cast<const float4 *>(Dl);
    while (go && it < A.maxit) {
        // ---- the chunk partials y_c = X_Jc'(X_Jc d) of this block's chunks ----
        for (int ch = b; ch < A.vc; ch += G) {
            float as[4 * NF4], ac[4 * NF4];
#pragma unroll
            for (int k = 0; k < 4 * NF4; ++k) as[k] = ac[k] = 0.f;
            const long long per = (A.p + A.vc - 1) / A.vc;
            const long long rbeg = (long long)ch * per;
            const long long rend = rbeg + per < A.p ? rbeg + per : A.p;
            // the row's dot with d (Dot2, butterfly), then its share of X_J't
            auto row_step = [&](const float4 (&xv)[NF4]) {
                float s = 0.f, cc = 0.f;
#pragma unroll
                for (int f = 0; f < NF4; ++f) {
                    const int c = lane + 32 * f;
                    const float4 dh = Dh4[c], dl = Dl4[c];   // zero beyond q
                    dot2_step(xv[f].x, make_float2(dh.x, dl.x), s, cc);
                    dot2_step(xv[f].y, make_float2(dh.y, dl.y), s, cc);
                    dot2_step(xv[f].z, make_float2(dh.z, dl.z), s, cc);
                    dot2_step(xv[f].w, make_float2(dh.w, dl.w), s, cc);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const float s2 = __shfl_xor_sync(0xffffffffu, s, o), c2 = __shfl_xor_sync(0xffffffffu, cc, o);
                    float sn, e;
                    two_sum(s, s2, sn, e);
                    s = sn;
                    cc += c2 + e;
                }
                float th, tl;
                two_sum(s, cc, th, tl);
                const float2 t = make_float2(th, tl);
#pragma unroll
                for (int f = 0; f < NF4; ++f) {
                    dot2_step(xv[f].x, t, as[4 * f + 0], ac[4 * f + 0]);
                    dot2_step(xv[f].y, t, as[4 * f + 1], ac[4 * f + 1]);
                    dot2_step(xv[f].z, t, as[4 * f + 2], ac[4 * f + 2]);
                    dot2_step(xv[f].w, t, as[4 * f + 3], ac[4 * f + 3]);
                }
            };
            auto load_row = [&](float4 (&xv)[NF4], int ii) {
                const float4 *row = reinterpret_cast<const float4 *>(A.X + (long long)ii * q);
#pragma unroll
                for (int f = 0; f < NF4; ++f) {
                    const int c = lane + 32 * f;
                    xv[f] = (4 * c < q) ? __ldcs(row + c) : make_float4(0.f, 0.f, 0.f, 0.f);
                }
            };
            // two rows in flight: the next row loads while this one is computed
            float4 xa[NF4], xb[NF4];
            for (long long c0 = rbeg + (long long)warp * 32; c0 < rend; c0 += (long long)nw * 32) {
                const int myi = (c0 + lane < rend) ? __ldg(&A.J[c0 + lane]) : 0;
                const int here = (int)(rend - c0 < 32 ? rend - c0 : 32);
                load_row(xa, __shfl_sync(0xffffffffu, myi, 0));
                for (int u = 0; u < here; u += 2) {
                    const int ib = __shfl_sync(0xffffffffu, myi, (u + 1) & 31);
                    const int ia = __shfl_sync(0xffffffffu, myi, (u + 2) & 31);
                    if (u + 1 < here) load_row(xb, ib);
                    row_step(xa);
                    if (u + 2 < here) load_row(xa, ia);
                    if (u + 1 < here) row_step(xb);
                }
            }
            // warps in order -> the block partial (double-float)
#pragma unroll
            for (int f = 0; f < NF4; ++f) {
                const int c = lane + 32 * f;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    float hi, lo;
                    two_sum(as[4 * f + k], ac[4 * f + k], hi, lo);
                    wb[warp * QW + 4 * c + k] = make_float2(hi, lo);
                }
            }
            __syncthreads();
            for (int j = tid; j < q; j += blockDim.x) {
                float s = 0.f, c = 0.f;
                for (int w = 0; w < nw; ++w) df_acc(s, c, wb[w * QW + j].x, wb[w * QW + j].y);
                float hi, lo;
                two_sum(s, c, hi, lo);
                A.part[(size_t)ch * q + j] = make_float2(hi, lo);
            }
            __syncthreads();   // wb is written again by the next chunk
        }
        if (!group_barrier(A.bar, A.err, b, G)) return;
        // ---- y = sum of the chunk partials in chunk order, by column slices ----
        {
            const int cs = (q + G - 1) / G;
            for (int k = warp; k < cs; k += nw) {
                const int j = b * cs + k;
                if (j >= q) break;
                float2 s = make_float2(0.f, 0.f);
                for (int bb = lane; bb < A.vc; bb += 32) s = dfx_add(s, __ldcg(&A.part[(size_t)bb * q + j]));
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) s = dfx_add(s, shfl_xor_f2(s, o));
                if (lane == 0) A.yg[j] = s;
            }
            if (!group_barrier(A.bar, A.err, b, G)) return;
        }
        for (int j = tid; j < QW; j += blockDim.x) Yv[j] = j < q ? __ldcg(&A.yg[j]) : make_float2(0.f, 0.f);
        __syncthreads();
        // ---- the CG step (identical in every block) ----
        const float2 hd = bc_dot(Hv, Dv, q, red);
        const float2 hdp = dfx_mul(hd, A.rp);
        for (int j = tid; j < QW; j += blockDim.x) {   // Ap = d + sigma (y - h (h'd) / p)
            const float2 corr = dfx_mul(Hv[j], hdp);
            APv[j] = j < q ? dfx_add(Dv[j], dfx_mul(A.sig, dfx_sub(Yv[j], corr))) : make_float2(0.f, 0.f);
        }
        __syncthreads();
        const float2 pap = bc_dot(Dv, APv, q, red);
        if (!(pap.x > 0.f)) break;   // breakdown: keep the current iterate
        const float2 al = dfx_div(rz, pap);
        for (int j = tid; j < QW; j += blockDim.x) {
            Xv[j] = dfx_add(Xv[j], dfx_mul(al, Dv[j]));
            ROv[j] = Rv[j];
            const float2 r = dfx_sub(Rv[j], dfx_mul(al, APv[j]));
            Rv[j] = r;
            Rf[j] = r.x + r.y;
        }
        __syncthreads();
        ++it;
        rr = bc_dot(Rv, Rv, q, red);
        go = rr.x > tol2;
        if (!go || it >= A.maxit) break;
        if (!precond()) return;
        const float2 rzn = bc_dot(Rv, Zv, q, red);
        const float2 rzo = bc_dot(ROv, Zv, q, red);
        float2 beta = dfx_div(dfx_sub(rzn, rzo), rz);
        if (!(beta.x > 0.f)) beta = make_float2(0.f, 0.f);
        rz = rzn;
        set_d(beta);
    }
    if (b != 0) return;
    for (int j = tid; j < q; j += blockDim.x) A.dv[j] = (double)Xv[j].x + (double)Xv[j].y;
    if (tid == 0 && A.info) {
        A.info[0] = it;
        A.info[1] = sqrt((double)fmaxf(rr.x, 0.f));
    }
    if (A.vdot) {
        // Algorithm 3, Step 2 quantities: rdots[2] = g'dv, rdots[3] = v'dv, rdots[4] = dv'dv
        for (int j = tid; j < q; j += blockDim.x) {
            const double a = A.g[j], c = A.vdot[j];
            const float ah = (float)a, ch = (float)c;
            APv[j] = make_float2(ah, (float)(a - (double)ah));
            Yv[j] = make_float2(ch, (float)(c - (double)ch));
        }
        __syncthreads();
        const float2 d0 = bc_dot(APv, Xv, q, red);
        const float2 d1 = bc_dot(Yv, Xv, q, red);
        const float2 d2 = bc_dot(Xv, Xv, q, red);
        if (tid == 0) {
            A.rdots[2] = (double)d0.x + (double)d0.y;
            A.rdots[3] = (double)d1.x + (double)d1.y;
            A.rdots[4] = (double)d2.x + (double)d2.y;
        }
    }
}

template <int NF4>
__global__ void __launch_bounds__(kMfwThreads, 1) newton_mfw_cg_kernel(const __grid_constant__ MfwArgs A)
{
    mfw_cg_body<NF4>(A, (int)blockIdx.x, (int)gridDim.x);
}

// several problems (the same q): groups of Gp consecutive blocks
template <int NF4>
__global__ void __launch_bounds__(kMfwThreads, 1) newton_mfw_cg_group_kernel(const MfwArgs *__restrict__ T, int ntask,
                                                                         int Gp)
{
    const int g = (int)blockIdx.x / Gp;
    if (g >= ntask) return;
    mfw_cg_body<NF4>(T[g], (int)blockIdx.x - g * Gp, Gp);
}

template <int NF4>
cudaError_t cg_attr()
{
    static int attr = 0;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(newton_mfw_cg_kernel<NF4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)mfw_smem(NF4));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(newton_mfw_cg_group_kernel<NF4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)mfw_smem(NF4));
        if (e != cudaSuccess) return e;
        attr = 1;
    }
    return cudaSuccess;
}

// one problem (T = nullptr: a) or ntask problems in groups of Gp blocks (T: device table)
template <int NF4>
cudaError_t launch_cg(const MfwArgs &a, const MfwArgs *T, int ntask, int Gp, int G, cudaStream_t st)
{
    const size_t smem = mfw_smem(NF4);
    cudaError_t e = cg_attr<NF4>();
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, newton_mfw_cg_kernel<NF4>, kMfwThreads, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    if (!T) {
        MfwArgs aa = a;
        void *args[] = {&aa};
        return cudaLaunchCooperativeKernel((const void *)newton_mfw_cg_kernel<NF4>, dim3(G), dim3(kMfwThreads), args,
                                           smem, st);
    }
    void *args[] = {(void *)&T, &ntask, &Gp};
    return cudaLaunchCooperativeKernel((const void *)newton_mfw_cg_group_kernel<NF4>, dim3(ntask * Gp),
                                       dim3(kMfwThreads), args, smem, st);
}

cudaError_t launch_cg_nf4(int q, const MfwArgs &a, const MfwArgs *T, int ntask, int Gp, int G, cudaStream_t st)
{
    switch ((q + 127) / 128) {
    case 2: return launch_cg<2>(a, T, ntask, Gp, G, st);
    case 3: return launch_cg<3>(a, T, ntask, Gp, G, st);
    case 4: return launch_cg<4>(a, T, ntask, Gp, G, st);
    case 5: return launch_cg<5>(a, T, ntask, Gp, G, st);
    case 6: return launch_cg<6>(a, T, ntask, Gp, G, st);
    case 7: return launch_cg<7>(a, T, ntask, Gp, G, st);
    default: return launch_cg<8>(a, T, ntask, Gp, G, st);
    }
}

int g_setup_attr = 0;

cudaError_t setup_attr()
{
    if (!g_setup_attr) {
        const int smem = (int)cg_fast_smem(kCgMaxQ);
        cudaError_t e = cudaFuncSetAttribute(newton_mfw_setup_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(newton_mfw_setup_group_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        g_setup_attr = 1;
    }
    return cudaSuccess;
}

// the reuse fraction in use (SVM_MFW_REUSE overrides it, 0 turns reuse off; for measurements)
double mfw_reuse_frac()
{
    static double v = -1.0;
    if (v < 0.0) {
        const char *e = getenv("SVM_MFW_REUSE");
        v = (e && atof(e) >= 0.0) ? atof(e) : kMfwReuseFrac;
        if (v < 0.0) v = 0.0;
    }
    return v;
}

float2 split2w(double v)
{
    const float hi = (float)v;
    return make_float2(hi, (float)(v - (double)hi));
}

}  // namespace

cudaError_t newton_mfw_alloc(Work &W)
{
    const size_t nwords = (size_t)((W.n + 31) / 32);
    if (cudaMalloc((void **)&W.mfw_mask, nwords * sizeof(unsigned)) != cudaSuccess) return cudaErrorMemoryAllocation;
    if (cudaMalloc((void **)&W.mfw_st, sizeof(MfwState)) != cudaSuccess) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaMemsetAsync(W.mfw_mask, 0, nwords * sizeof(unsigned), W.st);
    if (e == cudaSuccess) e = cudaMemsetAsync(W.mfw_st, 0, sizeof(MfwState), W.st);
    return e;
}

cudaError_t newton_mfw_reset(Work &W)
{
    return cudaMemsetAsync(W.mfw_st, 0, sizeof(MfwState), W.st);
}

// Large free set, 128 < q <= 1024 (dense FP32 X, q % 16 == 0): exact column
// sums -> tensor-core Gram -> M_pre -> preconditioner -> matrix-free CG.
// Workspace: the column sums' block partials in the region of the CG's chunk
// partials, then the Gram partials from the start of W.part (consumed by
// mfw_build_m_kernel), then W.part holds the 8 x 8 diagonal inverses, the
// inverse tiles, the CG's exchange vectors and the factor's flag; Pinv and h
// sit in W.M (unused by the mixed form), the factor in W.Lf.  prepare issues
// the ordinary launches and fills W.mfw_s / W.mfw_c; run (or the batch's
// grouped run) issues the two cooperative ones.
cudaError_t newton_mfw_prepare(Work &W, const int32_t *J, long long p, double sigma, const double *g, double *dv,
                               bool dots)
{
    const int q = (int)W.q;
    if (q <= kCgMaxQ || q > kBcMaxQ || q % 16 != 0 || !W.xf32 || p < 1 || !W.mfw_st) return cudaErrorInvalidValue;
    const int nblk = (q + kWdBlk - 1) / kWdBlk;
    const int Gc = 4 * W.nsm;   // column-sum blocks (and room for the W.nsm chunk partials of the CG)
    const size_t need = (size_t)q * kPb + (size_t)nblk * kWdBlk * kWdBlk + 2 * (size_t)Gc * q + 3 * (size_t)q + 4;
    if (need > 2 * W.part_len) return cudaErrorInvalidValue;
    double *info = W.red + 12;
    MfwState *st = W.mfw_st;
    const int *skip = &st->skip;
    // reuse decision and, on a rebuild, the bitmap of this J
    mfw_decide_kernel<<<W.nsm, 256, 0, W.st>>>(J, p, sigma, W.mfw_mask, st, info, mfw_reuse_frac(), kMfwStaleIt);
    mfw_mask_clear_kernel<<<W.nsm, 256, 0, W.st>>>(W.mfw_mask, (W.n + 31) / 32, st);
    mfw_mask_set_kernel<<<2 * W.nsm, 256, 0, W.st>>>(J, p, W.mfw_mask, st);
    W.nlaunch += 3;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int KS = gram_wide_splits(W, p);
    float *cpart = reinterpret_cast<float *>(W.part);
    float *Pinv = reinterpret_cast<float *>(W.M);
    float2 *H = reinterpret_cast<float2 *>(Pinv + (size_t)q * q);
    float *Dg = reinterpret_cast<float *>(W.part);
    float *Linv = Dg + (size_t)q * kPb;
    float2 *cgp = reinterpret_cast<float2 *>(Linv + (size_t)nblk * kWdBlk * kWdBlk);
    float2 *yg = cgp + (size_t)Gc * q;
    float *zg = reinterpret_cast<float *>(yg + q);
    int *fflag = reinterpret_cast<int *>(zg + q);
    // the exact h (the CG's operator needs it; M_pre too), its scratch the CG's
    // chunk partials (free until the CG); then the Gram and M_pre, which return
    // at once when the preconditioner is kept (the Gram partials reuse the
    // scratch after the column sums are done)
    e = launch_colsum(W, J, p, colsum_blocks(W, p, Gc), cgp, H);
    if (e == cudaSuccess) e = launch_gram_umma_wide(W, J, p, KS, cpart, skip);
    if (e != cudaSuccess) return e;
    {
        const long long nb = ((long long)q * q + 255) / 256;
        mfw_build_m_kernel<<<(unsigned)(nb < 8 * W.nsm ? nb : 8 * W.nsm), 256, 0, W.st>>>(
            q, KS, cpart, H, split2w(1.0 / (double)p), split2w(sigma), W.Mf, skip);
        ++W.nlaunch;
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    MfwSetupArgs &s = W.mfw_s;
    s.q = q;
    s.Mf = W.Mf;
    s.Lg = W.Lf;
    s.Dg = Dg;
    s.Linv = Linv;
    s.Pinv = Pinv;
    s.fflag = fflag;
    s.bar = W.bar;
    s.err = W.err;
    s.info = info;
    s.skip = skip;
    MfwArgs &a = W.mfw_c;
    a.X = (const float *)W.X;
    a.J = J;
    a.p = p;
    a.q = q;
    a.sig = split2w(sigma);
    a.rp = split2w(1.0 / (double)p);
    a.H = H;
    a.Pinv = Pinv;
    a.g = g;
    a.dv = dv;
    a.eta = (float)W.eta;
    a.tau = (float)W.tau;
    a.floor = (float)W.cg_floor;
    a.maxit = W.cg_maxit;
    a.info = info;
    a.err = W.err;
    a.vdot = dots ? W.v : nullptr;
    a.rdots = W.red;
    a.vc = W.nsm;
    a.part = cgp;
    a.yg = yg;
    a.zg = zg;
    a.bar = W.bar;
    return cudaGetLastError();
}

cudaError_t newton_mfw_run(Work &W)
{
    cudaError_t e = setup_attr();
    if (e != cudaSuccess) return e;
    const size_t smem = cg_fast_smem(kCgMaxQ);
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, newton_mfw_setup_kernel, kCgThreads, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    {
        MfwSetupArgs sa = W.mfw_s;
        void *args[] = {&sa};
        e = cudaLaunchCooperativeKernel((const void *)newton_mfw_setup_kernel, dim3(occ * W.nsm), dim3(kCgThreads),
                                        args, smem, W.st);
        if (e != cudaSuccess) return e;
    }
    e = launch_cg_nf4((int)W.q, W.mfw_c, nullptr, 1, W.nsm, W.nsm, W.st);
    W.nlaunch += 2;
    return e;
}

cudaError_t launch_newton_mfw(Work &W, const int32_t *J, long long p, double sigma, const double *g, double *dv,
                              bool dots)
{
    const cudaError_t e = newton_mfw_prepare(W, J, p, sigma, g, dv, dots);
    return e == cudaSuccess ? newton_mfw_run(W) : e;
}

// The prepared steps of ntask problems of one q (tables of their W.mfw_s /
// W.mfw_c in device memory): the set-up and the CG each in launches of up to
// nsm / 8 problems, a group of nsm / (problems in the launch) blocks each.
cudaError_t newton_mfw_run_group(Work &Wl, int q, const MfwSetupArgs *Ts, const MfwArgs *Tc, int ntask)
{
    if (ntask < 1) return cudaSuccess;
    if (q <= kCgMaxQ || q > kBcMaxQ || q % 16 != 0) return cudaErrorInvalidValue;
    cudaError_t e = setup_attr();
    if (e != cudaSuccess) return e;
    const int per_launch = Wl.nsm / 8 > 0 ? Wl.nsm / 8 : 1;
    const size_t smem = cg_fast_smem(kCgMaxQ);
    const MfwArgs unused{};
    for (int k0 = 0; k0 < ntask; k0 += per_launch) {
        int nt = ntask - k0 < per_launch ? ntask - k0 : per_launch;
        int Gp = Wl.nsm / nt;
        const MfwSetupArgs *Tsk = Ts + k0;
        void *args[] = {(void *)&Tsk, &nt, &Gp};
        e = cudaLaunchCooperativeKernel((const void *)newton_mfw_setup_group_kernel, dim3(nt * Gp), dim3(kCgThreads),
                                        args, smem, Wl.st);
        if (e != cudaSuccess) return e;
        e = launch_cg_nf4(q, unused, Tc + k0, nt, Gp, nt * Gp, Wl.st);
        if (e != cudaSuccess) return e;
        Wl.nlaunch += 2;
    }
    return cudaSuccess;
}

}  // namespace svm
