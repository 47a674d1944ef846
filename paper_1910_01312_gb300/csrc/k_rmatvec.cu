// k_rmatvec.cu -- the transposed product A' c over a row list or all rows
// (A' pi gives the gradient of eq. (3.10)), the double-float splits of
// n-vectors, and the small q-vector updates of Algorithm 3.
//
// PLAIN_FP64: FP64 products and sums.  MIXED: Dot2 sums of exact FP32
// products with double-float weights (Ogita, Rump and Oishi, 2005), block
// partials as double-float pairs, and a last-block reduction in block order.
#include <math.h>

#include "internal.cuh"

namespace svm {

// ----------------------------------------------------------------- A' c

// Block-partial of out_j = sum_r c_{i_r} y_{i_r} x_{i_r j} over this block's
// contiguous share of the row list; lane l owns columns l, l+32, ... (scalar
// columns, NCH per lane).  Also the absolute sums for the roundoff scale.
template <typename TX, int NCH>
__global__ void __launch_bounds__(256) rmatvec_part_kernel(const TX *__restrict__ X, const int8_t *__restrict__ y,
                                                           long long n, int q, const double *__restrict__ c,
                                                           const int32_t *__restrict__ idx,
                                                           const long long *__restrict__ cnt_dev,
                                                           double *__restrict__ part, double *__restrict__ apart)
{
    const long long cnt = idx ? *cnt_dev : n;
    const int G = gridDim.x;
    const long long per = (cnt + G - 1) / G;
    const long long r_beg = (long long)blockIdx.x * per;
    const long long r_end = r_beg + per < cnt ? r_beg + per : cnt;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double acc[NCH];
    float aac[NCH];
#pragma unroll
    for (int k = 0; k < NCH; ++k) { acc[k] = 0.0; aac[k] = 0.f; }
    for (long long r = r_beg + warp; r < r_end; r += nw) {
        const long long i = idx ? (long long)idx[r] : r;
        const double ci = c[i];
        if (ci == 0.0) continue;
        const double cy = (y[i] > 0) ? ci : -ci;
        const TX *row = X + i * (long long)q;
#pragma unroll
        for (int k = 0; k < NCH; ++k) {
            const int j = lane + 32 * k;
            if (j < q) {
                const double xv = (double)__ldcs(row + j);
                acc[k] = fma(cy, xv, acc[k]);
                aac[k] += (float)fabs(cy * xv);
            }
        }
    }
    extern __shared__ double sred[];   // [2][q]
    for (int j = threadIdx.x; j < 2 * q; j += blockDim.x) sred[j] = 0.0;
    __syncthreads();
    for (int w = 0; w < nw; ++w) {
        if (warp == w) {
#pragma unroll
            for (int k = 0; k < NCH; ++k) {
                const int j = lane + 32 * k;
                if (j < q) { sred[j] += acc[k]; sred[q + j] += (double)aac[k]; }
            }
        }
        __syncthreads();
    }
    for (int j = threadIdx.x; j < q; j += blockDim.x) {
        part[(size_t)blockIdx.x * q + j] = sred[j];
        apart[(size_t)blockIdx.x * q + j] = sred[q + j];
    }
}

// Mixed form.  Weights arrive as y_i c_i in FP32 (hi, lo) pairs; VW = 4:
// lane l owns the float4 column chunks l + 32k (q % 4 == 0), VW = 1: the
// scalar columns l + 32k.  Rows are in flight R at a time per warp.  The
// block's warps are combined by a tree over shared memory, and the block
// that finishes last (threadfence + counter) performs the fixed-order final
// reduction over all block partials, so one launch yields out = A'c.
// Last-block reduction of the double-float partials [G][3][q] (hi, lo, abs):
// per column, subs interleaved sub-sums over the blocks, combined in order.
__device__ void final_reduce_df(int G, int q, const float *__restrict__ part, const double *__restrict__ base,
                                const float *__restrict__ abase, double *__restrict__ out, float *__restrict__ aout,
                                double *__restrict__ red, int slot, float *sm, const GradOut go)
{
    __shared__ double gsh[32];
    double gsq = 0.0;
    const int subs = blockDim.x >> 7;
    const int tx = threadIdx.x & 127, sub = threadIdx.x >> 7;
    float2 *sp = reinterpret_cast<float2 *>(sm);   // [subs][128]
    float *sa = sm + 2 * subs * 128;               // [subs][128]
    float scale = 0.f;
    for (int c0 = 0; c0 < q; c0 += 128) {
        const int col = c0 + tx;
        float2 S = make_float2(0.f, 0.f);
        float A = 0.f;
        if (col < q) {
            // eight blocks' loads in flight per step, added in block order
            int b = sub;
            for (; b + 7 * subs < G; b += 8 * subs) {
                float h[8], l[8], ab[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const float *p = part + (size_t)(b + u * subs) * 3 * q;
                    h[u] = __ldcg(p + col);
                    l[u] = __ldcg(p + q + col);
                    ab[u] = __ldcg(p + 2 * q + col);
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    S = dfx_add(S, make_float2(h[u], l[u]));
                    A += ab[u];
                }
            }
            for (; b < G; b += subs) {
                const float *p = part + (size_t)b * 3 * q;
                S = dfx_add(S, make_float2(__ldcg(p + col), __ldcg(p + q + col)));
                A += __ldcg(p + 2 * q + col);
            }
        }
        sp[sub * 128 + tx] = S;
        sa[sub * 128 + tx] = A;
        __syncthreads();
        if (sub == 0 && col < q) {
            float2 T = make_float2(0.f, 0.f);
            float TA = 0.f;
            for (int k = 0; k < subs; ++k) { T = dfx_add(T, sp[k * 128 + tx]); TA += sa[k * 128 + tx]; }
            const double v = (double)T.x + (double)T.y;
            const double o = base ? base[col] + v : v;
            out[col] = o;
            if (go.g) {   // gradient at the (trial) point: g = (v + t dv) - A'pi
                double vt = go.v[col];
                if (go.dv) vt = fma(go.t, go.dv[col], vt);
                if (go.vt) go.vt[col] = vt;
                const double gg = vt - o;
                go.g[col] = gg;
                gsq = fma(gg, gg, gsq);
            }
            const float a = abase ? abase[col] + TA : TA;
            if (aout) aout[col] = a;
            scale = fmaf(a, a, scale);
        }
        __syncthreads();
    }
    if (slot >= 0) {
        if (sub == 0) {
            const float v = warp_sumf(scale);
            if ((tx & 31) == 0) sa[tx >> 5] = v;
        }
        __syncthreads();
        if (threadIdx.x == 0) red[slot] = (double)((sa[0] + sa[1]) + (sa[2] + sa[3]));
    }
    if (go.g) {
        if (sub == 0) {
            const double v = warp_sum(gsq);
            if ((tx & 31) == 0) gsh[tx >> 5] = v;
        }
        __syncthreads();
        if (threadIdx.x == 0) red[0] = (gsh[0] + gsh[1]) + (gsh[2] + gsh[3]);
    }
}

// out = base + sum_i wc_i x_i, aout = abase + sum_i wa_i |x_i| (wa null: |wc_i.hi|),
// red[slot] = |aout|^2, over idx (count *cnt_dev) or all rows.  Per-block
// partials are double-float; the last block to finish adds them in block order
// in double-float arithmetic (no FP64 beyond one conversion per column).
template <int VW, int NCH>
__global__ void __launch_bounds__(NCH * VW >= 8 ? 256 : 1024) rmatvec_mx_part_kernel(
    const float *__restrict__ X, long long n, int q, const float2 *__restrict__ wc, const float *__restrict__ wa,
    const int32_t *__restrict__ idx, const long long *__restrict__ cnt_dev, float *__restrict__ part,
    unsigned *__restrict__ counter, const double *__restrict__ base, const float *__restrict__ abase,
    double *__restrict__ out, float *__restrict__ aout, double *__restrict__ red, int slot, const GradOut go)
{
    const long long cnt = idx ? *cnt_dev : n;
    const int G = gridDim.x;
    const long long per = (cnt + G - 1) / G;
    const long long r_beg = (long long)blockIdx.x * per;
    const long long r_end = r_beg + per < cnt ? r_beg + per : cnt;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int nch = q / VW;
    float s[NCH][VW], c[NCH][VW], ab[NCH][VW];
#pragma unroll
    for (int k = 0; k < NCH; ++k)
#pragma unroll
        for (int e = 0; e < VW; ++e) { s[k][e] = 0.f; c[k][e] = 0.f; ab[k][e] = 0.f; }
    // A warp takes 32-row chunks of the block's range; its lanes load the 32 row
    // indices and weights at once, then rows are streamed R at a time with all
    // R row loads in flight before any arithmetic.
    constexpr int R = NCH >= 4 ? 2 : (NCH == 2 ? 4 : 8);
    for (long long c0 = r_beg + (long long)warp * 32; c0 < r_end; c0 += (long long)nw * 32) {
        const long long rl = c0 + lane;
        int myi = -1;
        float2 myw = make_float2(0.f, 0.f);
        float mya = 0.f;
        if (rl < r_end) {
            myi = idx ? idx[rl] : (int)rl;
            myw = wc[myi];
            mya = wa ? wa[myi] : fabsf(myw.x);
        }
        const int here = (int)((r_end - c0) < 32 ? (r_end - c0) : 32);
        for (int u0 = 0; u0 < here; u0 += R) {
            int ii[R];
            float2 w[R];
            float wab[R];
#pragma unroll
            for (int u = 0; u < R; ++u) {
                const int src = (u0 + u) & 31;
                ii[u] = __shfl_sync(0xffffffffu, myi, src);
                w[u].x = __shfl_sync(0xffffffffu, myw.x, src);
                w[u].y = __shfl_sync(0xffffffffu, myw.y, src);
                wab[u] = __shfl_sync(0xffffffffu, mya, src);
                if (u0 + u >= here) ii[u] = -1;
            }
            float xv[R][NCH][VW];
#pragma unroll
            for (int u = 0; u < R; ++u)
#pragma unroll
                for (int k = 0; k < NCH; ++k) {
                    const int ch = lane + 32 * k;
                    if (ii[u] >= 0 && ch < nch) {
                        if (VW == 4) {
                            const float4 x4 =
                                __ldcs(reinterpret_cast<const float4 *>(X + (long long)ii[u] * q) + ch);
                            xv[u][k][0] = x4.x; xv[u][k][VW > 1 ? 1 : 0] = x4.y;
                            xv[u][k][VW > 2 ? 2 : 0] = x4.z; xv[u][k][VW > 3 ? 3 : 0] = x4.w;
                        } else {
                            xv[u][k][0] = __ldcs(X + (long long)ii[u] * q + ch);
                        }
                    } else {
#pragma unroll
                        for (int e = 0; e < VW; ++e) xv[u][k][e] = 0.f;
                    }
                }
#pragma unroll
            for (int u = 0; u < R; ++u)
#pragma unroll
                for (int k = 0; k < NCH; ++k)
#pragma unroll
                    for (int e = 0; e < VW; ++e) {
                        dot2_step(xv[u][k][e], w[u], s[k][e], c[k][e]);
                        ab[k][e] = fmaf(fabsf(xv[u][k][e]), wab[u], ab[k][e]);
                    }
        }
    }
    // per-warp results to shared memory: [warp][3][q]
    extern __shared__ float sredf[];
#pragma unroll
    for (int k = 0; k < NCH; ++k) {
        const int ch = lane + 32 * k;
        if (ch < nch)
#pragma unroll
            for (int e = 0; e < VW; ++e) {
                const int j = ch * VW + e;
                float *b = sredf + (size_t)warp * 3 * q;
                b[j] = s[k][e];
                b[q + j] = c[k][e];
                b[2 * q + j] = ab[k][e];
            }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < q; j += blockDim.x) {
        float ss = 0.f, cc = 0.f, aa = 0.f;
        for (int wv = 0; wv < nw; ++wv) {
            const float *b = sredf + (size_t)wv * 3 * q;
            df_acc(ss, cc, b[j], b[q + j]);
            aa += b[2 * q + j];
        }
        float hi, lo;
        two_sum(ss, cc, hi, lo);
        float *pb = part + (size_t)blockIdx.x * 3 * q;
        pb[j] = hi;
        pb[q + j] = lo;
        pb[2 * q + j] = aa;
    }
    __threadfence();
    __syncthreads();
    __shared__ int is_last;
    if (threadIdx.x == 0) is_last = (atomicAdd(counter, 1u) == (unsigned)(G - 1));
    __syncthreads();
    if (is_last) {
        __threadfence();
        final_reduce_df(G, q, part, base, abase, out, aout, red, slot, sredf, go);
        if (threadIdx.x == 0) *counter = 0u;
    }
}

// The same for 128 < q <= 1024 (q % 4 == 0): a lane holding all q columns'
// sums needs ~3q/32 registers, which leaves one block of eight warps per SM
// with two rows in flight each.  Here the columns are cut into NSL slices of
// 256 (two float4 per lane) and the block's 16 warps are 16/NSL row groups x
// NSL slices: each warp streams its row group's 32-row chunks of the block's
// share for its slice, R rows in flight, so every byte of a row is read once
// per block.  Block partials and the last-block reduction as above.
constexpr int kRcThreads = 512;
template <int NSL>
__global__ void __launch_bounds__(kRcThreads, 1) rmatvec_mx_cols_kernel(
    const float *__restrict__ X, long long n, int q, const float2 *__restrict__ wc, const float *__restrict__ wa,
    const int32_t *__restrict__ idx, const long long *__restrict__ cnt_dev, float *__restrict__ part,
    unsigned *__restrict__ counter, const double *__restrict__ base, const float *__restrict__ abase,
    double *__restrict__ out, float *__restrict__ aout, double *__restrict__ red, int slot, const GradOut go)
{
    constexpr int NRG = (kRcThreads / 32) / NSL;
    constexpr int R = 8;
    const long long cnt = idx ? *cnt_dev : n;
    const int G = gridDim.x;
    const long long per = (cnt + G - 1) / G;
    const long long r_beg = (long long)blockIdx.x * per;
    const long long r_end = r_beg + per < cnt ? r_beg + per : cnt;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int sl = warp % NSL, rg = warp / NSL;
    const int nf4 = q / 4;
    float s[8], c[8], ab[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) { s[k] = 0.f; c[k] = 0.f; ab[k] = 0.f; }
    for (long long c0 = r_beg + (long long)rg * 32; c0 < r_end; c0 += (long long)NRG * 32) {
        const long long rl = c0 + lane;
        int myi = -1;
        float2 myw = make_float2(0.f, 0.f);
        float mya = 0.f;
        if (rl < r_end) {
            myi = idx ? idx[rl] : (int)rl;
            myw = wc[myi];
            mya = wa ? wa[myi] : fabsf(myw.x);
        }
        const int here = (int)((r_end - c0) < 32 ? (r_end - c0) : 32);
        for (int u0 = 0; u0 < here; u0 += R) {
            int ii[R];
            float2 w[R];
            float wab[R];
#pragma unroll
            for (int u = 0; u < R; ++u) {
                const int src = (u0 + u) & 31;
                ii[u] = __shfl_sync(0xffffffffu, myi, src);
                w[u].x = __shfl_sync(0xffffffffu, myw.x, src);
                w[u].y = __shfl_sync(0xffffffffu, myw.y, src);
                wab[u] = __shfl_sync(0xffffffffu, mya, src);
                if (u0 + u >= here) ii[u] = -1;
            }
            float4 xv[R][2];
#pragma unroll
            for (int u = 0; u < R; ++u)
#pragma unroll
                for (int f = 0; f < 2; ++f) {
                    const int c4 = sl * 64 + 32 * f + lane;
                    xv[u][f] = (ii[u] >= 0 && c4 < nf4)
                                   ? __ldcs(reinterpret_cast<const float4 *>(X + (long long)ii[u] * q) + c4)
                                   : make_float4(0.f, 0.f, 0.f, 0.f);
                }
#pragma unroll
            for (int u = 0; u < R; ++u)
#pragma unroll
                for (int f = 0; f < 2; ++f) {
                    const float xs[4] = {xv[u][f].x, xv[u][f].y, xv[u][f].z, xv[u][f].w};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        dot2_step(xs[e], w[u], s[4 * f + e], c[4 * f + e]);
                        ab[4 * f + e] = fmaf(fabsf(xs[e]), wab[u], ab[4 * f + e]);
                    }
                }
        }
    }
    // per-row-group results to shared memory: [rg][3][q], then the row groups in order
    extern __shared__ float sredf[];
#pragma unroll
    for (int f = 0; f < 2; ++f) {
        const int c4 = sl * 64 + 32 * f + lane;
        if (c4 < nf4) {
            float *b = sredf + (size_t)rg * 3 * q;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int j = 4 * c4 + e;
                b[j] = s[4 * f + e];
                b[q + j] = c[4 * f + e];
                b[2 * q + j] = ab[4 * f + e];
            }
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < q; j += blockDim.x) {
        float ss = 0.f, cc = 0.f, aa = 0.f;
        for (int g = 0; g < NRG; ++g) {
            const float *b = sredf + (size_t)g * 3 * q;
            df_acc(ss, cc, b[j], b[q + j]);
            aa += b[2 * q + j];
        }
        float hi, lo;
        two_sum(ss, cc, hi, lo);
        float *pb = part + (size_t)blockIdx.x * 3 * q;
        pb[j] = hi;
        pb[q + j] = lo;
        pb[2 * q + j] = aa;
    }
    __threadfence();
    __syncthreads();
    __shared__ int is_last;
    if (threadIdx.x == 0) is_last = (atomicAdd(counter, 1u) == (unsigned)(G - 1));
    __syncthreads();
    if (is_last) {
        __threadfence();
        final_reduce_df(G, q, part, base, abase, out, aout, red, slot, sredf, go);
        if (threadIdx.x == 0) *counter = 0u;
    }
}

// out_j = sum_b part[b][j] in a fixed order (8 interleaved sub-sums per
// column, then the 8 combined in order); red[slot] = sum_j (sum_b apart[b][j])^2.
// One block of 1024 threads: 128 columns x 8 sub-sums per round.
__global__ void __launch_bounds__(1024) rmatvec_final_kernel(int G, int q, const double *__restrict__ part,
                                                             const double *__restrict__ apart,
                                                             double *__restrict__ out, double *__restrict__ red,
                                                             int slot)
{
    __shared__ double sp[8][128], sa[8][128];
    __shared__ double sq[128];
    const int tx = threadIdx.x & 127, sub = threadIdx.x >> 7;
    double scale = 0.0;
    for (int c0 = 0; c0 < q; c0 += 128) {
        const int col = c0 + tx;
        double s = 0.0, a = 0.0;
        if (col < q) {
#pragma unroll 4
            for (int b = sub; b < G; b += 8) {
                s += __ldcg(part + (size_t)b * q + col);
                a += __ldcg(apart + (size_t)b * q + col);
            }
        }
        sp[sub][tx] = s;
        sa[sub][tx] = a;
        __syncthreads();
        if (sub == 0 && col < q) {
            double ts = 0.0, ta = 0.0;
#pragma unroll
            for (int k = 0; k < 8; ++k) { ts += sp[k][tx]; ta += sa[k][tx]; }
            out[col] = ts;
            scale = fma(ta, ta, scale);
        }
        __syncthreads();
    }
    if (sub == 0) sq[tx] = scale;
    __syncthreads();
    if (threadIdx.x == 0 && slot >= 0) {
        double t = 0.0;
        for (int k = 0; k < 128; ++k) t += sq[k];
        red[slot] = t;
    }
}

template <typename TX>
static cudaError_t rmatvec_t(Work &W, const double *c, const int32_t *idx, const long long *cnt_dev, double *out,
                             int scale_slot)
{
    const int q = (int)W.q;
    const int nch = (q + 31) / 32;
    const int G = W.rm_grid;
    double *part = W.part;
    double *apart = W.part + (size_t)G * q;
    const size_t smem = (size_t)2 * q * sizeof(double);
    const TX *X = (const TX *)W.X;
#define RM_CASE(K)                                                                                         \
    if (nch <= K) {                                                                                        \
        rmatvec_part_kernel<TX, K><<<G, 256, smem, W.st>>>(X, W.y, W.n, q, c, idx, cnt_dev, part, apart);  \
    } else
    RM_CASE(1) RM_CASE(2) RM_CASE(4) RM_CASE(8) RM_CASE(16) RM_CASE(32) { return cudaErrorInvalidValue; }
#undef RM_CASE
    rmatvec_final_kernel<<<1, 1024, 0, W.st>>>(G, q, part, apart, out, W.red, scale_slot);
    W.nlaunch += 2;
    return cudaGetLastError();
}

static int g_rmx_attr = 0;
static int g_rmc_attr = 0;

static cudaError_t rmatvec_mx(Work &W, const float2 *wc, const float *wa, const int32_t *idx,
                              const long long *cnt_dev, const double *base, const float *abase, double *out,
                              float *aout, int scale_slot, const GradOut &go)
{
    const int q = (int)W.q;
    const bool vec = (q % 4 == 0) && ((uintptr_t)W.X % 16 == 0);
    const int nch = vec ? (q / 4 + 31) / 32 : (q + 31) / 32;
    int nch_t = 1;
    while (nch_t < nch) nch_t <<= 1;
    const int threads = nch_t * (vec ? 4 : 1) >= 8 ? 256 : 1024;   // must match the kernel's launch bounds
    const int G = threads == 1024 ? W.nsm : W.nsm * 4;
    float *part = reinterpret_cast<float *>(W.part);
    size_t smem = (size_t)(threads / 32) * 3 * q * sizeof(float);
    const size_t smem_final = (size_t)3 * (threads / 128) * 128 * sizeof(float);
    if (smem < smem_final) smem = smem_final;
    if (!g_rmx_attr) {
        const void *fns[] = {(const void *)rmatvec_mx_part_kernel<4, 1>, (const void *)rmatvec_mx_part_kernel<4, 2>,
                             (const void *)rmatvec_mx_part_kernel<4, 4>, (const void *)rmatvec_mx_part_kernel<4, 8>,
                             (const void *)rmatvec_mx_part_kernel<1, 1>, (const void *)rmatvec_mx_part_kernel<1, 2>,
                             (const void *)rmatvec_mx_part_kernel<1, 4>, (const void *)rmatvec_mx_part_kernel<1, 8>,
                             (const void *)rmatvec_mx_part_kernel<1, 16>, (const void *)rmatvec_mx_part_kernel<1, 32>};
        for (const void *f : fns) {
            const cudaError_t ea = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
            if (ea != cudaSuccess) return ea;
        }
        g_rmx_attr = 1;
    }
    const float *X = (const float *)W.X;
#define RX_ARGS X, W.n, q, wc, wa, idx, cnt_dev, part, W.rm_counter, base, abase, out, aout, W.red, scale_slot, go
    if (vec && q > 128 && q <= 1024) {
        // column slices: one block of 16 warps per SM
        const int Gc = W.nsm;
        const int nsl = q <= 512 ? 2 : 4;
        const size_t smc = (size_t)((kRcThreads / 32) / nsl) * 3 * q * sizeof(float);
        if (!g_rmc_attr) {
            cudaError_t ea = cudaFuncSetAttribute(rmatvec_mx_cols_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  64 * 1024);
            if (ea == cudaSuccess)
                ea = cudaFuncSetAttribute(rmatvec_mx_cols_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          64 * 1024);
            if (ea != cudaSuccess) return ea;
            g_rmc_attr = 1;
        }
        if (nsl == 2) rmatvec_mx_cols_kernel<2><<<Gc, kRcThreads, smc, W.st>>>(RX_ARGS);
        else rmatvec_mx_cols_kernel<4><<<Gc, kRcThreads, smc, W.st>>>(RX_ARGS);
    } else if (vec) {
        if (nch <= 1) rmatvec_mx_part_kernel<4, 1><<<G, threads, smem, W.st>>>(RX_ARGS);
        else if (nch <= 2) rmatvec_mx_part_kernel<4, 2><<<G, threads, smem, W.st>>>(RX_ARGS);
        else if (nch <= 4) rmatvec_mx_part_kernel<4, 4><<<G, threads, smem, W.st>>>(RX_ARGS);
        else if (nch <= 8) rmatvec_mx_part_kernel<4, 8><<<G, threads, smem, W.st>>>(RX_ARGS);
        else return cudaErrorInvalidValue;
    } else {
        if (nch <= 1) rmatvec_mx_part_kernel<1, 1><<<G, threads, smem, W.st>>>(RX_ARGS);
        else if (nch <= 2) rmatvec_mx_part_kernel<1, 2><<<G, threads, smem, W.st>>>(RX_ARGS);
        else if (nch <= 4) rmatvec_mx_part_kernel<1, 4><<<G, threads, smem, W.st>>>(RX_ARGS);
        else if (nch <= 8) rmatvec_mx_part_kernel<1, 8><<<G, threads, smem, W.st>>>(RX_ARGS);
        else if (nch <= 16) rmatvec_mx_part_kernel<1, 16><<<G, threads, smem, W.st>>>(RX_ARGS);
        else if (nch <= 32) rmatvec_mx_part_kernel<1, 32><<<G, threads, smem, W.st>>>(RX_ARGS);
        else return cudaErrorInvalidValue;
    }
#undef RX_ARGS
    ++W.nlaunch;
    return cudaGetLastError();
}

__global__ void split_weights_kernel(long long n, const double *c, const int8_t *y, float2 *wc)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double v = (y[i] > 0) ? c[i] : -c[i];
        const float hi = (float)v;
        wc[i] = make_float2(hi, (float)(v - (double)hi));
    }
}

cudaError_t split_weights(Work &W, const double *c, float2 *wc)
{
    int blocks = (int)((W.n + 255) / 256);
    if (blocks > W.nsm * 8) blocks = W.nsm * 8;
    split_weights_kernel<<<blocks, 256, 0, W.st>>>(W.n, c, W.y, wc);
    ++W.nlaunch;
    return cudaGetLastError();
}

cudaError_t launch_rmatvec_df(Work &W, const float2 *wc, const float *wa, const int32_t *idx, const long long *cnt_dev,
                              const double *base, const float *abase, double *out, float *aout, int slot,
                              const GradOut &go)
{
    if (!W.xf32) return cudaErrorInvalidValue;
    return rmatvec_mx(W, wc, wa, idx, cnt_dev, base, abase, out, aout, slot, go);
}

__global__ void split_vector_kernel(long long n, const double *c, const int8_t *y, int sgn, float2 *a)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double v = (sgn && y[i] < 0) ? -c[i] : c[i];
        const float hi = (float)v;
        a[i] = make_float2(hi, (float)(v - (double)hi));
    }
}

// entries equal to the split of C (the projection's value at the upper bound)
// become C exactly
__global__ void join_vector_kernel(long long n, const float2 *a, const int8_t *y, int sgn, float2 Cd, double C,
                                   double *c)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float2 v = a[i];
        const bool neg = sgn && y[i] < 0;
        if (neg) v = make_float2(-v.x, -v.y);
        c[i] = (v.x == Cd.x && v.y == Cd.y) ? C : (double)v.x + (double)v.y;
    }
}

cudaError_t split_vector(Work &W, const double *c, bool signed_by_y, float2 *a)
{
    int blocks = (int)((W.n + 255) / 256);
    if (blocks > W.nsm * 8) blocks = W.nsm * 8;
    split_vector_kernel<<<blocks, 256, 0, W.st>>>(W.n, c, W.y, signed_by_y ? 1 : 0, a);
    ++W.nlaunch;
    return cudaGetLastError();
}

cudaError_t join_vector(Work &W, const float2 *a, bool signed_by_y, double *c)
{
    int blocks = (int)((W.n + 255) / 256);
    if (blocks > W.nsm * 8) blocks = W.nsm * 8;
    const float Ch = (float)W.C;
    const float2 Cd = make_float2(Ch, (float)(W.C - (double)Ch));
    join_vector_kernel<<<blocks, 256, 0, W.st>>>(W.n, a, W.y, signed_by_y ? 1 : 0, Cd, W.C, c);
    ++W.nlaunch;
    return cudaGetLastError();
}

cudaError_t launch_rmatvec(Work &W, const double *c, const float2 *wc, const int32_t *idx, const long long *cnt_dev,
                           double *out, int scale_slot)
{
    if (W.csr) return launch_rmatvec_csr(W, c, out, scale_slot);
    if (W.precision == 1 && W.xf32 && wc)
        return rmatvec_mx(W, wc, nullptr, idx, cnt_dev, nullptr, nullptr, out, nullptr, scale_slot, GradOut());
    return W.xf32 ? rmatvec_t<float>(W, c, idx, cnt_dev, out, scale_slot)
                  : rmatvec_t<double>(W, c, idx, cnt_dev, out, scale_slot);
}

// ------------------------------------------------------------- q-vectors

__device__ __forceinline__ double block_sum_1024(double v, double *sh)
{
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    return t;
}

__global__ void grad_kernel(int q, const double *v, const double *atp, double *g, double *red)
{
    __shared__ double sh[32];
    double s = 0.0;
    for (int j = threadIdx.x; j < q; j += blockDim.x) {
        const double gj = v[j] - atp[j];
        g[j] = gj;
        s = fma(gj, gj, s);
    }
    const double t = block_sum_1024(s, sh);
    if (threadIdx.x == 0) red[0] = t;
}

__global__ void dots_kernel(int q, const double *g, const double *v, const double *dv, double *red)
{
    __shared__ double sh[3][32];
    double a = 0.0, b = 0.0, c = 0.0;
    for (int j = threadIdx.x; j < q; j += blockDim.x) {
        a = fma(g[j], dv[j], a);
        b = fma(v[j], dv[j], b);
        c = fma(dv[j], dv[j], c);
    }
    a = warp_sum(a); b = warp_sum(b); c = warp_sum(c);
    if ((threadIdx.x & 31) == 0) { sh[0][threadIdx.x >> 5] = a; sh[1][threadIdx.x >> 5] = b; sh[2][threadIdx.x >> 5] = c; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ta = 0, tb = 0, tc = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { ta += sh[0][w]; tb += sh[1][w]; tc += sh[2][w]; }
        red[2] = ta; red[3] = tb; red[4] = tc;
    }
}

__global__ void axpy_kernel(long long n, double t, const double *x, double *y)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = fma(t, x[i], y[i]);
}

__global__ void negcopy_kernel(int q, const double *g, double *dv)
{
    for (int j = threadIdx.x; j < q; j += blockDim.x) dv[j] = -g[j];
}

cudaError_t launch_grad(Work &W)
{
    grad_kernel<<<1, 1024, 0, W.st>>>((int)W.q, W.v, W.atp, W.g, W.red);
    ++W.nlaunch;
    return cudaGetLastError();
}
cudaError_t launch_dots(Work &W)
{
    dots_kernel<<<1, 1024, 0, W.st>>>((int)W.q, W.g, W.v, W.dv, W.red);
    ++W.nlaunch;
    return cudaGetLastError();
}
cudaError_t launch_vaxpy(Work &W, double t)
{
    axpy_kernel<<<1, 1024, 0, W.st>>>(W.q, t, W.dv, W.v);
    ++W.nlaunch;
    return cudaGetLastError();
}

cudaError_t launch_negcopy(Work &W, const double *g, double *dv)
{
    negcopy_kernel<<<1, 1024, 0, W.st>>>((int)W.q, g, dv);
    ++W.nlaunch;
    return cudaGetLastError();
}

}  // namespace svm
