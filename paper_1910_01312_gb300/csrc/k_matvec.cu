// k_matvec.cu -- the A v and A' c products over the dense row-major data
// (z = A v is Q w in the paper's variables, eq. (3.3); A' pi gives the
// gradient of eq. (3.10)), plus the small q-vector updates of Algorithm 3.
//
// PLAIN_FP64 arithmetic: X elements are widened exactly to FP64 and every
// product and sum is FP64.  Rows are read with 16-byte vector loads by a
// group of G lanes per row (G chosen so each lane issues <= 4 loads per row),
// so every load instruction of a warp touches whole 32-byte sectors.
#include <math.h>

#include "internal.cuh"

namespace svm {

template <typename TX> struct Vec;
template <> struct Vec<float> { using T = float4; static constexpr int W = 4; };
template <> struct Vec<double> { using T = double2; static constexpr int W = 2; };

__device__ __forceinline__ void vload(const float4 *p, double *o)
{
    float4 t = __ldcs(p);
    o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
}
__device__ __forceinline__ void vload(const double2 *p, double *o)
{
    double2 t = __ldcs(p);
    o[0] = t.x; o[1] = t.y;
}

// z_i = y_i <x_i, v>; GL lanes per row; vectorised when VEC.
template <typename TX, int GL, bool VEC>
__global__ void __launch_bounds__(256) matvec_kernel(const TX *__restrict__ X, const int8_t *__restrict__ y,
                                                     long long n, int q, const double *__restrict__ v,
                                                     double *__restrict__ z)
{
    extern __shared__ double sv[];
    for (int j = threadIdx.x; j < q; j += blockDim.x) sv[j] = v[j];
    __syncthreads();
    constexpr int RPW = 32 / GL;   // rows per warp step
    const int lane = threadIdx.x & 31;
    const int sub = lane % GL, grp = lane / GL;
    const long long warps_total = (long long)gridDim.x * (blockDim.x >> 5);
    const long long wid = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    for (long long r0 = wid * RPW; r0 < n; r0 += warps_total * RPW) {
        long long i = r0 + grp;
        double acc = 0.0;
        if (i < n) {
            const TX *row = X + i * (long long)q;
            if (VEC) {
                using VT = typename Vec<TX>::T;
                constexpr int W = Vec<TX>::W;
                const VT *rv = reinterpret_cast<const VT *>(row);
                const int nv = q / W;
                for (int c = sub; c < nv; c += GL) {
                    double e[W];
                    vload(rv + c, e);
#pragma unroll
                    for (int k = 0; k < W; ++k) acc = fma(e[k], sv[c * W + k], acc);
                }
            } else {
                for (int c = sub; c < q; c += GL) acc = fma((double)row[c], sv[c], acc);
            }
        }
#pragma unroll
        for (int o = GL / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (i < n && sub == 0) z[i] = (y[i] > 0) ? acc : -acc;
    }
}

template <typename TX, bool VEC>
static cudaError_t matvec_dispatch(Work &W, const double *v, double *z)
{
    constexpr int Wd = VEC ? Vec<TX>::W : 1;
    int chunks = (int)((W.q + Wd - 1) / Wd);
    int gl = 1;
    while (gl < 32 && (chunks + gl - 1) / gl > 4) gl <<= 1;
    int blocks = W.nsm * 8;
    size_t smem = (size_t)W.q * sizeof(double);
    const TX *X = (const TX *)W.X;
#define MV_CASE(G)                                                                                         \
    case G:                                                                                                \
        matvec_kernel<TX, G, VEC><<<blocks, 256, smem, W.st>>>(X, W.y, W.n, (int)W.q, v, z);             \
        ++W.nlaunch;                                                                                       \
        break;
    switch (gl) {
        MV_CASE(1) MV_CASE(2) MV_CASE(4) MV_CASE(8) MV_CASE(16) MV_CASE(32)
    }
#undef MV_CASE
    return cudaGetLastError();
}

cudaError_t launch_matvec(Work &W, const double *v, double *z)
{
    size_t es = W.xf32 ? 4 : 8;
    bool vec = ((W.q * es) % 16 == 0) && ((uintptr_t)W.X % 16 == 0);
    if (W.xf32) return vec ? matvec_dispatch<float, true>(W, v, z) : matvec_dispatch<float, false>(W, v, z);
    return vec ? matvec_dispatch<double, true>(W, v, z) : matvec_dispatch<double, false>(W, v, z);
}

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
        long long i = idx ? (long long)idx[r] : r;
        double ci = c[i];
        if (ci == 0.0) continue;
        double cy = (y[i] > 0) ? ci : -ci;
        const TX *row = X + i * (long long)q;
#pragma unroll
        for (int k = 0; k < NCH; ++k) {
            int j = lane + 32 * k;
            if (j < q) {
                double xv = (double)__ldcs(row + j);
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
                int j = lane + 32 * k;
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

// out_j = sum_b part[b][j] (fixed order); red[slot] = sum_j (sum_b apart[b][j])^2
__global__ void rmatvec_final_kernel(int G, int q, const double *__restrict__ part,
                                     const double *__restrict__ apart, double *__restrict__ out,
                                     double *__restrict__ red, int slot)
{
    __shared__ double sh[32];
    double local = 0.0;
    for (int j = threadIdx.x; j < q; j += blockDim.x) {
        double s = 0.0, a = 0.0;
        for (int b = 0; b < G; ++b) { s += part[(size_t)b * q + j]; a += apart[(size_t)b * q + j]; }
        out[j] = s;
        local += a * a;
    }
    local = warp_sum(local);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = local;
    __syncthreads();
    if (threadIdx.x == 0 && slot >= 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        red[slot] = t;
    }
}

template <typename TX>
static cudaError_t rmatvec_t(Work &W, const double *c, const int32_t *idx, const long long *cnt_dev,
                             double *out, int scale_slot)
{
    int q = (int)W.q;
    int nch = (q + 31) / 32;
    int G = W.rm_grid;
    double *part = W.part;
    double *apart = W.part + (size_t)G * q;
    size_t smem = (size_t)2 * q * sizeof(double);
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

cudaError_t launch_rmatvec(Work &W, const double *c, const int32_t *idx, const long long *cnt_dev,
                           double *out, int scale_slot)
{
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
        double gj = v[j] - atp[j];
        g[j] = gj;
        s = fma(gj, gj, s);
    }
    double t = block_sum_1024(s, sh);
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
cudaError_t launch_zaxpy(Work &W, double t)
{
    int blocks = (int)((W.n + 1023) / 1024);
    if (blocks > W.nsm * 4) blocks = W.nsm * 4;
    axpy_kernel<<<blocks, 1024, 0, W.st>>>(W.n, t, W.dz, W.z);
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
