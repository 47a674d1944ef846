// k_matvec.cu -- the forward product z = A v over the dense row-major data
// (z = A v is Q w in the paper's variables, eq. (3.3)).  The transposed
// product and the q-vector updates are in k_rmatvec.cu.
//
// The product streams X once from HBM with 16-byte vector loads (every warp
// load instruction touches whole 32-byte sectors) and is bandwidth-shaped:
// X (512 MB at n = 1e6, q = 128 FP32) never fits in L2.
//
// PLAIN_FP64: X elements are widened exactly to FP64 and every product and
// sum is FP64.  On this part the FP64 pipe is ~1/64 of the FP32 rate, so this
// form is ALU-bound, not HBM-bound.
// MIXED: products and sums on the FP32 pipes with error-free transformations
// (Dot2 of Ogita, Rump and Oishi, SIAM J. Sci. Comput. 26(6), 2005): the FP64
// operand is split into FP32 hi + lo, x*hi is formed exactly with TwoProd,
// accumulated with TwoSum, and the rounding terms plus x*lo are carried in a
// compensation word.  The result is as accurate as FP64 accumulation (error
// ~2^-48 of the sum of |terms|), at HBM speed.
#include <math.h>

#include "internal.cuh"

namespace svm {

// ---------------------------------------------------------------- A v, FP64

// z_i = y_i <x_i, v> (and the same for a second vector); GL lanes per row.
template <typename TX, int GL, bool VEC, int NV>
__global__ void __launch_bounds__(256) matvec_kernel(const TX *__restrict__ X, const int8_t *__restrict__ y,
                                                     long long n, int q, const double *__restrict__ v0,
                                                     const double *__restrict__ v1, double *__restrict__ z0,
                                                     double *__restrict__ z1)
{
    extern __shared__ double sv[];   // [NV][q]
    for (int j = threadIdx.x; j < q; j += blockDim.x) {
        sv[j] = v0[j];
        if (NV == 2) sv[q + j] = v1[j];
    }
    __syncthreads();
    constexpr int RPW = 32 / GL;   // rows per warp step
    const int lane = threadIdx.x & 31;
    const int sub = lane % GL, grp = lane / GL;
    const long long warps_total = (long long)gridDim.x * (blockDim.x >> 5);
    const long long wid = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    for (long long r0 = wid * RPW; r0 < n; r0 += warps_total * RPW) {
        const long long i = r0 + grp;
        double acc[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) acc[k] = 0.0;
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
                    for (int k = 0; k < W; ++k) {
                        acc[0] = fma(e[k], sv[c * W + k], acc[0]);
                        if (NV == 2) acc[NV - 1] = fma(e[k], sv[q + c * W + k], acc[NV - 1]);
                    }
                }
            } else {
                for (int c = sub; c < q; c += GL) {
                    const double e = (double)row[c];
                    acc[0] = fma(e, sv[c], acc[0]);
                    if (NV == 2) acc[NV - 1] = fma(e, sv[q + c], acc[NV - 1]);
                }
            }
        }
#pragma unroll
        for (int o = GL / 2; o > 0; o >>= 1)
#pragma unroll
            for (int k = 0; k < NV; ++k) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
        if (i < n && sub == 0) {
            const bool pos = y[i] > 0;
            z0[i] = pos ? acc[0] : -acc[0];
            if (NV == 2) z1[i] = pos ? acc[NV - 1] : -acc[NV - 1];
        }
    }
}

// ---------------------------------------------------------- A v, mixed (Dot2)

// FP32 X, q % 4 == 0.  A warp covers 32 consecutive rows in GL sub-steps of
// 32/GL rows (GL lanes per row), then transposes so that lane L holds row
// base + L: the FP64 epilogue and the z store are then one coalesced
// warp-wide instruction per 32 rows.
// NV vectors share each pass over X: vector k has its own labels y[k] (the
// batched solve runs problems that share X but not y) and output z[k].  Each
// vector's sums are formed in the same order whatever NV is, so a product is
// bit-identical whether it ran alone or in a batch.
// OUTDF: write y_i * (s + c) as a normalised double-float pair (float2)
// instead of FP64 (no FP64 instruction at all in that case).
template <int NV>
struct MvArgs {
    const double *v[NV];
    void *z[NV];
    const int8_t *y[NV];
};

template <int GL, int NV, bool OUTDF>
__global__ void __launch_bounds__(256) matvec_mx_kernel(const float *__restrict__ X, long long n, int q, MvArgs<NV> a)
{
    extern __shared__ float2 svf[];   // [NV][q] FP32 (hi, lo) split of v
    for (int j = threadIdx.x; j < q; j += blockDim.x) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            const double d = a.v[k][j];
            const float h = (float)d;
            svf[k * q + j] = make_float2(h, (float)(d - (double)h));
        }
    }
    __syncthreads();
    constexpr int RPW = 32 / GL;
    const int lane = threadIdx.x & 31;
    const int sub = lane % GL, grp = lane / GL;
    const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
    const long long wid = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int nv4 = q >> 2;
    for (long long base = wid * 32; base < n; base += nwarps * 32) {
        float rs[NV], rc[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) { rs[k] = 0.f; rc[k] = 0.f; }
#pragma unroll 1
        for (int kk = 0; kk < GL; ++kk) {
            const long long i = base + kk * RPW + grp;
            float s[NV], c[NV];
#pragma unroll
            for (int k = 0; k < NV; ++k) { s[k] = 0.f; c[k] = 0.f; }
            if (i < n) {
                const float4 *rv = reinterpret_cast<const float4 *>(X + i * (long long)q);
#pragma unroll 8
                for (int ch = sub; ch < nv4; ch += GL) {
                    const float4 x4 = __ldcs(rv + ch);
                    const float xs[4] = {x4.x, x4.y, x4.z, x4.w};
#pragma unroll
                    for (int e = 0; e < 4; ++e)
#pragma unroll
                        for (int k = 0; k < NV; ++k) dot2_step(xs[e], svf[k * q + ch * 4 + e], s[k], c[k]);
                }
            }
#pragma unroll
            for (int o = GL / 2; o > 0; o >>= 1)
#pragma unroll
                for (int k = 0; k < NV; ++k) {
                    const float s2 = __shfl_xor_sync(0xffffffffu, s[k], o);
                    const float c2 = __shfl_xor_sync(0xffffffffu, c[k], o);
                    df_acc(s[k], c[k], s2, c2);
                }
            const int src = (lane % RPW) * GL;
#pragma unroll
            for (int k = 0; k < NV; ++k) {
                const float ts = __shfl_sync(0xffffffffu, s[k], src);
                const float tc = __shfl_sync(0xffffffffu, c[k], src);
                if (lane / RPW == kk) { rs[k] = ts; rc[k] = tc; }
            }
        }
        const long long i = base + lane;
        if (i < n) {
#pragma unroll
            for (int k = 0; k < NV; ++k) {
                const bool pos = a.y[k][i] > 0;
                if (OUTDF) {
                    const float hi = rs[k] + rc[k];
                    float2 v = make_float2(hi, rc[k] - (hi - rs[k]));
                    if (!pos) { v.x = -v.x; v.y = -v.y; }
                    reinterpret_cast<float2 *>(a.z[k])[i] = v;
                } else {
                    const double d = (double)rs[k] + (double)rc[k];
                    reinterpret_cast<double *>(a.z[k])[i] = pos ? d : -d;
                }
            }
        }
    }
}

template <typename TX, bool VEC, int NV>
static cudaError_t matvec_dispatch(Work &W, const double *v0, double *z0, const double *v1, double *z1)
{
    constexpr int Wd = VEC ? Vec<TX>::W : 1;
    const int chunks = (int)((W.q + Wd - 1) / Wd);
    int gl = 1;
    while (gl < 32 && (chunks + gl - 1) / gl > 4) gl <<= 1;
    const int blocks = W.nsm * 8;
    const size_t smem = (size_t)NV * W.q * sizeof(double);
    const TX *X = (const TX *)W.X;
#define MV_CASE(G)                                                                                         \
    case G:                                                                                                \
        matvec_kernel<TX, G, VEC, NV><<<blocks, 256, smem, W.st>>>(X, W.y, W.n, (int)W.q, v0, v1, z0, z1); \
        break;
    switch (gl) {
        MV_CASE(1) MV_CASE(2) MV_CASE(4) MV_CASE(8) MV_CASE(16) MV_CASE(32)
    }
#undef MV_CASE
    ++W.nlaunch;
    return cudaGetLastError();
}

// GL (lanes per row) depends on q only, so every NV sums a vector in the same order.
static int mx_lanes(long long q)
{
    const int nv4 = (int)(q / 4);
    int gl = 1;
    while (gl < 32 && (nv4 + gl - 1) / gl > 8) gl <<= 1;
    return gl;
}

// Blocks of one launch: every SM full (nsm x resident blocks per SM), one
// wave, so no block waits for another to finish (measured on GB300 at
// n = 1e6, q = 128: 84.7 us per isolated launch against 88.1 us with 8
// blocks per SM, of which only 5 fit).  Rows are assigned to warps by a grid
// stride, and each row's sum has the same order whatever the grid.
template <int GL, int NV, bool OUTDF>
static int mx_blocks(int nsm, size_t smem)
{
    int v = 0;   // a host-side calculation from the kernel's attributes
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, matvec_mx_kernel<GL, NV, OUTDF>, 256, smem) != cudaSuccess ||
        v < 1)
        v = 8;
    return nsm * v;
}

template <int NV, bool OUTDF>
static cudaError_t matvec_mx_dispatch(const float *X, long long n, int q, int nsm, cudaStream_t st, const MvArgs<NV> &a)
{
    const int gl = mx_lanes(q);
    const size_t smem = (size_t)NV * q * sizeof(float2);
    if (smem > 48 * 1024) {
        // larger tiles of vectors (NV >= 8 at q > 384) need the opt-in shared memory
        static int attr_set[6] = {0, 0, 0, 0, 0, 0};
        static void *const kern[6] = {(void *)matvec_mx_kernel<1, NV, OUTDF>, (void *)matvec_mx_kernel<2, NV, OUTDF>,
                                      (void *)matvec_mx_kernel<4, NV, OUTDF>, (void *)matvec_mx_kernel<8, NV, OUTDF>,
                                      (void *)matvec_mx_kernel<16, NV, OUTDF>, (void *)matvec_mx_kernel<32, NV, OUTDF>};
        int li = 0;
        while ((1 << li) < gl) ++li;
        if (!attr_set[li]) {
            const cudaError_t e = cudaFuncSetAttribute(kern[li], cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
            if (e != cudaSuccess) return e;
            attr_set[li] = 1;
        }
    }
#define MX_CASE(G)                                                                                          \
    case G:                                                                                                 \
        matvec_mx_kernel<G, NV, OUTDF><<<mx_blocks<G, NV, OUTDF>(nsm, smem), 256, smem, st>>>(X, n, q, a); \
        break;
    switch (gl) {
        MX_CASE(1) MX_CASE(2) MX_CASE(4) MX_CASE(8) MX_CASE(16) MX_CASE(32)
    }
#undef MX_CASE
    return cudaGetLastError();
}

template <int NV, bool OUTDF>
static cudaError_t matvec_mx_one(Work &W, const double *v0, void *z0, const double *v1, void *z1)
{
    MvArgs<NV> a;
    a.v[0] = v0; a.z[0] = z0; a.y[0] = W.y;
    if (NV == 2) { a.v[NV - 1] = v1; a.z[NV - 1] = z1; a.y[NV - 1] = W.y; }
    ++W.nlaunch;
    return matvec_mx_dispatch<NV, OUTDF>((const float *)W.X, W.n, (int)W.q, W.nsm, W.st, a);
}

cudaError_t launch_matvec_df(Work &W, const double *v0, float2 *z0, const double *v1, float2 *z1)
{
    if (!(!W.csr && W.xf32 && W.q % 4 == 0 && (uintptr_t)W.X % 16 == 0)) return cudaErrorInvalidValue;
    return v1 ? matvec_mx_one<2, true>(W, v0, z0, v1, z1) : matvec_mx_one<1, true>(W, v0, z0, v1, z1);
}

template <int NV>
static cudaError_t multi_pass(const Work &W, const MvItem *it)
{
    MvArgs<NV> a;
    for (int k = 0; k < NV; ++k) { a.v[k] = it[k].v; a.z[k] = it[k].z; a.y[k] = it[k].y; }
    return matvec_mx_dispatch<NV, true>((const float *)W.X, W.n, (int)W.q, W.nsm, W.st, a);
}

cudaError_t launch_matvec_df_multi(Work &W, const MvItem *items, int count, int nv)
{
    if (!(!W.csr && W.xf32 && W.q % 4 == 0 && (uintptr_t)W.X % 16 == 0)) return cudaErrorInvalidValue;
    if (count < 1 || (nv != 1 && nv != 2 && nv != 4 && nv != 8) || count != nv) return cudaErrorInvalidValue;
    ++W.nlaunch;
    switch (nv) {
    case 1: return multi_pass<1>(W, items);
    case 2: return multi_pass<2>(W, items);
    case 4: return multi_pass<4>(W, items);
    default: return multi_pass<8>(W, items);
    }
}

cudaError_t launch_matvec(Work &W, const double *v0, double *z0, const double *v1, double *z1)
{
    if (W.csr) return launch_matvec_csr(W, v0, z0, v1, z1);
    const size_t es = W.xf32 ? 4 : 8;
    const bool vec = ((W.q * es) % 16 == 0) && ((uintptr_t)W.X % 16 == 0);
    const bool two = v1 != nullptr;
    if (W.xf32 && vec && W.precision == 1)
        return two ? matvec_mx_one<2, false>(W, v0, z0, v1, z1) : matvec_mx_one<1, false>(W, v0, z0, v1, z1);
    if (W.xf32) {
        if (vec) return two ? matvec_dispatch<float, true, 2>(W, v0, z0, v1, z1)
                            : matvec_dispatch<float, true, 1>(W, v0, z0, v1, z1);
        return two ? matvec_dispatch<float, false, 2>(W, v0, z0, v1, z1)
                   : matvec_dispatch<float, false, 1>(W, v0, z0, v1, z1);
    }
    if (vec) return two ? matvec_dispatch<double, true, 2>(W, v0, z0, v1, z1)
                        : matvec_dispatch<double, true, 1>(W, v0, z0, v1, z1);
    return two ? matvec_dispatch<double, false, 2>(W, v0, z0, v1, z1)
               : matvec_dispatch<double, false, 1>(W, v0, z0, v1, z1);
}

}  // namespace svm
