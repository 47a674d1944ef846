// common.cuh -- device helpers shared by the solver's kernels (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#ifndef SVM_TPB
#define SVM_TPB 512
#endif

namespace svm {

constexpr int kTPB = SVM_TPB;          // threads per block of the vector kernels
constexpr int kWarps = kTPB / 32;

// Device error codes written to Workspace::err (first error wins).
enum DevErr : int { DEV_OK = 0, DEV_TIMEOUT = 1, DEV_ROOT = 2, DEV_CHOL = 3, DEV_NAN = 4 };

__device__ __forceinline__ void set_err(int *err, int code)
{
    atomicCAS(err, 0, code);
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_relaxed_i32(const int *p)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier for kernels launched cooperatively (all blocks resident).
// Sense reversal on the top bit of one counter: block 0 adds 2^31 - (G-1),
// the others add 1, so after every barrier the low 31 bits are unchanged and
// the counter needs no reset between launches.  The wait is bounded: after
// 2^24 polls (seconds) it records DEV_TIMEOUT and returns false instead of spinning on.
// Every block executes the same sequence of barriers.
// The same barrier over a group of G blocks of one cooperative launch (b = this
// block's rank in the group, bar = the group's own counter).
__device__ __forceinline__ bool group_barrier(unsigned *bar, int *err, int b, int G)
{
    __syncthreads();
    __shared__ int ok_sh;
    if (threadIdx.x == 0) {
        int ok = 1;
        unsigned add = (b == 0) ? (0x80000000u - ((unsigned)G - 1u)) : 1u;
        __threadfence();
        unsigned old = atomicAdd(bar, add);
        // poll without sleeping: a sleep here is far coarser than the wait itself;
        // each acquire load is an L2 round trip, so the poll rate is self-limited
        unsigned spins = 0;
        while (((old ^ ld_acquire_u32(bar)) & 0x80000000u) == 0u) {
            if (((++spins) & 255u) == 0u && (ld_relaxed_i32(err) == DEV_TIMEOUT || spins > (1u << 24))) {
                set_err(err, DEV_TIMEOUT);
                ok = 0;
                break;
            }
        }
        __threadfence();
        ok_sh = ok;
    }
    __syncthreads();
    return ok_sh != 0;
}

__device__ __forceinline__ bool grid_barrier(unsigned *bar, int *err)
{
    return group_barrier(bar, err, (int)blockIdx.x, (int)gridDim.x);
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sumf(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ long long warp_sum_ll(long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double warp_min(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// ---------------------------------------------------------------------------
// Double-float ("float-float") arithmetic: a value is hi + lo with |lo| <=
// ulp(hi)/2, both FP32.  Built only from the error-free transformations
// TwoSum (Knuth) and TwoProd via fused multiply-add (Ogita, Rump, Oishi,
// "Accurate sum and dot product", SIAM J. Sci. Comput. 26(6), 2005), so the
// accumulations run on the FP32 pipes, which on this part are ~64x the FP64
// rate.  Relative accuracy ~2^-44 per operation.
struct df {
    float hi, lo;
};

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e)
{
    p = a * b;
    e = fmaf(a, b, -p);
}
// hi/lo split of a double
__device__ __forceinline__ df df_from_double(double x)
{
    df r;
    r.hi = (float)x;
    r.lo = (float)(x - (double)r.hi);
    return r;
}
__device__ __forceinline__ double df_to_double(df a)
{
    return (double)a.hi + (double)a.lo;
}
__device__ __forceinline__ df df_add(df a, df b)
{
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e += a.lo + b.lo;
    df r;
    r.hi = s + e;
    r.lo = e - (r.hi - s);
    return r;
}

// ---------------------------------------------------------------------------
// Double-float values as float2 (x = hi, y = lo, normalised: |lo| <= ulp(hi)/2,
// so the sign and the order are decided by hi first).  Addition is the
// accurate form with two TwoSums (Hida, Li, Bailey, "Algorithms for
// quad-double precision floating point arithmetic", ARITH-15, 2001), which
// stays accurate under cancellation; products use TwoProd via FMA.
__device__ __forceinline__ float2 dfx_fast(float s, float e)   // requires |s| >= |e| or s == 0
{
    const float hi = s + e;
    return make_float2(hi, e - (hi - s));
}
__device__ __forceinline__ float2 dfx_add(float2 a, float2 b)
{
    float s, e, t, f;
    two_sum(a.x, b.x, s, e);
    two_sum(a.y, b.y, t, f);
    e += t;
    float2 r = dfx_fast(s, e);
    r.y += f;
    return dfx_fast(r.x, r.y);
}
__device__ __forceinline__ float2 dfx_neg(float2 a)
{
    return make_float2(-a.x, -a.y);
}
__device__ __forceinline__ float2 dfx_sub(float2 a, float2 b)
{
    return dfx_add(a, dfx_neg(b));
}
__device__ __forceinline__ float2 dfx_addf(float2 a, float b)
{
    float s, e;
    two_sum(a.x, b, s, e);
    e += a.y;
    return dfx_fast(s, e);
}
__device__ __forceinline__ float2 dfx_mul(float2 a, float2 b)
{
    float p, e;
    two_prod(a.x, b.x, p, e);
    e = fmaf(a.x, b.y, fmaf(a.y, b.x, e));
    return dfx_fast(p, e);
}
// an integer (|v| < 2^47) as an exact double-float
__device__ __forceinline__ float2 dfx_from_ll(long long v)
{
    const float hi = (float)v;
    return make_float2(hi, (float)(v - (long long)hi));
}
// a / b for b > 0: one correction step on the FP32 quotient (Dekker,
// "A floating-point technique for extending the available precision",
// Numer. Math. 18, 1971): q1 = a/b, r = a - q1 b exactly enough, q2 = r/b.
__device__ __forceinline__ float2 dfx_div(float2 a, float2 b)
{
    const float q1 = a.x / b.x;
    const float2 r = dfx_sub(a, dfx_mul(make_float2(q1, 0.f), b));
    const float q2 = r.x / b.x;
    return dfx_fast(q1, q2);
}
__device__ __forceinline__ bool dfx_gt(float2 a, float2 b)
{
    return a.x > b.x || (a.x == b.x && a.y > b.y);
}
__device__ __forceinline__ bool dfx_same(float2 a, float2 b)   // bitwise equality
{
    return __float_as_uint(a.x) == __float_as_uint(b.x) && __float_as_uint(a.y) == __float_as_uint(b.y);
}
__device__ __forceinline__ float2 shfl_xor_f2(float2 v, int o)
{
    return make_float2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o));
}

// ---------------------------------------------------------------------------
// Shared by the product kernels.
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

// One Dot2 step: (s, c) += x * (w.x + w.y), x exact FP32.
__device__ __forceinline__ void dot2_step(float x, float2 w, float &s, float &c)
{
    float p, e, sn, t;
    two_prod(x, w.x, p, e);
    two_sum(s, p, sn, t);
    s = sn;
    c = fmaf(x, w.y, c + (t + e));
}

// (s, c) += (s2, c2) for double-float pairs.
__device__ __forceinline__ void df_acc(float &s, float &c, float s2, float c2)
{
    float sn, e;
    two_sum(s, s2, sn, e);
    e += c + c2;
    s = sn + e;
    c = e - (s - sn);
}

}  // namespace svm

namespace svm {
// ---------------------------------------------------------------------------
// Bulk asynchronous copies (cp.async.bulk, the 1-D TMA path) and mbarriers.
__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// The CG's residual target for M dv = -g (|g| = gn): Algorithm 3's bound
// min(eta, |g|^{1+tau}), tightened to max(1e-10 |g|, floor) -- floor a
// fraction of the level at which the subproblem stops (0 at the step-level
// entry point: the step as exact as a direct solve) -- and never below
// 1e-14 |g|.
__device__ __forceinline__ float cg_tol(float gn, float eta, float tau, float floor)
{
    return fmaxf(fminf(fminf(eta, powf(gn, 1.f + tau)), fmaxf(1e-10f * gn, floor)), 1e-14f * gn);
}

__device__ __forceinline__ void mbar_arrive(unsigned long long *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// global -> shared bulk copy completing on bar; dst, src 16-byte aligned, bytes % 16 == 0
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait on a phase of bar: false (and DEV_TIMEOUT recorded) after ~1 s.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *bar, unsigned parity, int *err)
{
    for (unsigned it = 0; it < (1u << 22); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 1023u) == 1023u) {
            if (ld_relaxed_i32(err) == DEV_TIMEOUT) break;
            __nanosleep(64);
        }
    }
    set_err(err, DEV_TIMEOUT);
    return false;
}
}  // namespace svm
