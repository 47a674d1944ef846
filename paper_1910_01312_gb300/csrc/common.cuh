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
__device__ __forceinline__ bool grid_barrier(unsigned *bar, int *err)
{
    __syncthreads();
    __shared__ int ok_sh;
    if (threadIdx.x == 0) {
        int ok = 1;
        unsigned add = (blockIdx.x == 0) ? (0x80000000u - (gridDim.x - 1u)) : 1u;
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
