// k_noalloc.cu -- the transposed product out = A'c for callers that must not
// allocate memory.
//
// Who needs this: code that runs where cudaMalloc is not an option -- inside a
// framework that owns all device memory through its own pool (a raw
// cudaMalloc would bypass its accounting and can implicitly synchronise the
// device), in latency-critical loops where an allocation's synchronisation or
// failure is unacceptable, or on callers with a fixed memory budget set up
// ahead of time.  Such callers cannot create a solver handle (the handle owns
// a workspace), so this entry point takes only the caller's inputs and
// outputs and keeps its scratch -- the per-block partial sums and the
// last-block counter -- in one fixed-size array in device global memory that
// every GPU loading the library holds until the process exits.
//
// Arithmetic: the same Dot2 scheme as the mixed-form product of k_matvec.cu
// (FP32 products made exact with TwoProd, sums carried as FP32 hi/lo pairs),
// with the FP64 weights y_i c_i split per row inside the kernel, and the same
// fixed-order two-stage reduction (block partials, then the last block to
// finish adds them in block order).
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/svm_ssnalm.h"
#include "common.cuh"

namespace {

constexpr int kNoAllocMaxQ = 1024;      // largest q accepted
constexpr int kNoAllocMaxBlocks = 160;  // largest grid (one block per SM on this part)
constexpr int kNoAllocThreads = 256;
// [0, 256): last-block counter; then kNoAllocMaxBlocks x kNoAllocMaxQ FP64 partials
constexpr size_t kScratchHeader = 256;
constexpr size_t kScratchBytes = kScratchHeader + sizeof(double) * (size_t)kNoAllocMaxBlocks * kNoAllocMaxQ;

// The scratch.  Host code must not use this name as an address: it is only a
// host-side stand-in for the device symbol; the device address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

__device__ __forceinline__ void na_dot2(float x, float2 w, float &s, float &c)
{
    float p, e, sn, t;
    svm::two_prod(x, w.x, p, e);
    svm::two_sum(s, p, sn, t);
    s = sn;
    c = fmaf(x, w.y, c + (t + e));
}

__device__ __forceinline__ void na_dfacc(float &s, float &c, float s2, float c2)
{
    float sn, e;
    svm::two_sum(s, s2, sn, e);
    e += c + c2;
    s = sn + e;
    c = e - (s - sn);
}

// Lane l owns the scalar columns l + 32k (k < NCH).  A warp takes 32-row
// chunks of its block's row range: each lane loads and splits one row's
// weight, then the rows are streamed with shuffles.
template <int NCH>
__global__ void __launch_bounds__(kNoAllocThreads) rmatvec_noalloc_kernel(const float *__restrict__ X,
                                                                          const int8_t *__restrict__ y, long long n,
                                                                          int q, const double *__restrict__ c,
                                                                          double *__restrict__ out,
                                                                          unsigned char *__restrict__ scratch)
{
    unsigned *counter = reinterpret_cast<unsigned *>(scratch);
    double *part = reinterpret_cast<double *>(scratch + kScratchHeader);
    const int G = gridDim.x;
    const long long per = (n + G - 1) / G;
    const long long r_beg = (long long)blockIdx.x * per;
    const long long r_end = r_beg + per < n ? r_beg + per : n;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    float s[NCH], cc[NCH];
#pragma unroll
    for (int k = 0; k < NCH; ++k) { s[k] = 0.f; cc[k] = 0.f; }
    for (long long c0 = r_beg + (long long)warp * 32; c0 < r_end; c0 += (long long)nw * 32) {
        const long long rl = c0 + lane;
        float2 myw = make_float2(0.f, 0.f);
        if (rl < r_end) {
            const double v = (y[rl] > 0) ? c[rl] : -c[rl];
            const float hi = (float)v;
            myw = make_float2(hi, (float)(v - (double)hi));
        }
        const int here = (int)((r_end - c0) < 32 ? (r_end - c0) : 32);
        for (int u = 0; u < here; ++u) {
            const float2 w = make_float2(__shfl_sync(0xffffffffu, myw.x, u), __shfl_sync(0xffffffffu, myw.y, u));
            if (w.x == 0.f && w.y == 0.f) continue;   // warp-uniform
            const float *row = X + (c0 + u) * (long long)q;
#pragma unroll
            for (int k = 0; k < NCH; ++k) {
                const int j = lane + 32 * k;
                if (j < q) na_dot2(__ldcs(row + j), w, s[k], cc[k]);
            }
        }
    }
    // warps of the block combined in order through shared memory
    extern __shared__ float sbuf[];   // [nw][2][q]
#pragma unroll
    for (int k = 0; k < NCH; ++k) {
        const int j = lane + 32 * k;
        if (j < q) {
            sbuf[(size_t)warp * 2 * q + j] = s[k];
            sbuf[(size_t)warp * 2 * q + q + j] = cc[k];
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < q; j += blockDim.x) {
        float ss = 0.f, sc = 0.f;
        for (int wv = 0; wv < nw; ++wv) na_dfacc(ss, sc, sbuf[(size_t)wv * 2 * q + j], sbuf[(size_t)wv * 2 * q + q + j]);
        part[(size_t)blockIdx.x * q + j] = (double)ss + (double)sc;
    }
    __threadfence();
    __syncthreads();
    __shared__ int is_last;
    if (threadIdx.x == 0) is_last = (atomicAdd(counter, 1u) == (unsigned)(G - 1));
    __syncthreads();
    if (is_last) {
        __threadfence();
        for (int j = threadIdx.x; j < q; j += blockDim.x) {
            double t = 0.0;
            for (int b = 0; b < G; ++b) t += __ldcg(part + (size_t)b * q + j);
            out[j] = t;
        }
        if (threadIdx.x == 0) *counter = 0u;   // leave the counter at zero for the next call
    }
}

std::mutex g_mu;
constexpr int kMaxDevices = 64;
void *g_scratch_ptr[kMaxDevices] = {};
int g_nsm[kMaxDevices] = {};

}  // namespace

// Set-up is done by the first call on each device (with that device current):
// it looks up the device address of the scratch array once and caches it.
extern "C" svm_status svm_rmatvec_noalloc(const float *X, const int8_t *y, int64_t n, int64_t q, const double *c,
                                          double *out, void *stream)
{
    if (!X || !y || !c || !out || n < 1 || q < 1) return SVM_ERR_INVALID_ARG;
    if (q > kNoAllocMaxQ || n > 0x7fffffffLL) return SVM_ERR_UNSUPPORTED;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SVM_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return SVM_ERR_UNSUPPORTED;
    if (stream) {
        // the scratch address and the SM count below are the current device's:
        // a stream of another device would run the kernel on memory it cannot use
        int sdev = -1;
        if (cudaStreamGetDevice((cudaStream_t)stream, &sdev) != cudaSuccess) return SVM_ERR_CUDA;
        if (sdev != dev) return SVM_ERR_INVALID_ARG;
    }
    void *scr = nullptr;
    int nsm = 0;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_scratch_ptr[dev]) {
            void *p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) return SVM_ERR_CUDA;
            int m = 0;
            if (cudaDeviceGetAttribute(&m, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return SVM_ERR_CUDA;
            // dynamic shared memory above 48 KB (q > 768) needs the opt-in
            const void *fns[] = {(const void *)rmatvec_noalloc_kernel<1>, (const void *)rmatvec_noalloc_kernel<2>,
                                 (const void *)rmatvec_noalloc_kernel<4>, (const void *)rmatvec_noalloc_kernel<8>,
                                 (const void *)rmatvec_noalloc_kernel<16>, (const void *)rmatvec_noalloc_kernel<32>};
            for (const void *f : fns)
                if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (kNoAllocThreads / 32) * 2 * kNoAllocMaxQ * (int)sizeof(float)) != cudaSuccess)
                    return SVM_ERR_CUDA;
            g_nsm[dev] = m;
            g_scratch_ptr[dev] = p;
        }
        scr = g_scratch_ptr[dev];
        nsm = g_nsm[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int G = nsm < kNoAllocMaxBlocks ? (nsm > 0 ? nsm : 1) : kNoAllocMaxBlocks;
    // the counter must start at zero (a previous launch that did not finish could have left it set)
    if (cudaMemsetAsync(scr, 0, sizeof(unsigned), st) != cudaSuccess) return SVM_ERR_CUDA;
    const size_t smem = (size_t)(kNoAllocThreads / 32) * 2 * (size_t)q * sizeof(float);
    unsigned char *sp = static_cast<unsigned char *>(scr);
    const int nch = (int)((q + 31) / 32);
#define NA_CASE(K)                                                                                          \
    if (nch <= K) {                                                                                         \
        rmatvec_noalloc_kernel<K><<<G, kNoAllocThreads, smem, st>>>(X, y, (long long)n, (int)q, c, out, sp); \
    } else
    NA_CASE(1) NA_CASE(2) NA_CASE(4) NA_CASE(8) NA_CASE(16) NA_CASE(32) { return SVM_ERR_UNSUPPORTED; }
#undef NA_CASE
    return cudaGetLastError() == cudaSuccess ? SVM_OK : SVM_ERR_CUDA;
}
