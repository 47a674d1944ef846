// k_rff.cu -- random Fourier features (Sec. 4.3), the front-end that turns an
// RBF-kernel C-SVC into the linear one this library solves:
//
//     Z[i][2j] = cos(<x_i, omega_j>) / sqrt(N),   Z[i][2j+1] = sin(<x_i, omega_j>) / sqrt(N),
//
// so that z(x)'z(y) = (1/N) sum_j cos(omega_j'(x - y)), whose expectation over
// omega ~ N(0, I/alpha) is exp(-|x - y|^2 / (2 alpha)) (Bochner's theorem).
//
// One kernel: the product T = X Omega (n x q times q x N, FP32 inputs, FP32
// products summed in k order) in 64 x 64 output tiles -- 16-deep slices of X
// (stored transposed) and Omega staged in shared memory, 4 x 4 outputs per
// thread -- with the cos/sin of each entry and the 1/sqrt(N) scale in the
// epilogue, written as interleaved (cos, sin) pairs.  The dot products are
// short (q is the data dimension) and the sincos is the costlier part, so the
// kernel stays on the FP32 pipes; tensor cores would round the phases to TF32.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "../../include/svm_ssnalm.h"
#include "common.cuh"

namespace {

constexpr int kRfTM = 64, kRfTN = 64, kRfTK = 16, kRfThreads = 256;

__global__ void __launch_bounds__(kRfThreads) rff_kernel(const float *__restrict__ X, long long n, int q,
                                                         const float *__restrict__ Om, int N, float scale,
                                                         float *__restrict__ Z)
{
    __shared__ float sX[kRfTK][kRfTM + 4];   // X slice, transposed: sX[k][row]
    __shared__ float sO[kRfTK][kRfTN + 4];   // Omega slice: sO[k][frequency]
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int c0 = blockIdx.x * kRfTN;
    for (long long r0 = (long long)blockIdx.y * kRfTM; r0 < n; r0 += (long long)gridDim.y * kRfTM) {
        float acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
        for (int k0 = 0; k0 < q; k0 += kRfTK) {
            for (int e = threadIdx.x; e < kRfTM * kRfTK; e += kRfThreads) {
                const int rr = e / kRfTK, kk = e - rr * kRfTK;
                const long long r = r0 + rr;
                const int k = k0 + kk;
                sX[kk][rr] = (r < n && k < q) ? X[r * q + k] : 0.f;
            }
            for (int e = threadIdx.x; e < kRfTK * kRfTN; e += kRfThreads) {
                const int kk = e / kRfTN, cc = e - kk * kRfTN;
                const int k = k0 + kk, c = c0 + cc;
                sO[kk][cc] = (k < q && c < N) ? Om[(size_t)k * N + c] : 0.f;
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < kRfTK; ++kk) {
                float a[4], b[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) a[i] = sX[kk][ty * 4 + i];
#pragma unroll
                for (int j = 0; j < 4; ++j) b[j] = sO[kk][tx * 4 + j];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
            }
            __syncthreads();
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const long long r = r0 + ty * 4 + i;
            if (r >= n) continue;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c = c0 + tx * 4 + j;
                if (c >= N) continue;
                float sv, cv;
                sincosf(acc[i][j], &sv, &cv);
                *reinterpret_cast<float2 *>(Z + r * (2LL * N) + 2LL * c) = make_float2(cv * scale, sv * scale);
            }
        }
    }
}

}  // namespace

extern "C" svm_status svm_rff_features(const float *X, int64_t n, int64_t q, const float *Omega, int64_t N, float *Z,
                                       void *stream)
{
    if (!X || !Omega || !Z || n < 1 || q < 1 || N < 1) return SVM_ERR_INVALID_ARG;
    if (q > 0x7fffffffLL || N > (1LL << 28) || (uintptr_t)Z % 8 != 0) return SVM_ERR_UNSUPPORTED;
    const long long tiles = (n + kRfTM - 1) / kRfTM;
    const dim3 grid((unsigned)((N + kRfTN - 1) / kRfTN), (unsigned)(tiles < 65535 ? tiles : 65535));
    rff_kernel<<<grid, kRfThreads, 0, (cudaStream_t)stream>>>(X, n, (int)q, Omega, (int)N,
                                                             (float)(1.0 / sqrt((double)N)), Z);
    return cudaGetLastError() == cudaSuccess ? SVM_OK : SVM_ERR_CUDA;
}
