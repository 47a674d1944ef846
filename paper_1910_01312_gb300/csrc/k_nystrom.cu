// k_nystrom.cu -- the Nystrom front-end of Sec. 4.3 (include/svm_nystrom.h):
// k-means landmarks (Lloyd's iterations), the kernel blocks K_nr and K_rr of
// k(x, y) = exp(-|x - y|^2 / (2 alpha)), the Cholesky factor L of K_rr + s I,
// its inverse, and the features Z = K_nr L^{-T} (so that Z Z' equals
// K_nr (K_rr + s I)^{-1} K_nr').
//
// Every distance, kernel value and factor is FP64 (X is FP32, widened
// exactly); sums run in fixed orders, so results are deterministic.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "../../include/svm_nystrom.h"
#include "common.cuh"

namespace svm {
namespace {

constexpr int kDR = 64;    // rows per distance tile
constexpr int kDC = 32;    // centres per distance tile
constexpr int kDK = 64;    // features per staged chunk
constexpr int kMaxR = 1024;

// Squared distances between a tile of 64 rows of X and the centres, in
// tiles of 32 centres: thread t owns row t/4 and centres t%4 + 4s (s < 8),
// accumulating (x_ik - c_jk)^2 over staged 64-feature chunks (padded rows
// avoid bank conflicts).  ASSIGN: per row the nearest centre (ties to the
// lowest index) into labels and its distance into dmin.  KERNEL: every
// exp(-d2 / (2 alpha)) into K (row-major, ldk = r).
template <bool ASSIGN>
__global__ void __launch_bounds__(256) dist_kernel(const float *__restrict__ X, long long n, int q,
                                                   const double *__restrict__ Cn, int r, double inv2a,
                                                   int32_t *__restrict__ labels, double *__restrict__ dmin,
                                                   double *__restrict__ K)
{
    __shared__ float Xs[kDR][kDK + 1];
    __shared__ double Cs[kDC][kDK + 1];
    const int tid = threadIdx.x;
    const int rr = tid >> 2, cs = tid & 3;
    const long long r0 = (long long)blockIdx.x * kDR;
    const long long i = r0 + rr;
    double best = INFINITY;
    int bestj = 0;
    for (int c0 = 0; c0 < r; c0 += kDC) {
        double acc[8];
#pragma unroll
        for (int s = 0; s < 8; ++s) acc[s] = 0.0;
        for (int k0 = 0; k0 < q; k0 += kDK) {
            for (int e = tid; e < kDR * kDK; e += 256) {
                const int a = e / kDK, b = e % kDK;
                const long long gi = r0 + a;
                Xs[a][b] = (gi < n && k0 + b < q) ? X[gi * q + k0 + b] : 0.f;
            }
            for (int e = tid; e < kDC * kDK; e += 256) {
                const int a = e / kDK, b = e % kDK;
                Cs[a][b] = (c0 + a < r && k0 + b < q) ? Cn[(long long)(c0 + a) * q + k0 + b] : 0.0;
            }
            __syncthreads();
            const int kk = (q - k0) < kDK ? (q - k0) : kDK;
            for (int k = 0; k < kk; ++k) {
                const double xv = (double)Xs[rr][k];
#pragma unroll
                for (int s = 0; s < 8; ++s) {
                    const double d = xv - Cs[cs + 4 * s][k];
                    acc[s] = fma(d, d, acc[s]);
                }
            }
            __syncthreads();
        }
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            const int j = c0 + cs + 4 * s;
            if (j < r && i < n) {
                if (ASSIGN) {
                    if (acc[s] < best) { best = acc[s]; bestj = j; }   // j grows: ties keep the lowest
                } else {
                    K[i * (long long)r + j] = exp(-acc[s] * inv2a);
                }
            }
        }
    }
    if (ASSIGN) {
        // the four threads of a row (adjacent lanes) agree on the smallest (d, j)
#pragma unroll
        for (int o = 1; o <= 2; o <<= 1) {
            const double ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oj = __shfl_xor_sync(0xffffffffu, bestj, o);
            if (ob < best || (ob == best && oj < bestj)) { best = ob; bestj = oj; }
        }
        if (cs == 0 && i < n) {
            labels[i] = bestj;
            dmin[i] = best;
        }
    }
}

// Centre j <- mean of the rows labelled j, summed in ascending row order (one
// block per centre: labels scanned in tiles, members compacted by warp
// ballots, each thread owning columns t, t + 256, ...); no rows: kept.
__global__ void __launch_bounds__(256) update_kernel(const float *__restrict__ X, long long n, int q,
                                                     const int32_t *__restrict__ labels, double *__restrict__ Cn)
{
    constexpr int kT = 1024;
    __shared__ int32_t mem[kT];
    __shared__ int wcnt[8];
    __shared__ int tot;
    const int j = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    long long cnt = 0;
    for (long long t0 = 0; t0 < n; t0 += kT) {
        int base = 0;
        for (int sub = 0; sub < kT; sub += 256) {
            const long long i = t0 + sub + tid;
            const bool m = i < n && labels[i] == j;
            const unsigned bal = __ballot_sync(0xffffffffu, m);
            if (lane == 0) wcnt[warp] = __popc(bal);
            __syncthreads();
            int pos = base;
            for (int w = 0; w < warp; ++w) pos += wcnt[w];
            if (m) mem[pos + __popc(bal & ((1u << lane) - 1u))] = (int32_t)i;
            int all = 0;
            for (int w = 0; w < 8; ++w) all += wcnt[w];
            base += all;
            __syncthreads();
        }
        if (tid == 0) tot = base;
        __syncthreads();
        for (int m = 0; m < tot; ++m) {
            const long long row = mem[m];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int col = tid + 256 * c;
                if (col < q) acc[c] += (double)X[row * q + col];
            }
        }
        cnt += tot;
        __syncthreads();
    }
    if (cnt > 0) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int col = tid + 256 * c;
            if (col < q) Cn[(long long)j * q + col] = acc[c] / (double)cnt;
        }
    }
}

// sum of dmin in a fixed order (one block)
__global__ void __launch_bounds__(1024) sum_kernel(const double *__restrict__ v, long long n, double *out)
{
    __shared__ double sh[32];
    double s = 0.0;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) s += v[i];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        *out = t;
    }
}

// K_rr + shift I (r x r), one thread per entry
__global__ void krr_kernel(const double *__restrict__ Cn, int r, int q, double inv2a, double shift,
                           double *__restrict__ M)
{
    const long long rr = (long long)r * r;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < rr; e += (long long)gridDim.x * blockDim.x) {
        const int a = (int)(e / r), b = (int)(e % r);
        double d2 = 0.0;
        for (int k = 0; k < q; ++k) {
            const double d = Cn[(long long)a * q + k] - Cn[(long long)b * q + k];
            d2 = fma(d, d, d2);
        }
        M[e] = exp(-d2 * inv2a) + (a == b ? shift : 0.0);
    }
}

// In-place lower Cholesky of M (r x r, one block); err on a non-positive pivot.
__global__ void __launch_bounds__(1024) chol_kernel(int r, double *__restrict__ M, int *err)
{
    __shared__ int bad;
    const int tid = threadIdx.x;
    if (tid == 0) bad = 0;
    __syncthreads();
    for (int j = 0; j < r; ++j) {
        if (tid == 0) {
            double d = M[(size_t)j * r + j];
            if (!(d > 0.0) || !isfinite(d)) { bad = 1; d = 1.0; }
            M[(size_t)j * r + j] = sqrt(d);
        }
        __syncthreads();
        const double djj = M[(size_t)j * r + j];
        for (int i = j + 1 + tid; i < r; i += blockDim.x) M[(size_t)i * r + j] /= djj;
        __syncthreads();
        const int wy = tid >> 5, wx = tid & 31, ny = blockDim.x >> 5;
        for (int i = j + 1 + wy; i < r; i += ny) {
            const double lij = M[(size_t)i * r + j];
            for (int k = j + 1 + wx; k <= i; k += 32) M[(size_t)i * r + k] -= lij * M[(size_t)k * r + j];
        }
        __syncthreads();
    }
    if (tid == 0 && bad) atomicExch(err, 1);
}

// Linv = L^{-1} (lower, r x r, row-major; the upper part is zeroed): warp w of
// the grid computes column j = w by forward substitution, L x = e_j, each
// step's dot product split over the 32 lanes (column stored as it is formed).
__global__ void __launch_bounds__(256) trinv_kernel(int r, const double *__restrict__ L, double *__restrict__ Li)
{
    const int lane = threadIdx.x & 31;
    const int j = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
    if (j >= r) return;   // whole warps leave together
    for (int k = lane; k < j; k += 32) Li[(size_t)k * r + j] = 0.0;
    for (int k = j; k < r; ++k) {
        double s = 0.0;
        for (int m = j + lane; m < k; m += 32) s = fma(L[(size_t)k * r + m], Li[(size_t)m * r + j], s);
        s = warp_sum(s);
        if (lane == 0) Li[(size_t)k * r + j] = ((k == j ? 1.0 : 0.0) - s) / L[(size_t)k * r + k];
        __syncwarp();
        __threadfence_block();
    }
}

// Z[i][j] = sum_{k <= j} K[i][k] Li[j][k] (FP64; 64 x 64 tiles, k in steps of
// 16, 4 x 4 outputs per thread), stored as T.
template <typename T>
__global__ void __launch_bounds__(256) zgemm_kernel(const double *__restrict__ K, long long nc, int r,
                                                    const double *__restrict__ Li, T *__restrict__ Z)
{
    __shared__ double As[16][64 + 1], Bs[16][64 + 1];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const long long i0 = (long long)blockIdx.y * 64;
    const int j0 = blockIdx.x * 64;
    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
    const int kend = (j0 + 64 < r) ? j0 + 64 : r;   // Li is lower triangular: k <= j < j0 + 64
    for (int k0 = 0; k0 < kend; k0 += 16) {
        for (int e = tid; e < 16 * 64; e += 256) {
            const int kk = e / 64, c = e % 64;
            const long long gi = i0 + c;
            const int gk = k0 + kk;
            As[kk][c] = (gi < nc && gk < r) ? K[gi * r + gk] : 0.0;
            const int gj = j0 + c;
            Bs[kk][c] = (gj < r && gk < r) ? Li[(size_t)gj * r + gk] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            double av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = As[kk][ty + 16 * a];
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = Bs[kk][tx + 16 * b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const long long gi = i0 + ty + 16 * a;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int gj = j0 + tx + 16 * b;
            if (gi < nc && gj < r) Z[gi * r + gj] = (T)acc[a][b];
        }
    }
}

svm_status cuda_status(cudaError_t e) { return e == cudaSuccess ? SVM_OK : SVM_ERR_CUDA; }

}  // namespace
}  // namespace svm

using namespace svm;

extern "C" svm_status svm_nystrom_kmeans(const float *X, int64_t n, int64_t q, double *centres, int64_t r,
                                         int32_t iters, int32_t *labels, double *objective, void *stream)
{
    if (!X || !centres || n < 1 || q < 1 || r < 1 || iters < 1) return SVM_ERR_INVALID_ARG;
    if (q > 1024 || r > kMaxR || n > 0x7fffffffLL) return SVM_ERR_UNSUPPORTED;
    cudaStream_t st = (cudaStream_t)stream;
    int32_t *lab = nullptr;
    double *dmin = nullptr, *obj = nullptr;
    if (cudaMallocAsync(&lab, sizeof(int32_t) * n, st) != cudaSuccess ||
        cudaMallocAsync(&dmin, sizeof(double) * n, st) != cudaSuccess ||
        cudaMallocAsync(&obj, sizeof(double) * iters, st) != cudaSuccess) {
        if (lab) cudaFreeAsync(lab, st);
        if (dmin) cudaFreeAsync(dmin, st);
        cudaStreamSynchronize(st);
        return SVM_ERR_OOM;
    }
    const unsigned gb = (unsigned)((n + kDR - 1) / kDR);
    for (int it = 0; it < iters; ++it) {
        dist_kernel<true><<<gb, 256, 0, st>>>(X, n, (int)q, centres, (int)r, 0.0, lab, dmin, nullptr);
        sum_kernel<<<1, 1024, 0, st>>>(dmin, n, obj + it);
        update_kernel<<<(unsigned)r, 256, 0, st>>>(X, n, (int)q, lab, centres);
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && labels) e = cudaMemcpyAsync(labels, lab, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && objective) e = cudaMemcpyAsync(objective, obj, sizeof(double) * iters, cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(lab, st);
    cudaFreeAsync(dmin, st);
    cudaFreeAsync(obj, st);
    const cudaError_t e2 = cudaStreamSynchronize(st);
    return cuda_status(e != cudaSuccess ? e : e2);
}

extern "C" svm_status svm_nystrom_features(const float *X, int64_t n, int64_t q, const double *centres, int64_t r,
                                           double alpha, double shift, void *Z, int32_t z_dtype, void *stream)
{
    if (!X || !centres || !Z || n < 1 || q < 1 || r < 1) return SVM_ERR_INVALID_ARG;
    if (!(alpha > 0.0) || !isfinite(alpha) || !(shift >= 0.0) || !isfinite(shift)) return SVM_ERR_INVALID_ARG;
    if (z_dtype != SVM_F32 && z_dtype != SVM_F64) return SVM_ERR_INVALID_ARG;
    if (q > 1024 || r > kMaxR || n > 0x7fffffffLL) return SVM_ERR_UNSUPPORTED;
    if ((uintptr_t)Z % 16 != 0) return SVM_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const long long chunk = n < 32768 ? n : 32768;   // rows of K_nr held at a time
    double *M = nullptr, *Li = nullptr, *K = nullptr;
    int *err = nullptr;
    if (cudaMallocAsync(&M, sizeof(double) * r * r, st) != cudaSuccess ||
        cudaMallocAsync(&Li, sizeof(double) * r * r, st) != cudaSuccess ||
        cudaMallocAsync(&K, sizeof(double) * chunk * r, st) != cudaSuccess ||
        cudaMallocAsync(&err, sizeof(int), st) != cudaSuccess) {
        if (M) cudaFreeAsync(M, st);
        if (Li) cudaFreeAsync(Li, st);
        if (K) cudaFreeAsync(K, st);
        cudaStreamSynchronize(st);
        return SVM_ERR_OOM;
    }
    const double inv2a = 1.0 / (2.0 * alpha);
    cudaMemsetAsync(err, 0, sizeof(int), st);
    krr_kernel<<<256, 256, 0, st>>>(centres, (int)r, (int)q, inv2a, shift, M);
    chol_kernel<<<1, 1024, 0, st>>>((int)r, M, err);
    trinv_kernel<<<(unsigned)((r * 32 + 255) / 256), 256, 0, st>>>((int)r, M, Li);
    for (long long c0 = 0; c0 < n; c0 += chunk) {
        const long long nc = (n - c0) < chunk ? (n - c0) : chunk;
        dist_kernel<false><<<(unsigned)((nc + kDR - 1) / kDR), 256, 0, st>>>(X + c0 * q, nc, (int)q, centres, (int)r,
                                                                             inv2a, nullptr, nullptr, K);
        dim3 grid((unsigned)((r + 63) / 64), (unsigned)((nc + 63) / 64));
        if (z_dtype == SVM_F32)
            zgemm_kernel<float><<<grid, 256, 0, st>>>(K, nc, (int)r, Li, static_cast<float *>(Z) + c0 * r);
        else
            zgemm_kernel<double><<<grid, 256, 0, st>>>(K, nc, (int)r, Li, static_cast<double *>(Z) + c0 * r);
    }
    cudaError_t e = cudaGetLastError();
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(M, st);
    cudaFreeAsync(Li, st);
    cudaFreeAsync(K, st);
    cudaFreeAsync(err, st);
    const cudaError_t e2 = cudaStreamSynchronize(st);
    if (e != cudaSuccess || e2 != cudaSuccess) return SVM_ERR_CUDA;
    return herr ? SVM_ERR_NUMERIC : SVM_OK;
}
