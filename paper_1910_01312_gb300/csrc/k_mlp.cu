// k_mlp.cu -- the learned warm start (include/svm_mlp.h): features, the
// 132-256-256-3 network's forward and backward passes, the class-weighted
// cross-entropy, Adam and the start point alpha^0, as hand-written FP32
// kernels.  Every reduction has a fixed order (deterministic results).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <new>

#include "../../include/svm_mlp.h"
#include "common.cuh"

using namespace svm;

namespace {

constexpr int kIn = SVM_MLP_IN, kH = SVM_MLP_HIDDEN, kOut = SVM_MLP_OUT;
constexpr int oW1 = 0, ob1 = oW1 + kIn * kH, oW2 = ob1 + kH, ob2 = oW2 + kH * kH, oW3 = ob2 + kH,
              ob3 = oW3 + kH * kOut, kNParam = ob3 + kOut;
static_assert(kNParam == SVM_MLP_NPARAM, "parameter layout");
constexpr int kQ = 128;   // feature rows are q + 4 = 132 wide

__device__ __forceinline__ float gelu(float z)
{
    return 0.5f * z * (1.f + erff(z * 0.70710678118654752f));
}
__device__ __forceinline__ float gelu_prime(float z)
{
    return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

// ------------------------------------------------------------------- GEMM
// C[m][n] = sum_k opA(m, k) opB(k, n), opA(m, k) = A[k][m] if TA else A[m][k],
// opB(k, n) = B[n][k] if TB else B[k][n] (row-major operands), 64 x 64 tiles,
// 16-deep k steps, 4 x 4 outputs per thread, then the epilogue.  Split K:
// block z takes k in [z kc, (z + 1) kc) and writes its partial product to
// C + z cstride; with bsum set, blocks of the first tile row also write the
// column sums of opB over their k range to bsum + z cstride (the bias
// gradient of a layer whose weight gradient is A' B).
enum Epi : int { EPI_PLAIN = 0, EPI_BIAS = 1, EPI_BIAS_GELU = 2, EPI_GELU_BWD = 3 };

template <bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(256) gemm_kernel(int M, int N, int K, int kc, const float *__restrict__ A, int lda,
                                                   const float *__restrict__ B, int ldb, float *__restrict__ C,
                                                   int ldc, size_t cstride, float *__restrict__ bsum,
                                                   const float *__restrict__ bias, float *__restrict__ Zout,
                                                   const float *__restrict__ Zin)
{
    __shared__ __align__(16) float As[16][68], Bs[16][68];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int bm = blockIdx.y * 64, bn = blockIdx.x * 64;
    const int kb0 = blockIdx.z * kc, kb1 = kb0 + kc < K ? kb0 + kc : K;
    const bool colsum = bsum != nullptr && blockIdx.y == 0 && ty == 0;
    float acc[4][4], cs[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int k0 = kb0; k0 < kb1; k0 += 16) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int e = tid + 256 * u;
            int m, k;
            if (TA) { m = e & 63; k = e >> 6; }
            else { m = e >> 4; k = e & 15; }
            float v = 0.f;
            if (bm + m < M && k0 + k < kb1)
                v = TA ? A[(size_t)(k0 + k) * lda + bm + m] : A[(size_t)(bm + m) * lda + k0 + k];
            As[k][m] = v;
            int n, kb;
            if (TB) { n = e >> 4; kb = e & 15; }
            else { n = e & 63; kb = e >> 6; }
            float w = 0.f;
            if (bn + n < N && k0 + kb < kb1)
                w = TB ? B[(size_t)(bn + n) * ldb + k0 + kb] : B[(size_t)(k0 + kb) * ldb + bn + n];
            Bs[kb][n] = w;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            const float4 a = *reinterpret_cast<const float4 *>(&As[kk][ty * 4]);
            const float4 b = *reinterpret_cast<const float4 *>(&Bs[kk][tx * 4]);
            const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
            if (colsum) {
#pragma unroll
                for (int j = 0; j < 4; ++j) cs[j] += bv[j];
            }
        }
        __syncthreads();
    }
    C += blockIdx.z * cstride;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = bm + ty * 4 + i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = bn + tx * 4 + j;
            if (n >= N) continue;
            const size_t o = (size_t)m * ldc + n;
            const float v = acc[i][j];
            if (EPI == EPI_PLAIN) C[o] = v;
            else if (EPI == EPI_BIAS) C[o] = v + bias[n];
            else if (EPI == EPI_BIAS_GELU) { const float z = v + bias[n]; Zout[o] = z; C[o] = gelu(z); }
            else C[o] = v * gelu_prime(Zin[o]);
        }
    }
    if (colsum) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = bn + tx * 4 + j;
            if (n < N) bsum[blockIdx.z * cstride + n] = cs[j];
        }
    }
}

template <bool TA, bool TB, int EPI>
cudaError_t gemm(cudaStream_t st, int M, int N, int K, const float *A, int lda, const float *B, int ldb, float *C,
                 int ldc, const float *bias = nullptr, float *Zout = nullptr, const float *Zin = nullptr)
{
    dim3 grid((N + 63) / 64, (M + 63) / 64, 1);
    gemm_kernel<TA, TB, EPI><<<grid, 256, 0, st>>>(M, N, K, K, A, lda, B, ldb, C, ldc, 0, nullptr, bias, Zout, Zin);
    return cudaGetLastError();
}

// out[i] = sum_z part[z stride + i], z in order
__global__ void splitk_reduce_kernel(int S, int count, size_t stride, const float *__restrict__ part,
                                     float *__restrict__ out)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int z = 0; z < S; ++z) s += part[z * stride + i];
        out[i] = s;
    }
}

constexpr int kMaxSplit = 64;

// Weight and bias gradient of one layer, G = A' D (M x N) and g = column sums of
// D (N), into out[0 .. M N) and out[M N .. M N + N) (the parameter layout keeps
// a layer's bias right after its weights).  Deterministic: the split count
// depends on the sizes only and the partials are added in order.
cudaError_t weight_grad(cudaStream_t st, int M, int N, int K, const float *A, int lda, const float *D, float *part,
                        float *out)
{
    const int tiles = ((M + 63) / 64) * ((N + 63) / 64);
    int S = (304 + tiles - 1) / tiles;
    if (S > kMaxSplit) S = kMaxSplit;
    const int smax = (K + 127) / 128;
    if (S > smax) S = smax;
    if (S < 1) S = 1;
    int kc = (K + S - 1) / S;
    kc = (kc + 15) / 16 * 16;
    S = (K + kc - 1) / kc;
    const size_t stride = (size_t)M * N + N;
    dim3 grid((N + 63) / 64, (M + 63) / 64, S);
    gemm_kernel<true, false, EPI_PLAIN><<<grid, 256, 0, st>>>(M, N, K, kc, A, lda, D, N, part, N, stride,
                                                              part + (size_t)M * N, nullptr, nullptr, nullptr);
    const int count = M * N + N;
    splitk_reduce_kernel<<<(count + 255) / 256, 256, 0, st>>>(S, count, stride, part, out);
    return cudaGetLastError();
}

// ------------------------------------------------------------ small kernels
// softmax cross-entropy: D3 = cw[l] (p - onehot(l)) / n, loss = (1/n) sum cw[l] (lse - z_l);
// block partials, the last block to finish adds them in block order
__global__ void __launch_bounds__(256) ce_kernel(int n, const float *__restrict__ Z3, const int32_t *__restrict__ lab,
                                                 const float *__restrict__ cw, float *__restrict__ D3,
                                                 float *__restrict__ part, unsigned *__restrict__ counter,
                                                 float *__restrict__ loss)
{
    __shared__ float sh[8];
    __shared__ int is_last;
    float acc = 0.f;
    const float rn = 1.f / (float)n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float z0 = Z3[3 * i], z1 = Z3[3 * i + 1], z2 = Z3[3 * i + 2];
        const float mx = fmaxf(z0, fmaxf(z1, z2));
        const float e0 = expf(z0 - mx), e1 = expf(z1 - mx), e2 = expf(z2 - mx);
        const float s = e0 + e1 + e2, rs = 1.f / s;
        const int l = lab[i];
        const float w = cw[l];
        const float zl = l == 0 ? z0 : (l == 1 ? z1 : z2);
        acc += w * (logf(s) + mx - zl);
        const float f = w * rn;
        D3[3 * i] = f * (e0 * rs - (l == 0 ? 1.f : 0.f));
        D3[3 * i + 1] = f * (e1 * rs - (l == 1 ? 1.f : 0.f));
        D3[3 * i + 2] = f * (e2 * rs - (l == 2 ? 1.f : 0.f));
    }
    acc = warp_sumf(acc);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < 8; ++w) t += sh[w];
        part[blockIdx.x] = t;
        __threadfence();
        is_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (is_last && threadIdx.x == 0) {
        __threadfence();
        float t = 0.f;
        for (int b = 0; b < (int)gridDim.x; ++b) t += __ldcg(&part[b]);
        *loss = t * rn;
        *counter = 0u;
    }
}

__global__ void adam_kernel(int np, float *__restrict__ th, float *__restrict__ m, float *__restrict__ v,
                            const float *__restrict__ g, float lr, float wd, float c1, float c2)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = 0.9f * m[i] + 0.1f * gi;
        const float vi = 0.999f * v[i] + 0.001f * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float t = th[i];
        th[i] = t - lr * ((mi / c1) / (sqrtf(vi / c2) + 1e-8f) + wd * t);
    }
}

__global__ void start_kernel(int n, const float *__restrict__ Z3, double C, double *__restrict__ a0)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float z0 = Z3[3 * i], z1 = Z3[3 * i + 1], z2 = Z3[3 * i + 2];
        const int c = (z1 > z0 && z1 >= z2) ? 1 : ((z2 > z0) ? 2 : 0);   // argmax, first maximum on ties
        a0[i] = c == 0 ? 0.0 : (c == 1 ? 0.5 * C : C);
    }
}

__global__ void labels_kernel(long long n, const double *__restrict__ a, double C, int32_t *__restrict__ lab)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double v = a[i];
        lab[i] = v <= 0.0 ? 0 : (v >= C ? 2 : 1);
    }
}

// a warp per gathered row: 33 float4 of features and the label
__global__ void gather_kernel(const float *__restrict__ F, const int32_t *__restrict__ lab,
                              const int64_t *__restrict__ idx, long long nb, float *__restrict__ Fb,
                              int32_t *__restrict__ Lb)
{
    const int lane = threadIdx.x & 31;
    const long long w0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long r = w0; r < nb; r += nw) {
        const long long i = idx[r];
        const float4 *src = reinterpret_cast<const float4 *>(F + i * kIn);
        float4 *dst = reinterpret_cast<float4 *>(Fb + r * kIn);
        dst[lane] = src[lane];
        if (lane == 0) { dst[32] = src[32]; Lb[r] = lab[i]; }
    }
}

// class sums of the rows (y = +1 and y = -1) as block partials: part[b][0..q) and [q..2q), counts
__global__ void __launch_bounds__(kQ) class_sum_kernel(const float *__restrict__ X, const int8_t *__restrict__ y,
                                                       long long n, double *__restrict__ part,
                                                       long long *__restrict__ cnt)
{
    const int j = threadIdx.x;
    double sp = 0.0, sm = 0.0;
    long long np_ = 0, nm = 0;
    const long long per = (n + gridDim.x - 1) / gridDim.x, r0 = blockIdx.x * per, r1 = r0 + per < n ? r0 + per : n;
    for (long long r = r0; r < r1; ++r) {
        const float x = X[r * kQ + j];
        if (y[r] > 0) { sp += x; ++np_; } else { sm += x; ++nm; }
    }
    part[(size_t)blockIdx.x * 2 * kQ + j] = sp;
    part[(size_t)blockIdx.x * 2 * kQ + kQ + j] = sm;
    if (j == 0) { cnt[2 * blockIdx.x] = np_; cnt[2 * blockIdx.x + 1] = nm; }
}

// stats[0..q): w, stats[q]: b, stats[q+1]: 1/|w| (one block of q threads, blocks in order)
__global__ void __launch_bounds__(kQ) class_stats_kernel(int G, const double *__restrict__ part,
                                                         const long long *__restrict__ cnt, float *__restrict__ stats)
{
    __shared__ double red[2][kQ / 32];
    const int j = threadIdx.x;
    double sp = 0.0, sm = 0.0;
    long long np_ = 0, nm = 0;
    for (int b = 0; b < G; ++b) {
        sp += part[(size_t)b * 2 * kQ + j];
        sm += part[(size_t)b * 2 * kQ + kQ + j];
        np_ += cnt[2 * b];
        nm += cnt[2 * b + 1];
    }
    const double mp = sp / (double)np_, mm = sm / (double)nm;
    const double w = mp - mm;
    double t0 = w * (mp + mm), t1 = w * w;
    t0 = warp_sum(t0);
    t1 = warp_sum(t1);
    if ((j & 31) == 0) { red[0][j >> 5] = t0; red[1][j >> 5] = t1; }
    __syncthreads();
    stats[j] = (float)w;
    if (j == 0) {
        double a = 0.0, b2 = 0.0;
        for (int k = 0; k < kQ / 32; ++k) { a += red[0][k]; b2 += red[1][k]; }
        stats[kQ] = (float)(-0.5 * a);
        stats[kQ + 1] = b2 > 0.0 ? (float)(1.0 / sqrt(b2)) : 1.f;
    }
}

// F_i = [x_i, y_i, |x_i|/sqrt(q), y_i (w.x_i + b)/|w|, log10 C]: a warp per row
__global__ void features_kernel(const float *__restrict__ X, const int8_t *__restrict__ y, long long n,
                                const float *__restrict__ stats, float lc, float *__restrict__ F)
{
    const int lane = threadIdx.x & 31;
    const long long w0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const float4 wv = reinterpret_cast<const float4 *>(stats)[lane];
    const float b = stats[kQ], rw = stats[kQ + 1];
    for (long long i = w0; i < n; i += nw) {
        const float4 x = reinterpret_cast<const float4 *>(X + i * kQ)[lane];
        float *f = F + i * kIn;
        reinterpret_cast<float4 *>(f)[lane] = x;
        float d = x.x * wv.x + x.y * wv.y + x.z * wv.z + x.w * wv.w;
        float s = x.x * x.x + x.y * x.y + x.z * x.z + x.w * x.w;
        d = warp_sumf(d);
        s = warp_sumf(s);
        if (lane == 0) {
            const float yi = (float)y[i];
            reinterpret_cast<float4 *>(f)[kQ / 4] =
                make_float4(yi, sqrtf(s) * 0.08838834764831845f /* 1/sqrt(128) */, yi * (d + b) * rw, lc);
        }
    }
}

}  // namespace

struct svm_mlp {
    cudaStream_t st = nullptr;
    int64_t max_rows = 0;
    float *theta = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
    float *Z1 = nullptr, *H1 = nullptr, *Z2 = nullptr, *H2 = nullptr, *Z3 = nullptr, *D3 = nullptr, *D2 = nullptr,
          *D1 = nullptr;
    float *part = nullptr, *loss = nullptr, *wpart = nullptr;
    unsigned *counter = nullptr;
};

static void mlp_free(svm_mlp *m)
{
    void *p[] = {m->theta, m->m, m->v, m->grad, m->Z1, m->H1, m->Z2, m->H2, m->Z3, m->D3, m->D2, m->D1, m->part,
                 m->loss, m->counter, m->wpart};
    for (void *x : p)
        if (x) cudaFree(x);
}

static cudaError_t forward_keep(svm_mlp *m, const float *F, int n)
{
    cudaError_t e;
    if ((e = gemm<false, false, EPI_BIAS_GELU>(m->st, n, kH, kIn, F, kIn, m->theta + oW1, kH, m->H1, kH,
                                               m->theta + ob1, m->Z1)) != cudaSuccess)
        return e;
    if ((e = gemm<false, false, EPI_BIAS_GELU>(m->st, n, kH, kH, m->H1, kH, m->theta + oW2, kH, m->H2, kH,
                                               m->theta + ob2, m->Z2)) != cudaSuccess)
        return e;
    return gemm<false, false, EPI_BIAS>(m->st, n, kOut, kH, m->H2, kH, m->theta + oW3, kOut, m->Z3, kOut,
                                        m->theta + ob3);
}

extern "C" svm_status svm_mlp_create(svm_mlp_t **out, const float *params, int64_t max_rows, void *stream)
{
    if (out) *out = nullptr;
    if (!out || !params || max_rows < 1 || max_rows > (1 << 26)) return SVM_ERR_INVALID_ARG;
    svm_mlp *m = new (std::nothrow) svm_mlp();
    if (!m) return SVM_ERR_OOM;
    m->st = (cudaStream_t)stream;
    m->max_rows = max_rows;
    const size_t r = (size_t)max_rows;
    bool bad = cudaMalloc(&m->theta, sizeof(float) * kNParam) || cudaMalloc(&m->m, sizeof(float) * kNParam) ||
               cudaMalloc(&m->v, sizeof(float) * kNParam) || cudaMalloc(&m->grad, sizeof(float) * kNParam) ||
               cudaMalloc(&m->Z1, sizeof(float) * r * kH) || cudaMalloc(&m->H1, sizeof(float) * r * kH) ||
               cudaMalloc(&m->Z2, sizeof(float) * r * kH) || cudaMalloc(&m->H2, sizeof(float) * r * kH) ||
               cudaMalloc(&m->Z3, sizeof(float) * r * kOut) || cudaMalloc(&m->D3, sizeof(float) * r * kOut) ||
               cudaMalloc(&m->D2, sizeof(float) * r * kH) || cudaMalloc(&m->D1, sizeof(float) * r * kH) ||
               cudaMalloc(&m->part, sizeof(float) * 4096) || cudaMalloc(&m->loss, sizeof(float)) ||
               cudaMalloc(&m->counter, sizeof(unsigned)) ||
               cudaMalloc(&m->wpart, sizeof(float) * kMaxSplit * ((size_t)kH * kH + kH));
    if (bad) { mlp_free(m); delete m; return SVM_ERR_OOM; }
    bad = cudaMemcpyAsync(m->theta, params, sizeof(float) * kNParam, cudaMemcpyDefault, m->st) ||
          cudaMemsetAsync(m->m, 0, sizeof(float) * kNParam, m->st) ||
          cudaMemsetAsync(m->v, 0, sizeof(float) * kNParam, m->st) ||
          cudaMemsetAsync(m->counter, 0, sizeof(unsigned), m->st);
    if (bad) { mlp_free(m); delete m; return SVM_ERR_CUDA; }
    *out = m;
    return SVM_OK;
}

extern "C" void svm_mlp_destroy(svm_mlp_t *m)
{
    if (!m) return;
    if (m->st) cudaStreamSynchronize(m->st);
    mlp_free(m);
    delete m;
}

extern "C" svm_status svm_mlp_get_params(svm_mlp_t *m, float *params)
{
    if (!m || !params) return SVM_ERR_INVALID_ARG;
    return cudaMemcpyAsync(params, m->theta, sizeof(float) * kNParam, cudaMemcpyDefault, m->st) == cudaSuccess
               ? SVM_OK
               : SVM_ERR_CUDA;
}

extern "C" svm_status svm_mlp_features(const float *X, const int8_t *y, int64_t n, int64_t q, double C, float *F,
                                       void *stream)
{
    if (!X || !y || !F || n < 2 || q != kQ || !(C > 0.0)) return SVM_ERR_INVALID_ARG;
    if ((uintptr_t)X % 16 != 0 || (uintptr_t)F % 16 != 0) return SVM_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int G = 256;
    double *part = nullptr;
    long long *cnt = nullptr;
    float *stats = nullptr;
    if (cudaMallocAsync(&part, sizeof(double) * G * 2 * kQ, st) || cudaMallocAsync(&cnt, sizeof(long long) * 2 * G, st) ||
        cudaMallocAsync(&stats, sizeof(float) * (kQ + 4), st))
        return SVM_ERR_OOM;
    class_sum_kernel<<<G, kQ, 0, st>>>(X, y, n, part, cnt);
    class_stats_kernel<<<1, kQ, 0, st>>>(G, part, cnt, stats);
    features_kernel<<<1024, 256, 0, st>>>(X, y, n, stats, (float)log10(C), F);
    const cudaError_t e = cudaGetLastError();
    cudaFreeAsync(part, st);
    cudaFreeAsync(cnt, st);
    cudaFreeAsync(stats, st);
    return e == cudaSuccess ? SVM_OK : SVM_ERR_CUDA;
}

extern "C" svm_status svm_mlp_labels(const double *alpha, int64_t n, double C, int32_t *labels, void *stream)
{
    if (!alpha || !labels || n < 1 || !(C > 0.0)) return SVM_ERR_INVALID_ARG;
    labels_kernel<<<1024, 256, 0, (cudaStream_t)stream>>>(n, alpha, C, labels);
    return cudaGetLastError() == cudaSuccess ? SVM_OK : SVM_ERR_CUDA;
}

extern "C" svm_status svm_mlp_gather(const float *F, const int32_t *labels, const int64_t *idx, int64_t nb,
                                      float *Fb, int32_t *Lb, void *stream)
{
    if (!F || !labels || !idx || !Fb || !Lb || nb < 1) return SVM_ERR_INVALID_ARG;
    if ((uintptr_t)F % 16 != 0 || (uintptr_t)Fb % 16 != 0) return SVM_ERR_INVALID_ARG;
    const long long blocks = (nb + 7) / 8;
    gather_kernel<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, (cudaStream_t)stream>>>(F, labels, idx, nb, Fb,
                                                                                              Lb);
    return cudaGetLastError() == cudaSuccess ? SVM_OK : SVM_ERR_CUDA;
}

extern "C" svm_status svm_mlp_forward(svm_mlp_t *m, const float *F, int64_t n, float *logits)
{
    if (!m || !F || !logits || n < 1 || n > m->max_rows) return SVM_ERR_INVALID_ARG;
    if (forward_keep(m, F, (int)n) != cudaSuccess) return SVM_ERR_CUDA;
    return cudaMemcpyAsync(logits, m->Z3, sizeof(float) * n * kOut, cudaMemcpyDeviceToDevice, m->st) == cudaSuccess
               ? SVM_OK
               : SVM_ERR_CUDA;
}

extern "C" svm_status svm_mlp_loss_grad(svm_mlp_t *m, const float *F, const int32_t *labels, int64_t n,
                                        const float *cw, float *loss, float *grad)
{
    if (!m || !F || !labels || !cw || !grad || n < 1 || n > m->max_rows) return SVM_ERR_INVALID_ARG;
    const int N = (int)n;
    cudaStream_t st = m->st;
    cudaError_t e = forward_keep(m, F, N);
    if (e != cudaSuccess) return SVM_ERR_CUDA;
    const int G = (N + 255) / 256 < 4096 ? (N + 255) / 256 : 4096;
    ce_kernel<<<G, 256, 0, st>>>(N, m->Z3, labels, cw, m->D3, m->part, m->counter, loss ? loss : m->loss);
    // output layer: gW3 = H2' D3, gb3; D2 = (D3 W3') o gelu'(Z2)
    if (weight_grad(st, kH, kOut, N, m->H2, kH, m->D3, m->wpart, grad + oW3) ||
        gemm<false, true, EPI_GELU_BWD>(st, N, kH, kOut, m->D3, kOut, m->theta + oW3, kOut, m->D2, kH, nullptr,
                                        nullptr, m->Z2))
        return SVM_ERR_CUDA;
    // second layer: gW2 = H1' D2, gb2; D1 = (D2 W2') o gelu'(Z1)
    if (weight_grad(st, kH, kH, N, m->H1, kH, m->D2, m->wpart, grad + oW2) ||
        gemm<false, true, EPI_GELU_BWD>(st, N, kH, kH, m->D2, kH, m->theta + oW2, kH, m->D1, kH, nullptr, nullptr,
                                        m->Z1))
        return SVM_ERR_CUDA;
    // first layer: gW1 = F' D1, gb1
    if (weight_grad(st, kIn, kH, N, F, kIn, m->D1, m->wpart, grad + oW1)) return SVM_ERR_CUDA;
    return cudaGetLastError() == cudaSuccess ? SVM_OK : SVM_ERR_CUDA;
}

extern "C" svm_status svm_mlp_adam_step(svm_mlp_t *m, const float *grad, int64_t t, float lr, float wd)
{
    if (!m || !grad || t < 1 || !(lr > 0.f) || !(wd >= 0.f)) return SVM_ERR_INVALID_ARG;
    const float c1 = (float)(1.0 - pow(0.9, (double)t)), c2 = (float)(1.0 - pow(0.999, (double)t));
    adam_kernel<<<(kNParam + 255) / 256, 256, 0, m->st>>>(kNParam, m->theta, m->m, m->v, grad, lr, wd, c1, c2);
    return cudaGetLastError() == cudaSuccess ? SVM_OK : SVM_ERR_CUDA;
}

extern "C" svm_status svm_mlp_train_step(svm_mlp_t *m, const float *F, const int32_t *labels, int64_t n,
                                         const float *cw, int64_t t, float lr, float wd, float *loss)
{
    if (!m) return SVM_ERR_INVALID_ARG;
    const svm_status s = svm_mlp_loss_grad(m, F, labels, n, cw, loss, m->grad);
    return s == SVM_OK ? svm_mlp_adam_step(m, m->grad, t, lr, wd) : s;
}

// ---- the working set of the reduced warm-start solve (svm_ssnalm.cu) ----
// Row i is in the set when the network's probability of alpha_i = 0 (softmax
// of the logits) is below p0max: e^(z1 - z0) + e^(z2 - z0) > 1 / p0max - 1.
// Block b owns rows [b per, (b + 1) per); pass 1 counts its rows (and their
// positive labels), pass 2 writes them in ascending order at the block's
// offset (the counts of the blocks before it), warp ballots within a block.
__device__ __forceinline__ bool ws_in(const float *Z3, int i, float thr)
{
    const float z0 = Z3[3 * i], z1 = Z3[3 * i + 1], z2 = Z3[3 * i + 2];
    return expf(z1 - z0) + expf(z2 - z0) > thr;
}

__global__ void ws_count_kernel(int n, const float *__restrict__ Z3, const int8_t *__restrict__ y, float thr,
                                int2 *__restrict__ blk)
{
    const int per = (n + gridDim.x - 1) / gridDim.x;
    const int r0 = blockIdx.x * per, r1 = r0 + per < n ? r0 + per : n;
    int c = 0, cp = 0;
    for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x)
        if (ws_in(Z3, i, thr)) {
            ++c;
            cp += y[i] > 0;
        }
    __shared__ int sc[32], sp[32];
    for (int o = 16; o > 0; o >>= 1) {
        c += __shfl_xor_sync(0xffffffffu, c, o);
        cp += __shfl_xor_sync(0xffffffffu, cp, o);
    }
    if ((threadIdx.x & 31) == 0) { sc[threadIdx.x >> 5] = c; sp[threadIdx.x >> 5] = cp; }
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0, tp = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { t += sc[w]; tp += sp[w]; }
        blk[blockIdx.x] = make_int2(t, tp);
    }
}

__global__ void ws_compact_kernel(int n, const float *__restrict__ Z3, float thr, const int2 *__restrict__ blk,
                                  int32_t *__restrict__ idx, long long *__restrict__ total)
{
    const int per = (n + gridDim.x - 1) / gridDim.x;
    const int r0 = blockIdx.x * per, r1 = r0 + per < n ? r0 + per : n;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __shared__ int s_off;
    __shared__ int s_w[32];
    if (threadIdx.x == 0) {
        int o = 0;
        for (int b = 0; b < (int)blockIdx.x; ++b) o += blk[b].x;
        s_off = o;
        if (blockIdx.x == 0) {
            long long t = 0, tp = 0;
            for (int b = 0; b < (int)gridDim.x; ++b) { t += blk[b].x; tp += blk[b].y; }
            total[0] = t;
            total[1] = tp;
        }
    }
    __syncthreads();
    for (int base = r0; base < r1; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const bool in = i < r1 && ws_in(Z3, i, thr);
        const unsigned bal = __ballot_sync(0xffffffffu, in);
        if (lane == 0) s_w[warp] = __popc(bal);
        __syncthreads();
        int before = 0, all = 0;
        for (int w = 0; w < nw; ++w) {
            if (w < warp) before += s_w[w];
            all += s_w[w];
        }
        if (in) idx[s_off + before + __popc(bal & ((1u << lane) - 1u))] = i;
        __syncthreads();
        if (threadIdx.x == 0) s_off += all;
        __syncthreads();
    }
}

cudaError_t mlp_working_set(svm_mlp_t *m, const float *F, long long n, const int8_t *y, float p0max, int G,
                            int2 *blk, int32_t *idx, long long *total)
{
    if (!m || !F || n < 1 || n > m->max_rows || !(p0max > 0.f && p0max < 1.f) || G < 1) return cudaErrorInvalidValue;
    const cudaError_t e = forward_keep(m, F, (int)n);
    if (e != cudaSuccess) return e;
    const float thr = 1.f / p0max - 1.f;
    ws_count_kernel<<<G, 256, 0, m->st>>>((int)n, m->Z3, y, thr, blk);
    ws_compact_kernel<<<G, 256, 0, m->st>>>((int)n, m->Z3, thr, blk, idx, total);
    return cudaGetLastError();
}

extern "C" svm_status svm_mlp_start_point(svm_mlp_t *m, const float *F, int64_t n, double C, double *alpha0)
{
    if (!m || !F || !alpha0 || n < 1 || n > m->max_rows || !(C > 0.0)) return SVM_ERR_INVALID_ARG;
    if (forward_keep(m, F, (int)n) != cudaSuccess) return SVM_ERR_CUDA;
    start_kernel<<<256, 256, 0, m->st>>>((int)n, m->Z3, C, alpha0);
    return cudaGetLastError() == cudaSuccess ? SVM_OK : SVM_ERR_CUDA;
}
