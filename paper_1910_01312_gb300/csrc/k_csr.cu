// k_csr.cu -- the method's products over a sparse X stored as CSR (layout
// SVM_CSR): z = A v by rows (eq. (3.3)), A'c by columns of a CSC copy built
// once at create (eq. (3.10)), and the Newton system of Prop. 3.5 in q
// coordinates, (I + sigma (G - h h'/p)) dv = -g with G = X_J'X_J and h = X_J'1,
// solved matrix-free by conjugate gradients as Algorithm 3 prescribes
// (Jacobi preconditioner; G is never formed: q may be tens of thousands).
// FP64 accumulation; every reduction has a fixed order (deterministic).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <vector>

#include "internal.cuh"

namespace svm {

// device state of the CSR Newton CG (Jacobi-preconditioned)
struct CsrCg {
    double rz, hp, tol2, rr, alpha, beta;
    long long pc;
    int done, iters;
    unsigned counter;   // last-block counter of the CG phase kernels (back to 0 after each)
    int pad_;
    double bpart[3 * 1024];   // block partials (at most 1024 blocks)
};

namespace {

constexpr int kTaskLen = 2048;    // CSC entries per column task of the transposed product
constexpr int kCgBatch = 16;      // CG steps launched between two reads of the stop flag

__device__ __forceinline__ long long gwarp() { return (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; }
__device__ __forceinline__ long long nwarps() { return ((long long)gridDim.x * blockDim.x) >> 5; }

template <typename TV>
__device__ __forceinline__ double ldv(const TV *p, long long k) { return (double)p[k]; }

// ---------------------------------------------------------------- checks
// out[0] |= 1: a row's pointers or column indices are out of range or not
// strictly increasing; out[1] |= 1: a non-finite value.  A thread per row.
template <typename TV>
__global__ void csr_check_kernel(const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                 const TV *__restrict__ cv, long long n, long long q, long long nnz,
                                 int *__restrict__ out)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long b = rp[i], e = rp[i + 1];
        bool bad = b < 0 || e < b || e > nnz, nf = false;
        if (!bad) {
            long long prev = -1;
            for (long long k = b; k < e; ++k) {
                const long long c = ci[k];
                if (c <= prev || c >= q) { bad = true; break; }
                prev = c;
                if (!isfinite(ldv(cv, k))) nf = true;
            }
        }
        if (bad) atomicOr(out, 1);
        if (nf) atomicOr(out + 1, 1);
    }
}

// ------------------------------------------------------------- CSC build
// Deterministic transpose: rows are cut into R chunks of rpc rows; cnt[c q + j]
// counts column j in chunk c, then becomes the column's offset for that chunk,
// and one warp per chunk places its rows in order (a row's columns are
// distinct, so the lanes of a warp never touch the same counter at once).
__global__ void csc_count_kernel(const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                 const int32_t *__restrict__ rows, long long n, int q, long long rpc,
                                 int *__restrict__ cnt)
{
    const int lane = threadIdx.x & 31;
    for (long long r = gwarp(); r < n; r += nwarps()) {
        const long long i = rows ? (long long)rows[r] : r;
        const size_t c = (size_t)(r / rpc);
        for (long long k = rp[i] + lane; k < rp[i + 1]; k += 32) atomicAdd(&cnt[c * q + ci[k]], 1);
    }
}

__global__ void csc_colscan_kernel(int R, int q, int *__restrict__ cnt, int64_t *__restrict__ tot)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < q; j += gridDim.x * blockDim.x) {
        long long s = 0;
        for (int c = 0; c < R; ++c) {
            const int v = cnt[(size_t)c * q + j];
            cnt[(size_t)c * q + j] = (int)s;
            s += v;
        }
        tot[j] = s;
    }
}

// exclusive scan of m counts into out[0..m] (one block of 1024 threads)
__global__ void __launch_bounds__(1024) scan_kernel(long long m, const int64_t *__restrict__ cnt, int64_t *__restrict__ out)
{
    __shared__ long long sh[1024];
    const int t = threadIdx.x;
    const long long per = (m + 1023) / 1024, j0 = t * per, j1 = j0 + per < m ? j0 + per : m;
    long long s = 0;
    for (long long j = j0; j < j1; ++j) s += cnt[j];
    sh[t] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const long long v = t >= off ? sh[t - off] : 0;
        __syncthreads();
        sh[t] += v;
        __syncthreads();
    }
    long long base = t ? sh[t - 1] : 0;
    for (long long j = j0; j < j1; ++j) {
        out[j] = base;
        base += cnt[j];
    }
    if (t == 1023) out[m] = sh[1023];
}

template <typename TV>
__global__ void csc_place_kernel(const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                 const TV *__restrict__ cv, const int32_t *__restrict__ rows, long long n, int q,
                                 long long rpc, int R, int *cnt, const int64_t *__restrict__ cp,
                                 int32_t *__restrict__ cr, TV *__restrict__ cvv)
{
    const int lane = threadIdx.x & 31;
    for (long long c = gwarp(); c < R; c += nwarps()) {
        const long long r0 = c * rpc, r1 = r0 + rpc < n ? r0 + rpc : n;
        volatile int *cc = cnt + (size_t)c * q;
        for (long long r = r0; r < r1; ++r) {
            const long long i = rows ? (long long)rows[r] : r;
            for (long long k = rp[i] + lane; k < rp[i + 1]; k += 32) {
                const int j = ci[k];
                const int o = cc[j];
                cc[j] = o + 1;
                const long long pos = cp[j] + o;
                cr[pos] = (int32_t)i;
                cvv[pos] = cv[k];
            }
            __syncwarp();
        }
    }
}

// tasks of at most kTaskLen entries per column: tc[j] = ceil(len_j / kTaskLen)
__global__ void task_count_kernel(int q, const int64_t *__restrict__ cp, int64_t *__restrict__ tc)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < q; j += gridDim.x * blockDim.x)
        tc[j] = (cp[j + 1] - cp[j] + kTaskLen - 1) / kTaskLen;
}

// tb[ct[j] + t] = cp[j] + t kTaskLen, and tb[ct[q]] = cp[q]
__global__ void task_fill_kernel(int q, const int64_t *__restrict__ cp, const int64_t *__restrict__ ct,
                                 int64_t *__restrict__ tb)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < q; j += gridDim.x * blockDim.x)
        for (long long t = ct[j]; t < ct[j + 1]; ++t) tb[t] = cp[j] + (t - ct[j]) * kTaskLen;
    if (blockIdx.x == 0 && threadIdx.x == 0) tb[ct[q]] = cp[q];
}

// --------------------------------------------------------- row products
// z0_i = s_i <x_i, v0> (and z1 with v1), s_i = y_i when USE_Y, else 1, for the
// rows i = rows[r] (ROWLIST) or i = r; G lanes per row.
template <typename TV, int G, int NV, bool ROWLIST, bool USE_Y>
__global__ void __launch_bounds__(256) csr_rows_kernel(const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                                       const TV *__restrict__ cv, const int8_t *__restrict__ y,
                                                       long long nrows, const int32_t *__restrict__ rows,
                                                       const double *__restrict__ v0, const double *__restrict__ v1,
                                                       double *__restrict__ z0, double *__restrict__ z1,
                                                       const int *__restrict__ done)
{
    if (done && *done) return;
    constexpr int RPW = 32 / G;
    const int lane = threadIdx.x & 31, sub = lane & (G - 1), grp = lane / G;
    for (long long base = gwarp() * RPW; base < nrows; base += nwarps() * RPW) {
        const long long r = base + grp;
        // two accumulators per vector halve the dependent FMA chain
        double s0 = 0.0, s1 = 0.0, t0 = 0.0, t1 = 0.0;
        long long i = 0;
        if (r < nrows) {
            i = ROWLIST ? (long long)rows[r] : r;
            const long long e = rp[i + 1];
            long long k = rp[i] + sub;
            for (; k + G < e; k += 2 * G) {
                const double xa = ldv(cv, k), xb = ldv(cv, k + G);
                const int ja = ci[k], jb = ci[k + G];
                s0 = fma(xa, __ldg(v0 + ja), s0);
                t0 = fma(xb, __ldg(v0 + jb), t0);
                if (NV == 2) {
                    s1 = fma(xa, __ldg(v1 + ja), s1);
                    t1 = fma(xb, __ldg(v1 + jb), t1);
                }
            }
            if (k < e) {
                const double x = ldv(cv, k);
                const int j = ci[k];
                s0 = fma(x, __ldg(v0 + j), s0);
                if (NV == 2) s1 = fma(x, __ldg(v1 + j), s1);
            }
            s0 += t0;
            if (NV == 2) s1 += t1;
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            s0 += __shfl_xor_sync(0xffffffffu, s0, o);
            if (NV == 2) s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        }
        if (sub == 0 && r < nrows) {
            const bool neg = USE_Y && y[i] < 0;
            z0[i] = neg ? -s0 : s0;
            if (NV == 2) z1[i] = neg ? -s1 : s1;
        }
    }
}

// Mixed form (FP32 values): the same products with FP32 arithmetic, Dot2 of
// Ogita, Rump and Oishi (2005) against double-float (hi, lo) inputs: each
// product x (hi + lo) is formed with TwoProd and accumulated with TwoSum, so
// the row sums are as accurate as FP64 accumulation (~2^-48 of sum |terms|)
// on the FP32 pipes, which this part runs 64 times faster than FP64.
__global__ void split_q_kernel(int q, const double *__restrict__ v, float2 *__restrict__ vf)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < q; j += gridDim.x * blockDim.x) {
        const double d = v[j];
        const float h = (float)d;
        vf[j] = make_float2(h, (float)(d - (double)h));
    }
}

template <int G, int NV, bool ROWLIST, bool USE_Y, bool OUTDF>
__global__ void __launch_bounds__(256) csr_rows_df_kernel(const int64_t *__restrict__ rp,
                                                          const int32_t *__restrict__ ci, const float *__restrict__ cv,
                                                          const int8_t *__restrict__ y, long long nrows,
                                                          const int32_t *__restrict__ rows,
                                                          const float2 *__restrict__ v0, const float2 *__restrict__ v1,
                                                          void *__restrict__ z0, void *__restrict__ z1,
                                                          const int *__restrict__ done)
{
    if (done && *done) return;
    constexpr int RPW = 32 / G;
    const int lane = threadIdx.x & 31, sub = lane & (G - 1), grp = lane / G;
    for (long long base = gwarp() * RPW; base < nrows; base += nwarps() * RPW) {
        const long long r = base + grp;
        float s0 = 0.f, c0 = 0.f, s1 = 0.f, c1 = 0.f;
        long long i = 0;
        if (r < nrows) {
            i = ROWLIST ? (long long)rows[r] : r;
            const long long e = rp[i + 1];
            for (long long k = rp[i] + sub; k < e; k += G) {
                const float x = cv[k];
                const int j = ci[k];
                dot2_step(x, __ldg(v0 + j), s0, c0);
                if (NV == 2) dot2_step(x, __ldg(v1 + j), s1, c1);
            }
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            const float a = __shfl_xor_sync(0xffffffffu, s0, o), b = __shfl_xor_sync(0xffffffffu, c0, o);
            df_acc(s0, c0, a, b);
            if (NV == 2) {
                const float a1 = __shfl_xor_sync(0xffffffffu, s1, o), b1 = __shfl_xor_sync(0xffffffffu, c1, o);
                df_acc(s1, c1, a1, b1);
            }
        }
        if (sub == 0 && r < nrows) {
            const bool neg = USE_Y && y[i] < 0;
            if (OUTDF) {
                float hi, lo;
                two_sum(s0, c0, hi, lo);
                reinterpret_cast<float2 *>(z0)[i] = neg ? make_float2(-hi, -lo) : make_float2(hi, lo);
            } else {
                const double d0 = (double)s0 + (double)c0;
                reinterpret_cast<double *>(z0)[i] = neg ? -d0 : d0;
                if (NV == 2) {
                    const double d1 = (double)s1 + (double)c1;
                    reinterpret_cast<double *>(z1)[i] = neg ? -d1 : d1;
                }
            }
        }
    }
}

// ------------------------------------------------------ column products
// Task t sums the CSC entries [tb[t], tb[t+1]) of one column:
//   MODE 0: part[t] = sum c_i y_i x_ij,  part[cap + t] = sum |c_i| |x_ij|  (A'c and its roundoff scale)
//   MODE 1: part[t] = sum c_i x_ij,      part[cap + t] = sum c_i x_ij^2    (h and diag G for c = 1 on J)
//   MODE 2: part[t] = sum c_i x_ij                                       (X'c)
template <typename TV, int MODE>
// The task count is T, or *Tdev when Tdev is set (tasks built on the device).
__global__ void __launch_bounds__(256) csc_task_kernel(long long T, const long long *__restrict__ Tdev, long long cap,
                                                       const int64_t *__restrict__ tb,
                                                       const int32_t *__restrict__ cr, const TV *__restrict__ cvv,
                                                       const int8_t *__restrict__ y, const double *__restrict__ c,
                                                       double *__restrict__ part, const int *__restrict__ done)
{
    if (done && *done) return;
    if (Tdev) T = *Tdev;
    const int lane = threadIdx.x & 31;
    for (long long t = gwarp(); t < T; t += nwarps()) {
        // MODE 0's abs scale is a roundoff estimate: FP32 is enough for it
        double s = 0.0, a = 0.0;
        float af = 0.f;
        const long long e = tb[t + 1];
        for (long long k = tb[t] + lane; k < e; k += 32) {
            const int i = cr[k];
            const double x = ldv(cvv, k), ci = c[i];
            if (MODE == 0) {
                s = fma(y[i] > 0 ? ci : -ci, x, s);
                af = fmaf(fabsf((float)ci), fabsf((float)x), af);
            } else if (MODE == 1) {
                s = fma(ci, x, s);
                a = fma(ci * x, x, a);
            } else {
                s = fma(ci, x, s);
            }
        }
        s = warp_sum(s);
        if (MODE == 0) a = warp_sum((double)af);
        else if (MODE == 1) a = warp_sum(a);
        if (lane == 0) {
            part[t] = s;
            if (MODE != 2) part[cap + t] = a;
        }
    }
}

// Mixed form of the column products (FP32 values, double-float weights w):
//   MODE 0: part[t] = sum w_i x_ij (w = y o c split), part[cap + t] = sum |w_i| |x_ij| (FP32)
//   MODE 2: part[t] = sum w_i x_ij
template <int MODE>
__global__ void __launch_bounds__(256) csc_task_df_kernel(long long T, const long long *__restrict__ Tdev,
                                                          long long cap, const int64_t *__restrict__ tb,
                                                          const int32_t *__restrict__ cr,
                                                          const float *__restrict__ cvv,
                                                          const float2 *__restrict__ w, double *__restrict__ part,
                                                          const int *__restrict__ done)
{
    if (done && *done) return;
    if (Tdev) T = *Tdev;
    const int lane = threadIdx.x & 31;
    for (long long t = gwarp(); t < T; t += nwarps()) {
        float s = 0.f, c = 0.f, af = 0.f;
        const long long e = tb[t + 1];
        for (long long k = tb[t] + lane; k < e; k += 32) {
            const float x = cvv[k];
            const float2 wi = w[cr[k]];
            dot2_step(x, wi, s, c);
            if (MODE == 0) af = fmaf(fabsf(wi.x), fabsf(x), af);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float a = __shfl_xor_sync(0xffffffffu, s, o), b = __shfl_xor_sync(0xffffffffu, c, o);
            df_acc(s, c, a, b);
            if (MODE == 0) af += __shfl_xor_sync(0xffffffffu, af, o);
        }
        if (lane == 0) {
            part[t] = (double)s + (double)c;
            if (MODE == 0) part[cap + t] = (double)af;
        }
    }
}

// ---------------------------------------------------------------- Newton CG
__device__ double block_sum(double v, double *sh)
{
    v = warp_sum(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    return t;   // every thread gets the same value (fixed order)
}

__global__ void mark_kernel(long long p, const int32_t *__restrict__ J, double *__restrict__ tn)
{
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < p; r += (long long)gridDim.x * blockDim.x)
        tn[J[r]] = 1.0;
}

// Block partials of up to three sums; the last block to finish adds them in
// block order (deterministic) and returns true with the totals in tot.
template <int K>
__device__ bool last_block_sums(double (&v)[K], double *sh, double *bpart, unsigned *counter, double (&tot)[K])
{
    __shared__ int is_last;
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = block_sum(v[k], sh);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) bpart[(size_t)k * gridDim.x + blockIdx.x] = v[k];
        __threadfence();
        is_last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!is_last) return false;
    __threadfence();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double t = 0.0;
            for (unsigned b = 0; b < gridDim.x; ++b) t += __ldcg(&bpart[(size_t)k * gridDim.x + b]);
            tot[k] = t;
        }
        *counter = 0u;
    }
    return true;
}

// h, the Jacobi preconditioner 1/diag(M), x = 0, r = -g, z = Dinv r, d = z
__global__ void __launch_bounds__(256) cg_setup_kernel(int q, long long cap, const int64_t *__restrict__ ct,
                                                       const double *__restrict__ part, const double *__restrict__ g,
                                                       double sigma, long long pc, double eta, double tau,
                                                       double floor, CsrCg *st, double *__restrict__ h, double *__restrict__ dinv,
                                                       double *__restrict__ x, double *__restrict__ r,
                                                       double *__restrict__ z, double *__restrict__ d,
                                                       float2 *__restrict__ dsplit, double *__restrict__ bpart,
                                                       unsigned *__restrict__ counter)
{
    __shared__ double sh[32];
    const double rp = 1.0 / (double)pc;
    double v[3] = {0.0, 0.0, 0.0};   // r'z, h'd, |g|^2
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < q; j += gridDim.x * blockDim.x) {
        double hj = 0.0, gjj = 0.0;
        for (long long t = ct[j]; t < ct[j + 1]; ++t) {
            hj += part[t];
            gjj += part[cap + t];
        }
        const double dj = 1.0 + sigma * (gjj - hj * hj * rp);
        const double di = dj > 0.0 ? 1.0 / dj : 1.0;
        const double rj = -g[j], zj = di * rj;
        h[j] = hj;
        dinv[j] = di;
        x[j] = 0.0;
        r[j] = rj;
        z[j] = zj;
        d[j] = zj;
        if (dsplit) {
            const float hz = (float)zj;
            dsplit[j] = make_float2(hz, (float)(zj - (double)hz));
        }
        v[0] = fma(rj, zj, v[0]);
        v[1] = fma(hj, zj, v[1]);
        v[2] = fma(rj, rj, v[2]);
    }
    double tot[3];
    if (last_block_sums<3>(v, sh, bpart, counter, tot) && threadIdx.x == 0) {
        const double gn = sqrt(tot[2]);
        // as cg_tol (common.cuh) in FP64
        double tol = fmin(eta, pow(gn, 1.0 + tau));
        tol = fmin(tol, fmax(1e-10 * gn, floor));
        st->rz = tot[0];
        st->hp = tot[1];
        st->tol2 = tol * tol;
        st->rr = tot[2];
        st->pc = pc;
        st->done = tot[2] == 0.0;
        st->iters = 0;
    }
}

// One CG step in three launches once s = X_J'(X_J d) is in the task partials.
// Phase 1: M d = d + sigma (s - h (h'd)/p), alpha = r'z / d'Md.
__global__ void __launch_bounds__(256) cg_phase1_kernel(int q, const int64_t *__restrict__ ct,
                                                        const double *__restrict__ part, double sigma, CsrCg *st,
                                                        const double *__restrict__ h, const double *__restrict__ d,
                                                        double *__restrict__ md, double *__restrict__ bpart,
                                                        unsigned *__restrict__ counter)
{
    __shared__ double sh[32];
    if (st->done) return;
    const double hpp = st->hp / (double)st->pc;
    double v[1] = {0.0};
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < q; j += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (long long t = ct[j]; t < ct[j + 1]; ++t) s += part[t];
        const double dj = d[j];
        const double mj = dj + sigma * (s - h[j] * hpp);
        md[j] = mj;
        v[0] = fma(dj, mj, v[0]);
    }
    double tot[1];
    if (last_block_sums<1>(v, sh, bpart, counter, tot) && threadIdx.x == 0) {
        if (tot[0] > 0.0) st->alpha = st->rz / tot[0];
        else st->done = 2;   // no positive curvature: keep x
    }
}

// Phase 2: x += alpha d, r -= alpha Md, z = Dinv r; stop test on |r|; beta.
__global__ void __launch_bounds__(256) cg_phase2_kernel(int q, int maxit, CsrCg *st, const double *__restrict__ dinv,
                                                        const double *__restrict__ d, const double *__restrict__ md,
                                                        double *__restrict__ x, double *__restrict__ r,
                                                        double *__restrict__ z, double *__restrict__ bpart,
                                                        unsigned *__restrict__ counter)
{
    __shared__ double sh[32];
    if (st->done) return;
    const double a = st->alpha;
    double v[2] = {0.0, 0.0};   // r'z, r'r
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < q; j += gridDim.x * blockDim.x) {
        x[j] = fma(a, d[j], x[j]);
        const double rj = fma(-a, md[j], r[j]);
        const double zj = dinv[j] * rj;
        r[j] = rj;
        z[j] = zj;
        v[0] = fma(rj, zj, v[0]);
        v[1] = fma(rj, rj, v[1]);
    }
    double tot[2];
    if (last_block_sums<2>(v, sh, bpart, counter, tot) && threadIdx.x == 0) {
        const int it = st->iters + 1;
        st->iters = it;
        st->rr = tot[1];
        if (tot[1] <= st->tol2 || it >= maxit) {
            st->done = 1;
        } else {
            st->beta = tot[0] / st->rz;
            st->rz = tot[0];
        }
    }
}

// out_j = sum of column j's task partials (in task order); with slot >= 0 also
// red[slot] = sum_j (its abs-scale partials)^2 (block partials, last block).
__global__ void __launch_bounds__(256) csc_final_kernel(int q, long long cap, const int64_t *__restrict__ ct,
                                                        const double *__restrict__ part, double *__restrict__ out,
                                                        double *__restrict__ red, int slot, double *__restrict__ bpart,
                                                        unsigned *__restrict__ counter)
{
    __shared__ double sh[32];
    double v[1] = {0.0};
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < q; j += gridDim.x * blockDim.x) {
        double s = 0.0, a = 0.0;
        for (long long t = ct[j]; t < ct[j + 1]; ++t) {
            s += part[t];
            a += part[cap + t];
        }
        out[j] = s;
        v[0] = fma(a, a, v[0]);
    }
    if (slot < 0) return;
    double tot[1];
    if (last_block_sums<1>(v, sh, bpart, counter, tot) && threadIdx.x == 0) red[slot] = tot[0];
}

// Phase 3: d = z + beta d and h'd.
__global__ void __launch_bounds__(256) cg_phase3_kernel(int q, CsrCg *st, const double *__restrict__ h,
                                                        const double *__restrict__ z, double *__restrict__ d,
                                                        float2 *__restrict__ dsplit, double *__restrict__ bpart,
                                                        unsigned *__restrict__ counter)
{
    __shared__ double sh[32];
    if (st->done) return;
    const double b = st->beta;
    double v[1] = {0.0};
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < q; j += gridDim.x * blockDim.x) {
        const double dj = fma(b, d[j], z[j]);
        d[j] = dj;
        if (dsplit) {
            const float hd = (float)dj;
            dsplit[j] = make_float2(hd, (float)(dj - (double)hd));
        }
        v[0] = fma(h[j], dj, v[0]);
    }
    double tot[1];
    if (last_block_sums<1>(v, sh, bpart, counter, tot) && threadIdx.x == 0) st->hp = tot[0];
}

__global__ void cg_finish_kernel(int q, const CsrCg *st, const double *__restrict__ x, double *__restrict__ dv,
                                 double *__restrict__ info)
{
    for (int j = threadIdx.x; j < q; j += blockDim.x) dv[j] = x[j];
    if (threadIdx.x == 0) {
        info[0] = (double)st->iters;
        info[1] = sqrt(st->rr);
    }
}

// Lanes per row: few enough that the FP64 shuffle reduction (log2 G adds per
// lane) stays small against the row's own FMAs, and enough rows per warp.
int row_group(const Work &W)
{
    const double avg = W.n ? (double)W.nnz / (double)W.n : 0.0;
    return avg <= 16.0 ? 4 : (avg <= 256.0 ? 8 : (avg <= 1024.0 ? 16 : 32));
}

template <typename TV, int NV, bool ROWLIST, bool USE_Y>
cudaError_t rows_launch(Work &W, long long nrows, const int32_t *rows, const double *v0, const double *v1, double *z0,
                        double *z1, const int *done)
{
    const int G = row_group(W);
    const long long warps = (nrows * G + 31) / 32;
    long long blocks = (warps + 7) / 8;
    if (blocks > (long long)W.nsm * 16) blocks = (long long)W.nsm * 16;
    if (blocks < 1) blocks = 1;
    const TV *cv = (const TV *)W.csr_val;
#define RW_CASE(g)                                                                                              \
    case g:                                                                                                     \
        csr_rows_kernel<TV, g, NV, ROWLIST, USE_Y><<<(unsigned)blocks, 256, 0, W.st>>>(                         \
            W.csr_ptr, W.csr_idx, cv, W.y, nrows, rows, v0, v1, z0, z1, done);                                  \
        break;
    switch (G) {
        RW_CASE(4) RW_CASE(8) RW_CASE(16) RW_CASE(32)
    }
#undef RW_CASE
    ++W.nlaunch;
    return cudaGetLastError();
}

// A column view of X (the whole matrix, or the rows of a free set J): CSC
// arrays, column tasks and their partial sums (second half at offset cap).
struct ColSet {
    const int32_t *row;
    const void *val;
    const int64_t *tb, *ct;
    double *part;
    long long T, cap;
    const long long *Tdev;   // device task count (nullable: T)
};

ColSet full_cols(const Work &W)
{
    return ColSet{W.csc_row, W.csc_val, W.task_beg, W.col_task, W.task_part, W.ntask, W.ntask, nullptr};
}

ColSet free_cols(const Work &W)
{
    return ColSet{W.jcsc_row, W.jcsc_val, W.jtask_beg, W.jcol_task, W.jtask_part, W.jtask_cap, W.jtask_cap,
                  reinterpret_cast<const long long *>(W.jcol_task + W.q)};
}

template <typename TV, int MODE>
cudaError_t task_launch(Work &W, const ColSet &cs, const double *c, const int *done)
{
    long long blocks = (cs.T + 7) / 8;
    if (blocks > (long long)W.nsm * 16) blocks = (long long)W.nsm * 16;
    if (blocks < 1) blocks = 1;
    csc_task_kernel<TV, MODE><<<(unsigned)blocks, 256, 0, W.st>>>(cs.T, cs.Tdev, cs.cap, cs.tb, cs.row,
                                                                  (const TV *)cs.val, W.y, c, cs.part, done);
    ++W.nlaunch;
    return cudaGetLastError();
}

bool mixed_csr(const Work &W) { return W.precision == 1 && W.xf32; }

template <int NV, bool ROWLIST, bool USE_Y, bool OUTDF>
cudaError_t rows_df_launch(Work &W, long long nrows, const int32_t *rows, const float2 *v0, const float2 *v1, void *z0,
                           void *z1, const int *done)
{
    const int G = row_group(W);
    const long long warps = (nrows * G + 31) / 32;
    long long blocks = (warps + 7) / 8;
    if (blocks > (long long)W.nsm * 16) blocks = (long long)W.nsm * 16;
    if (blocks < 1) blocks = 1;
    const float *cv = (const float *)W.csr_val;
#define RD_CASE(g)                                                                                              \
    case g:                                                                                                     \
        csr_rows_df_kernel<g, NV, ROWLIST, USE_Y, OUTDF><<<(unsigned)blocks, 256, 0, W.st>>>(                   \
            W.csr_ptr, W.csr_idx, cv, W.y, nrows, rows, v0, v1, z0, z1, done);                                  \
        break;
    switch (G) {
        RD_CASE(4) RD_CASE(8) RD_CASE(16) RD_CASE(32)
    }
#undef RD_CASE
    ++W.nlaunch;
    return cudaGetLastError();
}

template <int MODE>
cudaError_t task_df_launch(Work &W, const ColSet &cs, const float2 *w, const int *done)
{
    long long blocks = (cs.T + 7) / 8;
    if (blocks > (long long)W.nsm * 16) blocks = (long long)W.nsm * 16;
    if (blocks < 1) blocks = 1;
    csc_task_df_kernel<MODE><<<(unsigned)blocks, 256, 0, W.st>>>(cs.T, cs.Tdev, cs.cap, cs.tb, cs.row,
                                                                 (const float *)cs.val, w, cs.part, done);
    ++W.nlaunch;
    return cudaGetLastError();
}

cudaError_t split_q(Work &W, const double *v, float2 *vf)
{
    const int q = (int)W.q;
    int blocks = (q + 255) / 256;
    if (blocks > W.nsm * 4) blocks = W.nsm * 4;
    split_q_kernel<<<blocks, 256, 0, W.st>>>(q, v, vf);
    ++W.nlaunch;
    return cudaGetLastError();
}

template <typename TV>
cudaError_t csc_build_t(Work &W)
{
    const long long n = W.n, nnz = W.nnz;
    const int q = (int)W.q;
    // chunk count: at most 4096 chunks and 512 MiB of counters
    long long R = ((long long)128 << 20) / (q > 0 ? q : 1);
    if (R > 4096) R = 4096;
    if (R > n) R = n;
    if (R < 1) R = 1;
    const long long rpc = (n + R - 1) / R;
    R = (n + rpc - 1) / rpc;
    int *cnt = nullptr;
    int64_t *tot = nullptr;
    cudaError_t e;
    if ((e = cudaMalloc(&cnt, sizeof(int) * (size_t)R * q)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&tot, sizeof(int64_t) * q)) != cudaSuccess) { cudaFree(cnt); return e; }
    cudaMemsetAsync(cnt, 0, sizeof(int) * (size_t)R * q, W.st);
    const TV *cv = (const TV *)W.csr_val;
    csc_count_kernel<<<W.nsm * 8, 256, 0, W.st>>>(W.csr_ptr, W.csr_idx, nullptr, n, q, rpc, cnt);
    csc_colscan_kernel<<<(q + 255) / 256, 256, 0, W.st>>>((int)R, q, cnt, tot);
    scan_kernel<<<1, 1024, 0, W.st>>>(q, tot, W.csc_ptr);
    csc_place_kernel<TV><<<(unsigned)((R + 7) / 8), 256, 0, W.st>>>(W.csr_ptr, W.csr_idx, cv, nullptr, n, q, rpc,
                                                                    (int)R, cnt, W.csc_ptr, W.csc_row,
                                                                    (TV *)W.csc_val);
    W.nlaunch += 4;
    e = cudaGetLastError();
    // column tasks (host side, from the column pointers)
    std::vector<int64_t> cp((size_t)q + 1);
    if (e == cudaSuccess) e = cudaMemcpyAsync(cp.data(), W.csc_ptr, sizeof(int64_t) * (q + 1), cudaMemcpyDeviceToHost, W.st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(W.st);
    cudaFree(cnt);
    cudaFree(tot);
    if (e != cudaSuccess) return e;
    if (cp[q] != nnz) return cudaErrorInvalidValue;
    std::vector<int64_t> tb, ct((size_t)q + 1);
    tb.reserve((size_t)q + (size_t)(nnz / kTaskLen) + 1);
    for (int j = 0; j < q; ++j) {
        ct[j] = (int64_t)tb.size();
        for (int64_t b = cp[j]; b < cp[j + 1]; b += kTaskLen) tb.push_back(b);
    }
    ct[q] = (int64_t)tb.size();
    W.ntask = (long long)tb.size();
    tb.push_back(nnz);
    if ((e = cudaMalloc(&W.task_beg, sizeof(int64_t) * tb.size())) != cudaSuccess) return e;
    if ((e = cudaMalloc(&W.col_task, sizeof(int64_t) * ct.size())) != cudaSuccess) return e;
    if ((e = cudaMalloc(&W.task_part, sizeof(double) * 2 * (size_t)(W.ntask > 0 ? W.ntask : 1))) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(W.task_beg, tb.data(), sizeof(int64_t) * tb.size(), cudaMemcpyHostToDevice, W.st)) != cudaSuccess)
        return e;
    if ((e = cudaMemcpyAsync(W.col_task, ct.data(), sizeof(int64_t) * ct.size(), cudaMemcpyHostToDevice, W.st)) != cudaSuccess)
        return e;
    return cudaStreamSynchronize(W.st);   // the host vectors go out of scope
}

// Columns of the rows of J (ascending), built on the device: chunked counts,
// column pointers, placement in row order, then column tasks.
template <typename TV>
cudaError_t free_cols_build(Work &W, const int32_t *J, long long p)
{
    const int q = (int)W.q;
    long long R = p / 64;
    if (R > W.jchunk_cap) R = W.jchunk_cap;
    if (R < 1) R = 1;
    const long long rpc = (p + R - 1) / R;
    R = (p + rpc - 1) / rpc;
    cudaError_t e;
    if ((e = cudaMemsetAsync(W.jcnt, 0, sizeof(int) * (size_t)R * q, W.st)) != cudaSuccess) return e;
    long long blocks = (p + 7) / 8;
    if (blocks > (long long)W.nsm * 8) blocks = (long long)W.nsm * 8;
    csc_count_kernel<<<(unsigned)blocks, 256, 0, W.st>>>(W.csr_ptr, W.csr_idx, J, p, q, rpc, W.jcnt);
    csc_colscan_kernel<<<(q + 255) / 256, 256, 0, W.st>>>((int)R, q, W.jcnt, W.jtot);
    scan_kernel<<<1, 1024, 0, W.st>>>(q, W.jtot, W.jcsc_ptr);
    csc_place_kernel<TV><<<(unsigned)((R + 7) / 8), 256, 0, W.st>>>(W.csr_ptr, W.csr_idx, (const TV *)W.csr_val, J,
                                                                    p, q, rpc, (int)R, W.jcnt, W.jcsc_ptr,
                                                                    W.jcsc_row, (TV *)W.jcsc_val);
    task_count_kernel<<<(q + 255) / 256, 256, 0, W.st>>>(q, W.jcsc_ptr, W.jtot);
    scan_kernel<<<1, 1024, 0, W.st>>>(q, W.jtot, W.jcol_task);
    task_fill_kernel<<<(q + 255) / 256, 256, 0, W.st>>>(q, W.jcsc_ptr, W.jcol_task, W.jtask_beg);
    W.nlaunch += 7;
    return cudaGetLastError();
}

template <typename TV>
cudaError_t newton_csr_t(Work &W, const int32_t *J, long long p, double sigma, const double *g, double *dv, bool dots)
{
    const int q = (int)W.q;
    CsrCg *st = W.csr_cg;
    int *done = &st->done;
    double *tn = W.csr_tn;
    cudaError_t e;
    if ((e = free_cols_build<TV>(W, J, p)) != cudaSuccess) return e;
    const ColSet cs = free_cols(W);
    if ((e = cudaMemsetAsync(tn, 0, sizeof(double) * W.n, W.st)) != cudaSuccess) return e;
    mark_kernel<<<(unsigned)((p + 255) / 256 < 4096 ? (p + 255) / 256 : 4096), 256, 0, W.st>>>(p, J, tn);
    ++W.nlaunch;
    if ((e = task_launch<TV, 1>(W, cs, tn, nullptr)) != cudaSuccess) return e;
    double *x = W.csr_q, *r = x + q, *z = r + q, *d = z + q, *md = d + q, *dinv = md + q;
    int G = (q + 255) / 256;
    if (G > 2 * W.nsm) G = 2 * W.nsm;
    if (G > 1024) G = 1024;
    // mixed form: the CG's two products run in Dot2 on the split of d, with
    // X_J d kept as double-float pairs (zero outside J)
    const bool mx = mixed_csr(W);
    float2 *dsp = mx ? W.csr_df : nullptr;
    if (mx && (e = cudaMemsetAsync(W.csr_tnf, 0, sizeof(float2) * W.n, W.st)) != cudaSuccess) return e;
    cg_setup_kernel<<<G, 256, 0, W.st>>>(q, cs.cap, cs.ct, cs.part, g, sigma, p, W.eta, W.tau, W.cg_floor, st, W.h, dinv, x, r, z,
                                         d, dsp, st->bpart, &st->counter);
    ++W.nlaunch;
    const int maxit = W.csr_cg_maxit;
    for (int it = 0; it < maxit; it += kCgBatch) {
        for (int b = 0; b < kCgBatch; ++b) {
            if (mx) {
                if ((e = rows_df_launch<1, true, false, true>(W, p, J, dsp, nullptr, W.csr_tnf, nullptr, done)) !=
                    cudaSuccess)
                    return e;
                if ((e = task_df_launch<2>(W, cs, W.csr_tnf, done)) != cudaSuccess) return e;
            } else {
                if ((e = rows_launch<TV, 1, true, false>(W, p, J, d, nullptr, tn, nullptr, done)) != cudaSuccess)
                    return e;
                if ((e = task_launch<TV, 2>(W, cs, tn, done)) != cudaSuccess) return e;
            }
            cg_phase1_kernel<<<G, 256, 0, W.st>>>(q, cs.ct, cs.part, sigma, st, W.h, d, md, st->bpart, &st->counter);
            cg_phase2_kernel<<<G, 256, 0, W.st>>>(q, maxit, st, dinv, d, md, x, r, z, st->bpart, &st->counter);
            cg_phase3_kernel<<<G, 256, 0, W.st>>>(q, st, W.h, z, d, dsp, st->bpart, &st->counter);
            W.nlaunch += 3;
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = cudaMemcpyAsync(W.h_csr_done, done, sizeof(int), cudaMemcpyDeviceToHost, W.st)) != cudaSuccess) return e;
        if ((e = cudaStreamSynchronize(W.st)) != cudaSuccess) return e;
        if (*W.h_csr_done) break;
    }
    cg_finish_kernel<<<1, 1024, 0, W.st>>>(q, st, x, dv, W.red + 12);
    ++W.nlaunch;
    e = cudaGetLastError();
    return (e == cudaSuccess && dots) ? launch_dots(W) : e;
}

}  // namespace

cudaError_t csr_validate(Work &W, int *dev_flags)
{
    const unsigned blocks = (unsigned)(W.nsm * 8);
    if (W.xf32)
        csr_check_kernel<float><<<blocks, 256, 0, W.st>>>(W.csr_ptr, W.csr_idx, (const float *)W.csr_val, W.n, W.q,
                                                          W.nnz, dev_flags);
    else
        csr_check_kernel<double><<<blocks, 256, 0, W.st>>>(W.csr_ptr, W.csr_idx, (const double *)W.csr_val, W.n, W.q,
                                                           W.nnz, dev_flags);
    ++W.nlaunch;
    return cudaGetLastError();
}

cudaError_t csr_setup(Work &W)
{
    const size_t es = W.xf32 ? 4 : 8;
    const size_t nz = (size_t)(W.nnz > 0 ? W.nnz : 1);
    cudaError_t e;
    if ((e = cudaMalloc(&W.csc_ptr, sizeof(int64_t) * (W.q + 1))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&W.csc_row, sizeof(int32_t) * nz)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&W.csc_val, es * nz)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&W.csr_tn, sizeof(double) * W.n)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&W.csr_q, sizeof(double) * 6 * W.q)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&W.csr_cg, sizeof(CsrCg))) != cudaSuccess) return e;
    if (mixed_csr(W)) {
        if ((e = cudaMalloc(&W.csr_vf, sizeof(float2) * 2 * W.q)) != cudaSuccess) return e;
        if ((e = cudaMalloc(&W.csr_df, sizeof(float2) * W.q)) != cudaSuccess) return e;
        if ((e = cudaMalloc(&W.csr_cf, sizeof(float2) * W.n)) != cudaSuccess) return e;
        if ((e = cudaMalloc(&W.csr_tnf, sizeof(float2) * W.n)) != cudaSuccess) return e;
    }
    if ((e = cudaMemsetAsync(W.csr_cg, 0, sizeof(CsrCg), W.st)) != cudaSuccess) return e;
    if ((e = cudaMallocHost(&W.h_csr_done, sizeof(int))) != cudaSuccess) return e;
    // the free set's columns (rebuilt for every Newton step): at most nnz entries
    // and q + nnz / kTaskLen tasks; chunk counters for up to 256 chunks (64 MiB cap)
    W.jtask_cap = W.q + (long long)(nz / kTaskLen) + 1;
    long long jc = ((long long)16 << 20) / (W.q > 0 ? W.q : 1);
    W.jchunk_cap = jc > 256 ? 256 : (jc < 1 ? 1 : jc);
    if ((e = cudaMalloc(&W.jcsc_ptr, sizeof(int64_t) * (W.q + 1))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&W.jcsc_row, sizeof(int32_t) * nz)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&W.jcsc_val, es * nz)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&W.jtot, sizeof(int64_t) * W.q)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&W.jcnt, sizeof(int) * (size_t)W.jchunk_cap * W.q)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&W.jcol_task, sizeof(int64_t) * (W.q + 1))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&W.jtask_beg, sizeof(int64_t) * (W.jtask_cap + 1))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&W.jtask_part, sizeof(double) * 2 * W.jtask_cap)) != cudaSuccess) return e;
    return W.xf32 ? csc_build_t<float>(W) : csc_build_t<double>(W);
}

cudaError_t launch_matvec_csr(Work &W, const double *v0, double *z0, const double *v1, double *z1)
{
    if (mixed_csr(W)) {
        float2 *f0 = W.csr_vf, *f1 = W.csr_vf + W.q;
        cudaError_t e = split_q(W, v0, f0);
        if (e == cudaSuccess && v1) e = split_q(W, v1, f1);
        if (e != cudaSuccess) return e;
        return v1 ? rows_df_launch<2, false, true, false>(W, W.n, nullptr, f0, f1, z0, z1, nullptr)
                  : rows_df_launch<1, false, true, false>(W, W.n, nullptr, f0, nullptr, z0, nullptr, nullptr);
    }
    if (W.xf32)
        return v1 ? rows_launch<float, 2, false, true>(W, W.n, nullptr, v0, v1, z0, z1, nullptr)
                  : rows_launch<float, 1, false, true>(W, W.n, nullptr, v0, nullptr, z0, nullptr, nullptr);
    return v1 ? rows_launch<double, 2, false, true>(W, W.n, nullptr, v0, v1, z0, z1, nullptr)
              : rows_launch<double, 1, false, true>(W, W.n, nullptr, v0, nullptr, z0, nullptr, nullptr);
}

cudaError_t launch_rmatvec_csr(Work &W, const double *c, double *out, int scale_slot)
{
    const ColSet cs = full_cols(W);
    cudaError_t e;
    if (mixed_csr(W)) {
        e = split_weights(W, c, W.csr_cf);   // y o c as double-float pairs
        if (e == cudaSuccess) e = task_df_launch<0>(W, cs, W.csr_cf, nullptr);
    } else {
        e = W.xf32 ? task_launch<float, 0>(W, cs, c, nullptr) : task_launch<double, 0>(W, cs, c, nullptr);
    }
    if (e != cudaSuccess) return e;
    int G = (int)((W.q + 255) / 256);
    if (G > 2 * W.nsm) G = 2 * W.nsm;
    if (G > 1024) G = 1024;
    csc_final_kernel<<<G, 256, 0, W.st>>>((int)W.q, cs.cap, cs.ct, cs.part, out, W.red, scale_slot, W.csr_cg->bpart,
                                          &W.csr_cg->counter);
    ++W.nlaunch;
    return cudaGetLastError();
}

cudaError_t launch_newton_csr(Work &W, const int32_t *J, long long p, double sigma, const double *g, double *dv,
                              bool dots)
{
    if (p <= 0) {
        const cudaError_t e = launch_negcopy(W, g, dv);
        return (e == cudaSuccess && dots) ? launch_dots(W) : e;
    }
    return W.xf32 ? newton_csr_t<float>(W, J, p, sigma, g, dv, dots) : newton_csr_t<double>(W, J, p, sigma, g, dv, dots);
}

}  // namespace svm
