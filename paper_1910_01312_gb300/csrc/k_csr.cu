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
    double rz, hp, tol2, rr;
    long long pc;
    int done, iters;
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
__global__ void csc_count_kernel(const int64_t *__restrict__ rp, const int32_t *__restrict__ ci, long long n, int q,
                                 long long rpc, int *__restrict__ cnt)
{
    const int lane = threadIdx.x & 31;
    for (long long i = gwarp(); i < n; i += nwarps()) {
        const size_t c = (size_t)(i / rpc);
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
                                 const TV *__restrict__ cv, long long n, int q, long long rpc, int R, int *cnt,
                                 const int64_t *__restrict__ cp, int32_t *__restrict__ cr, TV *__restrict__ cvv)
{
    const int lane = threadIdx.x & 31;
    for (long long c = gwarp(); c < R; c += nwarps()) {
        const long long r0 = c * rpc, r1 = r0 + rpc < n ? r0 + rpc : n;
        volatile int *cc = cnt + (size_t)c * q;
        for (long long i = r0; i < r1; ++i) {
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
        double s0 = 0.0, s1 = 0.0;
        long long i = 0;
        if (r < nrows) {
            i = ROWLIST ? (long long)rows[r] : r;
            const long long e = rp[i + 1];
            for (long long k = rp[i] + sub; k < e; k += G) {
                const double x = ldv(cv, k);
                const int j = ci[k];
                s0 = fma(x, __ldg(v0 + j), s0);
                if (NV == 2) s1 = fma(x, __ldg(v1 + j), s1);
            }
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

// ------------------------------------------------------ column products
// Task t sums the CSC entries [tb[t], tb[t+1]) of one column:
//   MODE 0: part[t] = sum c_i y_i x_ij,  part[T + t] = sum |c_i| |x_ij|  (A'c and its roundoff scale)
//   MODE 1: part[t] = sum c_i x_ij,      part[T + t] = sum c_i x_ij^2    (h and diag G for c = 1 on J)
//   MODE 2: part[t] = sum c_i x_ij                                       (X'c)
template <typename TV, int MODE>
__global__ void __launch_bounds__(256) csc_task_kernel(long long T, const int64_t *__restrict__ tb,
                                                       const int32_t *__restrict__ cr, const TV *__restrict__ cvv,
                                                       const int8_t *__restrict__ y, const double *__restrict__ c,
                                                       double *__restrict__ part, const int *__restrict__ done)
{
    if (done && *done) return;
    const int lane = threadIdx.x & 31;
    for (long long t = gwarp(); t < T; t += nwarps()) {
        double s = 0.0, a = 0.0;
        const long long e = tb[t + 1];
        for (long long k = tb[t] + lane; k < e; k += 32) {
            const int i = cr[k];
            const double x = ldv(cvv, k), ci = c[i];
            if (MODE == 0) {
                s = fma(y[i] > 0 ? ci : -ci, x, s);
                a = fma(fabs(ci), fabs(x), a);
            } else if (MODE == 1) {
                s = fma(ci, x, s);
                a = fma(ci * x, x, a);
            } else {
                s = fma(ci, x, s);
            }
        }
        s = warp_sum(s);
        if (MODE != 2) a = warp_sum(a);
        if (lane == 0) {
            part[t] = s;
            if (MODE != 2) part[T + t] = a;
        }
    }
}

// out_j = sum of column j's task partials (in task order); with slot >= 0 also
// red[slot] = sum_j (its abs-scale partials)^2.  One block of 1024 threads.
__global__ void __launch_bounds__(1024) csc_final_kernel(int q, long long T, const int64_t *__restrict__ ct,
                                                         const double *__restrict__ part, double *__restrict__ out,
                                                         double *__restrict__ red, int slot)
{
    __shared__ double sh[32];
    double sc = 0.0;
    for (int j = threadIdx.x; j < q; j += 1024) {
        double s = 0.0, a = 0.0;
        for (long long t = ct[j]; t < ct[j + 1]; ++t) {
            s += part[t];
            a += part[T + t];
        }
        out[j] = s;
        sc = fma(a, a, sc);
    }
    if (slot < 0) return;
    sc = warp_sum(sc);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = sc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 32; ++w) t += sh[w];
        red[slot] = t;
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

// h, the Jacobi preconditioner 1/diag(M), x = 0, r = -g, z = Dinv r, d = z
__global__ void __launch_bounds__(1024) cg_setup_kernel(int q, long long T, const int64_t *__restrict__ ct,
                                                        const double *__restrict__ part, const double *__restrict__ g,
                                                        double sigma, long long pc, double eta, double tau,
                                                        CsrCg *st, double *__restrict__ h, double *__restrict__ dinv,
                                                        double *__restrict__ x, double *__restrict__ r,
                                                        double *__restrict__ z, double *__restrict__ d)
{
    __shared__ double sh[32];
    const double rp = 1.0 / (double)pc;
    double rz = 0.0, hp = 0.0, gg = 0.0;
    for (int j = threadIdx.x; j < q; j += 1024) {
        double hj = 0.0, gjj = 0.0;
        for (long long t = ct[j]; t < ct[j + 1]; ++t) {
            hj += part[t];
            gjj += part[T + t];
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
        rz = fma(rj, zj, rz);
        hp = fma(hj, zj, hp);
        gg = fma(rj, rj, gg);
    }
    rz = block_sum(rz, sh);
    hp = block_sum(hp, sh);
    gg = block_sum(gg, sh);
    if (threadIdx.x == 0) {
        const double gn = sqrt(gg);
        double tol = fmin(eta, pow(gn, 1.0 + tau));
        tol = fmin(tol, 1e-10 * gn);
        st->rz = rz;
        st->hp = hp;
        st->tol2 = tol * tol;
        st->rr = gg;
        st->pc = pc;
        st->done = gg == 0.0;
        st->iters = 0;
    }
}

// One CG step after s = X_J'(X_J d) is in the task partials: M d = d + sigma (s - h (h'd)/p).
__global__ void __launch_bounds__(1024) cg_step_kernel(int q, long long T, const int64_t *__restrict__ ct,
                                                       const double *__restrict__ part, double sigma, int maxit,
                                                       CsrCg *st, const double *__restrict__ h,
                                                       const double *__restrict__ dinv, double *__restrict__ x,
                                                       double *__restrict__ r, double *__restrict__ z,
                                                       double *__restrict__ d, double *__restrict__ md)
{
    __shared__ double sh[32];
    __shared__ int stop;
    if (st->done) return;
    const double hpp = st->hp / (double)st->pc;
    double dmd = 0.0;
    for (int j = threadIdx.x; j < q; j += 1024) {
        double s = 0.0;
        for (long long t = ct[j]; t < ct[j + 1]; ++t) s += part[t];
        const double mj = d[j] + sigma * (s - h[j] * hpp);
        md[j] = mj;
        dmd = fma(d[j], mj, dmd);
    }
    dmd = block_sum(dmd, sh);
    if (threadIdx.x == 0) stop = !(dmd > 0.0);
    __syncthreads();
    if (stop) {
        if (threadIdx.x == 0) st->done = 2;
        return;
    }
    const double a = st->rz / dmd;
    double rz = 0.0, rr = 0.0;
    for (int j = threadIdx.x; j < q; j += 1024) {
        x[j] = fma(a, d[j], x[j]);
        const double rj = fma(-a, md[j], r[j]);
        const double zj = dinv[j] * rj;
        r[j] = rj;
        z[j] = zj;
        rz = fma(rj, zj, rz);
        rr = fma(rj, rj, rr);
    }
    rz = block_sum(rz, sh);
    rr = block_sum(rr, sh);
    const int it = st->iters + 1;
    if (rr <= st->tol2 || it >= maxit) {
        __syncthreads();
        if (threadIdx.x == 0) { st->rr = rr; st->iters = it; st->done = 1; }
        return;
    }
    const double b = rz / st->rz;
    double hp = 0.0;
    for (int j = threadIdx.x; j < q; j += 1024) {
        const double dj = fma(b, d[j], z[j]);
        d[j] = dj;
        hp = fma(h[j], dj, hp);
    }
    hp = block_sum(hp, sh);
    __syncthreads();
    if (threadIdx.x == 0) { st->rz = rz; st->hp = hp; st->rr = rr; st->iters = it; }
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

int row_group(const Work &W)
{
    const double avg = W.n ? (double)W.nnz / (double)W.n : 0.0;
    return avg <= 8.0 ? 4 : (avg <= 24.0 ? 8 : (avg <= 64.0 ? 16 : 32));
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

template <typename TV, int MODE>
cudaError_t task_launch(Work &W, const double *c, const int *done)
{
    long long blocks = (W.ntask + 7) / 8;
    if (blocks > (long long)W.nsm * 16) blocks = (long long)W.nsm * 16;
    if (blocks < 1) blocks = 1;
    csc_task_kernel<TV, MODE><<<(unsigned)blocks, 256, 0, W.st>>>(W.ntask, W.task_beg, W.csc_row,
                                                                  (const TV *)W.csc_val, W.y, c, W.task_part, done);
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
    csc_count_kernel<<<W.nsm * 8, 256, 0, W.st>>>(W.csr_ptr, W.csr_idx, n, q, rpc, cnt);
    csc_colscan_kernel<<<(q + 255) / 256, 256, 0, W.st>>>((int)R, q, cnt, tot);
    scan_kernel<<<1, 1024, 0, W.st>>>(q, tot, W.csc_ptr);
    csc_place_kernel<TV><<<(unsigned)((R + 7) / 8), 256, 0, W.st>>>(W.csr_ptr, W.csr_idx, cv, n, q, rpc, (int)R, cnt,
                                                                    W.csc_ptr, W.csc_row, (TV *)W.csc_val);
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

template <typename TV>
cudaError_t newton_csr_t(Work &W, const int32_t *J, long long p, double sigma, const double *g, double *dv, bool dots)
{
    const int q = (int)W.q;
    CsrCg *st = W.csr_cg;
    int *done = &st->done;
    double *tn = W.csr_tn;
    cudaError_t e;
    if ((e = cudaMemsetAsync(tn, 0, sizeof(double) * W.n, W.st)) != cudaSuccess) return e;
    mark_kernel<<<(unsigned)((p + 255) / 256 < 4096 ? (p + 255) / 256 : 4096), 256, 0, W.st>>>(p, J, tn);
    ++W.nlaunch;
    if ((e = task_launch<TV, 1>(W, tn, nullptr)) != cudaSuccess) return e;
    double *x = W.csr_q, *r = x + q, *z = r + q, *d = z + q, *md = d + q, *dinv = md + q;
    cg_setup_kernel<<<1, 1024, 0, W.st>>>(q, W.ntask, W.col_task, W.task_part, g, sigma, p, W.eta, W.tau, st, W.h,
                                          dinv, x, r, z, d);
    ++W.nlaunch;
    const int maxit = W.csr_cg_maxit;
    for (int it = 0; it < maxit; it += kCgBatch) {
        for (int b = 0; b < kCgBatch; ++b) {
            if ((e = rows_launch<TV, 1, true, false>(W, p, J, d, nullptr, tn, nullptr, done)) != cudaSuccess) return e;
            if ((e = task_launch<TV, 2>(W, tn, done)) != cudaSuccess) return e;
            cg_step_kernel<<<1, 1024, 0, W.st>>>(q, W.ntask, W.col_task, W.task_part, sigma, maxit, st, W.h, dinv, x,
                                                 r, z, d, md);
            ++W.nlaunch;
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
    if ((e = cudaMallocHost(&W.h_csr_done, sizeof(int))) != cudaSuccess) return e;
    return W.xf32 ? csc_build_t<float>(W) : csc_build_t<double>(W);
}

cudaError_t launch_matvec_csr(Work &W, const double *v0, double *z0, const double *v1, double *z1)
{
    if (W.xf32)
        return v1 ? rows_launch<float, 2, false, true>(W, W.n, nullptr, v0, v1, z0, z1, nullptr)
                  : rows_launch<float, 1, false, true>(W, W.n, nullptr, v0, nullptr, z0, nullptr, nullptr);
    return v1 ? rows_launch<double, 2, false, true>(W, W.n, nullptr, v0, v1, z0, z1, nullptr)
              : rows_launch<double, 1, false, true>(W, W.n, nullptr, v0, nullptr, z0, nullptr, nullptr);
}

cudaError_t launch_rmatvec_csr(Work &W, const double *c, double *out, int scale_slot)
{
    const cudaError_t e = W.xf32 ? task_launch<float, 0>(W, c, nullptr) : task_launch<double, 0>(W, c, nullptr);
    if (e != cudaSuccess) return e;
    csc_final_kernel<<<1, 1024, 0, W.st>>>((int)W.q, W.ntask, W.col_task, W.task_part, out, W.red, scale_slot);
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
