// k_gqp.cu -- kernels of the unified-QP solver (Sec. 1, eq. (1.5)): the
// products z = B v and B'y, the projection onto {a'x = d, l <= x <= u}
// (Sec. 3.2.1, Algorithm 2) with the free-set compaction, and the reduced
// Newton matrix of Proposition 3.5 with a general a:
//     (I + sigma (B_J'B_J - h h' / s)) dv = -g,  h = B_J'a_J,  s = a_J'a_J,
// the q-space form of Prop. 3.5 (v = B'w) with the HS-Jacobian of Theorem 3.2
// P = Diag(1_J) - (1_J o a)(1_J o a)'/s (case (b), P = 0 on J's complement and
// no rank-one term, when s = 0).
//
// Every quantity is FP64 (X may be stored FP32; its entries widen exactly).
// Reductions are two-stage in a fixed order (block partials, then one pass in
// block order), so every result is deterministic.
#include <math.h>

#include "gqp.cuh"

namespace svm {
namespace gqp {

constexpr int kPT = 256;            // threads of the projection / vector kernels
constexpr int kPW = kPT / 32;
constexpr int kMaxPass = 200;
constexpr int kRecStride = 8;       // doubles per block partial of the projection
constexpr int kGT = 32;             // Gram tile
constexpr int kGRows = 32;          // rows staged per Gram step

template <typename T>
__device__ __forceinline__ double ldx(const void *X, long long k)
{
    return (double)static_cast<const T *>(X)[k];
}

__device__ __forceinline__ double lane0(double v) { return __shfl_sync(0xffffffffu, v, 0); }

// w - lambda a rounded as written (a product, then a difference; no FMA), so
// that the projection is clip(w - lambda a, l, u) of the definition exactly.
__device__ __forceinline__ double shifted(double w, double lam, double a) { return __dsub_rn(w, __dmul_rn(lam, a)); }

// ---------------------------------------------------------------- z = B v

// Eight lanes per stored row (a warp takes four rows); lanes stride the
// columns, FP64 FMAs, then a three-level shuffle reduction.  STACKED writes
// row i of X to z_i and -(row i) to z_{m+i}.
template <typename T>
__global__ void __launch_bounds__(kPT) matvec_kernel(const void *__restrict__ X, long long m, int q, int layout,
                                                     const double *__restrict__ v, double *__restrict__ z)
{
    extern __shared__ double vs[];
    for (int j = threadIdx.x; j < q; j += blockDim.x) vs[j] = v[j];
    __syncthreads();
    const int lane = threadIdx.x & 31, sub = lane & 7;
    const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
    // r0 is the same for the whole warp, so the shuffles below run warp-uniformly
    for (long long r0 = ((long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 4; r0 < m;
         r0 += nwarps * 4) {
        const long long i = r0 + (lane >> 3);
        double s = 0.0;
        if (i < m) {
            const long long base = i * (long long)q;
            for (int j = sub; j < q; j += 8) s = fma(ldx<T>(X, base + j), vs[j], s);
        }
        s += __shfl_xor_sync(0xffffffffu, s, 4);
        s += __shfl_xor_sync(0xffffffffu, s, 2);
        s += __shfl_xor_sync(0xffffffffu, s, 1);
        if (i < m && sub == 0) {
            z[i] = s;
            if (layout == STACKED) z[m + i] = -s;
        }
    }
}

cudaError_t matvec(Ws &W, const double *v, double *z)
{
    const size_t smem = (size_t)W.q * sizeof(double);
    const int grid = W.nsm * 8;
    if (W.xf32)
        matvec_kernel<float><<<grid, kPT, smem, W.st>>>(W.X, W.m, W.q, W.layout, v, z);
    else
        matvec_kernel<double><<<grid, kPT, smem, W.st>>>(W.X, W.m, W.q, W.layout, v, z);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- B'y

// Block b sums its contiguous range of stored rows: thread j owns columns
// j, j + blockDim, ...; row weights (y_i, or y_i - y_{m+i} for STACKED) skip
// zero rows.  The absolute sums |B|'|y| ride along (the roundoff scale of B'y).
template <typename T>
__global__ void __launch_bounds__(kPT) rmatvec_part_kernel(const void *__restrict__ X, long long m, int q, int layout,
                                                           const double *__restrict__ y, double *__restrict__ part)
{
    const int G = gridDim.x;
    const long long per = (m + G - 1) / G;
    const long long r0 = (long long)blockIdx.x * per;
    const long long r1 = r0 + per < m ? r0 + per : m;
    double *po = part + (size_t)blockIdx.x * 2 * q;
    for (int j0 = 0; j0 < q; j0 += blockDim.x) {
        const int j = j0 + threadIdx.x;
        double s = 0.0, sa = 0.0;
        for (long long i = r0; i < r1; ++i) {
            double w = y[i], wa = fabs(w);
            if (layout == STACKED) {
                const double y2 = y[m + i];
                w -= y2;
                wa += fabs(y2);
            }
            if (wa == 0.0) continue;
            if (j < q) {
                const double xv = ldx<T>(X, i * (long long)q + j);
                s = fma(w, xv, s);
                sa = fma(wa, fabs(xv), sa);
            }
        }
        if (j < q) {
            po[j] = s;
            po[q + j] = sa;
        }
    }
}

// out_j = sum over blocks in order; scale = |(|B|'|y|)|^2 (one block)
__global__ void __launch_bounds__(1024) rmatvec_final_kernel(const double *__restrict__ part, int G, int q,
                                                              double *__restrict__ out, double *__restrict__ scale)
{
    __shared__ double sh[32];
    double acc = 0.0;
    for (int j = threadIdx.x; j < q; j += blockDim.x) {
        double s = 0.0, sa = 0.0;
        for (int b = 0; b < G; ++b) {
            s += part[(size_t)b * 2 * q + j];
            sa += part[(size_t)b * 2 * q + q + j];
        }
        out[j] = s;
        acc = fma(sa, sa, acc);
    }
    if (scale) {
        acc = warp_sum(acc);
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
            *scale = t;
        }
    }
}

cudaError_t rmatvec(Ws &W, const double *y, double *out, double *scale_dev)
{
    const int G = W.rm_grid;
    if (W.xf32)
        rmatvec_part_kernel<float><<<G, kPT, 0, W.st>>>(W.X, W.m, W.q, W.layout, y, W.part);
    else
        rmatvec_part_kernel<double><<<G, kPT, 0, W.st>>>(W.X, W.m, W.q, W.layout, y, W.part);
    rmatvec_final_kernel<<<1, 1024, 0, W.st>>>(W.part, G, W.q, out, scale_dev);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- projection

struct PArgs {
    long long n;
    const double *x, *z, *dz, *c, *a, *ainv, *lo, *hi;
    double sigma, t, d;
    const double *lam0;
    double *lam_out;
    double *w_out, *pi_out;
    int32_t *J;
    const double *pib, *wb;
    double *part;
    long long *cnt;
    unsigned *bar;
    int *err;
    ProjRec *rec;
};

// One component at lambda: its pi, its share of f = a'pi, the one-sided free
// flags (free just right / just left of lambda, for the slopes) and its
// breakpoint offsets (lambda' - lambda where r hits a bound).
struct Comp {
    double pi, fa;
    bool fr, fl;
    double o1, o2;
};

__device__ __forceinline__ Comp comp_at(double w, double a, double ainv, double lo, double hi, double lam)
{
    Comp o;
    const double r = shifted(w, lam, a);
    o.pi = r >= hi ? hi : (r <= lo ? lo : r);   // ties go to the bound (Sec. 3.2.1)
    o.fa = a * o.pi;
    const bool in_r = a > 0.0 ? (lo < r && r <= hi) : (lo <= r && r < hi);   // r moves by -eps a
    const bool in_l = a > 0.0 ? (lo <= r && r < hi) : (lo < r && r <= hi);
    o.fr = a != 0.0 && lo < hi && in_r;
    o.fl = a != 0.0 && lo < hi && in_l;
    o.o1 = (r - lo) * ainv;   // 0 when a = 0
    o.o2 = (r - hi) * ainv;
    return o;
}

// Block partials reduced in block order by warp 0 of every block (identical
// in every block, so every block takes the same decision).
__device__ __forceinline__ void reduce_pass(const double *part, int G, double *tot)
{
    const int lane = threadIdx.x & 31;
    double f = 0.0, fa = 0.0, sp = 0.0, sm = 0.0, dh = INFINITY, dl = -INFINITY;
    for (int b = lane; b < G; b += 32) {
        const double *p = part + (size_t)b * kRecStride;
        f += __ldcg(p + 0); fa += __ldcg(p + 1); sp += __ldcg(p + 2); sm += __ldcg(p + 3);
        dh = fmin(dh, __ldcg(p + 4)); dl = fmax(dl, __ldcg(p + 5));
    }
    tot[0] = lane0(warp_sum(f)); tot[1] = lane0(warp_sum(fa)); tot[2] = lane0(warp_sum(sp));
    tot[3] = lane0(warp_sum(sm)); tot[4] = lane0(warp_min(dh)); tot[5] = lane0(warp_max(dl));
}

// Projection of w = x - sigma (z + t dz + c) onto {a'y = d, l <= y <= u} in one
// cooperative launch.  lambda-hat is the root of the nonincreasing piecewise-
// linear f(lambda) = a' clip(w - lambda a, l, u) - d.  Instead of sorting the
// 2n breakpoints (Algorithm 2) all blocks iterate in lock-step: each pass
// reduces f, the one-sided slopes sum a_i^2 over the components free just
// right / left of lambda, and the nearest breakpoints on either side; a Newton
// step that stays inside the current linear piece is the root (f is linear
// there), a flat piece is crossed to its next breakpoint, and a bracket with
// forced bisection every third pass guarantees termination.  Then pi, the
// sums of the record and J (ascending, warp ballots + block scan) are written.
__global__ void __launch_bounds__(kPT) proj_kernel(PArgs A)
{
    const int G = gridDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long per = (A.n + G - 1) / G;
    const long long i0 = (long long)blockIdx.x * per;
    const long long i1 = i0 + per < A.n ? i0 + per : A.n;
    __shared__ double sh[kPW][8];
    __shared__ double s_lam;
    __shared__ int s_state;   // 0 searching, 1 found, 2 infeasible, 3 pass cap

    // prologue: w_i
    for (long long i = i0 + tid; i < i1; i += kPT) {
        double zz = A.z[i] + A.c[i];
        if (A.dz) zz = fma(A.t, A.dz[i], zz);
        A.w_out[i] = fma(-A.sigma, zz, A.x[i]);
    }
    // the search state (thread 0 of every block keeps an identical copy)
    double lam = 0.0, L = -INFINITY, U = INFINITY;
    if (tid == 0) {
        double l0 = A.lam0 ? __ldcg(A.lam0) : 0.0;
        lam = isfinite(l0) ? l0 : 0.0;
        s_lam = lam;
        s_state = 0;
    }
    __syncthreads();
    int pass = 0, pass_all = 0;   // pass: thread 0's count; pass_all: every thread's
    while (true) {
        const double lm = s_lam;
        double f = 0.0, fa = 0.0, sp = 0.0, smn = 0.0, dh = INFINITY, dl = -INFINITY;
        for (long long i = i0 + tid; i < i1; i += kPT) {
            const Comp o = comp_at(A.w_out[i], A.a[i], A.ainv[i], A.lo[i], A.hi[i], lm);
            f += o.fa;
            fa += fabs(o.fa);
            if (o.fr) sp = fma(A.a[i], A.a[i], sp);
            if (o.fl) smn = fma(A.a[i], A.a[i], smn);
            if (A.a[i] != 0.0) {
                if (o.o1 > 0.0) dh = fmin(dh, o.o1); else if (o.o1 < 0.0) dl = fmax(dl, o.o1);
                if (o.o2 > 0.0) dh = fmin(dh, o.o2); else if (o.o2 < 0.0) dl = fmax(dl, o.o2);
            }
        }
        f = warp_sum(f); fa = warp_sum(fa); sp = warp_sum(sp); smn = warp_sum(smn);
        dh = warp_min(dh); dl = warp_max(dl);
        if (lane == 0) {
            sh[warp][0] = f; sh[warp][1] = fa; sh[warp][2] = sp; sh[warp][3] = smn; sh[warp][4] = dh; sh[warp][5] = dl;
        }
        __syncthreads();
        if (tid == 0) {
            double t6[6] = {0.0, 0.0, 0.0, 0.0, INFINITY, -INFINITY};
            for (int w = 0; w < kPW; ++w) {
                t6[0] += sh[w][0]; t6[1] += sh[w][1]; t6[2] += sh[w][2]; t6[3] += sh[w][3];
                t6[4] = fmin(t6[4], sh[w][4]); t6[5] = fmax(t6[5], sh[w][5]);
            }
            // two buffers: a block can start the next pass while others still read this one
            double *p = A.part + ((size_t)(pass_all & 1) * G + blockIdx.x) * kRecStride;
            for (int k = 0; k < 6; ++k) p[k] = t6[k];
        }
        if (!grid_barrier(A.bar, A.err)) return;
        double tot[6];
        if (warp == 0) reduce_pass(A.part + (size_t)(pass_all & 1) * G * kRecStride, G, tot);
        ++pass_all;
        if (tid == 0) {
            ++pass;
            const double F = tot[0] - A.d;
            double nl = lm;
            int state = 0;
            if (F == 0.0) {
                state = 1;
            } else {
                const bool right = F > 0.0;   // f decreases with lambda: the root lies to the right
                if (right) L = fmax(L, lm); else U = fmin(U, lm);
                const double sd = right ? tot[2] : tot[3];     // one-sided slope (sum of a_i^2)
                const double edge = right ? tot[4] : tot[5];   // offset of the nearest breakpoint that way
                if (sd > 0.0) {
                    const double step = F / sd;
                    nl = lm + step;
                    if (right ? step <= edge : step >= edge) state = 1;   // inside the piece: the root
                } else if (isfinite(edge)) {
                    nl = lm + edge;   // flat piece: go to its end
                } else {
                    state = 2;        // f never reaches d on that side: the set is empty
                }
                if (state == 0) {
                    const bool both = isfinite(L) && isfinite(U);
                    if (both && (!(L < nl && nl < U) || pass % 3 == 0)) nl = 0.5 * (L + U);
                    if (both && !(L < nl && nl < U)) {
                        nl = L;       // the bracket is two adjacent doubles
                        state = 1;
                    } else if (nl == lm) {
                        nl = nextafter(lm, right ? INFINITY : -INFINITY);   // a step below rounding
                    }
                    if (state == 0 && pass >= kMaxPass) state = 3;
                }
            }
            s_lam = nl;
            s_state = state;
        }
        __syncthreads();
        if (s_state != 0) break;
    }
    const double lh = s_lam;
    const int state = s_state;

    // final phase: pi, sums, free flags, counts
    double dpx = 0.0, psi = 0.0, xx = 0.0, cx = 0.0, sJ = 0.0, feas = 0.0;
    long long pc = 0, nfx = 0;
    for (long long i = i0 + tid; i < i1; i += kPT) {
        const double w = A.w_out[i], a = A.a[i], lo = A.lo[i], hi = A.hi[i];
        const double r = shifted(w, lh, a);
        const double pi = r >= hi ? hi : (r <= lo ? lo : r);
        A.pi_out[i] = pi;
        const double xi = A.x[i];
        dpx = fma(pi - xi, pi - xi, dpx);
        double ps = pi * (2.0 * w - pi);
        if (A.pib) ps -= A.pib[i] * (2.0 * A.wb[i] - A.pib[i]);
        psi += ps;
        xx = fma(xi, xi, xx);
        cx = fma(A.c[i], xi, cx);
        feas = fma(a, xi, feas);
        if (r > lo && r < hi) {
            ++pc;
            sJ = fma(a, a, sJ);
        }
        nfx += (xi > lo && xi < hi) ? 1 : 0;
    }
    {
        dpx = warp_sum(dpx); psi = warp_sum(psi); xx = warp_sum(xx); cx = warp_sum(cx); sJ = warp_sum(sJ);
        feas = warp_sum(feas);
        pc = warp_sum_ll(pc); nfx = warp_sum_ll(nfx);
        __syncthreads();
        if (lane == 0) {
            sh[warp][0] = dpx; sh[warp][1] = psi; sh[warp][2] = xx; sh[warp][3] = cx; sh[warp][4] = sJ;
            sh[warp][5] = feas; sh[warp][6] = (double)pc; sh[warp][7] = (double)nfx;
        }
        __syncthreads();
        if (tid == 0) {
            double t8[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            for (int w = 0; w < kPW; ++w)
                for (int k = 0; k < 8; ++k) t8[k] += sh[w][k];
            double *p = A.part + ((size_t)2 * G + blockIdx.x) * kRecStride;
            for (int k = 0; k < 8; ++k) p[k] = t8[k];
            A.cnt[blockIdx.x] = (long long)t8[6];
        }
    }
    if (!grid_barrier(A.bar, A.err)) return;
    // compaction of J in ascending order: block offset, then warp ballots per tile
    if (A.J) {
        __shared__ long long s_base;
        __shared__ int s_wc[kPW];
        if (tid == 0) {
            long long off = 0;
            for (int b = 0; b < (int)blockIdx.x; ++b) off += __ldcg(A.cnt + b);
            s_base = off;
        }
        __syncthreads();
        for (long long t0 = i0; t0 < i1; t0 += kPT) {
            const long long i = t0 + tid;
            bool fr = false;
            if (i < i1) {
                const double r = shifted(A.w_out[i], lh, A.a[i]);
                fr = r > A.lo[i] && r < A.hi[i];
            }
            const unsigned bal = __ballot_sync(0xffffffffu, fr);
            if (lane == 0) s_wc[warp] = __popc(bal);
            __syncthreads();
            long long pos = s_base;
            for (int w = 0; w < warp; ++w) pos += s_wc[w];
            if (fr) A.J[pos + __popc(bal & ((1u << lane) - 1u))] = (int32_t)i;
            __syncthreads();
            if (tid == 0) {
                long long tt = 0;
                for (int w = 0; w < kPW; ++w) tt += s_wc[w];
                s_base += tt;
            }
            __syncthreads();
        }
    }
    if (blockIdx.x == 0 && tid == 0) {
        double t8[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int b = 0; b < G; ++b)
            for (int k = 0; k < 8; ++k) t8[k] += __ldcg(A.part + ((size_t)2 * G + b) * kRecStride + k);
        ProjRec R;
        R.lam = lh;
        R.dpx = t8[0]; R.psi = t8[1]; R.xx = t8[2]; R.cx = t8[3]; R.sJ = t8[4]; R.feas = t8[5] - A.d;
        R.p = (long long)t8[6];
        R.nfree_x = (long long)t8[7];
        R.passes = pass;
        R.status = state == 2 ? 2 : (state == 3 ? 1 : 0);
        *A.rec = R;
        if (A.lam_out) *A.lam_out = lh;   // every block read lam0 before the first grid barrier
    }
}

cudaError_t project(Ws &W, const ProjReq &r)
{
    PArgs A;
    A.n = W.n; A.x = r.x; A.z = r.z; A.dz = r.dz; A.c = W.c; A.a = W.a; A.ainv = W.ainv; A.lo = W.lo; A.hi = W.hi;
    A.sigma = r.sigma; A.t = r.t; A.d = W.d; A.lam0 = r.lam0; A.lam_out = r.lam_out; A.w_out = r.w_out; A.pi_out = r.pi_out; A.J = r.J;
    A.pib = r.pib; A.wb = r.wb; A.part = W.part; A.cnt = W.cnt; A.bar = W.bar; A.err = W.err; A.rec = W.rec;
    void *args[] = {&A};
    return cudaLaunchCooperativeKernel((const void *)proj_kernel, dim3(W.proj_grid), dim3(kPT), args, 0, W.st);
}

// ---------------------------------------------------------------- Newton

// Split-K Gram of the free rows: block (tile, k) accumulates the 32 x 32
// tile (ti <= tj) of sum_{r in chunk k} b_r b_r' over its share of J; blocks of
// diagonal tiles also accumulate h = sum a_r b_r for their columns.  Rows are
// staged 32 at a time in shared memory; each thread owns 4 entries.
template <typename T>
__global__ void __launch_bounds__(256) gram_kernel(const void *__restrict__ X, long long m, int q, int layout,
                                                   const double *__restrict__ a, const int32_t *__restrict__ J,
                                                   long long p, int ks, double *__restrict__ part,
                                                   double *__restrict__ hpart)
{
    const int nt = (q + kGT - 1) / kGT;
    int t = blockIdx.x, ti = 0;
    while (t >= nt - ti) { t -= nt - ti; ++ti; }
    const int tj = ti + t;
    const long long per = (p + ks - 1) / ks;
    const long long r0 = (long long)blockIdx.y * per;
    const long long r1 = r0 + per < p ? r0 + per : p;
    __shared__ double Ra[kGRows][kGT + 1], Rb[kGRows][kGT + 1];
    __shared__ double wr[kGRows];
    const int tid = threadIdx.x;
    const int ea = tid >> 3;          // row of the tile: 0..31
    const int eb0 = (tid & 7) * 4;    // 4 consecutive columns
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    double hacc = 0.0;
    for (long long rb = r0; rb < r1; rb += kGRows) {
        const int nr = (int)(r1 - rb < kGRows ? r1 - rb : kGRows);
        for (int e = tid; e < kGRows * kGT; e += 256) {
            const int rr = e / kGT, cc = e % kGT;
            double va = 0.0, vb = 0.0;
            if (rr < nr) {
                const long long gi = J[rb + rr];
                const long long row = (layout == STACKED && gi >= m) ? gi - m : gi;
                const int ca = ti * kGT + cc, cb = tj * kGT + cc;
                if (ca < q) va = ldx<T>(X, row * (long long)q + ca);
                if (cb < q) vb = ldx<T>(X, row * (long long)q + cb);
            }
            Ra[rr][cc] = va;
            Rb[rr][cc] = vb;
        }
        if (tid < kGRows) {
            double wv = 0.0;
            if (tid < nr) {
                const long long gi = J[rb + tid];
                wv = a[gi];
                if (layout == STACKED && gi >= m) wv = -wv;   // row sign of B = [X; -X]
            }
            wr[tid] = wv;
        }
        __syncthreads();
        for (int rr = 0; rr < nr; ++rr) {
            const double xa = Ra[rr][ea];
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[k] = fma(xa, Rb[rr][eb0 + k], acc[k]);
        }
        if (ti == tj && tid < kGT)
            for (int rr = 0; rr < nr; ++rr) hacc = fma(wr[rr], Ra[rr][tid], hacc);
        __syncthreads();
    }
    double *P = part + (size_t)blockIdx.y * q * q;
    const int ga = ti * kGT + ea;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int gb = tj * kGT + eb0 + k;
        if (ga < q && gb < q) P[(size_t)ga * q + gb] = acc[k];
    }
    if (ti == tj && tid < kGT && ti * kGT + tid < q) hpart[(size_t)blockIdx.y * q + ti * kGT + tid] = hacc;
}

// M = I + sigma (G - h h'/s): partials summed in block order; the tile
// holding (a, b) is (min, max) of their tiles, read transposed below the diagonal.
__global__ void build_m_kernel(int q, int ks, const double *__restrict__ part, const double *__restrict__ hpart,
                               double sJ, double sigma, double *__restrict__ M)
{
    const long long qq = (long long)q * q;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < qq; e += (long long)gridDim.x * blockDim.x) {
        const int ra = (int)(e / q), cb = (int)(e % q);
        const bool lower = ra / kGT > cb / kGT;
        const long long src = lower ? (long long)cb * q + ra : e;
        double g = 0.0, ha = 0.0, hb = 0.0;
        for (int k = 0; k < ks; ++k) {
            g += part[(size_t)k * qq + src];
            ha += hpart[(size_t)k * q + ra];
            hb += hpart[(size_t)k * q + cb];
        }
        double v = g;
        if (sJ > 0.0) v -= ha * hb / sJ;
        v *= sigma;
        if (ra == cb) v += 1.0;
        M[e] = v;
    }
}

__global__ void negcopy_kernel(int q, const double *__restrict__ g, double *__restrict__ dv)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < q; j += gridDim.x * blockDim.x) dv[j] = -g[j];
}

cudaError_t newton(Ws &W, const int32_t *J, long long p, double sJ, double sigma, const double *g, double *dv,
                   double *M)
{
    const int q = W.q;
    if (p <= 0) {
        negcopy_kernel<<<1, 1024, 0, W.st>>>(q, g, dv);   // case (b) of Prop. 3.5: P = 0
        return cudaGetLastError();
    }
    const int nt = (q + kGT - 1) / kGT;
    const int ntiles = nt * (nt + 1) / 2;
    const size_t qq = (size_t)q * q;
    long long ks = (p + 255) / 256;
    long long ks_cap = (long long)(W.part_len / (qq + q));
    if (ks_cap > 4 * W.nsm) ks_cap = 4 * W.nsm;
    if (ks > ks_cap) ks = ks_cap;
    if (ks < 1) ks = 1;
    double *part = W.part, *hpart = W.part + (size_t)ks * qq;
    dim3 grid(ntiles, (unsigned)ks);
    if (W.xf32)
        gram_kernel<float><<<grid, 256, 0, W.st>>>(W.X, W.m, q, W.layout, W.a, J, p, (int)ks, part, hpart);
    else
        gram_kernel<double><<<grid, 256, 0, W.st>>>(W.X, W.m, q, W.layout, W.a, J, p, (int)ks, part, hpart);
    build_m_kernel<<<W.nsm * 2, 256, 0, W.st>>>(q, (int)ks, part, hpart, sJ, sigma, M);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_chol_solve(q, M, g, dv, W.err, W.st);
}

// ---------------------------------------------------------------- q- and n-vectors

__global__ void __launch_bounds__(1024) qvec_kernel(int q, const double *__restrict__ v, const double *__restrict__ btp,
                                                    double *__restrict__ g, const double *__restrict__ dv,
                                                    double *__restrict__ red)
{
    __shared__ double sh[4][32];
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    for (int j = threadIdx.x; j < q; j += blockDim.x) {
        if (btp) {
            const double gj = v[j] - btp[j];
            g[j] = gj;
            s3 = fma(gj, gj, s3);
        }
        if (dv) {
            const double dj = dv[j];
            s0 = fma(g[j], dj, s0);
            s1 = fma(v[j], dj, s1);
            s2 = fma(dj, dj, s2);
        }
    }
    s0 = warp_sum(s0); s1 = warp_sum(s1); s2 = warp_sum(s2); s3 = warp_sum(s3);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) { sh[0][w] = s0; sh[1][w] = s1; sh[2][w] = s2; sh[3][w] = s3; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t[4] = {0, 0, 0, 0};
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k)
            for (int r = 0; r < 4; ++r) t[r] += sh[r][k];
        if (dv) { red[0] = t[0]; red[1] = t[1]; red[2] = t[2]; }
        if (btp) red[3] = t[3];
    }
}

cudaError_t qvec(Ws &W, const double *v, const double *btp, double *g, const double *dv, double *red)
{
    qvec_kernel<<<1, 1024, 0, W.st>>>(W.q, v, btp, g, dv, red);
    return cudaGetLastError();
}

__global__ void axpy_kernel(long long n, double *__restrict__ z, double t, const double *__restrict__ dz)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        z[i] = fma(t, dz[i], z[i]);
}

cudaError_t axpy_q(Ws &W, double *v, double t, const double *dv)
{
    axpy_kernel<<<1, 1024, 0, W.st>>>(W.q, v, t, dv);
    return cudaGetLastError();
}

cudaError_t axpy_n(Ws &W, double *z, double t, const double *dz)
{
    axpy_kernel<<<W.nsm * 4, 256, 0, W.st>>>(W.n, z, t, dz);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- set-up

__global__ void ainv_kernel(long long n, const double *__restrict__ a, double *__restrict__ ainv)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        ainv[i] = a[i] != 0.0 ? 1.0 / a[i] : 0.0;
}

template <typename T>
__global__ void validate_kernel(const void *__restrict__ X, long long nx, long long n, const double *__restrict__ c,
                                const double *__restrict__ a, const double *__restrict__ lo,
                                const double *__restrict__ hi, int *flags)
{
    int bx = 0, bv = 0, bb = 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nx; k += stride)
        if (!isfinite(ldx<T>(X, k))) bx = 1;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride) {
        if (!isfinite(c[i]) || !isfinite(a[i]) || !isfinite(lo[i]) || !isfinite(hi[i])) bv = 1;
        if (lo[i] > hi[i]) bb = 1;
    }
    if (bx) atomicOr(flags + 0, 1);
    if (bv) atomicOr(flags + 1, 1);
    if (bb) atomicOr(flags + 2, 1);
}

cudaError_t validate(Ws &W, int *flags)
{
    const long long nx = W.m * (long long)W.q;
    if (W.xf32)
        validate_kernel<float><<<W.nsm * 4, 256, 0, W.st>>>(W.X, nx, W.n, W.c, W.a, W.lo, W.hi, flags);
    else
        validate_kernel<double><<<W.nsm * 4, 256, 0, W.st>>>(W.X, nx, W.n, W.c, W.a, W.lo, W.hi, flags);
    return cudaGetLastError();
}

__global__ void svr_kernel(long long m, const double *__restrict__ y, double eps, double C, double *__restrict__ c,
                           double *__restrict__ a, double *__restrict__ lo, double *__restrict__ hi)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x) {
        const double yi = y[i];
        c[i] = eps + yi;
        c[m + i] = eps - yi;
        a[i] = 1.0;
        a[m + i] = -1.0;
        lo[i] = lo[m + i] = 0.0;
        hi[i] = hi[m + i] = C;
    }
}

cudaError_t svr_vectors(Ws &W, const double *y, double eps, double C, double *c, double *a, double *lo, double *hi)
{
    svr_kernel<<<W.nsm * 4, 256, 0, W.st>>>(W.m, y, eps, C, c, a, lo, hi);
    return cudaGetLastError();
}

cudaError_t setup(Ws &W)
{
    int occ = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, proj_kernel, kPT, 0);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    if (occ > 2) occ = 2;
    long long want = (W.n + kPT * 4 - 1) / (kPT * 4);   // at least ~4 elements per thread
    if (want < 1) want = 1;
    W.proj_grid = (int)(want < (long long)W.nsm * occ ? want : (long long)W.nsm * occ);
    long long rg = (W.m + 63) / 64;
    if (rg > 4LL * W.nsm) rg = 4LL * W.nsm;
    W.rm_grid = (int)(rg < 1 ? 1 : rg);
    ainv_kernel<<<W.nsm * 4, 256, 0, W.st>>>(W.n, W.a, W.ainv);
    return cudaGetLastError();
}

}  // namespace gqp
}  // namespace svm
