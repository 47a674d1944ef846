// k_proj.cu -- projection onto {x : y'x = 0, 0 <= x <= C} (Sec. 3.2.1):
// the multiplier lambda-hat, the clipped point pi, the free set J and the
// support S, in one cooperative launch.
//
// The paper finds lambda-hat by sorting the 2n breakpoints and bisecting on
// their index (Algorithm 2).  A sort per projection is the wrong shape for
// this GPU; instead each block keeps its slice of s_i = y_i u_i in registers
// and all blocks run, in lock-step, a safeguarded Newton iteration on the
// monotone piecewise-linear function f(lambda) = sum_i y_i clip(u_i - lambda
// y_i, 0, C) (= -grad phi of Sec. 3.2.1).  One pass reduces f, the one-sided
// slopes (free counts on each side) and the nearest breakpoint on each side;
// a Newton step that stays inside the current linear piece lands exactly on
// the root, otherwise the bracket shrinks (secant, then bisection, as
// safeguards).  The result is the same lambda-hat as Algorithm 2 up to
// rounding (and any point of the flat piece when the root set is an interval;
// pi is the same either way).  Ties follow the paper's clip: t >= C -> C,
// t <= 0 -> 0, so J uses strict inequalities.
#include <math.h>

#include "internal.cuh"

namespace svm {

constexpr int kMaxPass = 96;
constexpr int kPartStride = 8;   // doubles per block partial

struct ProjArgs {
    const double *a, *b;
    double c0, c1, c2;
    const int8_t *y;
    long long n;
    double C;
    int mode;
    const double *lam0;
    double *u_out, *pi_out;
    int32_t *J, *S;
    const double *pi_base;
    const double *alpha;
    double *part;      // [3][G][kPartStride]
    int *cnt;          // [EPT][G][2]
    unsigned *bar;
    int *err;
    ProjOut *out;
};

// Fixed-order reduction of the G block partials of one slot; every block
// calls it on the same data and gets bit-identical results.
__device__ __forceinline__ void reduce_partials(const double *slot, int G, double *tot)
{
    // warp 0 only; tot[0]=sum f, [1]=max blo, [2]=min bhi, [3]=sum pp, [4]=sum pm
    const int lane = threadIdx.x & 31;
    double F = 0.0, blo = -INFINITY, bhi = INFINITY, pp = 0.0, pm = 0.0;
    for (int bb = lane; bb < G; bb += 32) {
        const double *p = slot + (size_t)bb * kPartStride;
        F += __ldcg(p + 0);
        blo = fmax(blo, __ldcg(p + 1));
        bhi = fmin(bhi, __ldcg(p + 2));
        pp += __ldcg(p + 3);
        pm += __ldcg(p + 4);
    }
    F = warp_sum(F);
    blo = warp_max(blo);
    bhi = warp_min(bhi);
    pp = warp_sum(pp);
    pm = warp_sum(pm);
    tot[0] = F; tot[1] = blo; tot[2] = bhi; tot[3] = pp; tot[4] = pm;
}

template <int EPT>
__global__ void __launch_bounds__(kTPB) proj_kernel(ProjArgs A)
{
    const int G = gridDim.x, blk = blockIdx.x, tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const long long NT = (long long)G * kTPB;
    const double C = A.C;

    double s[EPT];
    float ys[EPT];
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
        long long i = k * NT + (long long)blk * kTPB + tid;
        if (i < A.n) {
            double u = A.c0 * A.a[i] + A.c2;
            if (A.b) u = fma(A.c1, A.b[i], u);
            float yy = (float)A.y[i];
            s[k] = (yy > 0.f) ? u : -u;
            ys[k] = yy;
        } else {
            s[k] = 0.0;
            ys[k] = 0.f;
        }
    }

    __shared__ double sh_d[kWarps][3];
    __shared__ double sh_c[kWarps][2];
    __shared__ double sh_tot[5];
    __shared__ double sh_lam;
    __shared__ int sh_done;

    double lam = A.lam0 ? __ldcg(A.lam0) : 0.0;
    if (!isfinite(lam)) lam = 0.0;
    // bracket: f(L) > 0 > f(U)
    double L = -INFINITY, U = INFINITY, FL = 0.0, FU = 0.0;
    double lam_hat = lam;
    int pass = 0;
    bool alive = true;

    for (;;) {
        double F = 0.0, blo = -INFINITY, bhi = INFINITY, pp = 0.0, pm = 0.0;
#pragma unroll
        for (int k = 0; k < EPT; ++k) {
            if (ys[k] != 0.f) {
                const bool pos = ys[k] > 0.f;
                double t = pos ? (s[k] - lam) : (lam - s[k]);
                double pk = fmin(fmax(t, 0.0), C);
                F += pos ? pk : -pk;
                bool open = (t > 0.0) && (t < C);
                bool at0 = (t == 0.0), atC = (t == C);
                // one-sided free counts: right (lambda + eps) and left (lambda - eps)
                pp += (open || (pos ? atC : at0)) ? 1.0 : 0.0;
                pm += (open || (pos ? at0 : atC)) ? 1.0 : 0.0;
                double b1 = pos ? s[k] - C : s[k];
                double b2 = pos ? s[k] : s[k] + C;
                if (b1 > lam) bhi = fmin(bhi, b1); else if (b1 < lam) blo = fmax(blo, b1);
                if (b2 > lam) bhi = fmin(bhi, b2); else if (b2 < lam) blo = fmax(blo, b2);
            }
        }
        F = warp_sum(F);
        blo = warp_max(blo);
        bhi = warp_min(bhi);
        pp = warp_sum(pp);
        pm = warp_sum(pm);
        if (lane == 0) {
            sh_d[warp][0] = F; sh_d[warp][1] = blo; sh_d[warp][2] = bhi;
            sh_c[warp][0] = pp; sh_c[warp][1] = pm;
        }
        __syncthreads();
        if (tid == 0) {
            double bF = 0.0, bl = -INFINITY, bh = INFINITY, bp = 0.0, bm = 0.0;
            for (int w = 0; w < kWarps; ++w) {
                bF += sh_d[w][0]; bl = fmax(bl, sh_d[w][1]); bh = fmin(bh, sh_d[w][2]);
                bp += sh_c[w][0]; bm += sh_c[w][1];
            }
            double *p = A.part + ((size_t)(pass & 1) * G + blk) * kPartStride;
            p[0] = bF; p[1] = bl; p[2] = bh; p[3] = bp; p[4] = bm;
        }
        if (!grid_barrier(A.bar, A.err)) { alive = false; break; }
        if (warp == 0) {
            double tot[5];
            reduce_partials(A.part + (size_t)(pass & 1) * G * kPartStride, G, tot);
            if (lane == 0) {
                for (int f = 0; f < 5; ++f) sh_tot[f] = tot[f];
                // ---- decision (identical in every block) ----
                double Ft = tot[0], bl = tot[1], bh = tot[2], pr = tot[3], pl = tot[4];
                int done = 0;
                double next = lam;
                if (Ft == 0.0) {
                    done = 1; lam_hat = lam;
                } else if (Ft > 0.0) {
                    L = lam; FL = Ft;
                    if (pr > 0.0) {
                        double lN = lam + Ft / pr;
                        if (lN <= bh) { done = 1; lam_hat = lN; }
                        else next = lN;
                    } else {
                        next = bh;
                    }
                } else {
                    U = lam; FU = Ft;
                    if (pl > 0.0) {
                        double lN = lam + Ft / pl;
                        if (lN >= bl) { done = 1; lam_hat = lN; }
                        else next = lN;
                    } else {
                        next = bl;
                    }
                }
                if (!done) {
                    if (!(next > L && next < U)) {
                        if (isfinite(L) && isfinite(U)) {
                            next = L - FL * (U - L) / (FU - FL);
                            if (!(next > L && next < U)) next = 0.5 * (L + U);
                        }
                    }
                    if (!(next > L && next < U) || !isfinite(next)) {
                        // no representable point strictly inside the bracket
                        done = 1;
                        lam_hat = (isfinite(L) && (!isfinite(U) || fabs(FL) <= fabs(FU))) ? L : U;
                        if (!isfinite(lam_hat)) lam_hat = lam;
                    } else if (pass + 1 >= kMaxPass) {
                        done = 1;
                        lam_hat = next;
                        if (blk == 0) set_err(A.err, DEV_ROOT);
                    }
                }
                sh_done = done;
                sh_lam = done ? lam_hat : next;
            }
        }
        __syncthreads();
        ++pass;
        if (sh_done) { lam_hat = sh_lam; break; }
        lam = sh_lam;
    }

    // ---------------- final phase: pi, sums, compaction ----------------
    const double lh = lam_hat;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    unsigned isJ = 0u, isS = 0u;   // bit k: element k is in J / S
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
        if (ys[k] == 0.f) continue;
        long long i = k * NT + (long long)blk * kTPB + tid;
        const bool pos = ys[k] > 0.f;
        double t = pos ? (s[k] - lh) : (lh - s[k]);
        double pk = fmin(fmax(t, 0.0), C);
        double u = pos ? s[k] : -s[k];
        if (t > 0.0 && t < C) isJ |= 1u << k;
        if (pk > 0.0) isS |= 1u << k;
        if (A.pi_out) A.pi_out[i] = pk;
        if (A.mode == PM_MAIN) {
            if (A.u_out) A.u_out[i] = u;
            double al = A.alpha[i];
            double d = pk - al;
            acc[0] = fma(d, d, acc[0]);
            acc[1] += pk * (2.0 * u - pk);
        } else if (A.mode == PM_TRIAL) {
            double ub = A.a[i], pb = A.pi_base[i];
            acc[0] += pk * (2.0 * u - pk) - pb * (2.0 * ub - pb);
        } else if (A.mode == PM_KKT) {
            double al = A.a[i];
            double d = al - pk;
            acc[0] = fma(d, d, acc[0]);
            acc[1] = fma(al, al, acc[1]);
            acc[2] += al;
            double qa = A.b[i];
            double marg = qa + (pos ? lh : -lh);
            acc[3] += fmax(0.0, 1.0 - marg);
        }
    }
    // per-(k, warp) compaction counts
    __shared__ int sh_wc[EPT > 0 ? EPT : 1][kWarps][2];
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
        unsigned bj = __ballot_sync(0xffffffffu, (isJ >> k) & 1u);
        unsigned bs = __ballot_sync(0xffffffffu, (isS >> k) & 1u);
        if (lane == 0) { sh_wc[k][warp][0] = __popc(bj); sh_wc[k][warp][1] = __popc(bs); }
    }
#pragma unroll
    for (int f = 0; f < 4; ++f) acc[f] = warp_sum(acc[f]);
    if (lane == 0) {
        sh_d[warp][0] = acc[0]; sh_d[warp][1] = acc[1]; sh_d[warp][2] = acc[2];
        sh_c[warp][0] = acc[3];
    }
    __syncthreads();
    if (tid < EPT) {
        int cj = 0, cs = 0;
        for (int w = 0; w < kWarps; ++w) { cj += sh_wc[tid][w][0]; cs += sh_wc[tid][w][1]; }
        A.cnt[((size_t)tid * G + blk) * 2 + 0] = cj;
        A.cnt[((size_t)tid * G + blk) * 2 + 1] = cs;
    }
    if (tid == 0) {
        double b0 = 0, b1 = 0, b2 = 0, b3 = 0;
        for (int w = 0; w < kWarps; ++w) { b0 += sh_d[w][0]; b1 += sh_d[w][1]; b2 += sh_d[w][2]; b3 += sh_c[w][0]; }
        double *p = A.part + ((size_t)2 * G + blk) * kPartStride;
        p[0] = b0; p[1] = b1; p[2] = b2; p[3] = b3;
    }
    if (!alive || !grid_barrier(A.bar, A.err)) return;

    // offsets: off(k) = sum_{k'<k} total(k') + sum_{b'<blk} cnt(k, b')
    __shared__ long long sh_off[EPT > 0 ? EPT : 1][2];
    __shared__ long long sh_tot2[EPT > 0 ? EPT : 1][2];
    for (int k = warp; k < EPT; k += kWarps) {
        long long tj = 0, ts = 0, pj = 0, ps = 0;
        for (int bb = lane; bb < G; bb += 32) {
            int cj = __ldcg(A.cnt + ((size_t)k * G + bb) * 2 + 0);
            int cs = __ldcg(A.cnt + ((size_t)k * G + bb) * 2 + 1);
            tj += cj; ts += cs;
            if (bb < blk) { pj += cj; ps += cs; }
        }
        tj = warp_sum_ll(tj); ts = warp_sum_ll(ts);
        pj = warp_sum_ll(pj); ps = warp_sum_ll(ps);
        if (lane == 0) { sh_tot2[k][0] = tj; sh_tot2[k][1] = ts; sh_off[k][0] = pj; sh_off[k][1] = ps; }
    }
    __syncthreads();
    if (tid == 0) {
        long long rj = 0, rs = 0;
        for (int k = 0; k < EPT; ++k) {
            long long oj = rj + sh_off[k][0], os = rs + sh_off[k][1];
            rj += sh_tot2[k][0]; rs += sh_tot2[k][1];
            sh_off[k][0] = oj; sh_off[k][1] = os;
        }
        if (blk == 0) {
            // block 0 publishes the results
            double r0 = 0, r1 = 0, r2 = 0, r3 = 0;
            for (int bb = 0; bb < G; ++bb) {
                const double *p = A.part + ((size_t)2 * G + bb) * kPartStride;
                r0 += __ldcg(p + 0); r1 += __ldcg(p + 1); r2 += __ldcg(p + 2); r3 += __ldcg(p + 3);
            }
            A.out->lam = lam_hat;
            A.out->sum[0] = r0; A.out->sum[1] = r1; A.out->sum[2] = r2; A.out->sum[3] = r3;
            A.out->p = rj;
            A.out->s = rs;
            A.out->passes = pass;
            A.out->status = 0;
        }
    }
    __syncthreads();
    if (A.J || A.S) {
        const unsigned lt = (1u << lane) - 1u;
#pragma unroll
        for (int k = 0; k < EPT; ++k) {
            long long i = k * NT + (long long)blk * kTPB + tid;
            unsigned bj = __ballot_sync(0xffffffffu, (isJ >> k) & 1u);
            unsigned bs = __ballot_sync(0xffffffffu, (isS >> k) & 1u);
            int wj = 0, ws = 0;
            for (int w = 0; w < warp; ++w) { wj += sh_wc[k][w][0]; ws += sh_wc[k][w][1]; }
            if (A.J && ((isJ >> k) & 1u)) A.J[sh_off[k][0] + wj + __popc(bj & lt)] = (int32_t)i;
            if (A.S && ((isS >> k) & 1u)) A.S[sh_off[k][1] + ws + __popc(bs & lt)] = (int32_t)i;
        }
    }
}

template <int EPT>
static void *kfun() { return (void *)proj_kernel<EPT>; }

static const int kEpts[] = {1, 2, 4, 8, 16, 32};

static void *kernel_for(int ept)
{
    switch (ept) {
    case 1: return kfun<1>();
    case 2: return kfun<2>();
    case 4: return kfun<4>();
    case 8: return kfun<8>();
    case 16: return kfun<16>();
    default: return kfun<32>();
    }
}

cudaError_t proj_setup(Work &W)
{
    // Largest co-resident grid for each instantiation; pick the smallest EPT
    // whose grid covers n.
    long long n = W.n;
    for (int ept : kEpts) {
        int occ = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel_for(ept), kTPB, 0);
        if (e != cudaSuccess) return e;
        if (occ < 1) continue;
        long long gmax = (long long)occ * W.nsm;
        long long need = (n + (long long)kTPB * ept - 1) / ((long long)kTPB * ept);
        if (need <= gmax) {
            W.proj_grid = (int)(need < 1 ? 1 : need);
            W.proj_ept = ept;
            return cudaSuccess;
        }
    }
    return cudaErrorInvalidValue;   // n too large for register-resident slices
}

cudaError_t launch_project(Work &W, const ProjIn &in, ProjOut *out)
{
    ProjArgs A;
    A.a = in.a; A.b = in.b; A.c0 = in.c0; A.c1 = in.c1; A.c2 = in.c2;
    A.y = W.y; A.n = W.n; A.C = W.C; A.mode = in.mode; A.lam0 = in.lam0;
    A.u_out = in.u_out; A.pi_out = in.pi_out; A.J = in.J; A.S = in.S;
    A.pi_base = in.pi_base; A.alpha = in.alpha;
    A.part = W.part; A.cnt = W.cnt; A.bar = W.bar; A.err = W.err; A.out = out;
    void *args[] = {&A};
    ++W.nlaunch;
    return cudaLaunchCooperativeKernel(kernel_for(W.proj_ept), dim3(W.proj_grid), dim3(kTPB), args, 0,
                                       W.st);
}

}  // namespace svm
