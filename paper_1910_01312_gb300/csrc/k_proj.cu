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
// the root.  Until the root is bracketed the steps grow geometrically; once
// it is, Newton steps inside the bracket alternate with secant steps and a
// forced bisection every third pass, so the bracket shrinks geometrically.
// The result is the same lambda-hat as Algorithm 2 up to rounding (and any
// point of the flat piece when the root set is an interval; pi is the same
// either way).  Ties follow the paper's clip: t >= C -> C, t <= 0 -> 0, so J
// uses strict inequalities.
//
// Precision.  This kernel is the plain form: it reads FP64 vectors and
// evaluates every component in FP64.  The mixed form runs the same iteration
// in double-float arithmetic (k_projdf.cu).
#include <math.h>

#include "internal.cuh"

namespace svm {

constexpr int kMaxPass = 256;
constexpr int kPartStride = 8;   // doubles per block partial

struct ProjArgs {
    const double *a, *b;
    double c1, c2;
    const int8_t *y;
    long long n;
    double C;
    int sums;
    const double *lam0;
    double *u_out;
    double *pi_out;
    float2 *wpi_out;
    int32_t *J, *S;
    const double *pi_base;
    const double *alpha;     // FP64 alpha (SF_DPA, SF_KKT)
    double *part;            // [3][G][kPartStride]
    int *cnt;                // [EPT][G][2]
    unsigned *bar;
    int *err;
    ProjOut *out;
};

struct PassAcc {
    double fex;         // exact part of f over the components evaluated in FP64
    int nup;            // (#upper with y=+1) - (#upper with y=-1): contributes C * nup
    int pp;             // free count just right of lambda
    int pm;             // free count just left of lambda
    int ex;             // some component was evaluated in FP64
    float fdhi, fdlo;   // conservative breakpoint offsets of FP32-classified components
    double ddhi, ddlo;  // breakpoint offsets of FP64-evaluated components
};

__device__ __forceinline__ void acc_init(PassAcc &A)
{
    A.fex = 0.0; A.nup = 0; A.pp = 0; A.pm = 0; A.ex = 0;
    A.fdhi = INFINITY; A.fdlo = -INFINITY; A.ddhi = INFINITY; A.ddlo = -INFINITY;
}

// Exact FP64 evaluation of one component at lambda.  Out of line so that only
// warps with such a component spend FP64 instructions on it.
struct ExactOut {
    double fex, dhi, dlo;
    int nup, pp, pm;
};

__device__ __noinline__ ExactOut eval_exact_ool(double s, bool pos, double lam, double C)
{
    ExactOut o;
    const double t = pos ? (s - lam) : (lam - s);
    o.nup = 0;
    o.fex = 0.0;
    if (t >= C) o.nup = pos ? 1 : -1;
    else if (t > 0.0) o.fex = pos ? t : -t;
    const bool open = (t > 0.0) && (t < C);
    const bool at0 = (t == 0.0), atC = (t == C);
    o.pp = (open || (pos ? atC : at0)) ? 1 : 0;
    o.pm = (open || (pos ? at0 : atC)) ? 1 : 0;
    // breakpoints at offsets (in lambda): y=+1: t, t - C;  y=-1: -t, C - t
    const double o1 = pos ? t : -t, o2 = pos ? t - C : C - t;
    o.dhi = INFINITY;
    o.dlo = -INFINITY;
    if (o1 > 0.0) o.dhi = o1; else if (o1 < 0.0) o.dlo = o1;
    if (o2 > 0.0) o.dhi = fmin(o.dhi, o2); else if (o2 < 0.0) o.dlo = fmax(o.dlo, o2);
    return o;
}

__device__ __forceinline__ void eval_exact(double s, bool pos, double lam, double C, PassAcc &A)
{
    const ExactOut o = eval_exact_ool(s, pos, lam, C);
    A.nup += o.nup;
    A.fex += o.fex;
    A.pp += o.pp;
    A.pm += o.pm;
    A.ex = 1;
    A.ddhi = fmin(A.ddhi, o.dhi);
    A.ddlo = fmax(A.ddlo, o.dlo);
}

// pi component in FP64 and its class (0: = 0, 1: free, 2: = C), out of line
__device__ __noinline__ double clip_exact_ool(double s, bool pos, double lam, double C, int &pc)
{
    const double t = pos ? (s - lam) : (lam - s);
    if (t >= C) { pc = 2; return C; }
    if (t <= 0.0) { pc = 0; return 0.0; }
    pc = 1;
    return t;
}

// Fixed-order reduction of the G block partials of one slot; every block
// calls it on the same data and gets bit-identical results (warp 0 only).
__device__ __forceinline__ void reduce_partials(const double *slot, int G, double *tot)
{
    const int lane = threadIdx.x & 31;
    double F = 0.0, nu = 0.0, pp = 0.0, pm = 0.0, dh = INFINITY, dlo = -INFINITY;
#pragma unroll 8
    for (int bb = lane; bb < G; bb += 32) {
        const double *p = slot + (size_t)bb * kPartStride;
        const double2 a = __ldcg(reinterpret_cast<const double2 *>(p));
        const double2 b = __ldcg(reinterpret_cast<const double2 *>(p + 2));
        const double2 c = __ldcg(reinterpret_cast<const double2 *>(p + 4));
        F += a.x; nu += a.y; pp += b.x; pm += b.y;
        dh = fmin(dh, c.x); dlo = fmax(dlo, c.y);
    }
    tot[0] = warp_sum(F); tot[1] = warp_sum(nu); tot[2] = warp_sum(pp); tot[3] = warp_sum(pm);
    tot[4] = warp_min(dh); tot[5] = warp_max(dlo);
}

__device__ __forceinline__ double flip_sign(double x, bool neg)
{
    return neg ? __longlong_as_double(__double_as_longlong(x) ^ (long long)0x8000000000000000ULL) : x;
}

// FP32 (hi, lo) split of a double
__device__ __forceinline__ float2 dfx_split(double v)
{
    const float hi = (float)v;
    return make_float2(hi, (float)(v - (double)hi));
}

template <int EPT>
__global__ void __launch_bounds__(kTPB, EPT >= 16 ? 1 : 2) proj_kernel(ProjArgs A)
{
    const int G = gridDim.x, blk = blockIdx.x, tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const long long NT = (long long)G * kTPB;
    const double C = A.C;

    // warm start lambda_0: read by one thread per block and broadcast
    __shared__ double sh_lam0;
    if (tid == 0) {
        double l0 = A.lam0 ? __ldcg(A.lam0) : 0.0;
        if (!isfinite(l0)) l0 = 0.0;
        sh_lam0 = l0;
    }
    __syncthreads();
    const double lam0 = sh_lam0;

    double sd[EPT];   // s_i = y_i u_i
    unsigned posm = 0u, valm = 0u;
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
        const long long i = k * NT + (long long)blk * kTPB + tid;
        sd[k] = 0.0;
        if (i < A.n) {
            const bool pos = A.y[i] > 0;
            double u = A.a[i] + A.c2;
            if (A.b) u = fma(A.c1, A.b[i], u);
            sd[k] = flip_sign(u, !pos);
            posm |= (pos ? 1u : 0u) << k;
            valm |= 1u << k;
        }
    }

    __shared__ double sh_d[kWarps][6];
    __shared__ double sh_lam;
    __shared__ int sh_done;

    // root-search state, kept in shared memory (only warp 0 lane 0 updates it)
    __shared__ double st_L, st_U, st_FL, st_FU, st_last_step;
    __shared__ int st_last_dir, st_nbr;
    if (tid == 0) {
        st_L = -INFINITY; st_U = INFINITY; st_FL = 0.0; st_FU = 0.0;   // bracket: f(L) > 0 > f(U)
        st_last_step = 0.0; st_last_dir = 0; st_nbr = 0;
    }
    __syncthreads();
    double lam = lam0;
    double lam_hat = lam;
    int pass = 0;
    bool alive = true;

    for (;;) {
        PassAcc acc;
        acc_init(acc);
#pragma unroll
        for (int k = 0; k < EPT; ++k)
            if ((valm >> k) & 1u) eval_exact(sd[k], (posm >> k) & 1u, lam, C, acc);
        {
            const int nup = __reduce_add_sync(0xffffffffu, acc.nup);
            const int pp = __reduce_add_sync(0xffffffffu, acc.pp);
            const int pm = __reduce_add_sync(0xffffffffu, acc.pm);
            // FP64 reductions only in warps where some lane evaluated a component
            // exactly (in the mixed form most warps have none)
            double fex = 0.0, dh, dlw;
            if (__any_sync(0xffffffffu, acc.ex)) {
                fex = warp_sum(acc.fex);
                dh = warp_min(fmin(acc.ddhi, (double)acc.fdhi));
                dlw = warp_max(fmax(acc.ddlo, (double)acc.fdlo));
            } else {
                float fh = acc.fdhi, fl = acc.fdlo;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    fh = fminf(fh, __shfl_xor_sync(0xffffffffu, fh, o));
                    fl = fmaxf(fl, __shfl_xor_sync(0xffffffffu, fl, o));
                }
                dh = (double)fh;
                dlw = (double)fl;
            }
            if (lane == 0) {
                sh_d[warp][0] = fex; sh_d[warp][1] = (double)nup; sh_d[warp][2] = (double)pp;
                sh_d[warp][3] = (double)pm; sh_d[warp][4] = dh; sh_d[warp][5] = dlw;
            }
        }
        __syncthreads();
        if (warp == 0) {
            const bool v = lane < kWarps;
            const double b0 = warp_sum(v ? sh_d[lane][0] : 0.0), b1 = warp_sum(v ? sh_d[lane][1] : 0.0);
            const double b2 = warp_sum(v ? sh_d[lane][2] : 0.0), b3 = warp_sum(v ? sh_d[lane][3] : 0.0);
            const double b4 = warp_min(v ? sh_d[lane][4] : INFINITY), b5 = warp_max(v ? sh_d[lane][5] : -INFINITY);
            if (lane == 0) {
                double *p = A.part + ((size_t)(pass & 1) * G + blk) * kPartStride;
                p[0] = b0; p[1] = b1; p[2] = b2; p[3] = b3; p[4] = b4; p[5] = b5;
            }
        }
        if (!grid_barrier(A.bar, A.err)) { alive = false; break; }
        if (warp == 0) {
            double tot[6];
            reduce_partials(A.part + (size_t)(pass & 1) * G * kPartStride, G, tot);
            if (lane == 0) {
                // ---- decision (identical in every block) ----
                double &L = st_L, &U = st_U, &FL = st_FL, &FU = st_FU, &last_step = st_last_step;
                int &last_dir = st_last_dir, &nbr = st_nbr;
                const double Ft = tot[0] + C * tot[1];
                const double pr = tot[2], pl = tot[3];
                const double bh = lam + tot[4], bl = lam + tot[5];
                int done = 0;
                double next = lam;
                int dir = 0;
                if (Ft == 0.0) {
                    done = 1; lam_hat = lam;
                } else if (Ft > 0.0) {
                    L = lam; FL = Ft; dir = 1;
                    if (pr > 0.0) {
                        const double lN = lam + Ft / pr;
                        if (lN <= bh) { done = 1; lam_hat = lN; }
                        else next = lN;
                    } else {
                        next = lam + 2.0 * (bh - lam);   // flat piece: go past its end
                    }
                } else {
                    U = lam; FU = Ft; dir = -1;
                    if (pl > 0.0) {
                        const double lN = lam + Ft / pl;
                        if (lN >= bl) { done = 1; lam_hat = lN; }
                        else next = lN;
                    } else {
                        next = lam + 2.0 * (bl - lam);
                    }
                }
                if (!done) {
                    if (!isfinite(L) || !isfinite(U)) {
                        // not bracketed yet: steps in one direction at least double
                        double step = next - lam;
                        if (dir == last_dir && fabs(step) < 2.0 * last_step) step = dir * 2.0 * last_step;
                        next = lam + step;
                        last_step = fabs(step);
                        last_dir = dir;
                    } else {
                        // bracketed: Newton point if inside, else secant; every third
                        // bracketed pass bisects, so the bracket at least halves
                        ++nbr;
                        if (nbr % 3 == 0) next = 0.5 * (L + U);
                        else if (!(next > L && next < U)) {
                            next = L - FL * (U - L) / (FU - FL);
                            if (!(next > L && next < U)) next = 0.5 * (L + U);
                        }
                    }
                    if (!isfinite(next) || ((isfinite(L) && isfinite(U)) && !(next > L && next < U))) {
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
    const float Cf = (float)C;
    const float2 Csplit = make_float2(Cf, (float)(C - (double)Cf));
    const long long Cbits = __double_as_longlong(C);
    double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0, acc3 = 0.0;
    unsigned isJ = 0u, isS = 0u;          // bit k: component k is in J / S
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
        if (!((valm >> k) & 1u)) continue;
        const long long i = k * NT + (long long)blk * kTPB + tid;
        const bool pos = (posm >> k) & 1u;
        int pc;   // class of pk: 0 (= 0), 1 (free), 2 (= C)
        const double pk = clip_exact_ool(sd[k], pos, lh, C, pc);
        if (pc == 1) isJ |= 1u << k;
        if (pc) isS |= 1u << k;
        if (A.pi_out) A.pi_out[i] = pk;
        if (A.wpi_out) {
            // y_i pi_i as an FP32 (hi, lo) pair, the weight of the mixed-form A'pi
            const float2 pkf = (pc == 2) ? Csplit : ((pc == 0) ? make_float2(0.f, 0.f) : dfx_split(pk));
            A.wpi_out[i] = pos ? pkf : make_float2(-pkf.x, -pkf.y);
        }
        const double u = flip_sign(sd[k], !pos);
        if (A.u_out) A.u_out[i] = u;
        if (A.sums & SF_DPA) {
            // |pi - alpha|^2: only components that moved need FP64
            const double al = A.alpha[i];
            if (__double_as_longlong(al) != __double_as_longlong(pk)) {
                const double d = pk - al;
                acc0 = fma(d, d, acc0);
            }
        }
        if (A.sums & SF_PSID) {
            // psi difference term by term in the multiplier-stationary form of
            // k_projdf.cu: pi^2 when free, C (2 (u - lambda y) - C) at C, 0 at 0
            const double pb = A.pi_base[i];
            const long long pbb = __double_as_longlong(pb);
            const int pbc = (pbb == Cbits) ? 2 : ((pbb << 1) == 0 ? 0 : 1);
            const double ub = A.a[i];
            if (pc == 2 && pbc == 2) {
                acc2 += u - ub;             // 2C (u - ub), factor applied below
                acc3 += pos ? 1.0 : -1.0;   // - 2C (lambda - lambda_b) y_i, below
            } else if (pc == 1 && pbc == 1) {
                acc1 = fma(pk - pb, pk + pb, acc1);
            } else if (pc != 0 || pbc != 0) {
                const double yl = pos ? lh : -lh, ylb = pos ? lam0 : -lam0;
                const double f = (pc == 1) ? pk * pk : ((pc == 2) ? C * (2.0 * (u - yl) - C) : 0.0);
                const double fb = (pbc == 1) ? pb * pb : ((pbc == 2) ? C * (2.0 * (ub - ylb) - C) : 0.0);
                acc1 += f - fb;
            }
        }
        if (A.sums & SF_KKT) {
            const double al = A.alpha[i];
            const long long ab = __double_as_longlong(al);
            if (ab != __double_as_longlong(pk)) {
                const double d = al - pk;
                acc0 = fma(d, d, acc0);
            }
            if ((ab << 1) != 0) { acc1 = fma(al, al, acc1); acc2 += al; }
            // hinge max(0, 1 - (Qalpha_i + y_i lambda))
            const double marg = A.b[i] + (pos ? lh : -lh);
            acc3 += fmax(0.0, 1.0 - marg);
        }
    }
    if (A.sums & SF_PSID) acc1 = fma(2.0 * C, acc2, acc1) - 2.0 * C * (lh - lam0) * acc3;
    if (!(A.sums & SF_KKT)) acc2 = acc3 = 0.0;
    // per-(k, warp) compaction counts
    __shared__ int sh_wc[EPT][kWarps][2];
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
        const unsigned bj = __ballot_sync(0xffffffffu, (isJ >> k) & 1u);
        const unsigned bs = __ballot_sync(0xffffffffu, (isS >> k) & 1u);
        if (lane == 0) { sh_wc[k][warp][0] = __popc(bj); sh_wc[k][warp][1] = __popc(bs); }
    }
    // reduce only the sums this launch asks for (FP64 shuffles are costly here)
    if (A.sums & (SF_DPA | SF_KKT)) acc0 = warp_sum(acc0);
    if (A.sums & (SF_PSID | SF_KKT)) acc1 = warp_sum(acc1);
    if (A.sums & SF_KKT) { acc2 = warp_sum(acc2); acc3 = warp_sum(acc3); }
    if (lane == 0) { sh_d[warp][0] = acc0; sh_d[warp][1] = acc1; sh_d[warp][2] = acc2; sh_d[warp][3] = acc3; }
    __syncthreads();
    if (tid < EPT) {
        int cj = 0, cs = 0;
        for (int w = 0; w < kWarps; ++w) { cj += sh_wc[tid][w][0]; cs += sh_wc[tid][w][1]; }
        A.cnt[((size_t)tid * G + blk) * 2 + 0] = cj;
        A.cnt[((size_t)tid * G + blk) * 2 + 1] = cs;
    }
    if (warp == 0) {
        const bool v = lane < kWarps;
        const double b0 = warp_sum(v ? sh_d[lane][0] : 0.0), b1 = warp_sum(v ? sh_d[lane][1] : 0.0);
        const double b2 = warp_sum(v ? sh_d[lane][2] : 0.0), b3 = warp_sum(v ? sh_d[lane][3] : 0.0);
        if (lane == 0) {
            double *p = A.part + ((size_t)2 * G + blk) * kPartStride;
            p[0] = b0; p[1] = b1; p[2] = b2; p[3] = b3;
        }
    }
    if (!alive || !grid_barrier(A.bar, A.err)) return;

    // offsets: off(k) = sum_{k'<k} total(k') + sum_{b'<blk} cnt(k, b')
    __shared__ long long sh_off[EPT][2];
    __shared__ long long sh_tot2[EPT][2];
    for (int k = warp; k < EPT; k += kWarps) {
        long long tj = 0, ts = 0, pj = 0, ps = 0;
#pragma unroll 8
        for (int bb = lane; bb < G; bb += 32) {
            const int2 cc = __ldcg(reinterpret_cast<const int2 *>(A.cnt + ((size_t)k * G + bb) * 2));
            const int cj = cc.x, cs = cc.y;
            tj += cj; ts += cs;
            if (bb < blk) { pj += cj; ps += cs; }
        }
        tj = warp_sum_ll(tj); ts = warp_sum_ll(ts);
        pj = warp_sum_ll(pj); ps = warp_sum_ll(ps);
        if (lane == 0) { sh_tot2[k][0] = tj; sh_tot2[k][1] = ts; sh_off[k][0] = pj; sh_off[k][1] = ps; }
    }
    __syncthreads();
    if (blk == 0 && warp == 0) {
        // block 0 publishes the totals (fixed-order lanes, then shuffles)
        double r0 = 0, r1 = 0, r2 = 0, r3 = 0;
#pragma unroll 8
        for (int bb = lane; bb < G; bb += 32) {
            const double *p = A.part + ((size_t)2 * G + bb) * kPartStride;
            const double2 a = __ldcg(reinterpret_cast<const double2 *>(p));
            const double2 b = __ldcg(reinterpret_cast<const double2 *>(p + 2));
            r0 += a.x; r1 += a.y; r2 += b.x; r3 += b.y;
        }
        r0 = warp_sum(r0); r1 = warp_sum(r1); r2 = warp_sum(r2); r3 = warp_sum(r3);
        if (lane == 0) {
            long long tj = 0, ts = 0;
            for (int k = 0; k < EPT; ++k) { tj += sh_tot2[k][0]; ts += sh_tot2[k][1]; }
            A.out->lam = lam_hat;
            A.out->sum[0] = r0; A.out->sum[1] = r1; A.out->sum[2] = r2; A.out->sum[3] = r3;
            A.out->p = tj;
            A.out->s = ts;
            A.out->passes = pass;
            A.out->status = 0;
            A.out->is_df = 0;
        }
    }
    if (tid == 0) {
        long long rj = 0, rs = 0;
        for (int k = 0; k < EPT; ++k) {
            const long long oj = rj + sh_off[k][0], os = rs + sh_off[k][1];
            rj += sh_tot2[k][0]; rs += sh_tot2[k][1];
            sh_off[k][0] = oj; sh_off[k][1] = os;
        }
    }
    // exclusive prefix of the per-warp counts, one thread per (k, list)
    for (int t = tid; t < 2 * EPT; t += kTPB) {
        const int k = t >> 1, l = t & 1;
        int run = 0;
        for (int w = 0; w < kWarps; ++w) {
            const int c = sh_wc[k][w][l];
            sh_wc[k][w][l] = run;
            run += c;
        }
    }
    __syncthreads();
    if (A.J || A.S) {
        const unsigned lt = (1u << lane) - 1u;
#pragma unroll
        for (int k = 0; k < EPT; ++k) {
            const long long i = k * NT + (long long)blk * kTPB + tid;
            const unsigned bj = __ballot_sync(0xffffffffu, (isJ >> k) & 1u);
            const unsigned bs = __ballot_sync(0xffffffffu, (isS >> k) & 1u);
            if (A.J && ((isJ >> k) & 1u)) A.J[sh_off[k][0] + sh_wc[k][warp][0] + __popc(bj & lt)] = (int32_t)i;
            if (A.S && ((isS >> k) & 1u)) A.S[sh_off[k][1] + sh_wc[k][warp][1] + __popc(bs & lt)] = (int32_t)i;
        }
    }
}


static const int kEpts[] = {1, 2, 4, 8, 16, 32};

static void *kernel_for(int ept)
{
    switch (ept) {
    case 1: return (void *)proj_kernel<1>;
    case 2: return (void *)proj_kernel<2>;
    case 4: return (void *)proj_kernel<4>;
    case 8: return (void *)proj_kernel<8>;
    case 16: return (void *)proj_kernel<16>;
    default: return (void *)proj_kernel<32>;
    }
}

cudaError_t proj_setup(Work &W)
{
    // Largest co-resident grid for each instantiation (FP64 and double-float
    // kernels share the geometry); pick the smallest EPT whose grid covers n.
    const long long n = W.n;
    for (int ept : kEpts) {
        int occ0 = 0, occ1 = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ0, kernel_for(ept), kTPB, 0);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ1, projdf_kernel_for(ept), kTPB, 0);
        if (e != cudaSuccess) return e;
        const int occ = occ0 < occ1 ? occ0 : occ1;
        if (occ < 1) continue;
        const long long gmax = (long long)occ * W.nsm;
        const long long need = (n + (long long)kTPB * ept - 1) / ((long long)kTPB * ept);
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
    // the psi difference takes lam0 as the base point's lambda-hat
    if ((in.sums & SF_PSID) && (!in.lam0 || !in.pi_base || (in.sums & SF_KKT))) return cudaErrorInvalidValue;
    ProjArgs A;
    A.a = in.a; A.b = in.b; A.c1 = in.c1; A.c2 = in.c2;
    A.y = W.y; A.n = W.n; A.C = W.C; A.sums = in.sums; A.lam0 = in.lam0;
    A.u_out = in.u_out; A.pi_out = in.pi_out; A.wpi_out = in.wpi_out;
    A.J = in.J; A.S = in.S;
    A.pi_base = in.pi_base; A.alpha = in.alpha;
    A.part = W.part; A.cnt = W.cnt; A.bar = W.bar; A.err = W.err; A.out = out;
    void *args[] = {&A};
    ++W.nlaunch;
    return cudaLaunchCooperativeKernel(kernel_for(W.proj_ept), dim3(W.proj_grid), dim3(kTPB), args, 0, W.st);
}

}  // namespace svm
