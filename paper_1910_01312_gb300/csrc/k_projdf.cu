// k_projdf.cu -- the projection of Sec. 3.2.1 onto {x : y'x = 0, 0 <= x <= C}
// in double-float arithmetic (the mixed form of the solver).
//
// Same iteration as the FP64 kernel of k_proj.cu: each block keeps its slice
// of the data in registers and all blocks run, in lock-step, a safeguarded
// Newton iteration on the monotone piecewise-linear function
//   f(lambda) = sum_i y_i clip(u_i - lambda y_i, 0, C),
// whose root lambda-hat gives pi = clip(u - lambda-hat y, 0, C).
//
// Why a second kernel: on this part an FP64 instruction has ~64 cycles of
// latency and a warp can issue one every ~64 cycles (FP64 divide ~640), so
// even a handful of FP64 operations per pass -- scalar reductions, the
// decision of the root search, int-to-double conversions -- cost more than
// the whole FP32 work of the pass.  Here nothing on the device is FP64:
//  * every n-vector is a double-float pair (hi + lo, ~2^-48 relative);
//  * lambda = lambda_0 + delta with lambda_0 the warm start and delta a
//    double-float; each component keeps d_i = s_i - lambda_0 (s_i = y_i u_i)
//    in registers, so t_i = y_i (d_i - delta);
//  * f(delta) = C nu + sum_{free} d_i - n_free delta, where nu counts the
//    components at C (signed by y) and the free sum is a double-float; a
//    component is classified in FP32 with an error margin (|d| + |delta| + C)
//    2^-20 when it is certainly below 0, above C or strictly inside, and with
//    an exact double-float comparison otherwise;
//  * block partials are floats and integers, every block reduces all partials
//    in one fixed order (bit-identical decisions everywhere), and thread 0
//    of each block takes the decision in double-float arithmetic.
// The Newton step F/p is the exact root whenever it stays inside the current
// linear piece, whose ends are known as conservative FP32 offsets.
//
// Outputs: u (double-float), y o pi, the free set J, and the delta set D of
// the components whose y_i pi_i differs from a base point, with the weights
// that update A'pi from the base point's product (the mixed form never
// recomputes A'pi over all rows).  Sums for the line search (SF_PSID: the
// psi difference term by term), the inner stopping test (SF_DPA) and the KKT
// residual (SF_KKT) come back as double-float pairs.
//
// The psi difference.  With u_i - pi_i = lambda y_i for a free component, the
// sum of pi_i (2 u_i - pi_i) is |u|^2 - |u - pi|^2, and adding -2 lambda y'pi
// (zero at the root) makes each term stationary in lambda: pi_i^2 when free,
// C (2 (u_i - lambda y_i) - C) at C, 0 at 0 -- the dual function of the
// projection, max over lambda of sum_i min_{0<=x_i<=C} [(u_i - x_i)^2 +
// 2 lambda y_i x_i].  The plain terms pi (2u - pi) are of size |u| |pi| with
// |u| ~ sigma, so the root's own precision (a shift of lambda by eps moves
// their sum by 2 lambda eps |J|) and the rounding of 2u - pi left a constant
// offset in the differences of trial points at large sigma that hid the
// Armijo decrease; the stationary terms are of size pi^2 and C |u - lambda y|.
#include <math.h>

#include "internal.cuh"

namespace svm {

namespace {

constexpr int kMaxPassDF = 256;
constexpr float kMargin = 9.5367431640625e-07f;   // 2^-20
constexpr int kStrideF = 16;                      // floats per block partial
constexpr int kStageG = 512;                      // grids up to this size stage partials in shared memory
constexpr int kTPBC = 1024;                       // threads per CTA of the cluster form

// ---- thread-block clusters: the cluster form of the kernel (one problem per
// cluster) exchanges its partials through distributed shared memory and
// synchronises with the hardware cluster barrier instead of a grid barrier ----
__device__ __forceinline__ unsigned cl_rank() { unsigned r; asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r)); return r; }
__device__ __forceinline__ unsigned cl_size() { unsigned r; asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r)); return r; }
__device__ __forceinline__ unsigned cl_id() { unsigned r; asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r)); return r; }
__device__ __forceinline__ void cl_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// address of `p` (this CTA's shared memory) in CTA `rank` of the cluster
__device__ __forceinline__ unsigned cl_map(const void *p, unsigned rank)
{
    unsigned a;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(a) : "r"(smem_u32(p)), "r"(rank));
    return a;
}
__device__ __forceinline__ float4 cl_ld4(unsigned a)
{
    float4 v;
    asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ int2 cl_ld2i(unsigned a)
{
    int2 v;
    asm volatile("ld.shared::cluster.v2.s32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(a) : "memory");
    return v;
}


__device__ __forceinline__ float2 u_at(const PDArgs &A, long long i, bool pos)
{
    float2 u = A.a[i];
    if (A.a_signed && !pos) u = dfx_neg(u);
    if (A.b) u = dfx_add(u, dfx_mul(A.c1, A.b[i]));
    return dfx_add(u, A.c2);
}

// conservative FP32 bounds of a double-float offset: never farther than o
__device__ __forceinline__ float toward_zero(float2 o)
{
    return o.x > 0.f ? __fmul_rd(o.x, 0.99999988f) : __fmul_ru(o.x, 0.99999988f);
}

struct Acc {
    float2 D;        // sum of d_i over free components
    int nu, nf;      // signed count at C; free count
    int ppx, pmx;    // components exactly at a breakpoint that count for the right / left slope
    float bhi, blo;  // nearest breakpoint offsets above / below (conservative)
};

__device__ __forceinline__ void acc_zero(Acc &a)
{
    a.D = make_float2(0.f, 0.f);
    a.nu = a.nf = a.ppx = a.pmx = 0;
    a.bhi = INFINITY;
    a.blo = -INFINITY;
}

// One component at delta.  t = y (d - delta); breakpoints (in delta) at
// offsets e = d - delta (t = 0) and e - y C (t = C).
__device__ __forceinline__ void eval_df(float2 d, bool pos, float2 dl, float2 Cd, Acc &a)
{
    const float r = d.x;
    const float tf = pos ? (r - dl.x) : (dl.x - r);
    const float er = (fabsf(r) + fabsf(dl.x) + Cd.x) * kMargin;
    if (tf > Cd.x + er) {                       // certainly above C
        a.nu += pos ? 1 : -1;
        if (pos) a.bhi = fminf(a.bhi, tf - Cd.x - er);
        else a.blo = fmaxf(a.blo, Cd.x - tf + er);
        return;
    }
    if (tf < -er) {                             // certainly below 0
        if (pos) a.blo = fmaxf(a.blo, tf + er);
        else a.bhi = fminf(a.bhi, -tf - er);
        return;
    }
    if (tf > er && tf < Cd.x - er) {            // certainly free
        a.D = dfx_add(a.D, d);
        ++a.nf;
        if (pos) { a.bhi = fminf(a.bhi, tf - er); a.blo = fmaxf(a.blo, tf - Cd.x + er); }
        else { a.blo = fmaxf(a.blo, -tf + er); a.bhi = fminf(a.bhi, Cd.x - tf - er); }
        return;
    }
    // near a breakpoint: exact double-float comparison
    const float2 e = dfx_sub(d, dl);
    const float2 t = pos ? e : dfx_neg(e);
    const float2 tc = dfx_sub(t, Cd);
    if (tc.x > 0.f) {
        a.nu += pos ? 1 : -1;
    } else if (tc.x == 0.f) {                   // at C
        a.nu += pos ? 1 : -1;
        if (pos) ++a.ppx; else ++a.pmx;
    } else if (t.x > 0.f) {
        a.D = dfx_add(a.D, d);
        ++a.nf;
    } else if (t.x == 0.f) {                    // at 0
        if (pos) ++a.pmx; else ++a.ppx;
    }
    const float2 o2 = pos ? tc : dfx_neg(tc);   // e - y C
    if (e.x > 0.f) a.bhi = fminf(a.bhi, toward_zero(e));
    else if (e.x < 0.f) a.blo = fmaxf(a.blo, toward_zero(e));
    if (o2.x > 0.f) a.bhi = fminf(a.bhi, toward_zero(o2));
    else if (o2.x < 0.f) a.blo = fmaxf(a.blo, toward_zero(o2));
}

__device__ __forceinline__ void acc_warp_reduce(Acc &a)
{
    a.nu = __reduce_add_sync(0xffffffffu, a.nu);
    a.nf = __reduce_add_sync(0xffffffffu, a.nf);
    a.ppx = __reduce_add_sync(0xffffffffu, a.ppx);
    a.pmx = __reduce_add_sync(0xffffffffu, a.pmx);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a.bhi = fminf(a.bhi, __shfl_xor_sync(0xffffffffu, a.bhi, o));
        a.blo = fmaxf(a.blo, __shfl_xor_sync(0xffffffffu, a.blo, o));
        a.D = dfx_add(a.D, shfl_xor_f2(a.D, o));
    }
}

struct SearchState {
    float2 Ld, Ud;
    float FL, FU, last_step;
    int hL, hU, last_dir, nbr;
};

__device__ __forceinline__ float2 dfx_half(float2 a)
{
    return make_float2(0.5f * a.x, 0.5f * a.y);
}

// the final sums of one thread / warp / block: four double-float values and a count
struct Sums {
    float2 s[4];
    int nupa;
};

__device__ __forceinline__ void sums_warp_reduce(Sums &v)
{
    v.nupa = __reduce_add_sync(0xffffffffu, v.nupa);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < 4; ++k) v.s[k] = dfx_add(v.s[k], shfl_xor_f2(v.s[k], o));
}

// The body of both forms.  CLU = false: G blocks of one cooperative launch
// (grid barrier, partials in global memory); CLU = true: the G CTAs of one
// cluster (cluster barrier, partials in distributed shared memory; every CTA
// runs the same sequence of cluster barriers, and a last one keeps each CTA's
// shared memory alive until the others have read it).
template <int EPT, bool CLU, int TPB>
__device__ __forceinline__ void projdf_body(const PDArgs &A, const int G, const int blk)
{
    constexpr int WARPS = TPB / 32;
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const long long NT = (long long)G * TPB;
    const float2 Cd = A.Cd;

    __shared__ float2 sh_l0;
    if (tid == 0) {
        float2 l0 = A.lam0 ? __ldcg(A.lam0) : make_float2(0.f, 0.f);
        if (!isfinite(l0.x) || !isfinite(l0.y)) l0 = make_float2(0.f, 0.f);
        sh_l0 = l0;
    }
    __syncthreads();
    const float2 l0 = sh_l0;

    // d_i = y_i u_i - lambda_0, register resident; u is written here
    float2 d[EPT];
    unsigned posm = 0u, valm = 0u;
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
        const long long i = k * NT + (long long)blk * TPB + tid;
        d[k] = make_float2(0.f, 0.f);
        if (i < A.n) {
            const bool pos = A.y[i] > 0;
            const float2 u = u_at(A, i, pos);
            if (A.u_out) A.u_out[i] = u;
            d[k] = dfx_sub(pos ? u : dfx_neg(u), l0);
            posm |= (pos ? 1u : 0u) << k;
            valm |= 1u << k;
        }
    }

    __shared__ float4 sh_wf[WARPS];
    __shared__ int4 sh_wi[WARPS];
    __shared__ float4 sh_stage[CLU ? 1 : 3 * kStageG];   // staged block partials (2 per pass partial, 3 per final one)
    __shared__ float4 sh_xp[2][2];                      // cluster form: this CTA's pass partial (double-buffered)
    __shared__ int2 sh_xc[EPT];                         // cluster form: this CTA's list counts per k
    __shared__ float4 sh_xs[3];                         // cluster form: this CTA's final sums
    __shared__ float2 sh_dl;
    __shared__ int sh_done;
    if (tid == 0) sh_dl = make_float2(0.f, 0.f);
    __syncthreads();

    // root-search state, used by thread 0 only (bracket in delta: f(L) > 0 > f(U))
    __shared__ SearchState ss;
    if (tid == 0) {
        ss.Ld = ss.Ud = make_float2(0.f, 0.f);
        ss.FL = ss.FU = ss.last_step = 0.f;
        ss.hL = ss.hU = 0;
        ss.last_dir = ss.nbr = 0;
    }
    int pass = 0;
    bool alive = true;

    for (;;) {
        const float2 dl = sh_dl;
        Acc a;
        acc_zero(a);
#pragma unroll
        for (int k = 0; k < EPT; ++k)
            if ((valm >> k) & 1u) eval_df(d[k], (posm >> k) & 1u, dl, Cd, a);
        acc_warp_reduce(a);
        if (lane == 0) {
            sh_wf[warp] = make_float4(a.D.x, a.D.y, a.bhi, a.blo);
            sh_wi[warp] = make_int4(a.nu, a.nf, a.ppx, a.pmx);
        }
        __syncthreads();
        if (warp == 0) {
            Acc b;
            acc_zero(b);
            if (lane < WARPS) {
                const float4 f = sh_wf[lane];
                const int4 c = sh_wi[lane];
                b.D = make_float2(f.x, f.y); b.bhi = f.z; b.blo = f.w;
                b.nu = c.x; b.nf = c.y; b.ppx = c.z; b.pmx = c.w;
            }
            acc_warp_reduce(b);
            if (lane == 0) {
                if (CLU) {
                    sh_xp[pass & 1][0] = make_float4(b.D.x, b.D.y, b.bhi, b.blo);
                    sh_xp[pass & 1][1] = make_float4(__int_as_float(b.nu), __int_as_float(b.nf), __int_as_float(b.ppx),
                                                     __int_as_float(b.pmx));
                } else {
                    float *p = A.part + ((size_t)(pass & 1) * G + blk) * kStrideF;
                    __stcg(reinterpret_cast<float4 *>(p), make_float4(b.D.x, b.D.y, b.bhi, b.blo));
                    __stcg(reinterpret_cast<int4 *>(p + 4), make_int4(b.nu, b.nf, b.ppx, b.pmx));
                }
            }
        }
        if (CLU) {
            cl_sync();
        } else if (!grid_barrier(A.bar, A.err)) {
            alive = false;
            break;
        }
        const float *slot = CLU ? nullptr : A.part + (size_t)(pass & 1) * G * kStrideF;
        const bool staged = !CLU && G <= kStageG;
        if (staged) {
            // every thread of the block fetches a share of the G partials at once
            // (one L2 round trip instead of G/32 dependent ones for warp 0)
            for (int e = tid; e < 2 * G; e += TPB)
                sh_stage[e] = __ldcg(reinterpret_cast<const float4 *>(slot + (size_t)(e >> 1) * kStrideF) + (e & 1));
            __syncthreads();
        }
        if (warp == 0) {
            // every block reduces all partials in the same order
            Acc t;
            acc_zero(t);
            for (int bb = lane; bb < G; bb += 32) {
                float4 f, cf;
                if (CLU) {   // CTA bb's partial, read from its shared memory
                    f = cl_ld4(cl_map(&sh_xp[pass & 1][0], (unsigned)bb));
                    cf = cl_ld4(cl_map(&sh_xp[pass & 1][1], (unsigned)bb));
                } else {
                    f = staged ? sh_stage[2 * bb] : __ldcg(reinterpret_cast<const float4 *>(slot + (size_t)bb * kStrideF));
                    cf = staged ? sh_stage[2 * bb + 1]
                                : __ldcg(reinterpret_cast<const float4 *>(slot + (size_t)bb * kStrideF + 4));
                }
                const int4 c = make_int4(__float_as_int(cf.x), __float_as_int(cf.y), __float_as_int(cf.z), __float_as_int(cf.w));
                t.D = dfx_add(t.D, make_float2(f.x, f.y));
                t.bhi = fminf(t.bhi, f.z);
                t.blo = fmaxf(t.blo, f.w);
                t.nu += c.x; t.nf += c.y; t.ppx += c.z; t.pmx += c.w;
            }
            acc_warp_reduce(t);
            if (lane == 0) {
                // ---- decision (identical in every block) ----
                float2 Ld = ss.Ld, Ud = ss.Ud;
                float FL = ss.FL, FU = ss.FU, last_step = ss.last_step;
                bool hL = ss.hL != 0, hU = ss.hU != 0;
                int last_dir = ss.last_dir, nbr = ss.nbr;
                const float2 F = dfx_add(dfx_add(dfx_mul(Cd, dfx_from_ll(t.nu)), t.D),
                                         dfx_neg(dfx_mul(dl, dfx_from_ll(t.nf))));
                const long long pr = (long long)t.nf + t.ppx, pl = (long long)t.nf + t.pmx;
                int done = 0, dir = 0;
                float2 next = dl, dhat = dl;
                if (F.x == 0.f) {
                    done = 1;
                } else if (F.x > 0.f) {
                    Ld = dl; FL = F.x; hL = true; dir = 1;
                    if (pr > 0) {
                        const float2 st = dfx_div(F, dfx_from_ll(pr));
                        next = dfx_add(dl, st);
                        if (st.x <= t.bhi) { done = 1; dhat = next; }
                    } else {
                        next = dfx_addf(dl, 2.f * t.bhi);   // flat piece: go past its end
                    }
                } else {
                    Ud = dl; FU = F.x; hU = true; dir = -1;
                    if (pl > 0) {
                        const float2 st = dfx_div(F, dfx_from_ll(pl));
                        next = dfx_add(dl, st);
                        if (st.x >= t.blo) { done = 1; dhat = next; }
                    } else {
                        next = dfx_addf(dl, 2.f * t.blo);
                    }
                }
                if (!done) {
                    if (!(hL && hU)) {
                        // not bracketed yet: steps in one direction at least double
                        float stf = dfx_sub(next, dl).x;
                        if (dir == last_dir && fabsf(stf) < 2.f * last_step) {
                            stf = dir * 2.f * last_step;
                            next = dfx_addf(dl, stf);
                        }
                        if (!(fabsf(stf) > 0.f)) {
                            stf = dir * fmaxf(fabsf(dl.x) * 1.1920929e-07f, 1e-30f);
                            next = dfx_addf(dl, stf);
                        }
                        last_step = fabsf(stf);
                        last_dir = dir;
                    } else {
                        // bracketed: Newton point if inside, else secant; every third
                        // bracketed pass bisects, so the bracket at least halves
                        ++nbr;
                        const bool inside = dfx_gt(next, Ld) && dfx_gt(Ud, next);
                        if (nbr % 3 == 0) {
                            next = dfx_half(dfx_add(Ld, Ud));
                        } else if (!inside) {
                            next = dfx_addf(Ld, dfx_sub(Ud, Ld).x * (FL / (FL - FU)));
                            if (!(dfx_gt(next, Ld) && dfx_gt(Ud, next))) next = dfx_half(dfx_add(Ld, Ud));
                        }
                    }
                    if (!isfinite(next.x) || (hL && hU && !(dfx_gt(next, Ld) && dfx_gt(Ud, next)))) {
                        // no representable point strictly inside the bracket
                        done = 1;
                        dhat = (hL && (!hU || fabsf(FL) <= fabsf(FU))) ? Ld : Ud;
                    } else if (pass + 1 >= kMaxPassDF) {
                        done = 1;
                        dhat = next;
                        if (blk == 0) set_err(A.err, DEV_ROOT);
                    }
                }
                sh_done = done;
                sh_dl = done ? dhat : next;
                ss.Ld = Ld; ss.Ud = Ud; ss.FL = FL; ss.FU = FU; ss.last_step = last_step;
                ss.hL = hL; ss.hU = hU; ss.last_dir = last_dir; ss.nbr = nbr;
            }
        }
        __syncthreads();
        ++pass;
        if (sh_done) break;
    }

    // ---------------- final phase: pi, sums, lists ----------------
    const float2 dh = sh_dl;                    // delta-hat
    const float2 lh = dfx_add(l0, dh);          // lambda-hat
    Sums sm;
#pragma unroll
    for (int k = 0; k < 4; ++k) sm.s[k] = make_float2(0.f, 0.f);
    sm.nupa = 0;
    float2 sq0 = make_float2(0.f, 0.f), sq1 = make_float2(0.f, 0.f);   // sums of squares
    unsigned isJ = 0u, isD = 0u;
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
        if (!((valm >> k) & 1u)) continue;
        const long long i = k * NT + (long long)blk * TPB + tid;
        const bool pos = (posm >> k) & 1u;
        // pi_i and its class: 0 (= 0), 1 (free), 2 (= C); ties as the paper's clip
        int pc;
        float2 pk;
        {
            const float r = d[k].x;
            const float tf = pos ? (r - dh.x) : (dh.x - r);
            const float er = (fabsf(r) + fabsf(dh.x) + Cd.x) * kMargin;
            if (tf > Cd.x + er) { pc = 2; pk = Cd; }
            else if (tf < -er) { pc = 0; pk = make_float2(0.f, 0.f); }
            else {
                const float2 e = dfx_sub(d[k], dh);
                const float2 t = pos ? e : dfx_neg(e);
                if (!(t.x > 0.f)) { pc = 0; pk = make_float2(0.f, 0.f); }
                else if (!dfx_gt(Cd, t)) { pc = 2; pk = Cd; }
                else { pc = 1; pk = t; }
            }
        }
        const float2 wp = (pc == 0) ? make_float2(0.f, 0.f) : (pos ? pk : dfx_neg(pk));
        if (A.wpi_out) A.wpi_out[i] = wp;
        if (pc == 1) isJ |= 1u << k;
        float2 bw = make_float2(0.f, 0.f);
        if (A.base_w) bw = A.base_w[i];
        if (A.D && !dfx_same(wp, bw)) {
            isD |= 1u << k;
            A.dw_out[i] = dfx_sub(wp, bw);
            A.dwa_out[i] = (pk.x + pk.y) - fabsf(bw.x + bw.y);
        }
        if (A.sums & SF_DPA) {
            const float2 aw = A.alpha_w[i];
            if (!dfx_same(aw, wp)) {
                const float2 dx = dfx_sub(wp, aw);
                sq0 = dfx_add(sq0, dfx_mul(dx, dx));
            }
        }
        if (A.sums & SF_PSID) {
            // psi difference term by term, each term in its multiplier-stationary
            // form pi (2u - pi - 2 lambda y) (equal to pi (2u - pi) summed, since
            // y'pi = 0): pi^2 when free, C (2 (u - lambda y) - C) at C, 0 at 0
            const float2 pb = pos ? bw : dfx_neg(bw);
            const int pbc = (bw.x == 0.f) ? 0 : (dfx_same(pb, Cd) ? 2 : 1);
            if (pc == 2 && pbc == 2) {
                sm.s[2] = dfx_add(sm.s[2], A.b[i]);   // 2C (u - ub) = 2C c1 b_i, factor applied below
                sm.nupa += pos ? 1 : -1;               // - 2C (lambda - lambda_b) y_i, below
            } else if (pc == 1 && pbc == 1) {
                sm.s[1] = dfx_add(sm.s[1], dfx_mul(dfx_sub(pk, pb), dfx_add(pk, pb)));
            } else if (pc != 0 || pbc != 0) {
                float2 f = make_float2(0.f, 0.f), fb = f;
                if (pc == 1) {
                    f = dfx_mul(pk, pk);
                } else if (pc == 2) {
                    const float2 e = dfx_sub(d[k], dh);              // y u - lambda
                    const float2 t = pos ? e : dfx_neg(e);           // u - lambda y
                    f = dfx_mul(Cd, dfx_sub(dfx_add(t, t), Cd));
                }
                if (pbc == 1) {
                    fb = dfx_mul(pb, pb);
                } else if (pbc == 2) {
                    const float2 ub = A.a[i];
                    const float2 eb = dfx_sub(pos ? ub : dfx_neg(ub), l0);   // y ub - lambda_b
                    const float2 tb = pos ? eb : dfx_neg(eb);
                    fb = dfx_mul(Cd, dfx_sub(dfx_add(tb, tb), Cd));
                }
                sm.s[1] = dfx_add(sm.s[1], dfx_sub(f, fb));
            }
        }
        if (A.sums & SF_KKT) {
            // alpha = a (y o alpha); |alpha - pi|^2, |alpha|^2, sum alpha, hinge
            const float2 aw = A.a[i];
            if (!dfx_same(aw, wp)) {
                const float2 dx = dfx_sub(wp, aw);
                sq0 = dfx_add(sq0, dfx_mul(dx, dx));
            }
            const float2 al = pos ? aw : dfx_neg(aw);
            if (dfx_same(al, Cd)) {
                ++sm.nupa;
            } else if (al.x != 0.f) {
                sq1 = dfx_add(sq1, dfx_mul(al, al));
                sm.s[2] = dfx_add(sm.s[2], al);
            }
            const float2 m = dfx_add(A.b[i], pos ? lh : dfx_neg(lh));
            const float2 h = dfx_sub(make_float2(1.f, 0.f), m);
            if (h.x > 0.f) sm.s[3] = dfx_add(sm.s[3], h);
        }
    }
    sm.s[0] = sq0;
    if (A.sums & SF_KKT) sm.s[1] = sq1;

    // per-(k, warp) list counts
    __shared__ int sh_wc[EPT][WARPS][2];
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
        const unsigned bj = __ballot_sync(0xffffffffu, (isJ >> k) & 1u);
        const unsigned bd = __ballot_sync(0xffffffffu, (isD >> k) & 1u);
        if (lane == 0) { sh_wc[k][warp][0] = __popc(bj); sh_wc[k][warp][1] = __popc(bd); }
    }
    __shared__ float4 sh_s[WARPS][2];
    __shared__ int sh_n[WARPS];
    if (A.sums) {
        sums_warp_reduce(sm);
        if (lane == 0) {
            sh_s[warp][0] = make_float4(sm.s[0].x, sm.s[0].y, sm.s[1].x, sm.s[1].y);
            sh_s[warp][1] = make_float4(sm.s[2].x, sm.s[2].y, sm.s[3].x, sm.s[3].y);
            sh_n[warp] = sm.nupa;
        }
    }
    __syncthreads();
    if (tid < EPT) {
        int cj = 0, cd = 0;
        for (int w = 0; w < WARPS; ++w) { cj += sh_wc[tid][w][0]; cd += sh_wc[tid][w][1]; }
        if (CLU) {
            sh_xc[tid] = make_int2(cj, cd);
        } else {
            A.cnt[((size_t)tid * G + blk) * 2 + 0] = cj;
            A.cnt[((size_t)tid * G + blk) * 2 + 1] = cd;
        }
    }
    if (A.sums && warp == 0) {
        Sums b;
#pragma unroll
        for (int k = 0; k < 4; ++k) b.s[k] = make_float2(0.f, 0.f);
        b.nupa = 0;
        if (lane < WARPS) {
            const float4 f0 = sh_s[lane][0], f1 = sh_s[lane][1];
            b.s[0] = make_float2(f0.x, f0.y); b.s[1] = make_float2(f0.z, f0.w);
            b.s[2] = make_float2(f1.x, f1.y); b.s[3] = make_float2(f1.z, f1.w);
            b.nupa = sh_n[lane];
        }
        sums_warp_reduce(b);
        if (lane == 0) {
            if (CLU) {
                sh_xs[0] = make_float4(b.s[0].x, b.s[0].y, b.s[1].x, b.s[1].y);
                sh_xs[1] = make_float4(b.s[2].x, b.s[2].y, b.s[3].x, b.s[3].y);
                sh_xs[2] = make_float4(__int_as_float(b.nupa), 0.f, 0.f, 0.f);
            } else {
                float *p = A.part + ((size_t)2 * G + blk) * kStrideF;
                __stcg(reinterpret_cast<float4 *>(p), make_float4(b.s[0].x, b.s[0].y, b.s[1].x, b.s[1].y));
                __stcg(reinterpret_cast<float4 *>(p + 4), make_float4(b.s[2].x, b.s[2].y, b.s[3].x, b.s[3].y));
                __stcg(reinterpret_cast<int *>(p + 8), b.nupa);
            }
        }
    }
    if (CLU) {
        cl_sync();
    } else if (!alive || !grid_barrier(A.bar, A.err)) {
        return;
    }

    // offsets: off(k) = sum_{k'<k} total(k') + sum_{b'<blk} cnt(k, b')
    __shared__ long long sh_off[EPT][2];
    __shared__ long long sh_tot2[EPT][2];
    for (int k = warp; k < EPT; k += WARPS) {
        long long tj = 0, td = 0, pj = 0, pd = 0;
#pragma unroll 8
        for (int bb = lane; bb < G; bb += 32) {
            const int2 cc = CLU ? cl_ld2i(cl_map(&sh_xc[k], (unsigned)bb))
                                : __ldcg(reinterpret_cast<const int2 *>(A.cnt + ((size_t)k * G + bb) * 2));
            tj += cc.x; td += cc.y;
            if (bb < blk) { pj += cc.x; pd += cc.y; }
        }
        tj = warp_sum_ll(tj); td = warp_sum_ll(td);
        pj = warp_sum_ll(pj); pd = warp_sum_ll(pd);
        if (lane == 0) { sh_tot2[k][0] = tj; sh_tot2[k][1] = td; sh_off[k][0] = pj; sh_off[k][1] = pd; }
    }
    __syncthreads();
    const bool staged_sums = !CLU && blk == 0 && A.sums && G <= kStageG;
    if (staged_sums) {
        // block 0 fetches the final-phase partials with all its threads at once
        for (int e = tid; e < 3 * G; e += TPB)
            sh_stage[e] = __ldcg(reinterpret_cast<const float4 *>(A.part + ((size_t)2 * G + e / 3) * kStrideF) + e % 3);
        __syncthreads();
    }
    if (blk == 0 && warp == 0) {
        // block 0 publishes lambda-hat and the sums (fixed-order reduction)
        Sums t;
#pragma unroll
        for (int k = 0; k < 4; ++k) t.s[k] = make_float2(0.f, 0.f);
        t.nupa = 0;
        if (A.sums) {
            for (int bb = lane; bb < G; bb += 32) {
                const float *p = CLU ? nullptr : A.part + ((size_t)2 * G + bb) * kStrideF;
                float4 f0, f1;
                int nu;
                if (CLU) {
                    f0 = cl_ld4(cl_map(&sh_xs[0], (unsigned)bb));
                    f1 = cl_ld4(cl_map(&sh_xs[1], (unsigned)bb));
                    nu = __float_as_int(cl_ld4(cl_map(&sh_xs[2], (unsigned)bb)).x);
                } else {
                    f0 = staged_sums ? sh_stage[3 * bb] : __ldcg(reinterpret_cast<const float4 *>(p));
                    f1 = staged_sums ? sh_stage[3 * bb + 1] : __ldcg(reinterpret_cast<const float4 *>(p + 4));
                    nu = staged_sums ? __float_as_int(sh_stage[3 * bb + 2].x) : __ldcg(reinterpret_cast<const int *>(p + 8));
                }
                t.s[0] = dfx_add(t.s[0], make_float2(f0.x, f0.y));
                t.s[1] = dfx_add(t.s[1], make_float2(f0.z, f0.w));
                t.s[2] = dfx_add(t.s[2], make_float2(f1.x, f1.y));
                t.s[3] = dfx_add(t.s[3], make_float2(f1.z, f1.w));
                t.nupa += nu;
            }
            sums_warp_reduce(t);
        }
        if (lane == 0) {
            long long tj = 0, td = 0;
            for (int k = 0; k < EPT; ++k) { tj += sh_tot2[k][0]; td += sh_tot2[k][1]; }
            float2 s1 = t.s[1], s2 = t.s[2];
            if (A.sums & SF_PSID) {
                // + 2C c1 sum_{both at C} b_i - 2C (lambda - lambda_b) sum_{both at C} y_i,
                // lambda - lambda_b = dh (lambda_b = l0)
                const float2 c2x = make_float2(2.f * Cd.x, 2.f * Cd.y);
                s1 = dfx_add(s1, dfx_mul(dfx_mul(c2x, A.c1), s2));
                s1 = dfx_sub(s1, dfx_mul(dfx_mul(c2x, dh), dfx_from_ll(t.nupa)));
                s2 = make_float2(0.f, 0.f);
            }
            if (A.sums & SF_KKT) {
                const float2 nc = dfx_mul(Cd, dfx_from_ll(t.nupa));
                s1 = dfx_add(s1, dfx_mul(nc, Cd));
                s2 = dfx_add(s2, nc);
            }
            A.out->lamf = lh;
            A.out->sumf[0] = t.s[0];
            A.out->sumf[1] = s1;
            A.out->sumf[2] = s2;
            A.out->sumf[3] = t.s[3];
            A.out->p = tj;
            A.out->s = td;
            A.out->passes = pass;
            A.out->status = 0;
            A.out->is_df = 1;
        }
    }
    if (tid == 0) {
        long long rj = 0, rd = 0;
        for (int k = 0; k < EPT; ++k) {
            const long long oj = rj + sh_off[k][0], od = rd + sh_off[k][1];
            rj += sh_tot2[k][0]; rd += sh_tot2[k][1];
            sh_off[k][0] = oj; sh_off[k][1] = od;
        }
    }
    // exclusive prefix of the per-warp counts, one thread per (k, list)
    for (int t = tid; t < 2 * EPT; t += TPB) {
        const int k = t >> 1, l = t & 1;
        int run = 0;
        for (int w = 0; w < WARPS; ++w) {
            const int c = sh_wc[k][w][l];
            sh_wc[k][w][l] = run;
            run += c;
        }
    }
    __syncthreads();
    if (A.J || A.D) {
        const unsigned lt = (1u << lane) - 1u;
#pragma unroll
        for (int k = 0; k < EPT; ++k) {
            const long long i = k * NT + (long long)blk * TPB + tid;
            const unsigned bj = __ballot_sync(0xffffffffu, (isJ >> k) & 1u);
            const unsigned bd = __ballot_sync(0xffffffffu, (isD >> k) & 1u);
            if (A.J && ((isJ >> k) & 1u)) A.J[sh_off[k][0] + sh_wc[k][warp][0] + __popc(bj & lt)] = (int32_t)i;
            if (A.D && ((isD >> k) & 1u)) A.D[sh_off[k][1] + sh_wc[k][warp][1] + __popc(bd & lt)] = (int32_t)i;
        }
    }
    if (CLU) cl_sync();   // no CTA leaves while another may still read its shared memory
}

template <int EPT>
__global__ void __launch_bounds__(kTPB, EPT >= 16 ? 1 : 2) projdf_kernel(PDArgs A)
{
    projdf_body<EPT, false, kTPB>(A, (int)gridDim.x, (int)blockIdx.x);
}

// One problem per thread-block cluster: table[cluster id] (a batch of
// problems) or A0 (one problem, table = nullptr).
template <int EPT>
__global__ void __launch_bounds__(kTPBC, 1) projdf_cluster_kernel(const __grid_constant__ PDArgs A0,
                                                                  const PDArgs *__restrict__ table)
{
    const PDArgs &A = table ? table[cl_id()] : A0;
    projdf_body<EPT, true, kTPBC>(A, (int)cl_size(), (int)cl_rank());
}

float2 split_host(double v)
{
    const float hi = (float)v;
    return make_float2(hi, (float)(v - (double)hi));
}

}  // namespace

void *projdf_kernel_for(int ept)
{
    switch (ept) {
    case 1: return (void *)projdf_kernel<1>;
    case 2: return (void *)projdf_kernel<2>;
    case 4: return (void *)projdf_kernel<4>;
    case 8: return (void *)projdf_kernel<8>;
    case 16: return (void *)projdf_kernel<16>;
    default: return (void *)projdf_kernel<32>;
    }
}

static void *projdf_cluster_kernel_for(int ept)
{
    switch (ept) {
    case 1: return (void *)projdf_cluster_kernel<1>;
    case 2: return (void *)projdf_cluster_kernel<2>;
    case 4: return (void *)projdf_cluster_kernel<4>;
    case 8: return (void *)projdf_cluster_kernel<8>;
    default: return (void *)projdf_cluster_kernel<16>;
    }
}

cudaError_t make_pdargs(const Work &W, const ProjDF &in, ProjOut *out, PDArgs *A)
{
    if ((in.sums & SF_DPA) && !in.alpha_w) return cudaErrorInvalidValue;
    if ((in.sums & SF_PSID) && (!in.base_w || !in.b || in.a_signed || !in.lam0 || (in.sums & SF_KKT)))
        return cudaErrorInvalidValue;
    if ((in.sums & SF_KKT) && (!in.b || !in.a_signed)) return cudaErrorInvalidValue;
    if (in.D && (!in.dw_out || !in.dwa_out)) return cudaErrorInvalidValue;
    A->a = in.a; A->a_signed = in.a_signed ? 1 : 0; A->b = in.b;
    A->c1 = split_host(in.c1); A->c2 = split_host(in.c2);
    A->y = W.y; A->n = W.n; A->Cd = split_host(W.C); A->sums = in.sums; A->lam0 = in.lam0;
    A->u_out = in.u_out; A->wpi_out = in.wpi_out; A->alpha_w = in.alpha_w; A->base_w = in.base_w;
    A->dw_out = in.dw_out; A->dwa_out = in.dwa_out; A->J = in.J; A->D = in.D;
    A->part = reinterpret_cast<float *>(W.part); A->cnt = W.cnt; A->bar = W.bar; A->err = W.err; A->out = out;
    return cudaSuccess;
}

// Cluster launches: clusters of W.proj_cl CTAs, one problem per cluster.
static cudaError_t launch_cluster(const Work &W, const PDArgs &A0, const PDArgs *table, int nprob)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(nprob * W.proj_cl));
    cfg.blockDim = dim3(kTPBC);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = W.st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)W.proj_cl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    void *args[] = {(void *)&A0, (void *)&table};
    return cudaLaunchKernelExC(&cfg, projdf_cluster_kernel_for(W.proj_cept), args);
}

cudaError_t launch_project_df(Work &W, const ProjDF &in, ProjOut *out)
{
    PDArgs A;
    cudaError_t e = make_pdargs(W, in, out, &A);
    if (e != cudaSuccess) return e;
    ++W.nlaunch;
    if (W.proj_cl > 0) return launch_cluster(W, A, nullptr, 1);
    void *args[] = {&A};
    return cudaLaunchCooperativeKernel(projdf_kernel_for(W.proj_ept), dim3(W.proj_grid), dim3(kTPB), args, 0, W.st);
}

cudaError_t launch_project_df_table(Work &W, const PDArgs *table_dev, int nprob)
{
    if (W.proj_cl <= 0 || nprob < 1 || !table_dev) return cudaErrorInvalidValue;
    PDArgs dummy = {};
    ++W.nlaunch;
    return launch_cluster(W, dummy, table_dev, nprob);
}

// The cluster form (opt-in: SVM_PROJ_CLUSTER=1 when the handle is created)
// serves problems that fit one cluster's registers: clusters of 16 CTAs (8
// where 16 cannot be scheduled) of 1024 threads with EPT <= 16 components each,
// i.e. n <= 262,144; the cooperative form serves the rest.  Measured on GB300
// at n = 1e5: 59 us per projection against 46 us for the cooperative form
// (one cluster holds 16 SMs), while a batched solve's per-phase cost falls by
// a fifth when all its problems' projections share one launch -- no net gain
// on the one-vs-rest workload, so the cooperative form is the default.
cudaError_t projdf_cluster_setup(Work &W)
{
    W.proj_cl = 0;
    W.proj_cept = 0;
    const char *env = getenv("SVM_PROJ_CLUSTER");
    if (!env || env[0] != '1') return cudaSuccess;
    static const int kEptC[] = {1, 2, 4, 8, 16};
    for (int cl : {16, 8}) {
        int ept = 0;
        for (int e : kEptC)
            if ((long long)cl * kTPBC * e >= W.n) { ept = e; break; }
        if (!ept) continue;
        void *k = projdf_cluster_kernel_for(ept);
        if (cl > 8) {
            if (cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
                cudaGetLastError();
                continue;
            }
        }
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)cl);
        cfg.blockDim = dim3(kTPBC);
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)cl;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int nclusters = 0;
        if (cudaOccupancyMaxActiveClusters(&nclusters, k, &cfg) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        if (nclusters >= 1) {
            W.proj_cl = cl;
            W.proj_cept = ept;
            return cudaSuccess;
        }
    }
    return cudaSuccess;
}

}  // namespace svm
