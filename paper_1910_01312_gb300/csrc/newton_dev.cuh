// newton_dev.cuh -- device routines shared by the Newton solvers of the reduced
// system of Proposition 3.5 (k_newton.cu, k_newton_wide.cu): the packed FP32
// Cholesky of one block, the grid-wide blocked Cholesky, the triangular
// inverse of a packed factor, and fixed-order double-float dot products.
#pragma once
#include "internal.cuh"

namespace svm {

constexpr int kCgThreads = 512;
constexpr int kCgMaxQ = 128;
constexpr int kPb = 8;   // panel width

__device__ __forceinline__ int lpos(int i, int j)   // packed lower triangle, row-major
{
    return ((i * (i + 1)) >> 1) + j;
}

struct CgSmem {
    float2 *M;    // qp x qp double-float M (zero padded)
    float *L;     // packed lower triangle of the factor
    float *D;     // (qp / kPb) blocks kPb x kPb: Dinv_b, row-major
    float *t;     // qp: preconditioner work vector
    float2 *X, *R, *P, *AP, *Z, *RO;
};

// Shared-memory layouts of a lower triangle: packed row by row (the one-block
// solver, short of room) or full rows of stride ld (ld odd: consecutive rows
// fall on different banks).
struct LayPacked {
    __device__ __forceinline__ int operator()(int i, int j) const { return lpos(i, j); }
};
struct LayFull {
    int ld;
    __device__ __forceinline__ int operator()(int i, int j) const { return i * ld + j; }
};

// warp 0, lanes 0..7: factor the diagonal block at kb and store its inverse;
// false if a pivot is not positive
template <class Lay>
__device__ __forceinline__ bool cg_diag8_t(float *L, int kb, float *Db, Lay lay)
{
    const int lane = threadIdx.x & 31;
    const bool on = lane < kPb;
    float a[kPb];
#pragma unroll
    for (int k = 0; k < kPb; ++k) a[k] = (on && k <= lane) ? L[lay(kb + lane, kb + k)] : 0.f;
    bool ok = true;
    float rsd = 1.f;   // this lane's 1 / L_ii
#pragma unroll
    for (int j = 0; j < kPb; ++j) {
        const float d = __shfl_sync(0xffffffffu, a[j], j);
        const bool okj = (d > 0.f) && isfinite(d);
        ok = ok && okj;
        const float rs = okj ? rsqrtf(d) : 1.f;
        if (lane == j) { a[j] = okj ? d * rs : 1.f; rsd = rs; }
        else if (lane > j) a[j] *= rs;
#pragma unroll
        for (int k = 1; k < kPb; ++k) {
            if (k > j) {
                const float lkj = __shfl_sync(0xffffffffu, a[j], k);
                if (lane >= k) a[k] = fmaf(-a[j], lkj, a[k]);
            }
        }
    }
    // lane c: column c of the inverse, x_i = (delta_ic - sum_{m<i} L_im x_m) / L_ii
    float x[kPb];
#pragma unroll
    for (int i = 0; i < kPb; ++i) {
        float s = (i == lane) ? 1.f : 0.f;
#pragma unroll
        for (int m = 0; m < kPb; ++m)
            if (m < i) s = fmaf(-__shfl_sync(0xffffffffu, a[m], i), x[m], s);
        const float ri = __shfl_sync(0xffffffffu, rsd, i);   // every lane takes part in the shuffle
        x[i] = (i >= lane) ? s * ri : 0.f;
    }
    if (on) {
#pragma unroll
        for (int k = 0; k < kPb; ++k) {
            if (k <= lane) L[lay(kb + lane, kb + k)] = a[k];
            Db[k * kPb + lane] = x[k];
        }
    }
    return ok;
}

// dst[lay(i, j)] = src[i * ld + j] for the lower triangle j <= i of an np x np
// tile (rows i >= n: the identity), by the whole block with eight loads in
// flight per thread (a load-then-store loop waits one L2 round trip per element)
template <class Lay>
__device__ __forceinline__ void load_lower(float *dst, Lay lay, const float *__restrict__ src, size_t ld, int n, int np)
{
    const int total = np * np;
    for (int e0 = threadIdx.x; e0 < total; e0 += 8 * blockDim.x) {
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int e = e0 + u * blockDim.x;
            const int i = e / np, j = e - i * np;
            v[u] = (e < total && j <= i && i < n) ? __ldcg(src + (size_t)i * ld + j) : (i == j ? 1.f : 0.f);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int e = e0 + u * blockDim.x;
            const int i = e / np, j = e - i * np;
            if (e < total && j <= i) dst[lay(i, j)] = v[u];
        }
    }
}

__device__ __forceinline__ bool cg_diag8(float *L, int kb, float *Db)
{
    return cg_diag8_t(L, kb, Db, LayPacked());
}

// In-place FP32 Cholesky of the qp x qp matrix in S.L (layout lay; qp % 32 ==
// 0, rows beyond the problem set to the identity), right-looking by 8-column
// panels; S.D receives the inverses of the 8 x 8 diagonal blocks.  Block-
// uniform result: false when a pivot is not positive.
template <class Lay>
static __device__ bool cg_factor_t(CgSmem &S, int qp, Lay lay)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int nb = qp / kPb;
    __shared__ int bad;
    if (tid == 0) bad = 0;
    __syncthreads();
    for (int b = 0; b < nb; ++b) {
        const int kb = b * kPb;
        if (warp == 0) {
            const bool ok = cg_diag8_t(S.L, kb, S.D + b * kPb * kPb, lay);
            if (!ok && lane == 0) bad = 1;
        }
        __syncthreads();
        if (bad || b + 1 == nb) break;
        {   // rows below: L_rc = sum_k A_rk Dinv_b[c][k]; 4 rows per warp, 8 lanes a row
            const int grp = lane >> 3, c = lane & 7;
            const float *Db = S.D + b * kPb * kPb;
            float dr[kPb];
#pragma unroll
            for (int k = 0; k < kPb; ++k) dr[k] = Db[c * kPb + k];
            for (int r0 = kb + kPb + warp * 4; r0 < qp; r0 += nw * 4) {
                const int r = r0 + grp;
                const float av = (r < qp) ? S.L[lay(r, kb + c)] : 0.f;
                float acc = 0.f;
#pragma unroll
                for (int k = 0; k < kPb; ++k) acc = fmaf(__shfl_sync(0xffffffffu, av, grp * 8 + k), dr[k], acc);
                if (r < qp) S.L[lay(r, kb + c)] = acc;
            }
        }
        __syncthreads();
        // trailing triangle, a warp per row: A_rc -= sum_k L_rk L_ck, kb + 8 <= c <= r
        for (int r = kb + kPb + warp; r < qp; r += nw) {
            float lr[kPb];
#pragma unroll
            for (int k = 0; k < kPb; ++k) lr[k] = S.L[lay(r, kb + k)];
            for (int c = kb + kPb + lane; c <= r; c += 32) {
                const int pc = lay(c, kb);
                float acc = 0.f;
#pragma unroll
                for (int k = 0; k < kPb; ++k) acc = fmaf(lr[k], S.L[pc + k], acc);
                S.L[lay(r, c)] -= acc;
            }
        }
        __syncthreads();
    }
    const bool ok = !bad;
    __syncthreads();
    return ok;
}

static __device__ bool cg_factor_packed(CgSmem &S, int qp)
{
    return cg_factor_t(S, qp, LayPacked());
}

constexpr int kBcNb = 128;     // panel width of the blocked factor
constexpr int kBcTile = 64;    // trailing-update tile
constexpr int kBcMaxQ = 1024;

// sum_j a_j b_j, j < q <= kBcMaxQ, double-float, fixed order; every thread of
// the block returns the same value (and every block, given equal inputs)
__device__ __forceinline__ float2 bc_dot(const float2 *a, const float2 *b, int q, float2 *red)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    float2 s = make_float2(0.f, 0.f);
    for (int j = tid; j < q; j += blockDim.x) s = dfx_add(s, dfx_mul(a[j], b[j]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s = dfx_add(s, shfl_xor_f2(s, o));
    if (lane == 0) red[warp] = s;
    __syncthreads();
    float2 t = red[0];
    for (int w = 1; w < nw; ++w) t = dfx_add(t, red[w]);
    __syncthreads();
    return t;
}

// Blocked FP32 Cholesky of fl32(M) (M the q x q double-float pairs Mf, q <=
// kBcMaxQ) by the whole cooperative grid, right-looking by 128-wide panels,
// three grid barriers a panel: block 0 factors the diagonal block in shared
// memory (cg_factor_packed; the inverses of its 8 x 8 diagonal blocks go to
// Dg), every block then solves a share of the panel's rows (x L_kk' = a, a
// warp per row), and every block updates a share of the 64 x 64 tiles of the
// trailing lower triangle.  A pivot that is not positive restarts the factor
// with a diagonal shift (1e-7 max diag, then x100, at most six attempts).
// The factor goes to Lg (row-major, row stride q, lower triangle).  S holds
// one 128-panel's packed factor (cg_fast_smem(kCgMaxQ) bytes); red has one
// slot per warp.  Returns 1 when factored (*shift_out = the shift used), 0
// when every attempt failed, -1 when a grid barrier timed out; the same value
// in every block.  b, G: this block's rank and the number of blocks that
// factor this matrix (a group of a larger cooperative launch, or all of it).
static __device__ int bc_factor(int q, const float2 *__restrict__ Mf, float *__restrict__ Lg, float *__restrict__ Dg,
                                int *fflag, unsigned *bar, int *err, CgSmem &S, float2 *red, float *shift_out,
                                int b, int G)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int gw = b * nw + warp, ngw = G * nw;
    constexpr int kLdF = kBcNb + 1;                     // odd row stride: rows on distinct banks
    float *LF = reinterpret_cast<float *>(S.M);         // a 128-panel's diagonal block (kBcNb x kLdF)
    CgSmem SF = S;
    SF.L = LF;
    // the largest diagonal entry (scale of the breakdown shift), in every block
    float md = 0.f;
    for (int j = tid; j < q; j += blockDim.x) md = fmaxf(md, Mf[(size_t)j * q + j].x);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) md = fmaxf(md, __shfl_xor_sync(0xffffffffu, md, o));
    if (lane == 0) red[warp].x = md;
    __syncthreads();
    float maxdiag = 0.f;
    for (int w = 0; w < nw; ++w) maxdiag = fmaxf(maxdiag, red[w].x);
    __syncthreads();
    float shift = 0.f;
    bool factored = false;
    for (int attempt = 0; attempt < 6 && !factored; ++attempt) {
        // fl32(M) + shift, lower triangle, into Lg
        for (long long e = (long long)b * blockDim.x + tid; e < (long long)q * q; e += (long long)G * blockDim.x) {
            const int i = (int)(e / q), j = (int)(e - (long long)i * q);
            if (j <= i) Lg[e] = Mf[e].x + (i == j ? shift : 0.f);
        }
        if (b == 0 && tid == 0) *fflag = 0;
        if (!group_barrier(bar, err, b, G)) return -1;
        bool bad = false;
        for (int kb = 0; kb < q && !bad; kb += kBcNb) {
            const int nbk = q - kb < kBcNb ? q - kb : kBcNb;
            const int qpk = (nbk + 31) & ~31;
            // (1) block 0: the diagonal block, in full rows of stride kLdF in the
            // (free) M region
            if (b == 0) {
                load_lower(LF, LayFull{kLdF}, Lg + (size_t)kb * q + kb, (size_t)q, nbk, qpk);
                __syncthreads();
                const bool ok = cg_factor_t(SF, qpk, LayFull{kLdF});
                if (!ok) {
                    if (tid == 0) atomicExch(fflag, 1);
                } else {
                    for (int i = warp; i < nbk; i += nw)
                        for (int j = lane; j <= i; j += 32) Lg[(size_t)(kb + i) * q + kb + j] = LF[i * kLdF + j];
                    for (int e = tid; e < ((nbk + kPb - 1) / kPb) * kPb * kPb; e += blockDim.x)
                        Dg[(size_t)kb * kPb + e] = S.D[e];
                }
            }
            if (!group_barrier(bar, err, b, G)) return -1;
            if (ld_relaxed_i32(fflag)) {
                // every block has read the flag before block 0 clears it for the next attempt
                bad = true;
                if (!group_barrier(bar, err, b, G)) return -1;
                break;
            }
            if (kb + nbk >= q) break;
            // (2) the panel's rows below: x L_kk' = a, a warp per row (every block
            // first copies L_kk into its shared memory, with 1 / L_cc in S.t)
            if (b != 0) load_lower(LF, LayFull{kLdF}, Lg + (size_t)kb * q + kb, (size_t)q, nbk, nbk);
            __syncthreads();
            for (int c = tid; c < nbk; c += blockDim.x) S.t[c] = 1.f / LF[c * kLdF + c];
            __syncthreads();
            for (int r = kb + nbk + gw; r < q; r += ngw) {
                float a[kBcNb / 32];
#pragma unroll
                for (int m = 0; m < kBcNb / 32; ++m) {
                    const int j = lane + 32 * m;
                    a[m] = j < nbk ? __ldcg(&Lg[(size_t)r * q + kb + j]) : 0.f;
                }
                for (int c = 0; c < nbk; ++c) {
                    const int own = c & 31, slot = c >> 5;
                    float ac = 0.f;
#pragma unroll
                    for (int m = 0; m < kBcNb / 32; ++m)
                        if (m == slot) ac = a[m];
                    const float xc = __shfl_sync(0xffffffffu, ac, own) * S.t[c];
#pragma unroll
                    for (int m = 0; m < kBcNb / 32; ++m) {
                        const int j = lane + 32 * m;
                        if (j > c && j < nbk) a[m] = fmaf(-LF[j * kLdF + c], xc, a[m]);
                        if (j == c) a[m] = xc;
                    }
                }
#pragma unroll
                for (int m = 0; m < kBcNb / 32; ++m) {
                    const int j = lane + 32 * m;
                    if (j < nbk) Lg[(size_t)r * q + kb + j] = a[m];
                }
            }
            if (!group_barrier(bar, err, b, G)) return -1;
            // (3) trailing update A_ij -= L_i,panel L_j,panel' over 64 x 64 tiles, j <= i
            {
                const int t0 = kb + nbk;
                const int nt = (q - t0 + kBcTile - 1) / kBcTile;
                const int ntiles = nt * (nt + 1) / 2;
                float *TA = reinterpret_cast<float *>(S.M);                 // [64][nbk + 1]
                float *TB = TA + kBcTile * (kBcNb + 1);                    // [64][nbk + 1]
                const int ld = kBcNb + 1;
                for (int tt = b; tt < ntiles; tt += G) {
                    int ti = 0, rem = tt;
                    while (rem > ti) { rem -= ti + 1; ++ti; }
                    const int tj = rem;
                    const int i0 = t0 + ti * kBcTile, j0 = t0 + tj * kBcTile;
                    // the two 64-row strips of the panel, four loads of each in flight per thread
                    for (int e0 = tid; e0 < kBcTile * nbk; e0 += 4 * blockDim.x) {
                        float va[4], vb[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int e = e0 + u * blockDim.x;
                            const int rr = e / nbk, m = e - rr * nbk;
                            const bool in = e < kBcTile * nbk;
                            va[u] = (in && i0 + rr < q) ? __ldcg(&Lg[(size_t)(i0 + rr) * q + kb + m]) : 0.f;
                            vb[u] = (in && j0 + rr < q) ? __ldcg(&Lg[(size_t)(j0 + rr) * q + kb + m]) : 0.f;
                        }
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int e = e0 + u * blockDim.x;
                            const int rr = e / nbk, m = e - rr * nbk;
                            if (e < kBcTile * nbk) {
                                TA[rr * ld + m] = va[u];
                                TB[rr * ld + m] = vb[u];
                            }
                        }
                    }
                    __syncthreads();
                    const int ii = tid >> 3, jc = tid & 7;   // row ii, columns jc + 8u
                    float acc[kBcTile / 8];
#pragma unroll
                    for (int u = 0; u < kBcTile / 8; ++u) acc[u] = 0.f;
                    for (int m = 0; m < nbk; ++m) {
                        const float av = TA[ii * ld + m];
#pragma unroll
                        for (int u = 0; u < kBcTile / 8; ++u) acc[u] = fmaf(av, TB[(jc + 8 * u) * ld + m], acc[u]);
                    }
                    const int i = i0 + ii;
#pragma unroll
                    for (int u = 0; u < kBcTile / 8; ++u) {
                        const int j = j0 + jc + 8 * u;
                        if (i < q && j < q && j <= i) {
                            float *lij = Lg + (size_t)i * q + j;
                            *lij = __ldcg(lij) - acc[u];   // other blocks updated it in earlier panels
                        }
                    }
                    __syncthreads();
                }
            }
            if (!group_barrier(bar, err, b, G)) return -1;
        }
        factored = !bad;
        if (!factored) shift = (shift == 0.f) ? 1e-7f * maxdiag : shift * 100.f;
    }
    *shift_out = shift;
    return factored ? 1 : 0;
}

// Y = L^{-1} for the packed lower-triangular factor in S.L (qp x qp, qp % 8 ==
// 0) whose 8 x 8 diagonal blocks have the inverses S.D: blocked forward
// substitution on the identity, Y_b = Dinv_b T_b for the block rows b, then
// T_r -= L_rb Y_b for every row r below.  Y row-major with row stride ld
// (shared memory); one block.
static __device__ void tri_inverse_packed(const CgSmem &S, int qp, float *Y, int ld)
{
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    const int nb = qp / kPb;
    for (int e = tid; e < qp * qp; e += nt) {
        const int i = e / qp, j = e - i * qp;
        Y[i * ld + j] = (i == j) ? 1.f : 0.f;
    }
    __syncthreads();
    for (int b = 0; b < nb; ++b) {
        const int kb = b * kPb;
        for (int c = tid; c < kb + kPb; c += nt) {   // column c of the block rows
            const float *Db = S.D + b * kPb * kPb;
            float yv[kPb], out[kPb];
#pragma unroll
            for (int k = 0; k < kPb; ++k) yv[k] = Y[(kb + k) * ld + c];
#pragma unroll
            for (int i = 0; i < kPb; ++i) {
                float a = 0.f;
#pragma unroll
                for (int k = 0; k < kPb; ++k) a = fmaf(Db[i * kPb + k], yv[k], a);
                out[i] = a;
            }
#pragma unroll
            for (int i = 0; i < kPb; ++i) Y[(kb + i) * ld + c] = out[i];
        }
        __syncthreads();
        // rows below, a warp per row, over the columns <= kb + 7
        for (int r = kb + kPb + warp; r < qp; r += nw) {
            float lr[kPb];
#pragma unroll
            for (int k = 0; k < kPb; ++k) lr[k] = S.L[lpos(r, kb + k)];
            for (int c = lane; c < kb + kPb; c += 32) {
                float a = 0.f;
#pragma unroll
                for (int k = 0; k < kPb; ++k) a = fmaf(lr[k], Y[(kb + k) * ld + c], a);
                Y[r * ld + c] -= a;
            }
        }
        __syncthreads();
    }
}

static inline size_t cg_fast_smem(int q)
{
    const size_t qp = (size_t)((q + 31) & ~31);
    return qp * qp * sizeof(float2) + ((qp * (qp + 1)) / 2 + (qp / kPb) * kPb * kPb + qp) * sizeof(float) +
           6 * qp * sizeof(float2);
}

}  // namespace svm
