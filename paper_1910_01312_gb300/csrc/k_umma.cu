// k_umma.cu -- Gram of the gathered free rows on the fifth-generation tensor
// cores (tcgen05 / UMMA, sm_103a), for the preconditioner of the large-free-set
// Newton solve (Proposition 3.5: the reduced matrix I + sigma (G - h h'/p)
// with G = X_J' X_J and h = X_J' 1).
//
// Each block takes a contiguous share of J and accumulates C_b = X_S' X_S
// (S = its rows) in tensor memory: D[m][n] += sum_k A[m][k] B[n][k] with
// A = B = the stage's rows transposed (feature m, sample k), one
// tcgen05.mma.cta_group::1.kind::tf32 per 8 samples (M = 128 features, zero
// padded above q; N = q).  The rows are gathered with plain coalesced loads
// (the rows of J are scattered, 4 bytes x 8 consecutive features per lane
// group) and stored into a K-major, unswizzled core-matrix layout in shared
// memory, two stages deep: while the tensor core works on one stage the block
// gathers the next.  The exact column sums h_b are kept beside it (FP32
// TwoSum compensation, double-float per block).  Products are TF32 (10-bit
// mantissa), sums FP32: the CG operator stays exact, so this rounding only
// sets how fast CG converges.
//
// Every wait is bounded: a commit that does not arrive within ~1 s records
// DEV_TIMEOUT, the block frees its tensor memory and returns.
#include "internal.cuh"

namespace svm {

namespace {

constexpr int kUmRows = 64;                          // gathered rows (K) per stage
constexpr int kUmM = 128;                            // MMA rows (features, zero padded)
constexpr int kUmStageBytes = kUmM * kUmRows * 4;    // 32 KB of FP32
constexpr unsigned kUmLbo = 128;                     // K-adjacent core matrices (8 rows x 16 B) are contiguous
constexpr unsigned kUmSbo = (kUmRows / 4) * 128;     // next 8 features: after the stage's K/4 core matrices
constexpr int kUmThreads = 256;
constexpr int kUmCols = 128;                         // tensor-memory columns allocated (N <= 128)
constexpr int kUmMaxQ = 128;
constexpr size_t kUmSmem = 2 * (size_t)kUmStageBytes + 1024;   // + alignment slack

// Shared-memory matrix descriptor (tcgen05): start address, leading-dimension
// byte offset (between core matrices adjacent in K for a K-major operand),
// stride byte offset (between core matrices adjacent in M/N), all in 16-byte
// units; descriptor version 1 (bits 46-47), no swizzle, base offset 0.
__device__ __forceinline__ unsigned long long umma_desc(unsigned saddr, unsigned lbo, unsigned sbo)
{
    unsigned long long d = 0;
    d |= (unsigned long long)((saddr >> 4) & 0x3FFFu);
    d |= (unsigned long long)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (unsigned long long)((sbo >> 4) & 0x3FFFu) << 32;
    d |= 1ull << 46;
    return d;
}

// Instruction descriptor of kind::tf32: D FP32 (bits 4-5 = 1), A and B TF32
// (bits 7-9, 10-12 = 2), both K-major (bits 15, 16 = 0), N >> 3 at bit 17,
// M >> 4 at bit 24.
__host__ __device__ constexpr unsigned umma_idesc_tf32(int M, int N)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((unsigned)(N >> 3) << 17) | ((unsigned)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_mma_tf32(unsigned dtmem, unsigned long long adesc, unsigned long long bdesc,
                                            unsigned idesc, int accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tc_commit(unsigned long long *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 32 lanes x 32 bits, 16 consecutive columns: thread t of the warp gets row
// (warp's lane quarter) + t, columns c..c+15.
__device__ __forceinline__ void tc_ld16(unsigned taddr, unsigned (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Thread (warp w, lane l) of a stage gathers, for u = 0..31, the element of
// sample k = 4 (w + 8 (u & 1)) + (l >> 3) and feature m = 8 (u >> 1) + (l & 7):
// eight lanes read 32 contiguous bytes of one row, and the 32 lanes of a warp
// store to 32 distinct banks of the core-matrix layout.
__device__ __forceinline__ int um_k(int warp, int lane, int u) { return 4 * (warp + 8 * (u & 1)) + (lane >> 3); }
__device__ __forceinline__ int um_m(int lane, int u) { return 8 * (u >> 1) + (lane & 7); }

__global__ void __launch_bounds__(kUmThreads) gram_umma_kernel(const float *__restrict__ X, int q,
                                                               const int32_t *__restrict__ J, long long p,
                                                               float *__restrict__ cpart, float2 *__restrict__ hpart,
                                                               int *err)
{
    extern __shared__ unsigned char um_dyn[];
    __shared__ __align__(8) unsigned long long mbar[2];
    __shared__ unsigned tmem_slot;
    __shared__ int jrow[kUmRows];
    __shared__ float2 hsm[kUmThreads / 32][kUmMaxQ];
    unsigned char *base =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(um_dyn) + 1023) & ~(uintptr_t)1023);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int G = gridDim.x;
    const long long per = (p + G - 1) / G;
    const long long r0 = (long long)blockIdx.x * per;
    const long long r1 = r0 + per < p ? r0 + per : p;
    const int nst = r1 > r0 ? (int)((r1 - r0 + kUmRows - 1) / kUmRows) : 0;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(kUmCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 32) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        mbar_fence_init();
    }
    // features m >= q stay zero in both stages
    for (int i = threadIdx.x; i < 2 * kUmStageBytes / 16; i += kUmThreads)
        reinterpret_cast<float4 *>(base)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = tmem_slot;
    const unsigned idesc = umma_idesc_tf32(kUmM, q);

    float hs[16], hc[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) hs[i] = hc[i] = 0.f;
    int ok = 1;
    for (int it = 0; it < nst; ++it) {
        const int b = it & 1;
        // the MMAs of stage it - 2 read this buffer: wait for their commit
        if (it >= 2 && ok) ok = mbar_wait_bounded(&mbar[b], (unsigned)((it - 2) >> 1) & 1u, err) ? 1 : 0;
        const long long rb = r0 + (long long)it * kUmRows;
        if (threadIdx.x < kUmRows) jrow[threadIdx.x] = (rb + threadIdx.x < r1) ? J[rb + threadIdx.x] : -1;
        if (!__syncthreads_and(ok)) { ok = 0; break; }
        float x[32];
#pragma unroll
        for (int u = 0; u < 32; ++u) {
            const int jr = jrow[um_k(warp, lane, u)], m = um_m(lane, u);
            x[u] = (jr >= 0 && m < q) ? __ldcs(X + (long long)jr * q + m) : 0.f;
        }
        unsigned char *st = base + b * kUmStageBytes;
#pragma unroll
        for (int u = 0; u < 32; ++u) {
            const int k = um_k(warp, lane, u), m = um_m(lane, u);
            const unsigned off = (unsigned)(m >> 3) * kUmSbo + (unsigned)(k >> 2) * kUmLbo + (unsigned)(m & 7) * 16u +
                                 (unsigned)(k & 3) * 4u;
            *reinterpret_cast<float *>(st + off) = x[u];
            float sn, er;
            two_sum(hs[u >> 1], x[u], sn, er);
            hs[u >> 1] = sn;
            hc[u >> 1] += er;
        }
        // the generic-proxy stores must be visible to the tensor core's (async proxy) reads
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0) {
            tc_fence_after();
            const unsigned sa = smem_u32(st);
#pragma unroll
            for (int s = 0; s < kUmRows / 8; ++s) {
                // 8 samples = two core matrices along K
                const unsigned long long d = umma_desc(sa + s * 2 * kUmLbo, kUmLbo, kUmSbo);
                tc_mma_tf32(tmem, d, d, idesc, (it > 0 || s > 0) ? 1 : 0);
            }
            tc_commit(&mbar[b]);
        }
    }
    if (nst > 0 && ok) ok = mbar_wait_bounded(&mbar[(nst - 1) & 1], (unsigned)((nst - 1) >> 1) & 1u, err) ? 1 : 0;
    tc_fence_after();
    ok = __syncthreads_and(ok);

    // C_b rows from tensor memory: warp w < 4 reads lanes 32w..32w+31 (features)
    float *C = cpart + (size_t)blockIdx.x * q * q;
    if (warp < 4) {
        const int m = 32 * warp + lane;
        for (int c0 = 0; c0 < q; c0 += 16) {
            unsigned r[16];
            if (nst > 0 && ok) {
                tc_ld16(tmem + ((unsigned)(32 * warp) << 16) + (unsigned)c0, r);
            } else {
#pragma unroll
                for (int j = 0; j < 16; ++j) r[j] = 0u;
            }
            if (m < q) {
#pragma unroll
                for (int j = 0; j < 16; j += 4)
                    *reinterpret_cast<float4 *>(&C[(size_t)m * q + c0 + j]) =
                        make_float4(__uint_as_float(r[j]), __uint_as_float(r[j + 1]), __uint_as_float(r[j + 2]),
                                    __uint_as_float(r[j + 3]));
            }
        }
    }
    // column sums: the four lanes of a feature (l, l ^ 8, l ^ 16, l ^ 24), then
    // the eight warps in order
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        float hi, lo;
        two_sum(hs[i], hc[i], hi, lo);
        float2 t = make_float2(hi, lo);
        t = dfx_add(t, shfl_xor_f2(t, 8));
        t = dfx_add(t, shfl_xor_f2(t, 16));
        if (lane < 8) hsm[warp][8 * i + lane] = t;
    }
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x < q) {
        float2 t = make_float2(0.f, 0.f);
        for (int w = 0; w < kUmThreads / 32; ++w) t = dfx_add(t, hsm[w][threadIdx.x]);
        hpart[(size_t)blockIdx.x * q + threadIdx.x] = t;
    }
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kUmCols) : "memory");
    }
}

// ---------------------------------------------------------------------------
// The same Gram for 128 < q <= 1024 (q % 16 == 0), where one tensor-memory
// accumulator cannot hold q x q.  The lower triangle is cut into pairs (ti, cj)
// -- features 128 ti .. 128 ti + 127 (the MMA's M = 128 rows, A) against
// features 256 cj .. 256 cj + 255 (N <= 256 columns, B) for each chunk cj that
// reaches the diagonal of row tile ti -- and blockIdx.y splits the rows of J
// (split-K).  A stage gathers 32 rows: B's features always, A's only when they
// lie outside B's range (otherwise A's descriptor points into B's panel).  The
// panels are K-major in the 128-byte swizzled layout (32 rows = 128 bytes of K
// per feature).  A thread loads 16 bytes (4 features of one row) and stores
// the 4 values at offsets fixed for the thread, the 32 lanes of a warp on 32
// distinct banks; the rows of the next stage load while a stage is stored and
// its MMAs issued.  The
// pair whose chunk holds A's features also sums A's columns (h).  Each
// feature is gathered by several pairs (about 6 x the rows' bytes at q =
// 784); products are TF32, sums FP32 -- the preconditioner's Gram, as above.
constexpr int kWgK = 32;                                 // gathered rows per stage
constexpr int kWgBN = 256;                               // B features (MMA N, max)
constexpr int kWgAM = 128;                               // A features (MMA M)
constexpr unsigned kWgSbo = 8 * kWgK * 4;                // next 8 features: one 1024-byte swizzle atom
constexpr int kWgBBytes = kWgBN * kWgK * 4;              // 32 KB
constexpr int kWgABytes = kWgAM * kWgK * 4;              // 16 KB
constexpr int kWgStageBytes = kWgBBytes + kWgABytes;
constexpr int kWgCols = 256;                             // tensor-memory columns
constexpr size_t kWgSmem = 2 * (size_t)kWgStageBytes + 1024;

__host__ __device__ inline int wg_chunks(int ti, int q)   // column chunks of row tile ti
{
    const int last = (128 * ti + 127 < q - 1) ? 128 * ti + 127 : q - 1;
    return last / kWgBN + 1;
}

__host__ __device__ inline int wg_pairs(int q)
{
    int n = 0;
    for (int ti = 0; ti * kWgAM < q; ++ti) n += wg_chunks(ti, q);
    return n;
}

// Shared-memory descriptor of a K-major operand in the 128-byte swizzled
// layout: each M/N row holds its 32 K values (128 bytes) with 16-byte chunk c
// stored at chunk c ^ (row & 7), eight rows form a 1024-byte atom, atoms SBO
// bytes apart (layout type 2 at bits 61-63; the leading offset is unused for
// this layout and set to 1).  A K step of 8 TF32 values advances the start
// address by 32 bytes inside the atom.
__device__ __forceinline__ unsigned long long umma_desc_sw128(unsigned saddr, unsigned sbo)
{
    unsigned long long d = 0;
    d |= (unsigned long long)((saddr >> 4) & 0x3FFFu);
    d |= 1ull << 16;
    d |= (unsigned long long)((sbo >> 4) & 0x3FFFu) << 32;
    d |= 1ull << 46;
    d |= 2ull << 61;
    return d;
}

// the 4 values of one lane (4 consecutive features of one gathered row) into
// the swizzled panel at st, at the lane's fixed offsets
__device__ __forceinline__ void wg_store4(unsigned char *st, const unsigned (&soff)[4], const float4 &v)
{
    *reinterpret_cast<float *>(st + soff[0]) = v.x;
    *reinterpret_cast<float *>(st + soff[1]) = v.y;
    *reinterpret_cast<float *>(st + soff[2]) = v.z;
    *reinterpret_cast<float *>(st + soff[3]) = v.w;
}

__global__ void __launch_bounds__(kUmThreads, 2) gram_umma_wide_kernel(const float *__restrict__ X, int q,
                                                                    const int32_t *__restrict__ J, long long p,
                                                                    float *__restrict__ cpart,
                                                                    float2 *__restrict__ hpart, int *err,
                                                                    const int *skip)
{
    if (skip && __ldcg(skip)) return;
    extern __shared__ unsigned char um_dyn[];
    __shared__ __align__(8) unsigned long long mbar[2];
    __shared__ unsigned tmem_slot;
    __shared__ float2 hsm[2][kWgAM];
    unsigned char *base =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(um_dyn) + 1023) & ~(uintptr_t)1023);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int t = blockIdx.x, ti = 0;
    while (t >= wg_chunks(ti, q)) {
        t -= wg_chunks(ti, q);
        ++ti;
    }
    const int cj = t;
    const int b0 = kWgBN * cj, a0 = kWgAM * ti;
    const int nb = (q - b0 < kWgBN) ? q - b0 : kWgBN;   // a multiple of 16
    const bool inside = (ti >> 1) == cj;                // A's features are B's 128 (ti & 1) .. + 127
    const int KS = gridDim.y, ks = blockIdx.y;
    const long long per = (p + KS - 1) / KS;
    const long long r0 = (long long)ks * per;
    const long long r1 = r0 + per < p ? r0 + per : p;
    const int nst = r1 > r0 ? (int)((r1 - r0 + kWgK - 1) / kWgK) : 0;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(kWgCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 32) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        mbar_fence_init();
    }
    for (int i = threadIdx.x; i < 2 * kWgStageBytes / 16; i += kUmThreads)
        reinterpret_cast<float4 *>(base)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = tmem_slot;
    const unsigned idesc = umma_idesc_tf32(kWgAM, nb);
    // lane -> data: lane bits 0-3 give the stage row within the warp's half of
    // the stage (rows 16 (w & 1) .. + 15), lane bit 4 and w >> 1 the lane's
    // 4-feature group c4 within each 32 features (two lanes cover 32
    // contiguous bytes of a row).  Feature m = 32 g + 4 c4 + j of row k sits at
    // g * 4096 + soff[j]; for a fixed j the 32 lanes of a warp hit 32 distinct
    // banks: (k >> 2) ^ (m & 7) takes 8 values, k & 3 four.
    const int kr = 16 * (warp & 1) + (lane & 15);
    const int c4 = 2 * (warp >> 1) + (lane >> 4);
    unsigned soff[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int mj = 4 * (c4 & 1) + j;
        soff[j] = (unsigned)(c4 >> 1) * kWgSbo + (unsigned)mj * 128u + ((unsigned)((kr >> 2) ^ mj) << 4) +
                  (unsigned)(kr & 3) * 4u;
    }
    const int gA = (ti & 1) * 4;             // A's first 32-feature group inside B

    float hs[16], hc[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) hs[i] = hc[i] = 0.f;
    // software pipeline: the rows of stage it + 1 load into registers while
    // stage it is stored and its MMAs issued; row indices two stages ahead
    auto row_of = [&](int st) -> int {
        const long long r = r0 + (long long)st * kWgK + kr;
        return (st < nst && r < r1) ? __ldg(&J[r]) : -1;
    };
    float4 vb[kWgBN / 32], va[kWgAM / 32];
    auto load_rows = [&](int jr) {
        const float *row = X + (long long)(jr < 0 ? 0 : jr) * q;
#pragma unroll
        for (int g = 0; g < kWgBN / 32; ++g) {
            const int m = b0 + 32 * g + 4 * c4;
            vb[g] = (jr >= 0 && m < q) ? __ldcg(reinterpret_cast<const float4 *>(row + m))
                                       : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        if (!inside) {
#pragma unroll
            for (int g = 0; g < kWgAM / 32; ++g) {
                const int m = a0 + 32 * g + 4 * c4;
                va[g] = (jr >= 0 && m < q) ? __ldcg(reinterpret_cast<const float4 *>(row + m))
                                           : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
    };
    int jnext = row_of(1);
    load_rows(row_of(0));
    int ok = 1;
    for (int it = 0; it < nst; ++it) {
        const int b = it & 1;
        if (it >= 2 && ok) ok = mbar_wait_bounded(&mbar[b], (unsigned)((it - 2) >> 1) & 1u, err) ? 1 : 0;
        if (!__syncthreads_and(ok)) { ok = 0; break; }
        unsigned char *st = base + b * kWgStageBytes;
#pragma unroll
        for (int g = 0; g < kWgBN / 32; ++g) wg_store4(st + g * 4 * kWgSbo, soff, vb[g]);
        if (!inside) {
#pragma unroll
            for (int g = 0; g < kWgAM / 32; ++g) wg_store4(st + kWgBBytes + g * 4 * kWgSbo, soff, va[g]);
        } else {
#pragma unroll
            for (int gg = 0; gg < kWgAM / 32; ++gg) {
                const float4 v = gA ? vb[4 + gg] : vb[gg];
                const float xs[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float sn, er;
                    two_sum(hs[4 * gg + j], xs[j], sn, er);
                    hs[4 * gg + j] = sn;
                    hc[4 * gg + j] += er;
                }
            }
        }
        // the next stage's rows (this stage's values are in shared memory now)
        const int jn2 = row_of(it + 2);
        load_rows(jnext);
        jnext = jn2;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0) {
            tc_fence_after();
            const unsigned sb = smem_u32(st);
            const unsigned sa = inside ? sb + (unsigned)(ti & 1) * 16u * kWgSbo : sb + (unsigned)kWgBBytes;
#pragma unroll
            for (int s = 0; s < kWgK / 8; ++s) {
                const unsigned long long ad = umma_desc_sw128(sa + s * 32u, kWgSbo);
                const unsigned long long bd = umma_desc_sw128(sb + s * 32u, kWgSbo);
                tc_mma_tf32(tmem, ad, bd, idesc, (it > 0 || s > 0) ? 1 : 0);
            }
            tc_commit(&mbar[b]);
        }
    }
    if (nst > 0 && ok) ok = mbar_wait_bounded(&mbar[(nst - 1) & 1], (unsigned)((nst - 1) >> 1) & 1u, err) ? 1 : 0;
    tc_fence_after();
    ok = __syncthreads_and(ok);

    // D rows from tensor memory: warp w reads lanes 32 (w & 3) .. + 31 (A's
    // features), columns 128 (w >> 2) .. + 127 of B
    {
        float *C = cpart + (size_t)ks * q * q;
        const int quarter = warp & 3, half = warp >> 2;
        const int a = a0 + 32 * quarter + lane;
        const int cend = (128 * half + 128 < nb) ? 128 * half + 128 : nb;
        for (int c0 = 128 * half; c0 < cend; c0 += 16) {
            unsigned r[16];
            if (nst > 0 && ok) {
                tc_ld16(tmem + ((unsigned)(32 * quarter) << 16) + (unsigned)c0, r);
            } else {
#pragma unroll
                for (int j = 0; j < 16; ++j) r[j] = 0u;
            }
            if (a < q) {
#pragma unroll
                for (int j = 0; j < 16; j += 4)
                    *reinterpret_cast<float4 *>(&C[(size_t)a * q + b0 + c0 + j]) =
                        make_float4(__uint_as_float(r[j]), __uint_as_float(r[j + 1]), __uint_as_float(r[j + 2]),
                                    __uint_as_float(r[j + 3]));
            }
        }
    }
    if (inside) {
        // A's column sums: the 16 lanes of a 4-feature group (lane bits 0-3 =
        // the row), then the two halves of the stage rows in order
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            float hi, lo;
            two_sum(hs[i], hc[i], hi, lo);
            float2 v = make_float2(hi, lo);
#pragma unroll
            for (int o = 1; o < 16; o <<= 1) v = dfx_add(v, shfl_xor_f2(v, o));
            if ((lane & 15) == 0) hsm[warp & 1][32 * (i >> 2) + 4 * c4 + (i & 3)] = v;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (inside && threadIdx.x < kWgAM && a0 + (int)threadIdx.x < q)
        hpart[(size_t)ks * q + a0 + threadIdx.x] = dfx_add(hsm[0][threadIdx.x], hsm[1][threadIdx.x]);
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kWgCols) : "memory");
    }
}

int g_wg_attr = 0;

// G = sum_b C_b and h = sum_b h_b in FP64, in block order (the step-level
// entry point); both triangles of G from the lower one of the partials
__global__ void gram_sum_kernel(int q, int nb, const float *__restrict__ cpart, const float2 *__restrict__ hpart,
                                double *__restrict__ Gout, double *__restrict__ hout)
{
    const long long qq = (long long)q * q;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < qq + q;
         t += (long long)gridDim.x * blockDim.x) {
        double s = 0.0;
        if (t < qq) {
            const long long a = t / q, c = t - a * q;
            const long long src = c <= a ? t : c * q + a;
            for (int b = 0; b < nb; ++b) s += (double)cpart[(size_t)b * qq + src];
            Gout[t] = s;
        } else {
            const long long j = t - qq;
            for (int b = 0; b < nb; ++b) {
                const float2 v = hpart[(size_t)b * q + j];
                s += (double)v.x + (double)v.y;
            }
            hout[j] = s;
        }
    }
}

int g_um_attr = 0;

}  // namespace

int gram_umma_blocks(const Work &W)
{
    return 2 * W.nsm;
}

size_t gram_umma_part_floats(const Work &W)
{
    const size_t q = (size_t)W.q;
    return (size_t)gram_umma_blocks(W) * (q * q + 2 * q);
}

cudaError_t launch_gram_umma(Work &W, const int32_t *J, long long p, float *cpart, float2 *hpart)
{
    const int q = (int)W.q;
    if (q < 16 || q > kUmMaxQ || q % 16 != 0 || !W.xf32) return cudaErrorInvalidValue;
    if (!g_um_attr) {
        const cudaError_t ea =
            cudaFuncSetAttribute(gram_umma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kUmSmem);
        if (ea != cudaSuccess) return ea;
        g_um_attr = 1;
    }
    gram_umma_kernel<<<gram_umma_blocks(W), kUmThreads, kUmSmem, W.st>>>((const float *)W.X, q, J, p, cpart, hpart,
                                                                          W.err);
    ++W.nlaunch;
    return cudaGetLastError();
}

int gram_wide_pairs(int q)
{
    return wg_pairs(q);
}

int gram_wide_splits(const Work &W, long long p)
{
    const long long q = W.q;
    const long long np = wg_pairs((int)q);
    long long cap = (long long)((2 * W.part_len) / (size_t)(q * q + 2 * q));
    long long ks = (2 * W.nsm + np - 1) / np;
    if (ks > cap) ks = cap;
    const long long rows = (p + kWgK - 1) / kWgK;
    if (ks > rows) ks = rows;
    return ks < 1 ? 1 : (int)ks;
}

cudaError_t launch_gram_umma_wide(Work &W, const int32_t *J, long long p, int KS, float *cpart, float2 *hpart,
                                  const int *skip)
{
    const int q = (int)W.q;
    if (q <= kUmMaxQ || q > 1024 || q % 16 != 0 || !W.xf32 || KS < 1) return cudaErrorInvalidValue;
    if ((size_t)KS * ((size_t)q * q + 2 * q) > 2 * W.part_len) return cudaErrorInvalidValue;
    if (!g_wg_attr) {
        const cudaError_t ea =
            cudaFuncSetAttribute(gram_umma_wide_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWgSmem);
        if (ea != cudaSuccess) return ea;
        g_wg_attr = 1;
    }
    gram_umma_wide_kernel<<<dim3((unsigned)wg_pairs(q), (unsigned)KS), kUmThreads, kWgSmem, W.st>>>(
        (const float *)W.X, q, J, p, cpart, hpart, W.err, skip);
    ++W.nlaunch;
    return cudaGetLastError();
}

cudaError_t launch_gram_umma_sum(Work &W, int nb, const float *cpart, const float2 *hpart, double *G, double *h)
{
    gram_sum_kernel<<<W.nsm, 256, 0, W.st>>>((int)W.q, nb, cpart, hpart, G, h);
    ++W.nlaunch;
    return cudaGetLastError();
}

}  // namespace svm
