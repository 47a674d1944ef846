// k_umma.cu -- Gram of the gathered free rows on the fifth-generation tensor
// cores (tcgen05 / UMMA, sm_103a), for the preconditioner of the large-free-set
// Newton solve (Proposition 3.5: the reduced matrix I + sigma (G - h h'/p)
// with G = X_J' X_J and h = X_J' 1).
//
// q <= 128 (gram_umma_kernel; the wide form for 128 < q <= 1024 follows it).
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
// TF32 operands must be K-major (samples contiguous), which X's rows are
// not: with the operand-transpose bits set, kind::tf32 returned zeros on
// sm_103a, while kind::f16 takes MN-major operands -- hence the gathered
// register staging here and the FP16 copy of X for the wide form.
//
// Every wait is bounded: a commit or copy that does not arrive within ~1 s
// records DEV_TIMEOUT, the block waits for what it issued, frees its tensor
// memory and returns.
#include <cuda_fp16.h>

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
// (split-K).
//
// The operands come from X16, an FP16 copy of X with a power-of-two scale
// 2^k_f per feature (made once per X, x16_prepare; rows padded to 128-byte
// multiples): FP16's 11-bit significand is TF32's, and the scale keeps every
// column inside FP16's range.  The gathered rows go straight into the MMA's
// operand layout, 16-byte cp.async copies into 128-byte swizzled MN-major
// panels (features contiguous, as in X): a 64-feature block of a stage is 32
// rows x 128 bytes, blocks 4 KB apart (the descriptor's leading offset), rows
// 8 at a time in 1024-byte swizzle atoms (the stride offset).  A stage holds
// B's blocks and A's when A's features lie outside B's (otherwise A's
// descriptor points into B's panel).  Seven warps copy (four stages, three in
// flight), warp 1 issues the MMAs (one elected lane, kind::f16, K = 16 rows
// each, FP32 accumulation in tensor memory).  The epilogue undoes the scales
// (C_ab = D_ab 2^-(k_a + k_b)).  The exact column sums h come from a separate
// pass over the FP32 rows.  (A TMA tile::gather4 producer -- one instruction
// per 4 rows x 128 bytes -- measured 1.13x slower here: at about 10 cycles per
// gathered 128-byte row per SM the copy engine set the pace.)
constexpr int kTgK = 32;                                 // gathered rows per stage
constexpr int kTgNS = 4;                                 // stages
constexpr int kTgBN = 256;                               // B features (MMA N, max)
constexpr int kTgAM = 128;                               // A features (MMA M)
constexpr int kTgF = 64;                                 // features of a 128-byte row of a block
constexpr int kTgBlk = kTgK * 128;                       // one 64-feature block of a stage: 4 KB
constexpr int kTgBBytes = (kTgBN / kTgF) * kTgBlk;       // 16 KB
constexpr int kTgABytes = (kTgAM / kTgF) * kTgBlk;       // 8 KB
constexpr int kTgStage = kTgBBytes + kTgABytes;          // 24 KB
constexpr int kTgCols = 256;                             // tensor-memory columns
constexpr size_t kTgSmem = kTgNS * (size_t)kTgStage + 1024;

__host__ __device__ inline int wg_chunks(int ti, int q)   // column chunks of row tile ti
{
    const int last = (128 * ti + 127 < q - 1) ? 128 * ti + 127 : q - 1;
    return last / kTgBN + 1;
}

__host__ __device__ inline int wg_pairs(int q)
{
    int n = 0;
    for (int ti = 0; ti * kTgAM < q; ++ti) n += wg_chunks(ti, q);
    return n;
}

// Shared-memory descriptor of an MN-major operand in the 128-byte swizzled
// layout: 128-byte rows of consecutive features (16-byte chunk c of row k at
// chunk c ^ (k & 7)), 8 rows (K) to a 1024-byte atom, K atoms SBO bytes
// apart, feature blocks (one row each) LBO bytes apart (layout type 2 at bits
// 61-63).
__device__ __forceinline__ unsigned long long umma_desc_mn_sw128(unsigned saddr, unsigned lbo, unsigned sbo)
{
    unsigned long long d = 0;
    d |= (unsigned long long)((saddr >> 4) & 0x3FFFu);
    d |= (unsigned long long)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (unsigned long long)((sbo >> 4) & 0x3FFFu) << 32;
    d |= 1ull << 46;
    d |= 2ull << 61;
    return d;
}

// Instruction descriptor of kind::f16 with FP16 A and B (bits 7-9, 10-12 = 0),
// FP32 D (bits 4-5 = 1), both operands MN-major (bits 15, 16), N >> 3 at bit
// 17, M >> 4 at bit 24.
__host__ __device__ constexpr unsigned umma_idesc_f16_mn(int M, int N)
{
    return (1u << 4) | (1u << 15) | (1u << 16) | ((unsigned)(N >> 3) << 17) | ((unsigned)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma_f16(unsigned dtmem, unsigned long long adesc, unsigned long long bdesc,
                                           unsigned idesc, int accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// the lane-0 result of a bounded wait, in every lane of the warp
__device__ __forceinline__ bool warp_wait(unsigned long long *bar, unsigned parity, int *err, int lane)
{
    int ok = 1;
    if (lane == 0) ok = mbar_wait_bounded(bar, parity, err) ? 1 : 0;
    return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

__global__ void __launch_bounds__(kUmThreads, 2) gram_f16_wide_kernel(const void *__restrict__ x16, int x16_ld, int q,
                                                                   const int *__restrict__ kf,
                                                                   const int32_t *__restrict__ J, long long p,
                                                                   float *__restrict__ cpart, int *err,
                                                                   const int *skip)
{
    if (skip && __ldcg(skip)) return;
    extern __shared__ unsigned char um_dyn[];
    __shared__ __align__(8) unsigned long long full[kTgNS], empty[kTgNS], done;
    __shared__ unsigned tmem_slot;
    __shared__ int abort_flag, mma_count;
    unsigned char *base =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(um_dyn) + 1023) & ~(uintptr_t)1023);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int t = blockIdx.x, ti = 0;
    while (t >= wg_chunks(ti, q)) {
        t -= wg_chunks(ti, q);
        ++ti;
    }
    const int cj = t;
    const int b0 = kTgBN * cj, a0 = kTgAM * ti;
    const int nb = (q - b0 < kTgBN) ? q - b0 : kTgBN;   // a multiple of 16
    const bool inside = (ti >> 1) == cj;                // A's features are B's 128 (ti & 1) .. + 127
    const int nbB = (nb + kTgF - 1) / kTgF;             // 64-feature blocks copied per stage
    const int nbA = inside ? 0 : ((q - a0 < kTgAM ? q - a0 : kTgAM) + kTgF - 1) / kTgF;
    const int KS = gridDim.y, ks = blockIdx.y;
    const long long per = (p + KS - 1) / KS;
    const long long r0 = (long long)ks * per;
    const long long r1 = r0 + per < p ? r0 + per : p;
    const int nst = r1 > r0 ? (int)((r1 - r0 + kTgK - 1) / kTgK) : 0;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(kTgCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 32) {
        for (int s = 0; s < kTgNS; ++s) {
            mbar_init(&full[s], kUmThreads - 32);   // every producer thread
            mbar_init(&empty[s], 1);   // the MMAs' commit
        }
        mbar_init(&done, 1);
        mbar_fence_init();
        abort_flag = 0;
        mma_count = 0;
    }
    // blocks that are never copied (features past q) stay zero
    for (int i = threadIdx.x; i < kTgNS * kTgStage / 16; i += kUmThreads)
        reinterpret_cast<float4 *>(base)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = tmem_slot;
    const unsigned sbase = smem_u32(base);

    if (warp != 1) {
        // ---- producers (every warp but the MMA warp): 16-byte cp.async copies of
        // stage it into the swizzled blocks once the MMAs of its previous use are
        // done; rows past the share's end are written as zeros.  A thread's copies
        // of stage it - kLag are complete once stage it is committed and at most
        // kLag groups remain; it then makes them visible to the tensor core (proxy
        // fence) and arrives on that stage's full barrier.
        constexpr int kLag = kTgNS - 1;
        const int pt = threadIdx.x < 32 ? threadIdx.x : threadIdx.x - 32;   // 0 .. kUmThreads - 33
        constexpr int kProd = kUmThreads - 32;
        static_assert(kProd % 8 == 0 && kProd / 8 == 28, "chunk stepping assumes 28 rows of 8 chunks per round");
        const int nblk = nbB + nbA;
        const int chunks = nblk * kTgK * 8;
        const __half *X16 = reinterpret_cast<const __half *>(x16);
        // chunk e = pt + kProd u: 16-byte chunk c = e & 7 (fixed per thread) of
        // block (e >> 3) % nblk of stage row (e >> 3) / nblk; (block, row)
        // advance by 28 blocks a round, i.e. by (28 / nblk, 28 % nblk)
        const int c = pt & 7;
        const int blk0 = (pt >> 3) % nblk, k0 = (pt >> 3) / nblk;
        const int dk = 28 / nblk, dblk = 28 % nblk;
        const int rounds = (chunks + kProd - 1) / kProd;   // the same in every warp
        // lane k holds the row index of stage row k, one stage ahead
        auto stage_row = [&](int st2) -> int {
            if (st2 >= nst) return 0;
            const long long r = r0 + (long long)st2 * kTgK + lane;
            return __ldg(&J[r < r1 ? r : r1 - 1]);
        };
        int jnext = stage_row(0);
        for (int it = 0; it < nst + kLag; ++it) {
            if (it < nst) {
                const int s = it % kTgNS;
                const int jrow = jnext;
                jnext = stage_row(it + 1);
                if (it >= kTgNS && !warp_wait(&empty[s], (unsigned)((it / kTgNS) - 1) & 1u, err, lane)) {
                    abort_flag = 1;
                    break;
                }
                if (*(volatile int *)&abort_flag) break;
                const long long rb = r0 + (long long)it * kTgK;
                const int valid = (int)(r1 - rb < kTgK ? r1 - rb : kTgK);
                const unsigned st = sbase + (unsigned)s * kTgStage;
                int blk = blk0, k = k0;
                for (int u = 0; u < rounds; ++u) {
                    const int row = __shfl_sync(0xffffffffu, jrow, k & 31);
                    if (pt + kProd * u < chunks) {
                        const bool isb = blk < nbB;
                        const unsigned dst = st +
                                             (isb ? (unsigned)blk * kTgBlk : (unsigned)kTgBBytes + (unsigned)(blk - nbB) * kTgBlk) +
                                             (unsigned)k * 128u + ((unsigned)(c ^ (k & 7)) << 4);
                        if (k < valid) {
                            const int x = (isb ? b0 + kTgF * blk : a0 + kTgF * (blk - nbB)) + 8 * c;
                            const __half *src = X16 + (long long)row * x16_ld + x;
                            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
                        } else {
                            asm volatile("st.shared.v4.u32 [%0], {%1, %1, %1, %1};" ::"r"(dst), "r"(0u) : "memory");
                        }
                    }
                    blk += dblk;
                    k += dk;
                    if (blk >= nblk) {
                        blk -= nblk;
                        ++k;
                    }
                }
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
            if (it >= kLag) {
                asm volatile("cp.async.wait_group %0;" ::"n"(kLag) : "memory");
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive(&full[(it - kLag) % kTgNS]);
            }
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
    } else if (warp == 1) {
        // ---- the MMAs of each stage: two per 32 rows, one for a last stage of <= 16 ----
        const unsigned idesc = umma_idesc_f16_mn(kTgAM, nb);
        int mmas = 0;
        for (int it = 0; it < nst; ++it) {
            const int s = it % kTgNS;
            if (!warp_wait(&full[s], (unsigned)(it / kTgNS) & 1u, err, lane)) {
                abort_flag = 1;
                break;
            }
            const long long rb = r0 + (long long)it * kTgK;
            const int valid = (int)(r1 - rb < kTgK ? r1 - rb : kTgK);
            if (lane == 0) {
                tc_fence_after();
                const unsigned sb = sbase + (unsigned)s * kTgStage;
                const unsigned sa = inside ? sb + (unsigned)(ti & 1) * 2u * kTgBlk : sb + (unsigned)kTgBBytes;
                for (int h = 0; 16 * h < valid; ++h) {
                    const unsigned long long ad = umma_desc_mn_sw128(sa + h * 2048u, kTgBlk, 1024);
                    const unsigned long long bd = umma_desc_mn_sw128(sb + h * 2048u, kTgBlk, 1024);
                    tc_mma_f16(tmem, ad, bd, idesc, (it > 0 || h > 0) ? 1 : 0);
                }
                tc_commit(&empty[s]);
            }
            __syncwarp();
            mmas = it + 1;
        }
        // done completes once every MMA issued has (on the normal path and after a wait gave up)
        if (lane == 0) {
            if (mmas > 0) tc_commit(&done);
            mma_count = mmas;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (mma_count > 0 && !mbar_wait_bounded(&done, 0u, err)) abort_flag = 1;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const int ok = !abort_flag && mma_count == nst;

    // D rows from tensor memory: warp w reads lanes 32 (w & 3) .. + 31 (A's
    // features), columns 128 (w >> 2) .. + 127 of B; the scales undone
    {
        float *C = cpart + (size_t)ks * q * q;
        const int quarter = warp & 3, half = warp >> 2;
        const int a = a0 + 32 * quarter + lane;
        const int ka = a < q ? __ldg(&kf[a]) : 0;
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
                float v[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) v[j] = ldexpf(__uint_as_float(r[j]), -(ka + __ldg(&kf[b0 + c0 + j])));
#pragma unroll
                for (int j = 0; j < 16; j += 4)
                    *reinterpret_cast<float4 *>(&C[(size_t)a * q + b0 + c0 + j]) =
                        make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTgCols) : "memory");
    }
}

// ---- the FP16 copy of X ----
// k_f = 15 - e_f with max_i |x_if| = m 2^e_f, m in [0.5, 1): the scaled
// column's largest magnitude lies in [2^14, 2^15), below FP16's 65504
__global__ void x16_colmax_kernel(const float *__restrict__ X, long long n, int q, unsigned *__restrict__ cmax)
{
    for (int f = threadIdx.x; f < q; f += blockDim.x) {
        unsigned m = 0u;
        for (long long i = blockIdx.x; i < n; i += gridDim.x) m = max(m, __float_as_uint(fabsf(X[i * q + f])));
        atomicMax(&cmax[f], m);
    }
}

__global__ void x16_scale_kernel(int q, const unsigned *__restrict__ cmax, int *__restrict__ kf)
{
    for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < q; f += gridDim.x * blockDim.x) {
        const float m = __uint_as_float(cmax[f]);
        int e = 0;
        if (m > 0.f && isfinite(m)) frexpf(m, &e);
        kf[f] = m > 0.f && isfinite(m) ? 15 - e : 0;
    }
}

// rows of ld >= q entries (a multiple of 64: every 128-byte box of a row
// starts on a 128-byte line), zero past q
__global__ void x16_convert_kernel(const float *__restrict__ X, long long n, int q, int ld,
                                   const int *__restrict__ kf, __half *__restrict__ X16)
{
    const long long total = n * ld;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long i = e / ld;
        const int f = (int)(e - i * ld);
        X16[e] = f < q ? __float2half_rn(ldexpf(X[i * q + f], __ldg(&kf[f]))) : __float2half_rn(0.f);
    }
}

int g_wg_attr = 0;

// Exact column sums of the gathered rows: block b sums its contiguous share
// of J in row order (TwoSum per feature, four features per thread) into
// part[b]; colsum_reduce_kernel then adds the nb partials of each column in
// block order (eight lanes per column, a fixed shuffle order), 32 columns per
// block.
__global__ void __launch_bounds__(256) colsum_kernel(const float *__restrict__ X, int q,
                                                     const int32_t *__restrict__ J, long long p,
                                                     float2 *__restrict__ part)
{
    const int G = gridDim.x, c = threadIdx.x;
    const bool has = 4 * c < q;
    const long long per = (p + G - 1) / G;
    const long long rbeg = (long long)blockIdx.x * per;
    const long long rend = rbeg + per < p ? rbeg + per : p;
    float hs[4] = {0.f, 0.f, 0.f, 0.f}, hc[4] = {0.f, 0.f, 0.f, 0.f};
    for (long long r0 = rbeg; r0 < rend; r0 += 4) {
        float4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const long long r = r0 + u;
            v[u] = (has && r < rend) ? __ldcs(reinterpret_cast<const float4 *>(X + (long long)J[r] * q) + c)
                                     : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float xs[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                float sn, e;
                two_sum(hs[k], xs[k], sn, e);
                hs[k] = sn;
                hc[k] += e;
            }
        }
    }
    if (has) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float hi, lo;
            two_sum(hs[k], hc[k], hi, lo);
            part[(size_t)blockIdx.x * q + 4 * c + k] = make_float2(hi, lo);
        }
    }
}

__global__ void __launch_bounds__(256) colsum_reduce_kernel(int q, int nb, const float2 *__restrict__ part,
                                                            float2 *__restrict__ H)
{
    const int lane = threadIdx.x & 31, sub = lane & 7;
    const int j0 = blockIdx.x * 32 + (threadIdx.x >> 3);
    const int j = j0 < q ? j0 : q - 1;
    float2 t = make_float2(0.f, 0.f);
    for (int b = sub; b < nb; b += 8) t = dfx_add(t, __ldcg(&part[(size_t)b * q + j]));
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) t = dfx_add(t, shfl_xor_f2(t, o));
    if (sub == 0 && j0 < q) H[j] = t;
}

// G = sum_b C_b and h = sum_b h_b in FP64, in block order (the step-level
// entry point); both triangles of G from the lower one of the partials
__global__ void gram_sum_kernel(int q, int nb, const float *__restrict__ cpart, int nbh,
                                const float2 *__restrict__ hpart, double *__restrict__ Gout, double *__restrict__ hout)
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
            for (int b = 0; b < nbh; ++b) {
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
    const long long rows = (p + kTgK - 1) / kTgK;
    if (ks > rows) ks = rows;
    return ks < 1 ? 1 : (int)ks;
}

cudaError_t x16_prepare(Work &W)
{
    if (W.x16) return cudaSuccess;
    const int q = (int)W.q;
    if (!W.xf32 || W.csr || q % 16 != 0 || W.n < 1 || W.n > 0x7fffffffLL) return cudaErrorInvalidValue;
    void *x16 = nullptr;
    int *kf = nullptr;
    const int ld = (q + kTgF - 1) / kTgF * kTgF;
    if (cudaMalloc(&x16, (size_t)W.n * ld * sizeof(__half)) != cudaSuccess) return cudaErrorMemoryAllocation;
    if (cudaMalloc((void **)&kf, 2 * (size_t)q * sizeof(int)) != cudaSuccess) {
        cudaFree(x16);
        return cudaErrorMemoryAllocation;
    }
    W.x16 = x16;
    W.x16_k = kf;
    W.x16_own = true;
    unsigned *cmax = reinterpret_cast<unsigned *>(kf + q);
    cudaError_t e = cudaMemsetAsync(cmax, 0, (size_t)q * sizeof(unsigned), W.st);
    if (e != cudaSuccess) return e;
    x16_colmax_kernel<<<4 * W.nsm, 256, 0, W.st>>>((const float *)W.X, W.n, q, cmax);
    x16_scale_kernel<<<(q + 255) / 256, 256, 0, W.st>>>(q, cmax, kf);
    x16_convert_kernel<<<8 * W.nsm, 256, 0, W.st>>>((const float *)W.X, W.n, q, ld, kf,
                                                    reinterpret_cast<__half *>(x16));
    W.nlaunch += 3;
    return cudaGetLastError();
}

cudaError_t launch_gram_umma_wide(Work &W, const int32_t *J, long long p, int KS, float *cpart, const int *skip)
{
    const int q = (int)W.q;
    if (q <= kUmMaxQ || q > 1024 || q % 16 != 0 || !W.xf32 || KS < 1) return cudaErrorInvalidValue;
    if ((size_t)KS * ((size_t)q * q + 2 * q) > 2 * W.part_len) return cudaErrorInvalidValue;
    cudaError_t e = x16_prepare(W);
    if (e != cudaSuccess) return e;
    if (!g_wg_attr) {
        e = cudaFuncSetAttribute(gram_f16_wide_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTgSmem);
        if (e != cudaSuccess) return e;
        g_wg_attr = 1;
    }
    const int ld = (q + kTgF - 1) / kTgF * kTgF;
    gram_f16_wide_kernel<<<dim3((unsigned)wg_pairs(q), (unsigned)KS), kUmThreads, kTgSmem, W.st>>>(
        W.x16, ld, q, W.x16_k, J, p, cpart, W.err, skip);
    ++W.nlaunch;
    return cudaGetLastError();
}

cudaError_t launch_gram_umma_sum(Work &W, int nb, const float *cpart, int nbh, const float2 *hpart, double *G,
                                 double *h)
{
    gram_sum_kernel<<<W.nsm, 256, 0, W.st>>>((int)W.q, nb, cpart, nbh, hpart, G, h);
    ++W.nlaunch;
    return cudaGetLastError();
}

int colsum_blocks(const Work &W, long long p, int max_blocks)
{
    long long nb = (p + 63) / 64;   // about 64 rows per block
    if (nb > 4 * W.nsm) nb = 4 * W.nsm;
    if (nb > max_blocks) nb = max_blocks;
    return nb < 1 ? 1 : (int)nb;
}

cudaError_t launch_colsum(Work &W, const int32_t *J, long long p, int nb, float2 *part, float2 *H)
{
    if (W.csr || !W.xf32 || W.q > 1024 || W.q % 4 != 0 || nb < 1) return cudaErrorInvalidValue;
    colsum_kernel<<<nb, 256, 0, W.st>>>((const float *)W.X, (int)W.q, J, p, part);
    colsum_reduce_kernel<<<(unsigned)((W.q + 31) / 32), 256, 0, W.st>>>((int)W.q, nb, part, H);
    W.nlaunch += 2;
    return cudaGetLastError();
}

}  // namespace svm
