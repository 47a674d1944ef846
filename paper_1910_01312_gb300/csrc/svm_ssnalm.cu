// svm_ssnalm.cu -- C ABI (include/svm_ssnalm.h) and the host-side control of
// the SSsNAL method: Algorithm 1 (augmented Lagrangian on the restricted dual,
// multiplier update of eq. (3.5)) around Algorithm 3 (semismooth Newton with
// Armijo line search), stopped by the relative KKT residual of eq. (4.1).
//
// Variables (paper -> here): x -> alpha (SVM dual, n); w in Ran(Q) -> v = A'w
// (q), so Q w = A v =: z (n), <w, Qw> = |v|^2 and grad psi = A g with
// g = v - A'Pi(u) (q).  Every vector step runs in the kernels of k_*.cu; the
// host only sequences launches and reads back the scalars that decide the
// next launch (|g|, free-set size, Armijo test, R_KKT).
//
// Readings where the paper leaves a choice open (identical in the FP64 CPU
// oracle used by the tests):
//  - sigma_0 = 1; sigma *= 5 (cap 1e6) when R_KKT fell by less than 1/2.
//  - Inner stop (A')/(B') measured in q-space: |g| <= min(eps_k, eps_k |pi -
//    alpha^k|)/sqrt(sigma_k), eps_k = 0.1 * 0.5^k, floored at 1e-15 times the
//    absolute-sum scale of A'pi (the roundoff level of g); at most 50
//    Newton steps; a failed line search ends the subproblem.
//  - Armijo: mu = 1e-4, delta = 0.5, at most 40 trials; psi differences are
//    summed term by term (the oracle's terms pi (2u - pi); here each less
//    2 lambda y pi, which sums to zero at the root but makes the terms
//    stationary in lambda and of size pi^2: see k_projdf.cu).
//  - z = A v is recomputed at the start of every subproblem.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <chrono>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "../../include/svm_mlp.h"
#include "../../include/svm_ssnalm.h"
#include "internal.cuh"

using namespace svm;

struct svm_ssnalm {
    Work W;
    svm_params P;
    svm_problem prob;
    std::string err;
    double lam_main = 0.0;
    long long npos = 0;   // number of +1 labels (checked at create)
    // instrumentation
    bool timing = false;
    std::vector<cudaEvent_t> evpool;
    size_t evused = 0;
    struct Rec { int kind, e0, e1; };
    std::vector<Rec> recs;
    long long kcalls[5] = {0, 0, 0, 0, 0};
    double kms[5] = {0, 0, 0, 0, 0};
    long long syncs = 0;
    long long launch_base = 0;
    bool trace = false;   // SVM_SSNALM_TRACE=1: one stderr line per Newton step
    // batched solves (svm_ssnalm_solve_batch): one sub-handle per problem,
    // sharing this handle's X and stream; the forward-product plan of the
    // autotuner; per-problem label counts; staging for host memory
    std::vector<svm_ssnalm *> subs;
    bool mv_tuned = false;
    float mv_ms[4] = {0.f, 0.f, 0.f, 0.f};   // ms per pass over X with 1, 2, 4, 8 vectors
    std::vector<int> mv_plan;                  // mv_plan[c]: vectors in the first pass for c products
    int *bat_cnt = nullptr;
    int8_t *bat_y = nullptr;
    double *bat_a = nullptr, *bat_w = nullptr;
    int bat_cap = 0;
    long long batch_ticks = 0;
    NewtonTask *nt_host = nullptr, *nt_dev = nullptr;   // batched Newton steps (pinned / device table)
    int nt_cap = 0;
    // batched wide Newton steps (128 < q <= 1024): the prepared set-up and CG
    // arguments of each problem (pinned / device tables)
    MfwSetupArgs *wt_s_host = nullptr, *wt_s_dev = nullptr;
    MfwArgs *wt_c_host = nullptr, *wt_c_dev = nullptr;
    int wt_cap = 0;
    svm_mlp_t *wsm = nullptr;   // warm-start network of svm_ssnalm_set_warmstart_model (owned)
    // batched projections: a sub-handle of a batched solve records its
    // double-float projection instead of launching it (proj_defer), and the
    // batch launches all recorded ones at once (one cluster per problem)
    bool proj_defer = false, proj_pending = false;
    ProjDF pend_in;
    ProjOut *pend_out = nullptr;
    PDArgs *pd_host = nullptr, *pd_dev = nullptr;   // parent: the phase's table (pinned / device)
    int pd_cap = 0;
};

enum { TK_MATVEC = 0, TK_RMATVEC = 1, TK_PROJ = 2, TK_NEWTON = 3, TK_MATVEC2 = 4 };

static int ev_take(svm_ssnalm *h)
{
    if (h->evused == h->evpool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return -1;
        h->evpool.push_back(e);
    }
    return (int)h->evused++;
}

// Run f() (which launches on the handle's stream); count it under `kind` and,
// when timing is on, bracket it with two events.
template <class F>
static cudaError_t timed(svm_ssnalm *h, int kind, F f)
{
    h->kcalls[kind]++;
    int e0 = h->timing ? ev_take(h) : -1;
    if (e0 >= 0) cudaEventRecord(h->evpool[e0], h->W.st);
    cudaError_t e = f();
    if (e0 >= 0) {
        int e1 = ev_take(h);
        if (e1 >= 0) {
            cudaEventRecord(h->evpool[e1], h->W.st);
            h->recs.push_back({kind, e0, e1});
        }
    }
    return e;
}

// Fold recorded event pairs into the totals (the stream must be idle).
static void flush_timing(svm_ssnalm *h)
{
    for (const auto &r : h->recs) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, h->evpool[r.e0], h->evpool[r.e1]) == cudaSuccess) h->kms[r.kind] += ms;
    }
    h->recs.clear();
    h->evused = 0;
}

static thread_local std::string g_create_err;

#define CK(call)                                                                                           \
    do {                                                                                                   \
        cudaError_t e_ = (call);                                                                           \
        if (e_ != cudaSuccess) {                                                                           \
            h->err = std::string(#call) + ": " + cudaGetErrorString(e_);                                   \
            return SVM_ERR_CUDA;                                                                           \
        }                                                                                                  \
    } while (0)

extern "C" void svm_default_params(svm_params *p)
{
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->C = 1.0;
    p->tol = 1e-6;
    p->max_outer = 200;
    p->max_inner = 50;
    p->max_ls = 40;
    p->precision = SVM_PREC_MIXED;
    p->sigma0 = 1.0;
    p->sigma_growth = 5.0;
    p->sigma_max = 1e6;
    p->mu = 1e-4;
    p->delta = 0.5;
    p->tau = 0.5;
    p->eta = 0.1;
    p->newton_mode = 0;
    p->deterministic = 1;
    p->stream = nullptr;
}

extern "C" const char *svm_ssnalm_last_error(const svm_ssnalm_t *h)
{
    if (!h) return g_create_err.c_str();
    return h->err.c_str();
}

static void free_work(Work &W)
{
    void *ptrs[] = {W.alpha, W.z, W.dz, W.qa, W.tmpn, W.zf, W.dzf, W.qaf, W.alphaw, W.dw, W.dwa, W.atpa,
                    W.atpa2, W.mf_st, W.mf_pinv, W.mf_counter, W.mfw_mask, W.mfw_st, W.v, W.vt, W.dv, W.g, W.atp, W.atp2, W.h, W.w, W.tmpq, W.M, W.Lf, W.Mf, W.part, W.cnt,
                    W.bar, W.rm_counter, W.err, W.pout, W.red, W.X_own, W.y_own, W.csc_ptr, W.csc_row,
                    W.csc_val, W.task_beg, W.col_task, W.task_part, W.csr_tn, W.csr_q, W.csr_cg,
                    W.csr_ptr_own, W.csr_idx_own, W.csr_val_own, W.jcsc_ptr, W.jtot, W.jcol_task, W.jtask_beg,
                    W.jcsc_row, W.jcsc_val, W.jcnt, W.jtask_part, W.csr_vf, W.csr_df, W.csr_cf, W.csr_tnf};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (W.x16_own) {
        cudaFree(W.x16);
        cudaFree(W.x16_k);
    }
    for (int b = 0; b < 2; ++b) {
        void *pp[] = {W.pb[b].u, W.pb[b].uf, W.pb[b].pi, W.pb[b].wpi, W.pb[b].J, W.pb[b].S};
        for (void *p : pp)
            if (p) cudaFree(p);
    }
    if (W.h_pout) cudaFreeHost(W.h_pout);
    if (W.h_red) cudaFreeHost(W.h_red);
    if (W.h_err) cudaFreeHost(W.h_err);
    if (W.h_csr_done) cudaFreeHost(W.h_csr_done);
    W = Work();
}

extern "C" void svm_ssnalm_destroy(svm_ssnalm_t *h)
{
    if (!h) return;
    if (h->W.st) cudaStreamSynchronize(h->W.st);
    for (cudaEvent_t e : h->evpool) cudaEventDestroy(e);
    for (svm_ssnalm *sb : h->subs) svm_ssnalm_destroy(sb);
    void *bp[] = {h->bat_cnt, h->bat_y, h->bat_a, h->bat_w, h->nt_dev, h->wt_s_dev, h->wt_c_dev};
    for (void *p : bp)
        if (p) cudaFree(p);
    if (h->nt_host) cudaFreeHost(h->nt_host);
    if (h->wt_s_host) cudaFreeHost(h->wt_s_host);
    if (h->wt_c_host) cudaFreeHost(h->wt_c_host);
    if (h->pd_dev) cudaFree(h->pd_dev);
    if (h->pd_host) cudaFreeHost(h->pd_host);
    svm_mlp_destroy(h->wsm);
    free_work(h->W);
    delete h;
}

__global__ void check_labels_kernel(const int8_t *y, long long n, int *out)
{
    // out[0]: count of invalid labels, out[1]: count of +1
    int bad = 0, pos = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        int8_t v = y[i];
        bad += (v != 1 && v != -1);
        pos += (v == 1);
    }
    for (int o = 16; o > 0; o >>= 1) {
        bad += __shfl_xor_sync(0xffffffffu, bad, o);
        pos += __shfl_xor_sync(0xffffffffu, pos, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (bad) atomicAdd(out, bad);
        if (pos) atomicAdd(out + 1, pos);
    }
}

__global__ void check_finite_kernel(const void *X, int f32, long long m, int *out)
{
    int bad = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x) {
        double v = f32 ? (double)((const float *)X)[i] : ((const double *)X)[i];
        bad += !isfinite(v);
    }
    for (int o = 16; o > 0; o >>= 1) bad += __shfl_xor_sync(0xffffffffu, bad, o);
    if ((threadIdx.x & 31) == 0 && bad) atomicAdd(out, bad);
}

template <typename T>
static cudaError_t dalloc(T **p, size_t count)
{
    return cudaMalloc((void **)p, (count ? count : 1) * sizeof(T));
}

// validate = false: the labels and X were checked by the caller (the
// sub-handles of a batched solve, which share the parent's X)
static svm_status create_impl(svm_ssnalm_t **out, const svm_problem *prob, const svm_params *params, bool validate)
{
    if (out) *out = nullptr;
    if (!out || !prob || !params) { g_create_err = "null argument"; return SVM_ERR_INVALID_ARG; }
    if (prob->n < 1 || prob->q < 1) { g_create_err = "n and q must be >= 1"; return SVM_ERR_INVALID_ARG; }
    if (prob->n > 0x7fffffffLL) { g_create_err = "n must fit in int32"; return SVM_ERR_UNSUPPORTED; }
    if (!(params->C > 0.0) || !isfinite(params->C)) { g_create_err = "C must be finite and > 0"; return SVM_ERR_INVALID_ARG; }
    if (!(params->tol > 0.0)) { g_create_err = "tol must be > 0"; return SVM_ERR_INVALID_ARG; }
    const bool csr = prob->layout == SVM_CSR;
    if (prob->layout != SVM_DENSE_ROWMAJOR && !csr) { g_create_err = "layout must be dense row-major or CSR"; return SVM_ERR_INVALID_ARG; }
    if (!prob->y || (!csr && !prob->X) || (csr && (!prob->indptr || (prob->nnz > 0 && (!prob->indices || !prob->values)))))
    { g_create_err = "X (or the CSR arrays) and y must be non-null"; return SVM_ERR_INVALID_ARG; }
    if (csr && (prob->nnz < 0 || prob->q > 0x7fffffffLL)) { g_create_err = "CSR: nnz >= 0 and q < 2^31 required"; return SVM_ERR_INVALID_ARG; }
    if (prob->dtype != SVM_F32 && prob->dtype != SVM_F64) { g_create_err = "dtype must be F32 or F64"; return SVM_ERR_INVALID_ARG; }
    if (prob->memory != SVM_MEM_DEVICE && prob->memory != SVM_MEM_HOST) { g_create_err = "bad memory kind"; return SVM_ERR_INVALID_ARG; }
    if (!csr && prob->q > 1024) { g_create_err = "dense q > 1024 not supported in this build"; return SVM_ERR_UNSUPPORTED; }
    if (params->max_outer < 1 || params->max_inner < 1 || params->max_ls < 1) { g_create_err = "iteration caps must be >= 1"; return SVM_ERR_INVALID_ARG; }
    if (params->precision != SVM_PREC_PLAIN_FP64 && params->precision != SVM_PREC_MIXED) { g_create_err = "bad precision"; return SVM_ERR_INVALID_ARG; }

    svm_ssnalm *h = new (std::nothrow) svm_ssnalm();
    if (!h) { g_create_err = "out of host memory"; return SVM_ERR_OOM; }
    h->P = *params;
    h->prob = *prob;
    Work &W = h->W;
    W.n = prob->n;
    W.q = prob->q;
    W.xf32 = prob->dtype == SVM_F32;
    W.C = params->C;
    W.precision = params->precision;
    W.eta = params->eta > 0.0 ? params->eta : 0.1;
    W.tau = params->tau > 0.0 ? params->tau : 0.5;
    W.st = (cudaStream_t)params->stream;
    auto fail = [&](svm_status st, const std::string &m) {
        g_create_err = m;
        free_work(h->W);
        delete h;
        return st;
    };
    cudaError_t e = cudaGetDevice(&W.dev);
    if (e != cudaSuccess) return fail(SVM_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    cudaDeviceGetAttribute(&W.nsm, cudaDevAttrMultiProcessorCount, W.dev);
    const size_t n = (size_t)W.n, q = (size_t)W.q;
    const size_t xbytes = n * q * (W.xf32 ? 4 : 8);
    W.csr = csr;
    if (csr) {
        W.nnz = prob->nnz;
        const size_t nz = (size_t)prob->nnz, es = W.xf32 ? 4 : 8;
        if (prob->memory == SVM_MEM_HOST) {
            if (cudaMalloc(&W.csr_ptr_own, (n + 1) * sizeof(int64_t)) != cudaSuccess ||
                cudaMalloc(&W.csr_idx_own, (nz ? nz : 1) * sizeof(int32_t)) != cudaSuccess ||
                cudaMalloc(&W.csr_val_own, (nz ? nz : 1) * es) != cudaSuccess || dalloc(&W.y_own, n) != cudaSuccess)
                return fail(SVM_ERR_OOM, "device allocation of the CSR/y copy failed");
            if (cudaMemcpyAsync(W.csr_ptr_own, prob->indptr, (n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, W.st) ||
                (nz && cudaMemcpyAsync(W.csr_idx_own, prob->indices, nz * sizeof(int32_t), cudaMemcpyHostToDevice, W.st)) ||
                (nz && cudaMemcpyAsync(W.csr_val_own, prob->values, nz * es, cudaMemcpyHostToDevice, W.st)) ||
                cudaMemcpyAsync(W.y_own, prob->y, n, cudaMemcpyHostToDevice, W.st))
                return fail(SVM_ERR_CUDA, "host-to-device copy of the CSR arrays/y failed");
            W.csr_ptr = W.csr_ptr_own;
            W.csr_idx = W.csr_idx_own;
            W.csr_val = W.csr_val_own;
            W.y = W.y_own;
        } else {
            W.csr_ptr = prob->indptr;
            W.csr_idx = prob->indices;
            W.csr_val = prob->values;
            W.y = prob->y;
        }
    } else if (prob->memory == SVM_MEM_HOST) {
        if (cudaMalloc(&W.X_own, xbytes) != cudaSuccess || dalloc(&W.y_own, n) != cudaSuccess)
            return fail(SVM_ERR_OOM, "device allocation of X/y copy failed");
        if (cudaMemcpyAsync(W.X_own, prob->X, xbytes, cudaMemcpyHostToDevice, W.st) != cudaSuccess ||
            cudaMemcpyAsync(W.y_own, prob->y, n, cudaMemcpyHostToDevice, W.st) != cudaSuccess)
            return fail(SVM_ERR_CUDA, "host-to-device copy of X/y failed");
        W.X = W.X_own;
        W.y = W.y_own;
    } else {
        W.X = prob->X;
        W.y = prob->y;
    }
    if (!csr && (uintptr_t)W.X % 16 != 0) return fail(SVM_ERR_INVALID_ARG, "X must be 16-byte aligned");
    // double-float n-vectors wherever the mixed-form matvec applies (dense FP32 X,
    // q % 4 == 0); CSR runs the FP64 form
    W.df = !csr && W.precision == SVM_PREC_MIXED && W.xf32 && q % 4 == 0;
    // workspace
    W.rm_grid = W.nsm * 4;
    // Gram split-K partials: at most 32 MiB (at least one q x q partial)
    size_t part_gram = (size_t)(4 * W.nsm) * (q * q + q);
    const size_t gram_cap = ((size_t)32 << 20) / sizeof(double);
    if (part_gram > gram_cap) part_gram = gram_cap > (q * q + q) ? gram_cap : (q * q + q);
    if (!csr && W.precision == SVM_PREC_MIXED && q > 128 && q <= 1024 && q % 16 == 0) {
        // the wide Gram's row splits: enough (128 x 256)-tile blocks for two per SM
        const size_t np = (size_t)gram_wide_pairs((int)q);
        const size_t ks = (2 * (size_t)W.nsm + np - 1) / np;
        const size_t need = (ks * (q * q + 2 * q) + 1) / 2;   // FP32 partials, counted in doubles
        if (part_gram < need) part_gram = need;
    }
    size_t part_rm = (size_t)2 * W.rm_grid * q;
    if (csr) part_gram = part_rm = 0;   // no dense Gram, no row-block partials
    const size_t qq = csr ? 1 : q * q;   // the dense q x q Newton matrices
    const size_t part_proj = (size_t)3 * 8 * 4 * W.nsm * 4;
    W.part_len = part_gram > part_rm ? part_gram : part_rm;
    if (W.part_len < part_proj) W.part_len = part_proj;
    bool bad = dalloc(&W.alpha, n) || dalloc(&W.qa, n) || dalloc(&W.tmpn, n) ||
               (W.df ? (dalloc(&W.zf, n) || dalloc(&W.dzf, n) || dalloc(&W.qaf, n) || dalloc(&W.alphaw, n) ||
                        dalloc(&W.dw, n) || dalloc(&W.dwa, n))
                     : (dalloc(&W.z, n) || dalloc(&W.dz, n))) ||
               dalloc(&W.atpa, q) || dalloc(&W.atpa2, q) || dalloc(&W.vt, q) ||
               dalloc(&W.v, q) || dalloc(&W.dv, q) || dalloc(&W.g, q) ||
               dalloc(&W.atp, q) || dalloc(&W.atp2, q) || dalloc(&W.h, q) || dalloc(&W.w, q) || dalloc(&W.tmpq, q) ||
               dalloc(&W.M, qq) || dalloc(&W.Lf, csr ? 1 : q * (q + 1)) || dalloc(&W.Mf, qq) || dalloc(&W.part, W.part_len) || dalloc(&W.bar, 4) || dalloc(&W.rm_counter, 4) || dalloc(&W.err, 4) ||
               dalloc(&W.pout, 4) || dalloc(&W.red, 16);
    for (int b = 0; b < 2 && !bad; ++b)
        bad = (W.df ? dalloc(&W.pb[b].uf, n) : dalloc(&W.pb[b].u, n)) || dalloc(&W.pb[b].pi, n) ||
              dalloc(&W.pb[b].wpi, n) ||
              dalloc(&W.pb[b].J, n) || dalloc(&W.pb[b].S, n);
    if (!bad && W.df && q <= 128) bad = newton_mf_alloc(W) != cudaSuccess;
    if (!bad && W.df && q > 128 && q <= 1024 && q % 16 == 0) bad = newton_mfw_alloc(W) != cudaSuccess;
    if (bad) return fail(SVM_ERR_OOM, "device workspace allocation failed");
    if (cudaMallocHost(&W.h_pout, 4 * sizeof(ProjOut)) != cudaSuccess ||
        cudaMallocHost(&W.h_red, 16 * sizeof(double)) != cudaSuccess ||
        cudaMallocHost(&W.h_err, 4 * sizeof(int)) != cudaSuccess)
        return fail(SVM_ERR_OOM, "pinned host allocation failed");
    e = proj_setup(W);
    if (e != cudaSuccess) return fail(SVM_ERR_UNSUPPORTED, "n too large for the projection kernel");
    if (W.df && (e = projdf_cluster_setup(W)) != cudaSuccess)
        return fail(SVM_ERR_CUDA, std::string("projection set-up: ") + cudaGetErrorString(e));
    W.cnt_len = (size_t)W.proj_ept * W.proj_grid * 2;
    if (dalloc(&W.cnt, W.cnt_len)) return fail(SVM_ERR_OOM, "device workspace allocation failed");
    cudaMemsetAsync(W.bar, 0, 4 * sizeof(unsigned), W.st);
    cudaMemsetAsync(W.rm_counter, 0, 4 * sizeof(unsigned), W.st);
    cudaMemsetAsync(W.err, 0, 4 * sizeof(int), W.st);
    cudaMemsetAsync(W.pout, 0, 4 * sizeof(ProjOut), W.st);
    if (!validate) {
        *out = h;
        return SVM_OK;
    }
    // validate labels and data on the device
    int *chk = nullptr;
    if (dalloc(&chk, 4)) return fail(SVM_ERR_OOM, "device allocation failed");
    cudaMemsetAsync(chk, 0, 4 * sizeof(int), W.st);
    check_labels_kernel<<<W.nsm * 2, 256, 0, W.st>>>(W.y, W.n, chk);
    int64_t ends[2] = {0, 0};
    if (csr) {
        // pointer ends, row structure and values (chk[2]: structure, chk[3]: non-finite)
        cudaMemcpyAsync(&ends[0], W.csr_ptr, sizeof(int64_t), cudaMemcpyDeviceToHost, W.st);
        cudaMemcpyAsync(&ends[1], W.csr_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, W.st);
        e = cudaStreamSynchronize(W.st);
        if (e == cudaSuccess && (ends[0] != 0 || ends[1] != W.nnz)) {
            cudaFree(chk);
            return fail(SVM_ERR_INVALID_ARG, "CSR: indptr[0] must be 0 and indptr[n] = nnz");
        }
        if (e == cudaSuccess) e = csr_validate(W, chk + 2);
    } else {
        check_finite_kernel<<<W.nsm * 4, 256, 0, W.st>>>(W.X, W.xf32, (long long)(n * q), chk + 2);
    }
    int hchk[4] = {0, 0, 0, 0};
    cudaMemcpyAsync(hchk, chk, sizeof(hchk), cudaMemcpyDeviceToHost, W.st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(W.st);
    cudaFree(chk);
    if (e != cudaSuccess) return fail(SVM_ERR_CUDA, std::string("create: ") + cudaGetErrorString(e));
    if (hchk[0]) return fail(SVM_ERR_INVALID_ARG, "labels must be +1 or -1");
    if (csr && hchk[2]) return fail(SVM_ERR_INVALID_ARG, "CSR: row pointers or column indices out of range, or columns not strictly increasing within a row");
    if (csr ? hchk[3] : hchk[2]) return fail(SVM_ERR_INVALID_ARG, "X has non-finite entries");
    h->npos = hchk[1];
    if (csr) {
        e = csr_setup(W);
        if (e != cudaSuccess) return fail(SVM_ERR_OOM, std::string("CSR setup: ") + cudaGetErrorString(e));
    }
    {
        const char *tr = getenv("SVM_SSNALM_TRACE");
        h->trace = tr && tr[0] == '1';
    }
    *out = h;
    return SVM_OK;
}

extern "C" svm_status svm_ssnalm_create(svm_ssnalm_t **out, const svm_problem *prob, const svm_params *params)
{
    return create_impl(out, prob, params, true);
}

// ------------------------------------------------------------ helpers

// Scalar read-back of a phase: the projection records, the small reductions
// and the device error flag, copied to pinned host memory (stream-ordered).
static svm_status readback_issue(svm_ssnalm *h)
{
    Work &W = h->W;
    CK(cudaMemcpyAsync(W.h_pout, W.pout, 4 * sizeof(ProjOut), cudaMemcpyDeviceToHost, W.st));
    CK(cudaMemcpyAsync(W.h_red, W.red, 16 * sizeof(double), cudaMemcpyDeviceToHost, W.st));
    CK(cudaMemcpyAsync(W.h_err, W.err, sizeof(int), cudaMemcpyDeviceToHost, W.st));
    return SVM_OK;
}

// The double-float projection of a phase: launched now, or -- in a batched
// solve whose problems fit the cluster form -- recorded, to be launched with
// the other problems' projections of the phase (h->proj_pending).
static svm_status proj_df(svm_ssnalm *h, const ProjDF &in, ProjOut *out)
{
    if (h->proj_defer) {
        h->pend_in = in;
        h->pend_out = out;
        h->proj_pending = true;
        h->kcalls[TK_PROJ]++;
        return SVM_OK;
    }
    CK(timed(h, TK_PROJ, [&] { return launch_project_df(h->W, in, out); }));
    return SVM_OK;
}

// After the stream has been synchronised: complete the double-float records
// and turn a device error flag into a status (the flag is cleared for the
// next call).
static svm_status readback_check(svm_ssnalm *h)
{
    Work &W = h->W;
    for (int k = 0; k < 4; ++k) {
        ProjOut &o = W.h_pout[k];
        if (!o.is_df) continue;
        o.lam = (double)o.lamf.x + (double)o.lamf.y;
        for (int j = 0; j < 4; ++j) o.sum[j] = (double)o.sumf[j].x + (double)o.sumf[j].y;
    }
    const int e = W.h_err[0];
    if (e) {
        cudaMemsetAsync(W.err, 0, sizeof(int), W.st);
        cudaMemsetAsync(W.bar, 0, sizeof(unsigned), W.st);
        if (e == DEV_TIMEOUT) { h->err = "device-side wait timed out"; return SVM_ERR_TIMEOUT; }
        if (e == DEV_ROOT) { h->err = "projection root search hit its pass cap"; return SVM_ERR_NUMERIC; }
        if (e == DEV_CHOL) { h->err = "Newton matrix not positive definite"; return SVM_ERR_NUMERIC; }
        h->err = "device numeric error";
        return SVM_ERR_NUMERIC;
    }
    return SVM_OK;
}

static svm_status sync_read(svm_ssnalm *h)
{
    svm_status st = readback_issue(h);
    if (st != SVM_OK) return st;
    CK(cudaStreamSynchronize(h->W.st));
    h->syncs++;
    if (h->timing) flush_timing(h);
    return readback_check(h);
}

// ProjOut slots: 0 step-level op, 1 + b for projection buffer b, 3 KKT.
enum { SLOT_OP = 0, SLOT_KKT = 3 };

// The KKT projection of eq. (4.1) at alpha given Q alpha in W.qa (FP64).
static svm_status kkt_project(svm_ssnalm *h, const double *alpha)
{
    Work &W = h->W;
    ProjIn in;
    in.a = alpha; in.b = W.qa; in.c1 = -1.0; in.c2 = 1.0;
    in.sums = SF_KKT; in.alpha = alpha;
    in.lam0 = &W.pout[SLOT_KKT].lam;
    CK(timed(h, TK_PROJ, [&] { return launch_project(W, in, &W.pout[SLOT_KKT]); }));
    return SVM_OK;
}

// The same in double-float form: alpha given as y o alpha, Q alpha in W.qaf.
static svm_status kkt_project_df(svm_ssnalm *h, const float2 *alpha_w)
{
    Work &W = h->W;
    ProjDF in;
    in.a = alpha_w; in.a_signed = true; in.b = W.qaf; in.c1 = -1.0; in.c2 = 1.0;
    in.sums = SF_KKT;
    in.lam0 = &W.pout[SLOT_KKT].lamf;
    return proj_df(h, in, &W.pout[SLOT_KKT]);
}

static double kkt_value(const ProjOut &o)
{
    return sqrt(o.sum[0]) / (1.0 + sqrt(o.sum[1]));
}

// red[0] += #{0 < a < C}, red[1] += #{a >= C}, red[2] += #{a > 0}
__global__ void count_kernel(long long n, const double *a, double C, double *red)
{
    unsigned long long f = 0, u = 0, s = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double v = a[i];
        f += (v > 0.0 && v < C);
        u += (v >= C);
        s += (v > 0.0);
    }
    for (int o = 16; o > 0; o >>= 1) {
        f += __shfl_xor_sync(0xffffffffu, f, o);
        u += __shfl_xor_sync(0xffffffffu, u, o);
        s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(red + 0, (double)f);
        atomicAdd(red + 1, (double)u);
        atomicAdd(red + 2, (double)s);
    }
}

// g = (v + t dv) - atp, red[0] = |g|^2 (the gradient at the trial point)
__global__ void grad_at_kernel(int q, const double *v, const double *dv, double t, const double *atp, double *g,
                               double *red)
{
    __shared__ double sh[32];
    double s = 0.0;
    for (int j = threadIdx.x; j < q; j += blockDim.x) {
        const double gj = fma(t, dv[j], v[j]) - atp[j];
        g[j] = gj;
        s = fma(gj, gj, s);
    }
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += sh[w];
        red[0] = r;
    }
}

__global__ void copyq_kernel(int q, const double *a, double *b)
{
    for (int j = threadIdx.x; j < q; j += blockDim.x) b[j] = a[j];
}

// ------------------------------------------------------------ solve

// One solve as a sequence of phases.  A phase issues kernels on the handle's
// stream, possibly with forward products A v in the middle (run_pre issues
// what comes before them and lists them in mv, run_post what comes after),
// and ends with the read-back of the scalars that decide the next phase
// (run_after, once the stream has been synchronised).  svm_ssnalm_solve runs
// one Run and synchronises after every phase; svm_ssnalm_solve_batch runs
// many in lockstep, with one pass over X for the forward products of all of
// them and one synchronisation per phase for all of them.
enum RunPhase { RP_INIT, RP_SUBSTART, RP_NEWTON, RP_TRIAL, RP_OUTER_END, RP_FINISH, RP_DONE };

struct MvReq {
    int nv = 0;
    const double *v[2] = {nullptr, nullptr};
    float2 *zf[2] = {nullptr, nullptr};   // double-float outputs (mixed form)
    double *z[2] = {nullptr, nullptr};    // FP64 outputs (other forms)
};

struct Run {
    svm_ssnalm *h = nullptr;
    const double *alpha0 = nullptr;
    svm_result *res = nullptr;
    RunPhase ph = RP_INIT;
    int cur = 0;          // projection buffer holding pi(u(v)) at the current point
    int k = 0, j = 0, mtr = 0, inner_total = 0;
    double sigma = 1.0, R = 0.0, Rprev = 0.0, t = 1.0, epsk = 0.1;
    svm_status status = SVM_ERR_NOT_CONVERGED;   // convergence status
    svm_status ret = SVM_OK;                     // return value once done
    MvReq mv;
    std::vector<double> hw;                      // w on the host (results)
    bool defer_newton = false;   // batched: leave a small-free-set Newton step to the batch launch
    bool has_task = false;       // ... and this phase's step was left there
    NewtonTask task;
    bool has_wtask = false;      // a wide step was prepared and left to the batch launch
    double t_in = 0.0;           // the level at which the current subproblem stops (|g| <= t_in)
    int cont = 0;                // batched: what follows a recorded projection (a RunCont)
};

// The kernels of a phase that follow its projection, when the projection was
// recorded for a batched launch (run_post_cont issues them after it).
enum RunCont { RC_NONE = 0, RC_READBACK = 1, RC_SUBSTART = 2, RC_TRIAL = 3 };

// The CG of a Newton step stops once its residual is below kCgFloor times the
// level at which the subproblem stops (and within Algorithm 3's bound): the
// step's new gradient is then about that residual, so the subproblem's last
// step still ends it, while earlier steps, whose gradients are far above the
// level, are not solved to 1e-10 of |g|.  (0.01 measured 2-3 % slower on the
// one-vs-rest batch and on gauss1m, with the same Newton step counts there.)
constexpr double kCgFloor = 0.1;

static void mv_add(Work &W, MvReq &m, const double *v, float2 *zf, double *z)
{
    (void)W;
    m.v[m.nv] = v;
    m.zf[m.nv] = zf;
    m.z[m.nv] = z;
    ++m.nv;
}

// The requested products of one run, one launch (both vectors in one pass).
static svm_status run_matvec_single(Run &r)
{
    svm_ssnalm *h = r.h;
    Work &W = h->W;
    const MvReq &m = r.mv;
    if (!m.nv) return SVM_OK;
    // one-vector and two-vector passes are timed apart (the second does twice the arithmetic per byte)
    CK(timed(h, m.nv > 1 ? TK_MATVEC2 : TK_MATVEC, [&] {
        return W.df ? launch_matvec_df(W, m.v[0], m.zf[0], m.nv > 1 ? m.v[1] : nullptr, m.nv > 1 ? m.zf[1] : nullptr)
                    : launch_matvec(W, m.v[0], m.z[0], m.nv > 1 ? m.v[1] : nullptr, m.nv > 1 ? m.z[1] : nullptr);
    }));
    return SVM_OK;
}

// A line-search trial at step t: project u - t sigma A dv into the other
// buffer and, speculatively, form A'pi and the gradient there, so an accepted
// trial is the next iterate's projection and gradient at no extra pass.
// A'pi at the trial point (over the delta list) and, in the epilogue,
// vt = v + t dv and g = vt - A'pi with |g|^2 (kept if the trial is accepted)
static svm_status trial_after_proj(Run &r)
{
    svm_ssnalm *h = r.h;
    Work &W = h->W;
    const int nxt = 1 - r.cur;
    ProjBuf &B = W.pb[nxt];
    GradOut go;
    go.v = W.v; go.dv = W.dv; go.t = r.t; go.g = W.tmpq; go.vt = W.vt;
    CK(timed(h, TK_RMATVEC, [&] {
        return launch_rmatvec_df(W, W.dw, W.dwa, B.S, &W.pout[1 + nxt].s, W.atp, W.atpa, W.atp2, W.atpa2, 1, go);
    }));
    return readback_issue(h);
}

static svm_status issue_trial(Run &r)
{
    svm_ssnalm *h = r.h;
    Work &W = h->W;
    const int cur = r.cur, nxt = 1 - cur;
    const double t = r.t, sigma = r.sigma;
    ProjBuf &B = W.pb[nxt];
    if (W.df) {
        ProjDF tr;
        tr.a = W.pb[cur].uf; tr.b = W.dzf; tr.c1 = -t * sigma; tr.c2 = 0.0;
        tr.sums = SF_PSID | SF_DPA; tr.alpha_w = W.alphaw; tr.base_w = W.pb[cur].wpi;
        tr.lam0 = &W.pout[1 + cur].lamf;
        tr.u_out = B.uf; tr.wpi_out = B.wpi; tr.dw_out = W.dw; tr.dwa_out = W.dwa; tr.J = B.J; tr.D = B.S;
        svm_status st = proj_df(h, tr, &W.pout[1 + nxt]);
        if (st != SVM_OK) return st;
        if (h->proj_pending) {
            r.cont = RC_TRIAL;
            return SVM_OK;
        }
        return trial_after_proj(r);
    } else {
        ProjIn tr;
        tr.a = W.pb[cur].u; tr.b = W.dz; tr.c1 = -t * sigma; tr.c2 = 0.0;
        tr.sums = SF_PSID | SF_DPA; tr.alpha = W.alpha; tr.pi_base = W.pb[cur].pi;
        tr.lam0 = &W.pout[1 + cur].lam;
        tr.u_out = B.u; tr.pi_out = B.pi; tr.wpi_out = B.wpi; tr.J = B.J; tr.S = B.S;
        CK(timed(h, TK_PROJ, [&] { return launch_project(W, tr, &W.pout[1 + nxt]); }));
        CK(timed(h, TK_RMATVEC, [&] { return launch_rmatvec(W, B.pi, B.wpi, B.S, &W.pout[1 + nxt].s, W.atp2, 1); }));
        grad_at_kernel<<<1, 1024, 0, W.st>>>((int)W.q, W.v, W.dv, t, W.atp2, W.tmpq, W.red);
        ++W.nlaunch;
        CK(cudaGetLastError());
    }
    return readback_issue(h);
}

// Degenerate labels (one class only): alpha = 0, b undefined.
static svm_status run_degenerate(Run &r)
{
    svm_ssnalm *h = r.h;
    Work &W = h->W;
    svm_result *res = r.res;
    const bool host_mem = h->prob.memory == SVM_MEM_HOST;
    CK(cudaMemsetAsync(W.alpha, 0, W.n * sizeof(double), W.st));
    CK(cudaMemsetAsync(W.w, 0, W.q * sizeof(double), W.st));
    cudaMemcpyKind kd = host_mem ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    CK(cudaMemcpyAsync(res->alpha, W.alpha, W.n * sizeof(double), kd, W.st));
    CK(cudaMemcpyAsync(res->w, W.w, W.q * sizeof(double), kd, W.st));
    CK(cudaStreamSynchronize(W.st));
    res->b = NAN; res->kkt = NAN; res->objective = 0.0; res->primal_objective = NAN; res->gap = NAN;
    res->sigma = h->P.sigma0; res->outer_iters = 0; res->inner_iters_total = 0;
    res->n_free = res->n_upper = res->n_sv = 0;
    res->status = SVM_ERR_DEGENERATE;
    h->err = "labels of one class only";
    r.ret = SVM_ERR_DEGENERATE;
    r.ph = RP_DONE;
    return SVM_OK;
}

// Kernels of the phase before its forward products.
static svm_status run_pre(Run &r)
{
    svm_ssnalm *h = r.h;
    Work &W = h->W;
    const svm_params &P = h->P;
    const bool host_mem = h->prob.memory == SVM_MEM_HOST;
    const long long n = W.n;
    const int q = (int)W.q;
    const bool df = W.df;
    r.mv = MvReq();
    r.has_task = false;
    r.has_wtask = false;
    switch (r.ph) {
    case RP_INIT: {
        // lambda warm starts restart at 0
        CK(cudaMemsetAsync(W.pout, 0, 4 * sizeof(ProjOut), W.st));
        r.cur = 0;
        r.sigma = P.sigma0;
        // start point: alpha^0 = Pi(alpha0) (or 0); the ALM dual starts at v = A'alpha^0
        // (w^0 = 0 when cold, Sec. 4.1)
        if (r.alpha0) {
            cudaMemcpyKind kin = host_mem ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
            CK(cudaMemcpyAsync(W.tmpn, r.alpha0, n * sizeof(double), kin, W.st));
            if (df) {
                // y o Pi(alpha0) and A'Pi(alpha0) (the delta list against 0 is the support)
                CK(split_vector(W, W.tmpn, false, W.pb[1].uf));
                ProjDF in;
                in.a = W.pb[1].uf;
                in.wpi_out = W.alphaw; in.dw_out = W.dw; in.dwa_out = W.dwa; in.D = W.pb[0].S;
                CK(timed(h, TK_PROJ, [&] { return launch_project_df(W, in, &W.pout[SLOT_OP]); }));
                CK(timed(h, TK_RMATVEC, [&] {
                    return launch_rmatvec_df(W, W.dw, W.dwa, W.pb[0].S, &W.pout[SLOT_OP].s, nullptr, nullptr, W.v,
                                             nullptr, -1);
                }));
            } else {
                ProjIn in;
                in.a = W.tmpn; in.pi_out = W.alpha; in.S = W.pb[0].S; in.wpi_out = W.pb[0].wpi;
                CK(timed(h, TK_PROJ, [&] { return launch_project(W, in, &W.pout[SLOT_OP]); }));
                CK(timed(h, TK_RMATVEC, [&] {
                    return launch_rmatvec(W, W.alpha, W.pb[0].wpi, W.pb[0].S, &W.pout[SLOT_OP].s, W.v, -1);
                }));
            }
            copyq_kernel<<<1, 1024, 0, W.st>>>(q, W.v, W.w);
            ++W.nlaunch;
            CK(cudaGetLastError());
            // Q alpha = A w and z = A v (equal here) in one pass
            mv_add(W, r.mv, W.w, W.qaf, W.qa);
            mv_add(W, r.mv, W.v, W.zf, W.z);
        } else {
            CK(cudaMemsetAsync(W.v, 0, q * sizeof(double), W.st));
            CK(cudaMemsetAsync(W.w, 0, q * sizeof(double), W.st));
            if (df) {
                CK(cudaMemsetAsync(W.alphaw, 0, n * sizeof(float2), W.st));
                CK(cudaMemsetAsync(W.qaf, 0, n * sizeof(float2), W.st));
                CK(cudaMemsetAsync(W.zf, 0, n * sizeof(float2), W.st));
            } else {
                CK(cudaMemsetAsync(W.alpha, 0, n * sizeof(double), W.st));
                CK(cudaMemsetAsync(W.qa, 0, n * sizeof(double), W.st));
                CK(cudaMemsetAsync(W.z, 0, n * sizeof(double), W.st));
            }
        }
        return SVM_OK;
    }
    case RP_SUBSTART:
    case RP_TRIAL:
    case RP_FINISH:
        return SVM_OK;
    case RP_NEWTON: {
        // Algorithm 3, Step 1: Newton direction on the free set J (with the
        // Armijo quantities g'dv, v'dv, dv'dv), then A dv = Q d
        const long long p = W.h_pout[1 + r.cur].p;
        const double sigma = r.sigma;
        const int cur = r.cur;
        // CG is run to kCgFloor x the subproblem's stopping level (within Algorithm 3's bound)
        W.cg_floor = kCgFloor * r.t_in;
        r.has_task = r.defer_newton && newton_task(W, W.pb[cur].J, p, sigma, W.g, W.dv, true, &r.task);
        r.has_wtask = !r.has_task && r.defer_newton && newton_is_wide(W, p);
        if (r.has_task) {
            h->kcalls[TK_NEWTON]++;
        } else if (r.has_wtask) {
            // Gram, M_pre and the column sums now; the set-up and the CG in the batch launch
            CK(timed(h, TK_NEWTON, [&] { return newton_mfw_prepare(W, W.pb[cur].J, p, sigma, W.g, W.dv, true); }));
        } else {
            CK(timed(h, TK_NEWTON, [&] {
                return launch_newton(W, W.pb[cur].J, p, &W.pout[1 + cur].p, sigma, W.g, W.dv, true);
            }));
        }
        mv_add(W, r.mv, W.dv, W.dzf, W.dz);
        return SVM_OK;
    }
    case RP_OUTER_END: {
        // alpha^{k+1} = Pi(u(w^{k+1}))  (eq. (3.5)): the buffer holding pi becomes
        // alpha (the old alpha buffer takes its place); A'alpha^{k+1} is the last A'pi
        if (df) std::swap(W.alphaw, W.pb[r.cur].wpi);
        else std::swap(W.alpha, W.pb[r.cur].pi);
        std::swap(W.w, W.atp);   // the next subproblem forms A'pi afresh into the other buffer
        // Q alpha = A w for the KKT test and z = A v for the next subproblem, one pass
        mv_add(W, r.mv, W.w, W.qaf, W.qa);
        mv_add(W, r.mv, W.v, W.zf, W.z);
        return SVM_OK;
    }
    case RP_DONE:
        return SVM_OK;
    }
    return SVM_OK;
}

// Kernels of the phase after its forward products, then the read-back.
// A'pi from scratch over the support at the start of a subproblem, and
// g = v - A'pi with |g|^2 in the same launch's epilogue
static svm_status substart_after_proj(Run &r)
{
    svm_ssnalm *h = r.h;
    Work &W = h->W;
    const int cur = r.cur;
    ProjBuf &B = W.pb[cur];
    GradOut go;
    go.v = W.v; go.g = W.g;
    CK(timed(h, TK_RMATVEC, [&] {
        return launch_rmatvec_df(W, W.dw, W.dwa, B.S, &W.pout[1 + cur].s, nullptr, nullptr, W.atp, W.atpa, 1, go);
    }));
    return readback_issue(h);
}

// The rest of a phase whose projection was launched with the batch's.
static svm_status run_post_cont(Run &r)
{
    const int c = r.cont;
    r.cont = RC_NONE;
    switch (c) {
    case RC_READBACK: return readback_issue(r.h);
    case RC_SUBSTART: return substart_after_proj(r);
    case RC_TRIAL: return trial_after_proj(r);
    default: return SVM_OK;
    }
}

static svm_status run_post(Run &r)
{
    svm_ssnalm *h = r.h;
    Work &W = h->W;
    const bool host_mem = h->prob.memory == SVM_MEM_HOST;
    const bool df = W.df;
    svm_status st;
    switch (r.ph) {
    case RP_INIT:
        if (r.alpha0) CK(cudaMemsetAsync(W.pout, 0, sizeof(ProjOut), W.st));
        if ((st = df ? kkt_project_df(h, W.alphaw) : kkt_project(h, W.alpha)) != SVM_OK) return st;
        if (h->proj_pending) { r.cont = RC_READBACK; return SVM_OK; }
        return readback_issue(h);
    case RP_SUBSTART: {
        // z = A v holds here (from the start or from the fused product of the
        // last phase).  u = alpha^k - sigma (z - e); pi = Pi(u); J   (eq. (3.3))
        r.epsk = 0.1 * pow(0.5, (double)r.k);
        const double sigma = r.sigma;
        const int cur = r.cur;
        ProjBuf &B = W.pb[cur];
        if (df) {
            // A'pi from scratch once per subproblem (the delta list against 0 is
            // the support): the incremental products of the line search then
            // carry roundoff from this subproblem only
            ProjDF in;
            in.a = W.alphaw; in.a_signed = true; in.b = W.zf; in.c1 = -sigma; in.c2 = sigma;
            in.sums = SF_DPA; in.alpha_w = W.alphaw;
            in.lam0 = &W.pout[1 + cur].lamf;
            in.u_out = B.uf; in.wpi_out = B.wpi; in.dw_out = W.dw; in.dwa_out = W.dwa; in.J = B.J; in.D = B.S;
            if ((st = proj_df(h, in, &W.pout[1 + cur])) != SVM_OK) return st;
            if (h->proj_pending) { r.cont = RC_SUBSTART; return SVM_OK; }
            return substart_after_proj(r);
        } else {
            ProjIn in;
            in.a = W.alpha; in.b = W.z; in.c1 = -sigma; in.c2 = sigma;
            in.sums = SF_DPA; in.alpha = W.alpha;
            in.lam0 = &W.pout[1 + cur].lam;
            in.u_out = B.u; in.pi_out = B.pi; in.wpi_out = B.wpi; in.J = B.J; in.S = B.S;
            CK(timed(h, TK_PROJ, [&] { return launch_project(W, in, &W.pout[1 + cur]); }));
            // g = v - A'pi (eq. (3.10) in q coordinates) and its roundoff scale
            CK(timed(h, TK_RMATVEC, [&] { return launch_rmatvec(W, B.pi, B.wpi, B.S, &W.pout[1 + cur].s, W.atp, 1); }));
            CK(launch_grad(W));
        }
        return readback_issue(h);
    }
    case RP_NEWTON:
        // Step 2: Armijo line search from t = 1
        r.t = 1.0;
        r.mtr = 0;
        return issue_trial(r);
    case RP_TRIAL:
        return issue_trial(r);
    case RP_OUTER_END:
        if ((st = df ? kkt_project_df(h, W.alphaw) : kkt_project(h, W.alpha)) != SVM_OK) return st;
        if (h->proj_pending) { r.cont = RC_READBACK; return SVM_OK; }
        return readback_issue(h);
    case RP_FINISH: {
        // results: alpha, w = A'alpha, b = lambda of the KKT projection, objective,
        // primal objective, gap, counts
        const long long n = W.n;
        const int q = (int)W.q;
        if (df) CK(join_vector(W, W.alphaw, true, W.alpha));
        cudaMemcpyKind kd = host_mem ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
        CK(cudaMemcpyAsync(r.res->alpha, W.alpha, n * sizeof(double), kd, W.st));
        CK(cudaMemcpyAsync(r.res->w, W.w, q * sizeof(double), kd, W.st));
        CK(cudaMemsetAsync(W.red + 8, 0, 3 * sizeof(double), W.st));
        count_kernel<<<W.nsm * 2, 256, 0, W.st>>>(n, W.alpha, W.C, W.red + 8);
        ++W.nlaunch;
        CK(cudaGetLastError());
        r.hw.resize((size_t)q);
        CK(cudaMemcpyAsync(r.hw.data(), W.w, q * sizeof(double), cudaMemcpyDeviceToHost, W.st));
        CK(cudaMemcpyAsync(W.h_red, W.red, 16 * sizeof(double), cudaMemcpyDeviceToHost, W.st));
        return SVM_OK;
    }
    case RP_DONE:
        return SVM_OK;
    }
    return SVM_OK;
}

// Algorithm 3's stopping test at the current point (host only): either
// another Newton step or the end of the subproblem.
static svm_status inner_check(Run &r)
{
    svm_ssnalm *h = r.h;
    Work &W = h->W;
    const svm_params &P = h->P;
    const ProjOut &m = W.h_pout[1 + r.cur];
    const double gn = sqrt(W.h_red[0]);
    const double dx = sqrt(m.sum[0]);
    const double tol_in = fmin(r.epsk, r.epsk * dx) / sqrt(r.sigma);
    const double floor_g = (W.df ? 32e-15 : 1e-15) * sqrt(W.h_red[1]);
    if (!isfinite(gn)) { h->err = "non-finite gradient"; return SVM_ERR_NUMERIC; }
    if (h->trace)
        fprintf(stderr, "[svm] k=%d j=%d sigma=%.3g p=%lld s=%lld |g|=%.3e tol=%.3e passes=%d lam=%.6g\n", r.k, r.j,
                r.sigma, (long long)m.p, (long long)m.s, gn, fmax(tol_in, floor_g), m.passes, m.lam);
    r.t_in = fmax(tol_in, floor_g);
    if (gn <= fmax(tol_in, floor_g) || r.j >= P.max_inner) {
        r.inner_total += r.j;
        r.ph = RP_OUTER_END;
    } else {
        r.ph = RP_NEWTON;
    }
    return SVM_OK;
}

// After the synchronisation that ends a phase: read its scalars and choose
// the next phase.
static svm_status run_after(Run &r)
{
    svm_ssnalm *h = r.h;
    Work &W = h->W;
    const svm_params &P = h->P;
    svm_status st;
    if (r.ph == RP_FINISH) {
        svm_result *res = r.res;
        const ProjOut &kk = W.h_pout[SLOT_KKT];
        double wsq = 0.0;
        for (double x : r.hw) wsq += x * x;
        res->kkt = kkt_value(kk);
        res->b = kk.lam;
        res->objective = 0.5 * wsq - kk.sum[2];
        res->primal_objective = 0.5 * wsq + W.C * kk.sum[3];
        res->gap = res->primal_objective + res->objective;
        res->sigma = r.sigma;
        res->outer_iters = r.k;
        res->inner_iters_total = r.inner_total;
        res->status = r.status;
        res->n_free = (int64_t)W.h_red[8];
        res->n_upper = (int64_t)W.h_red[9];
        res->n_sv = (int64_t)W.h_red[10];
        if (r.status != SVM_OK && h->err.empty()) h->err = "iteration cap reached";
        r.ret = r.status;
        r.ph = RP_DONE;
        return SVM_OK;
    }
    if ((st = readback_check(h)) != SVM_OK) return st;
    switch (r.ph) {
    case RP_INIT:
        r.R = kkt_value(W.h_pout[SLOT_KKT]);
        r.Rprev = r.R;
        r.k = 0;
        r.inner_total = 0;
        if (r.R <= P.tol) {
            r.status = SVM_OK;
            r.ph = RP_FINISH;
        } else {
            r.ph = RP_SUBSTART;
        }
        return SVM_OK;
    case RP_SUBSTART:
        r.j = 0;
        return inner_check(r);
    case RP_NEWTON:
    case RP_TRIAL: {
        const int nxt = 1 - r.cur;
        const double t = r.t;
        const double slope = W.h_red[2], vdv = W.h_red[3], dvdv = W.h_red[4];
        const double dpsi = t * vdv + 0.5 * t * t * dvdv + W.h_pout[1 + nxt].sum[1] / (2.0 * r.sigma);
        if (h->trace)
            fprintf(stderr, "[svm]   trial t=%.3g dpsi=%.3e slope=%.3e passes=%d cg=%g cg_res=%.2e\n", t, dpsi, slope,
                    W.h_pout[1 + nxt].passes, W.h_red[12], W.h_red[13]);
        if (dpsi <= P.mu * t * slope) {
            // Step 3 (z = A v is not read again before it is recomputed after the
            // inner loop: the trials project from the accepted point's u)
            if (W.df) {
                std::swap(W.v, W.vt);   // v + t dv, formed by the trial's epilogue
            } else {
                CK(launch_vaxpy(W, t));
            }
            std::swap(W.g, W.tmpq);     // the gradient at the accepted trial
            std::swap(W.atp, W.atp2);   // A'pi of the accepted trial
            std::swap(W.atpa, W.atpa2);
            r.cur = nxt;
            ++r.j;
            return inner_check(r);
        }
        r.t *= P.delta;
        if (++r.mtr < P.max_ls) {
            r.ph = RP_TRIAL;
        } else {
            // line search failed: the subproblem ends at the current point
            r.inner_total += r.j;
            r.ph = RP_OUTER_END;
        }
        return SVM_OK;
    }
    case RP_OUTER_END:
        r.R = kkt_value(W.h_pout[SLOT_KKT]);
        if (h->trace)
            fprintf(stderr, "[svm] outer k=%d inner=%d R_KKT=%.3e sigma=%.3g kkt_passes=%d\n", r.k, r.j, r.R, r.sigma,
                    W.h_pout[SLOT_KKT].passes);
        if (!isfinite(r.R)) {
            r.status = SVM_ERR_NUMERIC;
            h->err = "non-finite KKT residual";
            r.ph = RP_FINISH;
            return SVM_OK;
        }
        if (r.R <= P.tol) {
            r.status = SVM_OK;
            ++r.k;
            r.ph = RP_FINISH;
            return SVM_OK;
        }
        if (r.R > 0.5 * r.Rprev) r.sigma = fmin(P.sigma_max, P.sigma_growth * r.sigma);
        r.Rprev = r.R;
        ++r.k;
        r.ph = r.k < P.max_outer ? RP_SUBSTART : RP_FINISH;
        return SVM_OK;
    default:
        return SVM_OK;
    }
}

// Start a run: checks, then the degenerate case or the first phase.
// The arithmetic a solve of this handle runs (svm_form of the header).
static int32_t solve_form(const Work &W)
{
    const bool mixed = W.precision == SVM_PREC_MIXED;
    if (W.csr) return (mixed && W.xf32) ? SVM_FORM_COMPENSATED : SVM_FORM_FP64_CG;
    if (W.df) return SVM_FORM_MIXED;
    if (mixed) return W.xf32 ? SVM_FORM_COMPENSATED : SVM_FORM_FP64_CG;
    return SVM_FORM_FP64_DIRECT;
}

static svm_status run_begin(Run &r, svm_ssnalm *h, const double *alpha0, svm_result *res)
{
    r = Run();
    r.h = h;
    r.alpha0 = alpha0;
    r.res = res;
    res->form = solve_form(h->W);
    h->err.clear();
    // every solve builds its own Newton preconditioners: results never depend on
    // what the handle solved before
    if (h->W.mfw_st && newton_mfw_reset(h->W) != cudaSuccess) {
        h->err = "cudaMemsetAsync failed";
        return SVM_ERR_CUDA;
    }
    if (h->npos == 0 || h->npos == h->W.n) return run_degenerate(r);
    r.ph = RP_INIT;
    return SVM_OK;
}

static svm_status solve_mlp_impl(svm_ssnalm *h, svm_mlp_t *m, svm_result *res, int32_t *used_warm);

// One solve from alpha0 (NULL: the cold start), never the learned warm start.
static svm_status solve_direct(svm_ssnalm *h, const double *alpha0, svm_result *res)
{
    Run r;
    svm_status st = run_begin(r, h, alpha0, res);
    if (st != SVM_OK) return st;
    while (r.ph != RP_DONE) {
        if ((st = run_pre(r)) != SVM_OK) return st;
        if ((st = run_matvec_single(r)) != SVM_OK) return st;
        if ((st = run_post(r)) != SVM_OK) return st;
        CK(cudaStreamSynchronize(h->W.st));
        h->syncs++;
        if (h->timing) flush_timing(h);
        if ((st = run_after(r)) != SVM_OK) return st;
    }
    return r.ret;
}

extern "C" svm_status svm_ssnalm_solve(svm_ssnalm_t *h, const double *alpha0, svm_result *res)
{
    if (!h) return SVM_ERR_INVALID_ARG;
    if (!res || !res->alpha || !res->w) { h->err = "result buffers must be non-null"; return SVM_ERR_INVALID_ARG; }
    if (!alpha0 && h->wsm) return solve_mlp_impl(h, h->wsm, res, nullptr);
    return solve_direct(h, alpha0, res);
}

// ------------------------------------------------------------ batched solves

// Per-problem label checks: cnt[2b] = invalid labels, cnt[2b + 1] = +1 labels.
__global__ void batch_labels_kernel(const int8_t *__restrict__ Y, long long n, int *cnt)
{
    const int8_t *y = Y + (long long)blockIdx.y * n;
    int bad = 0, pos = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int8_t v = y[i];
        bad += (v != 1 && v != -1);
        pos += (v == 1);
    }
    for (int o = 16; o > 0; o >>= 1) {
        bad += __shfl_xor_sync(0xffffffffu, bad, o);
        pos += __shfl_xor_sync(0xffffffffu, pos, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (bad) atomicAdd(cnt + 2 * blockIdx.y, bad);
        if (pos) atomicAdd(cnt + 2 * blockIdx.y + 1, pos);
    }
}

// Severity order of per-problem outcomes for the batch's return value.
static int status_rank(svm_status st)
{
    if (st == SVM_OK) return 0;
    if (st == SVM_ERR_DEGENERATE) return 1;
    if (st == SVM_ERR_NOT_CONVERGED) return 2;
    return 3;
}

static const int kMvTile[4] = {1, 2, 4, 8};
constexpr int kMvPlanMax = 16;

// Autotuner of the batched forward product: time one pass over X with 1, 2,
// 4 and 8 vectors (CUDA events, after a warm-up) and plan, for every count
// c <= 16 of products, the split into passes of minimum measured time
// (dynamic programming); larger counts take whole passes of the tile with
// the lowest time per vector first.  The split changes no result: each
// product is bit-identical whatever tile it runs in.
static svm_status tune_batch_matvec(svm_ssnalm *h)
{
    Work &W = h->W;
    const long long n = W.n;
    const int q = (int)W.q;
    double *vs = nullptr;
    float2 *zs = nullptr;
    CK(cudaMalloc(&vs, sizeof(double) * 8 * q));
    if (cudaMalloc(&zs, sizeof(float2) * 8 * n) != cudaSuccess) {
        cudaFree(vs);
        h->err = "autotuner scratch allocation failed";
        return SVM_ERR_OOM;
    }
    cudaMemsetAsync(vs, 0, sizeof(double) * 8 * q, W.st);
    MvItem it[8];
    for (int k = 0; k < 8; ++k) it[k] = MvItem{vs + (size_t)k * q, zs + (size_t)k * n, W.y};
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaError_t err = cudaSuccess;
    for (int ti = 0; ti < 4 && err == cudaSuccess; ++ti) {
        const int nv = kMvTile[ti];
        err = launch_matvec_df_multi(W, it, nv, nv);   // warm-up
        cudaEventRecord(e0, W.st);
        for (int r = 0; r < 3 && err == cudaSuccess; ++r) err = launch_matvec_df_multi(W, it, nv, nv);
        cudaEventRecord(e1, W.st);
        if (err == cudaSuccess) err = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
        h->mv_ms[ti] = ms / 3.f;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(vs);
    cudaFree(zs);
    if (err != cudaSuccess) {
        h->err = std::string("autotuner: ") + cudaGetErrorString(err);
        return SVM_ERR_CUDA;
    }
    std::vector<double> cost(kMvPlanMax + 1, 0.0);
    h->mv_plan.assign(kMvPlanMax + 1, 1);
    for (int c = 1; c <= kMvPlanMax; ++c) {
        cost[c] = 1e300;
        for (int ti = 0; ti < 4; ++ti) {
            const int nv = kMvTile[ti];
            if (nv > c) break;
            const double cc = h->mv_ms[ti] + cost[c - nv];
            if (cc < cost[c]) { cost[c] = cc; h->mv_plan[c] = nv; }
        }
    }
    h->mv_tuned = true;
    return SVM_OK;
}

// All forward products of a lockstep phase in as few passes over X as the plan says.
static svm_status batch_matvec(svm_ssnalm *h, std::vector<MvItem> &items)
{
    Work &W = h->W;
    int best = 0;
    for (int ti = 1; ti < 4; ++ti)
        if (h->mv_ms[ti] / kMvTile[ti] < h->mv_ms[best] / kMvTile[best]) best = ti;
    size_t at = 0;
    while (at < items.size()) {
        const int left = (int)(items.size() - at);
        const int nv = left > kMvPlanMax ? kMvTile[best] : h->mv_plan[left];
        CK(timed(h, TK_MATVEC, [&] { return launch_matvec_df_multi(W, items.data() + at, nv, nv); }));
        at += (size_t)nv;
    }
    return SVM_OK;
}

extern "C" svm_status svm_ssnalm_solve_batch(svm_ssnalm_t *h, int32_t B, const int8_t *Y, const double *C,
                                             double *alpha, double *w, svm_result *results)
{
    if (!h) return SVM_ERR_INVALID_ARG;
    h->err.clear();
    if (B < 1 || !Y || !C || !alpha || !w || !results) {
        h->err = "batch: B >= 1 and non-null Y, C, alpha, w, results required";
        return SVM_ERR_INVALID_ARG;
    }
    for (int b = 0; b < B; ++b)
        if (!(C[b] > 0.0) || !isfinite(C[b])) { h->err = "batch: every C must be finite and > 0"; return SVM_ERR_INVALID_ARG; }
    Work &W = h->W;
    if (W.csr) { h->err = "batch: dense X only"; return SVM_ERR_UNSUPPORTED; }
    if (B > 65535) { h->err = "batch: at most 65535 problems per call"; return SVM_ERR_UNSUPPORTED; }
    const long long n = W.n;
    const int q = (int)W.q;
    const bool host_mem = h->prob.memory == SVM_MEM_HOST;
    // device copies of the labels and device outputs
    if (B > h->bat_cap) {
        void *bp[] = {h->bat_cnt, h->bat_y, h->bat_a, h->bat_w};
        for (void *p : bp)
            if (p) cudaFree(p);
        h->bat_cnt = nullptr; h->bat_y = nullptr; h->bat_a = nullptr; h->bat_w = nullptr;
        h->bat_cap = 0;
        if (cudaMalloc(&h->bat_cnt, sizeof(int) * 2 * B) != cudaSuccess ||
            (host_mem && (cudaMalloc(&h->bat_y, (size_t)B * n) != cudaSuccess ||
                          cudaMalloc(&h->bat_a, sizeof(double) * B * n) != cudaSuccess ||
                          cudaMalloc(&h->bat_w, sizeof(double) * B * q) != cudaSuccess))) {
            h->err = "batch: device allocation failed";
            return SVM_ERR_OOM;
        }
        h->bat_cap = B;
    }
    const int8_t *Yd = Y;
    double *Ad = alpha, *Wd = w;
    if (host_mem) {
        CK(cudaMemcpyAsync(h->bat_y, Y, (size_t)B * n, cudaMemcpyHostToDevice, W.st));
        Yd = h->bat_y;
        Ad = h->bat_a;
        Wd = h->bat_w;
    }
    CK(cudaMemsetAsync(h->bat_cnt, 0, sizeof(int) * 2 * B, W.st));
    batch_labels_kernel<<<dim3(2, B), 256, 0, W.st>>>(Yd, n, h->bat_cnt);
    ++W.nlaunch;
    CK(cudaGetLastError());
    std::vector<int> cnt((size_t)2 * B);
    CK(cudaMemcpyAsync(cnt.data(), h->bat_cnt, sizeof(int) * 2 * B, cudaMemcpyDeviceToHost, W.st));
    CK(cudaStreamSynchronize(W.st));
    for (int b = 0; b < B; ++b)
        if (cnt[2 * b]) { h->err = "batch: labels must be +1 or -1"; return SVM_ERR_INVALID_ARG; }
    // one sub-handle per problem: X borrowed from this handle, its own y, C and workspace
    while ((int)h->subs.size() < B) {
        svm_problem pr = h->prob;
        pr.memory = SVM_MEM_DEVICE;
        pr.X = W.X;
        pr.y = Yd;
        svm_params pa = h->P;
        pa.C = 1.0;
        svm_ssnalm *sb = nullptr;
        const svm_status st = create_impl(&sb, &pr, &pa, false);
        if (st != SVM_OK) { h->err = "batch: " + g_create_err; return st; }
        h->subs.push_back(sb);
    }
    const bool batched_mv = W.df;
    if (batched_mv && !h->mv_tuned) {
        const svm_status st = tune_batch_matvec(h);
        if (st != SVM_OK) return st;
    }
    if (B > h->nt_cap) {
        if (h->nt_dev) cudaFree(h->nt_dev);
        if (h->nt_host) cudaFreeHost(h->nt_host);
        h->nt_dev = nullptr;
        h->nt_host = nullptr;
        h->nt_cap = 0;
        if (cudaMalloc(&h->nt_dev, sizeof(NewtonTask) * B) != cudaSuccess ||
            cudaMallocHost(&h->nt_host, sizeof(NewtonTask) * B) != cudaSuccess) {
            h->err = "batch: allocation of the Newton task table failed";
            return SVM_ERR_OOM;
        }
        h->nt_cap = B;
    }
    if (B > h->wt_cap) {
        if (h->wt_s_dev) cudaFree(h->wt_s_dev);
        if (h->wt_c_dev) cudaFree(h->wt_c_dev);
        if (h->wt_s_host) cudaFreeHost(h->wt_s_host);
        if (h->wt_c_host) cudaFreeHost(h->wt_c_host);
        h->wt_s_dev = nullptr;
        h->wt_c_dev = nullptr;
        h->wt_s_host = nullptr;
        h->wt_c_host = nullptr;
        h->wt_cap = 0;
        if (cudaMalloc(&h->wt_s_dev, sizeof(MfwSetupArgs) * B) != cudaSuccess ||
            cudaMalloc(&h->wt_c_dev, sizeof(MfwArgs) * B) != cudaSuccess ||
            cudaMallocHost(&h->wt_s_host, sizeof(MfwSetupArgs) * B) != cudaSuccess ||
            cudaMallocHost(&h->wt_c_host, sizeof(MfwArgs) * B) != cudaSuccess) {
            h->err = "batch: allocation of the wide Newton tables failed";
            return SVM_ERR_OOM;
        }
        h->wt_cap = B;
    }
    // the projections of a phase in one launch (one cluster per problem) when
    // the problems fit the cluster form; each problem's result is bit-identical
    // to a single solve's, which runs the same cluster kernel
    const bool batched_proj = W.df && W.proj_cl > 0;
    if (batched_proj && B > h->pd_cap) {
        if (h->pd_dev) cudaFree(h->pd_dev);
        if (h->pd_host) cudaFreeHost(h->pd_host);
        h->pd_dev = nullptr;
        h->pd_host = nullptr;
        h->pd_cap = 0;
        if (cudaMalloc(&h->pd_dev, sizeof(PDArgs) * B) != cudaSuccess ||
            cudaMallocHost(&h->pd_host, sizeof(PDArgs) * B) != cudaSuccess) {
            h->err = "batch: allocation of the projection table failed";
            return SVM_ERR_OOM;
        }
        h->pd_cap = B;
    }
    // the wide Newton steps' FP16 copy of X: made once here, borrowed by every sub-handle
    if (W.mfw_st) {
        if (x16_prepare(W) != cudaSuccess) {
            h->err = "batch: the FP16 copy of X could not be made";
            return SVM_ERR_OOM;
        }
        for (svm_ssnalm *sb : h->subs) {
            if (sb->W.x16) continue;
            sb->W.x16 = W.x16;
            sb->W.x16_k = W.x16_k;
            sb->W.x16_own = false;
        }
    }
    std::vector<svm_result> res((size_t)B);
    std::vector<Run> runs((size_t)B);
    std::vector<long long> launch0((size_t)B);
    int active = 0;
    for (int b = 0; b < B; ++b) {
        svm_ssnalm *sb = h->subs[b];
        Work &S = sb->W;
        S.y = Yd + (size_t)b * n;
        sb->prob.y = S.y;
        S.C = C[b];
        sb->P = h->P;
        sb->P.C = C[b];
        sb->npos = cnt[2 * b + 1];
        sb->trace = h->trace;
        sb->timing = h->timing;
        sb->proj_defer = batched_proj && S.df && S.proj_cl == W.proj_cl && S.proj_cept == W.proj_cept;
        sb->proj_pending = false;
        launch0[b] = S.nlaunch;
        res[b] = svm_result();
        res[b].alpha = Ad + (size_t)b * n;
        res[b].w = Wd + (size_t)b * q;
        const svm_status st = run_begin(runs[b], sb, nullptr, &res[b]);
        runs[b].defer_newton = true;
        if (st != SVM_OK) { runs[b].ret = st; runs[b].ph = RP_DONE; res[b].status = st; }
        if (runs[b].ph != RP_DONE) ++active;
    }
    // lockstep: every active problem advances one phase per synchronisation
    std::vector<MvItem> items;
    std::vector<char> live((size_t)B);
    auto fail_run = [&](int b, svm_status st) {
        runs[b].ret = st;
        runs[b].ph = RP_DONE;
        res[b].status = st;
        live[b] = 0;
        --active;
    };
    while (active > 0) {
        items.clear();
        for (int b = 0; b < B; ++b) {
            live[b] = runs[b].ph != RP_DONE;
            if (!live[b]) continue;
            svm_status st = run_pre(runs[b]);
            if (st != SVM_OK) { fail_run(b, st); continue; }
            if (batched_mv) {
                const MvReq &m = runs[b].mv;
                for (int k = 0; k < m.nv; ++k) items.push_back(MvItem{m.v[k], m.zf[k], h->subs[b]->W.y});
            } else if ((st = run_matvec_single(runs[b])) != SVM_OK) {
                fail_run(b, st);
            }
        }
        // the small-free-set Newton steps of all problems: three launches
        int ntask = 0, ks_max = 0;
        for (int b = 0; b < B; ++b) {
            if (!live[b] || !runs[b].has_task) continue;
            h->nt_host[ntask++] = runs[b].task;
            if (runs[b].task.ks > ks_max) ks_max = runs[b].task.ks;
        }
        if (ntask > 0) {
            CK(cudaMemcpyAsync(h->nt_dev, h->nt_host, sizeof(NewtonTask) * ntask, cudaMemcpyHostToDevice, W.st));
            CK(timed(h, TK_NEWTON, [&] { return launch_newton_batch(W, h->nt_dev, ntask, ks_max); }));
            h->kcalls[TK_NEWTON]--;   // counted per problem when the steps were deferred
        }
        // the prepared wide Newton steps: their set-ups in one launch, their CGs in another
        int nwt = 0;
        for (int b = 0; b < B; ++b) {
            if (!live[b] || !runs[b].has_wtask) continue;
            h->wt_s_host[nwt] = h->subs[b]->W.mfw_s;
            h->wt_c_host[nwt] = h->subs[b]->W.mfw_c;
            ++nwt;
        }
        if (nwt > 0) {
            CK(cudaMemcpyAsync(h->wt_s_dev, h->wt_s_host, sizeof(MfwSetupArgs) * nwt, cudaMemcpyHostToDevice, W.st));
            CK(cudaMemcpyAsync(h->wt_c_dev, h->wt_c_host, sizeof(MfwArgs) * nwt, cudaMemcpyHostToDevice, W.st));
            CK(timed(h, TK_NEWTON, [&] { return newton_mfw_run_group(W, q, h->wt_s_dev, h->wt_c_dev, nwt); }));
            h->kcalls[TK_NEWTON]--;
        }
        if (!items.empty()) {
            const svm_status st = batch_matvec(h, items);
            if (st != SVM_OK) return st;
        }
        for (int b = 0; b < B; ++b) {
            if (!live[b]) continue;
            const svm_status st = run_post(runs[b]);
            if (st != SVM_OK) fail_run(b, st);
        }
        // the recorded projections of this phase: one launch, then each
        // problem's kernels that follow its projection
        int npd = 0;
        for (int b = 0; b < B; ++b) {
            svm_ssnalm *sb = h->subs[b];
            if (!live[b] || !sb->proj_pending) continue;
            if (make_pdargs(sb->W, sb->pend_in, sb->pend_out, &h->pd_host[npd]) != cudaSuccess) {
                sb->proj_pending = false;
                fail_run(b, SVM_ERR_CUDA);
                continue;
            }
            ++npd;
        }
        if (npd > 0) {
            CK(cudaMemcpyAsync(h->pd_dev, h->pd_host, sizeof(PDArgs) * npd, cudaMemcpyHostToDevice, W.st));
            CK(timed(h, TK_PROJ, [&] { return launch_project_df_table(W, h->pd_dev, npd); }));
            h->kcalls[TK_PROJ]--;   // counted per problem when the projections were recorded
        }
        for (int b = 0; b < B; ++b) {
            svm_ssnalm *sb = h->subs[b];
            if (!sb->proj_pending) continue;
            sb->proj_pending = false;
            if (!live[b]) continue;
            const svm_status st = run_post_cont(runs[b]);
            if (st != SVM_OK) fail_run(b, st);
        }
        CK(cudaStreamSynchronize(W.st));
        h->syncs++;
        h->batch_ticks++;
        for (int b = 0; b < B; ++b) {
            if (!live[b]) continue;
            svm_ssnalm *sb = h->subs[b];
            if (sb->timing) flush_timing(sb);
            const svm_status st = run_after(runs[b]);
            if (st != SVM_OK) { fail_run(b, st); continue; }
            if (runs[b].ph == RP_DONE) --active;
        }
    }
    if (h->timing) flush_timing(h);
    if (host_mem) {
        CK(cudaMemcpyAsync(alpha, Ad, sizeof(double) * B * n, cudaMemcpyDeviceToHost, W.st));
        CK(cudaMemcpyAsync(w, Wd, sizeof(double) * B * q, cudaMemcpyDeviceToHost, W.st));
        CK(cudaStreamSynchronize(W.st));
    }
    // results, and the problems' launches and step counts folded into this handle's counters
    svm_status worst = SVM_OK;
    for (int b = 0; b < B; ++b) {
        svm_ssnalm *sb = h->subs[b];
        results[b] = res[b];
        results[b].alpha = alpha + (size_t)b * n;
        results[b].w = w + (size_t)b * q;
        const svm_status st = runs[b].ret;
        results[b].status = st;
        if (status_rank(st) > status_rank(worst)) {
            worst = st;
            h->err = "batch problem " + std::to_string(b) + ": " + sb->err;
        }
        W.nlaunch += sb->W.nlaunch - launch0[b];
        sb->proj_defer = false;
        for (int k = 0; k < 5; ++k) {
            h->kcalls[k] += sb->kcalls[k];
            h->kms[k] += sb->kms[k];
            sb->kcalls[k] = 0;
            sb->kms[k] = 0.0;
        }
    }
    return worst;
}

// ------------------------------------------------------------ step-level ops

extern "C" svm_status svm_op_matvec(svm_ssnalm_t *h, const double *v, double *z)
{
    if (!h || !v || !z) return SVM_ERR_INVALID_ARG;
    CK(timed(h, TK_MATVEC, [&] { return launch_matvec(h->W, v, z); }));
    CK(cudaStreamSynchronize(h->W.st));
    return SVM_OK;
}

extern "C" svm_status svm_op_rmatvec(svm_ssnalm_t *h, const double *c, double *out)
{
    if (!h || !c || !out) return SVM_ERR_INVALID_ARG;
    Work &W = h->W;
    // the mixed form reads y_i c_i as FP32 (hi, lo) pairs: split them here
    const float2 *wc = nullptr;
    if (W.precision == SVM_PREC_MIXED && W.xf32) {
        split_weights(W, c, W.pb[0].wpi);
        wc = W.pb[0].wpi;
    }
    CK(timed(h, TK_RMATVEC, [&] { return launch_rmatvec(W, c, wc, nullptr, nullptr, out, -1); }));
    CK(cudaStreamSynchronize(W.st));
    return SVM_OK;
}

extern "C" svm_status svm_op_project(svm_ssnalm_t *h, const double *u, double *pi, double *lambda, int32_t *J,
                                     int64_t *p_out, int32_t *S, int64_t *s_out)
{
    if (!h || !u || !pi) return SVM_ERR_INVALID_ARG;
    Work &W = h->W;
    if (W.df) {
        // the double-float kernel of the mixed form: u split on the device, pi joined back
        CK(split_vector(W, u, false, W.pb[1].uf));
        ProjDF in;
        in.a = W.pb[1].uf; in.wpi_out = W.pb[1].wpi; in.J = J;
        if (S) { in.D = S; in.dw_out = W.dw; in.dwa_out = W.dwa; }   // the delta list against 0 is the support
        CK(timed(h, TK_PROJ, [&] { return launch_project_df(W, in, &W.pout[SLOT_OP]); }));
        CK(join_vector(W, W.pb[1].wpi, true, pi));
    } else {
        ProjIn in;
        in.a = u; in.pi_out = pi; in.J = J; in.S = S;
        CK(timed(h, TK_PROJ, [&] { return launch_project(W, in, &W.pout[SLOT_OP]); }));
    }
    svm_status st = sync_read(h);
    if (st != SVM_OK) return st;
    if (lambda) *lambda = W.h_pout[SLOT_OP].lam;
    if (p_out) *p_out = W.h_pout[SLOT_OP].p;
    if (s_out) *s_out = W.h_pout[SLOT_OP].s;
    return SVM_OK;
}

extern "C" svm_status svm_op_newton(svm_ssnalm_t *h, const int32_t *J, int64_t p, double sigma, const double *g,
                                    double *dv)
{
    if (!h || !g || !dv || p < 0 || (p > 0 && !J) || !(sigma > 0.0)) return SVM_ERR_INVALID_ARG;
    Work &W = h->W;
    W.cg_floor = 0.0;   // the step as exact as a direct solve
    CK(timed(h, TK_NEWTON, [&] { return launch_newton(W, J, p, nullptr, sigma, g, dv); }));
    return sync_read(h);
}

extern "C" svm_status svm_op_gram(svm_ssnalm_t *h, const int32_t *J, int64_t p, double *G, double *hsum)
{
    if (!h || !G || !hsum || p < 0 || (p > 0 && !J)) return SVM_ERR_INVALID_ARG;
    Work &W = h->W;
    const int64_t q = W.q;
    if (W.csr || !W.xf32 || q % 16 != 0 || q > 1024) {
        h->err = "svm_op_gram: dense FP32 X with q % 16 == 0 and q <= 1024 only";
        return SVM_ERR_UNSUPPORTED;
    }
    float *cpart = reinterpret_cast<float *>(W.part);
    if (q <= 128) {
        if (gram_umma_part_floats(W) > 2 * W.part_len) {
            h->err = "svm_op_gram: workspace too small";
            return SVM_ERR_UNSUPPORTED;
        }
        float2 *hpart = reinterpret_cast<float2 *>(cpart + (size_t)gram_umma_blocks(W) * q * q);
        CK(timed(h, TK_NEWTON, [&] { return launch_gram_umma(W, J, p, cpart, hpart); }));
        CK(launch_gram_umma_sum(W, gram_umma_blocks(W), cpart, gram_umma_blocks(W), hpart, G, hsum));
    } else {
        // the FP16 tensor-core Gram, then the exact column sums (scratch after the Gram partials)
        const int KS = gram_wide_splits(W, p);
        float2 *hs = reinterpret_cast<float2 *>(cpart + (size_t)KS * q * q);
        float2 *cs_part = hs + q;
        const long long room = ((long long)(2 * W.part_len) - (long long)KS * q * q - 2 * q) / (2 * q);
        if (room < 1) {
            h->err = "svm_op_gram: workspace too small";
            return SVM_ERR_UNSUPPORTED;
        }
        const int nbc = colsum_blocks(W, p, (int)(room < (1 << 20) ? room : (1 << 20)));
        CK(timed(h, TK_NEWTON, [&] { return launch_gram_umma_wide(W, J, p, KS, cpart); }));
        if (p > 0) {
            CK(launch_colsum(W, J, p, nbc, cs_part, hs));
        } else {
            CK(cudaMemsetAsync(hs, 0, q * sizeof(float2), W.st));
        }
        CK(launch_gram_umma_sum(W, KS, cpart, 1, hs, G, hsum));
    }
    return sync_read(h);
}

extern "C" svm_status svm_op_kkt(svm_ssnalm_t *h, const double *alpha, double *kkt, double *lambda)
{
    if (!h || !alpha) return SVM_ERR_INVALID_ARG;
    Work &W = h->W;
    const float2 *wc = nullptr;
    if (W.precision == SVM_PREC_MIXED && W.xf32) {
        split_weights(W, alpha, W.pb[0].wpi);
        wc = W.pb[0].wpi;
    }
    CK(timed(h, TK_RMATVEC, [&] { return launch_rmatvec(W, alpha, wc, nullptr, nullptr, W.w, -1); }));
    svm_status st;
    if (W.df) {
        // y o alpha split (pb[0].wpi) is the double-float alpha of the mixed form
        CK(timed(h, TK_MATVEC, [&] { return launch_matvec_df(W, W.w, W.qaf); }));
        st = kkt_project_df(h, W.pb[0].wpi);
    } else {
        CK(timed(h, TK_MATVEC, [&] { return launch_matvec(W, W.w, W.qa); }));
        st = kkt_project(h, alpha);
    }
    if (st != SVM_OK) return st;
    if ((st = sync_read(h)) != SVM_OK) return st;
    if (kkt) *kkt = kkt_value(W.h_pout[SLOT_KKT]);
    if (lambda) *lambda = W.h_pout[SLOT_KKT].lam;
    return SVM_OK;
}

extern "C" svm_status svm_ssnalm_set_timing(svm_ssnalm_t *h, int enable)
{
    if (!h) return SVM_ERR_INVALID_ARG;
    CK(cudaStreamSynchronize(h->W.st));
    flush_timing(h);
    h->timing = enable != 0;
    return SVM_OK;
}

extern "C" svm_status svm_ssnalm_get_stats(svm_ssnalm_t *h, svm_stats *out, int reset)
{
    if (!h || !out) return SVM_ERR_INVALID_ARG;
    CK(cudaStreamSynchronize(h->W.st));
    flush_timing(h);
    out->launches = h->W.nlaunch - h->launch_base;
    out->matvec_calls = h->kcalls[TK_MATVEC];
    out->matvec_ms = h->kms[TK_MATVEC];
    out->rmatvec_calls = h->kcalls[TK_RMATVEC];
    out->rmatvec_ms = h->kms[TK_RMATVEC];
    out->proj_calls = h->kcalls[TK_PROJ];
    out->proj_ms = h->kms[TK_PROJ];
    out->newton_calls = h->kcalls[TK_NEWTON];
    out->newton_ms = h->kms[TK_NEWTON];
    out->host_syncs = h->syncs;
    out->matvec2_calls = h->kcalls[TK_MATVEC2];
    out->matvec2_ms = h->kms[TK_MATVEC2];
    if (reset) {
        h->launch_base = h->W.nlaunch;
        for (int k = 0; k < 5; ++k) { h->kcalls[k] = 0; h->kms[k] = 0.0; }
        h->syncs = 0;
    }
    return SVM_OK;
}

// Warm start from the learned network (include/svm_mlp.h), with the cold solve
// as fallback.  The paper's own warm start is a cheaper solve of an
// approximating problem (Sec. 4.3); the network plays that role here.
// rows idx[0 .. m) of X (n x q FP32) and y into Xw (m x q) and yw
__global__ void gather_rows_kernel(const float *__restrict__ X, const int8_t *__restrict__ y, int q,
                                   const int32_t *__restrict__ idx, long long m, float *__restrict__ Xw,
                                   int8_t *__restrict__ yw)
{
    const int q4 = q / 4;
    for (long long r = blockIdx.x; r < m; r += gridDim.x) {
        const long long i = idx[r];
        const float4 *src = reinterpret_cast<const float4 *>(X + i * q);
        float4 *dst = reinterpret_cast<float4 *>(Xw + r * q);
        for (int c = threadIdx.x; c < q4; c += blockDim.x) dst[c] = __ldcs(src + c);
        if (threadIdx.x == 0) yw[r] = y[i];
    }
}

// a0 = 0, then a0[idx[r]] = aw[r]
__global__ void scatter_alpha_kernel(long long n, const int32_t *__restrict__ idx, long long m,
                                     const double *__restrict__ aw, double *__restrict__ a0)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        a0[i] = 0.0;
}
__global__ void scatter_alpha2_kernel(const int32_t *__restrict__ idx, long long m, const double *__restrict__ aw,
                                      double *__restrict__ a0)
{
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < m; r += (long long)gridDim.x * blockDim.x)
        a0[idx[r]] = aw[r];
}

// Probability of alpha_i = 0 below which a row joins the reduced solve's working
// set (SVM_WS_P0 overrides it for measurements).
static float ws_p0max()
{
    static float v = -1.f;
    if (v < 0.f) {
        const char *e = getenv("SVM_WS_P0");
        v = (e && atof(e) > 0.0 && atof(e) < 1.0) ? (float)atof(e) : 0.9f;
    }
    return v;
}

// The learned warm start: the network's working set J0 (rows not predicted to
// end at alpha = 0 with probability >= 0.9) is solved as an SVM of its own
// (same C and tolerance, cold), and its solution, zero elsewhere, starts the
// full solve; when J0 holds every support vector the full solve stops at its
// first KKT test.  A reduced problem larger than half of the rows costs about
// a full solve, and one that is degenerate (one class) is no problem at all:
// then the full problem is solved cold.
static svm_status solve_mlp_impl(svm_ssnalm *h, svm_mlp_t *m, svm_result *res, int32_t *used_warm)
{
    if (used_warm) *used_warm = 0;
    Work &W = h->W;
    if (W.csr || !W.xf32 || W.q != SVM_MLP_IN - 4) {
        h->err = "the warm-start network needs dense FP32 X with q = 128";
        return SVM_ERR_UNSUPPORTED;
    }
    const long long n = W.n;
    const int q = (int)W.q;
    const int G = 2 * W.nsm;
    float *F = nullptr, *Xw = nullptr;
    double *a0 = nullptr, *aw = nullptr, *ww = nullptr;
    int32_t *idx = nullptr;
    int8_t *yw = nullptr;
    int2 *blk = nullptr;
    long long *tot = nullptr;
    auto release = [&]() {
        void *p[] = {F, Xw, a0, aw, ww, idx, yw, blk, tot};
        for (void *x : p)
            if (x) cudaFreeAsync(x, W.st);
    };
    if (cudaMallocAsync(&F, sizeof(float) * n * SVM_MLP_IN, W.st) != cudaSuccess ||
        cudaMallocAsync(&a0, sizeof(double) * n, W.st) != cudaSuccess ||
        cudaMallocAsync(&idx, sizeof(int32_t) * n, W.st) != cudaSuccess ||
        cudaMallocAsync(&blk, sizeof(int2) * G, W.st) != cudaSuccess ||
        cudaMallocAsync(&tot, sizeof(long long) * 2, W.st) != cudaSuccess) {
        release();
        h->err = "device allocation of the warm-start buffers failed";
        return SVM_ERR_OOM;
    }
    svm_status st = svm_mlp_features((const float *)W.X, W.y, n, W.q, h->P.C, F, W.st);
    long long ht[2] = {0, 0};
    if (st == SVM_OK &&
        (mlp_working_set(m, F, n, W.y, ws_p0max(), G, blk, idx, tot) != cudaSuccess ||
         cudaMemcpyAsync(ht, tot, sizeof(ht), cudaMemcpyDeviceToHost, W.st) != cudaSuccess ||
         cudaStreamSynchronize(W.st) != cudaSuccess))
        st = SVM_ERR_CUDA;
    bool reduced = false;
    const long long mw = ht[0];
    if (st == SVM_OK && mw >= 2 && 2 * mw <= n && ht[1] > 0 && ht[1] < mw) {
        if (cudaMallocAsync(&Xw, sizeof(float) * mw * q, W.st) != cudaSuccess ||
            cudaMallocAsync(&yw, mw, W.st) != cudaSuccess ||
            cudaMallocAsync(&aw, sizeof(double) * mw, W.st) != cudaSuccess ||
            cudaMallocAsync(&ww, sizeof(double) * q, W.st) != cudaSuccess) {
            release();
            h->err = "device allocation of the warm-start buffers failed";
            return SVM_ERR_OOM;
        }
        gather_rows_kernel<<<(unsigned)(mw < 4096 ? mw : 4096), 32, 0, W.st>>>((const float *)W.X, W.y, q, idx, mw,
                                                                                Xw, yw);
        svm_problem pw = h->prob;
        pw.n = mw;
        pw.layout = SVM_DENSE_ROWMAJOR;
        pw.dtype = SVM_F32;
        pw.memory = SVM_MEM_DEVICE;
        pw.X = Xw;
        pw.y = yw;
        svm_ssnalm_t *sub = nullptr;
        const auto t0 = std::chrono::steady_clock::now();
        svm_status sc = cudaGetLastError() == cudaSuccess ? create_impl(&sub, &pw, &h->P, false) : SVM_ERR_CUDA;
        if (sc == SVM_OK) {
            sub->npos = ht[1];
            svm_result rw{};
            rw.alpha = aw;
            rw.w = ww;
            if (h->trace) cudaStreamSynchronize(W.st);
            const auto t1 = std::chrono::steady_clock::now();
            sc = solve_direct(sub, nullptr, &rw);
            if (h->trace) {
                cudaStreamSynchronize(W.st);
                const auto t2 = std::chrono::steady_clock::now();
                fprintf(stderr, "[svm] warm start: working set %lld of %lld rows; create %.2f ms, reduced solve %.2f ms "
                        "(%d outer, R_KKT %.2e)\n", mw, n, std::chrono::duration<double, std::milli>(t1 - t0).count(),
                        std::chrono::duration<double, std::milli>(t2 - t1).count(), rw.outer_iters, rw.kkt);
            }
            if (sc == SVM_OK || sc == SVM_ERR_NOT_CONVERGED) {
                scatter_alpha_kernel<<<W.nsm * 4, 256, 0, W.st>>>(n, idx, mw, aw, a0);
                scatter_alpha2_kernel<<<W.nsm * 4, 256, 0, W.st>>>(idx, mw, aw, a0);
                reduced = cudaGetLastError() == cudaSuccess;
            }
            svm_ssnalm_destroy(sub);
        }
    }
    std::vector<double> host_a0;
    if (st == SVM_OK && reduced && h->prob.memory == SVM_MEM_HOST) {
        host_a0.resize((size_t)n);
        if (cudaMemcpyAsync(host_a0.data(), a0, sizeof(double) * n, cudaMemcpyDeviceToHost, W.st) != cudaSuccess ||
            cudaStreamSynchronize(W.st) != cudaSuccess)
            st = SVM_ERR_CUDA;
    }
    if (st != SVM_OK) {
        release();
        h->err = "warm-start features or network failed";
        return st;
    }
    if (!reduced) {
        release();
        return solve_direct(h, nullptr, res);
    }
    st = solve_direct(h, h->prob.memory == SVM_MEM_HOST ? host_a0.data() : a0, res);
    release();
    if (st == SVM_ERR_NOT_CONVERGED || st == SVM_ERR_NUMERIC) return solve_direct(h, nullptr, res);
    if (used_warm) *used_warm = 1;
    return st;
}

extern "C" svm_status svm_ssnalm_solve_mlp(svm_ssnalm_t *h, svm_mlp_t *m, svm_result *res, int32_t *used_warm)
{
    if (used_warm) *used_warm = 0;
    if (!h || !m || !res || !res->alpha || !res->w) return SVM_ERR_INVALID_ARG;
    return solve_mlp_impl(h, m, res, used_warm);
}

extern "C" svm_status svm_ssnalm_set_warmstart_model(svm_ssnalm_t *h, const float *mlp_weights)
{
    if (!h) return SVM_ERR_INVALID_ARG;
    svm_mlp_destroy(h->wsm);
    h->wsm = nullptr;
    if (!mlp_weights) return SVM_OK;
    const Work &W = h->W;
    if (W.csr || !W.xf32 || W.q != SVM_MLP_IN - 4) {
        h->err = "the warm-start network needs dense FP32 X with q = 128";
        return SVM_ERR_UNSUPPORTED;
    }
    const svm_status st = svm_mlp_create(&h->wsm, mlp_weights, W.n, W.st);
    if (st != SVM_OK) {
        h->wsm = nullptr;
        h->err = "could not create the warm-start network (allocation or copy failed)";
    }
    return st;
}
