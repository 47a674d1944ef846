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
//    summed term by term.
//  - z = A v is recomputed at the start of every subproblem.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

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
    long long kcalls[4] = {0, 0, 0, 0};
    double kms[4] = {0, 0, 0, 0};
    long long syncs = 0;
    long long launch_base = 0;
    bool trace = false;   // SVM_SSNALM_TRACE=1: one stderr line per Newton step
};

enum { TK_MATVEC = 0, TK_RMATVEC = 1, TK_PROJ = 2, TK_NEWTON = 3 };

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
                    W.atpa2, W.mf_st, W.mf_pinv, W.mf_counter, W.v, W.vt, W.dv, W.g, W.atp, W.atp2, W.h, W.w, W.tmpq, W.M, W.Lf, W.Mf, W.part, W.cnt,
                    W.bar, W.rm_counter, W.err, W.pout, W.red, W.X_own, W.y_own, W.csc_ptr, W.csc_row,
                    W.csc_val, W.task_beg, W.col_task, W.task_part, W.csr_tn, W.csr_q, W.csr_cg,
                    W.csr_ptr_own, W.csr_idx_own, W.csr_val_own, W.jcsc_ptr, W.jtot, W.jcol_task, W.jtask_beg,
                    W.jcsc_row, W.jcsc_val, W.jcnt, W.jtask_part, W.csr_vf, W.csr_df, W.csr_cf, W.csr_tnf};
    for (void *p : ptrs)
        if (p) cudaFree(p);
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

extern "C" svm_status svm_ssnalm_create(svm_ssnalm_t **out, const svm_problem *prob, const svm_params *params)
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
    if (bad) return fail(SVM_ERR_OOM, "device workspace allocation failed");
    if (cudaMallocHost(&W.h_pout, 4 * sizeof(ProjOut)) != cudaSuccess ||
        cudaMallocHost(&W.h_red, 16 * sizeof(double)) != cudaSuccess ||
        cudaMallocHost(&W.h_err, 4 * sizeof(int)) != cudaSuccess)
        return fail(SVM_ERR_OOM, "pinned host allocation failed");
    e = proj_setup(W);
    if (e != cudaSuccess) return fail(SVM_ERR_UNSUPPORTED, "n too large for the projection kernel");
    W.cnt_len = (size_t)W.proj_ept * W.proj_grid * 2;
    if (dalloc(&W.cnt, W.cnt_len)) return fail(SVM_ERR_OOM, "device workspace allocation failed");
    cudaMemsetAsync(W.bar, 0, 4 * sizeof(unsigned), W.st);
    cudaMemsetAsync(W.rm_counter, 0, 4 * sizeof(unsigned), W.st);
    cudaMemsetAsync(W.err, 0, 4 * sizeof(int), W.st);
    cudaMemsetAsync(W.pout, 0, 4 * sizeof(ProjOut), W.st);
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

// ------------------------------------------------------------ helpers

static svm_status sync_read(svm_ssnalm *h)
{
    Work &W = h->W;
    CK(cudaMemcpyAsync(W.h_pout, W.pout, 4 * sizeof(ProjOut), cudaMemcpyDeviceToHost, W.st));
    CK(cudaMemcpyAsync(W.h_red, W.red, 16 * sizeof(double), cudaMemcpyDeviceToHost, W.st));
    CK(cudaMemcpyAsync(W.h_err, W.err, sizeof(int), cudaMemcpyDeviceToHost, W.st));
    CK(cudaStreamSynchronize(W.st));
    h->syncs++;
    if (h->timing) flush_timing(h);
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
    CK(timed(h, TK_PROJ, [&] { return launch_project_df(W, in, &W.pout[SLOT_KKT]); }));
    return SVM_OK;
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

extern "C" svm_status svm_ssnalm_solve(svm_ssnalm_t *h, const double *alpha0, svm_result *res)
{
    if (!h) return SVM_ERR_INVALID_ARG;
    if (!res || !res->alpha || !res->w) { h->err = "result buffers must be non-null"; return SVM_ERR_INVALID_ARG; }
    Work &W = h->W;
    const svm_params &P = h->P;
    const bool host_mem = h->prob.memory == SVM_MEM_HOST;
    const long long n = W.n;
    const int q = (int)W.q;
    const bool df = W.df;
    svm_status st;
    h->err.clear();

    // degenerate labels: one class only
    if (h->npos == 0 || h->npos == n) {
        CK(cudaMemsetAsync(W.alpha, 0, n * sizeof(double), W.st));
        CK(cudaMemsetAsync(W.w, 0, q * sizeof(double), W.st));
        cudaMemcpyKind k = host_mem ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
        CK(cudaMemcpyAsync(res->alpha, W.alpha, n * sizeof(double), k, W.st));
        CK(cudaMemcpyAsync(res->w, W.w, q * sizeof(double), k, W.st));
        CK(cudaStreamSynchronize(W.st));
        res->b = NAN; res->kkt = NAN; res->objective = 0.0; res->primal_objective = NAN; res->gap = NAN;
        res->sigma = P.sigma0; res->outer_iters = 0; res->inner_iters_total = 0;
        res->n_free = res->n_upper = res->n_sv = 0;
        res->status = SVM_ERR_DEGENERATE;
        h->err = "labels of one class only";
        return SVM_ERR_DEGENERATE;
    }

    // lambda warm starts restart at 0
    CK(cudaMemsetAsync(W.pout, 0, 4 * sizeof(ProjOut), W.st));
    int cur = 0;   // projection buffer holding pi(u(v)) at the current point

    // start point: alpha^0 = Pi(alpha0) (or 0); the ALM dual starts at v = A'alpha^0
    // (w^0 = 0 when cold, Sec. 4.1)
    if (alpha0) {
        cudaMemcpyKind k = host_mem ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
        CK(cudaMemcpyAsync(W.tmpn, alpha0, n * sizeof(double), k, W.st));
        if (df) {
            // y o Pi(alpha0) and A'Pi(alpha0) (the delta list against 0 is the support)
            CK(split_vector(W, W.tmpn, false, W.pb[1].uf));
            ProjDF in;
            in.a = W.pb[1].uf;
            in.wpi_out = W.alphaw; in.dw_out = W.dw; in.dwa_out = W.dwa; in.D = W.pb[0].S;
            CK(timed(h, TK_PROJ, [&] { return launch_project_df(W, in, &W.pout[SLOT_OP]); }));
            CK(timed(h, TK_RMATVEC, [&] {
                return launch_rmatvec_df(W, W.dw, W.dwa, W.pb[0].S, &W.pout[SLOT_OP].s, nullptr, nullptr, W.v, nullptr, -1);
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
        CK(timed(h, TK_MATVEC, [&] {
            return df ? launch_matvec_df(W, W.w, W.qaf, W.v, W.zf) : launch_matvec(W, W.w, W.qa, W.v, W.z);
        }));
        CK(cudaMemsetAsync(W.pout, 0, sizeof(ProjOut), W.st));
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
    double sigma = P.sigma0;
    if ((st = df ? kkt_project_df(h, W.alphaw) : kkt_project(h, W.alpha)) != SVM_OK) return st;
    if ((st = sync_read(h)) != SVM_OK) return st;
    double R = kkt_value(W.h_pout[SLOT_KKT]), Rprev = R;
    svm_status status = SVM_ERR_NOT_CONVERGED;
    int k = 0, inner_total = 0;
    if (R <= P.tol) status = SVM_OK;
    for (k = 0; k < P.max_outer && status != SVM_OK; ++k) {
        const double epsk = 0.1 * pow(0.5, (double)k);
        // z = A v holds here (from the start or from the fused product below).
        // u = alpha^k - sigma (z - e); pi = Pi(u); J   (eq. (3.3))
        {
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
                CK(timed(h, TK_PROJ, [&] { return launch_project_df(W, in, &W.pout[1 + cur]); }));
                // ... and g = v - A'pi with |g|^2 in the same launch's epilogue
                GradOut go;
                go.v = W.v; go.g = W.g;
                CK(timed(h, TK_RMATVEC, [&] {
                    return launch_rmatvec_df(W, W.dw, W.dwa, B.S, &W.pout[1 + cur].s, nullptr, nullptr, W.atp, W.atpa, 1,
                                             go);
                }));
            } else {
                ProjIn in;
                in.a = W.alpha; in.b = W.z; in.c1 = -sigma; in.c2 = sigma;
                in.sums = SF_DPA; in.alpha = W.alpha;
                in.lam0 = &W.pout[1 + cur].lam;
                in.u_out = B.u; in.pi_out = B.pi; in.wpi_out = B.wpi; in.J = B.J; in.S = B.S;
                CK(timed(h, TK_PROJ, [&] { return launch_project(W, in, &W.pout[1 + cur]); }));
                // g = v - A'pi (eq. (3.10) in q coordinates) and its roundoff scale
                CK(timed(h, TK_RMATVEC, [&] {
                    return launch_rmatvec(W, B.pi, B.wpi, B.S, &W.pout[1 + cur].s, W.atp, 1);
                }));
                CK(launch_grad(W));
            }
            if ((st = sync_read(h)) != SVM_OK) return st;
        }
        int j = 0;
        for (j = 0;; ++j) {
            const ProjOut &m = W.h_pout[1 + cur];
            const double gn = sqrt(W.h_red[0]);
            const double dx = sqrt(m.sum[0]);
            const double tol_in = fmin(epsk, epsk * dx) / sqrt(sigma);
            const double floor_g = (df ? 32e-15 : 1e-15) * sqrt(W.h_red[1]);
            if (!isfinite(gn)) { h->err = "non-finite gradient"; return SVM_ERR_NUMERIC; }
            if (h->trace)
                fprintf(stderr, "[svm] k=%d j=%d sigma=%.3g p=%lld s=%lld |g|=%.3e tol=%.3e passes=%d lam=%.6g\n", k, j,
                        sigma, (long long)m.p, (long long)m.s, gn, fmax(tol_in, floor_g), m.passes, m.lam);
            if (gn <= fmax(tol_in, floor_g) || j >= P.max_inner) break;
            // Algorithm 3, Step 1: Newton direction on the free set J
            const long long p = m.p;
            // (with the Armijo quantities g'dv, v'dv, dv'dv)
            CK(timed(h, TK_NEWTON, [&] {
                return launch_newton(W, W.pb[cur].J, p, &W.pout[1 + cur].p, sigma, W.g, W.dv, true);
            }));
            // A dv = Q d
            CK(timed(h, TK_MATVEC, [&] { return df ? launch_matvec_df(W, W.dv, W.dzf) : launch_matvec(W, W.dv, W.dz); }));
            // Step 2: Armijo line search.  Each trial projects u - t sigma A dv into the
            // other buffer and, speculatively, forms the gradient there, so an accepted
            // trial is the next iterate's projection and gradient at no extra pass.
            double t = 1.0;
            bool accepted = false;
            const int nxt = 1 - cur;
            for (int mtr = 0; mtr < P.max_ls; ++mtr) {
                ProjBuf &B = W.pb[nxt];
                if (df) {
                    ProjDF tr;
                    tr.a = W.pb[cur].uf; tr.b = W.dzf; tr.c1 = -t * sigma; tr.c2 = 0.0;
                    tr.sums = SF_PSID | SF_DPA; tr.alpha_w = W.alphaw; tr.base_w = W.pb[cur].wpi;
                    tr.lam0 = &W.pout[1 + cur].lamf;
                    tr.u_out = B.uf; tr.wpi_out = B.wpi; tr.dw_out = W.dw; tr.dwa_out = W.dwa; tr.J = B.J; tr.D = B.S;
                    CK(timed(h, TK_PROJ, [&] { return launch_project_df(W, tr, &W.pout[1 + nxt]); }));
                    // A'pi at the trial point and, in the epilogue, vt = v + t dv and
                    // g = vt - A'pi with |g|^2 (speculative: kept if the trial is accepted)
                    GradOut go;
                    go.v = W.v; go.dv = W.dv; go.t = t; go.g = W.tmpq; go.vt = W.vt;
                    CK(timed(h, TK_RMATVEC, [&] {
                        return launch_rmatvec_df(W, W.dw, W.dwa, B.S, &W.pout[1 + nxt].s, W.atp, W.atpa, W.atp2,
                                                 W.atpa2, 1, go);
                    }));
                } else {
                    ProjIn tr;
                    tr.a = W.pb[cur].u; tr.b = W.dz; tr.c1 = -t * sigma; tr.c2 = 0.0;
                    tr.sums = SF_PSID | SF_DPA; tr.alpha = W.alpha; tr.pi_base = W.pb[cur].pi;
                    tr.lam0 = &W.pout[1 + cur].lam;
                    tr.u_out = B.u; tr.pi_out = B.pi; tr.wpi_out = B.wpi; tr.J = B.J; tr.S = B.S;
                    CK(timed(h, TK_PROJ, [&] { return launch_project(W, tr, &W.pout[1 + nxt]); }));
                    CK(timed(h, TK_RMATVEC, [&] {
                        return launch_rmatvec(W, B.pi, B.wpi, B.S, &W.pout[1 + nxt].s, W.atp2, 1);
                    }));
                    grad_at_kernel<<<1, 1024, 0, W.st>>>(q, W.v, W.dv, t, W.atp2, W.tmpq, W.red);
                    ++W.nlaunch;
                    CK(cudaGetLastError());
                }
                if ((st = sync_read(h)) != SVM_OK) return st;
                const double slope = W.h_red[2], vdv = W.h_red[3], dvdv = W.h_red[4];
                const double dpsi = t * vdv + 0.5 * t * t * dvdv + W.h_pout[1 + nxt].sum[1] / (2.0 * sigma);
                if (h->trace)
                    fprintf(stderr, "[svm]   trial t=%.3g dpsi=%.3e slope=%.3e passes=%d cg=%g cg_res=%.2e\n", t, dpsi,
                            slope, W.h_pout[1 + nxt].passes, W.h_red[12], W.h_red[13]);
                if (dpsi <= P.mu * t * slope) { accepted = true; break; }
                t *= P.delta;
            }
            if (!accepted) break;   // line search failed: the subproblem ends at the current point
            // Step 3 (z = A v is not read again before it is recomputed after the
            // inner loop: the trials project from the accepted point's u)
            if (df) {
                std::swap(W.v, W.vt);   // v + t dv, formed by the trial's epilogue
            } else {
                CK(launch_vaxpy(W, t));
            }
            std::swap(W.g, W.tmpq);     // the gradient at the accepted trial
            std::swap(W.atp, W.atp2);   // A'pi of the accepted trial
            std::swap(W.atpa, W.atpa2);
            cur = nxt;
        }
        inner_total += j;
        // alpha^{k+1} = Pi(u(w^{k+1}))  (eq. (3.5)): the buffer holding pi becomes
        // alpha (the old alpha buffer takes its place); A'alpha^{k+1} is the last A'pi
        if (df) std::swap(W.alphaw, W.pb[cur].wpi);
        else std::swap(W.alpha, W.pb[cur].pi);
        std::swap(W.w, W.atp);   // the next subproblem forms A'pi afresh into the other buffer
        // Q alpha = A w for the KKT test and z = A v for the next subproblem, one pass
        CK(timed(h, TK_MATVEC, [&] {
            return df ? launch_matvec_df(W, W.w, W.qaf, W.v, W.zf) : launch_matvec(W, W.w, W.qa, W.v, W.z);
        }));
        if ((st = df ? kkt_project_df(h, W.alphaw) : kkt_project(h, W.alpha)) != SVM_OK) return st;
        if ((st = sync_read(h)) != SVM_OK) return st;
        R = kkt_value(W.h_pout[SLOT_KKT]);
        if (h->trace)
            fprintf(stderr, "[svm] outer k=%d inner=%d R_KKT=%.3e sigma=%.3g kkt_passes=%d\n", k, j, R, sigma,
                    W.h_pout[SLOT_KKT].passes);
        if (!isfinite(R)) { status = SVM_ERR_NUMERIC; h->err = "non-finite KKT residual"; break; }
        if (R <= P.tol) { status = SVM_OK; ++k; break; }
        if (R > 0.5 * Rprev) sigma = fmin(P.sigma_max, P.sigma_growth * sigma);
        Rprev = R;
    }
    // results: alpha, w = A'alpha, b = lambda of the KKT projection, objective,
    // primal objective, gap, counts
    const ProjOut &kk = W.h_pout[SLOT_KKT];
    {
        if (df) CK(join_vector(W, W.alphaw, true, W.alpha));
        cudaMemcpyKind kd = host_mem ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
        CK(cudaMemcpyAsync(res->alpha, W.alpha, n * sizeof(double), kd, W.st));
        CK(cudaMemcpyAsync(res->w, W.w, q * sizeof(double), kd, W.st));
        CK(cudaMemsetAsync(W.red + 8, 0, 3 * sizeof(double), W.st));
        count_kernel<<<W.nsm * 2, 256, 0, W.st>>>(n, W.alpha, W.C, W.red + 8);
        ++W.nlaunch;
        CK(cudaGetLastError());
        double *hw = (double *)malloc(q * sizeof(double));
        if (!hw) { h->err = "host allocation failed"; return SVM_ERR_OOM; }
        cudaError_t e1 = cudaMemcpyAsync(hw, W.w, q * sizeof(double), cudaMemcpyDeviceToHost, W.st);
        cudaError_t e2 = cudaMemcpyAsync(W.h_red, W.red, 16 * sizeof(double), cudaMemcpyDeviceToHost, W.st);
        cudaError_t e3 = cudaStreamSynchronize(W.st);
        if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
            free(hw);
            h->err = "result copy failed";
            return SVM_ERR_CUDA;
        }
        double wsq = 0.0;
        for (int jj = 0; jj < q; ++jj) wsq += hw[jj] * hw[jj];
        free(hw);
        res->kkt = kkt_value(kk);
        res->b = kk.lam;
        res->objective = 0.5 * wsq - kk.sum[2];
        res->primal_objective = 0.5 * wsq + W.C * kk.sum[3];
        res->gap = res->primal_objective + res->objective;
        res->sigma = sigma;
        res->outer_iters = k;
        res->inner_iters_total = inner_total;
        res->status = status;
        res->n_free = (int64_t)W.h_red[8];
        res->n_upper = (int64_t)W.h_red[9];
        res->n_sv = (int64_t)W.h_red[10];
    }
    if (h->timing) flush_timing(h);
    if (status != SVM_OK && h->err.empty()) h->err = "iteration cap reached";
    return status;
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
    CK(timed(h, TK_NEWTON, [&] { return launch_newton(W, J, p, nullptr, sigma, g, dv); }));
    return sync_read(h);
}

extern "C" svm_status svm_op_gram(svm_ssnalm_t *h, const int32_t *J, int64_t p, double *G, double *hsum)
{
    if (!h || !G || !hsum || p < 0 || (p > 0 && !J)) return SVM_ERR_INVALID_ARG;
    Work &W = h->W;
    const int64_t q = W.q;
    if (W.csr || !W.xf32 || q % 16 != 0 || q > 128) {
        h->err = "svm_op_gram: dense FP32 X with q % 16 == 0 and q <= 128 only";
        return SVM_ERR_UNSUPPORTED;
    }
    if (gram_umma_part_floats(W) > 2 * W.part_len) {
        h->err = "svm_op_gram: workspace too small";
        return SVM_ERR_UNSUPPORTED;
    }
    float *cpart = reinterpret_cast<float *>(W.part);
    float2 *hpart = reinterpret_cast<float2 *>(cpart + (size_t)gram_umma_blocks(W) * q * q);
    CK(timed(h, TK_NEWTON, [&] { return launch_gram_umma(W, J, p, cpart, hpart); }));
    CK(launch_gram_umma_sum(W, cpart, hpart, G, hsum));
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
    if (reset) {
        h->launch_base = h->W.nlaunch;
        for (int k = 0; k < 4; ++k) { h->kcalls[k] = 0; h->kms[k] = 0.0; }
        h->syncs = 0;
    }
    return SVM_OK;
}

// Warm start from the learned network (include/svm_mlp.h), with the cold solve
// as fallback.  The paper's own warm start is a cheaper solve of an
// approximating problem (Sec. 4.3); the network plays that role here.
extern "C" svm_status svm_ssnalm_solve_mlp(svm_ssnalm_t *h, svm_mlp_t *m, svm_result *res, int32_t *used_warm)
{
    if (used_warm) *used_warm = 0;
    if (!h || !m || !res) return SVM_ERR_INVALID_ARG;
    Work &W = h->W;
    if (W.csr || !W.xf32 || W.q != SVM_MLP_IN - 4) {
        h->err = "the warm-start network needs dense FP32 X with q = 128";
        return SVM_ERR_UNSUPPORTED;
    }
    const long long n = W.n;
    float *F = nullptr;
    double *a0 = nullptr;
    if (cudaMallocAsync(&F, sizeof(float) * n * SVM_MLP_IN, W.st) != cudaSuccess ||
        cudaMallocAsync(&a0, sizeof(double) * n, W.st) != cudaSuccess) {
        if (F) cudaFreeAsync(F, W.st);
        h->err = "device allocation of the warm-start buffers failed";
        return SVM_ERR_OOM;
    }
    svm_status st = svm_mlp_features((const float *)W.X, W.y, n, W.q, h->P.C, F, W.st);
    if (st == SVM_OK) st = svm_mlp_start_point(m, F, n, h->P.C, a0);
    std::vector<double> host_a0;
    if (st == SVM_OK && h->prob.memory == SVM_MEM_HOST) {
        host_a0.resize((size_t)n);
        if (cudaMemcpyAsync(host_a0.data(), a0, sizeof(double) * n, cudaMemcpyDeviceToHost, W.st) != cudaSuccess ||
            cudaStreamSynchronize(W.st) != cudaSuccess)
            st = SVM_ERR_CUDA;
    }
    if (st != SVM_OK) {
        cudaFreeAsync(F, W.st);
        cudaFreeAsync(a0, W.st);
        h->err = "warm-start features or network failed";
        return st;
    }
    st = svm_ssnalm_solve(h, h->prob.memory == SVM_MEM_HOST ? host_a0.data() : a0, res);
    cudaFreeAsync(F, W.st);
    cudaFreeAsync(a0, W.st);
    if (st == SVM_ERR_NOT_CONVERGED || st == SVM_ERR_NUMERIC) return svm_ssnalm_solve(h, nullptr, res);
    if (used_warm) *used_warm = 1;
    return st;
}
