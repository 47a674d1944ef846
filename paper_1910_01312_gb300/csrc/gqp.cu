// gqp.cu -- C ABI (include/svm_gqp.h) and host control of SSsNAL for the
// unified QP of Sec. 1, eq. (1.5):
//     min 1/2 x'Qx + c'x  s.t.  a'x = d,  l <= x <= u,   Q = B B',
// with the SVR dual of eq. (1.4) as the STACKED case B = [X; -X].
//
// The control follows the C-SVC solver's (svm_ssnalm.cu) and the paper's
// order: Algorithm 1 (x^{k+1} = Pi(u(w^{k+1})), eq. (3.5)) around Algorithm 3
// (Newton direction from Proposition 3.5, Armijo line search on psi of eq.
// (3.3)), stopped by R_KKT of eq. (4.1), in the coordinates v = B'w:
// Qw = B v =: z, <w, Qw> = |v|^2, grad psi = B g with g = v - B'pi.
// Readings where the paper leaves a choice (the same as the C-SVC solver's):
// sigma_0 = 1, sigma *= 5 (cap 1e6) when R_KKT fell by less than 1/2; inner
// stop |g| <= min(eps_k, eps_k |pi - x^k|)/sqrt(sigma), eps_k = 0.1 * 0.5^k,
// floored at 1e-15 | |B|'|pi| | (the roundoff level of g), at most max_inner
// Newton steps, a failed line search ends the subproblem; Armijo mu = 1e-4,
// delta = 0.5; z = B v recomputed at the start of every subproblem.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <new>
#include <string>

#include "../../include/svm_gqp.h"
#include "gqp.cuh"

using namespace svm;

struct svm_gqp {
    gqp::Ws W;
    svm_params P;
    int memory = SVM_MEM_DEVICE;
    std::string err;
    // owned storage (host-memory problems, SVR vectors)
    void *X_own = nullptr;
    double *vec_own = nullptr;   // c, a, l, u (4 n) when owned
    // n-vectors
    double *x = nullptr, *z = nullptr, *dz = nullptr, *zk = nullptr;
    double *wv[2] = {nullptr, nullptr}, *pi[2] = {nullptr, nullptr};
    int32_t *J[2] = {nullptr, nullptr};
    // q-vectors and the Newton matrix
    double *v = nullptr, *dv = nullptr, *g = nullptr, *btp = nullptr, *wq = nullptr, *M = nullptr;
    double *red = nullptr, *h_red = nullptr;   // device / pinned: 8 doubles
    double *lam = nullptr;                     // device: warm starts of the two projection slots + KKT
    gqp::ProjRec *h_rec = nullptr;             // pinned
    int *h_err = nullptr;                      // pinned
};

static thread_local std::string g_gqp_create_err;

#define GK(call)                                                                                           \
    do {                                                                                                   \
        cudaError_t e_ = (call);                                                                           \
        if (e_ != cudaSuccess) {                                                                           \
            h->err = std::string(#call) + ": " + cudaGetErrorString(e_);                                   \
            return SVM_ERR_CUDA;                                                                           \
        }                                                                                                  \
    } while (0)

static void gqp_free(svm_gqp *h)
{
    gqp::Ws &W = h->W;
    void *dp[] = {h->X_own, h->vec_own, h->x, h->z, h->dz, h->zk, h->wv[0], h->wv[1], h->pi[0], h->pi[1], h->J[0],
                  h->J[1], h->v, h->dv, h->g, h->btp, h->wq, h->M, h->red, h->lam, W.ainv, W.part, W.cnt,
                  W.bar, W.err, W.rec};
    for (void *p : dp)
        if (p) cudaFree(p);
    if (h->h_red) cudaFreeHost(h->h_red);
    if (h->h_rec) cudaFreeHost(h->h_rec);
    if (h->h_err) cudaFreeHost(h->h_err);
}

extern "C" void svm_gqp_destroy(svm_gqp_t *h)
{
    if (!h) return;
    if (h->W.st) cudaStreamSynchronize(h->W.st);
    gqp_free(h);
    delete h;
}

extern "C" const char *svm_gqp_last_error(const svm_gqp_t *h)
{
    if (!h) return g_gqp_create_err.c_str();
    return h->err.c_str();
}

template <class T>
static bool dmalloc(T **p, size_t count)
{
    return cudaMalloc((void **)p, (count ? count : 1) * sizeof(T)) == cudaSuccess;
}

// Read back the device error flag and the last projection record (syncs).
static svm_status sync_rec(svm_gqp *h, bool want_rec)
{
    gqp::Ws &W = h->W;
    if (want_rec) GK(cudaMemcpyAsync(h->h_rec, W.rec, sizeof(gqp::ProjRec), cudaMemcpyDeviceToHost, W.st));
    GK(cudaMemcpyAsync(h->h_red, h->red, 8 * sizeof(double), cudaMemcpyDeviceToHost, W.st));
    GK(cudaMemcpyAsync(h->h_err, W.err, sizeof(int), cudaMemcpyDeviceToHost, W.st));
    GK(cudaStreamSynchronize(W.st));
    if (*h->h_err == DEV_TIMEOUT) { h->err = "a device-side wait timed out"; return SVM_ERR_TIMEOUT; }
    if (*h->h_err == DEV_CHOL) { h->err = "the Newton matrix is not positive definite"; return SVM_ERR_NUMERIC; }
    if (*h->h_err) { h->err = "device error"; return SVM_ERR_NUMERIC; }
    if (want_rec && h->h_rec->status == 2) { h->err = "the set {a'x = d, l <= x <= u} is empty"; return SVM_ERR_INVALID_ARG; }
    if (want_rec && h->h_rec->status == 1) { h->err = "projection root search hit its pass cap"; return SVM_ERR_NUMERIC; }
    return SVM_OK;
}

// z_kkt = Q x = B (B'x) (w = B'x kept), then the KKT projection of x - Qx - c.
static svm_status kkt_eval(svm_gqp *h, double *R, double *lam_out)
{
    gqp::Ws &W = h->W;
    GK(gqp::rmatvec(W, h->x, h->wq, nullptr));
    GK(gqp::matvec(W, h->wq, h->zk));
    gqp::ProjReq r;
    r.x = h->x; r.z = h->zk; r.sigma = 1.0; r.lam0 = h->lam + 2; r.lam_out = h->lam + 2;
    r.w_out = h->wv[1]; r.pi_out = h->pi[1]; r.J = nullptr;
    GK(gqp::project(W, r));
    svm_status st = sync_rec(h, true);
    if (st != SVM_OK) return st;
    const gqp::ProjRec &k = *h->h_rec;
    *R = sqrt(k.dpx) / (1.0 + sqrt(k.xx));
    if (lam_out) *lam_out = k.lam;
    return SVM_OK;
}

static svm_status create_common(svm_gqp *h, const svm_params *params)
{
    gqp::Ws &W = h->W;
    h->P = *params;
    W.st = (cudaStream_t)params->stream;
    if (cudaGetDevice(&W.dev) != cudaSuccess) { h->err = "cudaGetDevice failed"; return SVM_ERR_CUDA; }
    cudaDeviceGetAttribute(&W.nsm, cudaDevAttrMultiProcessorCount, W.dev);
    const size_t n = (size_t)W.n, q = (size_t)W.q;
    if (!dmalloc(&W.ainv, n) || !dmalloc(&W.cnt, 4096) || !dmalloc(&W.bar, 4) || !dmalloc(&W.err, 4) ||
        !dmalloc(&W.rec, 1) || !dmalloc(&h->x, n) || !dmalloc(&h->z, n) || !dmalloc(&h->dz, n) ||
        !dmalloc(&h->zk, n) || !dmalloc(&h->wv[0], n) || !dmalloc(&h->wv[1], n) || !dmalloc(&h->pi[0], n) ||
        !dmalloc(&h->pi[1], n) || !dmalloc(&h->J[0], n) || !dmalloc(&h->J[1], n) || !dmalloc(&h->v, q) ||
        !dmalloc(&h->dv, q) || !dmalloc(&h->g, q) || !dmalloc(&h->btp, q) || !dmalloc(&h->wq, q) ||
        !dmalloc(&h->M, q * q) || !dmalloc(&h->red, 8) || !dmalloc(&h->lam, 4)) {
        h->err = "device workspace allocation failed";
        return SVM_ERR_OOM;
    }
    if (cudaMallocHost(&h->h_red, 8 * sizeof(double)) != cudaSuccess ||
        cudaMallocHost(&h->h_rec, sizeof(gqp::ProjRec)) != cudaSuccess ||
        cudaMallocHost(&h->h_err, sizeof(int)) != cudaSuccess) {
        h->err = "pinned host allocation failed";
        return SVM_ERR_OOM;
    }
    cudaError_t e = gqp::setup(W);
    if (e != cudaSuccess) { h->err = std::string("set-up: ") + cudaGetErrorString(e); return SVM_ERR_CUDA; }
    // partials: the projection's 3 G records, the product's 2 q per block, the
    // Gram's split-K q x q tiles (at least one, at most 32 MiB)
    size_t need = (size_t)3 * W.proj_grid * 8;
    if (need < (size_t)2 * W.rm_grid * q) need = (size_t)2 * W.rm_grid * q;
    size_t gram = (size_t)(4 * W.nsm) * (q * q + q);
    const size_t cap = ((size_t)32 << 20) / sizeof(double);
    if (gram > cap) gram = cap > (q * q + q) ? cap : (q * q + q);
    if (need < gram) need = gram;
    W.part_len = need;
    if (!dmalloc(&W.part, need) || W.proj_grid > 4096) { h->err = "device workspace allocation failed"; return SVM_ERR_OOM; }
    cudaMemsetAsync(W.bar, 0, 4 * sizeof(unsigned), W.st);
    cudaMemsetAsync(W.err, 0, sizeof(int), W.st);
    cudaMemsetAsync(h->lam, 0, 4 * sizeof(double), W.st);
    // validation: finite values, l <= u, then one projection (of -c) for a non-empty set
    int *flags = nullptr;
    if (!dmalloc(&flags, 4)) { h->err = "device allocation failed"; return SVM_ERR_OOM; }
    cudaMemsetAsync(flags, 0, 4 * sizeof(int), W.st);
    gqp::validate(W, flags);
    int hf[4] = {0, 0, 0, 0};
    cudaMemcpyAsync(hf, flags, sizeof(hf), cudaMemcpyDeviceToHost, W.st);
    e = cudaStreamSynchronize(W.st);
    cudaFree(flags);
    if (e != cudaSuccess) { h->err = std::string("create: ") + cudaGetErrorString(e); return SVM_ERR_CUDA; }
    if (hf[0]) { h->err = "B has non-finite entries"; return SVM_ERR_INVALID_ARG; }
    if (hf[1]) { h->err = "c, a, l or u has non-finite entries"; return SVM_ERR_INVALID_ARG; }
    if (hf[2]) { h->err = "l_i > u_i for some i"; return SVM_ERR_INVALID_ARG; }
    cudaMemsetAsync(h->x, 0, n * sizeof(double), W.st);
    cudaMemsetAsync(h->z, 0, n * sizeof(double), W.st);
    gqp::ProjReq r;
    r.x = h->x; r.z = h->z; r.sigma = 1.0; r.lam0 = h->lam; r.lam_out = h->lam; r.w_out = h->wv[0];
    r.pi_out = h->pi[0];
    if ((e = gqp::project(W, r)) != cudaSuccess) { h->err = std::string("create: ") + cudaGetErrorString(e); return SVM_ERR_CUDA; }
    return sync_rec(h, true);
}

static bool finite_d(double v) { return isfinite(v) != 0; }

extern "C" svm_status svm_gqp_create(svm_gqp_t **out, const svm_gqp_problem *prob, const svm_params *params)
{
    if (out) *out = nullptr;
    if (!out || !prob || !params) { g_gqp_create_err = "null argument"; return SVM_ERR_INVALID_ARG; }
    if (prob->n < 1 || prob->q < 1) { g_gqp_create_err = "n and q must be >= 1"; return SVM_ERR_INVALID_ARG; }
    if (prob->layout != SVM_GQP_DENSE && prob->layout != SVM_GQP_STACKED) { g_gqp_create_err = "bad layout"; return SVM_ERR_INVALID_ARG; }
    if (prob->layout == SVM_GQP_STACKED && prob->n % 2) { g_gqp_create_err = "STACKED needs an even n"; return SVM_ERR_INVALID_ARG; }
    if (prob->q > 1024) { g_gqp_create_err = "q > 1024 not supported in this build"; return SVM_ERR_UNSUPPORTED; }
    if (prob->n > 0x7fffffffLL) { g_gqp_create_err = "n must fit in int32"; return SVM_ERR_UNSUPPORTED; }
    if (prob->dtype != SVM_F32 && prob->dtype != SVM_F64) { g_gqp_create_err = "dtype must be F32 or F64"; return SVM_ERR_INVALID_ARG; }
    if (prob->memory != SVM_MEM_DEVICE && prob->memory != SVM_MEM_HOST) { g_gqp_create_err = "bad memory kind"; return SVM_ERR_INVALID_ARG; }
    if (!prob->B || !prob->c || !prob->a || !prob->l || !prob->u) { g_gqp_create_err = "B, c, a, l and u must be non-null"; return SVM_ERR_INVALID_ARG; }
    if (!finite_d(prob->d)) { g_gqp_create_err = "d must be finite"; return SVM_ERR_INVALID_ARG; }
    if (!(params->tol > 0.0) || params->max_outer < 1 || params->max_inner < 1 || params->max_ls < 1)
    { g_gqp_create_err = "tol > 0 and iteration caps >= 1 required"; return SVM_ERR_INVALID_ARG; }
    svm_gqp *h = new (std::nothrow) svm_gqp();
    if (!h) { g_gqp_create_err = "out of host memory"; return SVM_ERR_OOM; }
    gqp::Ws &W = h->W;
    W.n = prob->n;
    W.q = (int)prob->q;
    W.layout = prob->layout;
    W.m = prob->layout == SVM_GQP_STACKED ? prob->n / 2 : prob->n;
    W.xf32 = prob->dtype == SVM_F32;
    W.d = prob->d;
    h->memory = prob->memory;
    W.st = (cudaStream_t)params->stream;
    auto fail = [&](svm_status st, const std::string &m) {
        g_gqp_create_err = m;
        svm_gqp_destroy(h);
        return st;
    };
    const size_t n = (size_t)W.n, xb = (size_t)W.m * W.q * (W.xf32 ? 4 : 8);
    if (prob->memory == SVM_MEM_HOST) {
        if (!dmalloc((char **)&h->X_own, xb) || !dmalloc(&h->vec_own, 4 * n)) return fail(SVM_ERR_OOM, "device allocation of the problem copy failed");
        const double *src[4] = {prob->c, prob->a, prob->l, prob->u};
        if (cudaMemcpyAsync(h->X_own, prob->B, xb, cudaMemcpyHostToDevice, W.st) != cudaSuccess)
            return fail(SVM_ERR_CUDA, "host-to-device copy failed");
        for (int k = 0; k < 4; ++k)
            if (cudaMemcpyAsync(h->vec_own + k * n, src[k], n * sizeof(double), cudaMemcpyHostToDevice, W.st) != cudaSuccess)
                return fail(SVM_ERR_CUDA, "host-to-device copy failed");
        W.X = h->X_own;
        W.c = h->vec_own; W.a = h->vec_own + n; W.lo = h->vec_own + 2 * n; W.hi = h->vec_own + 3 * n;
    } else {
        W.X = prob->B;
        W.c = prob->c; W.a = prob->a; W.lo = prob->l; W.hi = prob->u;
    }
    if ((uintptr_t)W.X % 16 != 0) return fail(SVM_ERR_INVALID_ARG, "B must be 16-byte aligned");
    const svm_status st = create_common(h, params);
    if (st != SVM_OK) return fail(st, h->err);
    *out = h;
    return SVM_OK;
}

extern "C" svm_status svm_svr_create(svm_gqp_t **out, const void *X, int64_t m, int64_t q, int32_t dtype,
                                     int32_t memory, const double *y, double eps, const svm_params *params)
{
    if (out) *out = nullptr;
    if (!out || !X || !y || !params) { g_gqp_create_err = "null argument"; return SVM_ERR_INVALID_ARG; }
    if (m < 1 || q < 1) { g_gqp_create_err = "m and q must be >= 1"; return SVM_ERR_INVALID_ARG; }
    if (!(eps >= 0.0) || !finite_d(eps)) { g_gqp_create_err = "eps must be finite and >= 0"; return SVM_ERR_INVALID_ARG; }
    if (!(params->C > 0.0) || !finite_d(params->C)) { g_gqp_create_err = "C must be finite and > 0"; return SVM_ERR_INVALID_ARG; }
    if (q > 1024) { g_gqp_create_err = "q > 1024 not supported in this build"; return SVM_ERR_UNSUPPORTED; }
    if (2 * m > 0x7fffffffLL) { g_gqp_create_err = "2m must fit in int32"; return SVM_ERR_UNSUPPORTED; }
    if (dtype != SVM_F32 && dtype != SVM_F64) { g_gqp_create_err = "dtype must be F32 or F64"; return SVM_ERR_INVALID_ARG; }
    if (memory != SVM_MEM_DEVICE && memory != SVM_MEM_HOST) { g_gqp_create_err = "bad memory kind"; return SVM_ERR_INVALID_ARG; }
    if (!(params->tol > 0.0) || params->max_outer < 1 || params->max_inner < 1 || params->max_ls < 1)
    { g_gqp_create_err = "tol > 0 and iteration caps >= 1 required"; return SVM_ERR_INVALID_ARG; }
    svm_gqp *h = new (std::nothrow) svm_gqp();
    if (!h) { g_gqp_create_err = "out of host memory"; return SVM_ERR_OOM; }
    gqp::Ws &W = h->W;
    W.n = 2 * m;
    W.m = m;
    W.q = (int)q;
    W.layout = gqp::STACKED;
    W.xf32 = dtype == SVM_F32;
    W.d = 0.0;
    h->memory = memory;
    W.st = (cudaStream_t)params->stream;
    auto fail = [&](svm_status st, const std::string &msg) {
        g_gqp_create_err = msg;
        svm_gqp_destroy(h);
        return st;
    };
    const size_t n = (size_t)W.n, xb = (size_t)m * q * (W.xf32 ? 4 : 8);
    double *ydev = nullptr;
    if (!dmalloc(&h->vec_own, 4 * n + (size_t)m)) return fail(SVM_ERR_OOM, "device allocation failed");
    ydev = h->vec_own + 4 * n;
    if (memory == SVM_MEM_HOST) {
        if (!dmalloc((char **)&h->X_own, xb)) return fail(SVM_ERR_OOM, "device allocation of the X copy failed");
        if (cudaMemcpyAsync(h->X_own, X, xb, cudaMemcpyHostToDevice, W.st) != cudaSuccess ||
            cudaMemcpyAsync(ydev, y, (size_t)m * sizeof(double), cudaMemcpyHostToDevice, W.st) != cudaSuccess)
            return fail(SVM_ERR_CUDA, "host-to-device copy failed");
        W.X = h->X_own;
    } else {
        if (cudaMemcpyAsync(ydev, y, (size_t)m * sizeof(double), cudaMemcpyDeviceToDevice, W.st) != cudaSuccess)
            return fail(SVM_ERR_CUDA, "copy of y failed");
        W.X = X;
    }
    if ((uintptr_t)W.X % 16 != 0) return fail(SVM_ERR_INVALID_ARG, "X must be 16-byte aligned");
    double *c = h->vec_own, *a = c + n, *lo = c + 2 * n, *hi = c + 3 * n;
    W.c = c; W.a = a; W.lo = lo; W.hi = hi;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&W.nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return fail(SVM_ERR_CUDA, "device query failed");
    if (gqp::svr_vectors(W, ydev, eps, params->C, c, a, lo, hi) != cudaSuccess) return fail(SVM_ERR_CUDA, "SVR set-up failed");
    const svm_status st = create_common(h, params);
    if (st != SVM_OK) return fail(st, h->err == "c, a, l or u has non-finite entries" ? "y has non-finite entries" : h->err);
    *out = h;
    return SVM_OK;
}

extern "C" svm_status svm_gqp_solve(svm_gqp_t *h, svm_gqp_result *res)
{
    if (!h) return SVM_ERR_INVALID_ARG;
    if (!res || !res->x || !res->w) { h->err = "result buffers must be non-null"; return SVM_ERR_INVALID_ARG; }
    h->err.clear();
    gqp::Ws &W = h->W;
    const svm_params &P = h->P;
    const size_t n = (size_t)W.n, q = (size_t)W.q;
    svm_status st;
    GK(cudaMemsetAsync(h->x, 0, n * sizeof(double), W.st));
    GK(cudaMemsetAsync(h->v, 0, q * sizeof(double), W.st));
    GK(cudaMemsetAsync(h->lam, 0, 4 * sizeof(double), W.st));
    double sigma = P.sigma0 > 0.0 ? P.sigma0 : 1.0;
    const double growth = P.sigma_growth > 1.0 ? P.sigma_growth : 5.0;
    const double smax = P.sigma_max > 0.0 ? P.sigma_max : 1e6;
    const double mu = P.mu > 0.0 ? P.mu : 1e-4, delta = (P.delta > 0.0 && P.delta < 1.0) ? P.delta : 0.5;
    double R = 0.0, lamk = 0.0;
    if ((st = kkt_eval(h, &R, &lamk)) != SVM_OK) return st;
    double Rprev = R;
    int status = R <= P.tol ? SVM_OK : SVM_ERR_NOT_CONVERGED;
    int k = 0, inner_total = 0;
    for (; k < P.max_outer && status != SVM_OK; ++k) {
        const double epsk = 0.1 * pow(0.5, (double)k);
        GK(gqp::matvec(W, h->v, h->z));   // z = B v = Q w
        int cur = 0;
        GK(cudaMemcpyAsync(h->lam + 1, h->lam, sizeof(double), cudaMemcpyDeviceToDevice, W.st));
        gqp::ProjReq r0;
        r0.x = h->x; r0.z = h->z; r0.sigma = sigma; r0.lam0 = h->lam; r0.lam_out = h->lam;
        r0.w_out = h->wv[cur]; r0.pi_out = h->pi[cur]; r0.J = h->J[cur];
        GK(gqp::project(W, r0));
        if ((st = sync_rec(h, true)) != SVM_OK) return st;
        gqp::ProjRec rc = *h->h_rec;
        bool ls_fail = false;
        for (int j = 0;; ++j) {
            // g = v - B'pi (eq. (3.10)), |g|, the roundoff scale
            GK(gqp::rmatvec(W, h->pi[cur], h->btp, h->red + 4));
            GK(gqp::qvec(W, h->v, h->btp, h->g, nullptr, h->red));
            if ((st = sync_rec(h, false)) != SVM_OK) return st;
            const double gn = sqrt(h->h_red[3]);
            const double tol_in = fmin(epsk, epsk * sqrt(rc.dpx)) / sqrt(sigma);
            const double floor_g = 1e-15 * sqrt(h->h_red[4]);
            if (gn <= fmax(tol_in, floor_g) || j >= P.max_inner || ls_fail) break;
            // Algorithm 3, step 1: Newton direction on the free set
            GK(gqp::newton(W, h->J[cur], rc.p, rc.sJ, sigma, h->g, h->dv, h->M));
            GK(gqp::matvec(W, h->dv, h->dz));   // B dv = Q d
            GK(gqp::qvec(W, h->v, nullptr, h->g, h->dv, h->red));
            if ((st = sync_rec(h, false)) != SVM_OK) return st;
            const double slope = h->h_red[0], vdv = h->h_red[1], dvdv = h->h_red[2];
            // step 2: Armijo line search on psi (differences term by term)
            double t = 1.0;
            bool accepted = false;
            for (int mm = 0; mm < P.max_ls; ++mm) {
                gqp::ProjReq rt;
                rt.x = h->x; rt.z = h->z; rt.dz = h->dz; rt.t = t; rt.sigma = sigma;
                rt.lam0 = h->lam + 1; rt.lam_out = h->lam + 1;
                rt.w_out = h->wv[1 - cur]; rt.pi_out = h->pi[1 - cur]; rt.J = h->J[1 - cur];
                rt.pib = h->pi[cur]; rt.wb = h->wv[cur];
                GK(gqp::project(W, rt));
                if ((st = sync_rec(h, true)) != SVM_OK) return st;
                const gqp::ProjRec &tr = *h->h_rec;
                const double dpsi = t * vdv + 0.5 * t * t * dvdv + tr.psi / (2.0 * sigma);
                if (dpsi <= mu * t * slope) {
                    accepted = true;
                    rc = tr;
                    break;
                }
                t *= delta;
            }
            if (!accepted) { ls_fail = true; continue; }
            // step 3: v += t dv, z += t B dv; the trial's projection becomes the current one
            GK(gqp::axpy_q(W, h->v, t, h->dv));
            GK(gqp::axpy_n(W, h->z, t, h->dz));
            cur = 1 - cur;
            GK(cudaMemcpyAsync(h->lam, h->lam + 1, sizeof(double), cudaMemcpyDeviceToDevice, W.st));
            ++inner_total;
        }
        // Algorithm 1, step 2 (eq. (3.5)): x^{k+1} = pi
        GK(cudaMemcpyAsync(h->x, h->pi[cur], n * sizeof(double), cudaMemcpyDeviceToDevice, W.st));
        if ((st = kkt_eval(h, &R, &lamk)) != SVM_OK) return st;
        if (!isfinite(R)) { status = SVM_ERR_NUMERIC; h->err = "non-finite KKT residual"; ++k; break; }
        if (R <= P.tol) { status = SVM_OK; ++k; break; }
        if (R > 0.5 * Rprev) sigma = fmin(smax, growth * sigma);
        Rprev = R;
    }
    // results (the last kkt_eval left w = B'x in wq and its record in h_rec)
    const gqp::ProjRec kr = *h->h_rec;
    const cudaMemcpyKind kd = h->memory == SVM_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    GK(cudaMemcpyAsync(res->x, h->x, n * sizeof(double), kd, W.st));
    GK(cudaMemcpyAsync(res->w, h->wq, q * sizeof(double), kd, W.st));
    double *hw = new (std::nothrow) double[q];
    if (!hw) { h->err = "out of host memory"; return SVM_ERR_OOM; }
    GK(cudaMemcpyAsync(hw, h->wq, q * sizeof(double), cudaMemcpyDeviceToHost, W.st));
    GK(cudaStreamSynchronize(W.st));
    double wsq = 0.0;
    for (size_t j = 0; j < q; ++j) wsq += hw[j] * hw[j];
    delete[] hw;
    res->lambda = lamk;
    res->kkt = R;
    res->objective = 0.5 * wsq + kr.cx;
    res->sigma = sigma;
    res->outer_iters = k;
    res->inner_iters_total = inner_total;
    res->status = status;
    res->n_free = kr.nfree_x;
    res->feasibility = kr.feas;   // a'x - d of the final x (the KKT projection's base point)
    if (status != SVM_OK && h->err.empty()) h->err = "iteration cap reached";
    return (svm_status)status;
}

// ------------------------------------------------------------ step-level entry points

__global__ void gqp_copy_kernel(long long n, const double *__restrict__ s, double *__restrict__ d)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        d[i] = s[i];
}

__global__ void gqp_ajsq_kernel(const double *__restrict__ a, const int32_t *__restrict__ J, long long p, double *out)
{
    __shared__ double sh[32];
    double s = 0.0;
    for (long long r = threadIdx.x; r < p; r += blockDim.x) {
        const double v = a[J[r]];
        s = fma(v, v, s);
    }
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        *out = t;
    }
}

extern "C" svm_status svm_gqp_op_project(svm_gqp_t *h, const double *w, double *x, double *lambda, int32_t *J,
                                         int64_t *p_out)
{
    if (!h) return SVM_ERR_INVALID_ARG;
    if (!w || !x || !lambda) { h->err = "null argument"; return SVM_ERR_INVALID_ARG; }
    gqp::Ws &W = h->W;
    // sigma = 0 projects the base point itself: the input w is passed as x
    gqp::ProjReq r;
    r.x = w; r.z = h->zk; r.sigma = 0.0; r.lam0 = nullptr;
    r.w_out = h->wv[1]; r.pi_out = x; r.J = J;
    GK(cudaMemsetAsync(h->zk, 0, (size_t)W.n * sizeof(double), W.st));
    GK(gqp::project(W, r));
    svm_status st = sync_rec(h, true);
    if (st != SVM_OK) return st;
    *lambda = h->h_rec->lam;
    if (p_out) *p_out = h->h_rec->p;
    return SVM_OK;
}

extern "C" svm_status svm_gqp_op_newton(svm_gqp_t *h, const int32_t *J, int64_t p, double sigma, const double *g,
                                        double *dv)
{
    if (!h) return SVM_ERR_INVALID_ARG;
    if (!g || !dv || (p > 0 && !J) || p < 0 || p > h->W.n || !(sigma > 0.0)) { h->err = "bad argument"; return SVM_ERR_INVALID_ARG; }
    gqp::Ws &W = h->W;
    double sJ = 0.0;
    if (p > 0) {
        gqp_ajsq_kernel<<<1, 1024, 0, W.st>>>(W.a, J, p, h->red + 6);
        svm_status st = sync_rec(h, false);
        if (st != SVM_OK) return st;
        sJ = h->h_red[6];
    }
    GK(gqp::newton(W, J, p, sJ, sigma, g, dv, h->M));
    return sync_rec(h, false);
}

extern "C" svm_status svm_gqp_op_matvec(svm_gqp_t *h, const double *v, double *z)
{
    if (!h) return SVM_ERR_INVALID_ARG;
    if (!v || !z) { h->err = "null argument"; return SVM_ERR_INVALID_ARG; }
    GK(gqp::matvec(h->W, v, z));
    return sync_rec(h, false);
}

extern "C" svm_status svm_gqp_op_rmatvec(svm_gqp_t *h, const double *y, double *out)
{
    if (!h) return SVM_ERR_INVALID_ARG;
    if (!y || !out) { h->err = "null argument"; return SVM_ERR_INVALID_ARG; }
    GK(gqp::rmatvec(h->W, y, out, nullptr));
    return sync_rec(h, false);
}
