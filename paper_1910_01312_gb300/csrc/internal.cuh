// internal.cuh -- solver workspace and kernel launchers shared by the
// translation units of libsvm_ssnalm.so.  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace svm {

// Results of one projection launch, written by the device.  The FP64 kernel
// writes lam and sum; the double-float kernel writes lamf and sumf and sets
// is_df, and the host fills lam and sum from them after reading the record.
struct ProjOut {
    double lam;        // lambda-hat
    double sum[4];     // mode-dependent reductions (see ProjSums)
    long long p;       // |J|
    long long s;       // |S| (FP64 kernel) or the length of the delta list (double-float kernel)
    int passes;        // root-search passes
    int status;        // 0 ok, DEV_ROOT if the search hit its cap
    float2 lamf;       // lambda-hat as a double-float pair
    float2 sumf[4];
    int is_df;
    int pad_;
};

// What a projection launch reduces besides lambda-hat, J and S (bit flags).
enum ProjSums : int {
    SF_DPA = 1,    // sum[0] = |pi - alpha|^2                      (needs alpha)
    SF_PSID = 2,   // sum[1] = sum [pi(2u - pi) - pib(2ub - pib)]  (psi difference,
                   //          evaluated term by term in the multiplier-stationary
                   //          form pi (2u - pi - 2 lambda y); base u is `a`, base
                   //          pi is pi_base, lam0 must be the base's lambda-hat)
    SF_KKT = 4     // sum[0] = |alpha - pi|^2, sum[1] = |alpha|^2, sum[2] = sum alpha,
                   // sum[3] = sum max(0, 1 - (Qalpha_i + y_i lambda)); alpha = a, Qalpha = b
};

// FP64 projection: input u_i = a_i + c1 * b_i + c2 (b may be null), outputs.
struct ProjIn {
    const double *a = nullptr, *b = nullptr;
    double c1 = 0.0, c2 = 0.0;
    int sums = 0;
    const double *lam0 = nullptr;   // device: warm start for lambda (nullable)
    double *u_out = nullptr;
    double *pi_out = nullptr;
    float2 *wpi_out = nullptr;      // y_i pi_i as an FP32 (hi, lo) pair
    int32_t *J = nullptr, *S = nullptr;
    const double *pi_base = nullptr;
    const double *alpha = nullptr;  // alpha for SF_DPA and SF_KKT
};

// Double-float projection (mixed form): every n-vector is a float2 (hi, lo)
// pair.  u_i = a'_i + c1 b_i + c2 with a'_i = a_i, or y_i a_i when a_signed
// (a holds y o alpha).  Besides J it lists the delta set D = {i : y_i pi_i !=
// base_w_i} (base_w null = 0) with the weights dw_i = y_i pi_i - base_w_i and
// dwa_i = |pi_i| - |pi_base,i|, so that A'pi = A'pi_base + sum_D dw_i x_i.
struct ProjDF {
    const float2 *a = nullptr;
    bool a_signed = false;
    const float2 *b = nullptr;
    double c1 = 0.0, c2 = 0.0;
    int sums = 0;
    const float2 *lam0 = nullptr;     // device: warm start (nullable)
    float2 *u_out = nullptr;
    float2 *wpi_out = nullptr;        // y o pi
    const float2 *alpha_w = nullptr;  // y o alpha (SF_DPA)
    const float2 *base_w = nullptr;   // y o pi_base (SF_PSID; base of D)
    float2 *dw_out = nullptr;
    float *dwa_out = nullptr;
    int32_t *J = nullptr, *D = nullptr;
};

// One projection's output buffers (the solver keeps two and swaps them when a
// line-search trial is accepted).
struct ProjBuf {
    double *u = nullptr, *pi = nullptr;   // FP64 u (plain form) and pi
    float2 *uf = nullptr;                 // double-float u (mixed form)
    float2 *wpi = nullptr;
    int32_t *J = nullptr, *S = nullptr;
};

struct CsrCg;

// Arguments of one double-float projection launch (k_projdf.cu); the batched
// form takes a device table of them, one per problem.
struct PDArgs {
    const float2 *a;
    int a_signed;
    const float2 *b;
    float2 c1, c2;
    const int8_t *y;
    long long n;
    float2 Cd;               // C as a double-float pair
    int sums;
    const float2 *lam0;
    float2 *u_out;
    float2 *wpi_out;
    const float2 *alpha_w;
    const float2 *base_w;
    float2 *dw_out;
    float *dwa_out;
    int32_t *J, *D;
    float *part;             // cooperative form: [3][G][16] block partials
    int *cnt;                // cooperative form: [EPT][G][2] list counts
    unsigned *bar;
    int *err;
    ProjOut *out;
};

// The cooperative kernels of the wide Newton step (k_newton_wide.cu): the
// preconditioner's set-up and the CG, for one problem by a whole launch or by
// a group of blocks of a launch over several problems.
struct MfwSetupArgs {
    int q;
    const float2 *Mf;      // M_pre (value, 0) pairs
    float *Lg, *Dg, *Linv, *Pinv;
    int *fflag;
    unsigned *bar;         // the problem's own barrier counter
    int *err;
    double *info;
    const int *skip;       // this step keeps the preconditioner
};
struct MfwArgs {   // the CG
    const float *X;
    const int32_t *J;
    long long p;
    int q;
    float2 sig, rp;        // sigma and 1 / p, double-float
    const float2 *H;       // h = X_J'1, double-float
    const float *Pinv;     // q x q, row-major
    const double *g;
    double *dv;
    float eta, tau, floor;
    int maxit;
    double *info;          // [0] CG steps, [1] |residual| ([2] the factor's shift, from the set-up)
    int *err;
    const double *vdot;    // nullable: Armijo quantities into rdots[2..4]
    double *rdots;
    int vc;                // chunks of the rows of J (the same for any number of blocks)
    float2 *part;          // vc x q chunk partials of X_J'(X_J d)
    float2 *yg;            // q: their sum
    float *zg;             // q: Pinv r
    unsigned *bar;
};

struct Work {
    // problem
    int64_t n = 0, q = 0;
    int xf32 = 1;            // X (dense) or the CSR values are FP32 (else FP64)
    const void *X = nullptr;
    // CSR layout: row pointers, column indices (strictly increasing within a
    // row) and values, their CSC copy (built at create), the column tasks of
    // the transposed product (task t covers CSC entries [task_beg[t],
    // task_beg[t+1]); column j owns tasks [col_task[j], col_task[j+1])) and the
    // matrix-free Newton CG state
    bool csr = false;
    const int64_t *csr_ptr = nullptr;
    const int32_t *csr_idx = nullptr;
    const void *csr_val = nullptr;
    int64_t nnz = 0;
    int64_t *csc_ptr = nullptr;
    int32_t *csc_row = nullptr;
    void *csc_val = nullptr;
    int64_t *task_beg = nullptr, *col_task = nullptr;
    double *task_part = nullptr;
    long long ntask = 0;
    // the columns of the free set's rows, rebuilt for each Newton step
    int64_t *jcsc_ptr = nullptr, *jtot = nullptr, *jcol_task = nullptr, *jtask_beg = nullptr;
    int32_t *jcsc_row = nullptr;
    void *jcsc_val = nullptr;
    int *jcnt = nullptr;
    double *jtask_part = nullptr;
    long long jtask_cap = 0, jchunk_cap = 1;
    double *csr_tn = nullptr;   // n-vector: X_J d scattered to the rows of J
    // mixed form (FP32 values): split q-vectors (2 inputs of A v; the CG's d),
    // split y o c, and X_J d as double-float pairs
    float2 *csr_vf = nullptr, *csr_df = nullptr, *csr_cf = nullptr, *csr_tnf = nullptr;
    double *csr_q = nullptr;    // 6 q-vectors of the CG
    CsrCg *csr_cg = nullptr;
    int *h_csr_done = nullptr;  // pinned
    int csr_cg_maxit = 500;
    int64_t *csr_ptr_own = nullptr;
    int32_t *csr_idx_own = nullptr;
    void *csr_val_own = nullptr;
    const int8_t *y = nullptr;
    double C = 1.0;
    int precision = 1;
    cudaStream_t st = nullptr;
    int dev = 0, nsm = 0;
    // n-vectors (FP64) and index lists
    double *alpha = nullptr, *z = nullptr, *dz = nullptr, *qa = nullptr, *tmpn = nullptr;
    // the mixed form carries z = A v, dz = A dv, Q alpha and y o alpha as
    // double-float pairs instead (df = true; z, dz and pb[].u are then unused),
    // and forms A'pi incrementally over delta lists (weights dw, dwa)
    bool df = false;
    float2 *zf = nullptr, *dzf = nullptr, *qaf = nullptr, *alphaw = nullptr;
    float2 *dw = nullptr;
    float *dwa = nullptr;
    // sum_i |pi_i| |x_i| (the roundoff scale of A'pi) for atp and atp2
    float *atpa = nullptr, *atpa2 = nullptr;
    ProjBuf pb[2];            // current / trial projection buffers
    // q-vectors
    double *v = nullptr, *dv = nullptr, *g = nullptr, *atp = nullptr, *atp2 = nullptr, *h = nullptr,
           *w = nullptr, *tmpq = nullptr, *vt = nullptr;   // vt: v + t dv at a trial point
    // matrix-free Newton state for large free sets (mixed form, q <= 128)
    struct MfState *mf_st = nullptr;
    float *mf_pinv = nullptr;
    unsigned *mf_counter = nullptr;
    // wide matrix-free Newton state (mixed form, 128 < q <= 1024): the free
    // set (n bits) and sigma the preconditioner in M was built for
    unsigned *mfw_mask = nullptr;
    struct MfwState *mfw_st = nullptr;
    MfwSetupArgs mfw_s{};   // the step prepared by newton_mfw_prepare
    MfwArgs mfw_c{};
    // the FP16 copy of a dense FP32 X for the wide Gram (made on first use,
    // or borrowed from the handle of a batched solve): X16_if = fl16(x_if
    // 2^k_f) in rows padded to a multiple of 64 entries, and the per-feature
    // exponents k_f
    void *x16 = nullptr;
    int *x16_k = nullptr;
    bool x16_own = false;
    double *M = nullptr;      // q*q Newton matrix / Cholesky factor
    float *Lf = nullptr;      // q*(q+1) FP32 factor when it does not fit in shared memory
    float2 *Mf = nullptr;     // q*q FP32 (hi, lo) split of M (double-float CG operator)
    double eta = 0.1, tau = 0.5;   // inexact-Newton constants of Algorithm 3
    double cg_floor = 0.0;         // CG residual floor of the next Newton step (cg_tol)
    int cg_maxit = 50;
    double *part = nullptr;   // partial sums (size part_len doubles)
    size_t part_len = 0;
    int *cnt = nullptr;       // compaction counts
    size_t cnt_len = 0;
    unsigned *bar = nullptr;  // grid-barrier counter
    unsigned *rm_counter = nullptr;   // last-block counter of the mixed A'c
    int *err = nullptr;       // device error flag
    ProjOut *pout = nullptr;  // 4 slots indexed by ProjMode
    double *red = nullptr;    // 16 small reductions
    // owned copies (memory = HOST)
    void *X_own = nullptr;
    int8_t *y_own = nullptr;
    // host pinned mirror for scalar read-back
    ProjOut *h_pout = nullptr;
    double *h_red = nullptr;
    int *h_err = nullptr;
    // cooperative-launch geometry of the projection kernel
    int proj_grid = 0, proj_ept = 0;
    // the double-float projection's cluster form (n small enough for one cluster
    // per problem): cluster size (0: the cooperative form) and components per thread
    int proj_cl = 0, proj_cept = 0;
    // rmatvec geometry
    int rm_grid = 0;
    // kernels launched through this workspace (all kinds)
    long long nlaunch = 0;
};

// ---- launchers (return cudaError_t of the launch) ----
cudaError_t proj_setup(Work &W);
cudaError_t launch_project(Work &W, const ProjIn &in, ProjOut *out);
cudaError_t launch_project_df(Work &W, const ProjDF &in, ProjOut *out);
// the arguments of one double-float projection (for a batched launch)
cudaError_t make_pdargs(const Work &W, const ProjDF &in, ProjOut *out, PDArgs *A);
// nprob projections in one launch of the cluster form (table in device memory;
// every problem must have W's n and cluster geometry)
cudaError_t launch_project_df_table(Work &W, const PDArgs *table_dev, int nprob);
// choose the cluster form of the double-float projection when n allows it
cudaError_t projdf_cluster_setup(Work &W);
void *projdf_kernel_for(int ept);   // for the occupancy query of proj_setup

// z0 = A v0 (and z1 = A v1 when v1 != nullptr, in the same pass over X)
cudaError_t launch_matvec(Work &W, const double *v0, double *z0, const double *v1 = nullptr,
                          double *z1 = nullptr);
// the same with double-float outputs (mixed form, FP32 X with q % 4 == 0)
cudaError_t launch_matvec_df(Work &W, const double *v0, float2 *z0, const double *v1 = nullptr,
                             float2 *z1 = nullptr);
// One vector of a batched forward product: z_i = y_i <x_i, v> as a
// double-float pair (mixed form), labels y of that vector's problem.
struct MvItem {
    const double *v;
    float2 *z;
    const int8_t *y;
};
// nv (1, 2, 4 or 8) = count products in one pass over X (W's X, n, q and stream);
// each is bit-identical to launch_matvec_df of the same vector.
cudaError_t launch_matvec_df_multi(Work &W, const MvItem *items, int count, int nv);
// out = sum_i c_i y_i x_i over the index list idx (cnt entries, read from
// *cnt_dev on the device) or over all rows when idx == nullptr.  The mixed
// form reads the weights as y_i c_i FP32 pairs from wc (when non-null).
// Also red[slot] = sum_j (sum_i |c_i x_ij|)^2 when scale_slot >= 0.
cudaError_t launch_rmatvec(Work &W, const double *c, const float2 *wc, const int32_t *idx,
                           const long long *cnt_dev, double *out, int scale_slot);
// out = base + sum_{i in idx} wc_i x_i (double-float weights, Dot2 sums, the
// count read from *cnt_dev), aout = abase + sum_i wa_i |x_i| (FP32) and
// red[slot] = |aout|^2; base and abase may be null (zero).
// Optional epilogue of launch_rmatvec_df: vt = v + t dv (dv nullable), g = vt - out,
// red[0] = |g|^2 (the gradient of eq. (3.10) at the point whose A'pi was formed).
struct GradOut {
    const double *v = nullptr, *dv = nullptr;
    double t = 0.0;
    double *g = nullptr, *vt = nullptr;
};
cudaError_t launch_rmatvec_df(Work &W, const float2 *wc, const float *wa, const int32_t *idx, const long long *cnt_dev,
                              const double *base, const float *abase, double *out, float *aout, int slot,
                              const GradOut &go = GradOut());
// wc_i = y_i c_i as an FP32 (hi, lo) pair (input of the mixed A' c)
cudaError_t split_weights(Work &W, const double *c, float2 *wc);
// a_i = (y_i when signed, else 1) * c_i as a double-float pair
cudaError_t split_vector(Work &W, const double *c, bool signed_by_y, float2 *a);
// c_i = (y_i when signed, else 1) * (a_i.hi + a_i.lo) in FP64; the split of C maps to C
cudaError_t join_vector(Work &W, const float2 *a, bool signed_by_y, double *c);
// q-vector helpers
cudaError_t launch_grad(Work &W);            // g = v - atp; red[0] = |g|^2
cudaError_t launch_dots(Work &W);            // red[2] = g'dv, red[3] = v'dv, red[4] = dv'dv
cudaError_t launch_vaxpy(Work &W, double t); // v += t dv
cudaError_t launch_negcopy(Work &W, const double *g, double *dv); // dv = -g

// Newton direction (I + sigma A'PA) dv = -g on the free set J (p from *p_dev
// when p_host < 0); with dots, also red[2] = g'dv, red[3] = v'dv, red[4] = dv'dv.
cudaError_t launch_newton(Work &W, const int32_t *J, long long p_host, const long long *p_dev,
                          double sigma, const double *g, double *dv, bool dots = false);
// One Newton step of the mixed form with a small free set (q <= 128): the
// exact double-float Gram of the p rows J split over ks blocks (partials in
// part/hpart), M = I + sigma (G - h h'/p) into Mf, and the preconditioned CG
// for dv with the Armijo dot products (rdots[2..4], v = vdot; info = red + 12).
// newton_task fills one for W (returns false when the step takes another
// path: FP64 form, CSR, q > 128, p = 0 or the matrix-free large-p step);
// launch_newton_batch runs ntask of them (table in device memory) in three
// launches, each problem's arithmetic identical to launch_newton's.
struct NewtonTask {
    const int32_t *J;
    long long p;
    int ks, maxit;
    float2 *part, *hpart, *Mf;
    float2 pinv, sig;
    float eta, tau, floor;
    const double *g;
    double *dv, *info, *rdots;
    int *err;
    const double *vdot;
};
bool newton_task(const Work &W, const int32_t *J, long long p, double sigma, const double *g, double *dv, bool dots,
                 NewtonTask *t);
cudaError_t launch_newton_batch(Work &W, const NewtonTask *T_dev, int ntask, int ks_max);
// workspace of the large-free-set Newton solve (mixed form, FP32 X, q <= 128)
cudaError_t newton_mf_alloc(Work &W);
// Gram of the rows J on the tcgen05 tensor cores (k_umma.cu): per block b of
// gram_umma_blocks(W), cpart[b] = X_S' X_S (q x q FP32, TF32 products) and
// hpart[b] = X_S' 1 (double-float); dense FP32 X, q % 16 == 0, q <= 128.
// The partials need gram_umma_part_floats(W) floats.
int gram_umma_blocks(const Work &W);
size_t gram_umma_part_floats(const Work &W);
cudaError_t launch_gram_umma(Work &W, const int32_t *J, long long p, float *cpart, float2 *hpart);
// The same Gram for 128 < q <= 1024 (q % 16 == 0) from the FP16 copy of X,
// split over (row tile, column chunk) pairs and KS row splits: cpart[ks] (q x
// q, the entries b <= a and some above) for ks < KS (the column sums come
// from launch_colsum); gram_wide_splits(W, p) is the KS that fits the
// workspace.
int gram_wide_pairs(int q);
int gram_wide_splits(const Work &W, long long p);
// skip (nullable, device): when *skip != 0 the launch does nothing.
cudaError_t launch_gram_umma_wide(Work &W, const int32_t *J, long long p, int KS, float *cpart,
                                  const int *skip = nullptr);
// the FP16 copy of X for launch_gram_umma_wide (a no-op once made or borrowed)
cudaError_t x16_prepare(Work &W);
// H = X_J' 1 exactly (double-float, column sums in row order within each of
// nb blocks, the blocks' sums in block order, two launches); part: nb x q
// float2 scratch, nb = colsum_blocks(W, p) at most max_blocks
int colsum_blocks(const Work &W, long long p, int max_blocks);
cudaError_t launch_colsum(Work &W, const int32_t *J, long long p, int nb, float2 *part, float2 *H);
// M_pre = I + sigma (G - h h'/p) into W.Mf from G partials of tensor-core
// Grams (FP32) and Gh partials of the double-float column sums; h itself into
// H (nullable)
cudaError_t launch_build_m_tc(Work &W, int G, const float *cpart, int Gh, const float2 *hpart, long long p,
                              double sigma, float2 *H, const int *skip = nullptr);
// The Newton step for a large free set at 128 < q <= 1024 (k_newton_wide.cu)
// and its workspace (allocated at create for the mixed form)
cudaError_t launch_newton_mfw(Work &W, const int32_t *J, long long p, double sigma, const double *g, double *dv,
                              bool dots);
cudaError_t newton_mfw_alloc(Work &W);
// The wide step in two halves: prepare (reuse decision, Gram, M_pre, column
// sums: ordinary launches) fills W.mfw_s / W.mfw_c; run launches the set-up and
// the CG for this problem alone.  launch_newton_mfw is both.  The batched
// solve prepares several problems and runs them together (newton_mfw_run_group:
// one launch of the set-up and one of the CG, a group of blocks per problem;
// the same result as running each alone).
bool newton_is_wide(const Work &W, long long p);
cudaError_t newton_mfw_prepare(Work &W, const int32_t *J, long long p, double sigma, const double *g, double *dv,
                               bool dots);
cudaError_t newton_mfw_run(Work &W);
cudaError_t newton_mfw_run_group(Work &Wl, int q, const MfwSetupArgs *Ts_dev, const MfwArgs *Tc_dev, int ntask);
// forget the preconditioner (the next wide Newton step builds one)
cudaError_t newton_mfw_reset(Work &W);
// G = sum_b cpart[b], h = sum_b hpart[b] over nb partials in FP64 (block
// order), both triangles of G from the partials' lower one
cudaError_t launch_gram_umma_sum(Work &W, int nb, const float *cpart, int nbh, const float2 *hpart, double *G,
                                double *h);

// CSR layout: structure/value checks (dev_flags[0]: structure, [1]: non-finite),
// the CSC copy and column tasks, and the three products of the method
cudaError_t csr_validate(Work &W, int *dev_flags);
cudaError_t csr_setup(Work &W);
cudaError_t launch_matvec_csr(Work &W, const double *v0, double *z0, const double *v1, double *z1);
cudaError_t launch_rmatvec_csr(Work &W, const double *c, double *out, int scale_slot);
cudaError_t launch_newton_csr(Work &W, const int32_t *J, long long p, double sigma, const double *g, double *dv,
                              bool dots);

}  // namespace svm

// The working set of the reduced warm-start solve (k_mlp.cu, global scope like
// the network's handle): the rows whose predicted probability of alpha_i = 0
// is below p0max, ascending in idx; total[0] their number, total[1] how many
// have y = +1 (blk: G int2 of scratch).
struct svm_mlp;
cudaError_t mlp_working_set(svm_mlp *m, const float *F, long long n, const int8_t *y, float p0max, int G,
                            int2 *blk, int32_t *idx, long long *total);
