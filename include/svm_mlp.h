/* svm_mlp.h -- C ABI of the learned warm start for svm_ssnalm_solve.
 *
 * The paper starts SSsNAL from a random-feature solution (Sec. 4.3); here a
 * small network predicts, for every sample, whether its dual variable ends at
 * 0, strictly inside (0, C) or at C, from the sample and four statistics; the
 * rows not predicted at 0 form a reduced problem whose solution starts the
 * full solve (svm_ssnalm_solve_mlp; the cold start alpha^0 = 0 remains the
 * fallback).  The network is trained on labels
 * harvested from the solver's own solutions.
 *
 * Network: F (n x 132) -> Z1 = F W1 + b1 -> H1 = gelu(Z1) -> Z2 = H1 W2 + b2 ->
 * H2 = gelu(Z2) -> Z3 = H2 W3 + b3 (n x 3 logits; class 0: alpha = 0,
 * 1: free, 2: alpha = C), gelu(x) = x (1 + erf(x / sqrt 2)) / 2, FP32.
 * Parameters: one flat FP32 vector of SVM_MLP_NPARAM values laid out as
 * [W1 (132 x 256, row-major, input x output), b1 (256), W2 (256 x 256), b2 (256),
 *  W3 (256 x 3), b3 (3)].
 *
 * All pointers are device pointers on the network's stream (or on `stream`).
 * Calls return SVM_ERR_INVALID_ARG for null pointers or sizes out of range and
 * SVM_ERR_CUDA when a launch fails; they are stream-ordered and do not
 * synchronise unless they return a host value.
 */
#ifndef SVM_MLP_H
#define SVM_MLP_H

#include <stdint.h>

#include "svm_ssnalm.h"

#ifdef __cplusplus
extern "C" {
#endif

#define SVM_MLP_IN 132
#define SVM_MLP_HIDDEN 256
#define SVM_MLP_OUT 3
#define SVM_MLP_NPARAM 100611

typedef struct svm_mlp svm_mlp_t;

/* A network with the given initial parameters (copied) and workspace for up
 * to max_rows rows per call.  Adam moments start at zero. */
svm_status svm_mlp_create(svm_mlp_t **out, const float *params, int64_t max_rows, void *stream);
void svm_mlp_destroy(svm_mlp_t *m); /* NULL-safe */

/* Copies the current parameters (SVM_MLP_NPARAM floats) to params. */
svm_status svm_mlp_get_params(svm_mlp_t *m, float *params);

/* Features of n >= 2 samples of a q = 128 problem (X row-major FP32, labels y in
 * {-1, +1}, box bound C > 0; X and F 16-byte aligned): F_i = [x_i, y_i, |x_i|/sqrt(q), y_i (w.x_i + b)/|w|,
 * log10 C] with w = mu_+ - mu_- (difference of the class means) and
 * b = -w.(mu_+ + mu_-)/2.  F is n x 132, row-major.  Needs both classes. */
svm_status svm_mlp_features(const float *X, const int8_t *y, int64_t n, int64_t q, double C, float *F,
                            void *stream);

/* Training labels harvested from a solution alpha (n, FP64): 0 where
 * alpha_i <= 0, 2 where alpha_i >= C, 1 otherwise (the solver returns bound
 * components exactly at 0 or C). */
svm_status svm_mlp_labels(const double *alpha, int64_t n, double C, int32_t *labels, void *stream);

/* Minibatch gather: Fb[r] = F[idx[r]] (132 floats) and Lb[r] = labels[idx[r]]
 * for r < nb (idx: int64, each in [0, rows of F)). */
svm_status svm_mlp_gather(const float *F, const int32_t *labels, const int64_t *idx, int64_t nb, float *Fb,
                          int32_t *Lb, void *stream);

/* Logits (n x 3) of n <= max_rows rows of F. */
svm_status svm_mlp_forward(svm_mlp_t *m, const float *F, int64_t n, float *logits);

/* Class-weighted cross-entropy L = (1/n) sum_i cw[l_i] (logsumexp(Z3_i) - Z3_i[l_i])
 * of labels l_i in {0, 1, 2} (class weights cw: 3 floats) and its gradient with
 * respect to the parameters (SVM_MLP_NPARAM floats) by backpropagation; *loss is
 * a device float. */
svm_status svm_mlp_loss_grad(svm_mlp_t *m, const float *F, const int32_t *labels, int64_t n, const float *cw,
                             float *loss, float *grad);

/* One AdamW step (Adam of Kingma and Ba, 2015, with the decoupled weight decay
 * of Loshchilov and Hutter, 2019; beta1 = 0.9, beta2 = 0.999, eps = 1e-8,
 * bias-corrected): theta -= lr (m_hat / (sqrt(v_hat) + eps) + wd theta), with
 * gradient grad at step t >= 1, learning rate lr > 0 and decay wd >= 0. */
svm_status svm_mlp_adam_step(svm_mlp_t *m, const float *grad, int64_t t, float lr, float wd);

/* loss_grad followed by adam_step on the network's own gradient buffer. */
svm_status svm_mlp_train_step(svm_mlp_t *m, const float *F, const int32_t *labels, int64_t n, const float *cw,
                              int64_t t, float lr, float wd, float *loss);

/* The warm start: alpha0_i = 0, C/2 or C for the predicted class (argmax of
 * the logits) of each of the n <= max_rows rows of F (FP64 output, n). */
svm_status svm_mlp_start_point(svm_mlp_t *m, const float *F, int64_t n, double C, double *alpha0);

/* Warm-started solve of the problem behind h (dense FP32, q = 128, n <= the
 * network's max_rows).  The network's logits give the working set J0: the
 * rows whose predicted probability of alpha_i = 0 is below 0.9 (the
 * complement of the predicted active set at the lower bound).  When J0 holds
 * at most n/2 rows of both classes, the SVM restricted to J0 is solved first
 * (cold, the same C and tolerance, on an internal handle over a gathered copy
 * of those rows: stream-ordered allocations, freed before returning) and its
 * solution, zero elsewhere, is alpha^0 of svm_ssnalm_solve(h, alpha0, res);
 * when J0 holds every support vector that solve stops at its first KKT test.
 * Otherwise the problem is solved cold.  If the warm-started solve ends with
 * SVM_ERR_NOT_CONVERGED or SVM_ERR_NUMERIC, the problem is solved again from
 * alpha^0 = 0 and that result is returned.  *used_warm (nullable) is 1 when
 * the returned result is the warm-started one.  Other problems return
 * SVM_ERR_UNSUPPORTED. */
svm_status svm_ssnalm_solve_mlp(svm_ssnalm_t *h, svm_mlp_t *m, svm_result *res, int32_t *used_warm);

/* Attach a trained warm-start network to the handle (the learned counterpart
 * of the paper's warm start from an approximate solve, Sec. 4.3).
 * mlp_weights: device pointer to SVM_MLP_NPARAM FP32 parameters in the layout
 * above; they are copied, so the caller's buffer may be freed afterwards.
 * Afterwards every svm_ssnalm_solve(h, NULL, res) of this handle runs as
 * svm_ssnalm_solve_mlp with the attached network, cold fallback included; a
 * solve given a non-NULL alpha0 still starts from alpha0, and
 * svm_ssnalm_solve_batch still starts every problem cold.  mlp_weights = NULL
 * detaches the network (cold starts again).  The handle owns the network and
 * its workspace (about 6 KB of device memory per sample: the hidden
 * activations of all n rows); svm_ssnalm_destroy frees it.  Stream-ordered on
 * the handle's stream.  Returns SVM_ERR_INVALID_ARG for a NULL handle,
 * SVM_ERR_UNSUPPORTED unless the handle's problem is dense FP32 with q = 128
 * (the network's input width), SVM_ERR_OOM / SVM_ERR_CUDA when the network
 * cannot be created (the handle is then left without a network). */
svm_status svm_ssnalm_set_warmstart_model(svm_ssnalm_t *h, const float *mlp_weights);

#ifdef __cplusplus
}
#endif

#endif /* SVM_MLP_H */
