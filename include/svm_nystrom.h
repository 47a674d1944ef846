/*
 * svm_nystrom.h -- C ABI of the Nystrom front-end on GB300 (sm_103a): the
 * RBF-kernel C-SVC of arXiv 1910.01312, Sec. 4.3, turned into a linear
 * problem by a low-rank kernel approximation from r landmarks,
 *     K ~ K_nr (K_rr + s I)^{-1} K_nr',   K_ij = exp(-|x_i - c_j|^2 / (2 alpha)),
 * with s = 1e-3 in the paper's experiments.  The features Z = K_nr L^{-T},
 * L L' = K_rr + s I, make Z Z' that approximation exactly, so Z is passed as
 * the X of svm_ssnalm_create (q = r).  The paper chooses the landmarks by
 * k-means; svm_nystrom_kmeans runs Lloyd's iterations for them.
 *
 * Arithmetic: FP64 distances, kernel values, Cholesky factor and triangular
 * inverse (X is FP32 and widened exactly).  Both calls allocate their own
 * scratch with cudaMallocAsync on the stream and free it before returning;
 * both are stream-ordered and synchronise the stream before returning.
 * Pointers are device pointers unless marked host.  Errors: SVM_ERR_INVALID_ARG
 * for null pointers, sizes < 1, alpha <= 0, shift < 0 or non-finite scalars;
 * SVM_ERR_UNSUPPORTED for q > 1024, r > 1024 or n >= 2^31; SVM_ERR_NUMERIC
 * when K_rr + s I is not numerically positive definite; SVM_ERR_OOM;
 * SVM_ERR_CUDA.
 */
#ifndef SVM_NYSTROM_H
#define SVM_NYSTROM_H

#include <stdint.h>

#include "svm_ssnalm.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Lloyd's k-means on the rows of X (n x q, FP32, row-major).
 * centres (r x q, FP64, row-major): the initial centres on entry (for
 * example r distinct rows of X), the final centres on exit.  Each of the
 * iters >= 1 iterations assigns every row to the centre at the smallest FP64
 * squared Euclidean distance (ties to the lowest centre index), then replaces
 * each centre with the mean of its rows (FP64 sums in ascending row order);
 * a centre with no rows is kept.  labels (n int32, nullable): the assignment
 * of the last iteration.  objective (host, iters doubles, nullable): the sum
 * of squared distances to the assigned centres at each iteration's
 * assignment (non-increasing). */
svm_status svm_nystrom_kmeans(const float *X, int64_t n, int64_t q, double *centres, int64_t r, int32_t iters,
                              int32_t *labels, double *objective, void *stream);

/* Features Z (n x r, row-major) = K_nr L^{-T}, L L' = K_rr + shift I, for the
 * landmarks `centres` (r x q, FP64) and X (n x q, FP32): z_dtype SVM_F32
 * (Z float, ready for the mixed-precision solve when r % 4 == 0) or SVM_F64.
 * Z must be 16-byte aligned. */
svm_status svm_nystrom_features(const float *X, int64_t n, int64_t q, const double *centres, int64_t r,
                                double alpha, double shift, void *Z, int32_t z_dtype, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* SVM_NYSTROM_H */
