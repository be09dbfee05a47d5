/*
 * pjds_mlp.h — learned choice of the pJDS launch configuration: a small
 * multilayer perceptron predicts the kernel time of a candidate (b, threads
 * per row, dtype) from features of the matrix's sparsity pattern, and the
 * candidate with the smallest prediction is used; the exhaustive sweep of
 * pjds_tune.h produces its training data and judges its regret.
 *
 * Paper (arXiv:1112.5588): the best storage and launch parameters depend on
 * the row-length distribution (Sect. 2.1, Fig. 3: the data reduction and the
 * speed of pJDS vs ELLPACK-R follow the histogram's width) and on RHS reuse
 * (Eq. 1, alpha); the features below summarise both.
 *
 * Model: 13 inputs -> 64 ReLU -> 64 ReLU -> 1, fp32, inputs and target
 * standardised with the statistics stored in the model. Training (full or
 * mini-batch Adam on the mean squared error of the standardised log time) and
 * inference run in hand-written CUDA kernels; gradients are summed per CTA
 * and then across CTAs in a fixed order, so training is reproducible.
 * Conventions as in pjds.h. The caller provides every device workspace.
 */
#ifndef PJDS_MLP_H
#define PJDS_MLP_H

#include <stddef.h>
#include <stdint.h>

#include "pjds.h"
#include "pjds_tune.h"

#ifdef __cplusplus
extern "C" {
#endif

#define PJDS_MLP_IN 13
#define PJDS_MLP_HID 64
#define PJDS_MLP_FEATURES 8

/* Host-side model: weights (row-major [out][in]) and standardisation. */
typedef struct pjds_mlp {
  float w1[PJDS_MLP_HID * PJDS_MLP_IN], b1[PJDS_MLP_HID];
  float w2[PJDS_MLP_HID * PJDS_MLP_HID], b2[PJDS_MLP_HID];
  float w3[PJDS_MLP_HID], b3;
  float in_mean[PJDS_MLP_IN], in_std[PJDS_MLP_IN];
  float out_mean, out_std;
} pjds_mlp;

/* He-uniform weights from a counter-based generator, zero biases, identity
 * standardisation (mean 0, std 1). */
int pjds_mlp_init(pjds_mlp *m, uint64_t seed);

/* Set the model's standardisation from n samples X[n][13], y[n] (host):
 * population mean and standard deviation per column (1 where it is 0). */
int pjds_mlp_fit_scaling(pjds_mlp *m, const float *X, const float *y, int32_t n);

/* Device workspace bytes for training on n samples with mini-batches of
 * `batch` (and for pjds_mlp_predict on up to n inputs). */
int pjds_mlp_workspace_bytes(int32_t n, int32_t batch, size_t *bytes);

/*
 * Train in place: X[n][13], y[n] on the host (raw, standardised on upload
 * with m's statistics), `epochs` passes of mini-batches of `batch` samples
 * (batch >= n: full batch, no shuffling; otherwise each epoch uses a
 * permutation drawn from a counter-based generator seeded with `seed`),
 * Adam with learning rate lr (beta1 0.9, beta2 0.999, eps 1e-8).
 * loss_hist: NULL or `epochs` floats receiving the mean squared error of the
 * standardised target after each epoch. Synchronises the stream.
 */
int pjds_mlp_train(pjds_mlp *m, const float *X, const float *y, int32_t n, int32_t epochs, int32_t batch, float lr,
                   uint64_t seed, float *loss_hist, void *work, size_t work_bytes, void *stream);

/* Predictions (unstandardised) for n host inputs X[n][13] into out[n] (host). */
int pjds_mlp_predict(const pjds_mlp *m, const float *X, int32_t n, float *out, void *work, size_t work_bytes,
                     void *stream);

/*
 * Features of a CRS pattern (host): [0] log10 N, [1] log10 nnz,
 * [2] log2(1 + mean row length), [3] coefficient of variation of the row
 * lengths, [4] their skewness, [5] log2(1 + longest row), [6] mean |col - row|
 * / N, [7] fraction of entries with |col - row| <= 64.
 */
int pjds_features(int32_t n_rows, int32_t n_cols, const int64_t *row_ptr, const int32_t *col_idx,
                  float out[PJDS_MLP_FEATURES]);

/* Model inputs for n candidates: the 8 features, then log2(b / 32),
 * log2(threads per row), and a one-hot dtype (f64, f32, bf16). */
int pjds_tune_encode(const float feat[PJDS_MLP_FEATURES], const pjds_candidate *cands, int32_t n, float *out);

#ifdef __cplusplus
}
#endif

#endif /* PJDS_MLP_H */
