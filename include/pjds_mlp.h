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
 * Model: 15 inputs -> 64 ReLU -> 64 ReLU -> 1, fp32, inputs and target
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

#define PJDS_MLP_IN 15
#define PJDS_MLP_HID 64
#define PJDS_MLP_FEATURES 8

/* Host-side model: weights (row-major [out][in]) and standardisation. */
typedef struct pjds_mlp {
  float w1[PJDS_MLP_HID * PJDS_MLP_IN], b1[PJDS_MLP_HID];
  float w2[PJDS_MLP_HID * PJDS_MLP_HID], b2[PJDS_MLP_HID];
  float w3[PJDS_MLP_HID], b3;
  float in_mean[PJDS_MLP_IN], in_std[PJDS_MLP_IN];
  float out_mean, out_std;
  /* the matrix features the model was trained on span [feat_lo, feat_hi]
   * (pjds_mlp_fit_range); feat_lo > feat_hi means no range is set */
  float feat_lo[PJDS_MLP_FEATURES], feat_hi[PJDS_MLP_FEATURES];
} pjds_mlp;

/* He-uniform weights from a counter-based generator, zero biases, identity
 * standardisation (mean 0, std 1), no feature range. */
int pjds_mlp_init(pjds_mlp *m, uint64_t seed);

/* Set the model's feature range from the features of its n training
 * matrices, feat[n][8] (host): per feature the smallest and largest value. */
int pjds_mlp_fit_range(pjds_mlp *m, const float *feat, int32_t n);

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
 * log2(threads per row) (0 for the per-tile mapping), a one-hot dtype (f64,
 * f32, bf16), 1 for the per-tile mapping (plan = 1) else 0, and 1 when the
 * tiles are taken in the traversal table (tile_order = 1) else 0. */
int pjds_tune_encode(const float feat[PJDS_MLP_FEATURES], const pjds_candidate *cands, int32_t n, float *out);

#define PJDS_PICK_MODEL 0 /* the model's smallest predicted time */
#define PJDS_PICK_SWEEP 1 /* the fastest candidate of the exhaustive sweep */

/* The configuration pjds_tune_pick chose. */
typedef struct pjds_pick {
  pjds_candidate cand; /* the chosen candidate as given in cands */
  int32_t index;       /* its index in cands */
  int32_t source;      /* PJDS_PICK_MODEL or PJDS_PICK_SWEEP */
  double us;           /* its predicted (model) or measured (sweep) kernel time, microseconds */
  int32_t n_outside;   /* features outside the model's range (> 0 sent the choice to the sweep) */
  int32_t reserved;
} pjds_pick;

/*
 * Choose the launch configuration of the product for a CRS matrix (host
 * arrays) among n_cands candidates (e.g. pjds_tune_default_space for the
 * caller's dtype). The features of the matrix are compared with the model's
 * range, widened by 2% of its width on each side: inside it, the model
 * predicts every candidate's time (CUDA inference kernel) and the smallest
 * prediction wins; outside it, or with model = NULL, pjds_tune_sweep times
 * every candidate (reps repetitions, L2 flushed through flush when given)
 * and the fastest wins. work: device workspace of at least
 * pjds_mlp_workspace_bytes(n_cands, 1) bytes (unused without a model).
 * arena: the sweep's device arena (pjds_tune_arena_bytes), needed only when
 * the sweep runs; NULL then returns PJDS_EINVAL. The result is written to
 * *out: make a pJDS matrix with cand.b and cand.dtype and launch it with
 * pjds_spmv_cfg and the candidate's fields. Synchronises the stream.
 * Paper: Sect. 2.1 (the row-length distribution decides the format's
 * benefit) and Sect. 4 (sliced ELLR-T, threads per row).
 */
int pjds_tune_pick(int32_t n_rows, int32_t n_cols, const int64_t *row_ptr, const int32_t *col_idx, const double *val,
                   const pjds_mlp *model, const pjds_candidate *cands, int32_t n_cands, int32_t reps, void *work,
                   size_t work_bytes, void *arena, size_t arena_bytes, void *flush, size_t flush_bytes,
                   pjds_pick *out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* PJDS_MLP_H */
