/*
 * pjds_batch.h — batched pJDS products on one GPU:
 *   - pjds_spmm: one matrix, k right-hand sides (block product Y = A X);
 *   - pjds_batch_*: many matrices of uneven sizes in one persistent launch.
 *
 * Paper (arXiv:1112.5588): the product is the dominant step of iterative
 * solvers (Sect. 1.1) and is bandwidth bound (Eq. 1); reading the matrix once
 * for k vectors divides its bytes per flop by k, and one persistent launch
 * over many small matrices removes per-launch overhead and tail imbalance.
 * Conventions as in pjds.h (statuses, caller-owned device memory, streams).
 */
#ifndef PJDS_BATCH_H
#define PJDS_BATCH_H

#include <stddef.h>
#include <stdint.h>

#include "pjds.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Y = A X for k right-hand sides. X: n_cols x k, Y: n_rows x k, row-major
 * (element (r, c) at r*k + c), device memory of A's vector type (double for
 * PJDS_F64, float otherwise), 16-byte aligned. k: 1, or a multiple of 4 up to
 * 128 (float) / a multiple of 2 up to 64 (double). Each thread handles one
 * row and 16 or 32 bytes of its k columns (32 when that leaves at least two
 * threads per row, the rows are not widely spread in length and the launch
 * still has 2^19 threads), so the lanes of a row read each gathered row of X
 * as one contiguous segment. On block-structured matrices (pair_share >= 500,
 * at least 2^18 rows of 64 entries or more on average; see pjds_host) with
 * bf16 values and k a multiple of 8, or fp32 values and k = 8 or a multiple of
 * 8 from 64 on, each thread takes both rows of a pair of adjacent sorted rows
 * and 32 bytes of their columns, and one gathered segment of X serves both
 * rows where their columns agree. Column c of Y is
 * computed in the same order and with the same fused multiply-adds as
 * pjds_spmv with one thread per row on column c of X. Original basis (permute_cols = 0): row i of
 * the sorted matrix is written to row perm[i] of Y; permuted basis: to row i.
 */
int pjds_spmm(const pjds_dev *A, int32_t k, const void *X, void *Y, void *stream);

/*
 * Pattern product Y = S X for k >= 2 right-hand sides, S the sparsity pattern
 * of A (every stored entry taken as 1): the launch pjds_spmm makes, without
 * reading val, each column summed in order with plain additions. Its time is
 * a floor for pjds_spmm's on the same matrix and k: the gathered rows of X
 * (4 k or 8 k bytes per entry), the column stream and the stores of Y, the
 * gather ceiling the block product is measured against. Same arguments and
 * errors as pjds_spmm; k = 1 returns PJDS_EINVAL (use pjds_spmv_pattern).
 * The paper has no counterpart of this call.
 */
int pjds_spmm_pattern(const pjds_dev *A, int32_t k, const void *X, void *Y, void *stream);

/* Opaque host handle of a batch plan. */
typedef struct pjds_batch pjds_batch;

/*
 * Device bytes of the plan for these matrices: a work counter, one
 * descriptor per matrix and room for one entry per tile (an upper bound:
 * every tile holds at least 32 sorted rows).
 */
int pjds_batch_plan_bytes(int32_t n_mats, const pjds_dev *mats, size_t *bytes);

/*
 * Build a plan for y_m = A_m x_m, m < n_mats. mats[m] are device views of
 * pJDS matrices of one dtype (original or permuted basis each); xs[m], ys[m]
 * their device vectors. Each matrix is cut into tiles of sorted rows by the
 * length of the rows' block: 8 lanes per row from 256 entries, 4 from 64, 2
 * from 16 (tiles of 256 / lanes rows), else one thread for two adjacent rows
 * (tiles of 512 rows), or for four when the block has at most 2 entries and
 * val and col are 16-byte aligned (tiles of 1024 rows); one row per thread,
 * 256 rows, when val and col do not allow paired loads. The tiles are grouped by matrix,
 * the matrix with the most stored work per lane first, and inside a matrix
 * ordered by their stored work per lane, largest first, so that the CTAs
 * work on one or two matrices at a time (their x stays in L2: 18% faster
 * than one order over the tiles of all matrices on 64 Zipf matrices, where
 * every x competed for L2); the plan is copied into plan_dev (caller-owned
 * device memory of pjds_batch_plan_bytes). Reads each matrix's block lengths back
 * to the host once. *out receives a host handle (free with
 * pjds_batch_destroy). Errors: PJDS_EINVAL (mixed dtypes, sizes), ENOMEM,
 * ECUDA.
 */
int pjds_batch_create(int32_t n_mats, const pjds_dev *mats, const void *const *xs, void *const *ys,
                      void *plan_dev, size_t plan_bytes, pjds_batch **out, void *stream);

/*
 * pjds_batch_create with the lanes per row of each matrix given: lanes[m] in
 * {1, 2, 4, 8} cuts every tile of matrix m to 256 / lanes[m] rows with that
 * many lanes per row (the threads_per_row an autotuner chose for the matrix,
 * pjds_tune.h / pjds_mlp.h); 0 keeps the rule above. lanes = NULL is
 * pjds_batch_create. A row taken by T lanes gives the same bits as
 * pjds_spmv_cfg with threads_per_row = T. Errors as pjds_batch_create, and
 * PJDS_EINVAL for another lanes value.
 */
int pjds_batch_create_lanes(int32_t n_mats, const pjds_dev *mats, const void *const *xs, void *const *ys,
                            const int32_t *lanes, void *plan_dev, size_t plan_bytes, pjds_batch **out,
                            void *stream);

/*
 * pjds_batch_create with another block-length rule: a tile whose rows'
 * block holds at least min_len[2] entries gets 8 lanes per row, else 4 from
 * min_len[1], else 2 from min_len[0], else one thread per row (tiles of
 * 256 / lanes rows, two rows per thread below min_len[0] as above). The
 * built-in rule is {16, 64, 256}. Errors as
 * pjds_batch_create, and PJDS_EINVAL for a threshold below 1.
 */
int pjds_batch_create_rule(int32_t n_mats, const pjds_dev *mats, const void *const *xs, void *const *ys,
                           const int32_t *min_len, void *plan_dev, size_t plan_bytes, pjds_batch **out,
                           void *stream);

/*
 * Exhaustive autotuner of the batch's tiles (the f2 sweep applied to the
 * whole persistent launch): for each of n_rules rules (rules[3 r .. 3 r + 2],
 * as min_len above) builds the plan in plan_dev, runs it once, then times
 * `reps` runs with CUDA events on `stream` (flush, if not NULL, is
 * overwritten with cudaMemsetAsync before each timed run to empty L2) and
 * writes the median microseconds to us[r]; *best receives the fastest rule.
 * The vectors ys are overwritten. Errors as pjds_batch_create; PJDS_EINVAL
 * for reps outside [1, 1000].
 */
int pjds_batch_tune_rule(int32_t n_mats, const pjds_dev *mats, const void *const *xs, void *const *ys,
                         const int32_t *rules, int32_t n_rules, int32_t reps, void *plan_dev, size_t plan_bytes,
                         void *flush, size_t flush_bytes, double *us, int32_t *best, void *stream);

/*
 * Run the plan: reset the work counter and launch one persistent kernel
 * (one CTA per SM slot) whose CTAs take tiles from the counter until none is
 * left. use_graph = 1 records the two steps once into a CUDA graph kept in
 * the handle and replays it (the handle's first run with use_graph must not
 * happen while the stream is capturing).
 */
int pjds_batch_run(pjds_batch *h, int32_t use_graph, void *stream);

/*
 * The pattern products of the batch in one launch of the same plan (no graph):
 * y_m = S_m x_m, S_m the sparsity pattern of matrix m (every stored entry taken
 * as 1), with the batched kernel's instructions, registers and occupancy, its
 * values read from eight ones in L1 instead of each matrix's values. Its time
 * is a floor for pjds_batch_run's: the gathers, column streams and stores of
 * the whole batch, the gather ceiling it is measured against. Writes the same
 * ys as pjds_batch_run. The paper has no counterpart of this call.
 */
int pjds_batch_run_pattern(pjds_batch *h, void *stream);

/* Number of tiles and CTAs of the plan (for reporting). */
int pjds_batch_info(const pjds_batch *h, int32_t *n_tiles, int32_t *n_ctas);

int pjds_batch_destroy(pjds_batch *h);

#ifdef __cplusplus
}
#endif

#endif /* PJDS_BATCH_H */
