/*
 * pjds_tune.h — exhaustive autotuning of the pJDS product over its launch and
 * format parameters: block size b (Sect. 2.1: b "should be the warp size";
 * larger multiples trade padding for fewer blocks), threads per row (the
 * "sliced ELLR-T" idea the paper cites in Sect. 4) or rows per thread, CTA
 * size, unroll depth, and value precision (Table 1: single vs double).
 *
 * The sweep converts the CRS matrix once per (b, dtype) on the host, copies
 * the pJDS arrays into a caller-owned device arena, and times every candidate
 * with CUDA events on the given stream (median of `reps` launches, each after
 * an L2 flush written into the caller's flush buffer). Nothing is allocated on
 * the device by the library. Timings are of y = A x in the original basis with
 * x = 0 (the kernels' timing does not depend on the values).
 */
#ifndef PJDS_TUNE_H
#define PJDS_TUNE_H

#include <stddef.h>
#include <stdint.h>

#include "pjds.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pjds_candidate {
  int32_t b;               /* pJDS block size, a positive multiple of 32 */
  int32_t dtype;           /* PJDS_F64, PJDS_F32, PJDS_BF16 */
  int32_t rows_per_thread; /* as in pjds_launch (0 = default) */
  int32_t threads_per_row; /* as in pjds_launch (0 = default) */
  int32_t block_threads;   /* as in pjds_launch (0 = default) */
  int32_t unroll;          /* as in pjds_launch (0 = default) */
  int32_t staged;          /* as in pjds_launch */
  int32_t plan;            /* as in pjds_launch: 1 times the per-tile mapping of
                              the matrix's plan (the fields above then do not
                              apply); 0 with uniform fields set means -1 */
  int32_t tile_order;      /* as in pjds_launch: 0 automatic, 1 the traversal
                              table, -1 sorted order (uniform mappings) */
  int32_t reserved;        /* 0 */
} pjds_candidate;

typedef struct pjds_tune_entry {
  pjds_candidate cand;     /* with every 0 field resolved to the value launched */
  double us;               /* median kernel time in microseconds (< 0: not run) */
  int64_t n_stored;        /* stored entries of this b */
  int32_t status;          /* PJDS_OK, or the error that made the candidate invalid */
  int32_t reserved;
} pjds_tune_entry;

/*
 * Device arena bytes the sweep over `cands` needs for this CRS matrix: the
 * largest pJDS matrix among the candidates' (b, dtype) pairs (with its
 * traversal table and plan) plus x and y of the widest vector type, each
 * array 256-byte aligned.
 */
int pjds_tune_arena_bytes(int32_t n_rows, int32_t n_cols, const int64_t *row_ptr, const pjds_candidate *cands,
                          int32_t n_cands, size_t *bytes);

/*
 * Time every candidate (see above). out[n_cands] receives one entry per
 * candidate in the given order; *best the index of the fastest valid one
 * (-1 if none ran). reps in [1, 1000]. flush may be NULL (no L2 flush).
 * Errors: PJDS_EINVAL (arguments, arena too small), PJDS_ENOMEM, PJDS_ECUDA.
 * Invalid candidates (e.g. a vector load wider than the alignment allows)
 * are recorded with their status and skipped, not reported as errors.
 * Synchronises the stream.
 */
int pjds_tune_sweep(int32_t n_rows, int32_t n_cols, const int64_t *row_ptr, const int32_t *col_idx,
                    const double *val, const pjds_candidate *cands, int32_t n_cands, int32_t reps, void *arena,
                    size_t arena_bytes, void *flush, size_t flush_bytes, pjds_tune_entry *out, int32_t *best,
                    void *stream);

/*
 * The candidate space of the tuners, for each dtype in dtype_mask (bit d set
 * = include pjds_dtype d): b in {32, 64, 128, 256} x threads per row in
 * {1, 2, 4, 8} x tile order in {sorted (-1), traversal table (1)}, then the
 * per-tile mapping (plan = 1) for each b; 36 candidates per dtype, other
 * fields 0 (their defaults). Writes at most max_out entries and returns the
 * count in *n_out.
 */
int pjds_tune_default_space(int32_t dtype_mask, pjds_candidate *out, int32_t max_out, int32_t *n_out);

#ifdef __cplusplus
}
#endif

#endif /* PJDS_TUNE_H */
