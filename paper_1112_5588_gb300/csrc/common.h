// Internal declarations shared by the host converter and the CUDA entry points.
#pragma once

#include <stdint.h>

#include "pjds.h"

namespace pjds {

// Record a message for pjds_last_error() on this thread and return `code`.
int set_error(int code, const char *fmt, ...)
#if defined(__GNUC__)
    __attribute__((format(printf, 2, 3)))
#endif
    ;

// Clear the thread's message (called at the start of every entry point).
void clear_error();

// Bytes of one stored value of the given dtype (0 for an unknown dtype).
inline int value_bytes(int32_t dtype) {
  return dtype == PJDS_F64 ? 8 : (dtype == PJDS_F32 || dtype == PJDS_BF16) ? (dtype == PJDS_F32 ? 4 : 2) : 0;
}

// Bytes of one vector element (x, y) for the given dtype.
inline int vector_bytes(int32_t dtype) { return dtype == PJDS_F64 ? 8 : 4; }

// Automatic choice of the tile traversal table (pjds_launch.tile_order = 0):
// large matrices (n_rows >= 2^20) whose longest row is at most 4 times the
// mean row length.
inline bool auto_tile_order(const pjds_dev *A) {
  if (!A->tile_order || A->n_rows < (1 << 20)) return false;
  return (int64_t)A->n_max * A->n_rows <= 4 * A->nnz;
}

// Block-structured matrix on which one thread takes both rows of a pair
// (sorted rows 2k, 2k + 1): at least half the entries share the paired row's
// column (pair_share >= 500), at least 2^18 rows and 64 entries per row on
// average. The single product (fp32 / bf16) and the block product use it.
inline bool shared_pairs(const pjds_dev *A) {
  return A->pair_share >= 500 && A->n_rows >= (1 << 18) && A->nnz >= 64 * (int64_t)A->n_rows;
}

// Whether the per-tile mapping can run (a plan, 16-byte aligned plan, val and
// col: the tiles of two and four rows per thread use vector loads).
inline bool plan_usable(const pjds_dev *A) {
  return A->plan && A->n_plan > 0 && (uintptr_t)A->plan % 16 == 0 && (uintptr_t)A->val % 16 == 0 &&
         (uintptr_t)A->col % 16 == 0;
}

// Default use of the per-tile mapping: widely spread row lengths (the longest
// row above 4 times the mean), where no single threads-per-row count suits
// both the long and the short rows, from 2^16 rows (fp64), 2^17 (fp32) or
// 2^18 (bf16) on: below that, one tile per 32 to 1024 rows leaves too few
// CTAs and the uniform mapping's extra lanes win. Thresholds fitted on the
// timings of 2,000 Zipf matrices (10k-4M rows); on 200 held-out ones the
// default then runs at 0.870 / 0.941 / 0.980 of the best uniform mapping's
// time (geometric mean; the uniform rule alone 1.10 / 1.07 / 1.08). On the
// HMEp-like, stencil and block-dense matrices the uniform mapping with the
// tile order stays faster.
inline bool auto_plan(const pjds_dev *A) {
  const int32_t min_rows = A->dtype == PJDS_F64 ? (1 << 16) : A->dtype == PJDS_F32 ? (1 << 17) : (1 << 18);
  return plan_usable(A) && A->n_rows >= min_rows && (int64_t)A->n_max * A->n_rows > 4 * A->nnz;
}

}  // namespace pjds
