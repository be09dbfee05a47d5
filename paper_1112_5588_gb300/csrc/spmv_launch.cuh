// Typed launchers: pick the kernel instance for (value type, index width,
// rows per thread, threads per row, scatter) and launch it on a stream.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "common.h"
#include "spmv_kernels.cuh"
#include "spmv_staged.cuh"
#include "tiles.cuh"

namespace pjds {

struct LaunchCfg {
  int rows_per_thread;  // R: 1, 2, 4
  int threads_per_row;  // T: 1, 2, 4, 8
  int block_threads;    // CTA size
  int unroll;           // U: jagged diagonals per chunk of the j-loop
  int staged;           // 1: bulk-copy staged persistent kernel (R = T = 1)
  int index64;          // 1: 64-bit element offsets regardless of size
  int tile_order;       // 1: tiles taken in A->tile_order
  int plan;             // 1: per-tile mapping of A->plan (the fields above do not apply)
  int pattern = 0;      // 1: the pattern product (values taken as 1, val not read)
};

// Launch-status helper: a launch error becomes PJDS_ECUDA with a message.
inline int check_launch(const char *what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(PJDS_ECUDA, "%s: %s", what, cudaGetErrorString(e));
  return PJDS_OK;
}

template <typename TV, typename TX, typename IDX, bool SC>
int launch_staged(const pjds_dev *A, const TX *x, TX *y, cudaStream_t s) {
  const TV *val = static_cast<const TV *>(A->val);
  const int n_tiles = (A->n_pad + dev::ST_TR - 1) / dev::ST_TR;
  if (n_tiles <= 0) return PJDS_OK;
  int device = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&device);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dev::pjds_staged_kernel<TV, TX, IDX, SC>,
                                                                dev::ST_TR + 32, 0);
  if (e != cudaSuccess) return set_error(PJDS_ECUDA, "occupancy: %s", cudaGetErrorString(e));
  int grid = sms * (per_sm > 0 ? per_sm : 1);
  if (grid > n_tiles) grid = n_tiles;
  dev::pjds_staged_kernel<TV, TX, IDX, SC><<<grid, dev::ST_TR + 32, 0, s>>>(
      val, A->col, A->col_start, A->block_len, A->perm, x, y, A->n_rows, A->n_pad, A->b);
  return check_launch("pjds_spmv staged launch");
}

template <typename TV, typename TX, typename IDX, bool SC>
int launch_pjds_idx(const pjds_dev *A, const TX *x, TX *y, const LaunchCfg &c, cudaStream_t s) {
  if (c.staged) return launch_staged<TV, TX, IDX, SC>(A, x, y, s);
  const TV *val = static_cast<const TV *>(A->val);
  if (c.pattern) {  // the pattern kernels read their values from eight ones
    const void *ones = nullptr;
    const cudaError_t e = dev::pattern_ones_address<TV>(&ones);
    if (e != cudaSuccess) return set_error(PJDS_ECUDA, "pattern values: %s", cudaGetErrorString(e));
    val = static_cast<const TV *>(ones);
  }
  const int R = c.rows_per_thread, T = c.threads_per_row, nt = c.block_threads;
  const int64_t work = T > 1 ? (int64_t)A->n_pad * T : ((int64_t)A->n_pad + R - 1) / R;
  const int64_t grid = (work + nt - 1) / nt;
  if (grid <= 0) return PJDS_OK;
  if (grid > 0x7fffffffLL) return set_error(PJDS_EOVERFLOW, "grid too large");
  const dim3 g((unsigned)grid), blk((unsigned)nt);
  const int32_t *order = c.tile_order ? A->tile_order : nullptr;
#ifdef PJDS_CHECKED
  dev::set_extents(dev::Extents{A->n_stored, A->n_cols, A->n_rows, A->n_blocks, A->n_max + 1}, s);
#endif
#define PJDS_ARGS val, A->col, A->col_start, A->block_len, A->perm, order, x, y, A->n_rows, A->n_pad, A->b
  const int U = c.unroll;
#define PJDS_ROWS(RR, UU) dev::pjds_rows_kernel<TV, TX, IDX, RR, UU, SC><<<g, blk, 0, s>>>(PJDS_ARGS)
#define PJDS_PAT(RR, UU) dev::pjds_rows_kernel<TV, TX, IDX, RR, UU, SC, true><<<g, blk, 0, s>>>(PJDS_ARGS)
#define PJDS_TPR(TT, UU) dev::pjds_tpr_kernel<TV, TX, IDX, TT, UU, SC><<<g, blk, 0, s>>>(PJDS_ARGS)
#define PJDS_TPR_PAT(TT, UU) dev::pjds_tpr_kernel<TV, TX, IDX, TT, UU, SC, true><<<g, blk, 0, s>>>(PJDS_ARGS)
  if (c.pattern && T > 1) {
    if (U != 2 && U != 4) return set_error(PJDS_EINVAL, "unroll must be 2 or 4 with threads_per_row > 1");
    switch (T) {
      case 2: if (U == 2) PJDS_TPR_PAT(2, 2); else PJDS_TPR_PAT(2, 4); break;
      case 4: if (U == 2) PJDS_TPR_PAT(4, 2); else PJDS_TPR_PAT(4, 4); break;
      case 8: if (U == 2) PJDS_TPR_PAT(8, 2); else PJDS_TPR_PAT(8, 4); break;
      default: return set_error(PJDS_EINVAL, "threads_per_row must be 1, 2, 4 or 8");
    }
  } else if (c.pattern) {
    if (R == 1 && U == 4) PJDS_PAT(1, 4);
    else if (R == 1 && U == 8) PJDS_PAT(1, 8);
    else if (R == 1 && U == 16) PJDS_PAT(1, 16);
    else if (R == 2 && U == 2) PJDS_PAT(2, 2);
    else if (R == 2 && U == 4) PJDS_PAT(2, 4);
    else if (R == 2 && U == 8) PJDS_PAT(2, 8);
    else if (R == 4 && U == 2) PJDS_PAT(4, 2);
    else if (R == 4 && U == 4) PJDS_PAT(4, 4);
    else return set_error(PJDS_EINVAL, "unroll %d is not available for %d rows per thread", U, R);
  } else if (T == 1 && R == 1) {
    if (U == 4) PJDS_ROWS(1, 4);
    else if (U == 8) PJDS_ROWS(1, 8);
    else if (U == 16) PJDS_ROWS(1, 16);
    else return set_error(PJDS_EINVAL, "unroll must be 4, 8 or 16 for one row per thread");
  } else if (T == 1 && R == 2) {
    if (U == 2) PJDS_ROWS(2, 2);
    else if (U == 4) PJDS_ROWS(2, 4);
    else if (U == 8) PJDS_ROWS(2, 8);
    else return set_error(PJDS_EINVAL, "unroll must be 2, 4 or 8 for two rows per thread");
  } else if (T == 1 && R == 4) {
    if (U == 2) PJDS_ROWS(4, 2);
    else if (U == 4) PJDS_ROWS(4, 4);
    else return set_error(PJDS_EINVAL, "unroll must be 2 or 4 for four rows per thread");
  } else if (T == 1) {
    return set_error(PJDS_EINVAL, "rows_per_thread must be 1, 2 or 4");
  } else {
    if (U != 2 && U != 4) return set_error(PJDS_EINVAL, "unroll must be 2 or 4 with threads_per_row > 1");
    switch (T) {
      case 2: if (U == 2) PJDS_TPR(2, 2); else PJDS_TPR(2, 4); break;
      case 4: if (U == 2) PJDS_TPR(4, 2); else PJDS_TPR(4, 4); break;
      case 8: if (U == 2) PJDS_TPR(8, 2); else PJDS_TPR(8, 4); break;
      default: return set_error(PJDS_EINVAL, "threads_per_row must be 1, 2, 4 or 8");
    }
  }
#undef PJDS_ROWS
#undef PJDS_PAT
#undef PJDS_TPR_PAT
#undef PJDS_TPR
#undef PJDS_ARGS
  return check_launch("pjds_spmv launch");
}

// Per-tile mapping: one CTA per plan entry (tiles.cuh).
template <typename TV, typename TX>
int launch_plan(const pjds_dev *A, const TX *x, TX *y, const LaunchCfg &c, cudaStream_t s) {
  if (A->n_plan <= 0 || A->n_rows == 0) return PJDS_OK;
  tiles::Desc d;
  d.val = A->val;
  d.col = A->col;
  d.col_start = A->col_start;
  d.block_len = A->block_len;
  d.perm = A->perm;
  d.x = x;
  d.y = y;
  d.n_rows = A->n_rows;
  d.b = A->b;
  d.scatter = A->permute_cols ? 0 : 1;
  d.idx64 = c.index64 || A->n_stored + A->n_pad >= 0x7fffffffLL ? 1 : 0;
  d.stored = A->n_stored;
  d.n_cols = A->n_cols;
  d.n_blocks = A->n_blocks;
  d.n_diag = A->n_max + 1;
  d.reserved = 0;
  const int4 *plan = reinterpret_cast<const int4 *>(A->plan);
  if (c.pattern) {  // the pattern kernel reads its values from eight ones
    const cudaError_t e = dev::pattern_ones_address<TV>(&d.val);
    if (e != cudaSuccess) return set_error(PJDS_ECUDA, "pattern values: %s", cudaGetErrorString(e));
    if constexpr (std::is_same<TV, double>::value)
      tiles::pjds_plan_kernel_f64<true><<<(unsigned)A->n_plan, tiles::BT, 0, s>>>(d, plan, A->n_pad);
    else
      tiles::pjds_plan_kernel<TV, TX, true><<<(unsigned)A->n_plan, tiles::BT, 0, s>>>(d, plan, A->n_pad);
    return check_launch("pjds_spmv_pattern plan launch");
  }
  if constexpr (std::is_same<TV, double>::value)
    tiles::pjds_plan_kernel_f64<><<<(unsigned)A->n_plan, tiles::BT, 0, s>>>(d, plan, A->n_pad);
  else
    tiles::pjds_plan_kernel<TV, TX><<<(unsigned)A->n_plan, tiles::BT, 0, s>>>(d, plan, A->n_pad);
  return check_launch("pjds_spmv plan launch");
}

template <typename TV, typename TX>
int launch_pjds(const pjds_dev *A, const void *x, void *y, const LaunchCfg &c, cudaStream_t s) {
  const TX *xx = static_cast<const TX *>(x);
  TX *yy = static_cast<TX *>(y);
  if (c.plan) return launch_plan<TV, TX>(A, xx, yy, c, s);
  const bool small = A->n_stored + A->n_pad < 0x7fffffffLL && !c.index64;
  const bool scatter = !A->permute_cols;
  if (small)
    return scatter ? launch_pjds_idx<TV, TX, int32_t, true>(A, xx, yy, c, s)
                   : launch_pjds_idx<TV, TX, int32_t, false>(A, xx, yy, c, s);
  return scatter ? launch_pjds_idx<TV, TX, int64_t, true>(A, xx, yy, c, s)
                 : launch_pjds_idx<TV, TX, int64_t, false>(A, xx, yy, c, s);
}

// ELLPACK-R baseline: 4 diagonals per round of the j-loop, 128-thread CTAs
// (the caller's nt). A GB300 sweep of U in 1, 2, 4, 8 x 128, 256, 512
// threads put this configuration first or within 1% of the first on the
// HMEp-like (6.2M rows, fp64), stencil (4.5M rows, fp64 / fp32) and
// block-dense (280k rows, fp32) matrices, 10% behind U = 8 on the HMEp-like
// matrix in fp32; U = 8 with 256 threads (52 registers in fp64, half the
// warps resident) was 11-24% slower in fp64.
template <typename TV, typename TX>
int launch_ellr(const ellr_dev *A, const void *x, void *y, int nt, cudaStream_t s) {
  const int64_t grid = ((int64_t)A->n_rows + nt - 1) / nt;
  if (grid <= 0) return PJDS_OK;
  const TV *val = static_cast<const TV *>(A->val);
#ifdef PJDS_CHECKED
  dev::set_extents(dev::Extents{A->n_stored, A->n_cols, A->n_rows, 0, 0}, s);
#endif
  const TX *xx = static_cast<const TX *>(x);
  TX *yy = static_cast<TX *>(y);
  if (A->n_stored < 0x7fffffffLL)
    dev::ellr_kernel<TV, TX, int32_t, 4>
        <<<(unsigned)grid, nt, 0, s>>>(val, A->col, A->row_max, xx, yy, A->n_rows, A->n_pad);
  else
    dev::ellr_kernel<TV, TX, int64_t, 4>
        <<<(unsigned)grid, nt, 0, s>>>(val, A->col, A->row_max, xx, yy, A->n_rows, A->n_pad);
  return check_launch("ellr_spmv launch");
}

template <typename TX>
int launch_permute(const int32_t *perm, const void *src, void *dst, int32_t n, bool inverse, cudaStream_t s) {
  const int nt = 256;
  const int64_t grid = ((int64_t)n + nt - 1) / nt;
  if (grid <= 0) return PJDS_OK;
  if (inverse)
    dev::unpermute_kernel<TX><<<(unsigned)grid, nt, 0, s>>>(perm, static_cast<const TX *>(src), static_cast<TX *>(dst), n);
  else
    dev::permute_kernel<TX><<<(unsigned)grid, nt, 0, s>>>(perm, static_cast<const TX *>(src), static_cast<TX *>(dst), n);
  return check_launch("pjds_permute launch");
}

// Per-dtype entry points, each compiled in its own translation unit.
int pjds_launch_f64(const pjds_dev *A, const void *x, void *y, const LaunchCfg &c, cudaStream_t s);
int pjds_launch_f32(const pjds_dev *A, const void *x, void *y, const LaunchCfg &c, cudaStream_t s);
int pjds_launch_bf16(const pjds_dev *A, const void *x, void *y, const LaunchCfg &c, cudaStream_t s);
int ellr_launch_f64(const ellr_dev *A, const void *x, void *y, int nt, cudaStream_t s);
int ellr_launch_f32(const ellr_dev *A, const void *x, void *y, int nt, cudaStream_t s);
int ellr_launch_bf16(const ellr_dev *A, const void *x, void *y, int nt, cudaStream_t s);
int staged_status_f64(int *out, bool clear, cudaStream_t s);
int staged_wait_selftest(int which, cudaStream_t s);
int staged_status_f32(int *out, bool clear, cudaStream_t s);
int staged_status_bf16(int *out, bool clear, cudaStream_t s);
// First out-of-extent access the checked build met in each translation unit
// (0: none); the normal build returns cudaErrorNotSupported.
int check_word_f64(unsigned long long *w, bool clear, cudaStream_t s);
int check_word_f32(unsigned long long *w, bool clear, cudaStream_t s);
int check_word_bf16(unsigned long long *w, bool clear, cudaStream_t s);
int check_word_batch(unsigned long long *w, bool clear, cudaStream_t s);

template <typename = void>
int check_word_here(unsigned long long *w, bool clear, cudaStream_t s) {
#ifdef PJDS_CHECKED
  return (int)dev::read_check_word(w, clear, s);
#else
  (void)clear;
  (void)s;
  *w = 0;
  return (int)cudaErrorNotSupported;
#endif
}

}  // namespace pjds
