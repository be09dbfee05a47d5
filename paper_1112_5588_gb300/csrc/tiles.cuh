// Tiles of sorted pJDS rows, one CTA each, with the thread mapping of the
// plan entry (include/pjds.h, pjds_dev.plan): the routines shared by the
// per-tile mapping of the single product (pjds_plan_kernel, one CTA per plan
// entry) and the persistent batched launch (batch.cu). Every mapping sums a
// row's entries in the order of the other pJDS kernels with the same lanes
// per row, so a row gives the same bits here as there.
#pragma once

#include "spmv_kernels.cuh"

namespace pjds {
namespace tiles {

constexpr int BT = 256;  // threads per tile

// One matrix as the tile routines see it.
struct Desc {
  const void *val;
  const int32_t *col;
  const int64_t *col_start;
  const int32_t *block_len;
  const int32_t *perm;
  const void *x;
  void *y;
  int64_t stored;  // val, col elements
  int32_t n_rows, b, scatter, idx64;
  int32_t n_cols, n_blocks, n_diag, reserved;  // extents checked in the checked build (n_diag = n_max + 1)
};

// Store row i's sum (through perm in the original basis).
template <typename TX, typename TA>
__device__ __forceinline__ void store_row(const Desc &d, TX *y, int64_t i, TA v) {
  const int64_t r = d.scatter ? (int64_t)__ldcs(d.perm + i) : i;
  if (PJDS_IN(r, d.n_rows, dev::CHK_ROW)) y[r] = (TX)v;
}

// PAT (every routine below): the pattern product; d.val is then the address
// of eight ones (dev::pattern_ones_address), read at
// dev::pattern_slot(d.val + o) where the product reads d.val + o.
template <typename TV, typename TX, typename IDX, bool PAT = false>
__device__ __forceinline__ typename dev::Acc<TV>::T desc_row(const Desc &d, int64_t i) {
  using TA = typename dev::Acc<TV>::T;
  constexpr int U = 4;
  const TV *__restrict__ val = static_cast<const TV *>(d.val);
  const TX *__restrict__ x = static_cast<const TX *>(d.x);
  const int32_t L = PJDS_IN(i / d.b, d.n_blocks, dev::CHK_BLOCK) ? __ldg(d.block_len + (int32_t)(i / d.b)) : 0;
  TA acc = TA(0);
  for (int32_t j = 0; j < L; j += U) {
    int32_t c[U];
    TV v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      bool live = j + u < L && PJDS_IN(j + u, d.n_diag, dev::CHK_DIAG);
      IDX o = 0;
      if (live) {
        o = (IDX)__ldg(d.col_start + j + u) + (IDX)i;
        live = PJDS_IN(o, d.stored, dev::CHK_OFFSET);
      }
      if (live) {
        c[u] = __ldcs(d.col + o);
        v[u] = dev::ld_stream1(PAT ? val + dev::pattern_slot(val + o) : val + o);
      } else {
        c[u] = -1;
        v[u] = TV{};
      }
    }
    TX xv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) xv[u] = dev::gather_n(x, c[u], d.n_cols);
#pragma unroll
    for (int u = 0; u < U; ++u) acc = c[u] >= 0 ? dev::fma_acc(dev::to_acc(v[u]), (TA)xv[u], acc) : acc;
  }
  return acc;
}

// R adjacent sorted rows i .. i+R-1 (i a multiple of R: one block) with one
// vector load of col and of val per jagged diagonal, U diagonals per round;
// each row's arithmetic as in desc_row.
template <typename TV, typename TX, typename IDX, int R, int U, bool PAT = false>
__device__ __forceinline__ void desc_rows(const Desc &d, int64_t i, typename dev::Acc<TV>::T (&acc)[R]) {
  using TA = typename dev::Acc<TV>::T;
  const TV *__restrict__ val = static_cast<const TV *>(d.val);
  const TX *__restrict__ x = static_cast<const TX *>(d.x);
  const int32_t L = PJDS_IN(i / d.b, d.n_blocks, dev::CHK_BLOCK) ? __ldg(d.block_len + (int32_t)(i / d.b)) : 0;
#pragma unroll
  for (int r = 0; r < R; ++r) acc[r] = TA(0);
  for (int32_t j = 0; j < L; j += U) {
    int32_t c[U][R];
    TV v[U][R];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      bool live = j + u < L && PJDS_IN(j + u, d.n_diag, dev::CHK_DIAG);
      IDX o = 0;
      if (live) {
        o = (IDX)__ldg(d.col_start + j + u) + (IDX)i;
        live = PJDS_IN(o, d.stored, dev::CHK_OFFSET) && PJDS_IN((int64_t)o + (R - 1), d.stored, dev::CHK_OFFSET);
      }
      if (live) {
        dev::ld_stream<R>(d.col + o, c[u]);
        if constexpr (PAT)
          dev::ld_stream<R>(val + dev::pattern_slot(val + o), v[u]);
        else
          dev::ld_stream<R>(val + o, v[u]);
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) {
          c[u][r] = -1;
          v[u][r] = TV{};
        }
      }
    }
    TX xv[U][R];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int r = 0; r < R; ++r) xv[u][r] = dev::gather_n(x, c[u][r], d.n_cols);
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int r = 0; r < R; ++r)
        acc[r] = c[u][r] >= 0 ? dev::fma_acc(dev::to_acc(v[u][r]), (TA)xv[u][r], acc[r]) : acc[r];
  }
}

// R adjacent rows per thread from the tile's first row; rows past the tile
// or the matrix are not stored.
template <typename TV, typename TX, int R, int U, bool PAT = false>
__device__ __forceinline__ void rows_tile(const Desc &d, const int4 &tl, TX *y) {
  const int32_t k = R * (int32_t)threadIdx.x;
  const int64_t i = (int64_t)tl.y + k;
  if (k >= tl.z || i >= d.n_rows) return;
  typename dev::Acc<TV>::T acc[R];
  if (d.idx64)
    desc_rows<TV, TX, int64_t, R, U, PAT>(d, i, acc);
  else
    desc_rows<TV, TX, int32_t, R, U, PAT>(d, i, acc);
#pragma unroll
  for (int r = 0; r < R; ++r)
    if (k + r < tl.z && i + r < d.n_rows) store_row(d, y, i + r, acc[r]);
}

// LANES consecutive lanes share sorted row i: lane s takes jagged diagonals
// s, s + LANES, ...; the partial sums are added with shuffles (fixed tree).
template <typename TV, typename TX, typename IDX, int LANES, bool PAT = false>
__device__ __forceinline__ typename dev::Acc<TV>::T desc_row_lanes(const Desc &d, int64_t i, int32_t s, bool active) {
  using TA = typename dev::Acc<TV>::T;
  constexpr int U = 4;
  const TV *__restrict__ val = static_cast<const TV *>(d.val);
  const TX *__restrict__ x = static_cast<const TX *>(d.x);
  const int32_t L =
      active && PJDS_IN(i / d.b, d.n_blocks, dev::CHK_BLOCK) ? __ldg(d.block_len + (int32_t)(i / d.b)) : 0;
  TA acc = TA(0);
  for (int32_t j = s; j < L; j += U * LANES) {
    int32_t c[U];
    TV v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      bool live = j + u * LANES < L && PJDS_IN(j + u * LANES, d.n_diag, dev::CHK_DIAG);
      IDX o = 0;
      if (live) {
        o = (IDX)__ldg(d.col_start + j + u * LANES) + (IDX)i;
        live = PJDS_IN(o, d.stored, dev::CHK_OFFSET);
      }
      if (live) {
        c[u] = __ldcs(d.col + o);
        v[u] = dev::ld_stream1(PAT ? val + dev::pattern_slot(val + o) : val + o);
      } else {
        c[u] = -1;
        v[u] = TV{};
      }
    }
    TX xv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) xv[u] = dev::gather_n(x, c[u], d.n_cols);
#pragma unroll
    for (int u = 0; u < U; ++u) acc = c[u] >= 0 ? dev::fma_acc(dev::to_acc(v[u]), (TA)xv[u], acc) : acc;
  }
#pragma unroll
  for (int off = LANES / 2; off >= 1; off /= 2) acc += __shfl_down_sync(0xffffffffu, acc, off, LANES);
  return acc;
}

// A tile of BT / LANES rows with LANES lanes each; the whole CTA stays for the
// shuffles.
template <typename TV, typename TX, int LANES, bool PAT = false>
__device__ __forceinline__ void lanes_tile(const Desc &d, const int4 &tl, TX *y) {
  const int32_t r = threadIdx.x / LANES, s = threadIdx.x % LANES;
  const int64_t i = (int64_t)tl.y + r;
  const bool active = r < tl.z && i < d.n_rows;
  const auto acc = d.idx64 ? desc_row_lanes<TV, TX, int64_t, LANES, PAT>(d, i, s, active)
                           : desc_row_lanes<TV, TX, int32_t, LANES, PAT>(d, i, s, active);
  if (active && s == 0) store_row(d, y, i, acc);
}

// One plan entry tl = {matrix, first sorted row, rows, kind} of matrix d, by
// the whole CTA: kind 0 two rows per thread, 3 four rows per thread, 1 one
// row per thread, 2 / 4 / 8 lanes per row.
template <typename TV, typename TX, bool PAT = false>
__device__ __forceinline__ void run_tile(const Desc &d, const int4 &tl) {
  TX *y = static_cast<TX *>(d.y);
  if (tl.w == 0) {
    rows_tile<TV, TX, 2, 4, PAT>(d, tl, y);
  } else if (tl.w == 3) {  // blocks of at most 2 entries (PlanRule::quad_max_len)
    rows_tile<TV, TX, 4, 1, PAT>(d, tl, y);
  } else if (tl.w == 1) {
    const int64_t i = (int64_t)tl.y + threadIdx.x;
    if ((int32_t)threadIdx.x < tl.z && i < d.n_rows) {
      const auto acc = d.idx64 ? desc_row<TV, TX, int64_t, PAT>(d, i) : desc_row<TV, TX, int32_t, PAT>(d, i);
      store_row(d, y, i, acc);
    }
  } else if (tl.w == 2) {
    lanes_tile<TV, TX, 2, PAT>(d, tl, y);
  } else if (tl.w == 4) {
    lanes_tile<TV, TX, 4, PAT>(d, tl, y);
  } else {
    lanes_tile<TV, TX, 8, PAT>(d, tl, y);
  }
}

// An entry outside the matrix, of an unknown kind, with more rows than its
// kind maps, or of two or four rows per thread on a first row that is not a
// multiple of 2 or 4 (vector loads) does not describe a tile: it is skipped.
__device__ __forceinline__ bool plan_entry_ok(const int4 &tl, int32_t n_pad) {
  if (tl.y < 0 || tl.z <= 0 || (int64_t)tl.y + tl.z > n_pad) return false;
  switch (tl.w) {
    case 0: return tl.z <= 2 * BT && (tl.y & 1) == 0;
    case 3: return tl.z <= 4 * BT && (tl.y & 3) == 0;
    case 1: return tl.z <= BT;
    case 2: return tl.z <= BT / 2;
    case 4: return tl.z <= BT / 4;
    case 8: return tl.z <= BT / 8;
    default: return false;
  }
}

// Per-tile mapping of one product: CTA k takes plan entry k. The entries are
// ordered by their work per lane, largest first, so the block scheduler
// starts the long tiles first (on large matrices the short-row entries follow
// in the original order of their first rows). Any order gives the same
// results.
template <typename TV, typename TX, bool PAT = false>
__global__ void __launch_bounds__(BT) pjds_plan_kernel(const Desc d, const int4 *__restrict__ plan, int32_t n_pad) {
  const int4 tl = plan[blockIdx.x];
  if (!plan_entry_ok(tl, n_pad)) return;
  run_tile<TV, TX, PAT>(d, tl);
}

// fp64 values: bounded to six resident CTAs per SM (40 registers; unbounded
// the instance takes 42, allocated as 48: five CTAs per SM). fp32 and bf16
// stay unbounded (40 and 34 registers).
template <bool PAT = false>  // a template: instantiated only where it is launched
__global__ void __launch_bounds__(BT, 6)
    pjds_plan_kernel_f64(const Desc d, const int4 *__restrict__ plan, int32_t n_pad) {
  const int4 tl = plan[blockIdx.x];
  if (!plan_entry_ok(tl, n_pad)) return;
  run_tile<double, double, PAT>(d, tl);
}

}  // namespace tiles
}  // namespace pjds
