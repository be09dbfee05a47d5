// Window mapping of the pJDS product (host side): the plan pjds_create stores
// with a matrix whose entries sit mostly on a few fixed offsets from the
// diagonal (a band structure: the HMEp-like matrix's diagonals 0, +-1, +-64,
// +-4096, a stencil's neighbour offsets).
//
// Sect. 2.1 fixes which rows share a block and the column-major layout of the
// jagged diagonals, not which rows a CTA works on together. With the tiles in
// the traversal order (tiles listed by the original index of their first
// row), window w is the run of tiles whose first row lies in the original
// rows [w W, (w + 1) W); one CTA takes the whole window. Its rows then cover
// that stretch of the original numbering densely, whatever their length, so
// the x entries at the band offsets of all its rows form a few short
// intervals: the CTA copies them into shared memory once and serves the band
// gathers from there, and it collects the window's y entries in shared
// memory and writes them as whole lines. Only the entries off the band go to
// L2 one gather at a time. The per-row arithmetic is unchanged.
#pragma once

#include <stdint.h>

#include <algorithm>
#include <vector>

namespace pjds {

constexpr int WIN_MAX_RANGES = 4;
constexpr int32_t WIN_MIN_ROWS = 1 << 16;   // smaller matrices keep the uniform mapping
constexpr int32_t WIN_MAX_OFFSET = 1 << 16; // band offsets looked for in [-2^16, 2^16]
constexpr int32_t WIN_MERGE_GAP = 512;      // heavy offsets closer than this share one interval
constexpr int64_t WIN_SMEM_BUDGET = 96 * 1024;  // shared memory of one window CTA (two per SM)

struct WindowPlan {
  int32_t W = 0;  // original rows per window
  int32_t n_ranges = 0;
  int32_t lo[WIN_MAX_RANGES] = {0, 0, 0, 0};   // interval k holds x[a + lo[k], a + lo[k] + len[k])
  int32_t len[WIN_MAX_RANGES] = {0, 0, 0, 0};  // for the window starting at original row a
  std::vector<int32_t> win_ptr;                // n_win + 1 positions in the tile order
};

// Shared-memory entries of the staged intervals, each started on an even
// entry (16-byte boundary for fp64); the window's y and its row flags follow.
inline int64_t window_staged_entries(const WindowPlan &p) {
  int64_t s = 0;
  for (int k = 0; k < p.n_ranges; ++k) s += (p.len[k] + 1) / 2 * 2;
  return s;
}

inline int64_t window_smem_bytes(const WindowPlan &p, int vec_bytes) {
  return (window_staged_entries(p) + p.W) * vec_bytes + ((int64_t)p.W + 31) / 32 * 4;
}

// Build the plan, or return false when the matrix has no band structure the
// window mapping can use. The rule: at least WIN_MIN_ROWS rows; the offsets
// col - row present in at least 1/8 of the rows ("heavy" offsets, searched
// within +-WIN_MAX_OFFSET) together hold at least a quarter of the entries;
// heavy offsets closer than WIN_MERGE_GAP form one interval, and the
// intervals holding the most entries are kept while the CTA's shared memory
// stays within WIN_SMEM_BUDGET (at most WIN_MAX_RANGES). W = 2048 rows with
// 8-byte vectors, 4096 with 4-byte ones; each interval reaches W / 4 rows
// past the window, for the rows of its last tiles that lie beyond it.
// tile_order lists the n_pad / 32 tiles by the original index of their first
// row (tiles of padding rows only at the end).
inline bool window_plan_build(int32_t n_rows, const int64_t *row_ptr, const int32_t *col_idx,
                              const int32_t *perm, const int32_t *tile_order, int32_t n_tiles, int vec_bytes,
                              WindowPlan &out) {
  out = WindowPlan();
  if (n_rows < WIN_MIN_ROWS) return false;
  const int64_t nnz = row_ptr[n_rows];
  const int32_t D = WIN_MAX_OFFSET, H = 2 * D + 1;
  std::vector<int64_t> cnt((size_t)H, 0);
#pragma omp parallel
  {
    std::vector<int64_t> mine((size_t)H, 0);
#pragma omp for schedule(static)
    for (int32_t i = 0; i < n_rows; ++i)
      for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
        const int64_t d = (int64_t)col_idx[k] - i;
        if (d >= -D && d <= D) ++mine[(size_t)(d + D)];
      }
#pragma omp critical
    for (int32_t h = 0; h < H; ++h) cnt[(size_t)h] += mine[(size_t)h];
  }
  struct Cluster {
    int32_t lo, hi;
    int64_t cover;
  };
  std::vector<Cluster> cl;
  int64_t cover = 0;
  for (int32_t h = 0; h < H; ++h) {
    if (cnt[(size_t)h] * 8 < n_rows) continue;
    const int32_t d = h - D;
    cover += cnt[(size_t)h];
    if (!cl.empty() && d - cl.back().hi <= WIN_MERGE_GAP) {
      cl.back().hi = d;
      cl.back().cover += cnt[(size_t)h];
    } else {
      cl.push_back(Cluster{d, d, cnt[(size_t)h]});
    }
  }
  if (cl.empty() || cover * 4 < nnz) return false;
  std::stable_sort(cl.begin(), cl.end(), [](const Cluster &a, const Cluster &b) { return a.cover > b.cover; });
  WindowPlan p;
  p.W = vec_bytes == 8 ? 2048 : 4096;
  const int32_t E = p.W / 4;
  for (const Cluster &c : cl) {
    if (p.n_ranges == WIN_MAX_RANGES) break;
    WindowPlan q = p;
    q.lo[q.n_ranges] = c.lo;
    q.len[q.n_ranges] = p.W + E + (c.hi - c.lo);
    ++q.n_ranges;
    if (window_smem_bytes(q, vec_bytes) > WIN_SMEM_BUDGET) continue;
    p = q;
  }
  if (p.n_ranges == 0) return false;
  // windows: runs of the tile order by first row
  const int64_t n_win = ((int64_t)n_rows + p.W - 1) / p.W;
  p.win_ptr.assign((size_t)n_win + 1, 0);
  int32_t t = 0;
  for (int64_t w = 0; w <= n_win; ++w) {
    const int64_t limit = std::min<int64_t>(w * p.W, n_rows);
    while (t < n_tiles) {
      const int64_t first = (int64_t)tile_order[t] * 32;
      if (first >= n_rows || perm[first] >= limit) break;
      ++t;
    }
    p.win_ptr[(size_t)w] = t;
  }
  out = std::move(p);
  return true;
}

}  // namespace pjds
