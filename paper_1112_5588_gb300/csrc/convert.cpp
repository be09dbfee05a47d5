// Host-side format conversion CRS -> pJDS and CRS -> ELLPACK-R (Sect. 2.1),
// plus the error state of the C ABI.
//
// pJDS steps (Sect. 2.1): count row lengths; sort rows by descending length
// (a counting sort over lengths, which keeps equal-length rows in their
// original order); pad each block of b sorted rows to the block's first (and
// therefore longest) row; lay the padded matrix out column by column, where
// column j spans the first b * #{blocks longer than j} sorted rows, so entry j
// of sorted row i lands at col_start[j] + i (the addressing of Listing 2).
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <limits>
#include <new>
#include <vector>

#include "common.h"
#include "plan.h"

namespace pjds {

static thread_local char g_msg[512];

int set_error(int code, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
  va_end(ap);
  return code;
}

void clear_error() { g_msg[0] = '\0'; }

// fp64 -> bfloat16 bits, round to nearest, ties to even, straight from the
// binary64 encoding (a single rounding; no detour through binary32).
static inline uint16_t bf16_bits(double d) {
  uint64_t u;
  memcpy(&u, &d, sizeof(u));
  const uint16_t sign = (uint16_t)((u >> 48) & 0x8000u);
  const uint64_t mag = u & 0x7FFFFFFFFFFFFFFFull;
  if (mag > 0x7FF0000000000000ull) return sign | 0x7FC0u;   // NaN
  if (mag == 0x7FF0000000000000ull) return sign | 0x7F80u;  // inf
  const int e = (int)(mag >> 52);
  const uint64_t frac = mag & ((1ull << 52) - 1);
  const int ebf = e - 1023 + 127;  // bf16 biased exponent of the unrounded value
  if (ebf >= 1) {
    const uint64_t keep = frac >> 45, rest = frac & ((1ull << 45) - 1), half = 1ull << 44;
    uint32_t r = ((uint32_t)ebf << 7) | (uint32_t)keep;
    if (rest > half || (rest == half && (keep & 1))) ++r;  // a carry moves into the exponent
    if (r >= 0x7F80u) return sign | 0x7F80u;               // rounded past the largest finite
    return sign | (uint16_t)r;
  }
  if (e == 0) return sign;  // binary64 subnormals are far below half of 2^-133
  // bf16 subnormal: value / 2^-133 = (2^52 + frac) * 2^(e - 942)
  const int s = 942 - e;  // >= 46 here
  if (s >= 64) return sign;
  const uint64_t m = (1ull << 52) | frac;
  const uint64_t keep = m >> s, rest = m & ((1ull << s) - 1), half = 1ull << (s - 1);
  uint32_t r = (uint32_t)keep;
  if (rest > half || (rest == half && (keep & 1))) ++r;
  return sign | (uint16_t)r;
}

static inline void store_value(void *dst, int64_t o, double v, int32_t dtype) {
  if (dtype == PJDS_F64)
    static_cast<double *>(dst)[o] = v;
  else if (dtype == PJDS_F32)
    static_cast<float *>(dst)[o] = (float)v;
  else
    static_cast<uint16_t *>(dst)[o] = bf16_bits(v);
}

static void clear_values(void *dst, int64_t o, int64_t n, int32_t dtype) {
  memset(static_cast<char *>(dst) + o * value_bytes(dtype), 0, (size_t)n * value_bytes(dtype));
}

// Shared CRS validation; fills len[i].
static int check_crs(int32_t n_rows, int32_t n_cols, const int64_t *row_ptr, const int32_t *col_idx,
                     const double *val, int32_t dtype, std::vector<int32_t> &len, bool entries = true) {
  if (n_rows < 0 || n_cols < 1) return set_error(PJDS_EINVAL, "n_rows must be >= 0 and n_cols >= 1");
  if (!row_ptr) return set_error(PJDS_EINVAL, "row_ptr is NULL");
  if (value_bytes(dtype) == 0) return set_error(PJDS_EINVAL, "unknown dtype %d", dtype);
  if (row_ptr[0] != 0) return set_error(PJDS_EINVAL, "row_ptr[0] must be 0");
  const int64_t nnz = row_ptr[n_rows];
  if (entries && nnz > 0 && (!col_idx || !val)) return set_error(PJDS_EINVAL, "col_idx/val is NULL");
  len.resize((size_t)n_rows);
  for (int32_t i = 0; i < n_rows; ++i) {
    const int64_t l = row_ptr[i + 1] - row_ptr[i];
    if (l < 0) return set_error(PJDS_EINVAL, "row_ptr decreases at row %d", i);
    if (l > std::numeric_limits<int32_t>::max()) return set_error(PJDS_EOVERFLOW, "row %d too long", i);
    len[i] = (int32_t)l;
  }
  if (!entries) return PJDS_OK;
  int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
  for (int64_t k = 0; k < nnz; ++k) bad |= (col_idx[k] < 0 || col_idx[k] >= n_cols);
  if (bad) return set_error(PJDS_EINVAL, "a column index is outside [0, n_cols)");
  return PJDS_OK;
}

static void free_pjds(pjds_host *h) {
  if (!h) return;
  free(h->perm);
  free(h->inv_perm);
  free(h->block_len);
  free(h->row_len);
  free(h->col_start);
  free(h->col);
  free(h->val);
  free(h->tile_order);
  free(h->plan);
  free(h);
}

static void free_ellr(ellr_host *h) {
  if (!h) return;
  free(h->row_max);
  free(h->col);
  free(h->val);
  free(h);
}

template <typename T>
static T *alloc_n(int64_t n) {
  return static_cast<T *>(malloc((size_t)std::max<int64_t>(n, 1) * sizeof(T)));
}

}  // namespace pjds

using namespace pjds;

extern "C" const char *pjds_last_error(void) { return g_msg; }

extern "C" int32_t pjds_version(void) { return 6; }

extern "C" void pjds_abi_sizes(int32_t out[5]) {
  out[0] = (int32_t)sizeof(pjds_host);
  out[1] = (int32_t)sizeof(pjds_dev);
  out[2] = (int32_t)sizeof(pjds_launch);
  out[3] = (int32_t)sizeof(ellr_host);
  out[4] = (int32_t)sizeof(ellr_dev);
}

// pjds_create (fill = true) and pjds_create_shape (fill = false: the
// structure from the row lengths alone, col and val left NULL).
static int create_impl(int32_t n_rows, int32_t n_cols, const int64_t *row_ptr, const int32_t *col_idx,
                       const double *val, int32_t b, int32_t dtype, int32_t permute_cols, bool fill,
                       pjds_host **out) {
  if (!out) return set_error(PJDS_EINVAL, "out is NULL");
  *out = nullptr;
  if (b <= 0 || b % 32 != 0) return set_error(PJDS_EINVAL, "b = %d is not a positive multiple of 32", b);
  if (permute_cols && n_rows != n_cols) return set_error(PJDS_EINVAL, "permute_cols needs a square matrix");
  std::vector<int32_t> len;
  int rc = check_crs(n_rows, n_cols, row_ptr, col_idx, val, dtype, len, fill);
  if (rc) return rc;

  const int64_t n_pad64 = ((int64_t)n_rows + b - 1) / b * b;
  if (n_pad64 > std::numeric_limits<int32_t>::max()) return set_error(PJDS_EOVERFLOW, "padded row count overflows");
  const int32_t n_pad = (int32_t)n_pad64, n_blocks = n_pad / b;

  pjds_host *h = static_cast<pjds_host *>(calloc(1, sizeof(pjds_host)));
  if (!h) return set_error(PJDS_ENOMEM, "out of host memory");
  h->n_rows = n_rows;
  h->n_cols = n_cols;
  h->n_pad = n_pad;
  h->b = b;
  h->n_blocks = n_blocks;
  h->nnz = row_ptr[n_rows];
  h->dtype = dtype;
  h->permute_cols = permute_cols ? 1 : 0;
  h->perm = alloc_n<int32_t>(n_rows);
  h->inv_perm = alloc_n<int32_t>(n_rows);
  h->block_len = alloc_n<int32_t>(n_blocks);
  h->row_len = alloc_n<int32_t>(n_pad);
  if (!h->perm || !h->inv_perm || !h->block_len || !h->row_len) {
    free_pjds(h);
    return set_error(PJDS_ENOMEM, "out of host memory");
  }

  // sort step: counting sort by length, longest first, stable
  int32_t max_len = 0;
  for (int32_t i = 0; i < n_rows; ++i) max_len = std::max(max_len, len[i]);
  std::vector<int64_t> slot((size_t)max_len + 2, 0);
  for (int32_t i = 0; i < n_rows; ++i) ++slot[(size_t)(max_len - len[i]) + 1];
  for (size_t l = 1; l < slot.size(); ++l) slot[l] += slot[l - 1];
  for (int32_t i = 0; i < n_rows; ++i) h->perm[slot[(size_t)(max_len - len[i])]++] = i;
  for (int32_t k = 0; k < n_rows; ++k) h->inv_perm[h->perm[k]] = k;
  for (int32_t k = 0; k < n_pad; ++k) h->row_len[k] = k < n_rows ? len[h->perm[k]] : 0;

  // pad step: a block's first sorted row is its longest
  for (int32_t k = 0; k < n_blocks; ++k) h->block_len[k] = h->row_len[(int64_t)k * b];
  h->n_max = n_blocks > 0 ? h->block_len[0] : 0;

  // jagged-diagonal offsets
  h->col_start = alloc_n<int64_t>((int64_t)h->n_max + 1);
  if (!h->col_start) {
    free_pjds(h);
    return set_error(PJDS_ENOMEM, "out of host memory");
  }
  int64_t blocks_longer = n_blocks;
  h->col_start[0] = 0;
  for (int32_t j = 0; j < h->n_max; ++j) {
    while (blocks_longer > 0 && h->block_len[blocks_longer - 1] <= j) --blocks_longer;
    h->col_start[j + 1] = h->col_start[j] + blocks_longer * b;
  }
  h->n_stored = h->col_start[h->n_max];
  if (h->n_stored > ((int64_t)1 << 62) / 8) {
    free_pjds(h);
    return set_error(PJDS_EOVERFLOW, "stored element count too large");
  }
  const int32_t *perm = h->perm;
  if (fill) {
    h->col = alloc_n<int32_t>(h->n_stored);
    h->val = malloc((size_t)std::max<int64_t>(h->n_stored, 1) * value_bytes(dtype));
    if (!h->col || !h->val) {
      free_pjds(h);
      return set_error(PJDS_ENOMEM, "out of host memory (%lld stored elements)", (long long)h->n_stored);
    }
  }

  // fill: sorted row i, entry j -> col_start[j] + i; padding up to the block length
  const int64_t *cs = h->col_start;
  const int32_t *inv = h->inv_perm, *rl = h->row_len, *bl = h->block_len;
  int32_t *col = h->col;
  void *v = h->val;
  const int permc = h->permute_cols;
#pragma omp parallel for schedule(static, 4096) if (fill)
  for (int64_t i = 0; i < (fill ? n_pad : 0); ++i) {
    const int32_t L = bl[i / b], li = rl[i];
    if (li > 0) {
      const int64_t src = row_ptr[perm[i]];
      for (int32_t j = 0; j < li; ++j) {
        const int64_t o = cs[j] + i;
        const int32_t c = col_idx[src + j];
        col[o] = permc ? inv[c] : c;
        store_value(v, o, val[src + j], dtype);
      }
    }
    for (int32_t j = li; j < L; ++j) {
      const int64_t o = cs[j] + i;
      col[o] = -1;
      clear_values(v, o, 1, dtype);
    }
  }

  // pair_share: per mille of the stored entries whose column equals the one
  // of the paired row at the same jagged diagonal (sorted rows 2k and 2k + 1,
  // the rows one thread takes with two rows per thread): high on
  // block-structured matrices, whose adjacent rows share their columns
  if (fill && h->nnz > 0) {
    int64_t matches = 0;
#pragma omp parallel for schedule(static, 2048) reduction(+ : matches)
    for (int64_t k = 0; k < (int64_t)n_rows / 2; ++k) {
      const int64_t a = row_ptr[perm[2 * k]], c = row_ptr[perm[2 * k + 1]];
      const int32_t m = std::min(rl[2 * k], rl[2 * k + 1]);
      for (int32_t j = 0; j < m; ++j) matches += col_idx[a + j] == col_idx[c + j];
    }
    h->pair_share = (int32_t)(2000.0 * (double)matches / (double)h->nnz);
  }

  // traversal order of the 32-row tiles: by the original index of each tile's
  // first row (tiles of padding rows only at the end), stable
  const int32_t n_tiles = n_pad / 32;
  h->tile_order = alloc_n<int32_t>(n_tiles);
  if (!h->tile_order) {
    free_pjds(h);
    return set_error(PJDS_ENOMEM, "out of host memory");
  }
  {
    std::vector<int32_t> key((size_t)n_tiles);
    for (int32_t t = 0; t < n_tiles; ++t) {
      const int64_t first = (int64_t)t * 32;
      key[(size_t)t] = first < n_rows ? perm[first] : std::numeric_limits<int32_t>::max();
      h->tile_order[t] = t;
    }
    std::stable_sort(h->tile_order, h->tile_order + n_tiles,
                     [&](int32_t a, int32_t c) { return key[(size_t)a] < key[(size_t)c]; });
  }

  // per-tile mapping: tiles of the default rule (pair and quad kinds assume
  // 16-byte aligned device arrays; the launcher checks), by work per lane,
  // largest first (stable). From 2^21 rows on, the tiles of two or four short
  // rows per thread then move behind the others, in the original order of
  // their first rows: the short rows in flight at any moment lie close
  // together in the original numbering, and their scattered y stores fill
  // whole sectors before the lines leave L2, which the vectors no longer fit
  // beside the streams (smaller matrices gain nothing from it)
  {
    std::vector<PlanTile> cut;
    plan_cut(n_rows, b, h->block_len, k_plan_rule, 0, true, true, cut);
    std::stable_sort(cut.begin(), cut.end(), [](const PlanTile &a, const PlanTile &c) { return a.cost > c.cost; });
    if (n_rows >= k_plan_first_row_order_min_rows) {
      const auto long_rows = [](const PlanTile &t) { return t.kind != KIND_PAIR && t.kind != KIND_QUAD; };
      const auto tail = std::stable_partition(cut.begin(), cut.end(), long_rows);
      std::stable_sort(tail, cut.end(),
                       [&](const PlanTile &a, const PlanTile &c) { return perm[a.row0] < perm[c.row0]; });
    }
    h->n_plan = (int32_t)cut.size();
    h->plan = alloc_n<int32_t>(4 * std::max<int64_t>((int64_t)cut.size(), 1));
    if (!h->plan) {
      free_pjds(h);
      return set_error(PJDS_ENOMEM, "out of host memory");
    }
    for (size_t t = 0; t < cut.size(); ++t) {
      h->plan[4 * t + 0] = 0;
      h->plan[4 * t + 1] = cut[t].row0;
      h->plan[4 * t + 2] = cut[t].rows;
      h->plan[4 * t + 3] = cut[t].kind;
    }
  }
  *out = h;
  return PJDS_OK;
}

extern "C" int pjds_create(int32_t n_rows, int32_t n_cols, const int64_t *row_ptr, const int32_t *col_idx,
                           const double *val, int32_t b, int32_t dtype, int32_t permute_cols, pjds_host **out) {
  clear_error();
  return create_impl(n_rows, n_cols, row_ptr, col_idx, val, b, dtype, permute_cols, true, out);
}

extern "C" int pjds_create_shape(int32_t n_rows, int32_t n_cols, const int64_t *row_ptr, int32_t b, int32_t dtype,
                                 pjds_host **out) {
  clear_error();
  return create_impl(n_rows, n_cols, row_ptr, nullptr, nullptr, b, dtype, 0, false, out);
}

extern "C" int pjds_destroy(pjds_host *h) {
  clear_error();
  free_pjds(h);
  return PJDS_OK;
}

extern "C" int ellr_create(int32_t n_rows, int32_t n_cols, const int64_t *row_ptr, const int32_t *col_idx,
                           const double *val, int32_t dtype, ellr_host **out) {
  clear_error();
  if (!out) return set_error(PJDS_EINVAL, "out is NULL");
  *out = nullptr;
  std::vector<int32_t> len;
  int rc = check_crs(n_rows, n_cols, row_ptr, col_idx, val, dtype, len);
  if (rc) return rc;
  const int64_t n_pad64 = ((int64_t)n_rows + 31) / 32 * 32;
  if (n_pad64 > std::numeric_limits<int32_t>::max()) return set_error(PJDS_EOVERFLOW, "padded row count overflows");
  int32_t n_max = 0;
  for (int32_t i = 0; i < n_rows; ++i) n_max = std::max(n_max, len[i]);
  const int64_t n_stored = n_pad64 * n_max;
  if (n_stored > ((int64_t)1 << 62) / 8) return set_error(PJDS_EOVERFLOW, "stored element count too large");
  ellr_host *h = static_cast<ellr_host *>(calloc(1, sizeof(ellr_host)));
  if (!h) return set_error(PJDS_ENOMEM, "out of host memory");
  h->n_rows = n_rows;
  h->n_cols = n_cols;
  h->n_pad = (int32_t)n_pad64;
  h->n_max = n_max;
  h->nnz = row_ptr[n_rows];
  h->n_stored = n_stored;
  h->dtype = dtype;
  h->row_max = alloc_n<int32_t>(n_pad64);
  h->col = alloc_n<int32_t>(n_stored);
  h->val = malloc((size_t)std::max<int64_t>(n_stored, 1) * value_bytes(dtype));
  if (!h->row_max || !h->col || !h->val) {
    free_ellr(h);
    return set_error(PJDS_ENOMEM, "out of host memory (%lld stored elements)", (long long)n_stored);
  }
  const int64_t n_pad = n_pad64;
  int32_t *rm = h->row_max, *col = h->col;
  void *v = h->val;
#pragma omp parallel for schedule(static, 4096)
  for (int64_t i = 0; i < n_pad; ++i) {
    const int32_t li = i < n_rows ? len[i] : 0;
    rm[i] = li;
    const int64_t src = i < n_rows ? row_ptr[i] : 0;
    for (int32_t j = 0; j < n_max; ++j) {
      const int64_t o = (int64_t)j * n_pad + i;
      if (j < li) {
        col[o] = col_idx[src + j];
        store_value(v, o, val[src + j], dtype);
      } else {
        col[o] = -1;
        clear_values(v, o, 1, dtype);
      }
    }
  }
  *out = h;
  return PJDS_OK;
}

extern "C" int ellr_destroy(ellr_host *h) {
  clear_error();
  free_ellr(h);
  return PJDS_OK;
}
