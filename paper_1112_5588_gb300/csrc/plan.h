// Tile plans: the sorted rows of a pJDS matrix cut into tiles of one CTA
// (256 threads) each, every tile with the thread mapping that suits the
// length of its rows' block. Used by the per-tile mapping of the single
// product (pjds_create stores a plan with the matrix) and by the batched
// launch (one plan over many matrices). Host code only.
#pragma once

#include <stdint.h>

#include <algorithm>
#include <vector>

namespace pjds {

constexpr int PLAN_BT = 256;                      // threads per tile
constexpr int PLAN_MIN_TILE_ROWS = PLAN_BT / 8;   // the smallest tile: 8 lanes per row

// Tile kinds (the w field of a plan entry): 2, 4, 8 lanes per row; 1 one row
// per thread; 0 two adjacent rows per thread; 3 four adjacent rows per thread.
enum : int32_t { KIND_PAIR = 0, KIND_ONE = 1, KIND_QUAD = 3 };

// Block-length rule: 8 lanes per row from min_len[2] entries, 4 from
// min_len[1], 2 from min_len[0]; below that rows go one, two (pair) or four
// (quad, blocks of at most quad_max_len entries) to a thread.
struct PlanRule {
  int32_t min_len[3];
  int32_t quad_max_len;
};

// The rule both plans use by default: on 64 Zipf matrices (9.8M rows, 61% of
// them with one entry) four rows per thread for blocks of at most 2 entries
// took the batched launch from 253 to 237 us in fp64 (241 -> 214 us fp32)
// against two rows per thread, with the same bits.
constexpr PlanRule k_plan_rule = {{16, 64, 256}, 2};
// rows from which pjds_create orders a product's short-row tiles by first original row
constexpr int32_t k_plan_first_row_order_min_rows = 1 << 21;

struct PlanTile {
  int32_t row0, rows, kind;
  int64_t cost;  // stored entries of the tile's rows over its lanes per row
};

inline int32_t plan_lanes(int32_t kind) { return kind == KIND_PAIR || kind == KIND_QUAD ? 1 : kind; }

// Cut the n_rows sorted rows (blocks of b rows, block_len[k] entries each)
// into tiles, appended to out in row order. fixed > 0 gives every tile that
// many lanes per row. pair / quad: the matrix's val and col allow the 2- and
// 4-row vector loads. A tile ends where its rows' blocks fall into another
// kind, so every row gets the mapping of its own block's length; tiles start
// on multiples of 32 rows.
inline void plan_cut(int32_t n_rows, int32_t b, const int32_t *block_len, const PlanRule &rule, int32_t fixed,
                     bool pair, bool quad, std::vector<PlanTile> &out) {
  auto lanes_of = [&](int64_t L) -> int32_t {
    return fixed ? fixed
                 : L >= rule.min_len[2] ? 8 : L >= rule.min_len[1] ? 4 : L >= rule.min_len[0] ? 2 : 1;
  };
  auto kind_of = [&](int64_t L) -> int32_t {
    const int32_t ln = lanes_of(L);
    if (ln != 1 || fixed || !pair) return ln;
    return quad && L <= rule.quad_max_len ? KIND_QUAD : KIND_PAIR;
  };
  for (int64_t t0 = 0; t0 < n_rows;) {
    const int32_t kind = kind_of(block_len[t0 / b]);
    const int32_t ln = plan_lanes(kind);
    const int32_t per_tile = kind == KIND_QUAD ? 4 * PLAN_BT : kind == KIND_PAIR ? 2 * PLAN_BT : PLAN_BT / ln;
    int64_t end = std::min<int64_t>(t0 + per_tile, n_rows);
    for (int64_t blk = t0 / b + 1; blk * b < end; ++blk)
      if (kind_of(block_len[blk]) != kind) {
        end = blk * b;
        break;
      }
    int64_t cost = 0;
    for (int64_t r = t0; r < end;) {
      const int64_t blk = r / b, e = std::min<int64_t>((blk + 1) * b, end);
      cost += (e - r) * (int64_t)block_len[blk];
      r = e;
    }
    out.push_back(PlanTile{(int32_t)t0, (int32_t)(end - t0), kind, cost / ln});
    t0 = end;
  }
}

// Upper bound of plan_cut's tile count: every tile but a matrix's last holds
// at least PLAN_MIN_TILE_ROWS rows.
inline int64_t plan_max_tiles(int32_t n_rows) {
  return ((int64_t)n_rows + PLAN_MIN_TILE_ROWS - 1) / PLAN_MIN_TILE_ROWS;
}

}  // namespace pjds
