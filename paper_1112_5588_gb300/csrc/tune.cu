// Exhaustive autotuning of the pJDS product (include/pjds_tune.h).
//
// Candidates are grouped by (b, dtype) so that each pJDS conversion runs once
// on the host; the arrays are copied into the caller's device arena and every
// candidate of the group is timed with CUDA events on the caller's stream.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.h"
#include "pjds_tune.h"

namespace pjds {
namespace tune {

static inline size_t a256(size_t b) { return (b + 255) & ~(size_t)255; }

struct Shape {
  int64_t n_pad, n_blocks, n_max, n_stored;
};

// pJDS sizes for block size b from the row lengths alone: after the
// descending sort the first row of each block is its longest.
static Shape shape_for(int32_t n_rows, const int64_t *row_ptr, int32_t b) {
  int64_t max_len = 0;
  for (int32_t i = 0; i < n_rows; ++i) max_len = std::max(max_len, row_ptr[i + 1] - row_ptr[i]);
  std::vector<int64_t> count((size_t)max_len + 1, 0);
  for (int32_t i = 0; i < n_rows; ++i) ++count[(size_t)(row_ptr[i + 1] - row_ptr[i])];
  Shape s;
  s.n_pad = ((int64_t)n_rows + b - 1) / b * b;
  s.n_blocks = s.n_pad / b;
  s.n_max = n_rows > 0 ? max_len : 0;
  s.n_stored = 0;
  // walk the sorted lengths from the longest; row k of the sorted order starts block k / b
  int64_t k = 0;
  for (int64_t len = max_len; len >= 0 && k < n_rows; --len) {
    const int64_t c = count[(size_t)len];
    if (c == 0) continue;
    // rows k .. k+c-1 have length len; blocks whose first row falls here get length len
    const int64_t first_block = (k + b - 1) / b, last_row = k + c - 1;
    if (first_block * b <= last_row) s.n_stored += (last_row / b - first_block + 1) * b * len;
    k += c;
  }
  return s;
}

static size_t matrix_bytes(const Shape &s, int32_t n_rows, int32_t dtype) {
  return a256((size_t)n_rows * 4) + a256((size_t)s.n_blocks * 4) + a256((size_t)(s.n_max + 1) * 8) +
         a256((size_t)s.n_stored * 4) + a256((size_t)s.n_stored * value_bytes(dtype)) +
         a256((size_t)(s.n_pad / 32) * 4) + a256((size_t)(s.n_pad / 32) * 16);
}

static size_t arena_need(int32_t n_rows, int32_t n_cols, const int64_t *row_ptr, const pjds_candidate *c,
                         int32_t n) {
  size_t m = 0;
  for (int32_t i = 0; i < n; ++i) {
    if (c[i].b <= 0 || c[i].b % 32 || value_bytes(c[i].dtype) == 0) continue;
    m = std::max(m, matrix_bytes(shape_for(n_rows, row_ptr, c[i].b), n_rows, c[i].dtype));
  }
  return m + a256((size_t)n_cols * 8) + a256((size_t)n_rows * 8);
}

}  // namespace tune
}  // namespace pjds

using namespace pjds;
using namespace pjds::tune;

extern "C" int pjds_tune_arena_bytes(int32_t n_rows, int32_t n_cols, const int64_t *row_ptr,
                                     const pjds_candidate *cands, int32_t n_cands, size_t *bytes) {
  clear_error();
  if (n_rows < 0 || n_cols < 1 || !row_ptr || !cands || n_cands <= 0 || !bytes)
    return set_error(PJDS_EINVAL, "bad arguments");
  *bytes = arena_need(n_rows, n_cols, row_ptr, cands, n_cands);
  return PJDS_OK;
}

extern "C" int pjds_tune_default_space(int32_t dtype_mask, pjds_candidate *out, int32_t max_out, int32_t *n_out) {
  clear_error();
  if (!out || !n_out || max_out < 0) return set_error(PJDS_EINVAL, "bad arguments");
  int32_t n = 0;
  const int32_t bs[4] = {32, 64, 128, 256}, ts[4] = {1, 2, 4, 8}, os[2] = {-1, 1};
  auto add = [&](const pjds_candidate &c) {
    if (n < max_out) out[n] = c;
    ++n;
  };
  for (int32_t d = 0; d < 3; ++d) {
    if (!(dtype_mask & (1 << d))) continue;
    for (int32_t b : bs)
      for (int32_t t : ts)
        for (int32_t o : os) {
          pjds_candidate c;
          memset(&c, 0, sizeof(c));
          c.b = b;
          c.dtype = d;
          c.threads_per_row = t;
          c.tile_order = o;
          add(c);
        }
    for (int32_t b : bs) {
      pjds_candidate c;
      memset(&c, 0, sizeof(c));
      c.b = b;
      c.dtype = d;
      c.plan = 1;
      add(c);
    }
  }
  *n_out = std::min(n, max_out);
  return PJDS_OK;
}

extern "C" int pjds_tune_sweep(int32_t n_rows, int32_t n_cols, const int64_t *row_ptr, const int32_t *col_idx,
                               const double *val, const pjds_candidate *cands, int32_t n_cands, int32_t reps,
                               void *arena, size_t arena_bytes, void *flush, size_t flush_bytes,
                               pjds_tune_entry *out, int32_t *best, void *stream) {
  clear_error();
  if (!row_ptr || !cands || n_cands <= 0 || !out || !best || !arena || n_rows <= 0 || n_cols < 1)
    return set_error(PJDS_EINVAL, "bad arguments");
  if (reps < 1 || reps > 1000) return set_error(PJDS_EINVAL, "reps must be in [1, 1000]");
  if (arena_bytes < arena_need(n_rows, n_cols, row_ptr, cands, n_cands))
    return set_error(PJDS_EINVAL, "arena of %zu bytes is too small", arena_bytes);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  *best = -1;
  for (int32_t i = 0; i < n_cands; ++i) {
    memset(&out[i], 0, sizeof(out[i]));
    out[i].cand = cands[i];
    out[i].us = -1.0;
    out[i].status = PJDS_EINVAL;
  }
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  if (cudaEventCreate(&ev0) != cudaSuccess || cudaEventCreate(&ev1) != cudaSuccess) {
    if (ev0) cudaEventDestroy(ev0);
    return set_error(PJDS_ECUDA, "cudaEventCreate failed");
  }
  std::vector<char> done((size_t)n_cands, 0);
  int rc = PJDS_OK;
  for (int32_t g = 0; g < n_cands && rc == PJDS_OK; ++g) {
    if (done[g]) continue;
    const int32_t b = cands[g].b, dt = cands[g].dtype;
    pjds_host *h = nullptr;
    const int crc = pjds_create(n_rows, n_cols, row_ptr, col_idx, val, b, dt, 0, &h);
    if (crc != PJDS_OK) {
      for (int32_t i = g; i < n_cands; ++i)
        if (!done[i] && cands[i].b == b && cands[i].dtype == dt) {
          out[i].status = crc;
          done[i] = 1;
        }
      continue;
    }
    // lay the arrays out in the arena
    char *p = static_cast<char *>(arena);
    auto place = [&](const void *src, size_t bytes) -> void * {
      void *dst = p;
      p += a256(bytes);
      if (bytes) cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s);
      return dst;
    };
    pjds_dev d;
    memset(&d, 0, sizeof(d));
    d.n_rows = h->n_rows;
    d.n_cols = h->n_cols;
    d.n_pad = h->n_pad;
    d.b = h->b;
    d.n_blocks = h->n_blocks;
    d.n_max = h->n_max;
    d.nnz = h->nnz;
    d.n_stored = h->n_stored;
    d.dtype = h->dtype;
    d.permute_cols = 0;
    d.perm = static_cast<const int32_t *>(place(h->perm, (size_t)h->n_rows * 4));
    d.block_len = static_cast<const int32_t *>(place(h->block_len, (size_t)h->n_blocks * 4));
    d.row_len = nullptr;
    d.col_start = static_cast<const int64_t *>(place(h->col_start, (size_t)(h->n_max + 1) * 8));
    d.col = static_cast<const int32_t *>(place(h->col, (size_t)h->n_stored * 4));
    d.val = place(h->val, (size_t)h->n_stored * value_bytes(dt));
    d.tile_order = static_cast<const int32_t *>(place(h->tile_order, (size_t)(h->n_pad / 32) * 4));
    d.plan = static_cast<const int32_t *>(place(h->plan, (size_t)h->n_plan * 16));
    d.n_plan = h->n_plan;
    d.pair_share = h->pair_share;
    void *x = p;
    p += a256((size_t)n_cols * 8);
    void *y = p;
    cudaMemsetAsync(x, 0, (size_t)n_cols * vector_bytes(dt), s);
    cudaError_t e = cudaStreamSynchronize(s);
    const int64_t n_stored = h->n_stored;
    pjds_destroy(h);
    if (e != cudaSuccess) {
      rc = set_error(PJDS_ECUDA, "arena upload: %s", cudaGetErrorString(e));
      break;
    }
    for (int32_t i = g; i < n_cands && rc == PJDS_OK; ++i) {
      if (done[i] || cands[i].b != b || cands[i].dtype != dt) continue;
      done[i] = 1;
      pjds_launch in, res;
      memset(&in, 0, sizeof(in));
      in.staged = cands[i].staged;
      in.rows_per_thread = cands[i].rows_per_thread;
      in.threads_per_row = cands[i].threads_per_row;
      in.block_threads = cands[i].block_threads;
      in.unroll = cands[i].unroll;
      in.plan = cands[i].plan;
      in.tile_order = cands[i].plan == 1 ? 0 : cands[i].tile_order;
      const int r = pjds_spmv_resolve(&d, &in, &res);
      out[i].n_stored = n_stored;
      if (r != PJDS_OK) {
        out[i].status = r;
        continue;
      }
      out[i].cand.rows_per_thread = res.rows_per_thread;
      out[i].cand.threads_per_row = res.threads_per_row;
      out[i].cand.block_threads = res.block_threads;
      out[i].cand.unroll = res.unroll;
      out[i].cand.staged = res.staged;
      out[i].cand.plan = res.plan;
      out[i].cand.tile_order = res.plan == 1 ? 0 : res.tile_order;
      std::vector<float> t((size_t)reps);
      int lr = PJDS_OK;
      for (int w = 0; w < 2 && lr == PJDS_OK; ++w) lr = pjds_spmv_cfg(&d, x, y, &res, stream);
      for (int32_t k = 0; k < reps && lr == PJDS_OK; ++k) {
        if (flush && flush_bytes) cudaMemsetAsync(flush, k & 0xff, flush_bytes, s);
        cudaEventRecord(ev0, s);
        lr = pjds_spmv_cfg(&d, x, y, &res, stream);
        cudaEventRecord(ev1, s);
        e = cudaEventSynchronize(ev1);
        if (e != cudaSuccess) {
          lr = set_error(PJDS_ECUDA, "timing: %s", cudaGetErrorString(e));
          break;
        }
        cudaEventElapsedTime(&t[(size_t)k], ev0, ev1);
      }
      if (lr == PJDS_ECUDA) {
        rc = lr;
        break;
      }
      out[i].status = lr;
      if (lr == PJDS_OK) {
        std::sort(t.begin(), t.end());
        const float med = reps % 2 ? t[(size_t)reps / 2] : 0.5f * (t[(size_t)reps / 2 - 1] + t[(size_t)reps / 2]);
        out[i].us = 1e3 * (double)med;
      }
    }
  }
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  if (rc != PJDS_OK) return rc;
  double bt = 0.0;
  for (int32_t i = 0; i < n_cands; ++i)
    if (out[i].status == PJDS_OK && out[i].us >= 0.0 && (*best < 0 || out[i].us < bt)) {
      *best = i;
      bt = out[i].us;
    }
  clear_error();
  return PJDS_OK;
}
