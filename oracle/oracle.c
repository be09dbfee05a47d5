/*
 * CPU oracle for pJDS / ELLPACK-R sparse matrix-vector multiplication.
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, obviously correct reference
 * that the CUDA path is checked against. Only the test suite, the smoke check
 * and the benchmark's CPU-baseline leg may load it. It shares no code, header
 * or table with the library under paper_1112_5588_gb300/, and the library never
 * calls it.
 *
 * Everything is computed in fp64 with plain loops. Compile with
 * -ffp-contract=off so that every product and every sum is rounded on its own
 * (no fused multiply-add); this is the textbook CRS evaluation order.
 *
 * Paper: Kreutzer, Hager, Wellein, Fehske, Basermann, Bishop, "Sparse
 * matrix-vector multiplication on GPGPU clusters: A new storage format and a
 * scalable implementation" (arXiv:1112.5588).
 *
 * Functions and the passages they follow:
 *   oracle_crs_spmv        y = A x in CRS order (Sect. 1.1 problem statement;
 *                          the CRS CPU baseline of Table 1).
 *   oracle_crs_absmv       |A| |x|, the scale of the forward error bound.
 *   oracle_crs_spmm        Y = A X for k right-hand sides (k independent
 *                          products, each in CRS order).
 *   oracle_pjds_shape/fill pJDS conversion, Sect. 2.1: sort rows by descending
 *                          length, pad each block of b consecutive rows to the
 *                          block's longest row, store the padded matrix column
 *                          by column with a col_start[] offset per column.
 *   oracle_ellr_shape/fill ELLPACK-R conversion, Sect. 2.1: rows shifted left
 *                          into an N x N_max rectangle stored column by column,
 *                          N padded to a multiple of the warp size (footnote),
 *                          plus the per-row length array rowmax[].
 *   oracle_pjds_listing    the pJDS kernel's loop (Listing 2) run sequentially
 *                          over converted arrays.
 *   oracle_ellr_listing    the ELLPACK-R kernel's loop (Listing 1), sequential.
 *   oracle_round_f32/bf16  the value a reduced-precision store holds
 *                          (Table 1 compares single and double precision).
 *
 * Readings where the paper is silent:
 *   - equal-length rows keep their original order (stable sort);
 *   - pad entries hold value +0.0 and column index -1 and are never used;
 *   - rows are padded up to a multiple of b with empty rows;
 *   - col_start[] has N_max+1 entries, the last one being the stored count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

void oracle_set_threads(int t) {
#ifdef _OPENMP
  if (t > 0) omp_set_num_threads(t);
#else
  (void)t;
#endif
}

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* y_i = sum_k val_k * x[col_k] over row i, k ascending (CRS order). */
void oracle_crs_spmv(int64_t n_rows, const int64_t *row_ptr, const int32_t *col, const double *val,
                     const double *x, double *y) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n_rows; ++i) {
    double s = 0.0;
    for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) s = s + val[k] * x[col[k]];
    y[i] = s;
  }
}

/* s_i = sum_k |val_k| * |x[col_k]|: the scale in |y - y_ref| <= gamma_n (|A||x|)_i. */
void oracle_crs_absmv(int64_t n_rows, const int64_t *row_ptr, const int32_t *col, const double *val,
                      const double *x, double *s) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n_rows; ++i) {
    double a = 0.0;
    for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) a = a + fabs(val[k]) * fabs(x[col[k]]);
    s[i] = a;
  }
}

/* Y = A X for k right-hand sides, X (n_cols x k) and Y (n_rows x k) row-major:
 * Y[i][c] = sum_k val_k * X[col_k][c], CRS order per (i, c) — the definition of
 * k independent products y_c = A x_c (block product of the batched solvers). */
void oracle_crs_spmm(int64_t n_rows, const int64_t *row_ptr, const int32_t *col, const double *val, int64_t k,
                     const double *X, double *Y) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n_rows; ++i)
    for (int64_t c = 0; c < k; ++c) {
      double s = 0.0;
      for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) s = s + val[e] * X[(int64_t)col[e] * k + c];
      Y[i * k + c] = s;
    }
}

/* Evaluate only the listed rows (for sampled checks at full size). */
void oracle_crs_spmv_rows(const int64_t *row_ptr, const int32_t *col, const double *val, const double *x,
                          const int64_t *rows, int64_t n_sel, double *y_sel, double *abs_sel) {
  for (int64_t r = 0; r < n_sel; ++r) {
    int64_t i = rows[r];
    double s = 0.0, a = 0.0;
    for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
      s = s + val[k] * x[col[k]];
      a = a + fabs(val[k]) * fabs(x[col[k]]);
    }
    y_sel[r] = s;
    abs_sel[r] = a;
  }
}

/* ------------------------------------------------------------------------- */
/* pJDS conversion (Sect. 2.1)                                                 */
/* ------------------------------------------------------------------------- */

typedef struct {
  int64_t len;
  int64_t row;
} len_row;

/* longest row first; equal lengths keep ascending original index */
static int cmp_len_desc(const void *a, const void *b) {
  const len_row *p = (const len_row *)a, *q = (const len_row *)b;
  if (p->len != q->len) return p->len > q->len ? -1 : 1;
  return p->row < q->row ? -1 : (p->row > q->row ? 1 : 0);
}

/* The "sort" step: perm[new] = old. Returns 0, or -1 on allocation failure. */
static int sorted_rows(int64_t n_rows, const int64_t *row_ptr, int32_t *perm) {
  len_row *lr = (len_row *)malloc((size_t)(n_rows > 0 ? n_rows : 1) * sizeof(len_row));
  if (!lr) return -1;
  for (int64_t i = 0; i < n_rows; ++i) {
    lr[i].len = row_ptr[i + 1] - row_ptr[i];
    lr[i].row = i;
  }
  qsort(lr, (size_t)n_rows, sizeof(len_row), cmp_len_desc);
  for (int64_t k = 0; k < n_rows; ++k) perm[k] = (int32_t)lr[k].row;
  free(lr);
  return 0;
}

/* Sizes of the pJDS arrays: out = {n_pad, n_blocks, n_max, n_stored}. */
int oracle_pjds_shape(int64_t n_rows, const int64_t *row_ptr, int64_t b, int64_t *out) {
  if (n_rows < 0 || b <= 0) return -1;
  int64_t n_pad = (n_rows + b - 1) / b * b, n_blocks = n_pad / b;
  int32_t *perm = (int32_t *)malloc((size_t)(n_rows > 0 ? n_rows : 1) * sizeof(int32_t));
  if (!perm || sorted_rows(n_rows, row_ptr, perm)) { free(perm); return -1; }
  int64_t n_max = 0, n_stored = 0;
  for (int64_t blk = 0; blk < n_blocks; ++blk) {
    int64_t m = 0;
    for (int64_t k = blk * b; k < (blk + 1) * b && k < n_rows; ++k) {
      int64_t l = row_ptr[perm[k] + 1] - row_ptr[perm[k]];
      if (l > m) m = l;
    }
    if (m > n_max) n_max = m;
    n_stored += m * b;
  }
  free(perm);
  out[0] = n_pad;
  out[1] = n_blocks;
  out[2] = n_max;
  out[3] = n_stored;
  return 0;
}

/*
 * Fill the pJDS arrays. Sizes from oracle_pjds_shape:
 *   perm[n_rows], inv_perm[n_rows], block_len[n_blocks], row_len[n_pad],
 *   col_start[n_max+1], col_out[n_stored], val_out[n_stored].
 * permute_cols = 1 renumbers columns into the permuted basis (col -> inv_perm[col];
 * square matrices only), so that the product can run in the permuted basis
 * (Sect. 2.1: the iterative scheme works on permuted vectors).
 * The padded matrix is written column by column: column j holds, in row order,
 * every (padded, sorted) row whose block is longer than j.
 */
int oracle_pjds_fill(int64_t n_rows, int64_t n_cols, const int64_t *row_ptr, const int32_t *col,
                     const double *val, int64_t b, int permute_cols, int32_t *perm, int32_t *inv_perm,
                     int32_t *block_len, int32_t *row_len, int64_t *col_start, int32_t *col_out,
                     double *val_out) {
  if (n_rows < 0 || b <= 0) return -1;
  if (permute_cols && n_rows != n_cols) return -1;
  int64_t n_pad = (n_rows + b - 1) / b * b, n_blocks = n_pad / b;
  if (sorted_rows(n_rows, row_ptr, perm)) return -1;
  for (int64_t k = 0; k < n_rows; ++k) inv_perm[perm[k]] = (int32_t)k;
  /* rows of the sorted matrix; padding rows are empty */
  for (int64_t k = 0; k < n_pad; ++k)
    row_len[k] = k < n_rows ? (int32_t)(row_ptr[perm[k] + 1] - row_ptr[perm[k]]) : 0;
  /* the "pad" step: each block padded to its longest row */
  int64_t n_max = 0;
  for (int64_t blk = 0; blk < n_blocks; ++blk) {
    int32_t m = 0;
    for (int64_t k = blk * b; k < (blk + 1) * b; ++k)
      if (row_len[k] > m) m = row_len[k];
    block_len[blk] = m;
    if (m > n_max) n_max = m;
  }
  /* column-major storage of the padded, sorted matrix */
  int64_t pos = 0;
  for (int64_t j = 0; j < n_max; ++j) {
    col_start[j] = pos;
    for (int64_t k = 0; k < n_pad; ++k) {
      if (block_len[k / b] <= j) continue;
      if (j < row_len[k]) {
        int64_t src = row_ptr[perm[k]] + j;
        col_out[pos] = permute_cols ? inv_perm[col[src]] : col[src];
        val_out[pos] = val[src];
      } else {
        col_out[pos] = -1;
        val_out[pos] = 0.0;
      }
      ++pos;
    }
  }
  col_start[n_max] = pos;
  return 0;
}

/* ------------------------------------------------------------------------- */
/* ELLPACK-R conversion (Sect. 2.1)                                            */
/* ------------------------------------------------------------------------- */

/* out = {n_pad, n_max, n_stored}; rows padded to a multiple of pad_to. */
int oracle_ellr_shape(int64_t n_rows, const int64_t *row_ptr, int64_t pad_to, int64_t *out) {
  if (n_rows < 0 || pad_to <= 0) return -1;
  int64_t n_pad = (n_rows + pad_to - 1) / pad_to * pad_to, n_max = 0;
  for (int64_t i = 0; i < n_rows; ++i)
    if (row_ptr[i + 1] - row_ptr[i] > n_max) n_max = row_ptr[i + 1] - row_ptr[i];
  out[0] = n_pad;
  out[1] = n_max;
  out[2] = n_pad * n_max;
  return 0;
}

/* rowmax[n_pad], col_out/val_out[n_pad * n_max], element (i, j) at j*n_pad + i. */
int oracle_ellr_fill(int64_t n_rows, const int64_t *row_ptr, const int32_t *col, const double *val,
                     int64_t pad_to, int32_t *rowmax, int32_t *col_out, double *val_out) {
  int64_t sh[3];
  if (oracle_ellr_shape(n_rows, row_ptr, pad_to, sh)) return -1;
  int64_t n_pad = sh[0], n_max = sh[1];
  for (int64_t i = 0; i < n_pad; ++i) rowmax[i] = i < n_rows ? (int32_t)(row_ptr[i + 1] - row_ptr[i]) : 0;
  for (int64_t j = 0; j < n_max; ++j)
    for (int64_t i = 0; i < n_pad; ++i) {
      int64_t o = j * n_pad + i;
      if (j < rowmax[i]) {
        col_out[o] = col[row_ptr[i] + j];
        val_out[o] = val[row_ptr[i] + j];
      } else {
        col_out[o] = -1;
        val_out[o] = 0.0;
      }
    }
  return 0;
}

/* ------------------------------------------------------------------------- */
/* The kernels' loops (Listings 1 and 2), run sequentially on the CPU          */
/* ------------------------------------------------------------------------- */

/* pJDS: c[i] += val[col_start[j] + i] * rhs[col_idx[col_start[j] + i]] for
 * j < rowmax[i]. With scatter = 1 the result of sorted row i goes to y[perm[i]]
 * (original basis); with scatter = 0 it stays at y[i] (permuted basis). */
void oracle_pjds_listing(int64_t n_rows, const int32_t *perm, const int32_t *row_len, const int64_t *col_start,
                         const int32_t *col, const double *val, const double *x, int scatter, double *y) {
  for (int64_t i = 0; i < n_rows; ++i) {
    double c = 0.0;
    for (int64_t j = 0; j < row_len[i]; ++j) {
      int64_t off = col_start[j];
      c = c + val[off + i] * x[col[off + i]];
    }
    y[scatter ? perm[i] : i] = c;
  }
}

/* ELLPACK-R: c[i] += val[j*N + i] * rhs[col_idx[j*N + i]] for j < rowmax[i]. */
void oracle_ellr_listing(int64_t n_rows, int64_t n_pad, const int32_t *rowmax, const int32_t *col,
                         const double *val, const double *x, double *y) {
  for (int64_t i = 0; i < n_rows; ++i) {
    double c = 0.0;
    for (int64_t j = 0; j < rowmax[i]; ++j) c = c + val[j * n_pad + i] * x[col[j * n_pad + i]];
    y[i] = c;
  }
}

/* ------------------------------------------------------------------------- */
/* Reduced-precision storage                                                   */
/* ------------------------------------------------------------------------- */

/* IEEE binary32 round-to-nearest-even of each value (C conversion). */
void oracle_round_f32(const double *in, double *out, int64_t n) {
  for (int64_t i = 0; i < n; ++i) out[i] = (double)(float)in[i];
}

/*
 * bfloat16 (1 sign, 8 exponent, 7 fraction bits; binary32's exponent range)
 * nearest value, ties to even. Definition: with |v| = m * 2^e, 0.5 <= m < 1,
 * bf16 keeps 8 significant bits, so the spacing near v is 2^(e-8); below the
 * normal range (2^-126) the spacing is fixed at 2^-133. The result is
 * rint(v / q) * q (rint rounds half to even), and values at or beyond
 * 2^128 - 2^119 (half a spacing above the largest finite bf16) become inf.
 */
void oracle_round_bf16(const double *in, double *out, int64_t n) {
  for (int64_t i = 0; i < n; ++i) {
    double v = in[i];
    if (v == 0.0 || isnan(v) || isinf(v)) { out[i] = v; continue; }
    int e;
    frexp(v, &e);
    int qe = e - 8;
    if (qe < -133) qe = -133;
    double r = rint(ldexp(v, -qe));
    double res = ldexp(r, qe);
    if (fabs(res) >= ldexp(1.0, 128)) res = v > 0 ? INFINITY : -INFINITY;
    out[i] = res;
  }
}
