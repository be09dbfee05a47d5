/*
 * Seeded synthetic sparse matrices in CRS form (row_ptr int64, col int32, val fp64).
 *
 * These generators produce the inputs that both the CUDA path and the CPU oracle
 * consume. They hold none of the pJDS method's arithmetic: no row sorting by
 * length, no padding, no products. Every random draw comes from a counter-based
 * hash of (seed, stream, index), so a matrix depends only on its parameters and
 * the seed, not on the thread count or the machine.
 *
 * Shapes follow the paper's test matrices (Sect. 1.3): an HMEp-like Holstein-
 * Hubbard structure (N = 6.2e6, ~15 nonzeros per row, long off-diagonals), an
 * FEM-like 27-point stencil, a DLR-like matrix of dense 4x4 blocks, and a small
 * banded matrix with uniform row lengths. The real matrices are not available.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* splitmix64 output function (Steele, Lea, Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014), used as a 64-bit mixer. */
static inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

static inline uint64_t rnd(uint64_t seed, uint64_t stream, uint64_t idx) {
  return mix64(mix64(seed * 0x9E3779B97F4A7C15ULL + stream) + idx * 0xD1B54A32D192ED03ULL);
}

/* uniform in [0, 1) with 53 random bits */
static inline double u01(uint64_t r) { return (double)(r >> 11) * 0x1.0p-53; }
/* uniform in [-1, 1) */
static inline double um11(uint64_t r) { return 2.0 * u01(r) - 1.0; }
/* uniform integer in [lo, hi] (hi - lo < 2^32; modulo bias below 2^-32) */
static inline int64_t uint_in(uint64_t r, int64_t lo, int64_t hi) {
  return lo + (int64_t)((r >> 16) % (uint64_t)(hi - lo + 1));
}

/* Result holder handed to Python: it asks for nnz, then copies out and frees. */
typedef struct synth_crs {
  int64_t n_rows, n_cols, nnz;
  int64_t *row_ptr;
  int32_t *col;
  double *val;
  double param; /* generator-specific recorded parameter (e.g. geometric p) */
} synth_crs;

static synth_crs *crs_alloc(int64_t n_rows, int64_t n_cols) {
  synth_crs *m = (synth_crs *)calloc(1, sizeof(synth_crs));
  if (!m) return NULL;
  m->n_rows = n_rows;
  m->n_cols = n_cols;
  m->row_ptr = (int64_t *)calloc((size_t)n_rows + 1, sizeof(int64_t));
  if (!m->row_ptr) { free(m); return NULL; }
  return m;
}

static int crs_alloc_entries(synth_crs *m) {
  m->nnz = m->row_ptr[m->n_rows];
  m->col = (int32_t *)malloc((size_t)(m->nnz > 0 ? m->nnz : 1) * sizeof(int32_t));
  m->val = (double *)malloc((size_t)(m->nnz > 0 ? m->nnz : 1) * sizeof(double));
  return (m->col && m->val) ? 0 : -1;
}

void synth_free(synth_crs *m) {
  if (!m) return;
  free(m->row_ptr);
  free(m->col);
  free(m->val);
  free(m);
}

int64_t synth_nnz(const synth_crs *m) { return m->nnz; }
int64_t synth_n_rows(const synth_crs *m) { return m->n_rows; }
int64_t synth_n_cols(const synth_crs *m) { return m->n_cols; }
double synth_param(const synth_crs *m) { return m->param; }

/* Copy out into caller-owned arrays (row_ptr: n_rows+1, col/val: nnz), then free. */
void synth_take(synth_crs *m, int64_t *row_ptr, int32_t *col, double *val) {
  memcpy(row_ptr, m->row_ptr, (size_t)(m->n_rows + 1) * sizeof(int64_t));
  if (m->nnz > 0) {
    memcpy(col, m->col, (size_t)m->nnz * sizeof(int32_t));
    memcpy(val, m->val, (size_t)m->nnz * sizeof(double));
  }
  synth_free(m);
}

static void prefix_sum_counts(int64_t *row_ptr, int64_t n) {
  /* row_ptr[i+1] holds the count of row i on entry */
  row_ptr[0] = 0;
  for (int64_t i = 0; i < n; ++i) row_ptr[i + 1] += row_ptr[i];
}

static void insertion_sort_i32(int32_t *a, int64_t n) {
  for (int64_t k = 1; k < n; ++k) {
    int32_t v = a[k];
    int64_t p = k - 1;
    while (p >= 0 && a[p] > v) { a[p + 1] = a[p]; --p; }
    a[p + 1] = v;
  }
}

/* sort ascending and drop repeats; returns the new length */
static int64_t sort_unique_i32(int32_t *a, int64_t n) {
  if (n <= 48) {
    insertion_sort_i32(a, n);
  } else {
    /* longer rows: simple heap sort keeps this dependency-free */
    for (int64_t s = n / 2 - 1; s >= 0; --s) {
      int64_t r = s;
      for (;;) {
        int64_t c = 2 * r + 1;
        if (c >= n) break;
        if (c + 1 < n && a[c + 1] > a[c]) ++c;
        if (a[r] >= a[c]) break;
        int32_t t = a[r]; a[r] = a[c]; a[c] = t; r = c;
      }
    }
    for (int64_t e = n - 1; e > 0; --e) {
      int32_t t = a[0]; a[0] = a[e]; a[e] = t;
      int64_t r = 0;
      for (;;) {
        int64_t c = 2 * r + 1;
        if (c >= e) break;
        if (c + 1 < e && a[c + 1] > a[c]) ++c;
        if (a[r] >= a[c]) break;
        int32_t t2 = a[r]; a[r] = a[c]; a[c] = t2; r = c;
      }
    }
  }
  int64_t w = 0;
  for (int64_t k = 0; k < n; ++k)
    if (w == 0 || a[k] != a[w - 1]) a[w++] = a[k];
  return w;
}

/* ------------------------------------------------------------------------- */
/* Banded matrix with uniform row lengths.                                    */
/* Row i holds the diagonal plus (m_i - 1) distinct columns drawn uniformly   */
/* from [i-hw, i+hw] ∩ [0, n), m_i uniform in [m_lo, m_hi] (capped at the     */
/* window size). Values uniform in [-1, 1).                                   */
/* ------------------------------------------------------------------------- */
synth_crs *synth_banded_uniform(int64_t n, int32_t m_lo, int32_t m_hi, int64_t hw, uint64_t seed) {
  if (n <= 0 || n > 2147483647LL || m_lo < 1 || m_hi < m_lo || hw < 0) return NULL;
  synth_crs *m = crs_alloc(n, n);
  if (!m) return NULL;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    int64_t lo = i - hw < 0 ? 0 : i - hw, hi = i + hw >= n ? n - 1 : i + hw;
    int64_t want = uint_in(rnd(seed, 1, (uint64_t)i), m_lo, m_hi);
    if (want > hi - lo + 1) want = hi - lo + 1;
    m->row_ptr[i + 1] = want;
  }
  prefix_sum_counts(m->row_ptr, n);
  if (crs_alloc_entries(m)) { synth_free(m); return NULL; }
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t i = 0; i < n; ++i) {
    int64_t lo = i - hw < 0 ? 0 : i - hw, hi = i + hw >= n ? n - 1 : i + hw;
    int64_t beg = m->row_ptr[i], want = m->row_ptr[i + 1] - beg;
    int32_t *c = m->col + beg;
    int64_t have = 0;
    c[have++] = (int32_t)i;
    for (uint64_t t = 0; have < want; ++t) {
      int32_t cand = (int32_t)uint_in(rnd(seed, 2, ((uint64_t)i << 20) + t), lo, hi);
      int dup = 0;
      for (int64_t k = 0; k < have; ++k)
        if (c[k] == cand) { dup = 1; break; }
      if (!dup) c[have++] = cand;
    }
    insertion_sort_i32(c, want);
    for (int64_t k = 0; k < want; ++k)
      m->val[beg + k] = um11(rnd(seed, 3, (uint64_t)i * (uint64_t)n + (uint64_t)c[k]));
  }
  return m;
}

/* ------------------------------------------------------------------------- */
/* HMEp-like (Holstein-Hubbard) matrix, Sect. 1.3.                            */
/* Fixed diagonals at offsets 0, ±off1, ±off2, ±off3 (clipped at the edges)   */
/* plus random off-band entries: row i draws m_i from a geometric law         */
/* truncated to [m_lo, m_hi], emits ceil(m_i/2) entries (i, j) with j uniform */
/* in |j - i| <= n/8, and mirrors each to (j, i), so the pattern is           */
/* symmetric. Repeats are merged. Values uniform in [-1, 1), drawn per (i,j). */
/* The geometric parameter p is found by bisection so that the expected       */
/* number of nonzeros per row is target_nzr (recorded in synth_param).        */
/* ------------------------------------------------------------------------- */
static double trunc_geom_mean_half(double p, int m_lo, int m_hi) {
  /* E[ceil(m/2)] for P(m) ∝ (1-p)^(m-m_lo), m in [m_lo, m_hi] */
  double z = 0.0, s = 0.0, w = 1.0;
  for (int m = m_lo; m <= m_hi; ++m) {
    z += w;
    s += w * (double)((m + 1) / 2);
    w *= (1.0 - p);
  }
  return s / z;
}

synth_crs *synth_hmep(int64_t n, int32_t off1, int32_t off2, int32_t off3, int32_t m_lo, int32_t m_hi,
                      double target_nzr, uint64_t seed) {
  if (n <= 0 || n > 2147483647LL || m_lo < 1 || m_hi < m_lo || m_hi - m_lo + 1 > 64) return NULL;
  const int64_t offs[7] = {-(int64_t)off3, -(int64_t)off2, -(int64_t)off1, 0, off1, off2, off3};
  /* random entries per row, expected: 2 * E[ceil(m/2)] (own + mirrored) */
  double want_half = (target_nzr - 7.0) / 2.0;
  double plo = 1e-9, phi = 0.999;
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (plo + phi);
    if (trunc_geom_mean_half(mid, m_lo, m_hi) > want_half) plo = mid; else phi = mid;
  }
  double p = 0.5 * (plo + phi);
  int nm = m_hi - m_lo + 1;
  double cdf[64];
  {
    double z = 0.0, w = 1.0;
    for (int k = 0; k < nm; ++k) { z += w; cdf[k] = z; w *= (1.0 - p); }
    for (int k = 0; k < nm; ++k) cdf[k] /= z;
  }
  int64_t hw = n / 8;
  /* per-row own random count k_i = ceil(m_i / 2) */
  int32_t *k_own = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  int64_t *cnt = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
  if (!k_own || !cnt) { free(k_own); free(cnt); return NULL; }
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double u = u01(rnd(seed, 11, (uint64_t)i));
    int g = 0;
    while (g < nm - 1 && u >= cdf[g]) ++g;
    int mi = m_lo + g;
    k_own[i] = (mi + 1) / 2;
  }
  /* candidate counts: band + own + mirrored */
  for (int64_t i = 0; i < n; ++i) {
    int64_t b = 0;
    for (int d = 0; d < 7; ++d) b += (i + offs[d] >= 0 && i + offs[d] < n);
    cnt[i + 1] += b + k_own[i];
  }
  for (int64_t i = 0; i < n; ++i) {
    int64_t lo = i - hw < 0 ? 0 : i - hw, hi = i + hw >= n ? n - 1 : i + hw;
    for (int t = 0; t < k_own[i]; ++t) {
      int64_t j = uint_in(rnd(seed, 12, ((uint64_t)i << 5) + (uint64_t)t), lo, hi);
      cnt[j + 1] += 1;
    }
  }
  prefix_sum_counts(cnt, n);
  int64_t ncand = cnt[n];
  int32_t *cand = (int32_t *)malloc((size_t)ncand * sizeof(int32_t));
  int64_t *fill = (int64_t *)malloc((size_t)n * sizeof(int64_t));
  if (!cand || !fill) { free(k_own); free(cnt); free(cand); free(fill); return NULL; }
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    int64_t w = cnt[i];
    for (int d = 0; d < 7; ++d)
      if (i + offs[d] >= 0 && i + offs[d] < n) cand[w++] = (int32_t)(i + offs[d]);
    int64_t lo = i - hw < 0 ? 0 : i - hw, hi = i + hw >= n ? n - 1 : i + hw;
    for (int t = 0; t < k_own[i]; ++t)
      cand[w++] = (int32_t)uint_in(rnd(seed, 12, ((uint64_t)i << 5) + (uint64_t)t), lo, hi);
    fill[i] = w;
  }
  for (int64_t i = 0; i < n; ++i) {
    int64_t lo = i - hw < 0 ? 0 : i - hw, hi = i + hw >= n ? n - 1 : i + hw;
    for (int t = 0; t < k_own[i]; ++t) {
      int64_t j = uint_in(rnd(seed, 12, ((uint64_t)i << 5) + (uint64_t)t), lo, hi);
      cand[fill[j]++] = (int32_t)i;
    }
  }
  free(fill);
  free(k_own);
  synth_crs *m = crs_alloc(n, n);
  if (!m) { free(cnt); free(cand); return NULL; }
  m->param = p;
#pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t i = 0; i < n; ++i) {
    int64_t u = sort_unique_i32(cand + cnt[i], cnt[i + 1] - cnt[i]);
    m->row_ptr[i + 1] = u;
  }
  prefix_sum_counts(m->row_ptr, n);
  if (crs_alloc_entries(m)) { free(cnt); free(cand); synth_free(m); return NULL; }
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    int64_t beg = m->row_ptr[i], len = m->row_ptr[i + 1] - beg;
    for (int64_t k = 0; k < len; ++k) {
      int32_t c = cand[cnt[i] + k];
      m->col[beg + k] = c;
      m->val[beg + k] = um11(rnd(seed, 13, (uint64_t)i * (uint64_t)n + (uint64_t)c));
    }
  }
  free(cnt);
  free(cand);
  return m;
}

/* ------------------------------------------------------------------------- */
/* FEM-like 27-point stencil on a g^3 grid. Each off-diagonal pair (i,j)/(j,i)*/
/* is dropped with probability p_drop (decided once per unordered pair, so the*/
/* pattern stays symmetric). Off-diagonal values uniform in [-1, 0), equal for*/
/* (i,j) and (j,i). Diagonal = sum |off-diagonal| + 1, so the matrix is       */
/* symmetric, strictly diagonally dominant, hence SPD.                        */
/* ------------------------------------------------------------------------- */
static inline int stencil_keep(uint64_t seed, uint64_t a, uint64_t b, uint64_t n, double p_drop) {
  uint64_t lo = a < b ? a : b, hi = a < b ? b : a;
  return u01(rnd(seed, 21, lo * n + hi)) >= p_drop;
}
static inline double stencil_val(uint64_t seed, uint64_t a, uint64_t b, uint64_t n) {
  uint64_t lo = a < b ? a : b, hi = a < b ? b : a;
  return u01(rnd(seed, 22, lo * n + hi)) - 1.0;
}

synth_crs *synth_stencil27(int64_t g, double p_drop, uint64_t seed) {
  if (g <= 0 || g * g * g > 2147483647LL) return NULL;
  int64_t n = g * g * g;
  synth_crs *m = crs_alloc(n, n);
  if (!m) return NULL;
  m->param = p_drop;
  for (int pass = 0; pass < 2; ++pass) {
    if (pass == 1) {
      prefix_sum_counts(m->row_ptr, n);
      if (crs_alloc_entries(m)) { synth_free(m); return NULL; }
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      int64_t z = i / (g * g), y = (i / g) % g, x = i % g;
      int64_t w = pass ? m->row_ptr[i] : 0, diag_at = -1;
      double dsum = 0.0;
      for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            int64_t zz = z + dz, yy = y + dy, xx = x + dx;
            if (zz < 0 || zz >= g || yy < 0 || yy >= g || xx < 0 || xx >= g) continue;
            int64_t j = (zz * g + yy) * g + xx;
            if (j == i) {
              if (pass) { diag_at = w; m->col[w] = (int32_t)i; }
              ++w;
              continue;
            }
            if (!stencil_keep(seed, (uint64_t)i, (uint64_t)j, (uint64_t)n, p_drop)) continue;
            if (pass) {
              double v = stencil_val(seed, (uint64_t)i, (uint64_t)j, (uint64_t)n);
              m->col[w] = (int32_t)j;
              m->val[w] = v;
              dsum += fabs(v);
            }
            ++w;
          }
      if (pass) m->val[diag_at] = dsum + 1.0;
      else m->row_ptr[i + 1] = w;
    }
  }
  return m;
}

/* ------------------------------------------------------------------------- */
/* DLR-like matrix of dense bs x bs blocks (Sect. 1.3, DLR1/DLR2): n_brow     */
/* block rows, each with nb distinct block columns: the diagonal block plus   */
/* (nb-1) drawn uniformly within ±frac*n_brow block rows. Nonsymmetric values */
/* uniform in [-1, 1).                                                        */
/* ------------------------------------------------------------------------- */
synth_crs *synth_block_dense(int64_t n_brow, int32_t bs, int32_t nb, double frac, uint64_t seed) {
  if (n_brow <= 0 || bs <= 0 || nb <= 0 || n_brow * bs > 2147483647LL) return NULL;
  int64_t n = n_brow * bs;
  int64_t hw = (int64_t)(frac * (double)n_brow);
  if (hw < 1) hw = 1;
  synth_crs *m = crs_alloc(n, n);
  if (!m) return NULL;
  int32_t *bcols = (int32_t *)malloc((size_t)n_brow * (size_t)nb * sizeof(int32_t));
  int32_t *bcnt = (int32_t *)malloc((size_t)n_brow * sizeof(int32_t));
  if (!bcols || !bcnt) { free(bcols); free(bcnt); synth_free(m); return NULL; }
#pragma omp parallel for schedule(static)
  for (int64_t r = 0; r < n_brow; ++r) {
    int64_t lo = r - hw < 0 ? 0 : r - hw, hi = r + hw >= n_brow ? n_brow - 1 : r + hw;
    int64_t want = nb;
    if (want > hi - lo + 1) want = hi - lo + 1;
    int32_t *c = bcols + r * nb;
    int64_t have = 0;
    c[have++] = (int32_t)r;
    for (uint64_t t = 0; have < want; ++t) {
      int32_t cand = (int32_t)uint_in(rnd(seed, 31, ((uint64_t)r << 20) + t), lo, hi);
      int dup = 0;
      for (int64_t k = 0; k < have; ++k)
        if (c[k] == cand) { dup = 1; break; }
      if (!dup) c[have++] = cand;
    }
    sort_unique_i32(c, want);
    bcnt[r] = (int32_t)want;
  }
  for (int64_t i = 0; i < n; ++i) m->row_ptr[i + 1] = (int64_t)bcnt[i / bs] * bs;
  prefix_sum_counts(m->row_ptr, n);
  if (crs_alloc_entries(m)) { free(bcols); free(bcnt); synth_free(m); return NULL; }
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    int64_t r = i / bs, w = m->row_ptr[i];
    for (int32_t k = 0; k < bcnt[r]; ++k)
      for (int32_t e = 0; e < bs; ++e) {
        int64_t c = (int64_t)bcols[r * nb + k] * bs + e;
        m->col[w] = (int32_t)c;
        m->val[w] = um11(rnd(seed, 32, (uint64_t)i * (uint64_t)n + (uint64_t)c));
        ++w;
      }
  }
  free(bcols);
  free(bcnt);
  return m;
}

/* ------------------------------------------------------------------------- */
/* Power-law row lengths: row i has len_i drawn from a Zipf law with exponent */
/* s on [1, len_max] (inverse CDF on the normalised weights k^-s), columns    */
/* distinct, either uniform over [0, n) (banded = 0) or within ±bw of i       */
/* (banded = 1). Values uniform in [-1, 1).                                   */
/* ------------------------------------------------------------------------- */
synth_crs *synth_zipf(int64_t n, double s, int32_t len_max, int32_t banded, int64_t bw, uint64_t seed) {
  if (n <= 0 || n > 2147483647LL || len_max < 1 || s <= 0.0) return NULL;
  if (len_max > n) len_max = (int32_t)n;
  double *cdf = (double *)malloc((size_t)len_max * sizeof(double));
  if (!cdf) return NULL;
  double z = 0.0;
  for (int32_t k = 1; k <= len_max; ++k) { z += pow((double)k, -s); cdf[k - 1] = z; }
  for (int32_t k = 0; k < len_max; ++k) cdf[k] /= z;
  synth_crs *m = crs_alloc(n, n);
  if (!m) { free(cdf); return NULL; }
  m->param = s;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double u = u01(rnd(seed, 41, (uint64_t)i));
    int32_t lo = 0, hi = len_max - 1;
    while (lo < hi) { int32_t mid = (lo + hi) / 2; if (u < cdf[mid]) hi = mid; else lo = mid + 1; }
    int64_t len = lo + 1;
    if (banded) {
      int64_t a = i - bw < 0 ? 0 : i - bw, b = i + bw >= n ? n - 1 : i + bw;
      if (len > b - a + 1) len = b - a + 1;
    }
    m->row_ptr[i + 1] = len;
  }
  free(cdf);
  prefix_sum_counts(m->row_ptr, n);
  if (crs_alloc_entries(m)) { synth_free(m); return NULL; }
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t i = 0; i < n; ++i) {
    int64_t beg = m->row_ptr[i], want = m->row_ptr[i + 1] - beg;
    int64_t a = 0, b = n - 1;
    if (banded) { a = i - bw < 0 ? 0 : i - bw; b = i + bw >= n ? n - 1 : i + bw; }
    int32_t *c = m->col + beg;
    int64_t have = 0;
    /* draw with replacement, merge repeats, redraw until the row is full */
    uint64_t t = 0;
    while (have < want) {
      for (int64_t k = have; k < want; ++k)
        c[k] = (int32_t)uint_in(rnd(seed, 42, ((uint64_t)i << 24) + t++), a, b);
      have = sort_unique_i32(c, want);
    }
    for (int64_t k = 0; k < want; ++k)
      m->val[beg + k] = um11(rnd(seed, 43, (uint64_t)i * (uint64_t)n + (uint64_t)c[k]));
  }
  return m;
}

/* Dense vector with entries uniform in [-1, 1). */
void synth_vector(double *x, int64_t n, uint64_t seed, uint64_t stream) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) x[i] = um11(rnd(seed, 100 + stream, (uint64_t)i));
}

int synth_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
