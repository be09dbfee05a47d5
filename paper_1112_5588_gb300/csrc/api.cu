// C entry points for the device products (pjds_spmv*, ellr_spmv, basis
// changes): argument checks, the default kernel configuration, dtype dispatch.
#include <stdint.h>

#include "common.h"
#include "spmv_launch.cuh"

namespace pjds {

static int check_pjds_dev(const pjds_dev *A, const void *x, const void *y, bool need_vectors = true) {
  if (!A) return set_error(PJDS_EINVAL, "A is NULL");
  if (value_bytes(A->dtype) == 0) return set_error(PJDS_EINVAL, "unknown dtype %d", A->dtype);
  if (A->n_rows < 0 || A->n_cols < 1 || A->b <= 0 || A->b % 32 != 0)
    return set_error(PJDS_EINVAL, "bad sizes (n_rows %d, n_cols %d, b %d)", A->n_rows, A->n_cols, A->b);
  if ((int64_t)A->n_pad != ((int64_t)A->n_rows + A->b - 1) / A->b * A->b || A->n_blocks != A->n_pad / A->b)
    return set_error(PJDS_EINVAL, "n_pad/n_blocks inconsistent with n_rows and b");
  if (need_vectors && A->n_rows > 0 && (!x || !y)) return set_error(PJDS_EINVAL, "x or y is NULL");
  if (A->n_stored > 0 && (!A->val || !A->col || !A->col_start || !A->block_len))
    return set_error(PJDS_EINVAL, "a matrix array is NULL");
  if (A->n_rows > 0 && !A->permute_cols && !A->perm) return set_error(PJDS_EINVAL, "perm is NULL");
  if (A->permute_cols && A->n_rows != A->n_cols) return set_error(PJDS_EINVAL, "permuted basis needs a square matrix");
  // a plan holds at most one tile per 32 rows
  if (A->plan && (A->n_plan < 0 || A->n_plan > A->n_pad / 32))
    return set_error(PJDS_EINVAL, "n_plan %d outside [0, %d]", A->n_plan, A->n_pad / 32);
  return PJDS_OK;
}

static int dispatch_pjds(const pjds_dev *A, const void *x, void *y, const LaunchCfg &c, cudaStream_t s) {
  if (A->n_rows == 0) return PJDS_OK;
  if (A->n_stored == 0) {
    // no stored entries: every row sum is zero
    cudaError_t e = cudaMemsetAsync(y, 0, (size_t)A->n_rows * vector_bytes(A->dtype), s);
    return e == cudaSuccess ? PJDS_OK : set_error(PJDS_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
  }
  switch (A->dtype) {
    case PJDS_F64: return pjds_launch_f64(A, x, y, c, s);
    case PJDS_F32: return pjds_launch_f32(A, x, y, c, s);
    default: return pjds_launch_bf16(A, x, y, c, s);
  }
}

static int check_cfg(const pjds_dev *A, LaunchCfg &c) {
  const int R = c.rows_per_thread, T = c.threads_per_row;
  if (R != 1 && R != 2 && R != 4) return set_error(PJDS_EINVAL, "rows_per_thread must be 1, 2 or 4");
  if (T != 1 && T != 2 && T != 4 && T != 8) return set_error(PJDS_EINVAL, "threads_per_row must be 1, 2, 4 or 8");
  if (R > 1 && T > 1) return set_error(PJDS_EINVAL, "rows_per_thread > 1 needs threads_per_row = 1");
  if (c.staged) {
    c.tile_order = 0;
    if (R != 1 || T != 1) return set_error(PJDS_EINVAL, "the staged kernel runs one thread per row");
    if (((uintptr_t)A->val | (uintptr_t)A->col) & 15)
      return set_error(PJDS_EINVAL, "the staged kernel needs 16-byte aligned val and col");
  }
  if (c.unroll == 0) c.unroll = T > 1 ? 4 : (R == 1 ? (A->dtype == PJDS_F32 ? 8 : 4) : (R == 2 ? 4 : 2));
  const int U = c.unroll;
  const bool u_ok = T > 1 ? (U == 2 || U == 4)
                          : R == 1 ? (U == 4 || U == 8 || U == 16) : R == 2 ? (U == 2 || U == 4 || U == 8) : (U == 2 || U == 4);
  if (!u_ok) return set_error(PJDS_EINVAL, "unroll %d is not available for rows_per_thread %d, threads_per_row %d", U, R, T);
  if (c.block_threads < 32 || c.block_threads > 512 || c.block_threads % 32)
    return set_error(PJDS_EINVAL, "block_threads must be a multiple of 32 in [32, 512]");
  if (R > 1) {
    const uintptr_t va = (uintptr_t)A->val, ca = (uintptr_t)A->col;
    const int vb = value_bytes(A->dtype) * R, need_v = vb < 16 ? vb : 16, need_c = 4 * R < 16 ? 4 * R : 16;
    if (va % need_v || ca % need_c)
      return set_error(PJDS_EINVAL, "val/col not aligned for %d-row vector loads", R);
  }
  return PJDS_OK;
}

// Default mapping: T threads per row, T in 1, 2, 4, 8. A thread runs its
// row as a chain of about len / (T U) dependent rounds (a col load, then the
// x gather it addresses), while the whole product streams about
// nnz * (value + index bytes) from HBM; T grows until the longest row's chain
// fits under that stream time. With ratio = n_max * 2^20 / (nnz * entry
// bytes): T = 1 below 2, 2 below 8, 4 below 64, else 8; then T doubles (up
// to 8) while n_rows * T < 2^17 threads. Thresholds fitted to an exhaustive
// GB300 timing of T on 2,000 Zipf matrices (10k to 4M rows) and 100 more of
// 4M to 20M rows; on 200 held-out matrices the time over the best T is 8.2%
// / 5.2% / 4.9% (fp64 / fp32 / bf16; 17.5% / 15.5% / 13.9% with the earlier
// rule, T from n_rows * T >= 2^19 or 2^20 threads alone), and 1.9% over 45
// uniform-length cases (stencil, banded, block-dense and HMEp-like, 8k to
// 1M rows; 9.9% before). With one thread per row, fp32 / bf16 values take
// two adjacent rows per thread (one 8- or 4-byte load per jagged diagonal)
// from 2^21 rows on, when val and col are aligned for it, and every dtype
// runs 256-thread CTAs: on the 27-point stencil (4.5M rows) bf16 162 -> 136
// us, fp32 168 -> 160 us; on the HMEp-like matrix (6.2M rows) fp64 289 -> 283 us.
// Pairs of rows also from 2^18 rows on when the paired rows share their
// columns (pair_share >= 500: block-structured matrices) and rows hold 64
// entries or more on average: the two rows' gathers of one jagged diagonal
// then read the same x sector. Measured on block-dense matrices of 4x4 blocks
// (64 and 144 entries per row, 280k to 1.1M rows) fp32 0.89-0.94 and bf16
// 0.78-0.89 of the one-row time, on 128-thread CTAs (1-7% faster than 256
// there: the halved thread count spreads over more CTAs per SM); below 2^18 rows (too few threads), with
// 2x2 blocks of 40-entry rows (0.93-1.08), with fp64 values (0.98-1.33) or on
// banded rows of 80-150 entries that share no columns (1.14-1.42) it does not pay.
static int32_t default_threads_per_row(const pjds_dev *A) {
  const double entry = (double)(value_bytes(A->dtype) + 4);
  const double ratio = A->nnz > 0 ? (double)A->n_max * 1048576.0 / ((double)A->nnz * entry) : 0.0;
  int32_t t = ratio < 2.0 ? 1 : ratio < 8.0 ? 2 : ratio < 64.0 ? 4 : 8;
  while (t < 8 && (int64_t)A->n_rows * t < (1 << 17)) t *= 2;
  return t;
}

static LaunchCfg default_cfg(const pjds_dev *A) {
  LaunchCfg c;
  c.rows_per_thread = 1;
  const int32_t t = default_threads_per_row(A);
  c.threads_per_row = t;
  c.block_threads = A->dtype == PJDS_F32 ? 256 : 128;
  if (t == 1) {
    c.block_threads = 256;
    const uintptr_t va = (uintptr_t)A->val, ca = (uintptr_t)A->col;
    const bool paired = shared_pairs(A);
    if (A->dtype != PJDS_F64 && (A->n_rows >= (1 << 21) || paired) && va % (2 * value_bytes(A->dtype)) == 0 &&
        ca % 8 == 0) {
      c.rows_per_thread = 2;
      if (paired) c.block_threads = 128;  // half the threads: spread over more CTAs
    }
  }
  c.unroll = 0;  // filled in by check_cfg once R and T are final
  c.staged = 0;
  c.index64 = 0;
  c.tile_order = auto_tile_order(A) ? 1 : 0;
  c.plan = auto_plan(A) ? 1 : 0;
  return c;
}

}  // namespace pjds

using namespace pjds;

extern "C" int pjds_spmv(const pjds_dev *A, const void *x, void *y, void *stream) {
  clear_error();
  int rc = check_pjds_dev(A, x, y);
  if (rc) return rc;
  LaunchCfg c = default_cfg(A);
  rc = check_cfg(A, c);
  if (rc) return rc;
  return dispatch_pjds(A, x, y, c, static_cast<cudaStream_t>(stream));
}

static int resolve_cfg(const pjds_dev *A, const pjds_launch *cfg, LaunchCfg &c) {
  c = default_cfg(A);
  if (cfg) {
    // a field left at 0 keeps its default; asking for several rows per thread
    // implies one thread per row and vice versa
    if (cfg->rows_per_thread) c.rows_per_thread = cfg->rows_per_thread;
    if (cfg->threads_per_row) c.threads_per_row = cfg->threads_per_row;
    if (cfg->rows_per_thread > 1 && !cfg->threads_per_row) c.threads_per_row = 1;
    if (cfg->threads_per_row > 1 && !cfg->rows_per_thread) c.rows_per_thread = 1;
    if (cfg->block_threads) c.block_threads = cfg->block_threads;
    if (cfg->unroll) c.unroll = cfg->unroll;
    if (cfg->index64) c.index64 = 1;
    if (cfg->tile_order < -1 || cfg->tile_order > 1) return set_error(PJDS_EINVAL, "tile_order must be -1, 0 or 1");
    if (cfg->tile_order == 1 && !A->tile_order) return set_error(PJDS_EINVAL, "tile_order = 1 but A->tile_order is NULL");
    if (cfg->tile_order) c.tile_order = cfg->tile_order == 1;
    // the per-tile mapping: forced, switched off, or automatic unless the
    // caller asked for a uniform mapping
    if (cfg->plan < -1 || cfg->plan > 1) return set_error(PJDS_EINVAL, "plan must be -1, 0 or 1");
    if (cfg->plan == 1) {
      if (!plan_usable(A))
        return set_error(PJDS_EINVAL, "plan = 1 needs A->plan with entries and 16-byte aligned plan, val and col");
      if (cfg->staged) return set_error(PJDS_EINVAL, "staged and plan = 1 are exclusive");
      c.plan = 1;
    } else if (cfg->plan == -1 || cfg->rows_per_thread || cfg->threads_per_row || cfg->block_threads ||
               cfg->unroll || cfg->staged || cfg->tile_order) {
      c.plan = 0;
    }
    if (cfg->staged) {
      c.staged = 1;
      if (!cfg->rows_per_thread) c.rows_per_thread = 1;
      if (!cfg->threads_per_row) c.threads_per_row = 1;
    }
  }
  return check_cfg(A, c);
}

extern "C" int pjds_spmv_resolve(const pjds_dev *A, const pjds_launch *cfg, pjds_launch *out) {
  clear_error();
  if (!A || !out) return set_error(PJDS_EINVAL, "A or out is NULL");
  int rc = check_pjds_dev(A, nullptr, nullptr, false);
  if (rc) return rc;
  LaunchCfg c;
  rc = resolve_cfg(A, cfg, c);
  if (rc) return rc;
  out->rows_per_thread = c.rows_per_thread;
  out->threads_per_row = c.threads_per_row;
  out->block_threads = c.block_threads;
  out->unroll = c.unroll;
  out->staged = c.staged;
  out->index64 = c.index64;
  out->tile_order = c.tile_order ? 1 : -1;
  out->plan = c.plan ? 1 : -1;
  return PJDS_OK;
}

extern "C" int pjds_spmv_cfg(const pjds_dev *A, const void *x, void *y, const pjds_launch *cfg, void *stream) {
  clear_error();
  int rc = check_pjds_dev(A, x, y);
  if (rc) return rc;
  LaunchCfg c;
  rc = resolve_cfg(A, cfg, c);
  if (rc) return rc;
  return dispatch_pjds(A, x, y, c, static_cast<cudaStream_t>(stream));
}

extern "C" int pjds_spmv_pattern(const pjds_dev *A, const void *x, void *y, const pjds_launch *cfg, void *stream) {
  clear_error();
  int rc = check_pjds_dev(A, x, y);
  if (rc) return rc;
  LaunchCfg c;
  rc = resolve_cfg(A, cfg, c);
  if (rc) return rc;
  if (c.staged) return set_error(PJDS_EINVAL, "the pattern product does not run the staged kernel");
  c.pattern = 1;
  return dispatch_pjds(A, x, y, c, static_cast<cudaStream_t>(stream));
}

extern "C" int pjds_device_status(int32_t *status, int32_t clear, void *stream) {
  clear_error();
  if (!status) return set_error(PJDS_EINVAL, "status is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int a = 0, b = 0, c = 0;
  int e = staged_status_f64(&a, clear != 0, s);
  if (e == 0) e = staged_status_f32(&b, clear != 0, s);
  if (e == 0) e = staged_status_bf16(&c, clear != 0, s);
  if (e != 0) return set_error(PJDS_ECUDA, "reading the device status: %s", cudaGetErrorString((cudaError_t)e));
  *status = a | b | c;
  return PJDS_OK;
}

extern "C" int pjds_check_word(uint64_t *word, int32_t clear, void *stream) {
  clear_error();
  if (!word) return set_error(PJDS_EINVAL, "word is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned long long w[4] = {0, 0, 0, 0};
  int (*const readers[4])(unsigned long long *, bool, cudaStream_t) = {check_word_f64, check_word_f32,
                                                                      check_word_bf16, check_word_batch};
  for (int k = 0; k < 4; ++k) {
    const int e = readers[k](&w[k], clear != 0, s);
    if (e == (int)cudaErrorNotSupported) return set_error(PJDS_EINVAL, "not a checked build (PJDS_CHECKED)");
    if (e != 0) return set_error(PJDS_ECUDA, "reading the check word: %s", cudaGetErrorString((cudaError_t)e));
  }
  *word = 0;
  for (int k = 0; k < 4 && !*word; ++k) *word = w[k];
  return PJDS_OK;
}

extern "C" int pjds_wait_selftest(int32_t which, void *stream) {
  clear_error();
  if (which != 0 && which != 1) return set_error(PJDS_EINVAL, "which must be 0 or 1");
  return staged_wait_selftest(which, static_cast<cudaStream_t>(stream));
}

extern "C" int pjds_spmv_host(const pjds_dev *A, const void *x_host, void *y_host, void *x_dev, void *y_dev,
                              void *stream) {
  clear_error();
  int rc = check_pjds_dev(A, x_dev, y_dev);
  if (rc) return rc;
  if (A->n_rows > 0 && (!x_host || !y_host)) return set_error(PJDS_EINVAL, "host vector is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t vb = (size_t)vector_bytes(A->dtype);
  if (A->n_rows > 0) {
    cudaError_t e = cudaMemcpyAsync(x_dev, x_host, (size_t)A->n_cols * vb, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return set_error(PJDS_ECUDA, "copy x to device: %s", cudaGetErrorString(e));
    LaunchCfg c = default_cfg(A);
    rc = check_cfg(A, c);
    if (rc) return rc;
    rc = dispatch_pjds(A, x_dev, y_dev, c, s);
    if (rc) return rc;
    e = cudaMemcpyAsync(y_host, y_dev, (size_t)A->n_rows * vb, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return set_error(PJDS_ECUDA, "copy y to host: %s", cudaGetErrorString(e));
  }
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return set_error(PJDS_ECUDA, "stream synchronize: %s", cudaGetErrorString(e));
  return PJDS_OK;
}

extern "C" int pjds_spmv_host_stream(const pjds_dev *A, int32_t n_vec, const void *const *x_host,
                                     void *const *y_host, void *const *x_dev, void *const *y_dev, void *stream) {
  clear_error();
  if (n_vec < 0) return set_error(PJDS_EINVAL, "n_vec = %d", n_vec);
  if (!x_host || !y_host || !x_dev || !y_dev) return set_error(PJDS_EINVAL, "a pointer array is NULL");
  int rc = check_pjds_dev(A, x_dev[0], y_dev[0]);
  if (rc) return rc;
  if ((rc = check_pjds_dev(A, x_dev[1], y_dev[1]))) return rc;
  if (A->n_rows > 0) {
    const void *d[4] = {x_dev[0], x_dev[1], y_dev[0], y_dev[1]};
    for (int a = 0; a < 4; ++a)
      for (int b = a + 1; b < 4; ++b)
        if (d[a] == d[b]) return set_error(PJDS_EINVAL, "the four device buffers must be distinct");
    for (int32_t v = 0; v < n_vec; ++v)
      if (!x_host[v] || !y_host[v]) return set_error(PJDS_EINVAL, "host vector %d is NULL", v);
  }
  LaunchCfg c = default_cfg(A);
  if ((rc = check_cfg(A, c))) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (n_vec == 0 || A->n_rows == 0) {
    const cudaError_t e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? PJDS_OK : set_error(PJDS_ECUDA, "stream synchronize: %s", cudaGetErrorString(e));
  }
  const size_t vb = (size_t)vector_bytes(A->dtype), nx = (size_t)A->n_cols * vb, ny = (size_t)A->n_rows * vb;
  cudaStream_t cin = nullptr, cout = nullptr;
  // start, done, and per buffer: x ready, product done, y copied out
  cudaEvent_t ev[8] = {};
  cudaError_t e = cudaStreamCreateWithFlags(&cin, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cout, cudaStreamNonBlocking);
  for (int k = 0; k < 8 && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming);
  cudaEvent_t start = ev[0], done = ev[1], *xr = ev + 2, *kd = ev + 4, *yo = ev + 6;
  if (e == cudaSuccess) e = cudaEventRecord(start, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(cin, start, 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(cout, start, 0);
  for (int32_t v = 0; v < n_vec && e == cudaSuccess && rc == PJDS_OK; ++v) {
    const int b = v & 1;
    if (v >= 2) e = cudaStreamWaitEvent(cin, kd[b], 0);  // x buffer b: product v-2 has read it
    if (e == cudaSuccess) e = cudaMemcpyAsync(x_dev[b], x_host[v], nx, cudaMemcpyHostToDevice, cin);
    if (e == cudaSuccess) e = cudaEventRecord(xr[b], cin);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, xr[b], 0);
    if (e == cudaSuccess && v >= 2) e = cudaStreamWaitEvent(s, yo[b], 0);  // y buffer b: y_{v-2} is out
    if (e != cudaSuccess) break;
    rc = dispatch_pjds(A, x_dev[b], y_dev[b], c, s);
    if (rc) break;
    e = cudaEventRecord(kd[b], s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cout, kd[b], 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(y_host[v], y_dev[b], ny, cudaMemcpyDeviceToHost, cout);
    if (e == cudaSuccess) e = cudaEventRecord(yo[b], cout);
  }
  if (e == cudaSuccess && rc == PJDS_OK) e = cudaEventRecord(done, cout);
  if (e == cudaSuccess && rc == PJDS_OK) e = cudaStreamWaitEvent(s, done, 0);
  // drain every stream before releasing them, on success and on error alike
  cudaError_t es = cudaStreamSynchronize(s);
  if (cin) cudaStreamSynchronize(cin);
  if (cout) {
    const cudaError_t eo = cudaStreamSynchronize(cout);
    if (es == cudaSuccess) es = eo;
  }
  for (cudaEvent_t x : ev)
    if (x) cudaEventDestroy(x);
  if (cin) cudaStreamDestroy(cin);
  if (cout) cudaStreamDestroy(cout);
  if (rc) return rc;
  if (e != cudaSuccess) return set_error(PJDS_ECUDA, "host stream: %s", cudaGetErrorString(e));
  if (es != cudaSuccess) return set_error(PJDS_ECUDA, "host stream synchronize: %s", cudaGetErrorString(es));
  return PJDS_OK;
}

static int permute_common(const pjds_dev *A, const void *src, void *dst, bool inverse, void *stream) {
  clear_error();
  if (!A) return set_error(PJDS_EINVAL, "A is NULL");
  if (value_bytes(A->dtype) == 0) return set_error(PJDS_EINVAL, "unknown dtype %d", A->dtype);
  if (A->n_rows < 0) return set_error(PJDS_EINVAL, "bad n_rows");
  if (A->n_rows == 0) return PJDS_OK;
  if (!A->perm || !src || !dst) return set_error(PJDS_EINVAL, "perm or a vector is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (A->dtype == PJDS_F64) return launch_permute<double>(A->perm, src, dst, A->n_rows, inverse, s);
  return launch_permute<float>(A->perm, src, dst, A->n_rows, inverse, s);
}

extern "C" int pjds_permute(const pjds_dev *A, const void *v, void *v_perm, void *stream) {
  return permute_common(A, v, v_perm, false, stream);
}

extern "C" int pjds_unpermute(const pjds_dev *A, const void *v_perm, void *v, void *stream) {
  return permute_common(A, v_perm, v, true, stream);
}

extern "C" int ellr_spmv(const ellr_dev *A, const void *x, void *y, void *stream) {
  clear_error();
  if (!A) return set_error(PJDS_EINVAL, "A is NULL");
  if (value_bytes(A->dtype) == 0) return set_error(PJDS_EINVAL, "unknown dtype %d", A->dtype);
  if (A->n_rows < 0 || A->n_cols < 1 || (int64_t)A->n_pad != ((int64_t)A->n_rows + 31) / 32 * 32)
    return set_error(PJDS_EINVAL, "bad sizes");
  if (A->n_rows == 0) return PJDS_OK;
  if (!x || !y || !A->row_max) return set_error(PJDS_EINVAL, "x, y or row_max is NULL");
  if (A->n_stored > 0 && (!A->val || !A->col)) return set_error(PJDS_EINVAL, "val or col is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int nt = 128;
  switch (A->dtype) {
    case PJDS_F64: return ellr_launch_f64(A, x, y, nt, s);
    case PJDS_F32: return ellr_launch_f32(A, x, y, nt, s);
    default: return ellr_launch_bf16(A, x, y, nt, s);
  }
}
