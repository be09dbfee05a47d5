// Krylov drivers on pJDS matrices in the permuted basis (include/pjds_krylov.h):
// mixed-precision CG with fp64 residual refinement, Lanczos, fp64 Ritz refine.
//
// Every step runs in the kernels below; the host only sequences launches,
// reads one residual norm per outer CG step and solves the small tridiagonal
// eigenproblem. Scalars (alpha, beta, norms) live in device memory and are
// read by the kernels that need them, so a run of inner iterations has no
// host round trip and can be captured once in a CUDA graph. Inner products
// accumulate in fp64 with a fixed reduction order: per-CTA partial sums
// (warp shuffles, then one warp) into the workspace; the CTA that finishes
// last (a counter in the workspace) adds the partials in index order and
// applies the scalar update, inside the same launch. The summation pattern
// does not depend on which CTA is last — results are bitwise reproducible.
#include <float.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "common.h"
#include "pjds_krylov.h"
#include "spmv_kernels.cuh"

namespace pjds {
namespace kry {

constexpr int KT = 256;  // threads per CTA of the vector and product kernels

// slots of the device scalar block
// (slot S_CTR holds the 32-bit arrival counter of the reduction in flight; it
// is 0 between launches)
enum { S_RR = 0, S_PQ, S_ALPHA, S_BETA, S_NRM, S_INVNRM, S_AUX0, S_AUX1, S_AUX2, S_CTR = 15, S_COUNT = 16 };
// finalisation operations
enum { F_ALPHA = 0, F_BETA, F_RR, F_NORM, F_LALPHA, F_LBETA, F_STORE };

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sh[KT / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  if (w == 0) {
    s = l < KT / 32 ? sh[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  }
  return s;  // complete in thread 0
}

// Where a reduction's result goes: the partial-sum array (one slot per CTA),
// the scalar block (its S_CTR slot is the arrival counter) and the update.
struct Fin {
  double *partial;
  double *scal;
  double *out;
  int32_t op, j;
};

// The scalar update `op` with the complete sum v.
__device__ __forceinline__ void apply_op(double v, const Fin &f) {
  double *scal = f.scal;
  switch (f.op) {
    case F_ALPHA:  // alpha = (r, r) / (p, A p)
      scal[S_PQ] = v;
      scal[S_ALPHA] = v != 0.0 ? scal[S_RR] / v : 0.0;
      break;
    case F_BETA:  // beta = (r', r') / (r, r)
      scal[S_BETA] = scal[S_RR] != 0.0 ? v / scal[S_RR] : 0.0;
      scal[S_RR] = v;
      break;
    case F_RR:
      scal[S_RR] = v;
      break;
    case F_NORM: {
      const double nrm = sqrt(v);
      scal[S_NRM] = nrm;
      scal[S_INVNRM] = nrm > 0.0 ? 1.0 / nrm : 0.0;
      break;
    }
    case F_LALPHA:
      f.out[f.j] = v;
      break;
    case F_LBETA: {
      const double nrm = sqrt(v);
      f.out[f.j] = nrm;
      scal[S_INVNRM] = nrm > 0.0 ? 1.0 / nrm : 0.0;
      break;
    }
    default:  // F_STORE
      scal[f.j] = v;
      break;
  }
}

// End of a reducing kernel, called by every thread; thread 0 holds the CTA's
// sum s. The sum goes to partial[blockIdx.x], is made visible device-wide,
// and the CTA counts itself in. The CTA that arrives last adds all gridDim.x
// partials in index order (strided per thread, then the CTA tree: the same
// pattern whichever CTA it is), applies the update and puts the counter back
// to 0 for the next reduction on the stream.
__device__ __forceinline__ void finish(double s, const Fin &f) {
  __shared__ int last;
  unsigned *ctr = reinterpret_cast<unsigned *>(f.scal + S_CTR);
  if (threadIdx.x == 0) {
    f.partial[blockIdx.x] = s;
    __threadfence();
    last = atomicAdd(ctr, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double v = 0.0;
  for (uint32_t k = threadIdx.x; k < gridDim.x; k += KT) v += __ldcg(f.partial + k);
  v = block_sum(v);
  if (threadIdx.x == 0) {
    apply_op(v, f);
    *ctr = 0u;
  }
}

// One sorted row's product in the permuted basis (Listing 2 with the loop
// bound of the row's block; pads carry column -1 and are skipped).
template <typename TV, typename TX, typename IDX>
__device__ __forceinline__ typename dev::Acc<TV>::T row_product(const TV *__restrict__ val,
                                                                 const int32_t *__restrict__ col,
                                                                 const int64_t *__restrict__ col_start, int32_t L,
                                                                 int64_t i, const TX *__restrict__ x) {
  using TA = typename dev::Acc<TV>::T;
  constexpr int U = 4;
  TA acc = TA(0);
  for (int32_t j = 0; j < L; j += U) {
    int32_t c[U];
    TV v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (j + u < L) {
        const IDX o = (IDX)__ldg(col_start + j + u) + (IDX)i;
        c[u] = __ldcs(col + o);
        v[u] = dev::ld_stream1(val + o);
      } else {
        c[u] = -1;
        v[u] = TV{};
      }
    }
    TX xv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) xv[u] = dev::gather(x, c[u]);
#pragma unroll
    for (int u = 0; u < U; ++u) acc = c[u] >= 0 ? dev::fma_acc(dev::to_acc(v[u]), (TA)xv[u], acc) : acc;
  }
  return acc;
}

// Two adjacent sorted rows i, i+1 (i even, so both lie in one block): one
// paired load of col and of val per jagged diagonal, then each row's product
// exactly as row_product computes it.
template <typename TV, typename TX, typename IDX>
__device__ __forceinline__ void row_product2(const TV *__restrict__ val, const int32_t *__restrict__ col,
                                             const int64_t *__restrict__ col_start, int32_t L, int64_t i,
                                             const TX *__restrict__ x, typename dev::Acc<TV>::T (&acc)[2]) {
  using TA = typename dev::Acc<TV>::T;
  constexpr int U = 4;
  acc[0] = acc[1] = TA(0);
  for (int32_t j = 0; j < L; j += U) {
    int32_t c[U][2];
    TV v[U][2];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (j + u < L) {
        const IDX o = (IDX)__ldg(col_start + j + u) + (IDX)i;
        dev::ld_stream<2>(col + o, c[u]);
        dev::ld_stream<2>(val + o, v[u]);
      } else {
        c[u][0] = c[u][1] = -1;
        v[u][0] = v[u][1] = TV{};
      }
    }
    TX xv[U][2];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int r = 0; r < 2; ++r) xv[u][r] = dev::gather(x, c[u][r]);
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int r = 0; r < 2; ++r)
        acc[r] = c[u][r] >= 0 ? dev::fma_acc(dev::to_acc(v[u][r]), (TA)xv[u][r], acc[r]) : acc[r];
  }
}

// The reducing kernels below run a grid of at most as many CTAs as fit on the
// GPU at once and stride over the vectors (element i is taken by thread
// i mod KT of CTA (i / KT) mod gridDim.x); each thread accumulates its own
// elements in order, so the sum depends only on the grid size, which the host
// derives from the device and the kernel alone.

// MODE 0: y = A x and the reduction of sum x_i y_i.  MODE 1: y = bv - A x and
// the reduction of sum y_i^2 (the fp64 residual of the refinement loop). The
// value array arrives untyped so that every instance for one vector type has
// the same signature.
template <typename TV, typename TX, typename IDX, int MODE>
__global__ void __launch_bounds__(KT)
    spmv_dot_kernel(const void *__restrict__ val_, const int32_t *__restrict__ col,
                    const int64_t *__restrict__ col_start, const int32_t *__restrict__ block_len,
                    const TX *__restrict__ x, TX *__restrict__ y, const TX *__restrict__ bv, Fin f, int32_t n_rows,
                    int32_t b) {
  const TV *__restrict__ val = static_cast<const TV *>(val_);
  double contrib = 0.0;
  // rows in sorted order: the tile traversal table measured 1.7% slower here
  // (fp64 CG on the 27-point stencil, 4.5M rows)
  for (int64_t i = (int64_t)blockIdx.x * KT + threadIdx.x; i < n_rows; i += (int64_t)gridDim.x * KT) {
    const int32_t L = __ldg(block_len + (int32_t)(i / b));
    const auto acc = row_product<TV, TX, IDX>(val, col, col_start, L, i, x);
    TX yi;
    if constexpr (MODE == 0) {
      yi = (TX)acc;
      contrib += (double)x[i] * (double)yi;
    } else {
      yi = (TX)((double)bv[i] - (double)acc);
      contrib += (double)yi * (double)yi;
    }
    y[i] = yi;
  }
  const double s = block_sum(contrib);
  finish(s, f);
}

// y = A x and the reduction of sum x_i y_i with two adjacent rows per thread
// (row pair p: rows 2p, 2p+1; the second is a padding row when n_rows is odd)
template <typename TV, typename TX, typename IDX>
__global__ void __launch_bounds__(KT)
    spmv_dot2_kernel(const void *__restrict__ val_, const int32_t *__restrict__ col,
                     const int64_t *__restrict__ col_start, const int32_t *__restrict__ block_len,
                     const TX *__restrict__ x, TX *__restrict__ y, const TX *__restrict__ bv, Fin f, int32_t n_rows,
                     int32_t b) {
  const TV *__restrict__ val = static_cast<const TV *>(val_);
  const int64_t n_pairs = ((int64_t)n_rows + 1) / 2;
  double contrib = 0.0;
  for (int64_t p = (int64_t)blockIdx.x * KT + threadIdx.x; p < n_pairs; p += (int64_t)gridDim.x * KT) {
    const int64_t i = 2 * p;
    const int32_t L = __ldg(block_len + (int32_t)(i / b));
    typename dev::Acc<TV>::T acc[2];
    row_product2<TV, TX, IDX>(val, col, col_start, L, i, x, acc);
#pragma unroll
    for (int r = 0; r < 2; ++r)
      if (i + r < n_rows) {
        const TX yi = (TX)acc[r];
        contrib += (double)x[i + r] * (double)yi;
        y[i + r] = yi;
      }
  }
  const double s = block_sum(contrib);
  finish(s, f);
}

template <typename TX>
__global__ void __launch_bounds__(KT) sumsq_kernel(const TX *__restrict__ v, Fin f, int32_t n) {
  double contrib = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * KT + threadIdx.x; i < n; i += (int64_t)gridDim.x * KT) {
    const double x = (double)v[i];
    contrib += x * x;
  }
  const double s = block_sum(contrib);
  finish(s, f);
}

// 16-byte groups of workspace vectors (the workspace is 256-byte aligned):
// W elements per load and store.
template <typename TX>
struct G16 {
  static constexpr int W = 16 / (int)sizeof(TX);
  __device__ static void load(const TX *p, TX (&v)[W]) {
    const uint4 u = *reinterpret_cast<const uint4 *>(p);
    memcpy(v, &u, 16);
  }
  __device__ static void store(TX *p, const TX (&v)[W]) {
    uint4 u;
    memcpy(&u, v, 16);
    *reinterpret_cast<uint4 *>(p) = u;
  }
};

// d += alpha p; r -= alpha q; reduces sum r_i^2. Thread k takes 16-byte
// groups k, k + stride, ...; the last n mod W elements go one per thread.
template <typename TX>
__global__ void __launch_bounds__(KT)
    cg_update_kernel(TX *__restrict__ d, TX *__restrict__ r, const TX *__restrict__ p, const TX *__restrict__ q,
                     Fin f, int32_t n) {
  constexpr int W = G16<TX>::W;
  const TX a = (TX)f.scal[S_ALPHA];
  const int64_t ng = n / W, stride = (int64_t)gridDim.x * KT, t = (int64_t)blockIdx.x * KT + threadIdx.x;
  double contrib = 0.0;
  for (int64_t k = t; k < ng; k += stride) {
    TX dv[W], rv[W], pv[W], qv[W];
    G16<TX>::load(d + k * W, dv);
    G16<TX>::load(r + k * W, rv);
    G16<TX>::load(p + k * W, pv);
    G16<TX>::load(q + k * W, qv);
#pragma unroll
    for (int w = 0; w < W; ++w) {
      dv[w] = dv[w] + a * pv[w];
      rv[w] = rv[w] - a * qv[w];
      contrib += (double)rv[w] * (double)rv[w];
    }
    G16<TX>::store(d + k * W, dv);
    G16<TX>::store(r + k * W, rv);
  }
  for (int64_t i = ng * W + t; i < n; i += stride) {
    d[i] = d[i] + a * p[i];
    const TX ri = r[i] - a * q[i];
    r[i] = ri;
    contrib += (double)ri * (double)ri;
  }
  const double s = block_sum(contrib);
  finish(s, f);
}

// p = r + beta p: one 16-byte group per thread, then the last n mod W
// elements one per thread.
template <typename TX>
__global__ void __launch_bounds__(KT)
    cg_dir_kernel(TX *__restrict__ p, const TX *__restrict__ r, const double *__restrict__ scal, int32_t n) {
  constexpr int W = G16<TX>::W;
  const TX be = (TX)scal[S_BETA];
  const int64_t ng = n / W, k = (int64_t)blockIdx.x * KT + threadIdx.x;
  if (k < ng) {
    TX pv[W], rv[W];
    G16<TX>::load(p + k * W, pv);
    G16<TX>::load(r + k * W, rv);
#pragma unroll
    for (int w = 0; w < W; ++w) pv[w] = rv[w] + be * pv[w];
    G16<TX>::store(p + k * W, pv);
  }
  const int64_t i = ng * W + k;
  if (i < n) p[i] = r[i] + be * p[i];
}

// Start of an inner solve: r = p = (r64 / ||r64||) in the inner type, d = 0,
// reduces sum r_i^2.
template <typename TL>
__global__ void __launch_bounds__(KT)
    ir_start_kernel(const double *__restrict__ r64, TL *__restrict__ r, TL *__restrict__ p, TL *__restrict__ d,
                    Fin f, int32_t n) {
  const double inv = f.scal[S_INVNRM];
  double contrib = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * KT + threadIdx.x; i < n; i += (int64_t)gridDim.x * KT) {
    const TL ri = (TL)(r64[i] * inv);
    r[i] = ri;
    p[i] = ri;
    d[i] = TL(0);
    contrib += (double)ri * (double)ri;
  }
  const double s = block_sum(contrib);
  finish(s, f);
}

// x += ||r64|| d (fp64)
template <typename TL>
__global__ void __launch_bounds__(KT)
    ir_correct_kernel(double *__restrict__ x, const TL *__restrict__ d, const double *__restrict__ scal, int32_t n) {
  const int64_t i = (int64_t)blockIdx.x * KT + threadIdx.x;
  if (i < n) x[i] = fma(scal[S_NRM], (double)d[i], x[i]);
}

// v = v0 / ||v0||, vprev = 0
template <typename TX>
__global__ void __launch_bounds__(KT)
    lanczos_start_kernel(const TX *__restrict__ v0, TX *__restrict__ v, TX *__restrict__ vprev,
                         const double *__restrict__ scal, int32_t n) {
  const int64_t i = (int64_t)blockIdx.x * KT + threadIdx.x;
  if (i < n) {
    v[i] = (TX)((double)v0[i] * scal[S_INVNRM]);
    vprev[i] = TX(0);
  }
}

// w = w - alpha_j v - beta_j vprev (in fp64, stored in TX); reduces sum w_i^2
template <typename TX>
__global__ void __launch_bounds__(KT)
    lanczos_orth_kernel(TX *__restrict__ w, const TX *__restrict__ v, const TX *__restrict__ vprev,
                        const double *__restrict__ alpha, const double *__restrict__ beta, int32_t j, Fin f,
                        int32_t n) {
  constexpr int W = G16<TX>::W;
  const double aj = alpha[j], bj = beta[j];
  const int64_t ng = n / W, stride = (int64_t)gridDim.x * KT, t = (int64_t)blockIdx.x * KT + threadIdx.x;
  double contrib = 0.0;
  for (int64_t k = t; k < ng; k += stride) {
    TX wv[W], vv[W], pv[W];
    G16<TX>::load(w + k * W, wv);
    G16<TX>::load(v + k * W, vv);
    G16<TX>::load(vprev + k * W, pv);
#pragma unroll
    for (int e = 0; e < W; ++e) {
      const TX ws = (TX)((double)wv[e] - aj * (double)vv[e] - bj * (double)pv[e]);
      wv[e] = ws;
      contrib += (double)ws * (double)ws;
    }
    G16<TX>::store(w + k * W, wv);
  }
  for (int64_t i = ng * W + t; i < n; i += stride) {
    const double wi = (double)w[i] - aj * (double)v[i] - bj * (double)vprev[i];
    const TX ws = (TX)wi;
    w[i] = ws;
    contrib += (double)ws * (double)ws;
  }
  const double s = block_sum(contrib);
  finish(s, f);
}

// basis_row = v (optional); vprev = v; v = w / beta_{j+1}
template <typename TX>
__global__ void __launch_bounds__(KT)
    lanczos_next_kernel(TX *__restrict__ vprev, TX *__restrict__ v, const TX *__restrict__ w,
                        const double *__restrict__ scal, TX *__restrict__ basis_row, int32_t n) {
  constexpr int W = G16<TX>::W;
  const double inv = scal[S_INVNRM];
  const int64_t ng = n / W, k = (int64_t)blockIdx.x * KT + threadIdx.x;
  // the basis row is caller memory: 16-byte stores only when it is aligned
  const bool row16 = basis_row && ((uintptr_t)basis_row & 15) == 0;
  if (k < ng) {
    TX vv[W], wv[W], nv[W];
    G16<TX>::load(v + k * W, vv);
    G16<TX>::load(w + k * W, wv);
    if (row16) {
      G16<TX>::store(basis_row + k * W, vv);
    } else if (basis_row) {
#pragma unroll
      for (int e = 0; e < W; ++e) basis_row[k * W + e] = vv[e];
    }
    G16<TX>::store(vprev + k * W, vv);
#pragma unroll
    for (int e = 0; e < W; ++e) nv[e] = (TX)((double)wv[e] * inv);
    G16<TX>::store(v + k * W, nv);
  }
  const int64_t i = ng * W + k;
  if (i < n) {
    const TX vi = v[i];
    if (basis_row) basis_row[i] = vi;
    vprev[i] = vi;
    v[i] = (TX)((double)w[i] * inv);
  }
}

// y = sum_j s_j basis[j] (fp64); reduces sum y_i^2
template <typename TB>
__global__ void __launch_bounds__(KT)
    ritz_combine_kernel(const TB *__restrict__ basis, const double *__restrict__ s, int32_t k, int32_t n,
                        double *__restrict__ y, Fin f) {
  double contrib = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * KT + threadIdx.x; i < n; i += (int64_t)gridDim.x * KT) {
    double acc = 0.0;
    for (int32_t j = 0; j < k; ++j) acc = fma(s[j], (double)__ldcs(basis + (int64_t)j * n + i), acc);
    y[i] = acc;
    contrib += acc * acc;
  }
  const double sm = block_sum(contrib);
  finish(sm, f);
}

// reduces sum (w_i - theta y_i)^2 with theta = scal[S_AUX1] / scal[S_AUX0]
__global__ void __launch_bounds__(KT)
    ritz_residual_kernel(const double *__restrict__ w, const double *__restrict__ y, Fin f, int32_t n) {
  const double theta = f.scal[S_AUX1] / f.scal[S_AUX0];
  double contrib = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * KT + threadIdx.x; i < n; i += (int64_t)gridDim.x * KT) {
    const double e = w[i] - theta * y[i];
    contrib += e * e;
  }
  const double s = block_sum(contrib);
  finish(s, f);
}

// ----------------------------------------------------------------------------- host helpers

static inline size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }
static inline int32_t n_blocks_of(int32_t n) { return (int32_t)(((int64_t)n + KT - 1) / KT); }

struct Carve {
  char *base;
  size_t off, cap;
  template <typename T>
  T *take(size_t count) {
    T *p = reinterpret_cast<T *>(base + off);
    off += align256(count * sizeof(T));
    return p;
  }
};

static int launch_check(const char *what) {
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? PJDS_OK : set_error(PJDS_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Record the launches `body` issues into a graph on a private stream and
// instantiate it. Nothing executes while capturing.
template <typename F>
static int capture_graph(cudaGraphExec_t *exec, F body) {
  cudaStream_t cap = nullptr;
  cudaGraph_t g = nullptr;
  *exec = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) return set_error(PJDS_ECUDA, "graph stream: %s", cudaGetErrorString(e));
  e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    body(cap);
    const cudaError_t e_launch = cudaGetLastError();
    e = cudaStreamEndCapture(cap, &g);
    if (e == cudaSuccess) e = e_launch;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(exec, g, 0);
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cap);
  if (e != cudaSuccess) {
    if (*exec) cudaGraphExecDestroy(*exec);
    *exec = nullptr;
    return set_error(PJDS_ECUDA, "graph capture: %s", cudaGetErrorString(e));
  }
  return PJDS_OK;
}

static int check_square_permuted(const pjds_dev *A, const char *name) {
  if (!A) return set_error(PJDS_EINVAL, "%s is NULL", name);
  if (value_bytes(A->dtype) == 0) return set_error(PJDS_EINVAL, "%s: unknown dtype", name);
  if (!A->permute_cols || A->n_rows != A->n_cols)
    return set_error(PJDS_EINVAL, "%s must be square and created with permute_cols = 1", name);
  if (A->b <= 0 || A->b % 32 || (int64_t)A->n_pad != ((int64_t)A->n_rows + A->b - 1) / A->b * A->b)
    return set_error(PJDS_EINVAL, "%s: inconsistent n_pad / b", name);
  if (A->n_stored > 0 && (!A->val || !A->col || !A->col_start || !A->block_len))
    return set_error(PJDS_EINVAL, "%s: a matrix array is NULL", name);
  return PJDS_OK;
}

// CTAs of a reducing kernel: as many as are resident on all SMs at once at
// the kernel's occupancy (the grid-stride loops cover the rest), at most one
// per KT elements. Queried outside any stream capture.
template <typename K>
static int red_grid(K kernel, int32_t n, int32_t *grid) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, KT, 0);
  if (e != cudaSuccess) return set_error(PJDS_ECUDA, "occupancy query: %s", cudaGetErrorString(e));
  if (sms < 1 || per_sm < 1) return set_error(PJDS_ECUDA, "kernel does not fit on an SM");
  *grid = (int32_t)std::min<int64_t>(std::max<int32_t>(n_blocks_of(n), 1), (int64_t)sms * per_sm);
  return PJDS_OK;
}

// A product-and-reduce kernel chosen by value type and index width, with its
// grid.
template <typename TX, int MODE>
struct Dot {
  void (*fn)(const void *, const int32_t *, const int64_t *, const int32_t *, const TX *, TX *, const TX *, Fin,
             int32_t, int32_t);
  int32_t grid;
};

template <typename TV, typename TX, int MODE>
static int make_dot_typed(const pjds_dev *A, Dot<TX, MODE> *d) {
  if (A->n_stored + A->n_pad < 0x7fffffffLL)
    d->fn = spmv_dot_kernel<TV, TX, int32_t, MODE>;
  else
    d->fn = spmv_dot_kernel<TV, TX, int64_t, MODE>;
  return red_grid(d->fn, A->n_rows, &d->grid);
}

template <typename TX, int MODE>
static int make_dot(const pjds_dev *A, Dot<TX, MODE> *d);
template <>
int make_dot<double, 0>(const pjds_dev *A, Dot<double, 0> *d) {
  return make_dot_typed<double, double, 0>(A, d);
}
template <>
int make_dot<double, 1>(const pjds_dev *A, Dot<double, 1> *d) {
  return make_dot_typed<double, double, 1>(A, d);
}
// fp32 / bf16 values: two rows per thread when val and col allow the paired
// loads (one 8- or 4-byte value load and one 8-byte column load per diagonal)
template <typename TV>
static int make_dot2(const pjds_dev *A, Dot<float, 0> *d) {
  if (A->n_stored + A->n_pad < 0x7fffffffLL)
    d->fn = spmv_dot2_kernel<TV, float, int32_t>;
  else
    d->fn = spmv_dot2_kernel<TV, float, int64_t>;
  return red_grid(d->fn, (int32_t)(((int64_t)A->n_rows + 1) / 2), &d->grid);
}

template <>
int make_dot<float, 0>(const pjds_dev *A, Dot<float, 0> *d) {
  const bool pair = ((uintptr_t)A->val % (2 * value_bytes(A->dtype))) == 0 && ((uintptr_t)A->col % 8) == 0;
  if (pair) return A->dtype == PJDS_BF16 ? make_dot2<dev::bf16_t>(A, d) : make_dot2<float>(A, d);
  return A->dtype == PJDS_BF16 ? make_dot_typed<dev::bf16_t, float, 0>(A, d) : make_dot_typed<float, float, 0>(A, d);
}

template <typename T>
struct Same {
  using type = T;
};

// (the vector type is taken from the launcher alone)
template <typename TX, int MODE>
static void launch_dot(const Dot<TX, MODE> &d, const pjds_dev *A, const typename Same<TX>::type *x,
                       typename Same<TX>::type *y, const typename Same<TX>::type *bv, const Fin &f, cudaStream_t s) {
  d.fn<<<d.grid, KT, 0, s>>>(A->val, A->col, A->col_start, A->block_len, x, y, bv, f, A->n_rows, A->b);
}

// ----------------------------------------------------------------------------- CG

static size_t cg_bytes(int32_t n, int vec_bytes) {
  return align256((size_t)n_blocks_of(n) * 8) + align256(S_COUNT * 8) + 4 * align256((size_t)n * vec_bytes) +
         align256((size_t)n * 8);
}

template <typename TL>
static int cg_run(const pjds_dev *Ah, const pjds_dev *Al, const double *b, double *x, const pjds_cg_opts &o,
                  pjds_cg_result *res, void *work, cudaStream_t s) {
  const int32_t n = Ah->n_rows, nb = n_blocks_of(n);
  Carve cv{static_cast<char *>(work), 0, 0};
  double *partial = cv.take<double>((size_t)nb);
  double *scal = cv.take<double>(S_COUNT);
  TL *r = cv.take<TL>((size_t)n), *p = cv.take<TL>((size_t)n), *q = cv.take<TL>((size_t)n);
  TL *d = cv.take<TL>((size_t)n);
  double *r64 = cv.take<double>((size_t)n);
  auto fin = [&](int32_t op, int32_t j) { return Fin{partial, scal, nullptr, op, j}; };
  int rc;
  Dot<TL, 0> dot_lo;
  Dot<double, 1> dot_res;
  int32_t g_sumsq = 0, g_upd = 0, g_start = 0;
  if ((rc = make_dot(Al, &dot_lo)) || (rc = make_dot(Ah, &dot_res)) || (rc = red_grid(sumsq_kernel<double>, n, &g_sumsq)) ||
      (rc = red_grid(cg_update_kernel<TL>, n, &g_upd)) || (rc = red_grid(ir_start_kernel<TL>, n, &g_start)))
    return rc;
  // cg_dir: one thread per 16-byte group, and as many for the remainder
  const int64_t n_groups = n / G16<TL>::W, n_rem = n - n_groups * G16<TL>::W;
  const int32_t nb_dir = (int32_t)((std::max<int64_t>(std::max(n_groups, n_rem), 1) + KT - 1) / KT);

  // scalar block and reduction counter start at 0
  cudaError_t e = cudaMemsetAsync(scal, 0, S_COUNT * sizeof(double), s);
  if (e != cudaSuccess) return set_error(PJDS_ECUDA, "cg: %s", cudaGetErrorString(e));
  // ||b||
  sumsq_kernel<double><<<g_sumsq, KT, 0, s>>>(b, fin(F_STORE, S_AUX2), n);
  double bn2 = 0.0;
  if ((rc = launch_check("cg ||b||"))) return rc;
  e = cudaMemcpyAsync(&bn2, scal + S_AUX2, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return set_error(PJDS_ECUDA, "cg: %s", cudaGetErrorString(e));
  const double bnorm = sqrt(bn2);

  auto inner_step = [&](cudaStream_t st) {
    launch_dot(dot_lo, Al, p, q, nullptr, fin(F_ALPHA, 0), st);                  // q = A p, (p, q), alpha
    cg_update_kernel<TL><<<g_upd, KT, 0, st>>>(d, r, p, q, fin(F_BETA, 0), n);  // d, r, (r, r), beta
    cg_dir_kernel<TL><<<nb_dir, KT, 0, st>>>(p, r, scal, n);                    // p
  };

  cudaGraphExec_t exec = nullptr;
  if (o.use_graph) {
    // recorded on a private stream (nothing runs during capture; the legacy
    // default stream cannot be captured), replayed on the caller's stream
    rc = capture_graph(&exec, [&](cudaStream_t st) {
      for (int it = 0; it < o.inner_iters; ++it) inner_step(st);
    });
    if (rc) return rc;
  }

  pjds_cg_result out;
  memset(&out, 0, sizeof(out));
  double rel = 0.0;
  rc = PJDS_OK;
  for (int outer = 0;; ++outer) {
    launch_dot(dot_res, Ah, x, r64, b, fin(F_NORM, 0), s);  // r64 = b - A x, ||r64||
    if ((rc = launch_check("cg residual"))) break;
    double rn = 0.0;
    e = cudaMemcpyAsync(&rn, scal + S_NRM, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      rc = set_error(PJDS_ECUDA, "cg: %s", cudaGetErrorString(e));
      break;
    }
    rel = bnorm > 0.0 ? rn / bnorm : rn;
    if (out.n_history < PJDS_CG_HISTORY) out.history[out.n_history++] = rel;
    if (outer >= o.max_outer || rel <= o.tol || rn == 0.0) break;
    ir_start_kernel<TL><<<g_start, KT, 0, s>>>(r64, r, p, d, fin(F_RR, 0), n);
    if (exec) {
      e = cudaGraphLaunch(exec, s);
      if (e != cudaSuccess) {
        rc = set_error(PJDS_ECUDA, "cg graph launch: %s", cudaGetErrorString(e));
        break;
      }
    } else {
      for (int it = 0; it < o.inner_iters; ++it) inner_step(s);
    }
    ir_correct_kernel<TL><<<nb, KT, 0, s>>>(x, d, scal, n);
    if ((rc = launch_check("cg inner"))) break;
    out.outer = outer + 1;
    out.inner_total += o.inner_iters;
  }
  if (exec) cudaGraphExecDestroy(exec);
  out.rel_residual = rel;
  if (res) *res = out;
  return rc;
}

}  // namespace kry
}  // namespace pjds

using namespace pjds;
using namespace pjds::kry;

extern "C" int pjds_cg_workspace_bytes(int32_t n_rows, int32_t n_pad, int32_t vec_dtype, size_t *bytes) {
  clear_error();
  if (!bytes || n_rows < 0 || n_pad < n_rows) return set_error(PJDS_EINVAL, "bad arguments");
  *bytes = cg_bytes(n_rows, vec_dtype == PJDS_F64 ? 8 : 4);
  return PJDS_OK;
}

extern "C" int pjds_cg_solve(const pjds_dev *A_hi, const pjds_dev *A_lo, const double *b, double *x,
                             const pjds_cg_opts *opts, pjds_cg_result *res, void *work, size_t work_bytes,
                             void *stream) {
  clear_error();
  int rc = check_square_permuted(A_hi, "A_hi");
  if (rc) return rc;
  if (A_hi->dtype != PJDS_F64) return set_error(PJDS_EINVAL, "A_hi must hold fp64 values");
  if (!A_lo) A_lo = A_hi;
  if ((rc = check_square_permuted(A_lo, "A_lo"))) return rc;
  if (A_lo->n_rows != A_hi->n_rows) return set_error(PJDS_EINVAL, "A_lo and A_hi differ in size");
  if (A_hi->n_rows == 0) return PJDS_OK;
  if (!b || !x || !work) return set_error(PJDS_EINVAL, "b, x or work is NULL");
  pjds_cg_opts o{6, 50, 0.0, 1, 0};
  if (opts) {
    o = *opts;
    if (o.max_outer <= 0) o.max_outer = 6;
    if (o.inner_iters <= 0) o.inner_iters = 50;
  }
  if (o.inner_iters > 100000 || o.max_outer > 100000) return set_error(PJDS_EINVAL, "iteration counts too large");
  const bool low = A_lo->dtype != PJDS_F64;
  const size_t need = cg_bytes(A_hi->n_rows, low ? 4 : 8);
  if (work_bytes < need) return set_error(PJDS_EINVAL, "workspace of %zu bytes is smaller than %zu", work_bytes, need);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return low ? cg_run<float>(A_hi, A_lo, b, x, o, res, work, s) : cg_run<double>(A_hi, A_lo, b, x, o, res, work, s);
}

// ----------------------------------------------------------------------------- Lanczos

static size_t lanczos_bytes(int32_t n, int vec_bytes, int32_t steps) {
  return align256((size_t)n_blocks_of(n) * 8) + align256(S_COUNT * 8) + align256((size_t)steps * 8) +
         align256((size_t)(steps + 1) * 8) + 3 * align256((size_t)n * vec_bytes);
}

template <typename TX>
static int lanczos_run(const pjds_dev *A, const TX *v0, int32_t steps, double *alpha_h, double *beta_h, TX *basis,
                       int use_graph, void *work, cudaStream_t s) {
  const int32_t n = A->n_rows, nb = n_blocks_of(n);
  Carve cv{static_cast<char *>(work), 0, 0};
  double *partial = cv.take<double>((size_t)nb);
  double *scal = cv.take<double>(S_COUNT);
  double *alpha = cv.take<double>((size_t)steps);
  double *beta = cv.take<double>((size_t)steps + 1);
  TX *v = cv.take<TX>((size_t)n), *vp = cv.take<TX>((size_t)n), *w = cv.take<TX>((size_t)n);
  cudaError_t e = cudaMemsetAsync(beta, 0, sizeof(double) * ((size_t)steps + 1), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(scal, 0, S_COUNT * sizeof(double), s);
  if (e != cudaSuccess) return set_error(PJDS_ECUDA, "lanczos: %s", cudaGetErrorString(e));
  Dot<TX, 0> dot;
  int32_t g_sumsq = 0, g_orth = 0;
  int rc;
  if ((rc = make_dot(A, &dot)) || (rc = red_grid(sumsq_kernel<TX>, n, &g_sumsq)) ||
      (rc = red_grid(lanczos_orth_kernel<TX>, n, &g_orth)))
    return rc;
  // lanczos_next: one thread per 16-byte group, and as many for the remainder
  const int64_t n_groups = n / G16<TX>::W, n_rem = n - n_groups * G16<TX>::W;
  const int32_t nb_next = (int32_t)((std::max<int64_t>(std::max(n_groups, n_rem), 1) + KT - 1) / KT);
  sumsq_kernel<TX><<<g_sumsq, KT, 0, s>>>(v0, Fin{partial, scal, nullptr, F_NORM, 0}, n);
  lanczos_start_kernel<TX><<<nb, KT, 0, s>>>(v0, v, vp, scal, n);
  rc = launch_check("lanczos start");
  if (rc) return rc;
  auto step = [&](int32_t j, cudaStream_t st) {
    launch_dot(dot, A, v, w, nullptr, Fin{partial, scal, alpha, F_LALPHA, j}, st);  // w = A v, alpha_j = (v, w)
    lanczos_orth_kernel<TX>
        <<<g_orth, KT, 0, st>>>(w, v, vp, alpha, beta, j, Fin{partial, scal, beta, F_LBETA, j + 1}, n);  // beta_j+1
    lanczos_next_kernel<TX><<<nb_next, KT, 0, st>>>(vp, v, w, scal, basis ? basis + (int64_t)j * n : nullptr, n);
  };
  if (use_graph) {
    cudaGraphExec_t exec = nullptr;
    rc = capture_graph(&exec, [&](cudaStream_t st) {
      for (int32_t j = 0; j < steps; ++j) step(j, st);
    });
    if (rc) return rc;
    e = cudaGraphLaunch(exec, s);
    cudaGraphExecDestroy(exec);
    if (e != cudaSuccess) return set_error(PJDS_ECUDA, "lanczos graph launch: %s", cudaGetErrorString(e));
  } else {
    for (int32_t j = 0; j < steps; ++j) step(j, s);
  }
  if ((rc = launch_check("lanczos steps"))) return rc;
  e = cudaMemcpyAsync(alpha_h, alpha, sizeof(double) * (size_t)steps, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(beta_h, beta, sizeof(double) * ((size_t)steps + 1), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return set_error(PJDS_ECUDA, "lanczos: %s", cudaGetErrorString(e));
  return PJDS_OK;
}

extern "C" int pjds_lanczos_workspace_bytes(int32_t n_rows, int32_t n_pad, int32_t vec_dtype, int32_t steps,
                                            size_t *bytes) {
  clear_error();
  if (!bytes || n_rows < 0 || n_pad < n_rows || steps < 0) return set_error(PJDS_EINVAL, "bad arguments");
  *bytes = lanczos_bytes(n_rows, vec_dtype == PJDS_F64 ? 8 : 4, steps);
  return PJDS_OK;
}

extern "C" int pjds_lanczos(const pjds_dev *A, const void *v0, int32_t steps, double *alpha_host, double *beta_host,
                            void *basis, int32_t use_graph, void *work, size_t work_bytes, void *stream) {
  clear_error();
  int rc = check_square_permuted(A, "A");
  if (rc) return rc;
  if (steps <= 0 || steps > 100000) return set_error(PJDS_EINVAL, "steps must be in [1, 100000]");
  if (A->n_rows == 0) return set_error(PJDS_EINVAL, "empty matrix");
  if (!v0 || !alpha_host || !beta_host || !work) return set_error(PJDS_EINVAL, "a pointer argument is NULL");
  const int vb = vector_bytes(A->dtype);
  if (work_bytes < lanczos_bytes(A->n_rows, vb, steps)) return set_error(PJDS_EINVAL, "workspace too small");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (A->dtype == PJDS_F64)
    return lanczos_run<double>(A, static_cast<const double *>(v0), steps, alpha_host, beta_host,
                               static_cast<double *>(basis), use_graph, work, s);
  return lanczos_run<float>(A, static_cast<const float *>(v0), steps, alpha_host, beta_host,
                            static_cast<float *>(basis), use_graph, work, s);
}

// ----------------------------------------------------------------------------- tridiagonal eigenpair (host)

namespace {

// number of eigenvalues of T below t (LDL^T Sturm count)
int sturm_below(int32_t k, const double *a, const double *b, double t) {
  int cnt = 0;
  double d = a[0] - t;
  const double tiny = DBL_MIN * 1e3;
  for (int32_t i = 0;; ++i) {
    if (d == 0.0) d = -tiny;
    if (d < 0.0) ++cnt;
    if (i + 1 >= k) break;
    d = (a[i + 1] - t) - b[i + 1] * b[i + 1] / d;
  }
  return cnt;
}

// Solve (T - t I) z = rhs in place by Gaussian elimination with partial
// pivoting on the tridiagonal band (rows may swap with the next row).
void tridiag_solve_pivot(int32_t k, const double *a, const double *b, double t, double *z) {
  std::vector<double> d(k), du(k, 0.0), du2(k, 0.0), dl(k, 0.0);
  for (int32_t i = 0; i < k; ++i) d[i] = a[i] - t;
  for (int32_t i = 0; i + 1 < k; ++i) {
    du[i] = b[i + 1];
    dl[i] = b[i + 1];
  }
  const double eps = DBL_EPSILON * 4.0;
  double scale = 0.0;
  for (int32_t i = 0; i < k; ++i) scale = std::max(scale, fabs(a[i]) + (i ? fabs(b[i]) : 0.0));
  for (int32_t i = 0; i + 1 < k; ++i) {
    if (fabs(d[i]) >= fabs(dl[i])) {
      if (d[i] == 0.0) d[i] = eps * (scale > 0 ? scale : 1.0);
      const double f = dl[i] / d[i];
      d[i + 1] -= f * du[i];
      z[i + 1] -= f * z[i];
      dl[i] = 0.0;
    } else {  // swap rows i and i+1
      const double f = d[i] / dl[i];
      d[i] = dl[i];
      const double tmp = d[i + 1];
      d[i + 1] = du[i] - f * tmp;
      du[i] = tmp;
      if (i + 2 < k) {
        du2[i] = du[i + 1];
        du[i + 1] = -f * du2[i];
      }
      const double zt = z[i];
      z[i] = z[i + 1];
      z[i + 1] = zt - f * z[i + 1];
    }
  }
  if (d[k - 1] == 0.0) d[k - 1] = eps * (scale > 0 ? scale : 1.0);
  z[k - 1] /= d[k - 1];
  if (k > 1) z[k - 2] = (z[k - 2] - du[k - 2] * z[k - 1]) / d[k - 2];
  for (int32_t i = k - 3; i >= 0; --i) z[i] = (z[i] - du[i] * z[i + 1] - du2[i] * z[i + 2]) / d[i];
}

}  // namespace

extern "C" int pjds_tridiag_extreme(int32_t k, const double *alpha, const double *beta, int32_t which, double *theta,
                                    double *s) {
  clear_error();
  if (k <= 0 || !alpha || !beta || !theta) return set_error(PJDS_EINVAL, "bad arguments");
  double lo = alpha[0], hi = alpha[0];
  for (int32_t i = 0; i < k; ++i) {
    const double r = (i > 0 ? fabs(beta[i]) : 0.0) + (i + 1 < k ? fabs(beta[i + 1]) : 0.0);
    lo = std::min(lo, alpha[i] - r);
    hi = std::max(hi, alpha[i] + r);
  }
  const double span = std::max(hi - lo, DBL_MIN);
  lo -= 1e-12 * span;
  hi += 1e-12 * span;
  const int m = which == 0 ? k - 1 : 0;  // index of the wanted eigenvalue (ascending)
  for (int it = 0; it < 2000; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (sturm_below(k, alpha, beta, mid) > m)
      hi = mid;
    else
      lo = mid;
  }
  const double th = 0.5 * (lo + hi);
  *theta = th;
  if (s) {
    std::vector<double> z(k, 1.0);
    for (int it = 0; it < 4; ++it) {
      tridiag_solve_pivot(k, alpha, beta, th, z.data());
      double nrm = 0.0;
      for (double v : z) nrm += v * v;
      nrm = sqrt(nrm);
      if (!(nrm > 0.0) || !std::isfinite(nrm)) return set_error(PJDS_EINVAL, "inverse iteration failed");
      for (double &v : z) v /= nrm;
    }
    // sign convention: largest-magnitude component positive
    int32_t im = 0;
    for (int32_t i = 1; i < k; ++i)
      if (fabs(z[i]) > fabs(z[im])) im = i;
    const double sg = z[im] < 0 ? -1.0 : 1.0;
    for (int32_t i = 0; i < k; ++i) s[i] = sg * z[i];
  }
  return PJDS_OK;
}

// ----------------------------------------------------------------------------- Ritz refinement

static size_t ritz_bytes(int32_t n, int32_t k) {
  return align256((size_t)n_blocks_of(n) * 8) + align256(S_COUNT * 8) + align256((size_t)k * 8) +
         align256((size_t)n * 8);
}

extern "C" int pjds_ritz_workspace_bytes(int32_t n_rows, int32_t n_pad, int32_t k, size_t *bytes) {
  clear_error();
  if (!bytes || n_rows < 0 || n_pad < n_rows || k <= 0) return set_error(PJDS_EINVAL, "bad arguments");
  *bytes = ritz_bytes(n_rows, k);
  return PJDS_OK;
}

extern "C" int pjds_ritz_refine(const pjds_dev *A_hi, const void *basis, int32_t basis_dtype, int32_t k,
                                const double *s_host, double *y, double *theta, double *rel_residual, void *work,
                                size_t work_bytes, void *stream) {
  clear_error();
  int rc = check_square_permuted(A_hi, "A_hi");
  if (rc) return rc;
  if (A_hi->dtype != PJDS_F64) return set_error(PJDS_EINVAL, "A_hi must hold fp64 values");
  if (k <= 0 || !basis || !s_host || !y || !theta || !rel_residual || !work)
    return set_error(PJDS_EINVAL, "bad arguments");
  if (basis_dtype != PJDS_F64 && basis_dtype != PJDS_F32) return set_error(PJDS_EINVAL, "basis must be f64 or f32");
  const int32_t n = A_hi->n_rows, nb = n_blocks_of(n);
  if (n == 0) return set_error(PJDS_EINVAL, "empty matrix");
  if (work_bytes < ritz_bytes(n, k)) return set_error(PJDS_EINVAL, "workspace too small");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Carve cv{static_cast<char *>(work), 0, 0};
  double *partial = cv.take<double>((size_t)nb);
  double *scal = cv.take<double>(S_COUNT);
  double *sd = cv.take<double>((size_t)k);
  double *w = cv.take<double>((size_t)n);
  cudaError_t e = cudaMemcpyAsync(sd, s_host, sizeof(double) * (size_t)k, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(scal, 0, S_COUNT * sizeof(double), st);
  if (e != cudaSuccess) return set_error(PJDS_ECUDA, "ritz: %s", cudaGetErrorString(e));
  const Fin f_yy{partial, scal, nullptr, F_STORE, S_AUX0}, f_yw{partial, scal, nullptr, F_STORE, S_AUX1},
      f_ee{partial, scal, nullptr, F_STORE, S_AUX2};
  Dot<double, 0> dot;
  int32_t g_comb = 0, g_res = 0;
  if ((rc = make_dot(A_hi, &dot)) || (rc = red_grid(ritz_residual_kernel, n, &g_res)) ||
      (rc = basis_dtype == PJDS_F64 ? red_grid(ritz_combine_kernel<double>, n, &g_comb)
                                    : red_grid(ritz_combine_kernel<float>, n, &g_comb)))
    return rc;
  if (basis_dtype == PJDS_F64)
    ritz_combine_kernel<double><<<g_comb, KT, 0, st>>>(static_cast<const double *>(basis), sd, k, n, y, f_yy);
  else
    ritz_combine_kernel<float><<<g_comb, KT, 0, st>>>(static_cast<const float *>(basis), sd, k, n, y, f_yy);
  launch_dot(dot, A_hi, y, w, nullptr, f_yw, st);  // w = A y, (y, w)
  ritz_residual_kernel<<<g_res, KT, 0, st>>>(w, y, f_ee, n);
  if ((rc = launch_check("ritz refine"))) return rc;
  double h[3];
  e = cudaMemcpyAsync(h, scal + S_AUX0, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return set_error(PJDS_ECUDA, "ritz: %s", cudaGetErrorString(e));
  if (!(h[0] > 0.0)) return set_error(PJDS_EINVAL, "Ritz vector is zero");
  *theta = h[1] / h[0];
  *rel_residual = sqrt(h[2] / h[0]) / fabs(*theta);
  return PJDS_OK;
}

// ----------------------------------------------------------------------------- CG without any allocation

// pjds_cg_solve_static: the same solve as pjds_cg_solve, for callers that
// cannot provide a device workspace at all. Its workspace is this file-scope
// device array, which every GPU that loads the library holds until the
// process exits. The array's name is only a host-side stand-in in host code,
// so its device address is looked up once per device with
// cudaGetSymbolAddress and that address is handed to the kernels.
namespace pjds {
namespace kry {

constexpr int32_t CG_STATIC_MAX_ROWS = 131072;
constexpr size_t CG_STATIC_BYTES = (size_t)11 << 19;  // 5.5 MiB
static __device__ __align__(256) unsigned char g_cg_static_scratch[CG_STATIC_BYTES];

constexpr int kMaxDevices = 64;
static void *g_cg_static_ptr[kMaxDevices];
static std::mutex g_cg_static_mu;

// Device address of the static workspace on the current device (set up on
// the first call per device). The address is kept for the life of the
// process: after cudaDeviceReset the module is loaded again and the kept
// address no longer names the array, so the library must not be used across
// a reset of the device.
static int cg_static_workspace(void **out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_error(PJDS_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return set_error(PJDS_EINVAL, "device %d outside the supported range", dev);
  std::lock_guard<std::mutex> lock(g_cg_static_mu);
  if (!g_cg_static_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_cg_static_scratch);
    if (e != cudaSuccess || !p)
      return set_error(PJDS_ECUDA, "cudaGetSymbolAddress of the static workspace: %s", cudaGetErrorString(e));
    g_cg_static_ptr[dev] = p;
  }
  *out = g_cg_static_ptr[dev];
  return PJDS_OK;
}

}  // namespace kry
}  // namespace pjds

extern "C" int pjds_cg_solve_static(const pjds_dev *A_hi, const pjds_dev *A_lo, const double *b, double *x,
                                    const pjds_cg_opts *opts, pjds_cg_result *res, void *stream) {
  clear_error();
  int rc = check_square_permuted(A_hi, "A_hi");
  if (rc) return rc;
  if (A_hi->dtype != PJDS_F64) return set_error(PJDS_EINVAL, "A_hi must hold fp64 values");
  if (!A_lo) A_lo = A_hi;
  if ((rc = check_square_permuted(A_lo, "A_lo"))) return rc;
  if (A_lo->n_rows != A_hi->n_rows) return set_error(PJDS_EINVAL, "A_lo and A_hi differ in size");
  if (A_hi->n_rows > CG_STATIC_MAX_ROWS)
    return set_error(PJDS_EINVAL,
                     "pjds_cg_solve_static handles at most %d rows (got %d); use pjds_cg_solve with a workspace",
                     CG_STATIC_MAX_ROWS, A_hi->n_rows);
  if (A_hi->n_rows == 0) return PJDS_OK;
  if (!b || !x) return set_error(PJDS_EINVAL, "b or x is NULL");
  pjds_cg_opts o{6, 50, 0.0, 1, 0};
  if (opts) {
    o = *opts;
    if (o.max_outer <= 0) o.max_outer = 6;
    if (o.inner_iters <= 0) o.inner_iters = 50;
  }
  if (o.inner_iters > 100000 || o.max_outer > 100000) return set_error(PJDS_EINVAL, "iteration counts too large");
  // The inner steps are always launched one by one on the caller's stream:
  // recording them into a CUDA graph would create a stream and an executable
  // graph, driver objects this entry point promises not to create.
  o.use_graph = 0;
  const bool low = A_lo->dtype != PJDS_F64;
  const size_t need = cg_bytes(A_hi->n_rows, low ? 4 : 8);
  if (need > CG_STATIC_BYTES)
    return set_error(PJDS_EINVAL, "static workspace of %zu bytes is smaller than %zu", CG_STATIC_BYTES, need);
  void *work = nullptr;
  if ((rc = cg_static_workspace(&work))) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // The array keeps the previous call's contents: clear the partial sums and
  // the scalar block; every vector is written before it is read.
  const size_t head = align256((size_t)n_blocks_of(A_hi->n_rows) * 8) + align256(S_COUNT * 8);
  cudaError_t e = cudaMemsetAsync(work, 0, head, s);
  if (e != cudaSuccess) return set_error(PJDS_ECUDA, "clear static workspace: %s", cudaGetErrorString(e));
  return low ? cg_run<float>(A_hi, A_lo, b, x, o, res, work, s) : cg_run<double>(A_hi, A_lo, b, x, o, res, work, s);
}
