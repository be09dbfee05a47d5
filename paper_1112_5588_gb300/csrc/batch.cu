// Batched pJDS products (include/pjds_batch.h): the block product Y = A X for
// k right-hand sides, and one persistent launch over many matrices.
#include <string.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "common.h"
#include "pjds_batch.h"
#include "spmv_kernels.cuh"
#include "plan.h"
#include "tiles.cuh"

namespace pjds {
namespace bat {

using pjds::tiles::BT;  // threads per CTA

// 16-byte vectors of the vector type
template <typename TX>
struct V16;
template <>
struct V16<float> {
  static constexpr int W = 4;
  __device__ static void load(const float *p, float (&v)[4]) {
    const float4 a = __ldg(reinterpret_cast<const float4 *>(p));
    v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w;
  }
  __device__ static void store(float *p, const float (&v)[4]) {
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
};
template <>
struct V16<double> {
  static constexpr int W = 2;
  __device__ static void load(const double *p, double (&v)[2]) {
    const double2 a = __ldg(reinterpret_cast<const double2 *>(p));
    v[0] = a.x, v[1] = a.y;
  }
  __device__ static void store(double *p, const double (&v)[2]) {
    *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
  }
};

// Thread t: sorted row i = t / lr and, of its k columns, the CH 16-byte chunks
// [q W, q W + W), W = CH * (elements per chunk), q = t % lr (lr = k / W lanes
// per row). Wider lanes spread the loads of col_start, col and val and the
// address arithmetic over more fused multiply-adds. Row offsets into X and Y
// are 32-bit indices widened in the multiply (one wide multiply-add each).
// PAT: the pattern product Y = S X (every stored value taken as 1, the
// matrix's values not read): val is the address of eight ones
// (dev::pattern_ones_address), read where the product reads its values, so
// the kernel keeps the product's instructions, registers and occupancy and
// only the value stream is missing; fma(1, x, acc) is acc + x rounded once.
template <typename TV, typename TX, typename IDX, bool SCATTER, int CH, bool PAT = false>
__global__ void __launch_bounds__(BT)
    spmm_kernel(const TV *__restrict__ val, const int32_t *__restrict__ col, const int64_t *__restrict__ col_start,
                const int32_t *__restrict__ block_len, const int32_t *__restrict__ perm, const TX *__restrict__ X,
                TX *__restrict__ Y, int32_t n_rows, int32_t b, int32_t k, int32_t lr) {
  using TA = typename dev::Acc<TV>::T;
  constexpr int VW = V16<TX>::W, W = VW * CH, U = 4;
  const int64_t t = (int64_t)blockIdx.x * BT + threadIdx.x;
  const int64_t i = t / lr;
  const int32_t q = (int32_t)(t % lr);
  if (i >= n_rows) return;
  const int32_t L = PJDS_IN(i / b, PJDS_EXT(n_blocks), dev::CHK_BLOCK) ? __ldg(block_len + (int32_t)(i / b)) : 0;
  TA acc[W];
#pragma unroll
  for (int w = 0; w < W; ++w) acc[w] = TA(0);
  for (int32_t j = 0; j < L; j += U) {
    int32_t c[U];
    TV v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (j + u < L && PJDS_IN(j + u, PJDS_EXT(n_diag), dev::CHK_DIAG)) {
        const IDX o = (IDX)__ldg(col_start + j + u) + (IDX)i;
#ifdef PJDS_CHECKED
        if (!PJDS_IN(o, PJDS_EXT(stored), dev::CHK_OFFSET)) {
          c[u] = -1;
          v[u] = TV{};
          continue;
        }
#endif
        c[u] = __ldcs(col + o);
        v[u] = dev::ld_stream1(PAT ? val + dev::pattern_slot(val + o) : val + o);  // PAT: val holds the ones
      } else {
        c[u] = -1;
        v[u] = TV{};
      }
    }
    TX xv[U][W];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (c[u] >= 0 && PJDS_IN(c[u], PJDS_EXT(n_cols), dev::CHK_COLUMN)) {
#pragma unroll
        for (int h = 0; h < CH; ++h)
          V16<TX>::load(X + (int64_t)c[u] * k + (int64_t)q * W + h * VW,
                        *reinterpret_cast<TX(*)[VW]>(&xv[u][h * VW]));
      } else {
#pragma unroll
        for (int w = 0; w < W; ++w) xv[u][w] = TX(0);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int w = 0; w < W; ++w)
        acc[w] = c[u] >= 0 ? dev::fma_acc(dev::to_acc(v[u]), (TA)xv[u][w], acc[w]) : acc[w];
  }
  TX out[W];
#pragma unroll
  for (int w = 0; w < W; ++w) out[w] = (TX)acc[w];
  const int64_t r = SCATTER ? (int64_t)__ldcs(perm + i) : i;
  if (!PJDS_IN(r, PJDS_EXT(n_rows), dev::CHK_ROW)) return;
#pragma unroll
  for (int h = 0; h < CH; ++h)
    V16<TX>::store(Y + r * k + (int64_t)q * W + h * VW, *reinterpret_cast<const TX(*)[VW]>(&out[h * VW]));
}

// The pattern product's value address reduced to a slot of the ones (0 for
// every address the product reads), opaque to the compiler like
// dev::pattern_slot but without a volatile asm: a volatile statement also
// fixes its place in the schedule, which kept the paired kernel's loads of a
// round from interleaving (its pattern product of bf16 values at k = 32 ran
// 16% slower than the product itself).
template <typename TV>
__device__ __forceinline__ int pair_pattern_slot(const TV *p) {
  asm("" : "+l"(p));
  return (int)(reinterpret_cast<uintptr_t>(p) & 3);
}

// Two of the pattern product's ones, through L1 with the normal eviction priority.
__device__ __forceinline__ void ld_ones2(const double *p, double (&v)[2]) {
  const double2 a = __ldg(reinterpret_cast<const double2 *>(p));
  v[0] = a.x, v[1] = a.y;
}
__device__ __forceinline__ void ld_ones2(const float *p, float (&v)[2]) {
  const float2 a = __ldg(reinterpret_cast<const float2 *>(p));
  v[0] = a.x, v[1] = a.y;
}
__device__ __forceinline__ void ld_ones2(const dev::bf16_t *p, dev::bf16_t (&v)[2]) {
  const unsigned int a = __ldg(reinterpret_cast<const unsigned int *>(p));
  v[0].bits = (uint16_t)(a & 0xFFFFu);
  v[1].bits = (uint16_t)(a >> 16);
}

// Paired rows: thread t takes sorted rows 2p and 2p + 1 (p = t / lr) and the
// same CH chunks of their k columns as spmm_kernel. Where the two rows have
// the same column at a jagged diagonal (block-structured matrices), one
// gather of the X row serves both; otherwise row 2p + 1 gathers its own.
// Each row sums in the order and with the fused multiply-adds of
// spmm_kernel. Row 2p is at least as long as row 2p + 1 (sorted order), so
// a pad of the first is a pad of the second.
template <typename TV, typename TX, typename IDX, bool SCATTER, int CH, int U, bool PAT = false>
__global__ void __launch_bounds__(BT)
    spmm_pair_kernel(const TV *__restrict__ val, const int32_t *__restrict__ col, const int64_t *__restrict__ col_start,
                     const int32_t *__restrict__ block_len, const int32_t *__restrict__ perm, const TX *__restrict__ X,
                     TX *__restrict__ Y, int32_t n_rows, int32_t b, int32_t k, int32_t lr) {
  using TA = typename dev::Acc<TV>::T;
  constexpr int VW = V16<TX>::W, W = VW * CH;
  const int64_t t = (int64_t)blockIdx.x * BT + threadIdx.x;
  const int64_t i = 2 * (t / lr);
  const int32_t q = (int32_t)(t % lr);
  if (i >= n_rows) return;
  const int32_t L = PJDS_IN(i / b, PJDS_EXT(n_blocks), dev::CHK_BLOCK) ? __ldg(block_len + (int32_t)(i / b)) : 0;
  TA acc0[W], acc1[W];
#pragma unroll
  for (int w = 0; w < W; ++w) acc0[w] = acc1[w] = TA(0);
  for (int32_t j = 0; j < L; j += U) {
    int32_t c[U][2];
    TV v[U][2];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      bool live = j + u < L && PJDS_IN(j + u, PJDS_EXT(n_diag), dev::CHK_DIAG);
      IDX o = 0;
      if (live) {
        o = (IDX)__ldg(col_start + j + u) + (IDX)i;
        live = PJDS_IN(o, PJDS_EXT(stored), dev::CHK_OFFSET) && PJDS_IN((int64_t)o + 1, PJDS_EXT(stored), dev::CHK_OFFSET);
      }
      if (live) {
        dev::ld_stream<2>(col + o, c[u]);
        if constexpr (PAT)
          ld_ones2(val + pair_pattern_slot(val + o), v[u]);  // val holds the ones
        else
          dev::ld_stream<2>(val + o, v[u]);
      } else {
        c[u][0] = c[u][1] = -1;
        v[u][0] = v[u][1] = TV{};
      }
    }
    TX xv[U][W];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (c[u][0] >= 0 && PJDS_IN(c[u][0], PJDS_EXT(n_cols), dev::CHK_COLUMN)) {
#pragma unroll
        for (int h = 0; h < CH; ++h)
          V16<TX>::load(X + (int64_t)c[u][0] * k + (int64_t)q * W + h * VW,
                        *reinterpret_cast<TX(*)[VW]>(&xv[u][h * VW]));
      } else {
#pragma unroll
        for (int w = 0; w < W; ++w) xv[u][w] = TX(0);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
#pragma unroll
      for (int w = 0; w < W; ++w)
        acc0[w] = c[u][0] >= 0 ? dev::fma_acc(dev::to_acc(v[u][0]), (TA)xv[u][w], acc0[w]) : acc0[w];
      if (c[u][1] == c[u][0]) {
#pragma unroll
        for (int w = 0; w < W; ++w)
          acc1[w] = c[u][1] >= 0 ? dev::fma_acc(dev::to_acc(v[u][1]), (TA)xv[u][w], acc1[w]) : acc1[w];
      } else if (c[u][1] >= 0 && PJDS_IN(c[u][1], PJDS_EXT(n_cols), dev::CHK_COLUMN)) {
        TX x1[W];
#pragma unroll
        for (int h = 0; h < CH; ++h)
          V16<TX>::load(X + (int64_t)c[u][1] * k + (int64_t)q * W + h * VW, *reinterpret_cast<TX(*)[VW]>(&x1[h * VW]));
#pragma unroll
        for (int w = 0; w < W; ++w) acc1[w] = dev::fma_acc(dev::to_acc(v[u][1]), (TA)x1[w], acc1[w]);
      }
    }
  }
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int64_t ir = i + r;
    if (ir >= n_rows) break;
    TX out[W];
#pragma unroll
    for (int w = 0; w < W; ++w) out[w] = (TX)(r == 0 ? acc0[w] : acc1[w]);
    const int64_t row = SCATTER ? (int64_t)__ldcs(perm + ir) : ir;
    if (!PJDS_IN(row, PJDS_EXT(n_rows), dev::CHK_ROW)) continue;
#pragma unroll
    for (int h = 0; h < CH; ++h)
      V16<TX>::store(Y + row * k + (int64_t)q * W + h * VW, *reinterpret_cast<const TX(*)[VW]>(&out[h * VW]));
  }
}

// ----------------------------------------------------------------------------- persistent batch

using namespace pjds::tiles;


// CTAs take tiles (matrix, first sorted row, rows, lanes per row) from a work
// counter until none is left: tiles of one lane per row have one row per
// thread, tiles of 2, 4 or 8 lanes per row BT / lanes rows. No CTA ever waits
// for another.
// PAT: the pattern products of every matrix (ones: the address of eight
// ones, read in place of each matrix's values; see run_tile).
template <typename TV, typename TX, bool PAT = false>
__device__ __forceinline__ void
    batch_body(const Desc *__restrict__ descs, const int4 *__restrict__ tiles, int32_t n_tiles,
                 int32_t *__restrict__ counter, const void *ones) {
  __shared__ int32_t s_tile;
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(counter, 1);
    __syncthreads();
    const int32_t t = s_tile;
    __syncthreads();
    if (t >= n_tiles) return;
    const int4 tl = tiles[t];
    Desc d = descs[tl.x];
    if constexpr (PAT) d.val = ones;
    run_tile<TV, TX, PAT>(d, tl);
  }
}

template <typename TV, typename TX, bool PAT = false>
__global__ void __launch_bounds__(BT)
    batch_kernel(const Desc *__restrict__ descs, const int4 *__restrict__ tiles, int32_t n_tiles,
                 int32_t *__restrict__ counter, const void *ones) {
  batch_body<TV, TX, PAT>(descs, tiles, n_tiles, counter, ones);
}

// fp64 values: six resident CTAs per SM. Without the bound the four-row path
// takes the kernel from 40 to 48 registers and five CTAs per SM (253 against
// 237 us on the Zipf batch); fp32 and bf16 stay at 40 registers unbounded,
// while the same bound made fp32 spill (222 against 214 us).
template <bool PAT = false>
__global__ void __launch_bounds__(BT, 6)
    batch_kernel_f64(const Desc *__restrict__ descs, const int4 *__restrict__ tiles, int32_t n_tiles,
                     int32_t *__restrict__ counter, const void *ones) {
  batch_body<double, double, PAT>(descs, tiles, n_tiles, counter, ones);
}

static inline size_t a256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace bat

// The batched launch's translation unit's check word (checked build).
int check_word_batch(unsigned long long *w, bool clear, cudaStream_t s) {
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

using namespace pjds;
using namespace pjds::bat;

struct pjds_batch {
  int32_t dtype, n_mats, n_tiles, n_ctas;
  int32_t *counter;
  const Desc *descs;
  const int4 *tiles;
  cudaGraphExec_t exec;
};

// ----------------------------------------------------------------------------- spmm

// Chunks per lane, from a GB300 sweep (DLR-like, HMEp-like and Zipf
// matrices, k = 2..64): two chunks when that still leaves at least 2 lanes
// per row and n_rows * lanes >= 2^19 threads (DLR-like fp32, k = 32: 1.5x
// faster than one chunk), one chunk when the longest row has more than 4
// times the mean length (the longest rows' latency then sets the time and
// more lanes per row help) or otherwise. Four chunks were within 4% of two
// at best and are not built. Paired rows (shared_pairs: block-structured
// matrices, fp32 / bf16, k >= 8) run spmm_pair_kernel with two chunks:
// DLR-like matrices of 280k and 560k rows, against spmm_kernel, bf16
// 0.57-0.73 of the time (k = 8..64), fp32 0.85-0.92 at k = 8 and 0.87-0.94
// at k = 64, but 0.98-1.03 at k = 16 and 32 (not paired there); one chunk
// per lane, or fp64 values (bound by the fp64 pipe), gained nothing.
static int spmm_chunks(const pjds_dev *A, int32_t k, int vw) {
  if ((int64_t)A->n_max * A->n_rows > 4 * A->nnz) return 1;
  const int32_t lanes = k % (2 * vw) == 0 ? k / (2 * vw) : 0;
  return lanes >= 2 && (int64_t)A->n_rows * lanes >= (1 << 19) ? 2 : 1;
}

template <typename TV, typename TX, bool PAT = false>
static int launch_spmm(const pjds_dev *A, int32_t k, const void *X, void *Y, cudaStream_t s) {
  constexpr int VW = V16<TX>::W;
  int ch = spmm_chunks(A, k, VW), pair_u = 0;
  // block-structured matrices: one thread per pair of rows sharing their
  // columns, two chunks per lane (bf16 from k = 8, fp32 at k = 8 and from
  // k = 64); 4 jagged diagonals per round for bf16 values from k = 16, else 2
  const bool pair_k = A->dtype == PJDS_BF16 ? k >= 8 : (k == 8 || k >= 64);
  if (A->dtype != PJDS_F64 && shared_pairs(A) && pair_k && k % (2 * VW) == 0) {
    ch = 2;
    pair_u = A->dtype == PJDS_BF16 && k >= 16 ? 4 : 2;
  }
  const int32_t lr = k / (VW * ch);
  const int64_t threads = (pair_u ? ((int64_t)A->n_rows + 1) / 2 : (int64_t)A->n_rows) * lr;
  const int64_t grid = (threads + BT - 1) / BT;
  if (grid <= 0) return PJDS_OK;
  if (grid > 0x7fffffffLL) return set_error(PJDS_EOVERFLOW, "grid too large");
  const TV *val = static_cast<const TV *>(A->val);
  if constexpr (PAT) {
    const void *ones = nullptr;
    const cudaError_t e = dev::pattern_ones_address<TV>(&ones);
    if (e != cudaSuccess) return set_error(PJDS_ECUDA, "pattern values: %s", cudaGetErrorString(e));
    val = static_cast<const TV *>(ones);
  }
  const TX *x = static_cast<const TX *>(X);
  TX *y = static_cast<TX *>(Y);
  const bool small = A->n_stored + A->n_pad < 0x7fffffffLL, sc = !A->permute_cols;
#ifdef PJDS_CHECKED
  dev::set_extents(dev::Extents{A->n_stored, A->n_cols, A->n_rows, A->n_blocks, A->n_max + 1}, s);
#endif
#define SPMM(IDX, SC, CH)                                                                                        \
  spmm_kernel<TV, TX, IDX, SC, CH, PAT><<<(unsigned)grid, BT, 0, s>>>(val, A->col, A->col_start, A->block_len,    \
                                                                       A->perm, \
                                                                  x, y, A->n_rows, A->b, k, lr)
#define SPMM_CH(IDX, SC) \
  do {                   \
    if (ch == 2)         \
      SPMM(IDX, SC, 2);  \
    else                 \
      SPMM(IDX, SC, 1);  \
  } while (0)
#define SPMMP(IDX, SC, CH, UU)                                                                                 \
  spmm_pair_kernel<TV, TX, IDX, SC, CH, UU, PAT><<<(unsigned)grid, BT, 0, s>>>(val, A->col, A->col_start,        \
                                                                            A->block_len, A->perm, x, y, A->n_rows, \
                                                                            A->b, k, lr)
#define SPMMP_CH(IDX, SC)      \
  do {                         \
    if (pair_u == 2)           \
      SPMMP(IDX, SC, 2, 2);    \
    else                       \
      SPMMP(IDX, SC, 2, 4);    \
  } while (0)
  if (pair_u) {
    if (small) {
      if (sc) SPMMP_CH(int32_t, true);
      else SPMMP_CH(int32_t, false);
    } else {
      if (sc) SPMMP_CH(int64_t, true);
      else SPMMP_CH(int64_t, false);
    }
  } else if (small) {
    if (sc) SPMM_CH(int32_t, true);
    else SPMM_CH(int32_t, false);
  } else {
    if (sc) SPMM_CH(int64_t, true);
    else SPMM_CH(int64_t, false);
  }
#undef SPMMP_CH
#undef SPMMP
#undef SPMM_CH
#undef SPMM
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? PJDS_OK : set_error(PJDS_ECUDA, "pjds_spmm launch: %s", cudaGetErrorString(e));
}

template <bool PAT>
static int spmm_entry(const pjds_dev *A, int32_t k, const void *X, void *Y, void *stream) {
  clear_error();
  if (!A) return set_error(PJDS_EINVAL, "A is NULL");
  if (value_bytes(A->dtype) == 0) return set_error(PJDS_EINVAL, "unknown dtype %d", A->dtype);
  if (k == 1 && !PAT) return pjds_spmv(A, X, Y, stream);
  if (k == 1) return set_error(PJDS_EINVAL, "k = 1: use pjds_spmv_pattern");
  const int w = A->dtype == PJDS_F64 ? 2 : 4;
  if (k < w || k % w || k > 32 * w)
    return set_error(PJDS_EINVAL, "k = %d: use 1 or a multiple of %d up to %d", k, w, 32 * w);
  if (A->n_rows < 0 || A->n_cols < 1 || A->b <= 0 || A->b % 32 ||
      (int64_t)A->n_pad != ((int64_t)A->n_rows + A->b - 1) / A->b * A->b)
    return set_error(PJDS_EINVAL, "inconsistent matrix sizes");
  if (A->n_rows == 0) return PJDS_OK;
  if (!X || !Y) return set_error(PJDS_EINVAL, "X or Y is NULL");
  if (((uintptr_t)X | (uintptr_t)Y) & 15) return set_error(PJDS_EINVAL, "X and Y must be 16-byte aligned");
  if (A->n_stored > 0 && (!A->val || !A->col || !A->col_start || !A->block_len))
    return set_error(PJDS_EINVAL, "a matrix array is NULL");
  if (!A->permute_cols && !A->perm) return set_error(PJDS_EINVAL, "perm is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (A->n_stored == 0) {
    cudaError_t e = cudaMemsetAsync(Y, 0, (size_t)A->n_rows * k * vector_bytes(A->dtype), s);
    return e == cudaSuccess ? PJDS_OK : set_error(PJDS_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
  }
  switch (A->dtype) {
    case PJDS_F64: return launch_spmm<double, double, PAT>(A, k, X, Y, s);
    case PJDS_F32: return launch_spmm<float, float, PAT>(A, k, X, Y, s);
    default: return launch_spmm<dev::bf16_t, float, PAT>(A, k, X, Y, s);
  }
}

extern "C" int pjds_spmm(const pjds_dev *A, int32_t k, const void *X, void *Y, void *stream) {
  return spmm_entry<false>(A, k, X, Y, stream);
}

extern "C" int pjds_spmm_pattern(const pjds_dev *A, int32_t k, const void *X, void *Y, void *stream) {
  return spmm_entry<true>(A, k, X, Y, stream);
}

// ----------------------------------------------------------------------------- batch

// upper bound of a matrix's tiles (plan_cut)
static int64_t tiles_of(const pjds_dev &A) { return plan_max_tiles(A.n_rows); }

extern "C" int pjds_batch_plan_bytes(int32_t n_mats, const pjds_dev *mats, size_t *bytes) {
  clear_error();
  if (n_mats <= 0 || !mats || !bytes) return set_error(PJDS_EINVAL, "bad arguments");
  int64_t nt = 0;
  for (int32_t m = 0; m < n_mats; ++m) nt += tiles_of(mats[m]);
  *bytes = a256(sizeof(int32_t)) + a256(sizeof(Desc) * (size_t)n_mats) + a256(sizeof(int4) * (size_t)nt);
  return PJDS_OK;
}

// Plan: per matrix either fixed lanes (lanes[m] > 0) or the block-length
// rule min_len (2, 4 or 8 lanes from block lengths min_len[0], [1], [2]).
static int batch_plan(int32_t n_mats, const pjds_dev *mats, const void *const *xs, void *const *ys,
                      const int32_t *lanes, const int32_t *min_len, void *plan_dev, size_t plan_bytes,
                      pjds_batch **out, void *stream) {
  if (n_mats <= 0 || !mats || !xs || !ys || !plan_dev || !out) return set_error(PJDS_EINVAL, "bad arguments");
  if (lanes)
    for (int32_t m = 0; m < n_mats; ++m)
      if (lanes[m] != 0 && lanes[m] != 1 && lanes[m] != 2 && lanes[m] != 4 && lanes[m] != 8)
        return set_error(PJDS_EINVAL, "lanes[%d] = %d: use 0, 1, 2, 4 or 8", m, lanes[m]);
  for (int k = 0; k < 3; ++k)
    if (min_len[k] < 1) return set_error(PJDS_EINVAL, "min_len[%d] = %d must be positive", k, min_len[k]);
  *out = nullptr;
  size_t need = 0;
  int rc = pjds_batch_plan_bytes(n_mats, mats, &need);
  if (rc) return rc;
  if (plan_bytes < need) return set_error(PJDS_EINVAL, "plan buffer of %zu bytes is smaller than %zu", plan_bytes, need);
  const int32_t dt = mats[0].dtype;
  if (value_bytes(dt) == 0) return set_error(PJDS_EINVAL, "unknown dtype");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<Desc> descs((size_t)n_mats);
  struct T {
    int32_t m, row0, rows, lanes;
    int64_t cost;
  };
  std::vector<T> tiles;
  for (int32_t m = 0; m < n_mats; ++m) {
    const pjds_dev &A = mats[m];
    if (A.dtype != dt) return set_error(PJDS_EINVAL, "matrix %d has another dtype than matrix 0", m);
    if (A.n_rows < 0 || A.b <= 0 || A.b % 32 || (int64_t)A.n_pad != ((int64_t)A.n_rows + A.b - 1) / A.b * A.b)
      return set_error(PJDS_EINVAL, "matrix %d: inconsistent sizes", m);
    if (A.n_rows > 0 && (!xs[m] || !ys[m])) return set_error(PJDS_EINVAL, "matrix %d: x or y is NULL", m);
    if (A.n_stored > 0 && (!A.val || !A.col || !A.col_start || !A.block_len))
      return set_error(PJDS_EINVAL, "matrix %d: a matrix array is NULL", m);
    if (A.n_rows > 0 && !A.permute_cols && !A.perm) return set_error(PJDS_EINVAL, "matrix %d: perm is NULL", m);
    Desc &d = descs[(size_t)m];
    d.val = A.val;
    d.col = A.col;
    d.col_start = A.col_start;
    d.block_len = A.block_len;
    d.perm = A.perm;
    d.x = xs[m];
    d.y = ys[m];
    d.n_rows = A.n_rows;
    d.b = A.b;
    d.scatter = A.permute_cols ? 0 : 1;
    d.idx64 = A.n_stored + A.n_pad < 0x7fffffffLL ? 0 : 1;
    d.stored = A.n_stored;
    d.n_cols = A.n_cols;
    d.n_blocks = A.n_blocks;
    d.n_diag = A.n_max + 1;
    d.reserved = 0;
    if (A.n_rows == 0) continue;
    // block lengths back to the host once, to weigh the tiles
    std::vector<int32_t> bl((size_t)A.n_blocks);
    cudaError_t e = cudaMemcpyAsync(bl.data(), A.block_len, sizeof(int32_t) * bl.size(), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return set_error(PJDS_ECUDA, "read block lengths: %s", cudaGetErrorString(e));
    // one-lane tiles of the rule take two adjacent rows per thread when val
    // and col allow the paired loads, four when they allow 16-byte loads
    const int32_t fixed = lanes ? lanes[m] : 0;
    const bool pair = !fixed && ((uintptr_t)A.val % (2 * value_bytes(dt))) == 0 && ((uintptr_t)A.col % 8) == 0;
    const bool quad = pair && ((uintptr_t)A.val % 16) == 0 && ((uintptr_t)A.col % 16) == 0;
    const PlanRule rule = {{min_len[0], min_len[1], min_len[2]}, k_plan_rule.quad_max_len};
    std::vector<PlanTile> cut;
    plan_cut(A.n_rows, A.b, bl.data(), rule, fixed, pair, quad, cut);
    for (const PlanTile &c : cut) tiles.push_back(T{m, c.row0, c.rows, c.kind, c.cost});
  }
  // matrices by total work per lane (largest first), tiles by work per lane
  // inside each matrix: the CTAs share one or two matrices' x at a time
  std::vector<int64_t> mcost((size_t)n_mats, 0);
  for (const T &t : tiles) mcost[(size_t)t.m] += t.cost;
  std::stable_sort(tiles.begin(), tiles.end(), [&](const T &a, const T &b) {
    if (a.m != b.m) {
      const int64_t ca = mcost[(size_t)a.m], cb = mcost[(size_t)b.m];
      return ca != cb ? ca > cb : a.m < b.m;
    }
    return a.cost > b.cost;
  });
  int64_t bound = 0;
  for (int32_t m = 0; m < n_mats; ++m) bound += tiles_of(mats[m]);
  if ((int64_t)tiles.size() > bound)
    return set_error(PJDS_EINVAL, "plan of %zu tiles exceeds the %lld the plan buffer holds", tiles.size(),
                     (long long)bound);
  std::vector<int4> tl(tiles.size());
  for (size_t i = 0; i < tiles.size(); ++i) tl[i] = make_int4(tiles[i].m, tiles[i].row0, tiles[i].rows, tiles[i].lanes);
  char *p = static_cast<char *>(plan_dev);
  int32_t *counter = reinterpret_cast<int32_t *>(p);
  Desc *dd = reinterpret_cast<Desc *>(p + a256(sizeof(int32_t)));
  int4 *td = reinterpret_cast<int4 *>(p + a256(sizeof(int32_t)) + a256(sizeof(Desc) * (size_t)n_mats));
  cudaError_t e = cudaMemcpyAsync(dd, descs.data(), sizeof(Desc) * descs.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && !tl.empty())
    e = cudaMemcpyAsync(td, tl.data(), sizeof(int4) * tl.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return set_error(PJDS_ECUDA, "upload plan: %s", cudaGetErrorString(e));
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (dt == PJDS_F64)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel_f64<false>, BT, 0);
  else if (dt == PJDS_F32)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<float, float>, BT, 0);
  else
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<dev::bf16_t, float>, BT, 0);
  if (e != cudaSuccess) return set_error(PJDS_ECUDA, "occupancy: %s", cudaGetErrorString(e));
  pjds_batch *h = static_cast<pjds_batch *>(calloc(1, sizeof(pjds_batch)));
  if (!h) return set_error(PJDS_ENOMEM, "out of host memory");
  h->dtype = dt;
  h->n_mats = n_mats;
  h->n_tiles = (int32_t)tl.size();
  h->n_ctas = std::max(1, std::min(sms * std::max(per_sm, 1), std::max(h->n_tiles, 1)));
  h->counter = counter;
  h->descs = dd;
  h->tiles = td;
  h->exec = nullptr;
  *out = h;
  return PJDS_OK;
}

// the built-in rule: 2 lanes per row from block length 16, 4 from 64, 8 from
// 256 (the fastest of the tuner's candidate rules on 64 uneven Zipf
// matrices: 253 us against 281 us for 8 lanes from 64 and one below)
static const int32_t k_default_rule[3] = {k_plan_rule.min_len[0], k_plan_rule.min_len[1], k_plan_rule.min_len[2]};

extern "C" int pjds_batch_create(int32_t n_mats, const pjds_dev *mats, const void *const *xs, void *const *ys,
                                 void *plan_dev, size_t plan_bytes, pjds_batch **out, void *stream) {
  clear_error();
  return batch_plan(n_mats, mats, xs, ys, nullptr, k_default_rule, plan_dev, plan_bytes, out, stream);
}

extern "C" int pjds_batch_create_lanes(int32_t n_mats, const pjds_dev *mats, const void *const *xs,
                                       void *const *ys, const int32_t *lanes, void *plan_dev, size_t plan_bytes,
                                       pjds_batch **out, void *stream) {
  clear_error();
  return batch_plan(n_mats, mats, xs, ys, lanes, k_default_rule, plan_dev, plan_bytes, out, stream);
}

extern "C" int pjds_batch_create_rule(int32_t n_mats, const pjds_dev *mats, const void *const *xs,
                                      void *const *ys, const int32_t *min_len, void *plan_dev, size_t plan_bytes,
                                      pjds_batch **out, void *stream) {
  clear_error();
  if (!min_len) return set_error(PJDS_EINVAL, "min_len is NULL");
  return batch_plan(n_mats, mats, xs, ys, nullptr, min_len, plan_dev, plan_bytes, out, stream);
}

template <bool PAT = false>
static int batch_issue(pjds_batch *h, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(h->counter, 0, sizeof(int32_t), s);
  if (e != cudaSuccess) return set_error(PJDS_ECUDA, "reset counter: %s", cudaGetErrorString(e));
  const void *ones = nullptr;
  if constexpr (PAT) {
    e = h->dtype == PJDS_F64   ? dev::pattern_ones_address<double>(&ones)
        : h->dtype == PJDS_F32 ? dev::pattern_ones_address<float>(&ones)
                               : dev::pattern_ones_address<dev::bf16_t>(&ones);
    if (e != cudaSuccess) return set_error(PJDS_ECUDA, "pattern values: %s", cudaGetErrorString(e));
  }
  if (h->dtype == PJDS_F64)
    batch_kernel_f64<PAT><<<h->n_ctas, BT, 0, s>>>(h->descs, h->tiles, h->n_tiles, h->counter, ones);
  else if (h->dtype == PJDS_F32)
    batch_kernel<float, float, PAT><<<h->n_ctas, BT, 0, s>>>(h->descs, h->tiles, h->n_tiles, h->counter, ones);
  else
    batch_kernel<dev::bf16_t, float, PAT>
        <<<h->n_ctas, BT, 0, s>>>(h->descs, h->tiles, h->n_tiles, h->counter, ones);
  e = cudaGetLastError();
  return e == cudaSuccess ? PJDS_OK : set_error(PJDS_ECUDA, "batch launch: %s", cudaGetErrorString(e));
}

extern "C" int pjds_batch_run(pjds_batch *h, int32_t use_graph, void *stream) {
  clear_error();
  if (!h) return set_error(PJDS_EINVAL, "h is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (h->n_tiles == 0) return PJDS_OK;
  if (!use_graph) return batch_issue(h, s);
  if (!h->exec) {
    cudaStream_t cap = nullptr;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return set_error(PJDS_ECUDA, "graph stream: %s", cudaGetErrorString(e));
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    int rc = PJDS_OK;
    if (e == cudaSuccess) {
      rc = batch_issue(h, cap);
      e = cudaStreamEndCapture(cap, &g);
    }
    if (rc == PJDS_OK && e == cudaSuccess) e = cudaGraphInstantiate(&h->exec, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cap);
    if (rc != PJDS_OK) return rc;
    if (e != cudaSuccess) {
      h->exec = nullptr;
      return set_error(PJDS_ECUDA, "batch graph: %s", cudaGetErrorString(e));
    }
  }
  cudaError_t e = cudaGraphLaunch(h->exec, s);
  return e == cudaSuccess ? PJDS_OK : set_error(PJDS_ECUDA, "batch graph launch: %s", cudaGetErrorString(e));
}

extern "C" int pjds_batch_run_pattern(pjds_batch *h, void *stream) {
  clear_error();
  if (!h) return set_error(PJDS_EINVAL, "h is NULL");
  if (h->n_tiles == 0) return PJDS_OK;
  return batch_issue<true>(h, static_cast<cudaStream_t>(stream));
}

extern "C" int pjds_batch_info(const pjds_batch *h, int32_t *n_tiles, int32_t *n_ctas) {
  clear_error();
  if (!h) return set_error(PJDS_EINVAL, "h is NULL");
  if (n_tiles) *n_tiles = h->n_tiles;
  if (n_ctas) *n_ctas = h->n_ctas;
  return PJDS_OK;
}

extern "C" int pjds_batch_destroy(pjds_batch *h) {
  clear_error();
  if (!h) return PJDS_OK;
  if (h->exec) cudaGraphExecDestroy(h->exec);
  free(h);
  return PJDS_OK;
}

extern "C" int pjds_batch_tune_rule(int32_t n_mats, const pjds_dev *mats, const void *const *xs, void *const *ys,
                                    const int32_t *rules, int32_t n_rules, int32_t reps, void *plan_dev,
                                    size_t plan_bytes, void *flush, size_t flush_bytes, double *us, int32_t *best,
                                    void *stream) {
  clear_error();
  if (!rules || n_rules <= 0 || !us || !best) return set_error(PJDS_EINVAL, "bad arguments");
  if (reps < 1 || reps > 1000) return set_error(PJDS_EINVAL, "reps must be in [1, 1000]");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  if (cudaEventCreate(&ev0) != cudaSuccess || cudaEventCreate(&ev1) != cudaSuccess) {
    if (ev0) cudaEventDestroy(ev0);
    return set_error(PJDS_ECUDA, "cudaEventCreate failed");
  }
  *best = -1;
  int rc = PJDS_OK;
  for (int32_t r = 0; r < n_rules && rc == PJDS_OK; ++r) {
    us[r] = -1.0;
    pjds_batch *h = nullptr;
    rc = batch_plan(n_mats, mats, xs, ys, nullptr, rules + 3 * r, plan_dev, plan_bytes, &h, stream);
    if (rc) break;
    std::vector<float> t((size_t)reps);
    rc = batch_issue(h, s);  // warm-up
    for (int32_t k = 0; k < reps && rc == PJDS_OK; ++k) {
      if (flush && flush_bytes) cudaMemsetAsync(flush, k & 0xff, flush_bytes, s);
      cudaEventRecord(ev0, s);
      rc = batch_issue(h, s);
      cudaEventRecord(ev1, s);
      const cudaError_t e = cudaEventSynchronize(ev1);
      if (e != cudaSuccess && rc == PJDS_OK) rc = set_error(PJDS_ECUDA, "timing: %s", cudaGetErrorString(e));
      if (rc == PJDS_OK) cudaEventElapsedTime(&t[(size_t)k], ev0, ev1);
    }
    pjds_batch_destroy(h);
    if (rc) break;
    std::sort(t.begin(), t.end());
    const float med = reps % 2 ? t[(size_t)reps / 2] : 0.5f * (t[(size_t)reps / 2 - 1] + t[(size_t)reps / 2]);
    us[r] = 1e3 * (double)med;
    if (*best < 0 || us[r] < us[*best]) *best = r;
  }
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  return rc;
}
