// Window mapping of the pJDS product (device side; the plan is built by
// window.h): one CTA per window of W original rows. The CTA
//   1. copies the x intervals of the plan (the band offsets around its
//      window) into shared memory,
//   2. runs the window's 32-row tiles, one warp per tile at a time, each
//      thread one sorted row exactly as the one-thread-per-row kernel does
//      (same loads, same order of fused multiply-adds), taking x[c] from
//      shared memory when c lies in a staged interval and through the L1
//      path otherwise,
//   3. keeps the sums of rows inside the window in shared memory (a flag per
//      row marks the ones it computed) and writes them as whole lines at the
//      end; rows of its tiles beyond the window are stored directly.
// Every row keeps the bits of the one-thread-per-row mapping.
#pragma once

#include "spmv_kernels.cuh"

namespace pjds {
namespace win {

constexpr int MAX_RANGES = 4;

struct Desc {
  const void *val;
  const int32_t *col;
  const int64_t *col_start;
  const int32_t *block_len;
  const int32_t *perm;
  const int32_t *order;    // tile traversal table (tiles by first original row)
  const int32_t *win_ptr;  // window w: order[win_ptr[w] .. win_ptr[w+1])
  const void *x;
  void *y;
  int64_t stored;
  int32_t n_rows, n_cols, n_pad, b;
  int32_t W, n_ranges, n_blocks, n_diag;
  int32_t lo[MAX_RANGES], len[MAX_RANGES], soff[MAX_RANGES];
  int32_t staged;  // shared-memory entries of the intervals (soff[k] + len[k] <= staged)
  int32_t reserved;
};

// x[c] for a gather of the window starting at original row a.
template <typename TX>
__device__ __forceinline__ TX gather_win(const Desc &d, const TX *sx, const TX *__restrict__ x, int32_t c, int32_t a) {
  if (c < 0) return TX(0);
  const int32_t rel = c - a;  // both in [0, 2^31): no overflow
#pragma unroll
  for (int k = 0; k < MAX_RANGES; ++k) {
    if (k < d.n_ranges) {
      // unsigned wrap: the true difference lies within (-2^32, 2^32) - len
      const uint32_t e = (uint32_t)rel - (uint32_t)d.lo[k];
      if (e < (uint32_t)d.len[k]) return sx[d.soff[k] + (int32_t)e];
    }
  }
  return PJDS_IN(c, d.n_cols, dev::CHK_COLUMN) ? __ldg(x + c) : TX(0);
}

// One row's partial sum over jagged diagonals [j, j + U) (loads predicated on
// j + u < L; pads carry column -1 and add nothing).
template <typename TV, typename TX, typename IDX, int U, bool PAT>
__device__ __forceinline__ void row_chunk(const Desc &d, const TV *__restrict__ val, const TX *sx,
                                          const TX *__restrict__ x, int64_t i, int32_t L, int32_t j, int32_t a,
                                          typename dev::Acc<TV>::T &acc) {
  using TA = typename dev::Acc<TV>::T;
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
      if constexpr (!PAT) v[u] = dev::ld_stream1(val + o);
    } else {
      c[u] = -1;
      v[u] = TV{};
    }
  }
  TX xv[U];
#pragma unroll
  for (int u = 0; u < U; ++u) xv[u] = gather_win(d, sx, x, c[u], a);
#pragma unroll
  for (int u = 0; u < U; ++u) {
    if constexpr (PAT)
      acc = c[u] >= 0 ? acc + (TA)xv[u] : acc;
    else
      acc = c[u] >= 0 ? dev::fma_acc(dev::to_acc(v[u]), (TA)xv[u], acc) : acc;
  }
}

// RT tiles per warp at a time (RT rows per thread, from different tiles), so
// that each thread keeps RT independent chains of loads in flight.
template <typename TV, typename TX, typename IDX, int U, int RT, bool PAT, int NT>
__global__ void __launch_bounds__(NT, 2048 / NT) pjds_window_kernel(const Desc d) {
  using TA = typename dev::Acc<TV>::T;
  extern __shared__ __align__(16) unsigned char smem[];
  TX *sx = reinterpret_cast<TX *>(smem);
  TX *sy = sx + d.staged;
  uint32_t *flag = reinterpret_cast<uint32_t *>(sy + d.W);
  const TV *__restrict__ val = static_cast<const TV *>(d.val);
  const TX *__restrict__ x = static_cast<const TX *>(d.x);
  TX *__restrict__ y = static_cast<TX *>(d.y);
  const int32_t a = (int32_t)blockIdx.x * d.W;

  // 1. the plan's x intervals of this window (entries outside x read as 0
  //    and are never asked for: columns lie in [0, n_cols))
  for (int k = 0; k < d.n_ranges; ++k) {
    const int64_t g0 = (int64_t)a + d.lo[k];
    TX *dst = sx + d.soff[k];
    for (int32_t e = threadIdx.x; e < d.len[k]; e += NT) {
      const int64_t g = g0 + e;
      dst[e] = g >= 0 && g < d.n_cols ? __ldg(x + g) : TX(0);
    }
  }
  for (int32_t e = threadIdx.x; e < (d.W + 31) / 32; e += NT) flag[e] = 0u;
  __syncthreads();

  // 2. the window's tiles, RT per warp at a time
  const int32_t t0 = __ldg(d.win_ptr + blockIdx.x), t1 = __ldg(d.win_ptr + blockIdx.x + 1);
  const int32_t lane = threadIdx.x & 31;
  for (int32_t t = t0 + RT * (int32_t)(threadIdx.x >> 5); t < t1; t += RT * (NT / 32)) {
    int64_t i[RT];
    int32_t L[RT];
    int32_t Lmax = 0;
#pragma unroll
    for (int r = 0; r < RT; ++r) {
      L[r] = 0;
      i[r] = -1;
      if (t + r < t1) {
        const int32_t tile = __ldg(d.order + t + r);
        const int64_t ii = (int64_t)tile * 32 + lane;
        if ((uint32_t)tile < (uint32_t)(d.n_pad >> 5) && ii < d.n_rows && PJDS_IN(ii / d.b, d.n_blocks, dev::CHK_BLOCK)) {
          i[r] = ii;
          L[r] = __ldg(d.block_len + (int32_t)(ii / d.b));
        }
      }
      Lmax = max(Lmax, L[r]);
    }
    TA acc[RT];
#pragma unroll
    for (int r = 0; r < RT; ++r) acc[r] = TA(0);
    for (int32_t j = 0; j < Lmax; j += U) {
#pragma unroll
      for (int r = 0; r < RT; ++r) row_chunk<TV, TX, IDX, U, PAT>(d, val, sx, x, i[r], L[r], j, a, acc[r]);
    }
#pragma unroll
    for (int r = 0; r < RT; ++r) {
      if (i[r] < 0) continue;
      const int32_t p = __ldcs(d.perm + i[r]);
      if (!PJDS_IN(p, d.n_rows, dev::CHK_ROW)) continue;
      const uint32_t q = (uint32_t)(p - a);
      if (q < (uint32_t)d.W) {
        sy[q] = (TX)acc[r];
        atomicOr(flag + (q >> 5), 1u << (q & 31));
      } else {
        y[p] = (TX)acc[r];
      }
    }
  }
  __syncthreads();

  // 3. the window's own rows, as whole lines
  for (int32_t e = threadIdx.x; e < d.W; e += NT) {
    if ((int64_t)a + e >= d.n_rows) break;
    if ((flag[e >> 5] >> (e & 31)) & 1u) y[a + e] = sy[e];
  }
}

}  // namespace win
}  // namespace pjds
