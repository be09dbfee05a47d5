// pJDS and ELLPACK-R SpMV kernels for sm_103a (GB300).
//
// The product is bound by HBM bandwidth (about 0.15 flop per byte in fp64),
// not by arithmetic, and it is not a dense contraction, so there is no
// tensor-core path. What matters is keeping enough bytes in flight:
//   - val[] and col[] are streamed once: loads carry the evict-first hint in
//     L1 and L2 (ld.global.cs) so they do not push x out of the caches;
//   - a warp reads one jagged diagonal as one contiguous run (Listing 2
//     addressing col_start[j] + i), with optional 2- or 4-row vector loads;
//   - the gather x[col] goes through the read-only L1 path (ld.global.nc);
//   - the j-loop is unrolled so each thread issues U independent val/col
//     loads, then U gathers, before the dependent fused multiply-adds;
//   - the accumulator stays in a register and y is written once (scattered
//     through perm[] in the original basis);
//   - optionally the 32-row tiles are taken in the traversal order of
//     tile_order (by the original index of each tile's first row), so the
//     rows in flight are neighbours in the original numbering: their x
//     gathers share L2 sectors and their y stores fill whole sectors.
// Pad entries carry column -1 and are skipped, so every row's sum runs over
// exactly its own entries in CRS order, as in Listing 2 (with T threads per
// row, each lane over every T-th entry, then a fixed shuffle tree).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace pjds {
namespace dev {

// ----------------------------------------------------------------------------- value / vector types

struct bf16_t {
  uint16_t bits;
};

template <typename TV>
struct Acc;
template <>
struct Acc<double> {
  using T = double;
};
template <>
struct Acc<float> {
  using T = float;
};
template <>
struct Acc<bf16_t> {
  using T = float;
};

__device__ __forceinline__ double to_acc(double v) { return v; }
__device__ __forceinline__ float to_acc(float v) { return v; }
__device__ __forceinline__ float to_acc(bf16_t v) { return __uint_as_float(((uint32_t)v.bits) << 16); }

__device__ __forceinline__ double fma_acc(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fma_acc(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// ----------------------------------------------------------------------------- streaming loads

// R consecutive elements from a 16-byte-or-less aligned run, evict-first.
template <int R>
__device__ __forceinline__ void ld_stream(const double *p, double (&v)[R]) {
  if constexpr (R == 1) {
    v[0] = __ldcs(p);
  } else if constexpr (R == 2) {
    double2 a = __ldcs(reinterpret_cast<const double2 *>(p));
    v[0] = a.x;
    v[1] = a.y;
  } else {
    double2 a = __ldcs(reinterpret_cast<const double2 *>(p));
    double2 b = __ldcs(reinterpret_cast<const double2 *>(p) + 1);
    v[0] = a.x;
    v[1] = a.y;
    v[2] = b.x;
    v[3] = b.y;
  }
}

template <int R>
__device__ __forceinline__ void ld_stream(const float *p, float (&v)[R]) {
  if constexpr (R == 1) {
    v[0] = __ldcs(p);
  } else if constexpr (R == 2) {
    float2 a = __ldcs(reinterpret_cast<const float2 *>(p));
    v[0] = a.x;
    v[1] = a.y;
  } else {
    float4 a = __ldcs(reinterpret_cast<const float4 *>(p));
    v[0] = a.x;
    v[1] = a.y;
    v[2] = a.z;
    v[3] = a.w;
  }
}

template <int R>
__device__ __forceinline__ void ld_stream(const bf16_t *p, bf16_t (&v)[R]) {
  if constexpr (R == 1) {
    v[0].bits = __ldcs(reinterpret_cast<const unsigned short *>(p));
  } else if constexpr (R == 2) {
    unsigned int a = __ldcs(reinterpret_cast<const unsigned int *>(p));
    v[0].bits = (uint16_t)(a & 0xFFFFu);
    v[1].bits = (uint16_t)(a >> 16);
  } else {
    uint2 a = __ldcs(reinterpret_cast<const uint2 *>(p));
    v[0].bits = (uint16_t)(a.x & 0xFFFFu);
    v[1].bits = (uint16_t)(a.x >> 16);
    v[2].bits = (uint16_t)(a.y & 0xFFFFu);
    v[3].bits = (uint16_t)(a.y >> 16);
  }
}

template <int R>
__device__ __forceinline__ void ld_stream(const int32_t *p, int32_t (&v)[R]) {
  if constexpr (R == 1) {
    v[0] = __ldcs(p);
  } else if constexpr (R == 2) {
    int2 a = __ldcs(reinterpret_cast<const int2 *>(p));
    v[0] = a.x;
    v[1] = a.y;
  } else {
    int4 a = __ldcs(reinterpret_cast<const int4 *>(p));
    v[0] = a.x;
    v[1] = a.y;
    v[2] = a.z;
    v[3] = a.w;
  }
}

__device__ __forceinline__ double ld_stream1(const double *p) { return __ldcs(p); }
__device__ __forceinline__ float ld_stream1(const float *p) { return __ldcs(p); }
__device__ __forceinline__ bf16_t ld_stream1(const bf16_t *p) {
  bf16_t v;
  v.bits = __ldcs(reinterpret_cast<const unsigned short *>(p));
  return v;
}

// Values of the pattern products (every stored value taken as 1): the
// launcher passes the device address of these 8 ones as the kernel's val,
// and the pattern kernels read val + pattern_slot(val + o) (always a one)
// where the product reads val + o. They issue the product's instructions
// with its registers and occupancy, while the value stream stays in L1, and
// fma(1, x, acc) rounds acc + x once: the pattern product's sum exactly.
static __device__ __align__(16) double g_ones_f64[8] = {1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0};
static __device__ __align__(16) float g_ones_f32[8] = {1.0f, 1.0f, 1.0f, 1.0f, 1.0f, 1.0f, 1.0f, 1.0f};
static __device__ __align__(16) bf16_t g_ones_bf16[8] = {{0x3F80}, {0x3F80}, {0x3F80}, {0x3F80},
                                                         {0x3F80}, {0x3F80}, {0x3F80}, {0x3F80}};

// The product's value address, kept live (the compiler may not fold it
// away), reduced to a slot of the ones: 0 for every address the product
// reads (values are aligned to their size).
template <typename TV>
__device__ __forceinline__ int pattern_slot(const TV *p) {
  asm volatile("" : "+l"(p));
  return (int)(reinterpret_cast<uintptr_t>(p) & 3);
}

// Device address of this translation unit's ones of type TV (host code).
template <typename TV>
inline cudaError_t pattern_ones_address(const void **out) {
  void *p = nullptr;
  cudaError_t e;
  if constexpr (sizeof(TV) == 8)
    e = cudaGetSymbolAddress(&p, g_ones_f64);
  else if constexpr (sizeof(TV) == 4)
    e = cudaGetSymbolAddress(&p, g_ones_f32);
  else
    e = cudaGetSymbolAddress(&p, g_ones_bf16);
  *out = p;
  return e;
}

// Tile traversal order: logical row r is row r mod 32 of tile order[r / 32]
// (tiles of 32 sorted rows). Rewrites r in place; false for an entry outside
// the table's range (the thread then has no row).
__device__ __forceinline__ bool tile_row(const int32_t *__restrict__ order, int32_t n_pad, int64_t &r) {
  const int32_t t = __ldg(order + (r >> 5));
  if ((uint32_t)t >= (uint32_t)(n_pad >> 5)) return false;
  r = (int64_t)t * 32 + (r & 31);
  return true;
}

// Gather through the read-only L1 path; pads (c < 0) read nothing.
template <typename TX>
__device__ __forceinline__ TX gather(const TX *__restrict__ x, int32_t c) {
  return c >= 0 ? __ldg(x + c) : TX(0);
}

// ----------------------------------------------------------------------------- checked build

// Built with PJDS_CHECKED (libpjds_checked.so, a test build), the product
// kernels compare every jagged-diagonal index, element offset, gathered
// column, block index and stored row with its array's extent before the
// access. A violation skips the access and records its code and index in
// g_check_word (the first one; codes below); nothing traps. In the normal
// build PJDS_IN is `true` and the checks compile away.
enum CheckCode : unsigned { CHK_DIAG = 1, CHK_OFFSET = 2, CHK_COLUMN = 3, CHK_ROW = 4, CHK_BLOCK = 5 };

// Extents of the arrays one uniform-mapping launch reads (set by the
// launcher before each launch in the checked build).
struct Extents {
  int64_t stored;  // val, col
  int32_t n_cols;  // x
  int32_t n_rows;  // y (and perm)
  int32_t n_blocks;
  int32_t n_diag;  // col_start entries: n_max + 1
};

#ifdef PJDS_CHECKED
static __device__ Extents g_ext;
static __device__ unsigned long long g_check_word;
__device__ __forceinline__ bool in_extent(int64_t i, int64_t n, unsigned code) {
  if (i >= 0 && i < n) return true;
  atomicCAS(&g_check_word, 0ull, ((unsigned long long)code << 56) | ((unsigned long long)i & 0xFFFFFFFFFFFFFFull));
  return false;
}
#define PJDS_IN(i, n, code) ::pjds::dev::in_extent((int64_t)(i), (int64_t)(n), (code))
#define PJDS_EXT(field) ::pjds::dev::g_ext.field
#else
#define PJDS_IN(i, n, code) true
#define PJDS_EXT(field) 0
#endif

#ifdef PJDS_CHECKED
// This translation unit's check word (and optionally clear it); waits for s.
static inline cudaError_t read_check_word(unsigned long long *w, bool clear, cudaStream_t s) {
  cudaError_t e = cudaMemcpyFromSymbolAsync(w, g_check_word, sizeof(*w), 0, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess && clear) {
    const unsigned long long zero = 0;
    e = cudaMemcpyToSymbolAsync(g_check_word, &zero, sizeof(zero), 0, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  return e;
}

// Extents of a uniform-mapping launch, copied before the kernel on s.
static inline cudaError_t set_extents(const Extents &x, cudaStream_t s) {
  return cudaMemcpyToSymbolAsync(g_ext, &x, sizeof(x), 0, cudaMemcpyHostToDevice, s);
}
#endif

// gather with the extent of x checked in the checked build
template <typename TX>
__device__ __forceinline__ TX gather_n(const TX *__restrict__ x, int32_t c, int32_t n_cols) {
  (void)n_cols;
  return c >= 0 && PJDS_IN(c, n_cols, CHK_COLUMN) ? __ldg(x + c) : TX(0);
}

// ----------------------------------------------------------------------------- pJDS, R rows per thread

// Thread t owns sorted rows [R*t, R*t + R) of one block (b is a multiple of
// 32 >= R). Loop bound: the block's padded length; pads are skipped. The
// j-loop runs in chunks of U jagged diagonals; a chunk's loads are predicated
// on j < L, so a short row issues all of its loads in ceil(L/U) rounds.
// PAT: the pattern product (every stored value taken as 1, val not read):
// the same column stream, x gathers, fused multiply-adds (by the ones of
// pattern_ones, L1 hits) and y stores.
template <typename TV, typename TX, typename IDX, int R, int U, bool SCATTER, bool PAT = false>
__global__ void __launch_bounds__(512) pjds_rows_kernel(const TV *__restrict__ val, const int32_t *__restrict__ col,
                                                        const int64_t *__restrict__ col_start,
                                                        const int32_t *__restrict__ block_len,
                                                        const int32_t *__restrict__ perm,
                                                        const int32_t *__restrict__ order, const TX *__restrict__ x,
                                                        TX *__restrict__ y, int32_t n_rows, int32_t n_pad, int32_t b) {
  using TA = typename Acc<TV>::T;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t i0 = t * R;
  if (i0 >= n_pad) return;
  if (order && !tile_row(order, n_pad, i0)) return;
  if (!PJDS_IN(i0 / b, PJDS_EXT(n_blocks), CHK_BLOCK)) return;
  const int32_t L = __ldg(block_len + (int32_t)(i0 / b));
  TA acc[R];
#pragma unroll
  for (int r = 0; r < R; ++r) acc[r] = TA(0);

  for (int32_t j = 0; j < L; j += U) {
    int32_t c[U][R];
    TV v[U][R];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      bool live = j + u < L && PJDS_IN(j + u, PJDS_EXT(n_diag), CHK_DIAG);
      IDX o = 0;
      if (live) {
        o = (IDX)__ldg(col_start + j + u) + (IDX)i0;
        live = PJDS_IN(o, PJDS_EXT(stored), CHK_OFFSET) && PJDS_IN((int64_t)o + (R - 1), PJDS_EXT(stored), CHK_OFFSET);
      }
      if (live) {
        ld_stream<R>(col + o, c[u]);
        if constexpr (PAT)
          ld_stream<R>(val + pattern_slot(val + o), v[u]);  // val: the ones
        else
          ld_stream<R>(val + o, v[u]);
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) {
          c[u][r] = -1;
          v[u][r] = TV{};
        }
      }
    }
    TX xv[U][R];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int r = 0; r < R; ++r) xv[u][r] = gather_n(x, c[u][r], PJDS_EXT(n_cols));
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int r = 0; r < R; ++r) acc[r] = c[u][r] >= 0 ? fma_acc(to_acc(v[u][r]), (TA)xv[u][r], acc[r]) : acc[r];
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int64_t i = i0 + r;
    if (i < n_rows) {
      if constexpr (SCATTER) {
        const int32_t p = __ldcs(perm + i);
        if (PJDS_IN(p, PJDS_EXT(n_rows), CHK_ROW)) y[p] = (TX)acc[r];
      } else {
        y[i] = (TX)acc[r];
      }
    }
  }
}

// ----------------------------------------------------------------------------- pJDS, T threads per row

// T consecutive lanes share one sorted row: lane s takes jagged diagonals
// j = s, s+T, ...; the T partial sums are added with shuffles (fixed tree).
template <typename TV, typename TX, typename IDX, int T, int U, bool SCATTER, bool PAT = false>
__global__ void __launch_bounds__(512) pjds_tpr_kernel(const TV *__restrict__ val, const int32_t *__restrict__ col,
                                                        const int64_t *__restrict__ col_start,
                                                        const int32_t *__restrict__ block_len,
                                                        const int32_t *__restrict__ perm,
                                                        const int32_t *__restrict__ order, const TX *__restrict__ x,
                                                        TX *__restrict__ y, int32_t n_rows, int32_t n_pad, int32_t b) {
  using TA = typename Acc<TV>::T;
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t i = g / T;
  const int32_t s = (int32_t)(g % T);
  bool active = i < n_pad;  // whole warps stay for the shuffles
  if (active && order) active = tile_row(order, n_pad, i);
  if (active) active = PJDS_IN(i / b, PJDS_EXT(n_blocks), CHK_BLOCK);
  const int32_t L = active ? __ldg(block_len + (int32_t)(i / b)) : 0;
  TA acc = TA(0);
  for (int32_t j = s; j < L; j += U * T) {
    int32_t c[U];
    TV v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      bool live = j + u * T < L && PJDS_IN(j + u * T, PJDS_EXT(n_diag), CHK_DIAG);
      IDX o = 0;
      if (live) {
        o = (IDX)__ldg(col_start + j + u * T) + (IDX)i;
        live = PJDS_IN(o, PJDS_EXT(stored), CHK_OFFSET);
      }
      if (live) {
        c[u] = __ldcs(col + o);
        v[u] = ld_stream1(PAT ? val + pattern_slot(val + o) : val + o);  // PAT: val holds the ones
      } else {
        c[u] = -1;
        v[u] = TV{};
      }
    }
    TX xv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) xv[u] = gather_n(x, c[u], PJDS_EXT(n_cols));
#pragma unroll
    for (int u = 0; u < U; ++u) acc = c[u] >= 0 ? fma_acc(to_acc(v[u]), (TA)xv[u], acc) : acc;
  }
#pragma unroll
  for (int off = T / 2; off >= 1; off /= 2) acc += __shfl_down_sync(0xffffffffu, acc, off, T);
  if (s == 0 && active && i < n_rows) {
    if constexpr (SCATTER) {
      const int32_t p = __ldcs(perm + i);
      if (PJDS_IN(p, PJDS_EXT(n_rows), CHK_ROW)) y[p] = (TX)acc;
    } else {
      y[i] = (TX)acc;
    }
  }
}

// ----------------------------------------------------------------------------- ELLPACK-R (Listing 1)

// One thread per row in the original order; loop to the row's own length.
template <typename TV, typename TX, typename IDX, int U>
__global__ void __launch_bounds__(512) ellr_kernel(const TV *__restrict__ val, const int32_t *__restrict__ col,
                                                    const int32_t *__restrict__ row_max, const TX *__restrict__ x,
                                                    TX *__restrict__ y, int32_t n_rows, int32_t n_pad) {
  using TA = typename Acc<TV>::T;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_rows) return;
  const int32_t L = __ldcs(row_max + i);
  TA acc = TA(0);
  for (int32_t j = 0; j < L; j += U) {
    int32_t c[U];
    TV v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const IDX o = (IDX)(j + u) * (IDX)n_pad + (IDX)i;
      if (j + u < L && PJDS_IN(o, PJDS_EXT(stored), CHK_OFFSET)) {
        c[u] = __ldcs(col + o);
        v[u] = ld_stream1(val + o);
      } else {
        c[u] = -1;
        v[u] = TV{};
      }
    }
    TX xv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) xv[u] = gather_n(x, c[u], PJDS_EXT(n_cols));
#pragma unroll
    for (int u = 0; u < U; ++u) acc = c[u] >= 0 ? fma_acc(to_acc(v[u]), (TA)xv[u], acc) : acc;
  }
  y[i] = (TX)acc;
}

// ----------------------------------------------------------------------------- basis changes

template <typename TX>
__global__ void permute_kernel(const int32_t *__restrict__ perm, const TX *__restrict__ v, TX *__restrict__ vp,
                               int32_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) vp[i] = __ldg(v + __ldcs(perm + i));
}

template <typename TX>
__global__ void unpermute_kernel(const int32_t *__restrict__ perm, const TX *__restrict__ vp, TX *__restrict__ v,
                                 int32_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[__ldcs(perm + i)] = __ldcs(vp + i);
}

}  // namespace dev
}  // namespace pjds
