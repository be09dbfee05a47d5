// pJDS product with the streamed arrays staged by the bulk-copy engine.
//
// A persistent CTA owns tiles of TR consecutive sorted rows (one row per
// consumer thread). Within a tile, jagged diagonal j covers the tile's first
// n_j rows (blocks are sorted by length, so the rows of a diagonal form a
// prefix), and its val/col entries for those rows are one contiguous run at
// col_start[j] + row0. One producer thread issues a 1-D bulk copy
// (cp.async.bulk, completion counted in bytes on an mbarrier) for each run of
// a chunk of JC diagonals into a ring of S shared-memory stages; the consumer
// warps wait for a stage, read their row's entries from shared memory, gather
// x through L1 and accumulate, then release the stage. The L1 request path
// then carries only the x gathers. Every wait is bounded: after the limit the
// waiting thread records an error code in a device status word
// (pjds_device_status reads it) and leaves.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "spmv_kernels.cuh"

namespace pjds {
namespace dev {

constexpr int ST_TR = 128;        // rows per tile = consumer threads
constexpr int ST_JC = 8;          // jagged diagonals per stage
constexpr int ST_S = 3;           // stages in the ring (fp64: 36 KB of shared memory)
constexpr uint32_t ST_SPIN = 1u << 22;  // polls before a wait gives up

// Device status word of this translation unit: 0 = fine; bit 0: a consumer
// wait ran out; bit 1: a producer wait ran out. Internal linkage: each
// translation unit that launches the kernel has its own word and reads it
// with staged_status().
static __device__ int g_staged_status = 0;

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase of `parity` to complete; false after ST_SPIN polls.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  for (uint32_t it = 0; it < ST_SPIN; ++it) {
    if (mbar_test(bar, parity)) return true;
    if (it > 64) __nanosleep(64);
  }
  return false;
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Rows of diagonal j inside the tile starting at row0 (a prefix of the tile).
__device__ __forceinline__ int32_t diag_rows(const int64_t *__restrict__ col_start, int32_t j, int64_t row0) {
  const int64_t dl = __ldg(col_start + j + 1) - __ldg(col_start + j) - row0;
  return dl <= 0 ? 0 : (dl >= ST_TR ? ST_TR : (int32_t)dl);
}

template <typename TV, typename TX, typename IDX, bool SCATTER>
__global__ void __launch_bounds__(ST_TR + 32)
    pjds_staged_kernel(const TV *__restrict__ val, const int32_t *__restrict__ col,
                       const int64_t *__restrict__ col_start, const int32_t *__restrict__ block_len,
                       const int32_t *__restrict__ perm, const TX *__restrict__ x, TX *__restrict__ y, int32_t n_rows,
                       int32_t n_pad, int32_t b) {
  using TA = typename Acc<TV>::T;
  __shared__ __align__(128) TV s_val[ST_S][ST_JC][ST_TR];
  __shared__ __align__(128) int32_t s_col[ST_S][ST_JC][ST_TR];
  __shared__ __align__(8) uint64_t full[ST_S], empty[ST_S];
  const int tid = threadIdx.x;
  const int n_tiles = (n_pad + ST_TR - 1) / ST_TR;
  if (tid == 0) {
    for (int s = 0; s < ST_S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], ST_TR / 32);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  if (tid >= ST_TR) {  // producer warp: lane 0 issues every copy
    if (tid != ST_TR) return;
    uint32_t q = 0;  // running chunk index over all tiles of this CTA
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
      const int64_t row0 = (int64_t)tile * ST_TR;
      const int32_t L = __ldg(block_len + (int32_t)(row0 / b));
      for (int32_t j0 = 0; j0 < L; j0 += ST_JC, ++q) {
        const int s = q % ST_S;
        if (!mbar_wait(&empty[s], ((q / ST_S) & 1) ^ 1)) {
          atomicOr(&g_staged_status, 2);
          return;
        }
        uint32_t bytes = 0;
        int32_t nj[ST_JC];
#pragma unroll
        for (int jj = 0; jj < ST_JC; ++jj) {
          nj[jj] = j0 + jj < L ? diag_rows(col_start, j0 + jj, row0) : 0;
          bytes += (uint32_t)nj[jj] * (uint32_t)(sizeof(TV) + sizeof(int32_t));
        }
        mbar_expect_tx(&full[s], bytes);
#pragma unroll
        for (int jj = 0; jj < ST_JC; ++jj) {
          if (nj[jj] == 0) continue;
          const IDX o = (IDX)__ldg(col_start + j0 + jj) + (IDX)row0;
          bulk_g2s(&s_val[s][jj][0], val + o, (uint32_t)(nj[jj] * sizeof(TV)), &full[s]);
          bulk_g2s(&s_col[s][jj][0], col + o, (uint32_t)(nj[jj] * sizeof(int32_t)), &full[s]);
        }
      }
    }
    return;
  }

  // consumer threads: row row0 + tid of each tile
  uint32_t q = 0;
  bool ok = true;
  for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
    const int64_t row0 = (int64_t)tile * ST_TR;
    const int32_t L = __ldg(block_len + (int32_t)(row0 / b));
    TA acc = TA(0);
    for (int32_t j0 = 0; j0 < L; j0 += ST_JC, ++q) {
      const int s = q % ST_S;
      if (!mbar_wait(&full[s], (q / ST_S) & 1)) {
        atomicOr(&g_staged_status, 1);
        ok = false;
        break;
      }
      int32_t c[ST_JC];
      TV v[ST_JC];
#pragma unroll
      for (int jj = 0; jj < ST_JC; ++jj) {
        const bool in = j0 + jj < L && tid < diag_rows(col_start, j0 + jj, row0);
        c[jj] = in ? s_col[s][jj][tid] : -1;
        v[jj] = in ? s_val[s][jj][tid] : TV{};
      }
      __syncwarp();
      if ((tid & 31) == 0) mbar_arrive(&empty[s]);  // the stage may be refilled
      TX xv[ST_JC];
#pragma unroll
      for (int jj = 0; jj < ST_JC; ++jj) xv[jj] = gather(x, c[jj]);
#pragma unroll
      for (int jj = 0; jj < ST_JC; ++jj) acc = c[jj] >= 0 ? fma_acc(to_acc(v[jj]), (TA)xv[jj], acc) : acc;
    }
    const int64_t i = row0 + tid;
    if (ok && i < n_rows) {
      if constexpr (SCATTER)
        y[__ldcs(perm + i)] = (TX)acc;
      else
        y[i] = (TX)acc;
    }
  }
}

// Self-test of the bounded wait: one thread waits on an mbarrier that nothing
// will complete (which = 0: a fresh barrier's phase 0, as a consumer would;
// which = 1: the same wait from a producer's side) and must give up and set
// the matching status bit. No copy is ever issued, so nothing is in flight.
static __global__ void staged_wait_selftest_kernel(int which) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  if (!mbar_wait(&bar, 0)) atomicOr(&g_staged_status, which == 0 ? 1 : 2);
}

// Read (and optionally clear) this translation unit's status word; waits for the stream.
inline cudaError_t staged_status(int *out, bool clear, cudaStream_t s) {
  cudaError_t e = cudaMemcpyFromSymbolAsync(out, g_staged_status, sizeof(int), 0, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && clear) {
    static const int zero = 0;
    e = cudaMemcpyToSymbolAsync(g_staged_status, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e;
}

}  // namespace dev
}  // namespace pjds
