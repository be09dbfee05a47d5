/*
 * pjds_krylov.h — Krylov drivers on pJDS matrices in the permuted basis:
 * mixed-precision conjugate gradients with fp64 residual refinement, and the
 * Lanczos recurrence with an fp64-refined Ritz pair.
 *
 * Paper (arXiv:1112.5588): sparse matrix-vector multiplication is the
 * dominant operation of sparse eigenvalue and linear solvers (Sect. 1.1); with
 * pJDS the iterative scheme runs entirely on permuted vectors, permuting only
 * before the first and after the last step (Sect. 2.1); single-precision
 * values halve the matrix bytes (Table 1). Here the matrix is stored in fp32
 * or bf16 for the bandwidth-bound inner products and accuracy is recovered by
 * fp64 residuals (CG) and an fp64 Rayleigh quotient (Lanczos), the only fp64
 * work on the GPU.
 *
 * Conventions as in pjds.h (statuses, caller-owned device memory, streams).
 * Every matrix here must have been created with permute_cols = 1 (square,
 * permuted basis); vectors are in that basis (use pjds_permute/unpermute).
 * Scratch memory: every driver takes a caller-owned device workspace of at
 * least the size its *_workspace_bytes function reports, except
 * pjds_cg_solve_static, which uses a static device array instead; the
 * library never allocates device memory. Reductions are deterministic (fixed-order partial
 * sums per CTA, then one CTA), so repeated runs give identical results.
 */
#ifndef PJDS_KRYLOV_H
#define PJDS_KRYLOV_H

#include <stddef.h>
#include <stdint.h>

#include "pjds.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Options for pjds_cg_solve. max_outer = 0 / inner_iters = 0 take defaults
 * (6 and 50: 300 inner steps). use_graph = 1 captures the inner iterations in
 * a CUDA graph once and replays it every outer step (the stream must not be
 * capturing already). */
typedef struct pjds_cg_opts {
  int32_t max_outer;
  int32_t inner_iters;
  double tol;        /* stop when ||b - A x||_2 <= tol ||b||_2 (fp64 residual) */
  int32_t use_graph;
  int32_t reserved;
} pjds_cg_opts;

#define PJDS_CG_HISTORY 64

typedef struct pjds_cg_result {
  int32_t outer;            /* outer (refinement) steps taken */
  int32_t inner_total;      /* inner CG steps taken */
  double rel_residual;      /* final ||b - A_hi x||_2 / ||b||_2 in fp64 */
  double history[PJDS_CG_HISTORY]; /* relative fp64 residual before each outer step, then the final one */
  int32_t n_history;
  int32_t reserved;
} pjds_cg_result;

/* Workspace bytes for pjds_cg_solve on an n_rows x n_rows matrix (n_pad rows
 * padded), inner vectors of vec_dtype (PJDS_F64 or PJDS_F32). */
int pjds_cg_workspace_bytes(int32_t n_rows, int32_t n_pad, int32_t vec_dtype, size_t *bytes);

/*
 * Solve A x = b (A symmetric positive definite) by iterative refinement:
 *   repeat: r = b - A_hi x (fp64 pJDS product, fused with ||r||);
 *           inner CG on A_lo d = r / ||r|| for inner_iters steps (A_lo values
 *           fp32/bf16 with fp32 vectors and accumulation, or A_lo = A_hi/NULL
 *           for plain fp64 CG in every step);
 *           x += ||r|| d (fp64).
 * A_hi: PJDS_F64, permute_cols = 1. A_lo: NULL, or the same matrix in any
 * dtype, permute_cols = 1. b, x: device fp64 vectors of n_rows (x holds the
 * initial guess on entry). res may be NULL. Synchronises the stream once per
 * outer step (to read the residual norm).
 * Errors: PJDS_EINVAL (shapes, dtypes, bases, workspace too small), PJDS_ECUDA.
 */
int pjds_cg_solve(const pjds_dev *A_hi, const pjds_dev *A_lo, const double *b, double *x, const pjds_cg_opts *opts,
                  pjds_cg_result *res, void *work, size_t work_bytes, void *stream);

/*
 * pjds_cg_solve without a caller workspace. The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory for a
 * workspace at all — for example code that only ever receives the matrix, b
 * and x from a host application that owns every device allocation, or a hot
 * loop that must not pay for cudaMalloc/cudaFree (which can synchronise the
 * device) on each solve. It runs the same solve as pjds_cg_solve, with the
 * same arguments minus the workspace, using a 5.5 MiB array in device memory
 * that the library declares statically: every GPU that loads the library
 * holds it until the process exits. Limits and behaviour:
 *   - at most 131072 rows; larger matrices return PJDS_EINVAL (use
 *     pjds_cg_solve with a caller workspace);
 *   - the first call on a device (with that device current) looks up the
 *     array's device address once and keeps it for the life of the process;
 *     make that first call before any stream capture, and do not use the
 *     library across cudaDeviceReset (the kept address would then be stale);
 *   - opts->use_graph is ignored: the inner steps are launched one by one on
 *     `stream`, so the call creates no stream, graph or other driver object;
 *   - no cudaMalloc, cudaFree or allocating library call is made (the call
 *     issues kernels, one cudaMemsetAsync on the array and a small
 *     device-to-host copy of the residual norm per outer step);
 *   - all calls share the one array per device and it keeps the previous
 *     call's contents: each call clears the scalar block it reads and writes
 *     every vector before reading it, but calls that overlap on the GPU
 *     within one process (on two streams, or from two host threads) race on
 *     it and must be serialised by the caller.
 */
int pjds_cg_solve_static(const pjds_dev *A_hi, const pjds_dev *A_lo, const double *b, double *x,
                         const pjds_cg_opts *opts, pjds_cg_result *res, void *stream);

/* Workspace bytes for pjds_lanczos (vectors of A's vector type). */
int pjds_lanczos_workspace_bytes(int32_t n_rows, int32_t n_pad, int32_t vec_dtype, int32_t steps, size_t *bytes);

/*
 * `steps` steps of the symmetric Lanczos recurrence
 *   beta_{j+1} v_{j+1} = A v_j - alpha_j v_j - beta_j v_{j-1}
 * starting from v0 / ||v0||, without reorthogonalisation, with A's values in
 * its dtype, vectors in its vector type and every inner product accumulated
 * in fp64. alpha_host[steps] and beta_host[steps+1] (beta_host[0] = 0) receive
 * the tridiagonal T. basis: NULL, or device memory of steps * n_rows elements
 * of A's vector type that receives v_0 .. v_{steps-1} (row-major). A
 * breakdown (beta = 0) leaves the following vectors zero. Synchronises once.
 */
int pjds_lanczos(const pjds_dev *A, const void *v0, int32_t steps, double *alpha_host, double *beta_host,
                 void *basis, int32_t use_graph, void *work, size_t work_bytes, void *stream);

/*
 * Extreme eigenpair of the k x k symmetric tridiagonal T (diagonal alpha[k],
 * off-diagonal beta[1..k-1]) on the host: bisection on Sturm sequence counts
 * for the eigenvalue, then inverse iteration for a unit eigenvector s[k].
 * which = 0: largest, 1: smallest.
 */
int pjds_tridiag_extreme(int32_t k, const double *alpha, const double *beta, int32_t which, double *theta, double *s);

/* Workspace bytes for pjds_ritz_refine. */
int pjds_ritz_workspace_bytes(int32_t n_rows, int32_t n_pad, int32_t k, size_t *bytes);

/*
 * Ritz vector y = sum_j s[j] basis[j] (fp64, device, n_rows) from a Lanczos
 * basis of basis_dtype (PJDS_F64: double, PJDS_F32: float), then in fp64 with
 * A_hi (PJDS_F64, permute_cols = 1): the Rayleigh quotient
 * theta = (y, A y) / (y, y) and the residual ||A y - theta y|| / |theta|.
 * Synchronises once.
 */
int pjds_ritz_refine(const pjds_dev *A_hi, const void *basis, int32_t basis_dtype, int32_t k, const double *s_host,
                     double *y, double *theta, double *rel_residual, void *work, size_t work_bytes, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* PJDS_KRYLOV_H */
