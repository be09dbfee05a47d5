/*
 * pjds.h — C ABI of libpjds: sparse matrix-vector multiplication y = A x on a
 * GB300 (sm_103a) with A stored in padded jagged diagonals storage (pJDS), and
 * the ELLPACK-R format as the baseline.
 *
 * Paper: M. Kreutzer, G. Hager, G. Wellein, H. Fehske, A. Basermann,
 * A. R. Bishop, "Sparse matrix-vector multiplication on GPGPU clusters: A new
 * storage format and a scalable implementation", arXiv:1112.5588.
 *
 * Conventions for every entry point:
 *   - Return value: PJDS_OK (0) or a negative status below. pjds_last_error()
 *     returns a message for the last failure on the calling thread. Nothing
 *     aborts, no C++ exception crosses this boundary, and no error is signalled
 *     by a device fault.
 *   - Host arrays passed in are borrowed for the duration of the call only.
 *   - Device memory is never allocated by this library: every device pointer
 *     is owned by the caller (e.g. a torch tensor's data_ptr()).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream). Kernel launches are asynchronous on that stream; a launch
 *     error is reported as PJDS_ECUDA, execution errors surface at the
 *     caller's next synchronisation.
 *   - Indices are 0-based. Matrices have at most 2^31-1 rows and columns.
 */
#ifndef PJDS_H
#define PJDS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PJDS_OK 0
#define PJDS_EINVAL (-1)    /* null pointer, bad size, bad b, malformed CRS, dtype mismatch, misalignment */
#define PJDS_ENOMEM (-2)    /* host allocation failed */
#define PJDS_ECUDA (-3)     /* CUDA runtime error (launch configuration, copy) */
#define PJDS_EOVERFLOW (-4) /* stored element count or an index does not fit the format */

/* Storage type of the matrix values. Vectors x, y are double for PJDS_F64 and
 * float for PJDS_F32 and PJDS_BF16; products are accumulated in the vector
 * type (Table 1 compares single and double precision; BF16 halves the value
 * bytes again). */
typedef enum pjds_dtype { PJDS_F64 = 0, PJDS_F32 = 1, PJDS_BF16 = 2 } pjds_dtype;

/* Message for the last failing call on this thread ("" if none). The pointer
 * stays valid until the next call on the same thread. */
const char *pjds_last_error(void);

/* Library ABI version (increments when a struct layout changes). */
int32_t pjds_version(void);

/* sizeof of the ABI structs, for bindings to check their layouts:
 * out[0..4] = pjds_host, pjds_dev, pjds_launch, ellr_host, ellr_dev. */
void pjds_abi_sizes(int32_t out[5]);

/* ------------------------------------------------------------------------ */
/* pJDS (Sect. 2.1, Listing 2)                                               */
/* ------------------------------------------------------------------------ */

/*
 * Host-side pJDS arrays, created by pjds_create and owned by the library
 * until pjds_destroy. Layout (Sect. 2.1):
 *   - rows are sorted by descending length, equal lengths keeping their
 *     original order: perm[new] = old, inv_perm[old] = new;
 *   - rows are padded to n_pad = ceil(n_rows / b) * b with empty rows;
 *   - each block of b consecutive sorted rows is padded to its longest row,
 *     block_len[k] (non-increasing in k);
 *   - row_len[i] is the length of sorted row i (0 for padding rows);
 *   - the padded matrix is stored column by column ("jagged diagonals"):
 *     entry j of sorted row i sits at col_start[j] + i, for j < block_len of
 *     its block; col_start has n_max + 1 entries, col_start[n_max] = n_stored;
 *   - padding entries hold value +0 and column index -1.
 * With permute_cols = 1 the column indices are renumbered into the permuted
 * basis (col -> inv_perm[col]; square matrices only), the form in which an
 * iterative solver runs entirely on permuted vectors (Sect. 2.1).
 * val holds n_stored elements of dtype (double, float, or bfloat16 as uint16
 * bits, rounded to nearest even from the fp64 input).
 * tile_order is not part of the storage format: it is the order in which the
 * product kernels take the 32-row tiles of the sorted matrix (tile t = sorted
 * rows 32t .. 32t+31; n_pad / 32 tiles). Sect. 2.1 fixes which rows share a
 * block, not the order in which blocks are processed; pjds_create lists the
 * tiles by the original index of their first row (ascending, stable; tiles
 * holding only padding rows last), so that the rows in flight at any moment
 * lie close together in the original numbering, whatever their length. Their
 * x gathers then share L2 sectors and their scattered y stores fill whole
 * sectors while the lines are still in L2. Each row's arithmetic does not
 * depend on the order.
 * plan (n_plan entries of four int32) is not part of the format either: the
 * per-tile mapping, the sorted rows cut into one-CTA tiles each mapped by its
 * block's length (see pjds_dev). It assumes 16-byte aligned device arrays;
 * the launcher checks.
 * pair_share is a statistic of the matrix for the default mapping: the per
 * mille of stored entries whose column equals the column of the paired row
 * (sorted rows 2k and 2k + 1) at the same jagged diagonal, rounded down. It
 * is high on block-structured matrices (rows of one block row share their
 * columns), where one thread taking both rows of a pair reads each gathered x
 * sector once for both.
 */
typedef struct pjds_host {
  int32_t n_rows, n_cols, n_pad, b, n_blocks, n_max;
  int64_t nnz, n_stored;
  int32_t dtype, permute_cols;
  int32_t *perm;      /* [n_rows]   */
  int32_t *inv_perm;  /* [n_rows]   */
  int32_t *block_len; /* [n_blocks] */
  int32_t *row_len;   /* [n_pad]    */
  int64_t *col_start; /* [n_max+1]  */
  int32_t *col;       /* [n_stored] */
  void *val;          /* [n_stored] of dtype */
  int32_t *tile_order; /* [n_pad / 32] */
  int32_t *plan;       /* [4 * n_plan] per-tile mapping, see pjds_dev */
  int32_t n_plan;
  int32_t pair_share; /* per mille, see below; 0 from pjds_create_shape */
} pjds_host;

/*
 * Device-side view of the same arrays: the caller copies each host array into
 * a device buffer it owns and fills this struct (sizes copied from the host
 * struct). row_len and inv_perm are not read by the kernels and may be NULL.
 * tile_order may be NULL (tiles in sorted order); otherwise it must hold the
 * n_pad / 32 entries pjds_create wrote (a permutation of 0 .. n_pad/32 - 1).
 * The one-thread-per-row, several-rows-per-thread and several-threads-per-row
 * kernels follow it when pjds_launch.tile_order selects it (a kernel skips an
 * entry outside that range); the staged kernel, SpMM, the batched launch and
 * the Krylov products take tiles in sorted order.
 * plan (n_plan entries of four int32: 0, first sorted row, rows, kind) is
 * the per-tile mapping pjds_create wrote, or NULL: the sorted rows cut into
 * tiles of one 256-thread CTA each, every tile mapped by the length of its
 * rows' block: 8 lanes per row from 256 entries, 4 from 64, 2 from 16 (kinds
 * 8, 4, 2; 256 / lanes rows), else two adjacent rows per thread (kind 0, 512
 * rows) or four for blocks of at most 2 entries (kind 3, 1024 rows); a tile
 * ends where the kind changes. The entries are ordered by work per lane,
 * largest first; from 2^21 rows on, the entries of kinds 0 and 3 then follow
 * the others in the order of the original index of their first row (perm of
 * its first sorted row), so that the short rows in flight lie close together
 * in the original numbering. A row gives the same bits as with the same lanes per row in
 * the uniform mappings (one thread per row for kinds 0 and 3). The plan
 * kernel runs one CTA per entry; it needs plan, val and col 16-byte aligned
 * and skips an entry that does not describe a tile of the matrix.
 * val must be 16-byte aligned; all other pointers 4-byte aligned.
 */
typedef struct pjds_dev {
  int32_t n_rows, n_cols, n_pad, b, n_blocks, n_max;
  int64_t nnz, n_stored;
  int32_t dtype, permute_cols;
  const int32_t *perm;
  const int32_t *block_len;
  const int32_t *row_len;
  const int64_t *col_start;
  const int32_t *col;
  const void *val;
  const int32_t *tile_order; /* NULL: tiles in sorted order */
  const int32_t *plan;       /* NULL: no per-tile mapping */
  int32_t n_plan;
  int32_t pair_share; /* copied from pjds_host (0: unknown); read by the default mapping only */
} pjds_dev;

/*
 * Convert a CRS matrix (row_ptr[n_rows+1] int64, col_idx[nnz] int32 in
 * [0, n_cols), val[nnz] fp64; columns within a row are kept in the given
 * order, which fixes the summation order) into pJDS with block size b.
 * b must be a positive multiple of 32 (the warp width, Sect. 2.1: "b_r should
 * be the warp size"). On success *out receives a new handle.
 * Errors: PJDS_EINVAL (null pointers, n_rows < 0, n_cols < 1, bad b, row_ptr not
 * starting at 0 or decreasing, a column out of range, permute_cols on a
 * non-square matrix, unknown dtype), PJDS_ENOMEM, PJDS_EOVERFLOW.
 */
int pjds_create(int32_t n_rows, int32_t n_cols, const int64_t *row_ptr, const int32_t *col_idx,
                const double *val, int32_t b, int32_t dtype, int32_t permute_cols, pjds_host **out);

/*
 * The structure of the pJDS matrix from the row lengths alone (row_ptr[n_rows
 * + 1]): the sort, padding, jagged-diagonal offsets, traversal table and
 * per-tile plan of pjds_create (original basis), every array equal to
 * pjds_create's for any columns and values with these row lengths, but col
 * and val are left NULL and pair_share is 0: the caller fills the n_stored
 * entries itself (entry
 * j of sorted row i, perm[i] being its original row, at col_start[j] + i for
 * j < row_len[i]; pads, up to the block length, column -1 and value +0), for
 * example directly in device memory when the CRS arrays would not fit the
 * host. Nothing checks those entries. The paper has no counterpart of this
 * call. Errors as pjds_create; free with pjds_destroy.
 */
int pjds_create_shape(int32_t n_rows, int32_t n_cols, const int64_t *row_ptr, int32_t b, int32_t dtype,
                      pjds_host **out);

/* Free a handle from pjds_create or pjds_create_shape (NULL is accepted). */
int pjds_destroy(pjds_host *h);

/*
 * y = A x with A in pJDS (Listing 2): each sorted row i computes
 * sum_{j < len(i)} val[col_start[j] + i] * x[col[col_start[j] + i]] with
 * fused multiply-add, then
 *   - permute_cols = 0: writes y[perm[i]] (x and y in the original basis);
 *   - permute_cols = 1: writes y[i] (x and y in the permuted basis).
 * The basis is a property of the matrix handle, fixed by pjds_create's
 * permute_cols, not an argument of the call: in the permuted basis the column
 * indices themselves are renumbered, so one set of device arrays serves one
 * basis only (create the matrix twice to use both).
 * x: n_cols elements, y: n_rows elements, device memory of the vector type of
 * A->dtype; x and y must not overlap. Every element of y is written.
 * Mapping (the default of pjds_spmv_cfg): the per-tile mapping of A->plan
 * when the longest row has more than 4 times the mean row length and the
 * matrix has at least 2^16 rows (fp64), 2^17 (fp32) or 2^18 (bf16) (and
 * plan, val and col are 16-byte aligned); otherwise T threads per row for every
 * row, T in 1, 2, 4, 8, from the longest row against the size of the
 * product: with ratio =
 * n_max * 2^20 / (nnz * (value bytes + 4)), T = 1 below 2, 2 below 8, 4
 * below 64, else 8, then doubled (up to 8) while n_rows * T < 2^17. With
 * T = 1 each row sums in its original entry order; with T > 1 each lane sums
 * every T-th entry in order, then a fixed shuffle tree adds the T partial
 * sums. With one thread per row, fp32 and bf16 values take two adjacent
 * rows per thread (same per-row arithmetic) when val and col allow the paired
 * loads and either the matrix has at least 2^21 rows, or it has at least 2^18
 * rows of at least 64 entries on average with pair_share >= 500 (the paired
 * rows then share their x gathers; 128-thread CTAs in that case).
 * pjds_spmv_resolve reports the mapping chosen for a matrix.
 */
int pjds_spmv(const pjds_dev *A, const void *x, void *y, void *stream);

/*
 * Kernel configuration for pjds_spmv_cfg (tuning and autotuning):
 *   rows_per_thread  1, 2 or 4 adjacent sorted rows per thread, read with one
 *                    vector load per jagged diagonal (0 = default);
 *   threads_per_row  1, 2, 4 or 8 threads share one row, splitting its jagged
 *                    diagonals round-robin and adding partial sums at the end
 *                    (sliced ELLR-T style; changes the summation order);
 *   block_threads    threads per CTA, a multiple of 32 in [32, 512]
 *                    (0 = default);
 *   unroll           jagged diagonals loaded per round of the j-loop
 *                    (0 = default; R=1: 4, 8, 16; R=2: 2, 4, 8; R=4: 2, 4;
 *                    T>1: 2, 4);
 *   staged           1: a persistent kernel (one CTA per SM slot, tiles of
 *                    128 sorted rows) whose producer warp copies each tile's
 *                    jagged-diagonal runs of val and col into a 3-stage
 *                    shared-memory ring with bulk copies (cp.async.bulk,
 *                    mbarrier completion) while 4 consumer warps gather x
 *                    and accumulate; one thread per row, block_threads and
 *                    unroll are ignored, val and col must be 16-byte aligned.
 *                    Its waits are bounded; a wait that runs out sets a bit
 *                    in the device status word (pjds_device_status) and the
 *                    affected rows of y are not written.
 *   tile_order       0: automatic, 1: take the 32-row tiles in A->tile_order
 *                    (PJDS_EINVAL if A->tile_order is NULL), -1: in sorted
 *                    order. Automatic uses the table when there is one,
 *                    n_rows >= 2^20 and the longest row has at most 4 times
 *                    the mean row length (a measured GB300 rule: ordering
 *                    gains 4-23% there, while on smaller matrices nothing is
 *                    gained and on widely spread row lengths the sorted
 *                    order's longest-first schedule is worth more, 5-25%).
 *                    The staged kernel always takes sorted order.
 *   plan             0: automatic, 1: the per-tile mapping of A->plan
 *                    (PJDS_EINVAL if A->plan is NULL or plan, val or col is
 *                    not 16-byte aligned), -1: a uniform mapping. Automatic
 *                    uses the plan when it can, the longest row has more
 *                    than 4 times the mean row length and n_rows is at least
 *                    2^16 (fp64), 2^17 (fp32) or 2^18 (bf16), unless the caller sets
 *                    rows_per_thread, threads_per_row, block_threads, unroll,
 *                    staged or tile_order (a uniform mapping asked for). On
 *                    Zipf-distributed row lengths (1M-4M rows) the plan is
 *                    1.0-1.6x as fast as the best uniform threads per row;
 *                    over 200 held-out Zipf matrices (10k-4M rows) the
 *                    default takes 0.870 / 0.941 / 0.980 of the best uniform
 *                    mapping's time (fp64 / fp32 / bf16, geometric mean).
 *                    With the plan the other fields do not apply.
 * rows_per_thread > 1 and threads_per_row > 1 are exclusive, and staged
 * excludes plan = 1. Invalid values return PJDS_EINVAL.
 */
typedef struct pjds_launch {
  int32_t rows_per_thread;
  int32_t threads_per_row;
  int32_t block_threads;
  int32_t unroll;
  int32_t staged;
  int32_t index64;  /* 1: 64-bit element offsets even when 32 bits suffice (they are
                       used automatically from 2^31 stored entries on) */
  int32_t tile_order; /* 0 automatic, 1 the traversal table, -1 sorted order */
  int32_t plan;       /* 0 automatic, 1 the per-tile mapping of A->plan, -1 a uniform mapping */
} pjds_launch;

int pjds_spmv_cfg(const pjds_dev *A, const void *x, void *y, const pjds_launch *cfg, void *stream);

/*
 * The configuration pjds_spmv_cfg would launch for A and cfg (cfg = NULL: the
 * pjds_spmv default), with every 0 field replaced by its default, written to
 * *out; nothing is launched and no device memory is touched. Fields left at 0
 * take defaults; rows_per_thread > 1 alone implies threads_per_row = 1 and
 * vice versa. out->tile_order is 1 (the table is used) or -1 (sorted order);
 * out->plan is 1 (the per-tile mapping; the other fields then describe the
 * uniform mapping it replaces) or -1. Returns PJDS_EINVAL for a combination
 * pjds_spmv_cfg rejects.
 */
int pjds_spmv_resolve(const pjds_dev *A, const pjds_launch *cfg, pjds_launch *out);

/*
 * Pattern product y = S x, S the sparsity pattern of A (every stored entry
 * taken as 1): sorted row i sums x[col[col_start[j] + i]] for j < len(i), in
 * the order of the product with the same mapping, and writes y[perm[i]]
 * (y[i] in the permuted basis). It runs the traversal pjds_spmv_cfg would run for cfg (NULL: the
 * pjds_spmv default) without reading val: the column stream, the x gathers
 * and the y stores of the product and nothing else. Its time is therefore a
 * floor for the product's time with the same traversal, the gather ceiling
 * against which the product is measured besides HBM bandwidth (Eq. 1: the
 * alpha term, the traffic the right-hand side costs, is this part). Every
 * mapping but the staged kernel (PJDS_EINVAL): the kernel is the product's
 * own, with the values read from eight ones in L1 instead of val, so it keeps
 * the product's instructions, registers and occupancy; fma(1, x, acc) is
 * acc + x rounded once. The paper has no counterpart of this call.
 */
int pjds_spmv_pattern(const pjds_dev *A, const void *x, void *y, const pjds_launch *cfg, void *stream);

/*
 * Device status word of the staged kernel (see pjds_launch.staged): 0 when
 * every wait completed since the last clear, else bit 0 (a consumer wait ran
 * out) / bit 1 (a producer wait ran out). clear = 1 resets it. Waits for the
 * stream.
 */
int pjds_device_status(int32_t *status, int32_t clear, void *stream);

/*
 * Checked build only (libpjds_checked.so, compiled with PJDS_CHECKED; a test
 * build standing in for a memory checker): the product kernels with one or
 * T threads per row, several rows per thread, the per-tile mapping, the
 * batched launch and ELLPACK-R compare every jagged-diagonal index, element
 * offset, gathered column, block index and stored row with its array's
 * extent before the access, skip an access outside it and record the first
 * such access: *word = (code << 56) | index, code 1 jagged diagonal, 2
 * element offset, 3 gathered column, 4 stored row, 5 block index; 0 when
 * none. clear = 1 resets it. Waits for the stream. The normal build returns
 * PJDS_EINVAL.
 */
int pjds_check_word(uint64_t *word, int32_t clear, void *stream);

/*
 * Failure-detection self-test of the staged kernel's bounded waits: launches
 * one thread that waits on an mbarrier nothing completes (which = 0: as a
 * consumer, which = 1: as the producer). The wait gives up after its limit
 * (well under a second), sets status bit `which` and the kernel returns; the
 * context stays usable. Read the bit with pjds_device_status.
 */
int pjds_wait_selftest(int32_t which, void *stream);

/*
 * End-to-end product from host memory: copies x_host (n_cols elements) into
 * the caller's device buffer x_dev, runs pjds_spmv into y_dev, copies y_dev
 * back into y_host (n_rows elements) and waits for the stream. Host buffers
 * should be pinned for full copy bandwidth.
 */
int pjds_spmv_host(const pjds_dev *A, const void *x_host, void *y_host, void *x_dev, void *y_dev, void *stream);

/*
 * A stream of independent products from host memory: y_v = A x_v for
 * v < n_vec, x_host[v] holding n_cols and y_host[v] n_rows elements of A's
 * vector type (pinned host memory for full link bandwidth; the same host
 * buffer may appear more than once). x_dev[0..1] and y_dev[0..1] are two
 * caller-owned device buffers each (four distinct buffers), used in turn:
 * while product v runs on `stream`, x_{v+1} is copied in and y_{v-1} copied
 * out on two copy streams the call creates and orders with events. Eq. 2
 * adds the transfer time T_PCI to the product time T_MVM; here the two
 * overlap as far as the host link allows. Work already queued on `stream`
 * runs first; the call returns when every y_host[v] is written. Same mapping
 * and results as pjds_spmv. The paper has no counterpart of this call.
 * Errors: PJDS_EINVAL (n_vec < 0, a NULL pointer, a device buffer reused),
 * PJDS_ECUDA.
 */
int pjds_spmv_host_stream(const pjds_dev *A, int32_t n_vec, const void *const *x_host, void *const *y_host,
                          void *const *x_dev, void *const *y_dev, void *stream);

/*
 * Basis changes around an iterative solver (Sect. 2.1): for i < n_rows,
 *   pjds_permute:   v_perm[i] = v[perm[i]]   (original -> permuted basis)
 *   pjds_unpermute: v[perm[i]] = v_perm[i]   (permuted -> original basis)
 * Vectors are device memory of A's vector type and must not overlap.
 */
int pjds_permute(const pjds_dev *A, const void *v, void *v_perm, void *stream);
int pjds_unpermute(const pjds_dev *A, const void *v_perm, void *v, void *stream);

/* ------------------------------------------------------------------------ */
/* ELLPACK-R (Sect. 2.1, Listing 1)                                          */
/* ------------------------------------------------------------------------ */

/*
 * Host-side ELLPACK-R arrays, owned by the library until ellr_destroy. Rows
 * keep their original order and are padded to n_pad = ceil(n_rows/32)*32
 * (footnote to Sect. 2.1); each row's entries are shifted left into an
 * n_pad x n_max rectangle stored column by column: entry j of row i at
 * j * n_pad + i. row_max[i] is the length of row i (0 for padding rows);
 * padding entries hold value +0 and column -1.
 */
typedef struct ellr_host {
  int32_t n_rows, n_cols, n_pad, n_max;
  int64_t nnz, n_stored;
  int32_t dtype, reserved;
  int32_t *row_max; /* [n_pad]    */
  int32_t *col;     /* [n_stored] */
  void *val;        /* [n_stored] of dtype */
} ellr_host;

typedef struct ellr_dev {
  int32_t n_rows, n_cols, n_pad, n_max;
  int64_t nnz, n_stored;
  int32_t dtype, reserved;
  const int32_t *row_max;
  const int32_t *col;
  const void *val;
} ellr_dev;

/* Convert CRS to ELLPACK-R. Same arguments and errors as pjds_create. */
int ellr_create(int32_t n_rows, int32_t n_cols, const int64_t *row_ptr, const int32_t *col_idx,
                const double *val, int32_t dtype, ellr_host **out);

int ellr_destroy(ellr_host *h);

/*
 * y = A x with A in ELLPACK-R (Listing 1): one thread per row i computes
 * sum_{j < row_max[i]} val[j*n_pad + i] * x[col[j*n_pad + i]] with fused
 * multiply-add and writes y[i]. Same vector conventions as pjds_spmv.
 */
int ellr_spmv(const ellr_dev *A, const void *x, void *y, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* PJDS_H */
