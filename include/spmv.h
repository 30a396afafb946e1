/*
 * spmv.h -- C ABI of a GB300 (sm_103a) library for the CRS sparse matrix-vector
 * multiply of Schubert, Fehske, Hager and Wellein, "Hybrid-parallel sparse
 * matrix-vector multiplication with explicit communication overlap on current
 * multicore-based systems" (2011).
 *
 * Storage (Sect. 1.2): a matrix with n_rows rows is given by three arrays,
 *   row_ptr[n_rows+1]  starting offset of every row, row_ptr[0] == 0,
 *                      nondecreasing, row_ptr[n_rows] == nnz;
 *   col_idx[nnz]       column of every stored entry, 0 <= col_idx[k] < n_cols;
 *   val[nnz]           value of every stored entry, row by row.
 * Indices are 0-based (the paper's Fortran listing is 1-based).  Columns within a
 * row need not be sorted and repeated (row, col) entries are summed.
 *
 * Conventions for every call:
 *   - int32 indices; n_rows, n_cols, nnz < 2^31.
 *   - Vectors (x, y, g, grad_x, grad_val, X, Y) are caller-owned DEVICE pointers,
 *     borrowed for the duration of the call only.  Every compute call is
 *     asynchronous on the given stream (a cudaStream_t passed as void*; NULL is
 *     the legacy default stream).  A call returns once its work is enqueued.
 *   - Handles own device copies of what they hold and are not safe for concurrent
 *     applies from several host threads.
 *   - Errors are returned status codes; nothing is thrown across the ABI.  Errors
 *     of already-enqueued kernels surface as SPMV_ERR_CUDA on a later call.
 *   - beta == 0 means y is not read (NaN or Inf in y does not propagate).
 *   - Summation order within a row is unspecified; results match the FP64 row sum
 *     of Listing 1 to within |y - y_ref|_i <= 1e-13 * sum_j |a_ij x_j| for FP64
 *     operands and <= 1e-6 * sum_j |a_ij x_j| for FP32-stored operands, and are
 *     bit-exact when A and x are integer-valued with every partial sum exact.
 */
#ifndef SPMV_H
#define SPMV_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SPMV_OK = 0,
    SPMV_ERR_INVALID_ARG = 1,    /* null pointer, bad size, shape or dtype       */
    SPMV_ERR_INVALID_INDEX = 2,  /* row_ptr not a valid CRS offset array, or a
                                    column index outside [0, n_cols)             */
    SPMV_ERR_CUDA = 3,           /* a CUDA runtime call or kernel failed          */
    SPMV_ERR_ALLOC = 4,          /* device or host allocation failed              */
    SPMV_ERR_UNSUPPORTED = 5,    /* combination not provided by this library      */
    SPMV_ERR_TIMEOUT = 6,        /* a bounded on-device wait gave up              */
    SPMV_ERR_NOT_CONVERGED = 7   /* iterative solver hit its iteration cap        */
} spmv_status;

typedef enum { SPMV_F64 = 0, SPMV_F32 = 1 } spmv_dtype;

typedef struct spmv_matrix *spmv_handle;
typedef struct spmv_split *spmv_split_handle;
typedef struct spmv_batch *spmv_batch_handle;

/* Human-readable name of a status code (static storage). */
const char *spmv_status_string(spmv_status s);

/* Library version as 10000*major + 100*minor + patch. */
int32_t spmv_version(void);

/* ------------------------------------------------------------------------ */
/* Matrix handle (Sect. 1.2 storage; Listing 1 kernel)                        */
/* ------------------------------------------------------------------------ */

/* Create a handle from CRS arrays.  The arrays are validated (row_ptr[0] == 0,
 * nondecreasing, row_ptr[n_rows] == nnz, 0 <= col_idx < n_cols) and copied into
 * handle-owned device memory; the caller keeps ownership of its arrays.
 * is_device_ptr != 0: the three arrays are device pointers, else host pointers.
 * val_t selects FP64 or FP32 storage of the values.  The handle also derives,
 * from the row-length histogram, the kernel plan used by every apply (the tile
 * table and the per-thread nonzero count).  stream orders the copies; the call
 * synchronises the stream before returning.
 * Errors: SPMV_ERR_INVALID_ARG (null out, negative sizes, null arrays with
 * nnz > 0), SPMV_ERR_INVALID_INDEX (bad row_ptr or column), SPMV_ERR_ALLOC,
 * SPMV_ERR_CUDA.  *out is NULL on error. */
spmv_status spmv_create(spmv_handle *out, int32_t n_rows, int32_t n_cols, int64_t nnz,
                        const int32_t *row_ptr, const int32_t *col_idx, const void *val,
                        spmv_dtype val_t, int is_device_ptr, void *stream);

/* Release a handle and everything it owns (NULL is ignored).  Synchronises the
 * device work that may still use it. */
void spmv_destroy(spmv_handle h);

/* Symmetric CRS (Sect. 1.3.1: a symmetric matrix stored as its upper
 * triangle, which the paper names and sets aside).  The n x n matrix A is
 * given by U, its upper triangle with the diagonal: row_ptr[n+1], col_idx[nnz]
 * and val[nnz] as for spmv_create, every entry of row i having a column
 * j >= i (repeated entries are summed; columns need not be sorted), so each
 * off-diagonal value is stored once and serves a_ij and a_ji.  spmv_apply on
 * the handle computes y = alpha*A*x + beta*y with A = U + U_s^T (U_s: U
 * without its diagonal) in two passes of fixed summation order: the row sums
 * of U on the autotuned kernel (with beta), then the row sums of U_s^T added
 * onto y by the warp-chunk kernel that reads each value through its position
 * in U (a transposed index built once here, on the host: rows of U_s^T list
 * their entries by increasing position in U).  Results are deterministic.
 * spmv_set_values replaces U's values; spmv_apply (vector types as for
 * spmv_apply, except FP32 storage with an FP64 y), spmv_get_info, spmv_set_plan
 * (for the U pass), spmv_set_accumulator and spmv_destroy accept the handle;
 * the split form, block vectors, the reverse pass, the transposed structure,
 * the CG solvers and batches return SPMV_ERR_UNSUPPORTED.
 * Errors: as spmv_create, and SPMV_ERR_INVALID_INDEX for an entry left of the
 * diagonal. */
spmv_status spmv_create_symmetric(spmv_handle *out, int32_t n, int64_t nnz, const int32_t *row_ptr,
                                  const int32_t *col_idx, const void *val, spmv_dtype val_t,
                                  int is_device_ptr, void *stream);

/* Replace the stored values (same sparsity pattern) from a device pointer of
 * type t; t may differ from the handle's storage type only as FP64 -> FP32
 * storage or FP32 -> FP64 storage (converted on the device).  Asynchronous. */
spmv_status spmv_set_values(spmv_handle h, const void *val, spmv_dtype t, void *stream);

/* Shape and plan of a handle.  plan[0..7] receives: kernel family (as for
 * spmv_set_plan), entries per lane or thread segment E (family 5: the sorting
 * window sigma), threads per CTA, number of chunks, tiles or slices, rows per
 * chunk or tile cap (family 5: rows per slice), threads per row of the
 * row-vector kernel, number of rows longer than a chunk or tile (family 5: rows
 * of more than 128 entries), value dtype.  Any output may be NULL.  Builds the
 * plan's chunk table if needed (synchronises the device). */
spmv_status spmv_get_info(spmv_handle h, int32_t *n_rows, int32_t *n_cols, int64_t *nnz,
                          int32_t *plan);

/* Row-length histogram used by the autotuner: counts[L] = rows with exactly L
 * entries for L < nbins - 1, counts[nbins-1] = rows with >= nbins-1 entries.
 * counts is a HOST array of nbins int64. */
spmv_status spmv_row_histogram(spmv_handle h, int32_t nbins, int64_t *counts);

/* Override the autotuner's choice of kernel family and work per lane/thread.
 * family 0: warp-chunk kernel, param = entries per lane E (7 or 15: pipelined
 *           through a two-stage shared-memory ring; 8 or 16: direct loads);
 * family 1: row-vector kernel, param = threads per row (1,2,4,8,16,32);
 * family 2: staged tile kernel, param = entries per thread segment (odd, 3..31);
 * family 3: three-stage warp-chunk kernel (gathers one chunk ahead), E = 7, 11, 15;
 * family 4: slot-major warp-chunk kernel (values and column indices copied once
 *           into chunk-major, lane-interleaved order and loaded coalesced into
 *           registers; no shared-memory staging), E = 7, 9, 11, 15 (FP32 as well);
 *           the copy is built on first use and its values follow spmv_set_values;
 *           with FP32 storage and E = 7, 9 or 11 the default accumulator sums
 *           each lane's piece of a row (at most E entries) with FP32 FMAs and
 *           joins the pieces in float-float (see spmv_set_accumulator);
 * family 5: sorted row-slice kernel (SELL-C-sigma with C = 64: in each window
 *           of param rows, a power of two from 32 to 2^20, default 4096, the
 *           rows ordered by length and stored 64 rows at a time, two rows per
 *           lane; rows of more than 128 entries summed by a whole warp); FP64,
 *           and FP32 storage with the default accumulator (FP32 runs: a whole
 *           row when no row exceeds 9 entries, else blocks of 4 entries folded
 *           into float-float), other combinations run the slot-major kernel;
 *           copy built on first use, values follow spmv_set_values;
 * family 6: the slot-major kernel of family 4 with each chunk's values brought
 *           into a two-stage shared-memory ring per warp by 1-D bulk copies
 *           (cp.async.bulk) instead of register loads, so they bypass L1's miss
 *           handling; E = 7, 9 (FP64), 9, 15 (FP32 storage, float-float); FP64
 *           and FP32 vectors of the storage type, other combinations and the
 *           split form's row-mapped parts run family 4.  A bounded wait that
 *           gives up records a timeout (spmv_check_device_error).
 * param 0 keeps a default.  Results are unchanged up to summation order. */
spmv_status spmv_set_plan(spmv_handle h, int32_t family, int32_t param);

/* Accumulator of an FP32-storage handle: 0 = one FP64 FMA per entry (operands
 * widened exactly), 1 = FP32-pipe accumulation (default).  Setting 1 is, in the
 * slot-major kernel with E = 7, 9 or 11 (family 4 and the batched launch), FP32
 * FMA runs over each lane's piece of a row (at most E products: error at most
 * gamma_E = E u/(1 - E u) of sum |a_ij x_j|, u = 2^-24: 5.4e-7 for E = 9, 6.6e-7
 * for E = 11) joined across lanes by two-sum, and in the row-slice kernel
 * (family 5) FP32 FMA runs over a whole row of at most 11 entries or over blocks
 * of 4 entries folded into float-float
 * (gamma_4 ~ 2.4e-7); a row whose FP32 sum is not finite or below 2^-100 in
 * magnitude is summed again with FP64 FMAs.  Everywhere else it is exact-product
 * float-float accumulation (relative accuracy about 2^-44 of sum |a_ij x_j|),
 * which splits each product exactly only inside FP32's range: a row with a
 * nonzero product below 2^-100 in magnitude, an overflow of a product or of the
 * running sum, or an infinite or NaN operand is summed again with FP64 FMAs.
 * Either way every row is within 1e-6 * sum_j |a_ij x_j| of the FP64-accumulated
 * sum for every input (one more pass over a row's entries where the FP32 form
 * cannot guarantee it).  FP64 handles always accumulate with FP64 FMAs and
 * ignore this setting. */
spmv_status spmv_set_accumulator(spmv_handle h, int32_t acc);

/* Plain spMVM, Listing 1 generalised: y = alpha*A*x + beta*y.
 * x: n_cols entries of type xt; y: n_rows entries of type yt.  Supported
 * (value, x, y) types: (F64, F64, F64), (F32, F32, F32), (F32, F32, F64).  FP32
 * operands: the row sums are within 1e-6 * sum_j |a_ij x_j| of the FP64 sum of
 * the exact products over FP64's exponent range (FP32 runs or float-float, see
 * spmv_set_accumulator; rows outside FP32's range go through FP64 FMAs); an
 * FP32 y is then rounded once.
 * x and y must not overlap. */
spmv_status spmv_apply(spmv_handle h, double alpha, const void *x, spmv_dtype xt,
                       double beta, void *y, spmv_dtype yt, void *stream);

/* ------------------------------------------------------------------------ */
/* Local/nonlocal split form (Sect. 3.2 distribution; Sect. 3.4-3.5, Eq. 2)  */
/* ------------------------------------------------------------------------ */

/* Build the split plan of a square matrix once (the bookkeeping of Sect. 3.2):
 * nblocks contiguous row blocks (block_row_start: nblocks+1 HOST entries with
 * start[0] = 0, start[nblocks] = n_rows, nondecreasing; NULL = nonzeros balanced,
 * block b starting at the first row whose offset is >= ceil(b*nnz/nblocks)).  The
 * right-hand side is distributed like the rows, so column j is local to block b
 * iff start[b] <= j < start[b+1].  For each block the plan holds its halo map
 * (sorted distinct nonlocal columns), the local part A_loc and the nonlocal part
 * A_nl with columns renumbered into the concatenated halo buffer.
 * halo_count_out (optional HOST array of nblocks) receives the halo sizes.
 * The split handle references h, which must outlive it; its parts hold copies
 * of h's values taken at creation (after spmv_set_values on h, create the split
 * again).  Equal-rows blocks (the "constant rows" case of Fig. 6) are
 * block_row_start[b] = floor(b*n_rows/nblocks). */
spmv_status spmv_split_create(spmv_split_handle *out, spmv_handle h, int32_t nblocks,
                              const int32_t *block_row_start, int32_t *halo_count_out);
void spmv_split_destroy(spmv_split_handle hs);

/* Copy the plan out to HOST arrays (each optional): block_start[nblocks+1],
 * halo_count[nblocks], halo_map[total halo], nnz_local[nblocks],
 * nnz_nonlocal[nblocks]; *total_halo receives the halo length. */
spmv_status spmv_split_get_plan(spmv_split_handle hs, int32_t *nblocks, int32_t *block_start,
                                int32_t *halo_count, int64_t *total_halo, int32_t *halo_map,
                                int64_t *nnz_local, int64_t *nnz_nonlocal);

/* Split spMVM (task-mode analogue of Sect. 3.5, Fig. kernel_schemes (c)):
 *   s_compute: record "x ready";
 *   s_comm:    wait for it, gather halo[h] = x[halo_map[h]] (the stand-in for the
 *              MPI exchange), record "halo ready";
 *   s_compute: y = beta*y + alpha*A_loc*x over all blocks (overlaps the gather),
 *              wait for "halo ready", then y += alpha*A_nl*halo.
 * The result vector is written twice, as in Eq. 2.  FP64 x and y only.
 * s_comm may equal s_compute (naive overlap of Sect. 3.4 on one stream). */
spmv_status spmv_apply_split(spmv_split_handle hs, double alpha, const double *x, double beta,
                             double *y, void *s_compute, void *s_comm);

/* Split spMVM in vector mode (Sect. 3.4, Fig. kernel_schemes (a): the halo
 * exchange completes before any computation): on stream s, gather the whole
 * halo, then one pass over the full matrix, whose nonlocal columns are
 * renumbered into the extended vector [x | halo] at split creation, computes
 * y = alpha*A*x + beta*y, writing y once (Eq. 1 traffic plus the gather).  The
 * plan holds a handle-owned copy of the extended vector and of the renumbered
 * matrix.  FP64 x and y only; x and y are borrowed device pointers.
 * SPMV_ERR_UNSUPPORTED if n_rows + total halo does not fit in int32. */
spmv_status spmv_apply_split_vector(spmv_split_handle hs, double alpha, const double *x, double beta,
                                    double *y, void *stream);

/* Copy the halo buffer filled by the last spmv_apply_split (task mode) to a HOST array of
 * total-halo doubles (synchronises s). */
spmv_status spmv_split_get_halo(spmv_split_handle hs, double *halo_out, void *stream);

/* ------------------------------------------------------------------------ */
/* Block vectors                                                               */
/* ------------------------------------------------------------------------ */

/* Y = alpha*A*X + beta*Y for nrhs right-hand sides stored interleaved:
 * X[j*nrhs + r], Y[i*nrhs + r] (row-major, leading dimension nrhs).
 * 1 <= nrhs <= 64.  vt: SPMV_F64 (X, Y FP64; FP64 values) only.  Groups of 4
 * right-hand sides run on the sorted row slices of plan family 5 (built on first
 * use, whatever the handle's plan) when they pad at most 10 % and, for scattered
 * columns, X fits in L2; the rest on the tile kernel.  Results are unchanged up
 * to summation order. */
spmv_status spmm_apply(spmv_handle h, int32_t nrhs, double alpha, const void *X, double beta,
                       void *Y, spmv_dtype vt, void *stream);

/* ------------------------------------------------------------------------ */
/* Reverse pass                                                                */
/* ------------------------------------------------------------------------ */

/* Gradients of f = g^T y with y = alpha*A(val)*x:
 *   grad_x[j]   = alpha * sum_i a_ij g_i   (alpha*A^T g; n_cols entries), through a
 *                 transposed CRS built once on the device and kept in the handle;
 *   grad_val[k] = alpha * g[row(k)] * x[col_idx[k]]   (nnz entries, CRS order).
 * Both outputs are overwritten; either may be NULL.  FP64 handles take FP64 g,
 * x and outputs; FP32-storage handles take FP32 g, x and write FP32 outputs.
 * The first call after new values reads A^T's values through the permutation;
 * the second lays them out in A^T order once (kept until spmv_set_values) and
 * from then on grad_x runs on a copy of A^T (row slices for stencil-like
 * matrices with at least 12 entries per row, slot-major otherwise).  Results are
 * unchanged up to summation order. */
spmv_status spmv_backward(spmv_handle h, double alpha, const void *g, const void *x,
                          void *grad_x, void *grad_val, void *stream);

/* Copy the transposed structure to HOST arrays (builds it if needed):
 * rowT_ptr[n_cols+1], colT_idx[nnz] (row of A of each entry), perm[nnz] (position
 * in A of each entry of A^T).  Within a row of A^T, entries are in increasing
 * position of A. */
spmv_status spmv_get_transpose(spmv_handle h, int32_t *rowT_ptr, int32_t *colT_idx,
                               int32_t *perm, void *stream);

/* Transposed CRS build that allocates nothing (no counterpart in the paper).
 *
 * Some callers cannot allocate device memory at the moment they need this
 * result: real-time or latency-bound loops that must not wait on the allocator
 * or risk an out-of-memory failure mid-run, and programs whose device memory is
 * already reserved by another allocator (a pool that owns the whole device).
 * This entry point builds the same structure as spmv_get_transpose from CRS
 * arrays already on the device and writes it to caller-provided device
 * buffers; its scratch (one counter per column, the scans' block sums and the
 * histograms of the column sort, about 6.3 MB) is a fixed array compiled into
 * the library, which every GPU that loads the library holds until the process
 * exits.  It calls no cudaMalloc, cudaFree or other allocating routine.  Its
 * work is linear in nnz whatever the column lengths (a stable radix sort of
 * the entries by column).
 *
 *   row_ptr[n_rows+1], col_idx[nnz]: a valid CRS structure on the device;
 *   rowT_ptr[n_cols+1], colT_idx[nnz], perm[nnz]: device outputs, as for
 *   spmv_get_transpose (rows of A^T in increasing position of A).
 * n_cols must not exceed SPMV_NOALLOC_MAX_COLS (larger sizes return
 * SPMV_ERR_UNSUPPORTED before any work is enqueued).  The arrays are not
 * validated: a column outside [0, n_cols) is left out of rowT_ptr (and placed
 * after the last row of A^T), so the output is then not a transpose, but no
 * memory outside the arrays is touched.
 * The first call on a device looks up the scratch array's device address (once
 * per device, with that device current); make that first call before any
 * stream capture.  Every call shares the one array and re-clears the part it
 * uses, so calls that may overlap on the GPU (other streams, other host threads)
 * race and must be ordered by the caller.  Asynchronous on stream. */
#define SPMV_NOALLOC_MAX_COLS (1 << 20)
spmv_status spmv_transpose_noalloc(int32_t n_rows, int32_t n_cols, int64_t nnz,
                                   const int32_t *row_ptr, const int32_t *col_idx,
                                   int32_t *rowT_ptr, int32_t *colT_idx, int32_t *perm,
                                   void *stream);

/* ------------------------------------------------------------------------ */
/* Batched persistent launch                                                   */
/* ------------------------------------------------------------------------ */

/* Group count matrix handles (all FP64 or all FP32 storage) into one batch whose
 * apply is a single persistent kernel launch over the warp chunks of every
 * matrix (the slot-major chunk kernel on a concatenated slot-major copy of the
 * members, one per group of members tuned alike), captured once into a CUDA
 * graph and replayed.  spmv_batched_get_member_plan reports each member's
 * entries per lane.
 * The batch holds its own copy of the values: after spmv_set_values on a member,
 * the next spmv_batched_apply lays that member's values out again (on stream,
 * before the launch).  The handles must outlive the batch. */
spmv_status spmv_batched_create(spmv_batch_handle *out, int32_t count, const spmv_handle *mats);
void spmv_batched_destroy(spmv_batch_handle b);

/* y_m = alpha*A_m*x_m + beta*y_m for every matrix m.  x and y are HOST arrays of
 * count device pointers (vector types follow the storage type: FP64 or FP32).
 * When the pointer set or alpha/beta differ from the previous call the device
 * pointer table is rewritten and the graph re-instantiated; otherwise the
 * instantiated graph is replayed on stream. */
spmv_status spmv_batched_apply(spmv_batch_handle b, double alpha, const void *const *x,
                               double beta, void *const *y, void *stream);

/* plan[0..3]: E (0 when the members were tuned apart, see below), threads per
 * CTA, total chunks, persistent grid size (0 when the kernel sizes its
 * persistent grid at launch). */
spmv_status spmv_batched_get_info(spmv_batch_handle b, int32_t *plan);

/* The entries per lane each member runs with (HOST array of count int32).  The
 * batch tunes its members apart from their own row-length histograms (mean row
 * length below 4 entries: 7 per lane, else 9; a single matrix switches at 8,
 * but in a batch a separate group for members of 4-8 entries per row measured
 * slower than running them at 9); when both occur, the members of each group
 * share one slot-major copy and the one persistent launch walks both groups
 * (not in the paper). */
spmv_status spmv_batched_get_member_plan(spmv_batch_handle b, int32_t *entries_per_lane);

/* ------------------------------------------------------------------------ */
/* Mixed-precision iterative refinement CG                                     */
/* ------------------------------------------------------------------------ */

/* Solve A x = b for SPD A (FP64 handle) by iterative refinement:
 *   outer (FP64): r = b - A x (FP64 spMVM), ||r||_2, stop when
 *                 ||r||_2 <= outer_tol*||b||_2 or after max_outer steps;
 *   inner (FP32 storage): CG on A d = r with FP32 values and vectors, FP64
 *                 accumulation inside the spMVM and the dot products, stopped at
 *                 relative residual inner_tol or max_inner iterations;
 *   update (FP64): x += d.
 * b, x: device FP64 vectors of n_rows; x is overwritten (x0 = 0).
 * stats (optional HOST array of 4 doubles): outer steps, total inner iterations,
 * final relative residual ||b - A x||/||b|| (FP64, on the device), seconds.
 * Returns SPMV_ERR_NOT_CONVERGED if the outer cap is reached first.
 * Synchronises the stream (one scalar read-back every 8 inner iterations, so an
 * inner solve may run up to 7 iterations past its tolerance). */
spmv_status spmv_ir_cg(spmv_handle h, const double *b, double *x, double outer_tol,
                       int32_t max_outer, double inner_tol, int32_t max_inner,
                       double *stats, void *stream);

/* FP64 conjugate gradients on the device with the FP64 spMVM (the comparison
 * solver for spmv_ir_cg): x0 = 0, stop at ||r||_2 <= tol*||b||_2 (recursive
 * residual) or max_iter.  stats as for spmv_ir_cg (outer steps = 1). */
spmv_status spmv_cg(spmv_handle h, const double *b, double *x, double tol, int32_t max_iter,
                    double *stats, void *stream);

/* ------------------------------------------------------------------------ */
/* Error word                                                                  */
/* ------------------------------------------------------------------------ */

/* Read and clear the handle's device error word (synchronises stream).  Returns
 * SPMV_ERR_TIMEOUT if a bounded on-device wait gave up since the last check,
 * SPMV_OK otherwise. */
spmv_status spmv_check_device_error(spmv_handle h, void *stream);

/* Check a CRS structure held in DEVICE memory on the device (the checks
 * spmv_create applies on the host): row_ptr[0] == 0, row_ptr nondecreasing,
 * row_ptr[n_rows] == nnz, 0 <= col_idx[k] < n_cols.  row_ptr has n_rows + 1
 * entries and col_idx nnz; only those are read, whatever their values, and a
 * violation is recorded in a device word (no trap).  Synchronises stream.
 * Returns SPMV_ERR_INVALID_INDEX on a violation, SPMV_ERR_INVALID_ARG for
 * negative sizes, nnz >= 2^31 or null pointers. */
spmv_status spmv_validate_device(int32_t n_rows, int32_t n_cols, int64_t nnz, const int32_t *row_ptr,
                                 const int32_t *col_idx, void *stream);

/* Self-test of the failure detection: one warp waits on an on-device barrier
 * that nothing completes, with a wall-time limit of limit_ns (1 us .. 1 s, the
 * limit every on-device wait of the library uses); the wait gives up, records
 * the timeout in the handle's error word and the kernel returns, leaving the
 * context usable.  Synchronises stream; returns SPMV_ERR_TIMEOUT when the path
 * works (then the error word is clear again). */
spmv_status spmv_selftest_wait_timeout(spmv_handle h, int64_t limit_ns, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* SPMV_H */
