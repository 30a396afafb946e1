/*
 * Oracle for the CRS sparse matrix-vector multiply of Schubert, Fehske, Hager and
 * Wellein, "Hybrid-parallel sparse matrix-vector multiplication with explicit
 * communication overlap on current multicore-based systems" (2011).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct CPU
 * statement of what the GPU library computes.  Only the test suite, the smoke check
 * and the CPU-baseline leg of the benchmark may load it; the library never does.
 * It shares no code, header, table or helper with the CUDA path.
 *
 * Conventions (readings of the paper, which prints only the Fortran kernel of
 * Listing 1 with 1-based indices and an accumulating update C(i) = C(i) + ...):
 *   - indices are 0-based: row_ptr[0..n_rows], col_idx[0..nnz), val[0..nnz);
 *   - the update is generalised to y = alpha*A*x + beta*y; beta == 0 means y is not
 *     read (a NaN in y does not propagate);
 *   - the row sum runs over k in increasing order, in FP64, without FMA contraction
 *     (the file is compiled with -ffp-contract=off);
 *   - duplicate (row, col) entries are summed; columns need not be sorted;
 *   - empty rows give y_i = beta*y_i.
 * Everything is FP64.  FP32-stored operands are passed here after an exact
 * upcast to FP64.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Listing 1 (Sect. 1.2), generalised to alpha/beta.  absrow (nullable) receives
 * sum_k |val[k] * x[col_idx[k]]| per row, the scale of the tolerance bound. */
void oracle_spmv(int32_t n_rows, const int32_t *row_ptr, const int32_t *col_idx,
                 const double *val, const double *x, double alpha, double beta,
                 double *y, double *absrow)
{
    for (int32_t i = 0; i < n_rows; ++i) {
        double acc = 0.0, mag = 0.0;
        for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            double p = val[k] * x[col_idx[k]];
            acc = acc + p;
            mag = mag + fabs(p);
        }
        double yin = (beta == 0.0) ? 0.0 : y[i];
        if (beta == 0.0)
            y[i] = alpha * acc;
        else
            y[i] = alpha * acc + beta * yin;
        if (absrow)
            absrow[i] = fabs(alpha) * mag + fabs(beta * yin);
    }
}

/* Thread chunks of the explicit work distribution of Sect. 3.5: one contiguous,
 * nonzero-balanced range of rows per thread.  Thread t of T starts at the first
 * row whose starting offset is at least ceil(t*nnz/T) (the block rule of
 * Sect. 3.2 applied to threads); thread 0 starts at row 0 and the last thread
 * ends at n_rows.  bounds receives T+1 row indices. */
static int32_t first_row_at(int32_t n_rows, const int32_t *row_ptr, int64_t target)
{
    int32_t lo = 0, hi = n_rows;
    while (lo < hi) {
        int32_t mid = lo + (hi - lo) / 2;
        if (row_ptr[mid] < target)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

void oracle_thread_rows(int32_t n_rows, const int32_t *row_ptr, int32_t nthreads, int32_t *bounds)
{
    int64_t nnz = row_ptr[n_rows];
    bounds[0] = 0;
    for (int32_t t = 1; t < nthreads; ++t)
        bounds[t] = first_row_at(n_rows, row_ptr, ((int64_t)t * nnz + nthreads - 1) / nthreads);
    bounds[nthreads] = n_rows;
}

int oracle_num_threads(void);

static int32_t threads_or_max(int32_t nthreads)
{
    return nthreads > 0 ? nthreads : oracle_num_threads();
}

#ifdef _OPENMP
#define THREAD_ID() omp_get_thread_num()
#else
#define THREAD_ID() 0
#endif

/* Listing 1's row loop over rows [lo, hi), generalised to alpha/beta, with the
 * arithmetic of oracle_spmv (no magnitude sum). */
static void spmv_rows(int32_t lo, int32_t hi, const int32_t *row_ptr, const int32_t *col_idx,
                      const double *val, const double *x, double alpha, double beta, double *y)
{
    for (int32_t i = lo; i < hi; ++i) {
        double acc = 0.0;
        for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k)
            acc = acc + val[k] * x[col_idx[k]];
        if (beta == 0.0)
            y[i] = alpha * acc;
        else
            y[i] = alpha * acc + beta * y[i];
    }
}

/* The node-level parallelisation of Sect. 2 (the outer row loop of Listing 1
 * split across OpenMP threads) with the explicit work distribution of Sect. 3.5:
 * thread t computes the rows of oracle_thread_rows' chunk t.  nthreads <= 0 means
 * every available thread; 1 is the single-thread loop.  Same per-row arithmetic
 * as oracle_spmv, so the result does not depend on the thread count.  The
 * arrays are used where the caller placed them (see oracle_node_* for the
 * first-touch placement). */
void oracle_spmv_omp(int32_t n_rows, const int32_t *row_ptr, const int32_t *col_idx,
                     const double *val, const double *x, double alpha, double beta,
                     double *y, int32_t nthreads)
{
    int32_t T = threads_or_max(nthreads);
    int32_t *bounds = (int32_t *)malloc(sizeof(int32_t) * ((size_t)T + 1));
    oracle_thread_rows(n_rows, row_ptr, T, bounds);
#pragma omp parallel num_threads(T)
    {
        int32_t t = THREAD_ID();
        spmv_rows(bounds[t], bounds[t + 1], row_ptr, col_idx, val, x, alpha, beta, y);
    }
    free(bounds);
}

/* FP32-stored values and vectors with FP64 accumulation (the precision form of
 * the library, not in the paper): each product of two floats is formed exactly
 * in FP64, the row sum runs in FP64 in increasing k, and y_i = alpha*acc +
 * beta*y_i is rounded once to float.  Thread chunks as oracle_spmv_omp. */
void oracle_spmv_f32(int32_t n_rows, const int32_t *row_ptr, const int32_t *col_idx,
                     const float *val, const float *x, double alpha, double beta,
                     float *y, int32_t nthreads)
{
    int32_t T = threads_or_max(nthreads);
    int32_t *bounds = (int32_t *)malloc(sizeof(int32_t) * ((size_t)T + 1));
    oracle_thread_rows(n_rows, row_ptr, T, bounds);
#pragma omp parallel num_threads(T)
    {
        int32_t t = THREAD_ID();
        for (int32_t i = bounds[t]; i < bounds[t + 1]; ++i) {
            double acc = 0.0;
            for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k)
                acc = acc + (double)val[k] * (double)x[col_idx[k]];
            double out;
            if (beta == 0.0)
                out = alpha * acc;
            else
                out = alpha * acc + beta * (double)y[i];
            y[i] = (float)out;
        }
    }
    free(bounds);
}

/* Position of column j in the sorted list map[0..count), or -1. */
static int32_t find_sorted(const int32_t *map, int32_t count, int32_t j)
{
    int32_t lo = 0, hi = count;
    while (lo < hi) {
        int32_t mid = lo + (hi - lo) / 2;
        if (map[mid] < j)
            lo = mid + 1;
        else
            hi = mid;
    }
    return (lo < count && map[lo] == j) ? lo : -1;
}

/* The local/nonlocal split of one multiplication (Sect. 3.4), over the row
 * blocks of Sect. 3.2 (block_start: nblocks+1 row indices; halo_count and
 * halo_map as oracle_split_halo writes them).  For each block b with rows
 * [s_b, s_{b+1}):
 *   1. halo[h] = x[map_b[h]] (the nonlocal right-hand side elements it receives);
 *   2. local part:    y_i = alpha*sum_{local k} val[k]*x[col[k]] (+ beta*y_i),
 *                     k increasing, a column being local iff it lies in [s_b, s_{b+1});
 *   3. nonlocal part: y_i = y_i + alpha*sum_{nonlocal k} val[k]*halo[pos(col[k])],
 *                     k increasing, for rows with at least one nonlocal entry
 *                     (y is written a second time, the extra traffic of Eq. 2).
 * pos() is the binary search of the column in the block's sorted map.  halo is a
 * work array of the total halo length. */
void oracle_spmv_split(int32_t n_rows, const int32_t *row_ptr, const int32_t *col_idx,
                       const double *val, const double *x, double alpha, double beta,
                       double *y, int32_t nblocks, const int32_t *block_start,
                       const int32_t *halo_count, const int32_t *halo_map, double *halo)
{
    int64_t off = 0;
    (void)n_rows;
    for (int32_t b = 0; b < nblocks; ++b) {
        int32_t lo = block_start[b], hi = block_start[b + 1];
        const int32_t *map = halo_map + off;
        double *hb = halo + off;
        for (int32_t h = 0; h < halo_count[b]; ++h)
            hb[h] = x[map[h]];
        for (int32_t i = lo; i < hi; ++i) {
            double acc = 0.0;
            for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
                int32_t j = col_idx[k];
                if (j >= lo && j < hi)
                    acc = acc + val[k] * x[j];
            }
            if (beta == 0.0)
                y[i] = alpha * acc;
            else
                y[i] = alpha * acc + beta * y[i];
        }
        for (int32_t i = lo; i < hi; ++i) {
            double acc = 0.0;
            int32_t any = 0;
            for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
                int32_t j = col_idx[k];
                if (!(j >= lo && j < hi)) {
                    acc = acc + val[k] * hb[find_sorted(map, halo_count[b], j)];
                    any = 1;
                }
            }
            if (any)
                y[i] = y[i] + alpha * acc;
        }
        off += halo_count[b];
    }
}

/* ---------------------------------------------------------------------------
 * The node-level CPU code as the paper runs it (Sect. 2 and 3.5), for timing:
 * every array the multiplication touches is copied into memory that is first
 * touched by the thread that later computes with it (NUMA-aware placement by
 * first touch), and each thread owns one contiguous, nonzero-balanced chunk of
 * rows (oracle_thread_rows).  The node holds the FP64 matrix and vectors, the
 * FP32-stored copies of values and vectors, and the split form over nblocks row
 * blocks (local and nonlocal entries of each row stored apart, nonlocal columns
 * replaced once by their position in the concatenated halo buffer: the
 * bookkeeping of Sect. 3.2, done once).  Every product is the same arithmetic as
 * oracle_spmv (plain), oracle_spmv_f32 (FP32 storage) and oracle_spmv_split
 * (split form), row by row.
 * ------------------------------------------------------------------------- */
typedef struct oracle_node {
    int32_t n_rows, n_cols, T, nblocks;
    int32_t *bounds;                  /* T+1 thread chunk bounds */
    int32_t *rp, *ci;                 /* CRS */
    double *val, *x, *y;
    float *val32, *x32, *y32;
    /* split form */
    int32_t *blk_lo, *blk_hi;         /* block of each row: [lo, hi) */
    int32_t *rpl, *cil, *rpn, *cin;   /* local / nonlocal CRS (cin: halo positions) */
    double *vall, *valn;
    int32_t *hmap;                    /* concatenated halo maps */
    double *halo;
    int64_t total_halo;
    int32_t *hbounds;                 /* T+1 chunk bounds of the halo gather */
} oracle_node;

static void *alloc_untouched(size_t bytes)
{
    void *p = NULL;
    if (bytes == 0)
        bytes = 64;
    if (posix_memalign(&p, 64, bytes) != 0)
        return NULL;
    return p;
}

void oracle_node_destroy(oracle_node *nd);

oracle_node *oracle_node_create(int32_t n_rows, int32_t n_cols, const int32_t *row_ptr,
                                const int32_t *col_idx, const double *val, const double *x,
                                int32_t nthreads, int32_t nblocks, const int32_t *block_start,
                                const int32_t *halo_count, const int32_t *halo_map)
{
    oracle_node *nd = (oracle_node *)calloc(1, sizeof(oracle_node));
    int64_t nnz = row_ptr[n_rows];
    nd->n_rows = n_rows;
    nd->n_cols = n_cols;
    nd->T = threads_or_max(nthreads);
    nd->nblocks = nblocks;
    nd->bounds = (int32_t *)malloc(sizeof(int32_t) * ((size_t)nd->T + 1));
    oracle_thread_rows(n_rows, row_ptr, nd->T, nd->bounds);
    nd->rp = (int32_t *)alloc_untouched(sizeof(int32_t) * ((size_t)n_rows + 1));
    nd->ci = (int32_t *)alloc_untouched(sizeof(int32_t) * (size_t)nnz);
    nd->val = (double *)alloc_untouched(sizeof(double) * (size_t)nnz);
    nd->val32 = (float *)alloc_untouched(sizeof(float) * (size_t)nnz);
    nd->x = (double *)alloc_untouched(sizeof(double) * (size_t)n_cols);
    nd->x32 = (float *)alloc_untouched(sizeof(float) * (size_t)n_cols);
    nd->y = (double *)alloc_untouched(sizeof(double) * (size_t)n_rows);
    nd->y32 = (float *)alloc_untouched(sizeof(float) * (size_t)n_rows);
    /* split bookkeeping on one thread (once), into staging arrays */
    int32_t *cnt_l = (int32_t *)calloc((size_t)n_rows + 1, sizeof(int32_t));
    int32_t *cnt_n = (int32_t *)calloc((size_t)n_rows + 1, sizeof(int32_t));
    int32_t *blo = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n_rows + 1));
    int32_t *bhi = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n_rows + 1));
    int64_t *hoff = (int64_t *)calloc((size_t)nblocks + 1, sizeof(int64_t));
    for (int32_t b = 0; b < nblocks; ++b)
        hoff[b + 1] = hoff[b] + halo_count[b];
    nd->total_halo = nblocks > 0 ? hoff[nblocks] : 0;
    for (int32_t b = 0; b < nblocks; ++b)
        for (int32_t i = block_start[b]; i < block_start[b + 1]; ++i) {
            blo[i] = block_start[b];
            bhi[i] = block_start[b + 1];
        }
    for (int32_t i = 0; i < n_rows; ++i)
        for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            int32_t j = col_idx[k];
            if (j >= blo[i] && j < bhi[i])
                cnt_l[i + 1] += 1;
            else
                cnt_n[i + 1] += 1;
        }
    for (int32_t i = 0; i < n_rows; ++i) {
        cnt_l[i + 1] += cnt_l[i];
        cnt_n[i + 1] += cnt_n[i];
    }
    int64_t nl = cnt_l[n_rows], nn = cnt_n[n_rows];
    int32_t *s_cil = (int32_t *)malloc(sizeof(int32_t) * ((size_t)nl + 1));
    int32_t *s_cin = (int32_t *)malloc(sizeof(int32_t) * ((size_t)nn + 1));
    double *s_vall = (double *)malloc(sizeof(double) * ((size_t)nl + 1));
    double *s_valn = (double *)malloc(sizeof(double) * ((size_t)nn + 1));
    for (int32_t b = 0; b < nblocks; ++b)
        for (int32_t i = block_start[b]; i < block_start[b + 1]; ++i) {
            int32_t pl = cnt_l[i], pn = cnt_n[i];
            for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
                int32_t j = col_idx[k];
                if (j >= blo[i] && j < bhi[i]) {
                    s_cil[pl] = j;
                    s_vall[pl++] = val[k];
                } else {
                    s_cin[pn] = (int32_t)(hoff[b] + find_sorted(halo_map + hoff[b], halo_count[b], j));
                    s_valn[pn++] = val[k];
                }
            }
        }
    nd->blk_lo = (int32_t *)alloc_untouched(sizeof(int32_t) * (size_t)n_rows);
    nd->blk_hi = (int32_t *)alloc_untouched(sizeof(int32_t) * (size_t)n_rows);
    nd->rpl = (int32_t *)alloc_untouched(sizeof(int32_t) * ((size_t)n_rows + 1));
    nd->rpn = (int32_t *)alloc_untouched(sizeof(int32_t) * ((size_t)n_rows + 1));
    nd->cil = (int32_t *)alloc_untouched(sizeof(int32_t) * (size_t)nl);
    nd->cin = (int32_t *)alloc_untouched(sizeof(int32_t) * (size_t)nn);
    nd->vall = (double *)alloc_untouched(sizeof(double) * (size_t)nl);
    nd->valn = (double *)alloc_untouched(sizeof(double) * (size_t)nn);
    nd->hmap = (int32_t *)alloc_untouched(sizeof(int32_t) * (size_t)nd->total_halo);
    nd->halo = (double *)alloc_untouched(sizeof(double) * (size_t)nd->total_halo);
    nd->hbounds = (int32_t *)malloc(sizeof(int32_t) * ((size_t)nd->T + 1));
    for (int32_t t = 0; t <= nd->T; ++t)
        nd->hbounds[t] = (int32_t)(nd->total_halo * t / nd->T);
    /* first touch: each thread writes the parts it computes with */
#pragma omp parallel num_threads(nd->T)
    {
        int32_t t = THREAD_ID();
        int32_t lo = nd->bounds[t], hi = nd->bounds[t + 1];
        for (int32_t i = lo; i < hi; ++i) {
            nd->rp[i] = row_ptr[i];
            nd->rpl[i] = cnt_l[i];
            nd->rpn[i] = cnt_n[i];
            nd->blk_lo[i] = blo[i];
            nd->blk_hi[i] = bhi[i];
            nd->y[i] = 0.0;
            nd->y32[i] = 0.0f;
        }
        if (t == nd->T - 1) {
            nd->rp[n_rows] = row_ptr[n_rows];
            nd->rpl[n_rows] = cnt_l[n_rows];
            nd->rpn[n_rows] = cnt_n[n_rows];
        }
        for (int64_t k = row_ptr[lo]; k < row_ptr[hi]; ++k) {
            nd->ci[k] = col_idx[k];
            nd->val[k] = val[k];
            nd->val32[k] = (float)val[k];
        }
        for (int64_t k = cnt_l[lo]; k < cnt_l[hi]; ++k) {
            nd->cil[k] = s_cil[k];
            nd->vall[k] = s_vall[k];
        }
        for (int64_t k = cnt_n[lo]; k < cnt_n[hi]; ++k) {
            nd->cin[k] = s_cin[k];
            nd->valn[k] = s_valn[k];
        }
        /* x is distributed like the rows (Sect. 3.2); columns past n_rows go
         * to the last thread */
        int32_t xlo = lo < n_cols ? lo : n_cols, xhi = hi < n_cols ? hi : n_cols;
        if (t == nd->T - 1)
            xhi = n_cols;
        for (int32_t j = xlo; j < xhi; ++j) {
            nd->x[j] = x[j];
            nd->x32[j] = (float)x[j];
        }
        for (int32_t h = nd->hbounds[t]; h < nd->hbounds[t + 1]; ++h) {
            nd->hmap[h] = halo_map[h];
            nd->halo[h] = 0.0;
        }
    }
    free(cnt_l);
    free(cnt_n);
    free(blo);
    free(bhi);
    free(hoff);
    free(s_cil);
    free(s_cin);
    free(s_vall);
    free(s_valn);
    return nd;
}

void oracle_node_destroy(oracle_node *nd)
{
    if (!nd)
        return;
    free(nd->bounds); free(nd->rp); free(nd->ci); free(nd->val); free(nd->x); free(nd->y);
    free(nd->val32); free(nd->x32); free(nd->y32);
    free(nd->blk_lo); free(nd->blk_hi); free(nd->rpl); free(nd->cil); free(nd->rpn); free(nd->cin);
    free(nd->vall); free(nd->valn); free(nd->hmap); free(nd->halo); free(nd->hbounds);
    free(nd);
}

/* y = alpha*A*x + beta*y on the node's own arrays (plain FP64). */
void oracle_node_spmv(oracle_node *nd, double alpha, double beta)
{
#pragma omp parallel num_threads(nd->T)
    {
        int32_t t = THREAD_ID();
        spmv_rows(nd->bounds[t], nd->bounds[t + 1], nd->rp, nd->ci, nd->val, nd->x, alpha, beta, nd->y);
    }
}

/* The FP32-storage product on the node's float copies (arithmetic of
 * oracle_spmv_f32). */
void oracle_node_spmv_f32(oracle_node *nd, double alpha, double beta)
{
#pragma omp parallel num_threads(nd->T)
    {
        int32_t t = THREAD_ID();
        for (int32_t i = nd->bounds[t]; i < nd->bounds[t + 1]; ++i) {
            double acc = 0.0;
            for (int32_t k = nd->rp[i]; k < nd->rp[i + 1]; ++k)
                acc = acc + (double)nd->val32[k] * (double)nd->x32[nd->ci[k]];
            double out;
            if (beta == 0.0)
                out = alpha * acc;
            else
                out = alpha * acc + beta * (double)nd->y32[i];
            nd->y32[i] = (float)out;
        }
    }
}

/* The split form on the node (arithmetic of oracle_spmv_split): halo gather,
 * then the local part of every row, then the nonlocal part of every row that has
 * nonlocal entries; each thread on its own chunk, with a barrier between the
 * steps (the halo must be complete before any nonlocal part runs). */
void oracle_node_spmv_split(oracle_node *nd, double alpha, double beta)
{
#pragma omp parallel num_threads(nd->T)
    {
        int32_t t = THREAD_ID();
        for (int32_t h = nd->hbounds[t]; h < nd->hbounds[t + 1]; ++h)
            nd->halo[h] = nd->x[nd->hmap[h]];
        int32_t lo = nd->bounds[t], hi = nd->bounds[t + 1];
        for (int32_t i = lo; i < hi; ++i) {
            double acc = 0.0;
            for (int32_t k = nd->rpl[i]; k < nd->rpl[i + 1]; ++k)
                acc = acc + nd->vall[k] * nd->x[nd->cil[k]];
            if (beta == 0.0)
                nd->y[i] = alpha * acc;
            else
                nd->y[i] = alpha * acc + beta * nd->y[i];
        }
#pragma omp barrier
        for (int32_t i = lo; i < hi; ++i) {
            if (nd->rpn[i + 1] == nd->rpn[i])
                continue;
            double acc = 0.0;
            for (int32_t k = nd->rpn[i]; k < nd->rpn[i + 1]; ++k)
                acc = acc + nd->valn[k] * nd->halo[nd->cin[k]];
            nd->y[i] = nd->y[i] + alpha * acc;
        }
    }
}

void oracle_node_set_y(oracle_node *nd, const double *y, const float *y32)
{
    for (int32_t i = 0; i < nd->n_rows; ++i) {
        if (y)
            nd->y[i] = y[i];
        if (y32)
            nd->y32[i] = y32[i];
    }
}

void oracle_node_get_y(const oracle_node *nd, double *y, float *y32)
{
    for (int32_t i = 0; i < nd->n_rows; ++i) {
        if (y)
            y[i] = nd->y[i];
        if (y32)
            y32[i] = nd->y32[i];
    }
}

int32_t oracle_node_threads(const oracle_node *nd)
{
    return nd->T;
}

/* Symmetric CRS (the storage Sect. 1.3.1 mentions and sets aside): a symmetric
 * matrix given by its upper triangle with the diagonal, each row i listing the
 * entries a_ij with j >= i.  The product walks the stored entries once, row by
 * row in increasing k: entry (i, j, a) adds a*x[j] to row i's sum and, when
 * j != i, a*x[i] to row j's sum (the mirrored entry a_ji = a).  Then
 * y_i = alpha*t_i (+ beta*y_i).  absrow (nullable) receives
 * |alpha|*sum_j |a_ij x_j| over the full row plus |beta*y_i|. */
void oracle_spmv_sym(int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                     const double *val, const double *x, double alpha, double beta,
                     double *y, double *absrow)
{
    double *t = (double *)calloc((size_t)n + 1, sizeof(double));
    double *mag = (double *)calloc((size_t)n + 1, sizeof(double));
    for (int32_t i = 0; i < n; ++i)
        for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            int32_t j = col_idx[k];
            double p = val[k] * x[j];
            t[i] = t[i] + p;
            mag[i] = mag[i] + fabs(p);
            if (j != i) {
                double q = val[k] * x[i];
                t[j] = t[j] + q;
                mag[j] = mag[j] + fabs(q);
            }
        }
    for (int32_t i = 0; i < n; ++i) {
        double yin = (beta == 0.0) ? 0.0 : y[i];
        if (beta == 0.0)
            y[i] = alpha * t[i];
        else
            y[i] = alpha * t[i] + beta * yin;
        if (absrow)
            absrow[i] = fabs(alpha) * mag[i] + fabs(beta * yin);
    }
    free(t);
    free(mag);
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Block vectors: Y[i][r] = alpha*sum_k val[k]*X[col_idx[k]][r] + beta*Y[i][r], with
 * X and Y stored interleaved (row-major, leading dimension nrhs).  Computed one
 * right-hand side at a time with the plain kernel's loop. */
void oracle_spmm(int32_t n_rows, const int32_t *row_ptr, const int32_t *col_idx,
                 const double *val, int32_t nrhs, const double *X, double alpha,
                 double beta, double *Y, double *absY)
{
    for (int32_t r = 0; r < nrhs; ++r) {
        for (int32_t i = 0; i < n_rows; ++i) {
            double acc = 0.0, mag = 0.0;
            for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
                double p = val[k] * X[(int64_t)col_idx[k] * nrhs + r];
                acc = acc + p;
                mag = mag + fabs(p);
            }
            int64_t o = (int64_t)i * nrhs + r;
            double yin = (beta == 0.0) ? 0.0 : Y[o];
            if (beta == 0.0)
                Y[o] = alpha * acc;
            else
                Y[o] = alpha * acc + beta * yin;
            if (absY)
                absY[o] = fabs(alpha) * mag + (beta == 0.0 ? 0.0 : fabs(beta * yin));
        }
    }
}

/* Transposed CRS: rows of A^T are the columns of A.  Entries of each A^T row are
 * listed in increasing original position k (hence increasing row of A), which makes
 * the result unique.  perm[p] = k maps A^T position p to the A position it copies.
 * Counting sort: count entries per column, exclusive prefix sum, stable fill. */
void oracle_transpose(int32_t n_rows, int32_t n_cols, const int32_t *row_ptr,
                      const int32_t *col_idx, int32_t *rowT_ptr, int32_t *colT_idx,
                      int32_t *perm)
{
    int32_t nnz = row_ptr[n_rows];
    int32_t *next = (int32_t *)calloc((size_t)n_cols + 1, sizeof(int32_t));
    for (int32_t j = 0; j <= n_cols; ++j)
        rowT_ptr[j] = 0;
    for (int32_t k = 0; k < nnz; ++k)
        rowT_ptr[col_idx[k] + 1] += 1;
    for (int32_t j = 0; j < n_cols; ++j)
        rowT_ptr[j + 1] += rowT_ptr[j];
    for (int32_t j = 0; j < n_cols; ++j)
        next[j] = rowT_ptr[j];
    for (int32_t i = 0; i < n_rows; ++i) {
        for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            int32_t p = next[col_idx[k]]++;
            colT_idx[p] = i;
            perm[p] = k;
        }
    }
    free(next);
}

/* Reverse pass of f = g^T (alpha*A(val)*x):
 *   grad_x[j]   = alpha * sum_i a_ij g_i      (= alpha * A^T g, scattered row by row)
 *   grad_val[k] = alpha * g[row(k)] * x[col(k)]
 * Either output may be NULL.  absgx (nullable) receives sum_i |a_ij g_i| per column. */
void oracle_backward(int32_t n_rows, int32_t n_cols, const int32_t *row_ptr,
                     const int32_t *col_idx, const double *val, double alpha,
                     const double *g, const double *x, double *grad_x,
                     double *grad_val, double *absgx)
{
    if (grad_x) {
        double *acc = (double *)calloc((size_t)n_cols + 1, sizeof(double));
        double *mag = (double *)calloc((size_t)n_cols + 1, sizeof(double));
        for (int32_t i = 0; i < n_rows; ++i)
            for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
                double p = val[k] * g[i];
                acc[col_idx[k]] = acc[col_idx[k]] + p;
                mag[col_idx[k]] = mag[col_idx[k]] + fabs(p);
            }
        for (int32_t j = 0; j < n_cols; ++j) {
            grad_x[j] = alpha * acc[j];
            if (absgx)
                absgx[j] = fabs(alpha) * mag[j];
        }
        free(acc);
        free(mag);
    }
    if (grad_val) {
        for (int32_t i = 0; i < n_rows; ++i)
            for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k)
                grad_val[k] = alpha * (g[i] * x[col_idx[k]]);
    }
}

/* Row-block distribution of Sect. 3.2: nonzeros balanced across nblocks contiguous
 * row blocks.  Block b starts at the first row whose starting offset is at least
 * ceil(b*nnz/nblocks); block 0 starts at row 0 and the last block ends at n_rows. */
void oracle_split_blocks(int32_t n_rows, const int32_t *row_ptr, int32_t nblocks,
                         int32_t *block_start)
{
    int64_t nnz = row_ptr[n_rows];
    block_start[0] = 0;
    for (int32_t b = 1; b < nblocks; ++b) {
        int64_t target = (b * nnz + nblocks - 1) / nblocks;
        int32_t r = 0;
        while (r < n_rows && row_ptr[r] < target)
            ++r;
        block_start[b] = r;
    }
    block_start[nblocks] = n_rows;
}

/* Halo bookkeeping of Sect. 3.2 (done once per sparsity pattern): for each block b
 * with rows [s_b, s_{b+1}), the columns referenced by its rows that lie outside
 * [s_b, s_{b+1}) (the right-hand side is distributed like the rows), sorted and
 * without repeats.  halo_count[b] receives the number of such columns; if halo_map
 * is non-NULL the maps of all blocks are written one after the other.  Also counts
 * the local and nonlocal entries of each block. */
int64_t oracle_split_halo(int32_t n_rows, int32_t n_cols, const int32_t *row_ptr,
                          const int32_t *col_idx, int32_t nblocks,
                          const int32_t *block_start, int32_t *halo_count,
                          int32_t *halo_map, int64_t *nnz_local, int64_t *nnz_nonlocal)
{
    unsigned char *used = (unsigned char *)malloc((size_t)n_cols + 1);
    int64_t total = 0;
    (void)n_rows;
    for (int32_t b = 0; b < nblocks; ++b) {
        int32_t lo = block_start[b], hi = block_start[b + 1];
        memset(used, 0, (size_t)n_cols + 1);
        int64_t nl = 0, nn = 0;
        for (int32_t i = lo; i < hi; ++i)
            for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
                int32_t j = col_idx[k];
                if (j >= lo && j < hi) {
                    ++nl;
                } else {
                    ++nn;
                    used[j] = 1;
                }
            }
        int32_t cnt = 0;
        for (int32_t j = 0; j < n_cols; ++j)
            if (used[j]) {
                if (halo_map)
                    halo_map[total + cnt] = j;
                ++cnt;
            }
        halo_count[b] = cnt;
        if (nnz_local)
            nnz_local[b] = nl;
        if (nnz_nonlocal)
            nnz_nonlocal[b] = nn;
        total += cnt;
    }
    free(used);
    return total;
}

/* Textbook conjugate gradients (Hestenes-Stiefel) in FP64 for SPD A, x0 = 0,
 * stopped when ||r||_2 <= tol*||b||_2 or after maxit iterations.  Returns the
 * iteration count; x receives the iterate. */
int32_t oracle_cg(int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                  const double *val, const double *b, double tol, int32_t maxit,
                  double *x)
{
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    double *p = (double *)malloc(sizeof(double) * (size_t)n);
    double *q = (double *)malloc(sizeof(double) * (size_t)n);
    double bb = 0.0, rr = 0.0;
    for (int32_t i = 0; i < n; ++i) {
        x[i] = 0.0;
        r[i] = b[i];
        p[i] = b[i];
        bb += b[i] * b[i];
    }
    rr = bb;
    int32_t it = 0;
    while (it < maxit && sqrt(rr) > tol * sqrt(bb)) {
        oracle_spmv(n, row_ptr, col_idx, val, p, 1.0, 0.0, q, NULL);
        double pq = 0.0;
        for (int32_t i = 0; i < n; ++i)
            pq += p[i] * q[i];
        double a = rr / pq;
        double rr_new = 0.0;
        for (int32_t i = 0; i < n; ++i) {
            x[i] = x[i] + a * p[i];
            r[i] = r[i] - a * q[i];
            rr_new += r[i] * r[i];
        }
        double beta = rr_new / rr;
        for (int32_t i = 0; i < n; ++i)
            p[i] = r[i] + beta * p[i];
        rr = rr_new;
        ++it;
    }
    free(r);
    free(p);
    free(q);
    return it;
}

/* Row-length histogram: counts[L] = number of rows with exactly L entries, for
 * L < nbins; longer rows are counted in the last bin. */
void oracle_row_histogram(int32_t n_rows, const int32_t *row_ptr, int32_t nbins,
                          int64_t *counts)
{
    for (int32_t b = 0; b < nbins; ++b)
        counts[b] = 0;
    for (int32_t i = 0; i < n_rows; ++i) {
        int32_t len = row_ptr[i + 1] - row_ptr[i];
        counts[len < nbins ? len : nbins - 1] += 1;
    }
}
