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

/* The node-level parallelisation of Sect. 2: the outer (row) loop of Listing 1
 * split statically across OpenMP threads.  Same arithmetic per row as oracle_spmv.
 * Used only as the timed CPU baseline. */
void oracle_spmv_omp(int32_t n_rows, const int32_t *row_ptr, const int32_t *col_idx,
                     const double *val, const double *x, double alpha, double beta,
                     double *y)
{
#pragma omp parallel for schedule(static)
    for (int32_t i = 0; i < n_rows; ++i) {
        double acc = 0.0;
        for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k)
            acc = acc + val[k] * x[col_idx[k]];
        if (beta == 0.0)
            y[i] = alpha * acc;
        else
            y[i] = alpha * acc + beta * y[i];
    }
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
