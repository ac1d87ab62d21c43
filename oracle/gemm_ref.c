/*
 * FP64 reference GEMM — TEST INFRASTRUCTURE ONLY.
 *
 * This file is part of the oracle: a plain, slow, obviously correct CPU
 * statement of what every GEMM implementation variant must compute.  It is
 * used only by the tests, by the smoke check and by the benchmark's CPU
 * baseline leg.  The product path never calls it, and it shares no code or
 * header with the CUDA library.
 *
 * What it computes (the matrix-multiply component "mmul" that COMPAR exposes
 * through several interchangeable implementation variants, Sec. 2.1 and the
 * matrix-multiply row of Table 2; every variant is an implementation of this
 * one function):
 *
 *     C[i][j] = alpha * sum_{p=0}^{K-1} A[i][p] * B[p][j]  +  beta * C0[i][j]
 *
 * with A (M x K), B (K x N), C (M x N) row-major with leading dimensions
 * lda, ldb, ldc.  All arithmetic is IEEE double; the build passes
 * -ffp-contract=off so no fused multiply-add changes the rounding.
 * Following the BLAS convention, beta == 0 means C0 is not read.
 *
 * The loop order is i, p, j (row of C accumulated in a private buffer), which
 * changes nothing but the summation order inside fp64; OpenMP splits the i
 * loop across host cores.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* One output row: acc[j] = sum_p A[i][p] * B[p][j]. */
static void row_product(int64_t n, int64_t k, const double *a_row,
                        const double *B, int64_t ldb, double *acc)
{
    for (int64_t j = 0; j < n; ++j) acc[j] = 0.0;
    for (int64_t p = 0; p < k; ++p) {
        const double a = a_row[p];
        const double *b_row = B + p * ldb;
        for (int64_t j = 0; j < n; ++j) acc[j] += a * b_row[j];
    }
}

/* Full GEMM.  Returns 0, or -1 on bad arguments / allocation failure. */
int oracle_gemm_f64(int64_t m, int64_t n, int64_t k, double alpha,
                    const double *A, int64_t lda, const double *B, int64_t ldb,
                    double beta, double *C, int64_t ldc)
{
    if (m < 0 || n < 0 || k < 0) return -1;
    if (m == 0 || n == 0) return 0;
    if (lda < k || ldb < n || ldc < n) return -1;
    int failed = 0;
#pragma omp parallel
    {
        double *acc = (double *)malloc((size_t)n * sizeof(double));
        if (!acc) {
#pragma omp atomic write
            failed = 1;
        }
#pragma omp for schedule(dynamic, 1)
        for (int64_t i = 0; i < m; ++i) {
            if (!acc) continue;
            row_product(n, k, A + i * lda, B, ldb, acc);
            double *c_row = C + i * ldc;
            for (int64_t j = 0; j < n; ++j)
                c_row[j] = (beta == 0.0) ? alpha * acc[j]
                                         : alpha * acc[j] + beta * c_row[j];
        }
        free(acc);
    }
    return failed ? -1 : 0;
}

/*
 * The same definition evaluated for a chosen subset of rows only (used to
 * check products too large for the full triple loop).  rows[r] names the row
 * of C; the result row r is written to Out + r * n (packed).  C0 (may be NULL
 * when beta == 0) is the full M x N input C with leading dimension ldc.
 */
int oracle_gemm_rows_f64(int64_t m, int64_t n, int64_t k, double alpha,
                         const double *A, int64_t lda, const double *B,
                         int64_t ldb, double beta, const double *C0,
                         int64_t ldc, const int64_t *rows, int64_t nrows,
                         double *Out)
{
    if (m < 0 || n < 0 || k < 0 || nrows < 0) return -1;
    if (lda < k || ldb < n) return -1;
    if (beta != 0.0 && (C0 == NULL || ldc < n)) return -1;
    for (int64_t r = 0; r < nrows; ++r)
        if (rows[r] < 0 || rows[r] >= m) return -1;
    int failed = 0;
#pragma omp parallel
    {
        double *acc = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
        if (!acc) {
#pragma omp atomic write
            failed = 1;
        }
#pragma omp for schedule(dynamic, 1)
        for (int64_t r = 0; r < nrows; ++r) {
            if (!acc) continue;
            const int64_t i = rows[r];
            row_product(n, k, A + i * lda, B, ldb, acc);
            double *o = Out + r * n;
            for (int64_t j = 0; j < n; ++j)
                o[j] = (beta == 0.0) ? alpha * acc[j]
                                     : alpha * acc[j] + beta * C0[i * ldc + j];
        }
        free(acc);
    }
    return failed ? -1 : 0;
}

/* Number of threads the OpenMP loops above use (for reporting). */
int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
