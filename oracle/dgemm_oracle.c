/*
 * CPU oracle for the FP64 GEMM  C <- alpha*A*B + beta*C  (Section 4.2, "Performance":
 * the DGEMM definition with dense square matrices filled with random values).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests, the smoke check and the CPU-baseline leg of
 * the benchmark may load this file's library.  It shares no code, header or
 * constant with the CUDA path.
 *
 * Layout: row-major.  A is m x k with leading dimension lda >= k, B is k x n with
 * ldb >= n, C is m x n with ldc >= n (the pitched rows of Section 3.4.4, "Memory").
 *
 * Readings of the definition where the paper is silent (BLAS convention):
 *   - beta == 0: C is not read, so NaN/Inf already in C does not propagate.
 *   - alpha == 0 or k == 0: C <- beta*C, and A and B are not read.
 *   - m == 0 or n == 0: nothing happens.
 *
 * Compiled with -O2 -fno-fast-math -ffp-contract=off: every product and every sum
 * is one IEEE double rounding, the sum over l runs from 0 to k-1, and no fused
 * multiply-add is formed.
 */
#include <stdint.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* The definition, loop order i, j, l.  For each (i, j):
 *   s = ((A[i,0]*B[0,j] + A[i,1]*B[1,j]) + ...) ;  C[i,j] = alpha*s + beta*C[i,j]. */
void oracle_dgemm(int64_t m, int64_t n, int64_t k, double alpha,
                  const double* A, int64_t lda, const double* B, int64_t ldb,
                  double beta, double* C, int64_t ldc) {
    for (int64_t i = 0; i < m; ++i) {
        for (int64_t j = 0; j < n; ++j) {
            double* c = &C[i * ldc + j];
            if (alpha == 0.0 || k == 0) {
                *c = (beta == 0.0) ? 0.0 : beta * (*c);
                continue;
            }
            double s = 0.0;
            for (int64_t l = 0; l < k; ++l) s += A[i * lda + l] * B[l * ldb + j];
            *c = (beta == 0.0) ? alpha * s : alpha * s + beta * (*c);
        }
    }
}

/* The same definition for a subset of rows: output row r of Cr (leading dimension
 * ldcr) is row rows[r] of the full result; Cr holds the matching rows of C on entry
 * (read only when beta != 0). */
void oracle_dgemm_rows(int64_t nrows, const int64_t* rows, int64_t n, int64_t k,
                       double alpha, const double* A, int64_t lda, const double* B,
                       int64_t ldb, double beta, double* Cr, int64_t ldcr) {
    for (int64_t r = 0; r < nrows; ++r) {
        const double* a = &A[rows[r] * lda];
        oracle_dgemm(1, n, k, alpha, a, lda, B, ldb, beta, &Cr[r * ldcr], ldcr);
    }
}

/* The same definition, rows spread over OpenMP threads and loop order i, l, j.
 * Every C[i,j] still accumulates l = 0, 1, ..., k-1 in order with separate
 * rounded products and sums, so the result is bit-identical to oracle_dgemm.
 * `work` must hold n doubles per thread (nthreads * n). Returns threads used. */
int oracle_dgemm_omp(int64_t m, int64_t n, int64_t k, double alpha,
                     const double* A, int64_t lda, const double* B, int64_t ldb,
                     double beta, double* C, int64_t ldc, int nthreads, double* work) {
    int used = 1;
#ifdef _OPENMP
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel num_threads(nthreads)
    {
#pragma omp single
        used = omp_get_num_threads();
        double* s = &work[(int64_t)omp_get_thread_num() * n];
#pragma omp for schedule(static)
        for (int64_t i = 0; i < m; ++i) {
#else
    {
        double* s = work;
        (void)nthreads;
        for (int64_t i = 0; i < m; ++i) {
#endif
            double* c = &C[i * ldc];
            if (alpha == 0.0 || k == 0) {
                for (int64_t j = 0; j < n; ++j) c[j] = (beta == 0.0) ? 0.0 : beta * c[j];
                continue;
            }
            for (int64_t j = 0; j < n; ++j) s[j] = 0.0;
            for (int64_t l = 0; l < k; ++l) {
                const double a = A[i * lda + l];
                const double* b = &B[l * ldb];
                for (int64_t j = 0; j < n; ++j) s[j] += a * b[j];
            }
            for (int64_t j = 0; j < n; ++j)
                c[j] = (beta == 0.0) ? alpha * s[j] : alpha * s[j] + beta * c[j];
        }
    }
    return used;
}

/* ---- High-precision reference for measuring error (not for timing) ----------------
 * Error-free transformations: TwoSum (Knuth, TAOCP vol. 2, 4.2.2) and the
 * product split by a correctly rounded fma (C99 fma): a*b = p + e exactly.
 * The products are accumulated in double-double arithmetic; the result
 * hi + lo approximates sum_l A[i,l]*B[l,j] with relative error ~ k * 2^-104
 * of sum_l |A[i,l]*B[l,j]|, far below any FP64 rounding bound.
 * Rows `rows[r]` (all rows when rows == NULL and nrows == m). */
static inline void two_sum(double a, double b, double* s, double* e) {
    double x = a + b;
    double z = x - a;
    *e = (a - (x - z)) + (b - z);
    *s = x;
}

void oracle_dgemm_dd_rows(int64_t nrows, const int64_t* rows, int64_t n, int64_t k,
                          const double* A, int64_t lda, const double* B, int64_t ldb,
                          double* hi, double* lo, int64_t ldo) {
    /* Loop order r, l, j with the running (hi, lo) pair of every output kept in
     * the output rows: each entry still takes l = 0, 1, ..., k-1 in order through
     * the same steps as an i, j, l loop, so the bits do not depend on the order;
     * rows and blocks of 256 columns go to OpenMP threads. */
    const int64_t JB = 256;
    const int64_t nb = (n + JB - 1) / JB;
#ifdef _OPENMP
#pragma omp parallel for collapse(2) schedule(dynamic)
#endif
    for (int64_t r = 0; r < nrows; ++r) {
        for (int64_t b = 0; b < nb; ++b) {
            const int64_t i = rows ? rows[r] : r;
            const int64_t j0 = b * JB, j1 = (j0 + JB < n) ? j0 + JB : n;
            double* h = &hi[r * ldo];
            double* o = &lo[r * ldo];
            for (int64_t j = j0; j < j1; ++j) h[j] = o[j] = 0.0;
            for (int64_t l = 0; l < k; ++l) {
                const double a = A[i * lda + l];
                const double* bl = &B[l * ldb];
                for (int64_t j = j0; j < j1; ++j) {
                    const double p = a * bl[j];
                    const double pe = fma(a, bl[j], -p);
                    double t, te;
                    two_sum(h[j], p, &t, &te);
                    te += pe + o[j];
                    two_sum(t, te, &h[j], &o[j]);
                }
            }
        }
    }
}

/* ---- DAXPY  Y <- alpha X + Y  (Section 4.1, "Conceptual Comparison") ----------------
 * Reading: each element is evaluated with one rounding, y_i <- fma(alpha, x_i, y_i)
 * (C99 fma, correctly rounded).  n == 0 does nothing; alpha == 0 leaves Y unchanged
 * and does not read X. */
void oracle_daxpy(int64_t n, double alpha, const double* x, double* y) {
    if (alpha == 0.0) return;
    for (int64_t i = 0; i < n; ++i) y[i] = fma(alpha, x[i], y[i]);
}
