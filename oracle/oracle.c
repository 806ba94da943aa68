/*
 * CPU FP64 oracle for the tile Cholesky path -- TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may load
 * this library.  It shares no code with the CUDA path.
 *
 * Everything here is the plain textbook definition, in IEEE double precision:
 *   - Cholesky factor A = L L^T (Section III-A of the paper: the factor every
 *     tile algorithm reaches), computed column by column:
 *         L_jj = sqrt(a_jj - sum_{k<j} L_jk^2)
 *         L_ij = (a_ij - sum_{k<j} L_ik L_jk) / L_jj          (i > j)
 *     A non-positive pivot stops the factorization and returns the 1-based
 *     column (LAPACK's convention; the paper does not define failure).
 *   - Forward substitution L z = b and back substitution L^T x = z (used for
 *     y^T Sigma^{-1} y in Eq. 1 and for the solve).
 * Storage: dense row-major n x n, leading dimension ld >= n.
 * The only parallelism is an OpenMP loop over independent rows i inside one
 * column j, which does not change any operation or its order per entry.
 */
#include <math.h>
#include <stdint.h>

static double dot_prefix(const double *x, const double *y, int64_t len) {
    double s = 0.0;
    for (int64_t k = 0; k < len; ++k) s += x[k] * y[k];
    return s;
}

/* In-place lower Cholesky of the row-major matrix A (only the lower triangle is
 * read and written).  Returns 0 on success, j+1 if the pivot of column j is not
 * positive. */
int oracle_potrf(int64_t n, double *A, int64_t ld) {
    for (int64_t j = 0; j < n; ++j) {
        double *rj = A + j * ld;
        double d = rj[j] - dot_prefix(rj, rj, j);
        if (!(d > 0.0)) return (int)(j + 1);
        double ljj = sqrt(d);
        rj[j] = ljj;
#pragma omp parallel for schedule(static)
        for (int64_t i = j + 1; i < n; ++i) {
            double *ri = A + i * ld;
            ri[j] = (ri[j] - dot_prefix(ri, rj, j)) / ljj;
        }
    }
    return 0;
}

/* Solve L Z = B in place; B is row-major n x nrhs with leading dimension ldb. */
void oracle_trsm_lower(int64_t n, const double *L, int64_t ld, int64_t nrhs, double *B, int64_t ldb) {
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < nrhs; ++c) {
        for (int64_t i = 0; i < n; ++i) {
            const double *ri = L + i * ld;
            double s = B[i * ldb + c];
            for (int64_t k = 0; k < i; ++k) s -= ri[k] * B[k * ldb + c];
            B[i * ldb + c] = s / ri[i];
        }
    }
}

/* Solve L^T X = B in place (back substitution with the transposed factor). */
void oracle_trsm_lower_trans(int64_t n, const double *L, int64_t ld, int64_t nrhs, double *B, int64_t ldb) {
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < nrhs; ++c) {
        for (int64_t i = n - 1; i >= 0; --i) {
            double s = B[i * ldb + c];
            for (int64_t k = i + 1; k < n; ++k) s -= L[k * ld + i] * B[k * ldb + c];
            B[i * ldb + c] = s / L[i * ld + i];
        }
    }
}

/* Number of OpenMP threads the loops above use (1 without OpenMP). */
int oracle_threads(void) {
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
