/*
 * CPU FP64 oracle for the triangular solve (TRSM), the LU factorisation with
 * partial pivoting (GETRF) and the Cholesky factorisation (POTRF) built on the
 * out-of-core GEMM.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark use it.  It shares no code, header or constant with the CUDA
 * library.
 *
 * Section VII of the libhclooc paper (arXiv:1808.05056) names the rest of
 * level-3 BLAS and the out-of-core factorisations (LU, QR, Cholesky) that use
 * the out-of-core DGEMM as their building block as the next step.  The paper
 * defines neither operation; the oracle is the textbook definition of each,
 * written out as plain loops:
 *
 *   TRSM  side 'L': solve op(A) X = alpha B,  side 'R': solve X op(A) = alpha B,
 *         A triangular (uplo 'L' or 'U'; only that triangle is read), op(A) =
 *         A or A^T, diag 'U' takes the diagonal as ones (not read); X
 *         overwrites B.  Each right-hand side is one substitution: unknown t
 *         is (alpha b_t - sum over the unknowns already found of coefficient x
 *         unknown) / diagonal coefficient, the sum in ascending index order.
 *
 *   GETRF A = P L U with partial pivoting (row interchanges), L unit lower
 *         triangular, U upper triangular, stored over A (L below the diagonal,
 *         U on and above it).  Right-looking, column by column: for j = 0 ..
 *         n-1 the pivot is the first row p >= j with the largest |a[p][j]|;
 *         rows j and p are exchanged across all n columns and ipiv[j] = p;
 *         then a[i][j] /= a[j][j] and a[i][k] -= a[i][j] a[j][k] for i, k > j
 *         (k ascending per row).  A zero pivot skips the division and the
 *         update of that column and sets info = j + 1 (first one only).
 *
 *   POTRF uplo 'L': A = L L^T with L lower triangular, positive diagonal,
 *         computed column by column (Cholesky-Crout): for j = 0 .. n-1,
 *           L[j][j] = sqrt(A[j][j] - sum_{k<j} L[j][k]^2),
 *           L[i][j] = (A[i][j] - sum_{k<j} L[i][k] L[j][k]) / L[j][j], i > j;
 *         uplo 'U': A = U^T U, U = L^T stored in the upper triangle.  Only the
 *         uplo triangle is read and overwritten.  Returns 0, or j + 1 when the
 *         j-th pivot is not positive (then the columns before j are final).
 *
 * Storage is row-major (element (r, c) of X is X[r * ldx + c]).  No blocking,
 * no reordering, no fused multiply-add contraction (-ffp-contract=off).  The
 * independent right-hand sides (TRSM) and the rows below the pivot (GETRF,
 * POTRF) are split over host threads, which changes no arithmetic.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>

static int is_t(char t) { return t == 'T' || t == 't'; }
static int is_l(char t) { return t == 'L' || t == 'l'; }
static int is_u(char t) { return t == 'U' || t == 'u'; }

/* ------------------------------------------------------------------ TRSM */

typedef struct {
    char side, uplo, ta, diag;
    int64_t M, N;
    double alpha;
    const double* A;
    int64_t lda;
    double* B;
    int64_t ldb;
    int64_t v0, v1; /* right-hand sides [v0, v1): columns (side L) or rows (side R) of B */
} trsm_job;

/* op(A)[i][k], reading only the stored triangle (zero elsewhere, one on a unit diagonal) */
static double opa(const trsm_job* j, int64_t i, int64_t k)
{
    const int64_t r = is_t(j->ta) ? k : i, c = is_t(j->ta) ? i : k;  /* stored position */
    if (r == c) return is_u(j->diag) ? 1.0 : j->A[r * j->lda + c];
    if (is_l(j->uplo) ? c > r : c < r) return 0.0;
    return j->A[r * j->lda + c];
}

static void* trsm_run(void* p)
{
    const trsm_job* j = (const trsm_job*)p;
    const int64_t n = is_l(j->side) ? j->M : j->N;  /* order of the triangular system */
    /* op(A) lower triangular: uplo 'L' untransposed or uplo 'U' transposed */
    const int op_lower = is_l(j->uplo) != is_t(j->ta);
    for (int64_t v = j->v0; v < j->v1; ++v) {
        /* element t of this right-hand side */
        double* base = is_l(j->side) ? j->B + v : j->B + v * j->ldb;
        const int64_t step = is_l(j->side) ? j->ldb : 1;
        /* side L, op(A) x = alpha b: row t of op(A) couples x_t with x_k, k != t.
         * side R, x op(A) = alpha b: column t of op(A) couples x_t with x_k.
         * Forward order when the coupled unknowns come first. */
        const int forward = is_l(j->side) ? op_lower : !op_lower;
        for (int64_t q = 0; q < n; ++q) {
            const int64_t t = forward ? q : n - 1 - q;
            double s = 0.0;
            if (forward) {
                for (int64_t k = 0; k < t; ++k)
                    s += (is_l(j->side) ? opa(j, t, k) : opa(j, k, t)) * base[k * step];
            } else {
                for (int64_t k = t + 1; k < n; ++k)
                    s += (is_l(j->side) ? opa(j, t, k) : opa(j, k, t)) * base[k * step];
            }
            const double rhs = j->alpha * base[t * step] - s;
            base[t * step] = is_u(j->diag) ? rhs : rhs / opa(j, t, t);
        }
    }
    return NULL;
}

int oracle_dtrsm(char side, char uplo, char ta, char diag, int64_t M, int64_t N, double alpha,
                 const double* A, int64_t lda, double* B, int64_t ldb, int nthreads)
{
    if (M <= 0 || N <= 0) return 0;
    const int64_t nv = is_l(side) ? N : M;  /* independent right-hand sides */
    if (nthreads < 1) nthreads = 1;
    if (nthreads > nv) nthreads = (int)nv;
    trsm_job* jobs = (trsm_job*)calloc((size_t)nthreads, sizeof(trsm_job));
    pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !th) {
        free(jobs);
        free(th);
        return -1;
    }
    for (int t = 0; t < nthreads; ++t) {
        trsm_job j = {side, uplo, ta, diag, M, N, alpha, A, lda, B, ldb, nv * t / nthreads, nv * (t + 1) / nthreads};
        jobs[t] = j;
    }
    int started = 0;
    for (int t = 1; t < nthreads; ++t)
        if (pthread_create(&th[t], NULL, trsm_run, &jobs[t]) == 0) started = t;
        else break;
    trsm_run(&jobs[0]);
    for (int t = 1; t <= started; ++t) pthread_join(th[t], NULL);
    for (int t = started + 1; t < nthreads; ++t) trsm_run(&jobs[t]);
    free(jobs);
    free(th);
    return nthreads;
}

/* ----------------------------------------------------------------- POTRF */

typedef struct {
    int lower;
    int64_t n, j;
    double* A;
    int64_t lda;
    int64_t i0, i1; /* rows (lower) / columns (upper) i > j of column j handled by this thread */
} potrf_job;

/* element (r, c) of the factor's storage for the lower form, (c, r) for the upper form */
static double* fac(const potrf_job* p, int64_t r, int64_t c)
{
    return p->lower ? &p->A[r * p->lda + c] : &p->A[c * p->lda + r];
}

static void* potrf_col(void* q)
{
    const potrf_job* p = (const potrf_job*)q;
    const int64_t j = p->j;
    const double d = *fac(p, j, j);
    for (int64_t i = p->i0; i < p->i1; ++i) {
        double s = 0.0;
        for (int64_t k = 0; k < j; ++k) s += *fac(p, i, k) * *fac(p, j, k);
        *fac(p, i, j) = (*fac(p, i, j) - s) / d;
    }
    return NULL;
}

int64_t oracle_dpotrf(char uplo, int64_t n, double* A, int64_t lda, int nthreads)
{
    if (n <= 0) return 0;
    if (nthreads < 1) nthreads = 1;
    pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
    potrf_job* jobs = (potrf_job*)calloc((size_t)nthreads, sizeof(potrf_job));
    if (!th || !jobs) {
        free(th);
        free(jobs);
        return -1;
    }
    const int lower = is_l(uplo);
    int64_t info = 0;
    for (int64_t j = 0; j < n && !info; ++j) {
        potrf_job base = {lower, n, j, A, lda, 0, 0};
        double s = 0.0;
        for (int64_t k = 0; k < j; ++k) s += *fac(&base, j, k) * *fac(&base, j, k);
        const double piv = *fac(&base, j, j) - s;
        if (!(piv > 0.0)) {
            info = j + 1;
            break;
        }
        *fac(&base, j, j) = sqrt(piv);
        const int64_t rows = n - j - 1;
        int nt = nthreads;
        if ((int64_t)nt > rows / 64) nt = (int)(rows / 64);  /* threads only for long columns */
        if (nt < 1) nt = 1;
        for (int t = 0; t < nt; ++t) {
            jobs[t] = base;
            jobs[t].i0 = j + 1 + rows * t / nt;
            jobs[t].i1 = j + 1 + rows * (t + 1) / nt;
        }
        int started = 0;
        for (int t = 1; t < nt; ++t)
            if (pthread_create(&th[t], NULL, potrf_col, &jobs[t]) == 0) started = t;
            else break;
        potrf_col(&jobs[0]);
        for (int t = 1; t <= started; ++t) pthread_join(th[t], NULL);
        for (int t = started + 1; t < nt; ++t) potrf_col(&jobs[t]);
    }
    free(th);
    free(jobs);
    return info;
}

/* ----------------------------------------------------------------- GETRF */

typedef struct {
    int64_t n, j, lda;
    double* A;
    int64_t i0, i1; /* rows below the pivot handled by this thread */
} getrf_job;

static void* getrf_rows(void* q)
{
    const getrf_job* p = (const getrf_job*)q;
    const int64_t j = p->j, n = p->n, lda = p->lda;
    double* A = p->A;
    const double d = A[j * lda + j];
    for (int64_t i = p->i0; i < p->i1; ++i) {
        const double l = A[i * lda + j] / d;
        A[i * lda + j] = l;
        for (int64_t k = j + 1; k < n; ++k) A[i * lda + k] -= l * A[j * lda + k];
    }
    return NULL;
}

int64_t oracle_dgetrf(int64_t n, double* A, int64_t lda, int64_t* ipiv, int nthreads)
{
    if (n <= 0) return 0;
    if (nthreads < 1) nthreads = 1;
    pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
    getrf_job* jobs = (getrf_job*)calloc((size_t)nthreads, sizeof(getrf_job));
    if (!th || !jobs) {
        free(th);
        free(jobs);
        return -1;
    }
    int64_t info = 0;
    for (int64_t j = 0; j < n; ++j) {
        int64_t p = j;
        double best = fabs(A[j * lda + j]);
        for (int64_t i = j + 1; i < n; ++i) {
            const double v = fabs(A[i * lda + j]);
            if (v > best) {
                best = v;
                p = i;
            }
        }
        ipiv[j] = p;
        if (p != j)
            for (int64_t k = 0; k < n; ++k) {
                const double t = A[j * lda + k];
                A[j * lda + k] = A[p * lda + k];
                A[p * lda + k] = t;
            }
        if (best == 0.0) {
            if (!info) info = j + 1;
            continue;
        }
        const int64_t rows = n - j - 1;
        int nt = nthreads;
        if ((int64_t)nt > rows / 64) nt = (int)(rows / 64);
        if (nt < 1) nt = 1;
        for (int t = 0; t < nt; ++t) {
            getrf_job jb = {n, j, lda, A, j + 1 + rows * t / nt, j + 1 + rows * (t + 1) / nt};
            jobs[t] = jb;
        }
        int started = 0;
        for (int t = 1; t < nt; ++t)
            if (pthread_create(&th[t], NULL, getrf_rows, &jobs[t]) == 0) started = t;
            else break;
        getrf_rows(&jobs[0]);
        for (int t = 1; t <= started; ++t) pthread_join(th[t], NULL);
        for (int t = started + 1; t < nt; ++t) getrf_rows(&jobs[t]);
    }
    free(th);
    free(jobs);
    return info;
}
