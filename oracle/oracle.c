/*
 * CPU FP64 oracle for C = alpha * op(A) * op(B) + beta * C.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark use it.  It shares no code, header or constant with the CUDA
 * library.
 *
 * What it computes is the problem statement of Section IV of the libhclooc
 * paper (arXiv:1808.05056): C = alpha x A B + beta x C with A of M x K,
 * B of K x N and C of M x N, alpha and beta scalars.  The per-block form
 * c_ij = alpha a_i b_j + beta c_ij of the DGEMM pipeline stage (Section IV,
 * five-stage pipeline list) is the same sum restricted to a block, so the
 * plain definition over the whole matrix is the oracle for every partition.
 *
 * Conventions (the paper states none; these are the library's):
 *   - row-major storage; element (r, c) of a stored matrix X with leading
 *     dimension ldx is X[r * ldx + c];
 *   - op(X) = X for trans 'N'/'n', X^T for 'T'/'t' (then X is stored K x M
 *     for A, N x K for B);
 *   - the k-sum runs k = 0, 1, ..., K-1 in FP64, then
 *     C = alpha * acc + beta * C; C is not read when beta == 0 (BLAS rule,
 *     so NaN in C is ignored), and K == 0 gives C = beta * C.
 *
 * The loops are the definition written out; there is no blocking, no
 * reordering and no fused multiply-add contraction (built with
 * -ffp-contract=off).  Rows are split over host threads, which changes no
 * arithmetic: every C element is computed by one thread in the order above.
 */
#include <stdint.h>
#include <stdlib.h>
#include <pthread.h>

static int is_t(char t) { return t == 'T' || t == 't'; }

/* op(A)[i,k] */
static double elem_a(const double* A, int64_t lda, char ta, int64_t i, int64_t k)
{
    return is_t(ta) ? A[k * lda + i] : A[i * lda + k];
}
/* op(B)[k,j] */
static double elem_b(const double* B, int64_t ldb, char tb, int64_t k, int64_t j)
{
    return is_t(tb) ? B[j * ldb + k] : B[k * ldb + j];
}
static double elem_af(const float* A, int64_t lda, char ta, int64_t i, int64_t k)
{
    return (double)(is_t(ta) ? A[k * lda + i] : A[i * lda + k]);
}
static double elem_bf(const float* B, int64_t ldb, char tb, int64_t k, int64_t j)
{
    return (double)(is_t(tb) ? B[j * ldb + k] : B[k * ldb + j]);
}

/*
 * One output element of Section IV's C = alpha x A B + beta x C.
 * cold is the old C value (ignored when beta == 0).
 */
static double one_element_d(char ta, char tb, int64_t K, double alpha,
                            const double* A, int64_t lda, const double* B, int64_t ldb,
                            double beta, double cold, int64_t i, int64_t j)
{
    double acc = 0.0;
    for (int64_t k = 0; k < K; ++k)
        acc += elem_a(A, lda, ta, i, k) * elem_b(B, ldb, tb, k, j);
    double r = alpha * acc;
    if (beta != 0.0) r += beta * cold;
    return r;
}

static double one_element_f(char ta, char tb, int64_t K, double alpha,
                            const float* A, int64_t lda, const float* B, int64_t ldb,
                            double beta, double cold, int64_t i, int64_t j)
{
    double acc = 0.0;
    for (int64_t k = 0; k < K; ++k)
        acc += elem_af(A, lda, ta, i, k) * elem_bf(B, ldb, tb, k, j);
    double r = alpha * acc;
    if (beta != 0.0) r += beta * cold;
    return r;
}

typedef struct {
    int fp32;  /* inputs are float, widened to double */
    char ta, tb;
    int64_t i0, j0, rows, cols, K;
    double alpha, beta;
    const void *A, *B;
    int64_t lda, ldb;
    const double* Cold;   /* rows x cols block of the old C, or NULL */
    int64_t ldco;
    double* out;          /* rows x cols result */
    int64_t ldo;
    int64_t r_begin, r_end;
} job_t;

static void* run_rows(void* p)
{
    job_t* jb = (job_t*)p;
    for (int64_t r = jb->r_begin; r < jb->r_end; ++r) {
        for (int64_t c = 0; c < jb->cols; ++c) {
            double cold = (jb->beta != 0.0) ? jb->Cold[r * jb->ldco + c] : 0.0;
            double v;
            if (jb->fp32)
                v = one_element_f(jb->ta, jb->tb, jb->K, jb->alpha, (const float*)jb->A, jb->lda,
                                  (const float*)jb->B, jb->ldb, jb->beta, cold, jb->i0 + r, jb->j0 + c);
            else
                v = one_element_d(jb->ta, jb->tb, jb->K, jb->alpha, (const double*)jb->A, jb->lda,
                                  (const double*)jb->B, jb->ldb, jb->beta, cold, jb->i0 + r, jb->j0 + c);
            jb->out[r * jb->ldo + c] = v;
        }
    }
    return NULL;
}

static int run_block(job_t base, int nthreads)
{
    if (base.rows <= 0 || base.cols <= 0) return 0;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > base.rows) nthreads = (int)base.rows;
    if (nthreads > 256) nthreads = 256;
    job_t jobs[256];
    pthread_t th[256];
    int64_t per = base.rows / nthreads, rem = base.rows % nthreads, r = 0;
    for (int t = 0; t < nthreads; ++t) {
        jobs[t] = base;
        jobs[t].r_begin = r;
        r += per + (t < rem ? 1 : 0);
        jobs[t].r_end = r;
    }
    int started = 0;
    for (int t = 1; t < nthreads; ++t) {
        if (pthread_create(&th[t], NULL, run_rows, &jobs[t]) != 0) break;
        started = t;
    }
    run_rows(&jobs[0]);
    for (int t = 1; t <= started; ++t) pthread_join(th[t], NULL);
    /* rows of threads that failed to start are done here */
    for (int t = started + 1; t < nthreads; ++t) run_rows(&jobs[t]);
    return nthreads;
}

/*
 * Rows i0 .. i0+rows-1 and columns j0 .. j0+cols-1 of
 * alpha * op(A) * op(B) + beta * Cold, FP64 inputs.  A and B are the whole
 * operands (with their leading dimensions); Cold and out are rows x cols
 * blocks.  Returns the number of threads used.
 */
int oracle_dgemm_block(char ta, char tb, int64_t i0, int64_t j0, int64_t rows, int64_t cols,
                       int64_t K, double alpha, const double* A, int64_t lda,
                       const double* B, int64_t ldb, double beta, const double* Cold,
                       int64_t ldco, double* out, int64_t ldo, int nthreads)
{
    job_t b = {0, ta, tb, i0, j0, rows, cols, K, alpha, beta, A, B, lda, ldb,
               Cold, ldco, out, ldo, 0, 0};
    return run_block(b, nthreads);
}

/* Same for FP32 inputs: every element is widened to FP64 before use. */
int oracle_sgemm_block(char ta, char tb, int64_t i0, int64_t j0, int64_t rows, int64_t cols,
                       int64_t K, double alpha, const float* A, int64_t lda,
                       const float* B, int64_t ldb, double beta, const double* Cold,
                       int64_t ldco, double* out, int64_t ldo, int nthreads)
{
    job_t b = {1, ta, tb, i0, j0, rows, cols, K, alpha, beta, A, B, lda, ldb,
               Cold, ldco, out, ldo, 0, 0};
    return run_block(b, nthreads);
}

/*
 * Whole-matrix form, in place on C (M x N, leading dimension ldc), the
 * signature of the problem statement.  Uses a temporary so that the old C
 * values are read before they are overwritten.
 */
int oracle_dgemm(char ta, char tb, int64_t M, int64_t N, int64_t K, double alpha,
                 const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
                 double* C, int64_t ldc, int nthreads)
{
    if (M <= 0 || N <= 0) return 0;
    double* tmp = (double*)malloc((size_t)M * (size_t)N * sizeof(double));
    if (!tmp) return -1;
    int t = oracle_dgemm_block(ta, tb, 0, 0, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc,
                               tmp, N, nthreads);
    for (int64_t i = 0; i < M; ++i)
        for (int64_t j = 0; j < N; ++j) C[i * ldc + j] = tmp[i * N + j];
    free(tmp);
    return t;
}
