/*
 * Seeded synthetic matrices, shared by the tests, the benchmark and the
 * oracle's callers.  This file holds no arithmetic of the GEMM method: it only
 * turns (seed, stream, element index) into numbers.
 *
 * Generator: Philox4x32-10, the counter-based generator of Salmon, Moraes,
 * Dror and Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11):
 * a 4 x 32-bit counter and a 2 x 32-bit key, ten rounds of two 32x32->64
 * multiplications with the round constants 0xD2511F53 / 0xCD9E8D57 and the
 * Weyl key increments 0x9E3779B9 / 0xBB67AE85.  Element e of matrix stream s
 * under seed q uses counter (e_lo, e_hi, s, 0) and key (q_lo, q_hi), so any
 * entry can be regenerated alone and the fill is deterministic under any
 * thread split.  e is the logical row-major index r * cols + c (not the
 * storage offset), so a matrix has the same values whatever its leading
 * dimension.
 *
 * Distributions (kind):
 *   0  uniform [-1, 1)                    2u - 1, u from 53 bits
 *   1  normal N(0, 1)                     Box-Muller on two uniforms
 *   2  sign * 10^U(-4, 4)                 sign from one bit, exponent uniform
 *   3  integers uniform in [-p, p]        p = param (exact in FP32/FP64)
 *   4  dyadic: integer in [-p, p] * 2^-8  exact in FP64
 */
#include <stdint.h>
#include <math.h>
#include <pthread.h>

typedef struct { uint32_t v[4]; } ph4;

static inline void mulhilo(uint32_t a, uint32_t b, uint32_t* hi, uint32_t* lo)
{
    uint64_t p = (uint64_t)a * (uint64_t)b;
    *hi = (uint32_t)(p >> 32);
    *lo = (uint32_t)p;
}

static ph4 philox4x32_10(ph4 c, uint32_t k0, uint32_t k1)
{
    for (int r = 0; r < 10; ++r) {
        uint32_t hi0, lo0, hi1, lo1;
        mulhilo(0xD2511F53u, c.v[0], &hi0, &lo0);
        mulhilo(0xCD9E8D57u, c.v[2], &hi1, &lo1);
        ph4 n;
        n.v[0] = hi1 ^ c.v[1] ^ k0;
        n.v[1] = lo1;
        n.v[2] = hi0 ^ c.v[3] ^ k1;
        n.v[3] = lo0;
        c = n;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

/* one uniform in (0, 1) from 64 bits: 53 bits, offset by half an ulp */
static inline double u01(uint32_t hi, uint32_t lo)
{
    uint64_t x = ((uint64_t)hi << 32) | lo;
    return ((double)(x >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

static double draw(uint64_t seed, uint32_t stream, uint64_t e, int kind, double param)
{
    ph4 c = {{(uint32_t)e, (uint32_t)(e >> 32), stream, 0u}};
    ph4 r = philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    switch (kind) {
    case 0:
        return 2.0 * u01(r.v[0], r.v[1]) - 1.0;
    case 1: {
        double u1 = u01(r.v[0], r.v[1]), u2 = u01(r.v[2], r.v[3]);
        return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
    }
    case 2: {
        double x = -4.0 + 8.0 * u01(r.v[0], r.v[1]);
        double s = (r.v[2] & 1u) ? -1.0 : 1.0;
        return s * pow(10.0, x);
    }
    case 3:
    case 4: {
        int64_t p = (int64_t)param;
        uint64_t span = (uint64_t)(2 * p + 1);
        uint64_t x = (((uint64_t)r.v[0] << 32) | r.v[1]) % span;
        double v = (double)((int64_t)x - p);
        return kind == 3 ? v : v * (1.0 / 256.0);
    }
    default:
        return 0.0;
    }
}

typedef struct {
    uint64_t seed; uint32_t stream; int kind; double param;
    int64_t rows, cols, ld, r0, r1;
    void* out; int fp32;
} fill_job;

static void* fill_rows(void* p)
{
    fill_job* j = (fill_job*)p;
    for (int64_t r = j->r0; r < j->r1; ++r)
        for (int64_t c = 0; c < j->cols; ++c) {
            double v = draw(j->seed, j->stream, (uint64_t)(r * j->cols + c), j->kind, j->param);
            if (j->fp32) ((float*)j->out)[r * j->ld + c] = (float)v;
            else ((double*)j->out)[r * j->ld + c] = v;
        }
    return NULL;
}

/*
 * Fill a rows x cols row-major matrix (leading dimension ld, in elements)
 * with stream `stream` of seed `seed`.  fp32 != 0 writes float (the double
 * draw rounded to nearest), else double.  Returns the threads used.
 */
int synth_fill(void* out, int fp32, int64_t rows, int64_t cols, int64_t ld,
               uint64_t seed, uint32_t stream, int kind, double param, int nthreads)
{
    if (rows <= 0 || cols <= 0) return 0;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if (nthreads > rows) nthreads = (int)rows;
    fill_job jobs[256];
    pthread_t th[256];
    int64_t per = rows / nthreads, rem = rows % nthreads, r = 0;
    for (int t = 0; t < nthreads; ++t) {
        fill_job j = {seed, stream, kind, param, rows, cols, ld, r, 0, out, fp32};
        r += per + (t < rem ? 1 : 0);
        j.r1 = r;
        jobs[t] = j;
    }
    int started = 0;
    for (int t = 1; t < nthreads; ++t) {
        if (pthread_create(&th[t], NULL, fill_rows, &jobs[t]) != 0) break;
        started = t;
    }
    fill_rows(&jobs[0]);
    for (int t = 1; t <= started; ++t) pthread_join(th[t], NULL);
    for (int t = started + 1; t < nthreads; ++t) fill_rows(&jobs[t]);
    return nthreads;
}

/* Raw Philox4x32-10 block, for the known-answer test of the generator. */
void synth_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    ph4 c = {{ctr[0], ctr[1], ctr[2], ctr[3]}};
    ph4 r = philox4x32_10(c, key[0], key[1]);
    for (int i = 0; i < 4; ++i) out[i] = r.v[i];
}
