// Out-of-core triangular solve (TRSM), Cholesky (POTRF) and LU with partial
// pivoting (GETRF) built on the out-of-core GEMM -- the step Section VII of the
// paper names after its DGEMM: the rest of level-3 BLAS and the factorisations
// that use the out-of-core DGEMM as their building block.
//
// TRSM and Cholesky are left-looking over panels of the solution / factor:
//   1. the panel is brought up to date with one out-of-core GEMM (GEMMT with a
//      triangle mask for Cholesky) over everything already solved, streamed
//      from host memory by the Section IV pipeline (ooc_api.cu);
//   2. the panel is solved / factored in device memory by a recursive
//      blocked algorithm: triangular blocks of at most 64 by the substitution
//      and Cholesky kernels below, everything else by the tile kernels.
// LU is right-looking: each panel is factored in device memory (recursive
// halving down to a cooperative 64-column kernel), then the trailing matrix
// gets one out-of-core GEMM.  So nearly all flops run in the pipelined GEMM,
// in the caller's form (FP64 tiles, or the FP64-accurate Ozaki tensor-core form).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <string>
#include <thread>
#include <vector>

#include "device_sync.cuh"
#include "ooc_internal.hpp"

namespace ooc {

namespace {

constexpr int kSmall = 64;     // order of the triangular blocks the small kernels take

// Solve Tm x = alpha p for nvec vectors p of n <= 64 elements, where
// Tm[r][c] = T[c][r] if t_trans else T[r][c], lower or upper triangular (only
// that triangle of the stored T is read), unit diagonal (not read) or not.
// Element e of vector v lives at P[e * es + v * vs].  kVecs right-hand sides
// per CTA, one per thread (the launcher picks 128, 64 or 32 so that the grid
// still fills the SMs).
template <int kVecs>
__global__ void __launch_bounds__(kVecs) trsm_small_kernel(const double* __restrict__ T, int64_t ldt, int n,
                                                           int t_trans, int lower, int unit, double* P, int64_t es,
                                                           int64_t vs, int64_t nvec, double alpha)
{
    // dynamic shared memory (above the 48 KB static limit): the block, then the vectors
    extern __shared__ double smem_f64[];
    double (*Ts)[kSmall + 1] = reinterpret_cast<double (*)[kSmall + 1]>(smem_f64);
    double (*Xs)[kSmall + 1] = reinterpret_cast<double (*)[kSmall + 1]>(smem_f64 + kSmall * (kSmall + 1));
    const int tid = threadIdx.x;
    const int64_t v0 = (int64_t)blockIdx.x * kVecs;
    for (int idx = tid; idx < n * n; idx += blockDim.x) {
        const int r = idx / n, c = idx % n;
        double t = 0.0;
        if (r == c) t = unit ? 1.0 : T[(int64_t)r * ldt + c];
        else if (lower ? c < r : c > r) t = t_trans ? T[(int64_t)c * ldt + r] : T[(int64_t)r * ldt + c];
        Ts[r][c] = t;
    }
    // stage the vectors, the unit-stride index fastest for coalescing
    const bool v_fast = vs == 1;
    for (int idx = tid; idx < n * kVecs; idx += blockDim.x) {
        const int e = v_fast ? idx / kVecs : idx % n;
        const int v = v_fast ? idx % kVecs : idx / n;
        if (v0 + v < nvec) Xs[v][e] = P[(int64_t)e * es + (v0 + v) * vs];
    }
    __syncthreads();
    if (v0 + tid < nvec) {
        // one right-hand side per thread; four partial sums break the dependent FMA chain
        double* x = Xs[tid];
        for (int q = 0; q < n; ++q) {
            const int r = lower ? q : n - 1 - q;
            const int c0 = lower ? 0 : r + 1, c1 = lower ? r : n;
            double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
            int c = c0;
            for (; c + 3 < c1; c += 4) {
                s0 = fma(Ts[r][c], x[c], s0);
                s1 = fma(Ts[r][c + 1], x[c + 1], s1);
                s2 = fma(Ts[r][c + 2], x[c + 2], s2);
                s3 = fma(Ts[r][c + 3], x[c + 3], s3);
            }
            for (; c < c1; ++c) s0 = fma(Ts[r][c], x[c], s0);
            const double s = alpha * x[r] - ((s0 + s1) + (s2 + s3));
            x[r] = unit ? s : s / Ts[r][r];
        }
    }
    __syncthreads();
    for (int idx = tid; idx < n * kVecs; idx += blockDim.x) {
        const int e = v_fast ? idx / kVecs : idx % n;
        const int v = v_fast ? idx % kVecs : idx / n;
        if (v0 + v < nvec) P[(int64_t)e * es + (v0 + v) * vs] = Xs[v][e];
    }
}

// Cholesky of one n x n block (n <= 64) in place: the lower triangle of T
// becomes L with L L^T = T (upper != 0: the upper triangle becomes U = L^T
// with U^T U = T).  Only that triangle is read and written.  A pivot that is
// not positive stops the block and records gofs + its column + 1 in *info
// (first failure wins).
__global__ void __launch_bounds__(256) potrf_small_kernel(double* T, int64_t ldt, int n, int upper, int64_t gofs,
                                                          unsigned long long* info)
{
    __shared__ double S[kSmall][kSmall + 1];
    __shared__ int fail;
    const int tid = threadIdx.x;
    for (int idx = tid; idx < n * n; idx += blockDim.x) {
        const int r = idx / n, c = idx % n;
        if (c <= r) S[r][c] = upper ? T[(int64_t)c * ldt + r] : T[(int64_t)r * ldt + c];
    }
    if (tid == 0) fail = 0;
    __syncthreads();
    for (int j = 0; j < n; ++j) {
        if (tid == 0) {
            const double d = S[j][j];
            if (d > 0.0) S[j][j] = sqrt(d);
            else fail = j + 1;
        }
        __syncthreads();
        if (fail) break;
        for (int i = j + 1 + tid; i < n; i += blockDim.x) S[i][j] = S[i][j] / S[j][j];
        __syncthreads();
        const int m = n - j - 1;
        for (int idx = tid; idx < m * m; idx += blockDim.x) {
            const int i = j + 1 + idx / m, k = j + 1 + idx % m;
            if (k <= i) S[i][k] -= S[i][j] * S[k][j];
        }
        __syncthreads();
    }
    if (tid == 0 && fail) atomicCAS(info, 0ull, (unsigned long long)(gofs + fail));
    for (int idx = tid; idx < n * n; idx += blockDim.x) {
        const int r = idx / n, c = idx % n;
        if (c <= r) {
            if (upper) T[(int64_t)c * ldt + r] = S[r][c];
            else T[(int64_t)r * ldt + c] = S[r][c];
        }
    }
}

// ---- LU with partial pivoting ------------------------------------------------
constexpr int kLuThreads = 256;
constexpr int kLuWarps = kLuThreads / 32;
constexpr size_t kLuSmemMax = 200 * 1024;  // dynamic shared memory for a CTA's rows

// Barrier across the CTAs of a cooperative launch (all co-resident), bounded:
// a CTA that waits longer than kWaitLimitNs records kErrGridBarrier and gets
// false (the caller returns), so a lost arrival ends the kernel with an error.
// bar[0] counts arrivals, bar[1] is the generation.
__device__ bool grid_barrier(unsigned* bar, int* err)
{
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned* gen = bar + 1;
        const unsigned g = *gen;
        __threadfence();
        if (atomicAdd(bar, 1u) == gridDim.x - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            const uint64_t t0 = globaltimer_ns();
            while (*gen == g) {
                if (globaltimer_ns() - t0 > kWaitLimitNs) {
                    atomicCAS(err, 0, kErrGridBarrier);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

// Unblocked LU with partial pivoting of an m x nw panel (nw <= 64), in place,
// row-major with leading dimension ldp: the first largest |a| of each column
// at or below the diagonal is the pivot (piv[j] = its row), rows are swapped
// across the nw columns, the rows below are scaled and updated.  CTA g owns
// rows [g * rows_per_cta, (g + 1) * rows_per_cta) and is the only one that
// writes them; with kInSmem they stay in shared memory (stride kLuLd) from the
// first column to the last.  Per column each CTA publishes its candidate
// (largest |a|, smallest row on ties) together with that row's current
// values, and the owner of row j publishes row j; one grid barrier; then
// every CTA picks the same global winner and reads the pivot row and row j
// from the published copies.  The published slots alternate between two
// buffers by column parity: a CTA can only rewrite a column's slots two
// columns later, after the next barrier, which every CTA reaches only when
// it has finished reading them.  A zero pivot records gofs + j + 1 in *info
// (first failure wins) and skips the update; a column with no comparable
// entry (all NaN) keeps row j as its pivot.
constexpr int kLuLd = kSmall + 1;  // shared-memory row stride (doubles): column reads hit distinct banks

template <bool kInSmem>
__device__ __forceinline__ double& lu_at(double* S, double* P, int64_t ldp, int64_t r0, int64_t i, int k)
{
    if constexpr (kInSmem) return S[(i - r0) * kLuLd + k];
    else return P[i * ldp + k];
}

template <bool kInSmem>
__global__ void __launch_bounds__(kLuThreads) narrow_lu_kernel(double* P, int64_t ldp, int64_t m, int nw,
                                                               int64_t rows_per_cta, int64_t* piv, double* cand_v,
                                                               int64_t* cand_i, double* cand_row, double* jrow_buf,
                                                               unsigned* bar, int* err, unsigned long long* info,
                                                               int64_t gofs)
{
    extern __shared__ double S[];  // kInSmem: the CTA's rows
    __shared__ double prow[kSmall], jrow[kSmall];
    __shared__ double wv[kLuWarps];
    __shared__ int64_t wi[kLuWarps];
    __shared__ int64_t s_bi, s_p;
    __shared__ int s_found;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned G = gridDim.x;
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_cta, r1 = min(m, r0 + rows_per_cta);
    if constexpr (kInSmem) {
        const int64_t n = (r1 > r0 ? r1 - r0 : 0) * nw;
        for (int64_t e = tid; e < n; e += kLuThreads) {
            const int64_t r = e / nw;
            const int k = (int)(e % nw);
            S[r * kLuLd + k] = P[(r0 + r) * ldp + k];
        }
    }
    for (int j = 0; j < nw; ++j) {
        const int b = j & 1;
        __syncthreads();
        // local candidate: largest |a[i][j]| over own rows i >= j, smallest row on ties
        double bv = -1.0;
        int64_t bi = INT64_MAX;
        for (int64_t i = max(r0, (int64_t)j) + tid; i < r1; i += kLuThreads) {
            const double v = fabs(lu_at<kInSmem>(S, P, ldp, r0, i, j));
            if (v > bv) { bv = v; bi = i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_down_sync(0xffffffffu, bv, o);
            const int64_t oi = __shfl_down_sync(0xffffffffu, bi, o);
            if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
        }
        if (lane == 0) { wv[warp] = bv; wi[warp] = bi; }
        __syncthreads();
        if (tid == 0) {
            for (int w = 1; w < kLuWarps; ++w)
                if (wv[w] > bv || (wv[w] == bv && wi[w] < bi)) { bv = wv[w]; bi = wi[w]; }
            cand_v[b * G + blockIdx.x] = bv;
            cand_i[b * G + blockIdx.x] = bi;
            s_bi = bi;
        }
        __syncthreads();
        // publish the candidate row and, from its owner, row j
        const int64_t cb = s_bi;
        double* crow = cand_row + ((int64_t)b * G + blockIdx.x) * kSmall;
        for (int k = tid; k < nw; k += kLuThreads) {
            if (cb != INT64_MAX) crow[k] = lu_at<kInSmem>(S, P, ldp, r0, cb, k);
            if (j >= r0 && j < r1) jrow_buf[b * kSmall + k] = lu_at<kInSmem>(S, P, ldp, r0, j, k);
        }
        if (!grid_barrier(bar, err)) return;
        // every CTA reduces the candidates the same way: the global first maximum
        if (warp == 0) {
            double gv = -1.0;
            int64_t gi = INT64_MAX;
            for (unsigned g = lane; g < G; g += 32) {
                const double v = __ldcg(cand_v + b * G + g);
                const int64_t i = __ldcg(cand_i + b * G + g);
                if (v > gv || (v == gv && i < gi)) { gv = v; gi = i; }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const double ov = __shfl_down_sync(0xffffffffu, gv, o);
                const int64_t oi = __shfl_down_sync(0xffffffffu, gi, o);
                if (ov > gv || (ov == gv && oi < gi)) { gv = ov; gi = oi; }
            }
            if (lane == 0) {
                s_found = gi != INT64_MAX;
                s_p = gi != INT64_MAX ? gi : (int64_t)j;
            }
        }
        __syncthreads();
        const int64_t p = s_p;
        const double* src = s_found ? cand_row + ((int64_t)b * G + (unsigned)(p / rows_per_cta)) * kSmall
                                    : jrow_buf + b * kSmall;
        for (int k = tid; k < nw; k += kLuThreads) {
            prow[k] = __ldcg(src + k);
            jrow[k] = __ldcg(jrow_buf + b * kSmall + k);
        }
        if (blockIdx.x == 0 && tid == 0) piv[j] = p;
        __syncthreads();
        const double pv = prow[j];
        const bool zero = pv == 0.0;
        if (zero && blockIdx.x == 0 && tid == 0) atomicCAS(info, 0ull, (unsigned long long)(gofs + j + 1));
        // the interchange on own rows: row j becomes the pivot row, row p the old row j
        for (int k = tid; k < nw; k += kLuThreads) {
            if (j >= r0 && j < r1) lu_at<kInSmem>(S, P, ldp, r0, j, k) = prow[k];
            if (p != j && p >= r0 && p < r1) lu_at<kInSmem>(S, P, ldp, r0, p, k) = jrow[k];
        }
        __syncthreads();
        if (zero) continue;
        // own rows below j, one warp per row: multiplier a[j] / pivot, then the rank-1 update
        for (int64_t i = max(r0, (int64_t)j + 1) + warp; i < r1; i += kLuWarps) {
            const int k0 = lane, k1 = lane + 32;
            double a0 = 0.0, a1 = 0.0;
            if (k0 < nw) a0 = lu_at<kInSmem>(S, P, ldp, r0, i, k0);
            if (k1 < nw) a1 = lu_at<kInSmem>(S, P, ldp, r0, i, k1);
            const double aj = __shfl_sync(0xffffffffu, j < 32 ? a0 : a1, j & 31);
            const double l = aj / pv;
            if (k0 > j && k0 < nw) a0 = fma(-l, prow[k0], a0);
            if (k1 > j && k1 < nw) a1 = fma(-l, prow[k1], a1);
            if (k0 == j) a0 = l;
            if (k1 == j) a1 = l;
            if (k0 < nw) lu_at<kInSmem>(S, P, ldp, r0, i, k0) = a0;
            if (k1 < nw) lu_at<kInSmem>(S, P, ldp, r0, i, k1) = a1;
        }
    }
    if constexpr (kInSmem) {
        __syncthreads();
        const int64_t n = (r1 > r0 ? r1 - r0 : 0) * nw;
        for (int64_t e = tid; e < n; e += kLuThreads) {
            const int64_t r = e / nw;
            const int k = (int)(e % nw);
            P[(r0 + r) * ldp + k] = S[r * kLuLd + k];
        }
    }
}

// Row interchanges k <-> piv[k] for k in [k0, k1), in order, over columns [0, ncols) of P
// (one thread per column).
__global__ void laswp_kernel(double* P, int64_t ldp, int64_t ncols, const int64_t* piv, int64_t k0, int64_t k1)
{
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ncols; c += (int64_t)gridDim.x * blockDim.x)
        for (int64_t k = k0; k < k1; ++k) {
            const int64_t p = piv[k];
            if (p != k) {
                const double t = P[k * ldp + c];
                P[k * ldp + c] = P[p * ldp + c];
                P[p * ldp + c] = t;
            }
        }
}

__global__ void add_offset_kernel(int64_t* v, int64_t n, int64_t off)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v[i] += off;
}

__global__ void scale_kernel(double* P, int64_t ld, int64_t rows, int64_t cols, double alpha)
{
    const int64_t n = rows * cols;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / cols, c = i % cols;
        P[r * ld + c] *= alpha;
    }
}

template <int kVecs>
constexpr size_t trsm_smem() { return (size_t)(kSmall + kVecs) * (kSmall + 1) * sizeof(double); }

template <int kVecs>
int launch_trsm_small(const double* T, int64_t ldt, int n, bool t_trans, bool lower, bool unit, double* P,
                      int64_t es, int64_t vs, int64_t nv, cudaStream_t st, std::string& why)
{
    static const cudaError_t attr = cudaFuncSetAttribute(
        trsm_small_kernel<kVecs>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)trsm_smem<kVecs>());
    if (attr != cudaSuccess) {
        why = std::string("trsm_small_kernel shared memory: ") + cudaGetErrorString(attr);
        return OOC_ERR_CUDA;
    }
    const int64_t grid = (nv + kVecs - 1) / kVecs;
    trsm_small_kernel<kVecs><<<(unsigned)grid, kVecs, trsm_smem<kVecs>(), st>>>(
        T, ldt, n, t_trans ? 1 : 0, lower ? 1 : 0, unit ? 1 : 0, P, es, vs, nv, 1.0);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        why = std::string("trsm_small_kernel: ") + cudaGetErrorString(e);
        return OOC_ERR_CUDA;
    }
    return OOC_OK;
}

int check_launch(const char* what, std::string& why)
{
    const cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) return OOC_OK;
    why = std::string(what) + ": " + cudaGetErrorString(e);
    return OOC_ERR_CUDA;
}

// Device state of one driver call.
struct Dev {
    cudaStream_t st = nullptr;
    int* err = nullptr;                  // error word of the tile kernels' bounded waits
    unsigned long long* info = nullptr;  // first failed Cholesky pivot (global column + 1)
    int64_t launches = 0;
    // LU panel scratch: grid barrier words, per-CTA pivot candidates and their rows
    // (two buffers each, by column parity), the published row j; lu_grid bounds the grid
    unsigned* bar = nullptr;
    double* cand_v = nullptr;
    int64_t* cand_i = nullptr;
    double* cand_row = nullptr;
    double* jrow = nullptr;
    int lu_grid = 0;
    bool lu_rows_global = false;  // keep the panel's rows in global memory (the path for very tall panels)
    // Ozaki form for the in-HBM updates: digit-plane scratch (null: FP64 tiles)
    char* oz = nullptr;
    size_t oz_bytes = 0;
    int oz_slices = kOzakiSlicesFactor;
};

// One in-HBM update C = alpha op(A) op(B) + beta C: the Ozaki form when the call
// asked for it and its digit planes fit the scratch, else the FP64 tile kernel.
int dev_gemm(Dev& d, bool a_k, bool b_k, int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t lda,
             const double* B, int64_t ldb, double beta, bool read_c, double* C, int64_t ldc, std::string& why,
             int tri = 0, int64_t tri_off = 0)
{
    if (d.oz && K > 0 && ozaki_device_scratch(M, N, K, d.oz_slices) <= d.oz_bytes) {
        d.launches += 7;  // two splits of three kernels each, one tensor-core launch
        return ozaki_gemm_device(a_k, b_k, M, N, K, alpha, A, lda, B, ldb, beta, read_c, C, ldc, d.oz_slices, d.oz,
                                 d.oz_bytes, d.err, d.st, why, tri, tri_off);
    }
    ++d.launches;
    return launch_fp64_tile(a_k, b_k, M, N, K, alpha, A, lda, B, ldb, beta, read_c, C, ldc, d.err, d.st, why, tri,
                            tri_off);
}

// Split n > 64 at a multiple of 64 near its middle (keeps sub-blocks 16-byte aligned for TMA).
int64_t split_point(int64_t n) { return std::max<int64_t>(kSmall, (n / 2) / kSmall * kSmall); }

// The stored position of the sub-block of op(T) at (r0, c0), as a tile-kernel
// operand: as an A operand it is "rows x K" stored (a_kmajor) unless T is
// transposed; as a B operand it is "cols x K" stored (b_kmajor) iff T is.
const double* opT_block(const double* T, int64_t ldt, bool t_trans, int64_t r0, int64_t c0)
{
    return t_trans ? T + c0 * ldt + r0 : T + r0 * ldt + c0;
}

// In device memory: solve op(T) X = P (left) or X op(T) = P (right) in place
// in P, op(T) of order n lower (op_lower) or upper triangular; P is n x nv
// (left) or nv x n (right), row-major with leading dimension ldp.
int incore_trsm(bool left, bool op_lower, const double* T, int64_t ldt, bool t_trans, bool unit, int64_t n,
                double* P, int64_t ldp, int64_t nv, Dev& d, std::string& why)
{
    if (n <= 0 || nv <= 0) return OOC_OK;
    if (n <= kSmall) {
        // the substitution kernel solves Tm x = p: Tm = op(T) (left) or op(T)^T (right)
        const bool tm_lower = left ? op_lower : !op_lower;
        const bool tm_trans = left ? t_trans : !t_trans;
        const int64_t es = left ? ldp : 1, vs = left ? 1 : ldp;
        // the most right-hand sides per CTA (more warps per SM) that still gives two CTAs per SM
        const int64_t want = 2 * (int64_t)device_sm_count();
        ++d.launches;
        if ((nv + 127) / 128 >= want)
            return launch_trsm_small<128>(T, ldt, (int)n, tm_trans, tm_lower, unit, P, es, vs, nv, d.st, why);
        if ((nv + 63) / 64 >= want)
            return launch_trsm_small<64>(T, ldt, (int)n, tm_trans, tm_lower, unit, P, es, vs, nv, d.st, why);
        return launch_trsm_small<32>(T, ldt, (int)n, tm_trans, tm_lower, unit, P, es, vs, nv, d.st, why);
    }
    const int64_t n1 = split_point(n), n2 = n - n1;
    const double* T11 = T;
    const double* T22 = T + n1 * ldt + n1;
    int rc;
    auto gemm = [&](bool a_k, bool b_k, int64_t M, int64_t N, int64_t K, const double* A, int64_t lda,
                    const double* B, int64_t ldb, double* C) {
        return dev_gemm(d, a_k, b_k, M, N, K, -1.0, A, lda, B, ldb, 1.0, true, C, ldp, why);
    };
    if (left) {
        double* P1 = P;
        double* P2 = P + n1 * ldp;
        if (op_lower) {  // X1 = T11 \ P1;  P2 -= T21 X1;  X2 = T22 \ P2
            if ((rc = incore_trsm(left, op_lower, T11, ldt, t_trans, unit, n1, P1, ldp, nv, d, why))) return rc;
            if ((rc = gemm(!t_trans, false, n2, nv, n1, opT_block(T, ldt, t_trans, n1, 0), ldt, P1, ldp, P2)))
                return rc;
            return incore_trsm(left, op_lower, T22, ldt, t_trans, unit, n2, P2, ldp, nv, d, why);
        }
        // upper: X2 = T22 \ P2;  P1 -= T12 X2;  X1 = T11 \ P1
        if ((rc = incore_trsm(left, op_lower, T22, ldt, t_trans, unit, n2, P2, ldp, nv, d, why))) return rc;
        if ((rc = gemm(!t_trans, false, n1, nv, n2, opT_block(T, ldt, t_trans, 0, n1), ldt, P2, ldp, P1))) return rc;
        return incore_trsm(left, op_lower, T11, ldt, t_trans, unit, n1, P1, ldp, nv, d, why);
    }
    double* P1 = P;        // columns [0, n1)
    double* P2 = P + n1;   // columns [n1, n)
    if (op_lower) {  // X2 = P2 / T22;  P1 -= X2 T21;  X1 = P1 / T11
        if ((rc = incore_trsm(left, op_lower, T22, ldt, t_trans, unit, n2, P2, ldp, nv, d, why))) return rc;
        if ((rc = gemm(true, t_trans, nv, n1, n2, P2, ldp, opT_block(T, ldt, t_trans, n1, 0), ldt, P1))) return rc;
        return incore_trsm(left, op_lower, T11, ldt, t_trans, unit, n1, P1, ldp, nv, d, why);
    }
    // upper: X1 = P1 / T11;  P2 -= X1 T12;  X2 = P2 / T22
    if ((rc = incore_trsm(left, op_lower, T11, ldt, t_trans, unit, n1, P1, ldp, nv, d, why))) return rc;
    if ((rc = gemm(true, t_trans, nv, n2, n1, P1, ldp, opT_block(T, ldt, t_trans, 0, n1), ldt, P2))) return rc;
    return incore_trsm(left, op_lower, T22, ldt, t_trans, unit, n2, P2, ldp, nv, d, why);
}

// In device memory: Cholesky of the n x n block T in place (lower: L L^T,
// upper: U^T U); gofs is the block's first global column (for info).
int incore_potrf(bool upper, double* T, int64_t ldt, int64_t n, int64_t gofs, Dev& d, std::string& why)
{
    if (n <= kSmall) {
        potrf_small_kernel<<<1, 256, 0, d.st>>>(T, ldt, (int)n, upper ? 1 : 0, gofs, d.info);
        ++d.launches;
        return check_launch("potrf_small_kernel", why);
    }
    const int64_t n1 = split_point(n), n2 = n - n1;
    double* T22 = T + n1 * ldt + n1;
    int rc;
    if ((rc = incore_potrf(upper, T, ldt, n1, gofs, d, why))) return rc;
    if (!upper) {
        // L21 = T21 L11^{-T} (right solve with op = transpose of the stored lower L11, an upper op)
        double* T21 = T + n1 * ldt;
        if ((rc = incore_trsm(false, false, T, ldt, true, false, n1, T21, ldt, n2, d, why))) return rc;
        // T22 -= L21 L21^T on the lower triangle
        if ((rc = dev_gemm(d, true, true, n2, n2, n1, -1.0, T21, ldt, T21, ldt, 1.0, true, T22, ldt, why, 1, 0)))
            return rc;
    } else {
        // U12 = U11^{-T} T12 (left solve with op = transpose of the stored upper U11, a lower op)
        double* T12 = T + n1;
        if ((rc = incore_trsm(true, true, T, ldt, true, false, n1, T12, ldt, n2, d, why))) return rc;
        // T22 -= U12^T U12 on the upper triangle
        if ((rc = dev_gemm(d, false, false, n2, n2, n1, -1.0, T12, ldt, T12, ldt, 1.0, true, T22, ldt, why, 2, 0)))
            return rc;
    }
    return incore_potrf(upper, T22, ldt, n2, gofs + n1, d, why);
}

int launch_laswp(double* P, int64_t ldp, int64_t ncols, const int64_t* piv, int64_t k0, int64_t k1, Dev& d,
                 std::string& why)
{
    if (ncols <= 0 || k1 <= k0) return OOC_OK;
    const int64_t grid = std::min<int64_t>((ncols + 255) / 256, 4096);
    laswp_kernel<<<(unsigned)grid, 256, 0, d.st>>>(P, ldp, ncols, piv, k0, k1);
    ++d.launches;
    return check_launch("laswp_kernel", why);
}

// In device memory: LU with partial pivoting of the m x n panel P (m >= n),
// recursive halving at multiples of 64 (Toledo's recursive LU): factor the
// left half, interchange the right half's rows, U12 = L11^{-1} A12, A22 -=
// L21 U12 on the tile kernel, factor A22, interchange the left half's rows.
// piv (device, n entries) receives panel-relative pivot rows; gofs is the
// panel's first global column (for info).
int panel_lu(double* P, int64_t ldp, int64_t m, int64_t n, int64_t* piv, int64_t gofs, Dev& d, std::string& why)
{
    if (n <= kSmall) {
        // rows in shared memory when a co-resident grid's slices fit, else in global memory
        int64_t grid = std::max<int64_t>(1, std::min<int64_t>(d.lu_grid, (m + 31) / 32));
        const int sms = device_sm_count();
        bool in_smem = !d.lu_rows_global;
        size_t smem = 0;
        while (in_smem) {
            smem = (size_t)((m + grid - 1) / grid) * kLuLd * sizeof(double);
            int occ = 0;
            if (smem > kLuSmemMax ||
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, narrow_lu_kernel<true>, kLuThreads, smem) !=
                    cudaSuccess ||
                occ == 0) {
                cudaGetLastError();
                in_smem = false;
                break;
            }
            if ((int64_t)occ * sms >= grid) break;
            grid = (int64_t)occ * sms;  // fewer, taller slices until the grid is co-resident
        }
        if (!in_smem) {
            grid = std::max<int64_t>(1, std::min<int64_t>(d.lu_grid, (m + 31) / 32));
            smem = 0;
        }
        int64_t rows_per_cta = (m + grid - 1) / grid;
        unsigned* bar = d.bar;
        int nw = (int)n;
        void* args[] = {&P,         &ldp,    &m,    &nw,   &rows_per_cta, &piv,  &d.cand_v,
                        &d.cand_i,  &d.cand_row, &d.jrow, &bar, &d.err, &d.info, &gofs};
        if (cudaMemsetAsync(d.bar, 0, 2 * sizeof(unsigned), d.st) != cudaSuccess) {
            why = "barrier reset failed";
            return OOC_ERR_CUDA;
        }
        const void* fn = in_smem ? (const void*)narrow_lu_kernel<true> : (const void*)narrow_lu_kernel<false>;
        const cudaError_t e =
            cudaLaunchCooperativeKernel(fn, dim3((unsigned)grid), dim3(kLuThreads), args, smem, d.st);
        ++d.launches;
        if (e != cudaSuccess) {
            cudaGetLastError();
            why = std::string("narrow_lu_kernel cooperative launch: ") + cudaGetErrorString(e);
            return OOC_ERR_CUDA;
        }
        return OOC_OK;
    }
    const int64_t n1 = split_point(n), n2 = n - n1;
    int rc;
    if ((rc = panel_lu(P, ldp, m, n1, piv, gofs, d, why))) return rc;
    if ((rc = launch_laswp(P + n1, ldp, n2, piv, 0, n1, d, why))) return rc;
    if ((rc = incore_trsm(true, true, P, ldp, false, true, n1, P + n1, ldp, n2, d, why))) return rc;
    if (m > n1) {
        if ((rc = dev_gemm(d, true, false, m - n1, n2, n1, -1.0, P + n1 * ldp, ldp, P + n1, ldp, 1.0, true,
                           P + n1 * ldp + n1, ldp, why)))
            return rc;
        if ((rc = panel_lu(P + n1 * ldp + n1, ldp, m - n1, n2, piv + n1, gofs + n1, d, why))) return rc;
        add_offset_kernel<<<1, 256, 0, d.st>>>(piv + n1, n2, n1);
        ++d.launches;
        if ((rc = check_launch("add_offset_kernel", why))) return rc;
        if ((rc = launch_laswp(P, ldp, n1, piv, n1, n, d, why))) return rc;
    }
    return OOC_OK;
}

int64_t round_up64(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

bool is_l(char c) { return c == 'L' || c == 'l'; }
bool is_r(char c) { return c == 'R' || c == 'r'; }
bool is_u(char c) { return c == 'U' || c == 'u'; }
bool is_n(char c) { return c == 'N' || c == 'n'; }
bool is_t(char c) { return c == 'T' || c == 't'; }

int fail(int code, const std::string& msg)
{
    set_error(msg);
    return code;
}

// One driver call: a device arena of the budget (its first 256 bytes hold the
// error word and the pivot word), one stream, the running statistics.
struct Driver {
    char* arena = nullptr;
    size_t bytes = 0;
    Dev d;
    double h2d = 0, d2h = 0, kernel_s = 0, split_s = 0;
    int64_t steps = 0, launches = 0;
    ooc_opts gemm_opts;
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();

    ~Driver()
    {
        if (d.st) {
            cudaStreamSynchronize(d.st);
            cudaStreamDestroy(d.st);
        }
        if (arena) cudaFree(arena);
        cudaGetLastError();
    }

    int init(size_t budget, const ooc_opts* opts, std::string& why)
    {
        std::memset(&gemm_opts, 0, sizeof(gemm_opts));
        if (opts) gemm_opts = *opts;
        if (gemm_opts.form == OOC_FORM_OZAKI) {
            // the factors must track FP64's: 9 digits of 6 bits (54 bits) unless the caller chose
            if (gemm_opts.slices == 0) gemm_opts.slices = kOzakiSlicesFactor;
            if (gemm_opts.slices < 2 || gemm_opts.slices > kOzakiMaxSlices) {
                why = "opts->slices must be 0 or 2.." + std::to_string(kOzakiMaxSlices);
                return OOC_ERR_INVALID_ARG;
            }
            d.oz_slices = gemm_opts.slices;
        }
        if (gemm_opts.workspace) {
            why = "the TRSM / Cholesky drivers allocate their own arena (opts->workspace must be NULL)";
            return OOC_ERR_INVALID_ARG;
        }
        bytes = budget;
        if (cudaMalloc(&arena, bytes) != cudaSuccess) {
            cudaGetLastError();
            arena = nullptr;
            why = "device arena of " + std::to_string(bytes) + " bytes";
            return OOC_ERR_ALLOC;
        }
        if (cudaStreamCreateWithFlags(&d.st, cudaStreamNonBlocking) != cudaSuccess) {
            why = "stream creation failed";
            return OOC_ERR_CUDA;
        }
        d.err = reinterpret_cast<int*>(arena);
        d.info = reinterpret_cast<unsigned long long*>(arena + 8);
        if (cudaMemsetAsync(arena, 0, 256, d.st) != cudaSuccess) return OOC_ERR_CUDA;
        gemm_opts.workspace = arena + 256;
        gemm_opts.workspace_bytes = bytes - 256;
        return OOC_OK;
    }

    // one out-of-core GEMM over host operands, in the arena
    int gemm(char ta, char tb, int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t lda,
             const double* B, int64_t ldb, double beta, double* C, int64_t ldc, int tri)
    {
        if (cudaStreamSynchronize(d.st) != cudaSuccess) return fail(OOC_ERR_CUDA, "stream synchronise failed");
        ooc_stats st;
        const int rc = run_gemm_host(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, 8, bytes - 256,
                                     &gemm_opts, &st, tri, 0);
        if (rc) return rc;
        h2d += st.h2d_bytes;
        d2h += st.d2h_bytes;
        kernel_s += st.kernel_seconds;
        split_s += st.split_seconds;
        launches += st.kernel_launches;
        ++steps;
        return OOC_OK;
    }

    int copy_in(double* dst, int64_t ldd, const double* src, int64_t lds, int64_t rows, int64_t cols)
    {
        if (rows <= 0 || cols <= 0) return OOC_OK;
        if (cudaMemcpy2DAsync(dst, ldd * 8, src, lds * 8, cols * 8, rows, cudaMemcpyHostToDevice, d.st) !=
            cudaSuccess)
            return fail(OOC_ERR_CUDA, "panel copy to the device failed");
        h2d += (double)rows * cols * 8;
        return OOC_OK;
    }

    int copy_out(double* dst, int64_t ldd, const double* src, int64_t lds, int64_t rows, int64_t cols)
    {
        if (rows <= 0 || cols <= 0) return OOC_OK;
        if (cudaMemcpy2DAsync(dst, ldd * 8, src, lds * 8, cols * 8, rows, cudaMemcpyDeviceToHost, d.st) !=
            cudaSuccess)
            return fail(OOC_ERR_CUDA, "panel copy to the host failed");
        d2h += (double)rows * cols * 8;
        return OOC_OK;
    }

    // wait for the stream and turn a device-side error word into a status
    int drain()
    {
        if (cudaStreamSynchronize(d.st) != cudaSuccess)
            return fail(OOC_ERR_CUDA, std::string("panel stream: ") + cudaGetErrorString(cudaGetLastError()));
        int herr = 0;
        if (cudaMemcpy(&herr, d.err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
            return fail(OOC_ERR_CUDA, "error word read failed");
        if (herr) return fail(OOC_ERR_TIMEOUT, "a device-side wait gave up (status " + std::to_string(herr) + ")");
        return OOC_OK;
    }

    void finish(ooc_stats* stats, double flops)
    {
        if (!stats) return;
        std::memset(stats, 0, sizeof(*stats));
        stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        stats->device_seconds = stats->seconds;
        stats->kernel_seconds = kernel_s;
        stats->split_seconds = split_s;
        stats->tflops = stats->seconds > 0 ? flops / stats->seconds / 1e12 : 0.0;
        stats->h2d_bytes = h2d;
        stats->d2h_bytes = d2h;
        stats->form = gemm_opts.form;
        if (gemm_opts.form == OOC_FORM_OZAKI) {
            stats->slices = gemm_opts.slices;
            stats->products = gemm_opts.slices * (gemm_opts.slices + 1) / 2;
        }
        stats->steps = steps;
        stats->device_bytes = (int64_t)bytes;
        stats->kernel_launches = launches + d.launches;
    }
};

// Split a region between a chunk of right-hand sides of a t-order solve (rows:
// vectors are rows of ld round_up(t, 16); else columns of a t-row block) and,
// for Ozaki updates, the digit-plane scratch of the largest in-HBM update
// (order t, the chunk's vectors); sets the Dev's scratch and returns the chunk.
int64_t chunk_and_scratch(Driver& dr, char* region, size_t region_bytes, int64_t t, bool rows, int64_t nv_max)
{
    const int64_t lt = round_up64(t, 16);
    auto bytes_of = [&](int64_t c) {
        const size_t b = rows ? (size_t)c * lt * 8 : (size_t)t * round_up64(c, 16) * 8;
        return (b + 255) / 256 * 256;
    };
    int64_t c = rows ? (int64_t)(region_bytes / (8 * (size_t)lt)) : (int64_t)(region_bytes / (8 * (size_t)t)) / 16 * 16;
    c = std::max<int64_t>(kSmall, std::min(c, round_up64(std::max<int64_t>(nv_max, kSmall), 16)));
    dr.d.oz = nullptr;
    dr.d.oz_bytes = 0;
    if (dr.gemm_opts.form == OOC_FORM_OZAKI) {
        while (c > kSmall && bytes_of(c) + ozaki_device_scratch(t, c, t, dr.d.oz_slices) > region_bytes)
            c = std::max<int64_t>(kSmall, c / 2 / 16 * 16);
        if (bytes_of(c) + ozaki_device_scratch(t, c, t, dr.d.oz_slices) <= region_bytes) {
            dr.d.oz = region + bytes_of(c);
            dr.d.oz_bytes = region_bytes - bytes_of(c);
        }
    }
    return c;
}

// Row interchanges k <-> ipiv[k] for k in [k0, k1), in order, over host columns
// [c0, c1) of A; the columns are split over host threads (each applies every
// interchange to its columns, so the order is kept).
void host_laswp(double* A, int64_t lda, int64_t c0, int64_t c1, const int64_t* ipiv, int64_t k0, int64_t k1)
{
    if (c1 <= c0 || k1 <= k0) return;
    const int64_t ncols = c1 - c0;
    const int64_t hw = std::max<unsigned>(1u, std::thread::hardware_concurrency());
    const int nt = (int)std::max<int64_t>(1, std::min<int64_t>({hw, 32, ncols / 64}));
    auto work = [=](int64_t a, int64_t b) {
        for (int64_t k = k0; k < k1; ++k) {
            const int64_t p = ipiv[k];
            if (p != k) std::swap_ranges(A + k * lda + a, A + k * lda + b, A + p * lda + a);
        }
    };
    std::vector<std::thread> th;
    int started = 1;
    try {
        for (int t = 1; t < nt; ++t, ++started) th.emplace_back(work, c0 + ncols * t / nt, c0 + ncols * (t + 1) / nt);
    } catch (...) {
    }
    work(c0, c0 + ncols / nt);
    for (int t = started; t < nt; ++t) work(c0 + ncols * t / nt, c0 + ncols * (t + 1) / nt);
    for (auto& x : th) x.join();
}

// Panel order for a budget: t x t triangular block plus at least 64 vectors of t.
int64_t panel_order(int64_t n, size_t budget)
{
    const double usable = (double)budget * 0.45;  // the block and one chunk of right-hand sides
    int64_t t = (int64_t)(std::sqrt(usable / 8.0)) / kSmall * kSmall;
    t = std::min<int64_t>(t, 1024);
    if (t < kSmall) t = kSmall;
    return std::min<int64_t>(t, n);
}

// The left-looking out-of-core TRSM of ooc_dtrsm in the driver's arena (also
// the U12 solve of the LU driver).  Arguments as for ooc_dtrsm, already checked.
int trsm_run(Driver& dr, bool left, char uplo, char transA, char diag, int64_t M, int64_t N, double alpha,
             const double* A, int64_t lda, double* B, int64_t ldb)
{
    std::string why;
    int rc = OOC_OK;
    const int64_t n = left ? M : N;
    const int64_t t = panel_order(n, dr.bytes);
    const int64_t ldt = round_up64(t, 16);
    const bool trans = is_t(transA), unit = is_u(diag);
    const bool op_lower = is_l(uplo) != trans;
    const bool forward = left ? op_lower : !op_lower;  // the coupled unknowns come first
    double* dT = reinterpret_cast<double*>(dr.arena + 256);
    double* dP = dT + t * ldt;
    const size_t p_bytes = dr.bytes - 256 - (size_t)(t * ldt * 8);
    const int64_t np = (n + t - 1) / t;
    for (int64_t q = 0; q < np; ++q) {
        const int64_t k = forward ? q : np - 1 - q;
        const int64_t r0 = k * t, tk = std::min(t, n - r0);
        // the unknowns already solved: [0, r0) going forward, [r0 + tk, n) going backward
        const int64_t s0 = forward ? 0 : r0 + tk, ks = forward ? r0 : n - (r0 + tk);
        if (ks > 0) {
            // panel -= op(A)[panel, solved] X[solved] (side L), X[:, solved] op(A)[solved, panel] (side R);
            // beta = alpha applies the scale of the right-hand side once, here
            if (left)
                rc = dr.gemm(trans ? 'T' : 'N', 'N', tk, N, ks, -1.0, trans ? A + s0 * lda + r0 : A + r0 * lda + s0,
                             lda, B + s0 * ldb, ldb, alpha, B + r0 * ldb, ldb, 0);
            else
                rc = dr.gemm('N', trans ? 'T' : 'N', M, tk, ks, -1.0, B + s0, ldb,
                             trans ? A + r0 * lda + s0 : A + s0 * lda + r0, lda, alpha, B + r0, ldb, 0);
            if (rc) return rc;
        }
        const double scale = ks > 0 ? 1.0 : alpha;
        // the triangular block A_kk (as stored) and the panel in chunks of right-hand sides
        if ((rc = dr.copy_in(dT, ldt, A + r0 * lda + r0, lda, tk, tk))) return rc;
        const int64_t lp = round_up64(left ? 1 : tk, 16);  // leading dimension of a right-side chunk
        const int64_t nv_total = left ? N : M;
        const int64_t chunk = chunk_and_scratch(dr, reinterpret_cast<char*>(dP), p_bytes, tk, !left, nv_total);
        for (int64_t v0 = 0; v0 < nv_total; v0 += chunk) {
            const int64_t nv = std::min(chunk, nv_total - v0);
            const int64_t ldp = left ? round_up64(nv, 16) : lp;
            double* hP = left ? B + r0 * ldb + v0 : B + v0 * ldb + r0;
            const int64_t rows = left ? tk : nv, cols = left ? nv : tk;
            if ((rc = dr.copy_in(dP, ldp, hP, ldb, rows, cols))) return rc;
            if (scale != 1.0) {
                scale_kernel<<<1024, 256, 0, dr.d.st>>>(dP, ldp, rows, cols, scale);
                ++dr.d.launches;
                if ((rc = check_launch("scale_kernel", why))) return fail(rc, why);
            }
            if ((rc = incore_trsm(left, op_lower, dT, ldt, trans, unit, tk, dP, ldp, nv, dr.d, why)))
                return fail(rc, why);
            if ((rc = dr.copy_out(hP, ldb, dP, ldp, rows, cols))) return rc;
            if ((rc = dr.drain())) return rc;
        }
    }
    return OOC_OK;
}

}  // namespace

}  // namespace ooc

using namespace ooc;

int ooc_dtrsm(char side, char uplo, char transA, char diag, int64_t M, int64_t N, double alpha, const double* A,
              int64_t lda, double* B, int64_t ldb, size_t device_budget_bytes, const ooc_opts* opts,
              ooc_stats* stats)
{
    if (stats) std::memset(stats, 0, sizeof(*stats));
    if (!(is_l(side) || is_r(side)) || !(is_l(uplo) || is_u(uplo)) || !(is_n(transA) || is_t(transA)) ||
        !(is_n(diag) || is_u(diag)))
        return fail(OOC_ERR_INVALID_ARG, "side, uplo, transA or diag out of range");
    if (M < 0 || N < 0) return fail(OOC_ERR_INVALID_ARG, "negative dimension");
    const bool left = is_l(side);
    const int64_t n = left ? M : N;  // order of A
    if (lda < std::max<int64_t>(1, n) || ldb < std::max<int64_t>(1, N))
        return fail(OOC_ERR_INVALID_ARG, "leading dimension below the row width");
    if (M == 0 || N == 0) return OOC_OK;
    if (!A || !B) return fail(OOC_ERR_INVALID_ARG, "null operand pointer");
    std::string why;
    int rc = device_check(why);
    if (rc) return fail(rc, why);
    if (!host_range_pinned(A, n, n, lda, 8) || !host_range_pinned(B, M, N, ldb, 8))
        return fail(OOC_ERR_NOT_PINNED, "host operands must be page-locked (cudaHostAlloc / cudaHostRegister)");
    const int64_t t = panel_order(n, device_budget_bytes);
    const int64_t ldt = round_up64(t, 16);
    if ((size_t)(t * ldt * 8 + 256 + 64 * ldt * 8 + 4096) > device_budget_bytes)
        return fail(OOC_ERR_BUDGET, "budget below one 64 x 64 triangular block and its right-hand sides");
    Driver dr;
    if ((rc = dr.init(device_budget_bytes, opts, why))) return fail(rc, why);
    if (alpha == 0.0) {
        // X = 0 without reading B (the BLAS rule for alpha == 0)
        for (int64_t r = 0; r < M; ++r) std::memset(B + r * ldb, 0, (size_t)N * 8);
        dr.finish(stats, 0.0);
        return OOC_OK;
    }
    if ((rc = trsm_run(dr, left, uplo, transA, diag, M, N, alpha, A, lda, B, ldb))) return rc;
    dr.finish(stats, left ? (double)M * M * N : (double)M * N * N);
    return OOC_OK;
}

int ooc_dpotrf(char uplo, int64_t N, double* A, int64_t lda, size_t device_budget_bytes, const ooc_opts* opts,
               ooc_stats* stats, int64_t* info)
{
    if (stats) std::memset(stats, 0, sizeof(*stats));
    if (info) *info = 0;
    if (!(is_l(uplo) || is_u(uplo))) return fail(OOC_ERR_INVALID_ARG, "uplo must be 'L' or 'U'");
    if (N < 0 || lda < std::max<int64_t>(1, N)) return fail(OOC_ERR_INVALID_ARG, "bad order or leading dimension");
    if (N == 0) return OOC_OK;
    if (!A || !info) return fail(OOC_ERR_INVALID_ARG, "null matrix or info pointer");
    std::string why;
    int rc = device_check(why);
    if (rc) return fail(rc, why);
    if (!host_range_pinned(A, N, N, lda, 8))
        return fail(OOC_ERR_NOT_PINNED, "host operands must be page-locked (cudaHostAlloc / cudaHostRegister)");
    const int64_t t = panel_order(N, device_budget_bytes);
    const int64_t ldt = round_up64(t, 16);
    if ((size_t)(t * ldt * 8 + 256 + 64 * ldt * 8 + 4096) > device_budget_bytes)
        return fail(OOC_ERR_BUDGET, "budget below one 64 x 64 diagonal block and its panel rows");
    Driver dr;
    if ((rc = dr.init(device_budget_bytes, opts, why))) return fail(rc, why);
    const bool upper = is_u(uplo);
    double* dT = reinterpret_cast<double*>(dr.arena + 256);
    double* dP = dT + t * ldt;
    const size_t p_bytes = dr.bytes - 256 - (size_t)(t * ldt * 8);
    for (int64_t c0 = 0; c0 < N; c0 += t) {
        const int64_t tk = std::min(t, N - c0), rest = N - c0;
        if (c0 > 0) {
            // panel -= L[c0:, 0:c0] L[c0:c0+tk, 0:c0]^T on the lower triangle (upper: the transposed form)
            if (!upper)
                rc = dr.gemm('N', 'T', rest, tk, c0, -1.0, A + c0 * lda, lda, A + c0 * lda, lda, 1.0,
                             A + c0 * lda + c0, lda, 1);
            else
                rc = dr.gemm('T', 'N', tk, rest, c0, -1.0, A + c0, lda, A + c0, lda, 1.0, A + c0 * lda + c0, lda, 2);
            if (rc) return rc;
        }
        // right-hand-side chunks of the panel below (and the Ozaki scratch, also used by the diagonal block)
        const int64_t nv_total = rest - tk;
        const int64_t lp = round_up64(tk, 16);
        const int64_t chunk = chunk_and_scratch(dr, reinterpret_cast<char*>(dP), p_bytes, tk, !upper, nv_total);
        // factor the diagonal block
        double* hD = A + c0 * lda + c0;
        if ((rc = dr.copy_in(dT, ldt, hD, lda, tk, tk))) return rc;
        if ((rc = incore_potrf(upper, dT, ldt, tk, c0, dr.d, why))) return fail(rc, why);
        if ((rc = dr.copy_out(hD, lda, dT, ldt, tk, tk))) return rc;
        if ((rc = dr.drain())) return rc;
        unsigned long long hinfo = 0;
        if (cudaMemcpy(&hinfo, dr.d.info, sizeof(hinfo), cudaMemcpyDeviceToHost) != cudaSuccess)
            return fail(OOC_ERR_CUDA, "pivot word read failed");
        if (hinfo) {
            *info = (int64_t)hinfo;
            dr.finish(stats, 0.0);
            return OOC_OK;
        }
        // the rest of the panel: X L11^T = P (lower) or U11^T X = P (upper), in chunks
        for (int64_t v0 = 0; v0 < nv_total; v0 += chunk) {
            const int64_t nv = std::min(chunk, nv_total - v0);
            double* hP = upper ? A + c0 * lda + c0 + tk + v0 : A + (c0 + tk + v0) * lda + c0;
            const int64_t ldp = upper ? round_up64(nv, 16) : lp;
            const int64_t rows = upper ? tk : nv, cols = upper ? nv : tk;
            if ((rc = dr.copy_in(dP, ldp, hP, lda, rows, cols))) return rc;
            // stored L11 read transposed is upper (right solve); stored U11 read transposed is lower (left solve)
            if ((rc = incore_trsm(upper, upper, dT, ldt, true, false, tk, dP, ldp, nv, dr.d, why)))
                return fail(rc, why);
            if ((rc = dr.copy_out(hP, lda, dP, ldp, rows, cols))) return rc;
            if ((rc = dr.drain())) return rc;
        }
    }
    dr.finish(stats, (double)N * N * N / 3.0);
    return OOC_OK;
}

int ooc_dgetrf(int64_t N, double* A, int64_t lda, int64_t* ipiv, size_t device_budget_bytes, const ooc_opts* opts,
               ooc_stats* stats, int64_t* info)
{
    if (stats) std::memset(stats, 0, sizeof(*stats));
    if (info) *info = 0;
    if (N < 0 || lda < std::max<int64_t>(1, N)) return fail(OOC_ERR_INVALID_ARG, "bad order or leading dimension");
    if (N == 0) return OOC_OK;
    if (!A || !ipiv || !info) return fail(OOC_ERR_INVALID_ARG, "null matrix, pivot or info pointer");
    std::string why;
    int rc = device_check(why);
    if (rc) return fail(rc, why);
    if (!host_range_pinned(A, N, N, lda, 8))
        return fail(OOC_ERR_NOT_PINNED, "host operands must be page-locked (cudaHostAlloc / cudaHostRegister)");
    // panel width: the whole N x t panel, its pivots and the candidates in the arena
    if (cudaFuncSetAttribute(narrow_lu_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLuSmemMax) !=
        cudaSuccess) {
        cudaGetLastError();
        return fail(OOC_ERR_CUDA, "narrow_lu_kernel shared-memory attribute");
    }
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, narrow_lu_kernel<false>, kLuThreads, 0);
    // panel kernel grid: co-resident, at most two CTAs per SM and one per 32 rows of the tallest panel
    const int lu_grid =
        (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)occ * device_sm_count(), 304, (N + 31) / 32}));
    // its scratch: candidate values and rows (two buffers each), the published row j
    const size_t lu_scratch = (size_t)lu_grid * 2 * (8 + 8 + kSmall * 8) + 2 * kSmall * 8;
    const size_t fixed = 256 + 4096 + lu_scratch + 8 * 1024;
    auto panel_bytes = [&](int64_t w) { return (size_t)N * round_up64(w, 16) * 8; };
    const bool oz = opts && opts->form == OOC_FORM_OZAKI;
    const int oz_s = oz && opts->slices > 0 ? opts->slices : kOzakiSlicesFactor;
    auto oz_of = [&](int64_t w) { return oz ? ozaki_device_scratch(N, w, w, oz_s) + 256 : (size_t)0; };
    auto too_big = [&](int64_t w) {
        return fixed + panel_bytes(w) + oz_of(w) + (size_t)64 * round_up64(w, 16) * 8 + 512 > device_budget_bytes ||
               (size_t)(w * round_up64(w, 16) * 8 + 256 + 64 * 8 * round_up64(w, 16) + 4096) > device_budget_bytes;
    };
    // N itself when it fits (up to 1024), else the largest multiple of 64 that fits
    int64_t t = N <= 1024 ? N : 1024;
    while (t > kSmall && too_big(t)) t = (t - 1) / kSmall * kSmall;
    if (too_big(t)) return fail(OOC_ERR_BUDGET, "budget below one N x 64 panel");
    const size_t oz_bytes = oz_of(t) ? oz_of(t) - 256 : 0;
    Driver dr;
    if ((rc = dr.init(device_budget_bytes, opts, why))) return fail(rc, why);
    const int64_t ldp = round_up64(t, 16);
    double* dP = reinterpret_cast<double*>(dr.arena + 256);
    char* after = dr.arena + 256 + panel_bytes(t);
    int64_t* dpiv = reinterpret_cast<int64_t*>(after);
    char* lu = after + 8 * 1024;
    dr.d.cand_v = reinterpret_cast<double*>(lu);
    dr.d.cand_i = reinterpret_cast<int64_t*>(lu + (size_t)lu_grid * 16);
    dr.d.cand_row = reinterpret_cast<double*>(lu + (size_t)lu_grid * 32);
    dr.d.jrow = reinterpret_cast<double*>(lu + (size_t)lu_grid * 32 + (size_t)lu_grid * 2 * kSmall * 8);
    dr.d.bar = reinterpret_cast<unsigned*>(dr.arena + 16);
    dr.d.lu_grid = lu_grid;
    // OOC_LU_ROWS_GLOBAL=1: the panel kernel keeps its rows in global memory, the path taken
    // when a co-resident grid's row slices do not fit shared memory (tests use it on small panels)
    if (const char* g = std::getenv("OOC_LU_ROWS_GLOBAL")) dr.d.lu_rows_global = std::atoi(g) != 0;
    std::vector<int64_t> hpiv((size_t)t);
    // Ozaki updates: digit-plane scratch for the panel's largest in-HBM update (rows N, order t),
    // then the U12 row panel in column chunks
    size_t used = (256 + panel_bytes(t) + 8 * 1024 + lu_scratch + 255) / 256 * 256;
    if (oz_bytes) {
        dr.d.oz = dr.arena + used;
        dr.d.oz_bytes = oz_bytes;
        used += (oz_bytes + 255) / 256 * 256;
    }
    const size_t u_bytes = dr.bytes > used ? dr.bytes - used : 0;
    double* dU = reinterpret_cast<double*>(dr.arena + used);
    const int64_t u_chunk = std::max<int64_t>(16, (int64_t)(u_bytes / (8 * (size_t)round_up64(t, 16)) / 16 * 16) - 16);
    // OOC_TRACE=<file>: one line per panel with the host time of each phase (ms)
    std::unique_ptr<FILE, int (*)(FILE*)> trace_file(nullptr, std::fclose);
    if (const char* tp = std::getenv("OOC_TRACE")) trace_file.reset(std::fopen(tp, "a"));
    FILE* trace = trace_file.get();
    if (trace) std::fprintf(trace, "# getrf N=%lld t=%lld: c0,panel,laswp,u12,gemm\n", (long long)N, (long long)t);
    auto now = [] { return std::chrono::steady_clock::now(); };
    auto ms = [](std::chrono::steady_clock::time_point a, std::chrono::steady_clock::time_point b) {
        return std::chrono::duration<double, std::milli>(b - a).count();
    };
    // Right-looking over panels of t columns: every trailing update is one large
    // out-of-core GEMM (a full-occupancy output of (N - c0 - t)^2).
    for (int64_t c0 = 0; c0 < N; c0 += t) {
        const int64_t tk = std::min(t, N - c0), m = N - c0, rest = N - c0 - tk;
        const auto p0 = now();
        // 1. the panel A[c0:, c0:c0+tk] (up to date) factored in device memory
        if ((rc = dr.copy_in(dP, ldp, A + c0 * lda + c0, lda, m, tk))) return rc;
        if ((rc = panel_lu(dP, ldp, m, tk, dpiv, c0, dr.d, why))) return fail(rc, why);
        if ((rc = dr.copy_out(A + c0 * lda + c0, lda, dP, ldp, m, tk))) return rc;
        if ((rc = dr.drain())) return rc;
        if (cudaMemcpy(hpiv.data(), dpiv, (size_t)tk * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
            return fail(OOC_ERR_CUDA, "pivot read failed");
        for (int64_t q = 0; q < tk; ++q) ipiv[c0 + q] = c0 + hpiv[q];
        const auto p1 = now();
        // 2. its interchanges on every other column (L to the left, the trailing matrix to the right)
        host_laswp(A, lda, 0, c0, ipiv, c0, c0 + tk);
        host_laswp(A, lda, c0 + tk, N, ipiv, c0, c0 + tk);
        const auto p2 = now();
        // 3. U12 = L11^{-1} A12 in device memory, L11 still in the panel buffer, A12 in column chunks
        for (int64_t v0 = 0; v0 < rest; v0 += u_chunk) {
            const int64_t nv = std::min(u_chunk, rest - v0);
            const int64_t ldu = round_up64(nv, 16);
            double* hU = A + c0 * lda + c0 + tk + v0;
            if ((rc = dr.copy_in(dU, ldu, hU, lda, tk, nv))) return rc;
            if ((rc = incore_trsm(true, true, dP, ldp, false, true, tk, dU, ldu, nv, dr.d, why))) return fail(rc, why);
            if ((rc = dr.copy_out(hU, lda, dU, ldu, tk, nv))) return rc;
            if ((rc = dr.drain())) return rc;
        }
        const auto p3 = now();
        // 4. A22 -= L21 U12 over the trailing matrix, out of core
        if (rest > 0 &&
            (rc = dr.gemm('N', 'N', rest, rest, tk, -1.0, A + (c0 + tk) * lda + c0, lda, A + c0 * lda + c0 + tk, lda,
                          1.0, A + (c0 + tk) * lda + c0 + tk, lda, 0)))
            return rc;
        const auto p4 = now();
        if (trace)
            std::fprintf(trace, "%lld,%.2f,%.2f,%.2f,%.2f\n", (long long)c0, ms(p0, p1), ms(p1, p2), ms(p2, p3),
                         ms(p3, p4));
    }
    trace_file.reset();
    unsigned long long hinfo = 0;
    if (cudaMemcpy(&hinfo, dr.d.info, sizeof(hinfo), cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(OOC_ERR_CUDA, "pivot word read failed");
    *info = (int64_t)hinfo;
    dr.finish(stats, 2.0 * (double)N * N * N / 3.0);
    return OOC_OK;
}
