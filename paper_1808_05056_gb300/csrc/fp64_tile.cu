// Plain FP64 tile contraction for sm_103a: the compute stage of the Section IV
// pipeline (its per-block update c_ij = alpha a_i b_j + beta c_ij) on the FP64
// tensor-core MMA (mma.sync m8n8k4 .f64), fed by TMA tile loads.
//
// Shape: CTA tile 64 x 64, K step 16, a 4-stage ring of TMA-filled shared
// memory stages guarded by full/empty mbarriers.  Warp 4 is the producer (one
// elected lane issues the tensor copies); warps 0-3 each own a 32 x 32 part of
// the tile as 4 x 4 MMA fragments in registers.  The grid is persistent: each
// CTA walks tiles blockIdx.x, blockIdx.x + gridDim.x, ... with the stage ring
// running on across tile boundaries, so the copies of the next tile overlap
// the epilogue of the current one.  Ragged edges come from the tensor maps:
// reads outside the operand are zero-filled by TMA and the epilogue masks
// stores.
//
// GB300 has a small FP64 rate, so this kernel is bound by the FP64 pipe; the
// 64 x 64 tile keeps wave quantisation low on large blocks.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "device_sync.cuh"
#include "ooc_internal.hpp"

namespace ooc {

namespace {

constexpr int BM = 64, BN = 64, BK = 16, STAGES = 4;
constexpr int CONSUMER_WARPS = 4;
constexpr int THREADS = (CONSUMER_WARPS + 1) * 32;
constexpr int STAGE_A = BM * BK;  // doubles
constexpr int STAGE_B = BN * BK;
constexpr uint32_t STAGE_BYTES = (STAGE_A + STAGE_B) * 8;
constexpr size_t SMEM_BYTES = (size_t)STAGES * STAGE_BYTES + 2 * STAGES * sizeof(uint64_t) + 1024;

struct Fp64Args {
    int64_t M, N, K;
    int64_t tiles_n, tiles;
    double alpha, beta;
    int read_c;
    double* C;
    int64_t ldc;
    int* err;
};

__device__ __forceinline__ void dmma_8x8x4(double& d0, double& d1, double a, double b)
{
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                 : "+d"(d0), "+d"(d1)
                 : "d"(a), "d"(b));
}

template <bool A_KMAJOR, bool B_KMAJOR>
__global__ void __launch_bounds__(THREADS) fp64_tile_kernel(const __grid_constant__ CUtensorMap tmA,
                                                            const __grid_constant__ CUtensorMap tmB,
                                                            Fp64Args p)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte alignment of the stage ring
    unsigned char* base = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    double* stages = reinterpret_cast<double*>(base);
    uint64_t* full = reinterpret_cast<uint64_t*>(base + STAGES * STAGE_BYTES);
    uint64_t* empty = full + STAGES;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], CONSUMER_WARPS);
        }
        mbar_fence_init();
    }
    __syncthreads();

    const int64_t nk = (p.K + BK - 1) / BK;
    const int64_t my_tiles = p.tiles > blockIdx.x ? (p.tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const int64_t total = my_tiles * nk;

    if (warp == CONSUMER_WARPS) {
        // ---------------- producer ----------------
        if (lane == 0 && total > 0) {
            tma_prefetch_desc(&tmA);
            tma_prefetch_desc(&tmB);
            int64_t it = 0;
            bool ok = true;
            for (; it < total; ++it) {
                const int s = (int)(it % STAGES);
                const uint32_t ph = (uint32_t)((it / STAGES) & 1);
                if (!mbar_wait(&empty[s], ph ^ 1u, p.err, kErrWaitEmpty)) { ok = false; break; }
                const int64_t tl = it / nk, ks = it % nk;
                const int64_t tile = blockIdx.x + tl * gridDim.x;
                const int32_t tm = (int32_t)(tile / p.tiles_n), tn = (int32_t)(tile % p.tiles_n);
                double* sA = stages + (size_t)s * (STAGE_A + STAGE_B);
                double* sB = sA + STAGE_A;
                mbar_arrive_expect_tx(&full[s], STAGE_BYTES);
                const int32_t k0 = (int32_t)(ks * BK);
                if (A_KMAJOR) tma_load_2d(sA, &tmA, &full[s], k0, tm * BM);
                else tma_load_2d(sA, &tmA, &full[s], tm * BM, k0);
                if (B_KMAJOR) tma_load_2d(sB, &tmB, &full[s], k0, tn * BN);
                else tma_load_2d(sB, &tmB, &full[s], tn * BN, k0);
            }
            if (!ok) {
                // let the copies already issued land before the CTA exits
                for (int64_t q = (it > STAGES ? it - STAGES : 0); q < it; ++q) {
                    const int s = (int)(q % STAGES);
                    const uint64_t t0 = globaltimer_ns();
                    while (!mbar_try_wait(smem_u32(&full[s]), (uint32_t)((q / STAGES) & 1)) &&
                           globaltimer_ns() - t0 < kWaitLimitNs) {
                    }
                }
            }
        }
        return;
    }

    // ---------------- consumers ----------------
    const int wm = warp >> 1, wn = warp & 1;  // 2 x 2 warps of 32 x 32
    const int fr = lane >> 2, fc = lane & 3;  // fragment row / column of this lane
    double acc[4][4][2];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b][0] = acc[a][b][1] = 0.0;

    auto epilogue = [&](int64_t tile) {
        const int64_t tm = tile / p.tiles_n, tn = tile % p.tiles_n;
#pragma unroll
        for (int mi = 0; mi < 4; ++mi) {
            const int64_t row = tm * BM + wm * 32 + mi * 8 + fr;
#pragma unroll
            for (int ni = 0; ni < 4; ++ni) {
                const int64_t col = tn * BN + wn * 32 + ni * 8 + fc * 2;
                if (row < p.M) {
                    double* c = p.C + row * p.ldc + col;
                    if (col + 1 < p.N) {
                        double2 v;
                        v.x = p.alpha * acc[mi][ni][0];
                        v.y = p.alpha * acc[mi][ni][1];
                        if (p.read_c) {
                            const double2 o = *reinterpret_cast<const double2*>(c);
                            v.x += p.beta * o.x;
                            v.y += p.beta * o.y;
                        }
                        *reinterpret_cast<double2*>(c) = v;
                    } else if (col < p.N) {
                        double v = p.alpha * acc[mi][ni][0];
                        if (p.read_c) v += p.beta * c[0];
                        c[0] = v;
                    }
                }
                acc[mi][ni][0] = acc[mi][ni][1] = 0.0;
            }
        }
    };

    if (nk == 0) {  // K == 0: C = beta * C (or 0)
        for (int64_t tl = 0; tl < my_tiles; ++tl) epilogue(blockIdx.x + tl * gridDim.x);
        return;
    }

    for (int64_t it = 0; it < total; ++it) {
        const int s = (int)(it % STAGES);
        if (!mbar_wait(&full[s], (uint32_t)((it / STAGES) & 1), p.err, kErrWaitFull)) return;
        const double* sA = stages + (size_t)s * (STAGE_A + STAGE_B);
        const double* sB = sA + STAGE_A;
#pragma unroll
        for (int kk = 0; kk < BK; kk += 4) {
            double af[4], bf[4];
#pragma unroll
            for (int mi = 0; mi < 4; ++mi) {
                const int r = wm * 32 + mi * 8 + fr, k = kk + fc;
                af[mi] = A_KMAJOR ? sA[r * BK + k] : sA[k * BM + r];
            }
#pragma unroll
            for (int ni = 0; ni < 4; ++ni) {
                const int n = wn * 32 + ni * 8 + fr, k = kk + fc;
                bf[ni] = B_KMAJOR ? sB[n * BK + k] : sB[k * BN + n];
            }
#pragma unroll
            for (int mi = 0; mi < 4; ++mi)
#pragma unroll
                for (int ni = 0; ni < 4; ++ni) dmma_8x8x4(acc[mi][ni][0], acc[mi][ni][1], af[mi], bf[ni]);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
        if (it % nk == nk - 1) epilogue(blockIdx.x + (it / nk) * gridDim.x);
    }
}

template <bool AK, bool BKM>
int launch_variant(const CUtensorMap& ma, const CUtensorMap& mb, const Fp64Args& a, cudaStream_t st,
                   std::string& why)
{
    static int occ = 0, sms = 0;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaFuncSetAttribute(fp64_tile_kernel<AK, BKM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)SMEM_BYTES);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fp64_tile_kernel<AK, BKM>, THREADS, SMEM_BYTES);
        sms = device_sm_count();
    });
    if (occ <= 0) {
        why = "fp64 tile kernel cannot be resident (occupancy 0)";
        return OOC_ERR_CUDA;
    }
    const int64_t grid = std::min<int64_t>(a.tiles > 0 ? a.tiles : 1, (int64_t)occ * sms);
    fp64_tile_kernel<AK, BKM><<<(unsigned)grid, THREADS, SMEM_BYTES, st>>>(ma, mb, a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        why = std::string("fp64 tile launch: ") + cudaGetErrorString(e);
        return OOC_ERR_CUDA;
    }
    return OOC_OK;
}

}  // namespace

int launch_fp64_tile(bool a_kmajor, bool b_kmajor, int64_t M, int64_t N, int64_t K, double alpha,
                     const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
                     bool read_c, double* C, int64_t ldc, int* err, void* stream, std::string& why)
{
    if (M <= 0 || N <= 0) return OOC_OK;
    CUtensorMap ma, mbm;
    std::memset(&ma, 0, sizeof(ma));
    std::memset(&mbm, 0, sizeof(mbm));
    if (K > 0) {
        int rc = a_kmajor ? encode_map_2d(&ma, 0, A, (uint64_t)K, (uint64_t)M, (uint64_t)lda, BK, BM, 0, why)
                          : encode_map_2d(&ma, 0, A, (uint64_t)M, (uint64_t)K, (uint64_t)lda, BM, BK, 0, why);
        if (rc != OOC_OK) return rc;
        rc = b_kmajor ? encode_map_2d(&mbm, 0, B, (uint64_t)K, (uint64_t)N, (uint64_t)ldb, BK, BN, 0, why)
                      : encode_map_2d(&mbm, 0, B, (uint64_t)N, (uint64_t)K, (uint64_t)ldb, BN, BK, 0, why);
        if (rc != OOC_OK) return rc;
    }
    Fp64Args a;
    a.M = M; a.N = N; a.K = K;
    a.tiles_n = (N + BN - 1) / BN;
    a.tiles = ((M + BM - 1) / BM) * a.tiles_n;
    a.alpha = alpha; a.beta = beta; a.read_c = read_c ? 1 : 0;
    a.C = C; a.ldc = ldc; a.err = err;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (a_kmajor && b_kmajor) return launch_variant<true, true>(ma, mbm, a, st, why);
    if (a_kmajor && !b_kmajor) return launch_variant<true, false>(ma, mbm, a, st, why);
    if (!a_kmajor && b_kmajor) return launch_variant<false, true>(ma, mbm, a, st, why);
    return launch_variant<false, false>(ma, mbm, a, st, why);
}

}  // namespace ooc
