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
// the epilogue of the current one (tiles are taken in a grouped raster order,
// see tile_of).  Ragged edges come from the tensor maps:
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

// Tiles of a triangular update (GEMMT / SYRK blocks that straddle the
// diagonal).  With square tiles of side T, tile (tm, tn) holds an element with
// col - row <= off (lower) iff tn - tm <= floor((off + T - 1) / T), and one
// with col - row >= off (upper) iff tn - tm >= ceil((off - T + 1) / T).  So
// the kept tiles of tile row tm are one run of columns whose length is
//   lower: clamp(tm + a, 0, tiles_n), starting at column 0,
//   upper: clamp(a - tm, 0, tiles_n), ending at the last column,
// and the run lengths have closed-form prefix sums, which map a kept-tile
// index to its (tm, tn) by a binary search over tile rows.
struct TriTiles {
    int mode;  // 0 every tile, 1 lower, 2 upper
    int64_t a, tiles_m, tiles_n;
};

__host__ __device__ inline int64_t clamp64(int64_t v, int64_t lo, int64_t hi) { return v < lo ? lo : (v > hi ? hi : v); }
__host__ __device__ inline int64_t floor_div(int64_t a, int64_t b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

__host__ __device__ inline int64_t tri_run(const TriTiles& t, int64_t tm)
{
    return t.mode == 1 ? clamp64(tm + t.a, 0, t.tiles_n) : clamp64(t.a - tm, 0, t.tiles_n);
}

// number of kept tiles in tile rows [0, x)
__host__ __device__ inline int64_t tri_prefix(const TriTiles& t, int64_t x)
{
    const int64_t T = t.tiles_n, a = t.a;
    if (t.mode == 1) {
        const int64_t z = clamp64(1 - a, 0, x);    // rows before z keep no tile
        const int64_t s = clamp64(T - a, z, x);    // rows from s on keep all T
        const int64_t n = s - z;
        return n * (z + s - 1) / 2 + n * a + (x - s) * T;
    }
    const int64_t s = clamp64(a - T + 1, 0, x);    // rows before s keep all T
    const int64_t z = clamp64(a, s, x);            // rows from z on keep none
    const int64_t n = z - s;
    return s * T + n * a - n * (s + z - 1) / 2;
}

__host__ __device__ inline TriTiles tri_tiles(int mode, int64_t off, int64_t tiles_m, int64_t tiles_n, int64_t T)
{
    TriTiles t{mode, 0, tiles_m, tiles_n};
    if (mode == 1) t.a = floor_div(off + T - 1, T) + 1;
    else if (mode == 2) t.a = tiles_n + floor_div(-(off - T + 1), T);  // tiles_n - ceil((off - T + 1) / T)
    return t;
}

struct Fp64Args {
    int64_t M, N, K;
    int64_t tiles_n, tiles;
    double alpha, beta;
    int read_c;
    double* C;
    int64_t ldc;
    int* err;
    int tri;          // 0 full update, 1 lower (col - row <= tri_off), 2 upper (col - row >= tri_off)
    int64_t tri_off;
    TriTiles tt;
};

// Tile order of a full update: groups of kRasterRows tile rows, column-major
// inside a group, so that the ~456 tiles in flight span 16 rows and ~29
// columns and re-read their A and B tiles from L2 rather than DRAM.
constexpr int64_t kRasterRows = 16;

__device__ __forceinline__ void tile_of(const Fp64Args& p, int64_t tile, int64_t& tm, int64_t& tn)
{
    if (p.tri == 0) {
        const int64_t tiles_m = p.tiles / p.tiles_n;
        const int64_t per_group = kRasterRows * p.tiles_n;
        const int64_t g = tile / per_group, r = tile % per_group;
        const int64_t first = g * kRasterRows;
        const int64_t rows = tiles_m - first < kRasterRows ? tiles_m - first : kRasterRows;
        tm = first + r % rows;
        tn = r / rows;
        return;
    }
    int64_t lo = 0, hi = p.tt.tiles_m - 1;  // largest tm with prefix(tm) <= tile
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (tri_prefix(p.tt, mid) <= tile) lo = mid;
        else hi = mid - 1;
    }
    tm = lo;
    const int64_t first = p.tri == 1 ? 0 : p.tiles_n - tri_run(p.tt, lo);
    tn = first + (tile - tri_prefix(p.tt, lo));
}

__device__ __forceinline__ bool kept(const Fp64Args& p, int64_t row, int64_t col)
{
    return p.tri == 0 || (p.tri == 1 ? col - row <= p.tri_off : col - row >= p.tri_off);
}

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
                int64_t tm64, tn64;
                tile_of(p, tile, tm64, tn64);
                const int32_t tm = (int32_t)tm64, tn = (int32_t)tn64;
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
        int64_t tm, tn;
        tile_of(p, tile, tm, tn);
#pragma unroll
        for (int mi = 0; mi < 4; ++mi) {
            const int64_t row = tm * BM + wm * 32 + mi * 8 + fr;
#pragma unroll
            for (int ni = 0; ni < 4; ++ni) {
                const int64_t col = tn * BN + wn * 32 + ni * 8 + fc * 2;
                if (row < p.M && p.tri != 0) {  // masked: element by element
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        if (col + e >= p.N || !kept(p, row, col + e)) continue;
                        double* c = p.C + row * p.ldc + col + e;
                        double v = p.alpha * acc[mi][ni][e];
                        if (p.read_c) v += p.beta * c[0];
                        c[0] = v;
                    }
                } else if (row < p.M) {
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

// ---------------------------------------------------------------- grouped --
// One launch over the tiles of up to kGroupMax independent problems whose
// operands are all resident (a batch of uneven GEMMs): the CTAs walk the
// concatenated list of (problem, tile) items -- each problem's tiles in the
// raster order of tile_of -- with the stage ring running on across items and
// problems, so one launch's tail and pipeline fill are paid once per group of
// problems instead of once per problem.  Each problem's tensor maps live in
// the kernel parameters (no device-side descriptor copy, so the launch can be
// captured in a CUDA graph).
struct GroupProb {
    CUtensorMap ma, mb;
    double* C;
    int64_t ldc, M, N, K;
    int64_t tiles_n, tile_begin;  // tiles per row of tiles; first item of this problem
    double alpha, beta;
    int read_c, pad;
};

struct GroupArgs {
    int count;
    int64_t tiles;  // items in all problems
    int* err;
    GroupProb p[kGroupMax];
};

// the problem holding item t (tile_begin ascending, first entry 0)
__device__ __forceinline__ int group_problem(const GroupArgs& g, int64_t t)
{
    int lo = 0, hi = g.count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (g.p[mid].tile_begin <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ void group_tile(const GroupProb& q, int64_t t, int64_t& tm, int64_t& tn)
{
    const int64_t local = t - q.tile_begin;
    const int64_t tiles_m = (q.M + BM - 1) / BM;
    const int64_t per_group = kRasterRows * q.tiles_n;
    const int64_t gr = local / per_group, r = local % per_group;
    const int64_t first = gr * kRasterRows;
    const int64_t rows = tiles_m - first < kRasterRows ? tiles_m - first : kRasterRows;
    tm = first + r % rows;
    tn = r / rows;
}

template <bool A_KMAJOR, bool B_KMAJOR>
__global__ void __launch_bounds__(THREADS) fp64_group_kernel(const __grid_constant__ GroupArgs g)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
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

    if (warp == CONSUMER_WARPS) {
        // ---------------- producer ----------------
        if (lane != 0) return;
        int64_t it = 0;  // stages issued so far (ring position)
        bool ok = true;
        for (int64_t t = blockIdx.x; t < g.tiles && ok; t += gridDim.x) {
            const GroupProb& q = g.p[group_problem(g, t)];
            int64_t tm64, tn64;
            group_tile(q, t, tm64, tn64);
            const int32_t tm = (int32_t)tm64, tn = (int32_t)tn64;
            const int64_t nk = (q.K + BK - 1) / BK;
            for (int64_t ks = 0; ks < nk; ++ks, ++it) {
                const int s = (int)(it % STAGES);
                if (!mbar_wait(&empty[s], (uint32_t)((it / STAGES) & 1) ^ 1u, g.err, kErrWaitEmpty)) {
                    ok = false;
                    break;
                }
                double* sA = stages + (size_t)s * (STAGE_A + STAGE_B);
                double* sB = sA + STAGE_A;
                mbar_arrive_expect_tx(&full[s], STAGE_BYTES);
                const int32_t k0 = (int32_t)(ks * BK);
                if (A_KMAJOR) tma_load_2d(sA, &q.ma, &full[s], k0, tm * BM);
                else tma_load_2d(sA, &q.ma, &full[s], tm * BM, k0);
                if (B_KMAJOR) tma_load_2d(sB, &q.mb, &full[s], k0, tn * BN);
                else tma_load_2d(sB, &q.mb, &full[s], tn * BN, k0);
            }
        }
        if (!ok) {
            // let the copies already issued land before the CTA exits
            for (int64_t w = (it > STAGES ? it - STAGES : 0); w < it; ++w) {
                const int s = (int)(w % STAGES);
                const uint64_t t0 = globaltimer_ns();
                while (!mbar_try_wait(smem_u32(&full[s]), (uint32_t)((w / STAGES) & 1)) &&
                       globaltimer_ns() - t0 < kWaitLimitNs) {
                }
            }
        }
        return;
    }

    // ---------------- consumers ----------------
    const int wm = warp >> 1, wn = warp & 1;
    const int fr = lane >> 2, fc = lane & 3;
    double acc[4][4][2];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b][0] = acc[a][b][1] = 0.0;
    int64_t it = 0;
    for (int64_t t = blockIdx.x; t < g.tiles; t += gridDim.x) {
        const GroupProb& q = g.p[group_problem(g, t)];
        const int64_t nk = (q.K + BK - 1) / BK;
        for (int64_t ks = 0; ks < nk; ++ks, ++it) {
            const int s = (int)(it % STAGES);
            if (!mbar_wait(&full[s], (uint32_t)((it / STAGES) & 1), g.err, kErrWaitFull)) return;
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
        }
        // epilogue of item t: C = alpha acc + beta C (K == 0: beta C)
        int64_t tm, tn;
        group_tile(q, t, tm, tn);
#pragma unroll
        for (int mi = 0; mi < 4; ++mi) {
            const int64_t row = tm * BM + wm * 32 + mi * 8 + fr;
#pragma unroll
            for (int ni = 0; ni < 4; ++ni) {
                const int64_t col = tn * BN + wn * 32 + ni * 8 + fc * 2;
                if (row < q.M) {
                    double* c = q.C + row * q.ldc + col;
                    if (col + 1 < q.N) {
                        double2 v;
                        v.x = q.alpha * acc[mi][ni][0];
                        v.y = q.alpha * acc[mi][ni][1];
                        if (q.read_c) {
                            const double2 o = *reinterpret_cast<const double2*>(c);
                            v.x += q.beta * o.x;
                            v.y += q.beta * o.y;
                        }
                        *reinterpret_cast<double2*>(c) = v;
                    } else if (col < q.N) {
                        double v = q.alpha * acc[mi][ni][0];
                        if (q.read_c) v += q.beta * c[0];
                        c[0] = v;
                    }
                }
                acc[mi][ni][0] = acc[mi][ni][1] = 0.0;
            }
        }
    }
}

template <bool AK, bool BKM>
int launch_group_variant(const GroupArgs& a, cudaStream_t st, std::string& why)
{
    static int occ = 0, sms = 0;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaFuncSetAttribute(fp64_group_kernel<AK, BKM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)SMEM_BYTES);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fp64_group_kernel<AK, BKM>, THREADS, SMEM_BYTES);
        sms = device_sm_count();
    });
    if (occ <= 0) {
        why = "fp64 group kernel cannot be resident (occupancy 0)";
        return OOC_ERR_CUDA;
    }
    const int64_t grid = std::min<int64_t>(a.tiles > 0 ? a.tiles : 1, (int64_t)occ * sms);
    fp64_group_kernel<AK, BKM><<<(unsigned)grid, THREADS, SMEM_BYTES, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        why = std::string("fp64 group launch: ") + cudaGetErrorString(e);
        return OOC_ERR_CUDA;
    }
    return OOC_OK;
}

}  // namespace

int launch_fp64_tile(bool a_kmajor, bool b_kmajor, int64_t M, int64_t N, int64_t K, double alpha,
                     const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
                     bool read_c, double* C, int64_t ldc, int* err, void* stream, std::string& why, int tri,
                     int64_t tri_off)
{
    if (M <= 0 || N <= 0) return OOC_OK;
    static_assert(BM == BN, "the triangular tile map assumes square tiles");
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
    a.tri = tri; a.tri_off = tri_off;
    a.tt = tri_tiles(tri, tri_off, (M + BM - 1) / BM, a.tiles_n, BM);
    if (tri) {
        a.tiles = tri_prefix(a.tt, a.tt.tiles_m);
        if (a.tiles == 0) return OOC_OK;  // nothing of C is updated
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (a_kmajor && b_kmajor) return launch_variant<true, true>(ma, mbm, a, st, why);
    if (a_kmajor && !b_kmajor) return launch_variant<true, false>(ma, mbm, a, st, why);
    if (!a_kmajor && b_kmajor) return launch_variant<false, true>(ma, mbm, a, st, why);
    return launch_variant<false, false>(ma, mbm, a, st, why);
}

int launch_fp64_group(bool a_kmajor, bool b_kmajor, const Fp64GroupSpec* probs, int count, int* err, void* stream,
                      std::string& why, int64_t* tiles_out)
{
    if (count <= 0 || count > kGroupMax) {
        why = "grouped launch: problem count outside 1.." + std::to_string(kGroupMax);
        return OOC_ERR_INVALID_ARG;
    }
    static GroupArgs a;  // 24 KB of kernel parameters: not on the stack
    static std::mutex mu;
    std::lock_guard<std::mutex> lk(mu);
    std::memset(&a, 0, sizeof(a));
    a.err = err;
    int n = 0;
    int64_t tiles = 0;
    for (int i = 0; i < count; ++i) {
        const Fp64GroupSpec& s = probs[i];
        if (s.M <= 0 || s.N <= 0) continue;
        GroupProb& q = a.p[n];
        if (s.K > 0) {
            int rc = a_kmajor ? encode_map_2d(&q.ma, 0, s.A, (uint64_t)s.K, (uint64_t)s.M, (uint64_t)s.lda, BK, BM, 0, why)
                              : encode_map_2d(&q.ma, 0, s.A, (uint64_t)s.M, (uint64_t)s.K, (uint64_t)s.lda, BM, BK, 0, why);
            if (rc != OOC_OK) return rc;
            rc = b_kmajor ? encode_map_2d(&q.mb, 0, s.B, (uint64_t)s.K, (uint64_t)s.N, (uint64_t)s.ldb, BK, BN, 0, why)
                          : encode_map_2d(&q.mb, 0, s.B, (uint64_t)s.N, (uint64_t)s.K, (uint64_t)s.ldb, BN, BK, 0, why);
            if (rc != OOC_OK) return rc;
        }
        q.C = s.C; q.ldc = s.ldc;
        q.M = s.M; q.N = s.N; q.K = s.K;
        q.tiles_n = (s.N + BN - 1) / BN;
        q.tile_begin = tiles;
        q.alpha = s.alpha; q.beta = s.beta; q.read_c = s.read_c ? 1 : 0;
        tiles += ((s.M + BM - 1) / BM) * q.tiles_n;
        ++n;
    }
    if (tiles_out) *tiles_out = tiles;
    if (n == 0) return OOC_OK;
    a.count = n;
    a.tiles = tiles;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (a_kmajor && b_kmajor) return launch_group_variant<true, true>(a, st, why);
    if (a_kmajor && !b_kmajor) return launch_group_variant<true, false>(a, st, why);
    if (!a_kmajor && b_kmajor) return launch_group_variant<false, true>(a, st, why);
    return launch_group_variant<false, false>(a, st, why);
}

}  // namespace ooc
