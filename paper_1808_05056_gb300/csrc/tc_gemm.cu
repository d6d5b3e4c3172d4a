// Split-product tile contraction on the 5th-generation tensor cores (sm_103a):
// the compute stage of the out-of-core pipeline for the two tensor-core forms.
//
//   BF16x3 (FP32-accurate, ooc_sgemm): each FP32 operand is split into three
//   bf16 pieces x = h + m + l (each piece the bf16 rounding of what is left),
//   and C = sum of the six products hh, hm, mh, hl, mm, lh (the dropped ml, lm,
//   ll are below 2^-24 relative).  hh and the five small products use two TMEM
//   accumulators, drained every `chunk` of K (two K blocks) into a double-float
//   FP32 pair per output with TwoSum, which keeps the tensor cores' one-ulp,
//   round-toward-zero accumulator bias far below the 1e-6 target.
//
//   Ozaki (FP64-accurate, ooc_dgemm with OOC_FORM_OZAKI), after Ozaki, Ogita,
//   Oishi and Rump's error-free splitting of matrix products: every row of A
//   (column of B) is scaled by a power of two 2^e so that its largest entry is
//   below 1 in magnitude, and its 2^-(S*beta) fixed-point value is cut into S
//   digits of beta bits, a = 2^e * sum_s d_s 2^(-beta s), |d_s| < 2^beta.  Each
//   digit plane is exact in bf16; each product of digit planes accumulates
//   exactly in FP32 over K chunks of at most 2^24 / (2^beta - 1)^2 elements;
//   the products with s + t <= S + 1 are added into FP64 with their weight
//   2^(-beta (s+t)), and the epilogue applies 2^(e_i + f_j), alpha and beta.
//
// Kernel shape (both forms): persistent CTAs, one per SM, tile 128 x 128.
//   warp 0      TMA producer: for each (tile, K chunk, group, K block of 64
//               or 32) loads the group's bf16 plane tiles (128 rows x the K
//               block, 128- or 64-byte swizzle) into a ring of stages;
//   warp 1      allocates all 512 TMEM columns (two buffers x two 128-column
//               accumulators) and issues tcgen05.mma (M=128, N=128, K=16):
//               pair 0 of the group into accumulator 0, the other pairs into
//               accumulator 1, committing stage releases and buffer-full
//               events to mbarriers;
//   warps 2-17  epilogue: read a finished accumulator with tcgen05.ld, add it
//               (times the group weight) into FP64 (Ozaki) or double-float
//               FP32 (BF16x3) registers, 32 columns per warp, release it, and
//               after the last chunk write alpha*acc*2^(e_i+f_j) + beta*C_old.
// The two buffers let the tensor cores run the next group while the epilogue
// drains the previous one.  Every wait is bounded (device_sync.cuh).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>

#include "ooc_internal.hpp"
#include "tc_common.cuh"

namespace ooc {

namespace {

constexpr int BM = 128, BN = 128;
constexpr uint32_t RING_BYTES = 192u * 1024u;       // single-CTA stage ring
constexpr uint32_t RING_BYTES_PAIR = 216u * 1024u;  // pair stage ring (three 72 KiB BF16x3 stages)
constexpr int EPI_WARPS = 16;            // 4 per TMEM lane quadrant, 32 columns each
constexpr int THREADS = (2 + EPI_WARPS) * 32;
constexpr int MAX_GROUPS = 64;
constexpr size_t SMEM_BYTES = 1024 + RING_BYTES + 1024;
constexpr size_t SMEM_BYTES_PAIR = 1024 + RING_BYTES_PAIR + 1024;

struct TcGroup {
    int8_t na, nb, np, pad0;
    int8_t aplane[4];
    int8_t bplane[4];
    int8_t pa[6];
    int8_t pb[6];
    int16_t scale_exp;   // weight of accumulator 0 (pair 0)
    int16_t scale_exp2;  // weight of accumulator 1 (pairs 1.., Ozaki)
    int16_t pad1[2];
};
static_assert(sizeof(TcGroup) == 32, "group record layout");

struct TcArgs {
    int M, N;
    int kblocks, chunk_kblocks, nchunks;
    int ngroups;
    int tiles_m, tiles_n, tiles;
    int nstages;
    uint32_t stage_bytes;
    double alpha, beta;
    int read_c, c_fp32;
    void* C;
    int64_t ldc;
    const int* row_exp;
    const int* col_exp;
    int* err;
    int tri;          // 0 full update, 1 lower (col - row <= tri_off), 2 upper (col - row >= tri_off)
    int64_t tri_off;
    TcGroup g[MAX_GROUPS];
};

// Tile order: groups of kRasterRows tile rows, column-major inside a group, so
// that the ~152 tiles in flight at once span few rows and few columns and
// share their A and B plane tiles in L2.
constexpr int kRasterRows = 8;
__device__ __forceinline__ void tile_coords(int tile, int tiles_m, int tiles_n, int& tm, int& tn)
{
    const int per_group = kRasterRows * tiles_n;
    const int g = tile / per_group, r = tile % per_group;
    const int first = g * kRasterRows;
    const int rows = min(tiles_m - first, kRasterRows);
    tm = first + r % rows;
    tn = r / rows;
}

// Exact FP32 integer x (|x| < 2^24) times 2^e as a double, built from the bit
// fields with integer operations (no conversion or multiply on the FP64 pipe).
__device__ __forceinline__ double scaled_f32_to_f64(uint32_t xb, int e)
{
    if ((xb & 0x7FFFFFFFu) == 0u) return 0.0;
    const uint64_t sign = (uint64_t)(xb >> 31) << 63;
    const uint64_t ex = (uint64_t)((int)((xb >> 23) & 0xFFu) - 127 + 1023 + e) << 52;
    const uint64_t man = (uint64_t)(xb & 0x7FFFFFu) << 29;
    return __longlong_as_double((long long)(sign | ex | man));
}

// DF32 = true (BF16x3): the first pair of a group (the leading product) and the
// other pairs use two separate TMEM accumulators, drained into an unbiased
// double-float (hi, lo) FP32 pair per output with TwoSum; the tensor cores
// round their FP32 accumulator toward zero, so each accumulator add is biased
// by up to one ulp and the leading product must not absorb the small ones.
// DF32 = false (Ozaki): each of the group's (at most two) pairs has its own
// accumulator of exact integer partial sums, drained into FP64 with its
// power-of-two weight; the two pairs share the A digit plane.
// BK: K block of one stage (64 bf16, 128-byte swizzle).
// PAIR: two CTAs of a cluster compute one 256 x 128 tile with cta_group::2
// MMAs issued by rank 0: each CTA loads its 128 rows of every A plane tile and
// 64 of the 128 rows of every B plane tile, so a CTA moves and reads a quarter
// less per MMA than a single-CTA 128 x 128 tile and the ring holds a third
// stage for BF16x3.  Rank 1's copies complete on rank 0's stage barriers; the
// MMA completions are multicast to both CTAs; both CTAs' epilogues report a
// drained accumulator to rank 0.
template <bool DF32, int BK, bool PAIR>
__global__ void __launch_bounds__(THREADS, 1) tc_terms_kernel(const __grid_constant__ CUtensorMap tmA,
                                                              const __grid_constant__ CUtensorMap tmB,
                                                              const __grid_constant__ TcArgs p)
{
    constexpr uint32_t A_TILE = 128u * BK * 2u;                  // 128 rows x BK bf16
    constexpr uint32_t B_TILE = (PAIR ? 64u : 128u) * BK * 2u;   // this CTA's rows of a B tile
    constexpr uint32_t RING = PAIR ? RING_BYTES_PAIR : RING_BYTES;
    constexpr int PM = PAIR ? 2 * BM : BM;                       // C rows per tile
    constexpr uint32_t kAccCols = 2 * BN;  // TMEM columns of one buffer: accumulators 0 and 1
    constexpr uint32_t kTmemCols = 2 * kAccCols;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* ring = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                           ~uintptr_t(1023));
    uint64_t* full = reinterpret_cast<uint64_t*>(ring + RING);
    uint64_t* empty = full + 16;
    uint64_t* acc_full = empty + 16;
    uint64_t* acc_empty = acc_full + 2;
    uint64_t* drain = acc_empty + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = PAIR ? cluster_ctarank() : 0u;
    const bool leader = rank == 0;
    const int unit0 = PAIR ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;  // tile-walking unit (CTA or pair)
    const int nunits = PAIR ? (int)(gridDim.x >> 1) : (int)gridDim.x;
    if (warp == 1) {
        if constexpr (PAIR) {
            tmem_alloc_pair(tmem_slot, kTmemCols);
            tmem_relinquish_pair();
        } else {
            tmem_alloc(tmem_slot, kTmemCols);
            tmem_relinquish();
        }
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < p.nstages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], EPI_WARPS * (PAIR ? 2 : 1));
        }
        mbar_init(drain, 1);
        mbar_fence_init();
    }
    tc_fence_before();
    if constexpr (PAIR) cluster_sync_all(); else __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    const int64_t my_tiles = p.tiles > unit0 ? (p.tiles - 1 - unit0) / nunits + 1 : 0;

    if (warp == 0) {
        // ------------------------------------------------ TMA producer (each CTA loads its own halves)
        if (lane == 0) {
            tma_prefetch_desc(&tmA);
            tma_prefetch_desc(&tmB);
            uint32_t it = 0;
            bool ok = true;
            for (int64_t tl = 0; tl < my_tiles && ok; ++tl) {
                const int tile = unit0 + (int)tl * nunits;
                int tm, tn;
                tile_coords(tile, p.tiles_m, p.tiles_n, tm, tn);
                const int arow = tm * PM + (int)rank * BM;
                const int brow = tn * BN + (PAIR ? (int)rank * (BN / 2) : 0);
                for (int c = 0; c < p.nchunks && ok; ++c) {
                    const int kb0 = c * p.chunk_kblocks, kb1 = min(p.kblocks, kb0 + p.chunk_kblocks);
                    for (int gi = 0; gi < p.ngroups && ok; ++gi) {
                        const TcGroup& g = p.g[gi];
                        for (int kb = kb0; kb < kb1; ++kb, ++it) {
                            const int s = (int)(it % (uint32_t)p.nstages);
                            const uint32_t ph = (it / (uint32_t)p.nstages) & 1u;
                            if (!mbar_wait(&empty[s], ph ^ 1u, p.err, kErrWaitEmpty)) { ok = false; break; }
                            unsigned char* st = ring + (size_t)s * p.stage_bytes;
                            const uint32_t bytes = (uint32_t)g.na * A_TILE + (uint32_t)g.nb * B_TILE;
                            if constexpr (PAIR) {
                                // rank 0's barrier counts both CTAs' bytes; both CTAs' copies complete on it
                                if (leader) mbar_arrive_expect_tx(&full[s], 2u * bytes);
                                const uint32_t bar = mapa_shared(smem_u32(&full[s]), 0);
                                for (int a = 0; a < g.na; ++a)
                                    tma_load_3d_pair(st + a * A_TILE, &tmA, bar, kb * BK, arow, g.aplane[a]);
                                for (int b = 0; b < g.nb; ++b)
                                    tma_load_3d_pair(st + g.na * A_TILE + b * B_TILE, &tmB, bar, kb * BK, brow,
                                                     g.bplane[b]);
                            } else {
                                mbar_arrive_expect_tx(&full[s], bytes);
                                for (int a = 0; a < g.na; ++a)
                                    tma_load_3d(st + a * A_TILE, &tmA, &full[s], kb * BK, arow, g.aplane[a]);
                                for (int b = 0; b < g.nb; ++b)
                                    tma_load_3d(st + g.na * A_TILE + b * B_TILE, &tmB, &full[s], kb * BK, brow,
                                                g.bplane[b]);
                            }
                        }
                    }
                }
            }
            if (!ok && (!PAIR || leader)) {
                // let the copies already issued land before the CTA exits
                const uint32_t first = it > (uint32_t)p.nstages ? it - (uint32_t)p.nstages : 0u;
                for (uint32_t q = first; q < it; ++q) {
                    const int s = (int)(q % (uint32_t)p.nstages);
                    const uint64_t t0 = globaltimer_ns();
                    while (!mbar_try_wait(smem_u32(&full[s]), (q / (uint32_t)p.nstages) & 1u) &&
                           globaltimer_ns() - t0 < kWaitLimitNs) {
                    }
                }
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer (rank 0 of a pair)
        if (lane == 0 && leader) {
            const uint32_t idesc = idesc_bf16_f32(PM, BN);
            uint32_t it = 0, unit = 0;
            bool ok = true;
            for (int64_t tl = 0; tl < my_tiles && ok; ++tl) {
                for (int c = 0; c < p.nchunks && ok; ++c) {
                    const int kb0 = c * p.chunk_kblocks, kb1 = min(p.kblocks, kb0 + p.chunk_kblocks);
                    for (int gi = 0; gi < p.ngroups && ok; ++gi, ++unit) {
                        const TcGroup& g = p.g[gi];
                        const int buf = (int)(unit & 1u);
                        if (!mbar_wait(&acc_empty[buf], ((unit >> 1) & 1u) ^ 1u, p.err, kErrWaitAcc)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t d_tmem = tmem_base + (uint32_t)buf * kAccCols;
                        uint32_t accumulate = 0, accumulate2 = 0;
                        for (int kb = kb0; kb < kb1; ++kb, ++it) {
                            const int s = (int)(it % (uint32_t)p.nstages);
                            if (!mbar_wait(&full[s], (it / (uint32_t)p.nstages) & 1u, p.err, kErrWaitFull)) {
                                ok = false;
                                break;
                            }
                            tc_fence_after();
                            const uint32_t st = smem_u32(ring + (size_t)s * p.stage_bytes);
                            for (int q = 0; q < g.np; ++q) {
                                const uint32_t a0 = st + (uint32_t)g.pa[q] * A_TILE;
                                const uint32_t b0 = st + (uint32_t)g.na * A_TILE + (uint32_t)g.pb[q] * B_TILE;
                                const bool second = q > 0;
                                const uint32_t d = second ? d_tmem + BN : d_tmem;
#pragma unroll
                                for (int k = 0; k < BK / 16; ++k) {
                                    const uint64_t da = sw128_kmajor_desc(a0 + k * 32);
                                    const uint64_t db = sw128_kmajor_desc(b0 + k * 32);
                                    if constexpr (PAIR)
                                        tc_mma_bf16_pair(d, da, db, idesc, second ? accumulate2 : accumulate);
                                    else
                                        tc_mma_bf16(d, da, db, idesc, second ? accumulate2 : accumulate);
                                    if (second) accumulate2 = 1; else accumulate = 1;
                                }
                            }
                            if constexpr (PAIR) tc_commit_pair(&empty[s], 3); else tc_commit(&empty[s]);
                        }
                        if (ok) {
                            if constexpr (PAIR) tc_commit_pair(&acc_full[buf], 3); else tc_commit(&acc_full[buf]);
                        }
                    }
                }
            }
            // every MMA issued so far has completed before TMEM is released
            if constexpr (PAIR) tc_commit_pair(drain, 1); else tc_commit(drain);
            const uint64_t t0 = globaltimer_ns();
            while (!mbar_try_wait(smem_u32(drain), 0u) && globaltimer_ns() - t0 < kWaitLimitNs) {
            }
        }
    } else {
        // ------------------------------------------------ epilogue warps
        const int q = warp & 3;                 // TMEM lane quadrant this warp may access
        const int quarter = (warp - 2) >> 2;    // column quarter of the tile
        const int row_in_tile = (int)rank * BM + q * 32 + lane;
        const uint32_t lane_off = (uint32_t)(q * 32) << 16;
        // DF32: a double-float (hi, lo) per output; FP64: one double per output
        float hi[DF32 ? 32 : 1], lo[DF32 ? 32 : 1];
        double acc[DF32 ? 1 : 32];
#pragma unroll
        for (int j = 0; j < (DF32 ? 32 : 1); ++j) hi[j] = lo[j] = 0.f;
#pragma unroll
        for (int j = 0; j < (DF32 ? 1 : 32); ++j) acc[j] = 0.0;
        uint32_t unit = 0;
        bool ok = true;
        for (int64_t tl = 0; tl < my_tiles && ok; ++tl) {
            const int tile = unit0 + (int)tl * nunits;
            int tm, tn;
            tile_coords(tile, p.tiles_m, p.tiles_n, tm, tn);
            for (int c = 0; c < p.nchunks && ok; ++c) {
                for (int gi = 0; gi < p.ngroups; ++gi, ++unit) {
                    const int buf = (int)(unit & 1u);
                    if (!mbar_wait(&acc_full[buf], (unit >> 1) & 1u, p.err, kErrWaitMma)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t t0 = tmem_base + lane_off + (uint32_t)buf * kAccCols + (uint32_t)(quarter * 32);
                    if constexpr (DF32) {
                        const bool has_small = p.g[gi].np > 1;
#pragma unroll
                        for (int cc = 0; cc < 2; ++cc) {
                            uint32_t v[16];
                            tmem_ld_32x32b_x16(t0 + cc * 16, v);
                            tmem_wait_ld();
#pragma unroll
                            for (int j = 0; j < 16; ++j) {
                                const int o = cc * 16 + j;
                                const float x = __uint_as_float(v[j]);
                                // TwoSum: hi + x = sum + e exactly
                                const float sum = __fadd_rn(hi[o], x);
                                const float bp = __fsub_rn(sum, hi[o]);
                                const float e = __fadd_rn(__fsub_rn(hi[o], __fsub_rn(sum, bp)), __fsub_rn(x, bp));
                                hi[o] = sum;
                                lo[o] = __fadd_rn(lo[o], e);
                            }
                            if (has_small) {
                                tmem_ld_32x32b_x16(t0 + BN + cc * 16, v);
                                tmem_wait_ld();
#pragma unroll
                                for (int j = 0; j < 16; ++j) lo[cc * 16 + j] = __fadd_rn(lo[cc * 16 + j], __uint_as_float(v[j]));
                            }
                        }
                    } else {
                        const int e0 = p.g[gi].scale_exp, e1 = p.g[gi].scale_exp2;
                        const bool has_second = p.g[gi].np > 1;
#pragma unroll
                        for (int cc = 0; cc < 2; ++cc) {
                            uint32_t v[16];
                            tmem_ld_32x32b_x16(t0 + cc * 16, v);
                            tmem_wait_ld();
#pragma unroll
                            for (int j = 0; j < 16; ++j) acc[cc * 16 + j] += scaled_f32_to_f64(v[j], e0);
                            if (has_second) {
                                tmem_ld_32x32b_x16(t0 + BN + cc * 16, v);
                                tmem_wait_ld();
#pragma unroll
                                for (int j = 0; j < 16; ++j) acc[cc * 16 + j] += scaled_f32_to_f64(v[j], e1);
                            }
                        }
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) {
                        if constexpr (PAIR) mbar_arrive_cluster(mapa_shared(smem_u32(&acc_empty[buf]), 0));
                        else mbar_arrive(&acc_empty[buf]);
                    }
                }
            }
            if (!ok) break;
            // final epilogue of this tile
            const int64_t row = (int64_t)tm * PM + row_in_tile;
            const int64_t col0 = (int64_t)tn * BN + quarter * 32;
            if (row < p.M) {
                const int re = p.row_exp ? p.row_exp[row] : 0;
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int64_t col = col0 + j;
                    const bool keep = p.tri == 0 || (p.tri == 1 ? col - row <= p.tri_off : col - row >= p.tri_off);
                    if (col < p.N && keep) {
                        double a;
                        if constexpr (DF32) a = (double)hi[j] + (double)lo[j];
                        else a = acc[j];
                        const int ce = p.col_exp ? p.col_exp[col] : 0;
                        double v = p.alpha * ldexp(a, re + ce);
                        if (p.c_fp32) {
                            float* cp = static_cast<float*>(p.C) + row * p.ldc + col;
                            if (p.read_c) v = fma(p.beta, (double)*cp, v);
                            *cp = (float)v;
                        } else {
                            double* cp = static_cast<double*>(p.C) + row * p.ldc + col;
                            if (p.read_c) v = fma(p.beta, *cp, v);
                            *cp = v;
                        }
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < (DF32 ? 32 : 1); ++j) hi[j] = lo[j] = 0.f;
#pragma unroll
            for (int j = 0; j < (DF32 ? 1 : 32); ++j) acc[j] = 0.0;
        }
    }
    tc_fence_before();
    if constexpr (PAIR) cluster_sync_all(); else __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        if constexpr (PAIR) tmem_dealloc_pair(tmem_base, kTmemCols);
        else tmem_dealloc(tmem_base, kTmemCols);
    }
}

// ---------------------------------------------------------------- splits --
// Operand views: element (r, k) of a slot is X[r * sr + k * sk] with either
// sk == 1 (K-major rows) or sr == 1 (K runs down the stored rows).  Planes are
// K-major [rows_pad x k_pad] bf16, zero outside rows x K.

constexpr int ST = 64;  // split tile: 64 rows x 64 K

// x = h + m + l, each the bf16 rounding of the remainder (the remainders are
// exact in FP32 because each bf16 rounding keeps the leading bits).
__global__ void __launch_bounds__(256) split_bf16x3_kernel(const float* __restrict__ X, int64_t sr, int64_t sk,
                                                           int rows, int K, int rows_pad, int k_pad,
                                                           __nv_bfloat16* __restrict__ planes)
{
    __shared__ float t[ST][ST + 1];
    const int r0 = blockIdx.y * ST, k0 = blockIdx.x * ST;
    const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;  // 64 x 4
    for (int i = ty; i < ST; i += 4) {
        // coalesced along the stored contiguous dimension
        int r, k;
        if (sk == 1) { r = r0 + i; k = k0 + tx; } else { r = r0 + tx; k = k0 + i; }
        float v = 0.f;
        if (r < rows && k < K) v = X[(int64_t)r * sr + (int64_t)k * sk];
        if (sk == 1) t[i][tx] = v; else t[tx][i] = v;
    }
    __syncthreads();
    const size_t plane = (size_t)rows_pad * k_pad;
    for (int i = ty; i < ST; i += 4) {
        const int r = r0 + i, k = k0 + tx;
        if (r >= rows_pad || k >= k_pad) continue;
        const float x = t[i][tx];
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        const float r1 = x - __bfloat162float(h);
        const __nv_bfloat16 m = __float2bfloat16_rn(r1);
        const float r2 = r1 - __bfloat162float(m);
        const __nv_bfloat16 l = __float2bfloat16_rn(r2);
        const size_t o = (size_t)r * k_pad + k;
        planes[o] = h;
        planes[plane + o] = m;
        planes[2 * plane + o] = l;
    }
}

// max |x| over each row (as the bit pattern of a non-negative double, which
// orders like its value); rowmax must start at zero
__global__ void __launch_bounds__(256) rowmax_f64_kernel(const double* __restrict__ X, int64_t sr, int64_t sk,
                                                         int rows, int K, unsigned long long* __restrict__ rowmax)
{
    __shared__ unsigned long long t[ST];
    const int r0 = blockIdx.y * ST, k0 = blockIdx.x * ST;
    const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;
    if (threadIdx.x < ST) t[threadIdx.x] = 0ull;
    __syncthreads();
    for (int i = ty; i < ST; i += 4) {
        int r, k;
        if (sk == 1) { r = r0 + i; k = k0 + tx; } else { r = r0 + tx; k = k0 + i; }
        if (r < rows && k < K) {
            const unsigned long long b =
                (unsigned long long)__double_as_longlong(fabs(X[(int64_t)r * sr + (int64_t)k * sk]));
            atomicMax(&t[r - r0], b);
        }
    }
    __syncthreads();
    if (threadIdx.x < ST && r0 + (int)threadIdx.x < rows && t[threadIdx.x]) atomicMax(&rowmax[r0 + threadIdx.x], t[threadIdx.x]);
}

// exponent e with max|x| < 2^e (0 for an all-zero row)
__global__ void rowexp_kernel(const unsigned long long* __restrict__ rowmax, int rows, int rows_pad,
                              int* __restrict__ rowexp)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows_pad) return;
    int e = 0;
    if (r < rows && rowmax[r]) {
        const int biased = (int)((rowmax[r] >> 52) & 0x7FF);
        e = (biased ? biased - 1023 : -1022) + 1;
    }
    rowexp[r] = e;
}

// Digits of the fixed-point value |x| * 2^(S*beta - e), truncated, from the
// most significant: d_s = (F >> beta*(S-s)) & (2^beta - 1), signed like x.
// Integer arithmetic only, so the digits are exact.
__global__ void __launch_bounds__(256) split_ozaki_kernel(const double* __restrict__ X, int64_t sr, int64_t sk,
                                                          int rows, int K, int rows_pad, int k_pad,
                                                          const int* __restrict__ rowexp, int S, int beta,
                                                          __nv_bfloat16* __restrict__ planes)
{
    __shared__ double t[ST][ST + 1];
    const int r0 = blockIdx.y * ST, k0 = blockIdx.x * ST;
    const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;
    for (int i = ty; i < ST; i += 4) {
        int r, k;
        if (sk == 1) { r = r0 + i; k = k0 + tx; } else { r = r0 + tx; k = k0 + i; }
        double v = 0.0;
        if (r < rows && k < K) v = X[(int64_t)r * sr + (int64_t)k * sk];
        if (sk == 1) t[i][tx] = v; else t[tx][i] = v;
    }
    __syncthreads();
    const size_t plane = (size_t)rows_pad * k_pad;
    const unsigned long long mask = (1ull << beta) - 1ull;
    for (int i = ty; i < ST; i += 4) {
        const int r = r0 + i, k = k0 + tx;
        if (r >= rows_pad || k >= k_pad) continue;
        const unsigned long long bits = (unsigned long long)__double_as_longlong(t[i][tx]);
        const int biased = (int)((bits >> 52) & 0x7FF);
        unsigned long long mant = bits & ((1ull << 52) - 1ull);
        if (biased) mant |= 1ull << 52;
        const int ex = biased ? biased - 1023 : -1022;  // |x| = mant * 2^(ex - 52)
        const int e = r < rows ? rowexp[r] : 0;
        const int shift = ex - 52 + S * beta - e;       // <= S*beta - 53 for entries of this row
        unsigned long long F = 0;
        if (mant) {
            if (shift >= 0) F = shift < 64 ? (mant << shift) : 0ull;
            else F = -shift < 64 ? (mant >> (-shift)) : 0ull;
        }
        const bool neg = (bits >> 63) != 0;
        const size_t o = (size_t)r * k_pad + k;
        for (int s = 1; s <= S; ++s) {
            const int d = (int)((F >> (beta * (S - s))) & mask);
            planes[(size_t)(s - 1) * plane + o] = __int2bfloat16_rn(neg ? -d : d);
        }
    }
}

std::once_flag g_attr_once;
int g_sms = 0;
int g_pairs = 0;  // resident CTA pairs of the pair kernel (0: pairs unavailable)

}  // namespace

int tc_max_groups() { return MAX_GROUPS; }

int launch_split_bf16x3(const float* X, int64_t sr, int64_t sk, int rows, int K, int rows_pad, int k_pad, void* planes,
                        void* stream, std::string& why)
{
    dim3 grid((unsigned)((k_pad + ST - 1) / ST), (unsigned)((rows_pad + ST - 1) / ST));
    split_bf16x3_kernel<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(
        X, sr, sk, rows, K, rows_pad, k_pad, static_cast<__nv_bfloat16*>(planes));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { why = std::string("split_bf16x3: ") + cudaGetErrorString(e); return OOC_ERR_CUDA; }
    return OOC_OK;
}

int launch_split_ozaki(const double* X, int64_t sr, int64_t sk, int rows, int K, int rows_pad, int k_pad, int S,
                       int beta, void* planes, int* rowexp, unsigned long long* rowmax, void* stream,
                       std::string& why)
{
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(rowmax, 0, sizeof(unsigned long long) * (size_t)rows_pad, st) != cudaSuccess) {
        why = "rowmax clear";
        return OOC_ERR_CUDA;
    }
    dim3 grid((unsigned)((k_pad + ST - 1) / ST), (unsigned)((rows_pad + ST - 1) / ST));
    if (K > 0) rowmax_f64_kernel<<<grid, 256, 0, st>>>(X, sr, sk, rows, K, rowmax);
    rowexp_kernel<<<(unsigned)((rows_pad + 255) / 256), 256, 0, st>>>(rowmax, rows, rows_pad, rowexp);
    split_ozaki_kernel<<<grid, 256, 0, st>>>(X, sr, sk, rows, K, rows_pad, k_pad, rowexp, S, beta,
                                             static_cast<__nv_bfloat16*>(planes));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { why = std::string("split_ozaki: ") + cudaGetErrorString(e); return OOC_ERR_CUDA; }
    return OOC_OK;
}

int launch_tc_terms(const TcProblem& P, void* stream, std::string& why)
{
    if (P.M <= 0 || P.N <= 0) return OOC_OK;
    if (P.ngroups <= 0 || P.ngroups > MAX_GROUPS) { why = "bad group count"; return OOC_ERR_INVALID_ARG; }
    std::call_once(g_attr_once, [] {
        cudaFuncSetAttribute(tc_terms_kernel<true, 64, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)SMEM_BYTES);
        cudaFuncSetAttribute(tc_terms_kernel<false, 64, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)SMEM_BYTES);
        cudaFuncSetAttribute(tc_terms_kernel<true, 64, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)SMEM_BYTES_PAIR);
        cudaFuncSetAttribute(tc_terms_kernel<false, 64, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)SMEM_BYTES_PAIR);
        g_sms = device_sm_count();
        // CTA pairs that can be resident at once (clusters are placed inside GPCs)
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(2 * 76);
        cfg.blockDim = dim3(THREADS);
        cfg.dynamicSmemBytes = SMEM_BYTES_PAIR;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 2;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, tc_terms_kernel<true, 64, true>, &cfg) != cudaSuccess) {
            cudaGetLastError();
            n = 0;
        }
        g_pairs = n;
    });
    // 64-wide K blocks (128-byte swizzle) measured faster than 32-wide ones for
    // both forms on GB300 (BF16x3 166 vs 136, Ozaki 28 vs 18 logical TFLOP/s)
    const int BK = 64;
    if (P.kblock != BK) { why = "only 64-wide K blocks are built"; return OOC_ERR_INVALID_ARG; }
    const bool pair = P.pair && g_pairs > 0;
    const uint32_t A_TILE = 128u * (uint32_t)BK * 2u;
    const uint32_t B_TILE = (pair ? 64u : 128u) * (uint32_t)BK * 2u;
    const int PM = pair ? 2 * BM : BM;
    TcArgs a;
    std::memset(&a, 0, sizeof(a));
    a.M = (int)P.M; a.N = (int)P.N;
    if (P.k_pad % BK || P.chunk % BK) { why = "K padding / chunk not a multiple of the K block"; return OOC_ERR_INVALID_ARG; }
    a.kblocks = (int)(P.k_pad / BK);
    a.chunk_kblocks = std::max(1, P.chunk / BK);
    a.nchunks = (a.kblocks + a.chunk_kblocks - 1) / a.chunk_kblocks;
    a.ngroups = P.ngroups;
    a.tiles_n = (int)((P.N + BN - 1) / BN);
    a.tiles_m = (int)((P.M + PM - 1) / PM);
    a.tiles = a.tiles_m * a.tiles_n;
    uint32_t max_stage = 0;
    for (int g = 0; g < P.ngroups; ++g) {
        const TcGroupSpec& s = P.groups[g];
        TcGroup& d = a.g[g];
        if (s.na < 1 || s.na > 4 || s.nb < 1 || s.nb > 4 || s.np < 1 || s.np > 6) {
            why = "bad group shape";
            return OOC_ERR_INVALID_ARG;
        }
        d.na = (int8_t)s.na; d.nb = (int8_t)s.nb; d.np = (int8_t)s.np;
        for (int i = 0; i < 4; ++i) { d.aplane[i] = (int8_t)s.aplane[i]; d.bplane[i] = (int8_t)s.bplane[i]; }
        for (int i = 0; i < 6; ++i) { d.pa[i] = (int8_t)s.pa[i]; d.pb[i] = (int8_t)s.pb[i]; }
        d.scale_exp = (int16_t)s.scale_exp;
        d.scale_exp2 = (int16_t)s.scale_exp2;
        if (!P.df32 && s.np > 2) {
            why = "exact (Ozaki) groups hold at most two pairs";
            return OOC_ERR_INVALID_ARG;
        }
        max_stage = std::max(max_stage, (uint32_t)s.na * A_TILE + (uint32_t)s.nb * B_TILE);
    }
    a.stage_bytes = max_stage;
    a.nstages = std::min<int>(16, (int)((pair ? RING_BYTES_PAIR : RING_BYTES) / a.stage_bytes));  // 16 barrier slots
    if (a.nstages < 2) { why = "stage ring too small"; return OOC_ERR_INVALID_ARG; }
    a.alpha = P.alpha; a.beta = P.beta;
    a.read_c = P.read_c ? 1 : 0; a.c_fp32 = P.c_fp32 ? 1 : 0;
    a.C = P.C; a.ldc = P.ldc;
    a.row_exp = P.row_exp; a.col_exp = P.col_exp;
    a.err = P.err;
    a.tri = P.tri; a.tri_off = P.tri_off;

    CUtensorMap ma, mb;
    std::memset(&ma, 0, sizeof(ma));
    std::memset(&mb, 0, sizeof(mb));
    if (a.kblocks > 0) {  // K == 0 runs the epilogue only (C = beta * C)
        // rows past the padded planes (the last pair tile) read as zeros from TMA
        int rc = encode_map_3d_bf16(&ma, P.a_planes, (uint64_t)P.k_pad, (uint64_t)P.a_rows_pad,
                                    (uint64_t)P.a_nplanes, BK, BM, why);
        if (rc) return rc;
        rc = encode_map_3d_bf16(&mb, P.b_planes, (uint64_t)P.k_pad, (uint64_t)P.b_rows_pad, (uint64_t)P.b_nplanes,
                                BK, pair ? BN / 2 : BN, why);
        if (rc) return rc;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (pair) {
        const int pairs = std::min(a.tiles, g_pairs);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(2 * pairs));
        cfg.blockDim = dim3(THREADS);
        cfg.dynamicSmemBytes = SMEM_BYTES_PAIR;
        cfg.stream = st;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 2;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        e = P.df32 ? cudaLaunchKernelEx(&cfg, tc_terms_kernel<true, 64, true>, ma, mb, a)
                   : cudaLaunchKernelEx(&cfg, tc_terms_kernel<false, 64, true>, ma, mb, a);
    } else {
        const int grid = std::min(a.tiles, g_sms > 0 ? g_sms : 152);
        if (P.df32) tc_terms_kernel<true, 64, false><<<grid, THREADS, SMEM_BYTES, st>>>(ma, mb, a);
        else tc_terms_kernel<false, 64, false><<<grid, THREADS, SMEM_BYTES, st>>>(ma, mb, a);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) { why = std::string("tc_terms launch: ") + cudaGetErrorString(e); return OOC_ERR_CUDA; }
    return OOC_OK;
}

}  // namespace ooc
