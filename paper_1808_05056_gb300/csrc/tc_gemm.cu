// Split-product tile contraction on the 5th-generation tensor cores (sm_103a):
// the compute stage of the out-of-core pipeline for the two tensor-core forms.
//
//   BF16x3 (FP32-accurate, ooc_sgemm): each FP32 operand is split into three
//   bf16 pieces x = h + m + l (each piece the bf16 rounding of what is left),
//   and C = sum of the six products hh, hm, mh, hl, mm, lh (the dropped ml, lm,
//   ll are below 2^-24 relative).  The tensor cores round their FP32
//   accumulator toward zero, so each accumulator addition is biased by up to
//   one ulp: the leading product hh has its own accumulator, drained every
//   `chunk` of K (512: 32 additions) into an unbiased double-float (hi, lo)
//   pair per output with TwoSum; the five small products, 2^-8 of hh and
//   below, share a second accumulator drained every 2048 of K straight into
//   lo.  The drains run on the epilogue warps, four of which share the MMA
//   thread's sub-partition (TMEM lane quarters tie warps to sub-partitions):
//   draining hh every 128 of K took enough of that thread's issue slots to
//   cost a fifth of the tensor-core rate.
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
//   warp 0      TMA producer: for each (tile, K chunk, group, K block of 64)
//               loads the group's bf16 plane tiles (128-byte swizzle) into a
//               ring of stages;
//   warp 1      allocates all 512 TMEM columns and issues tcgen05.mma (M=128,
//               N=128, K=16), committing stage releases and accumulator-full
//               events to mbarriers;
//   warps 2-17  epilogue: drain finished accumulators with tcgen05.ld into
//               FP64 (Ozaki) or packed double-float FP32 (BF16x3) registers,
//               32 columns of one row per thread, release them, and after the
//               last chunk write alpha*acc*2^(e_i+f_j) + beta*C_old, each store
//               covering 8 rows x 4 consecutive columns (4 x 4 transposes by
//               shuffles inside groups of 4 lanes).
// TMEM: Ozaki uses two buffers of two 128-column accumulators (the group's two
// products), so the tensor cores run the next group while the epilogue drains
// the previous one; BF16x3 uses three buffers for hh and one accumulator for
// the small products.
//
// The single issuing thread keeps its per-stage work to the MMAs themselves
// (descriptor offsets precomputed per group, ring positions advanced without
// division): at 64 cycles per 128 x 128 x 16 MMA, anything more starves the
// tensor pipe.  For the same reason the ring releases whole stages: finer
// slots (one 16 KiB plane tile each, with a wait and a release per tile) ran
// at half the rate for both forms, even with the same shared-memory layout.
// CTA pairs (cta_group::2, 256 x 128 tiles with half of each B
// tile per CTA) were measured slower on GB300 for both forms (BF16x3 1216 vs
// 1384, Ozaki 1337 vs 1374 bf16 TFLOP/s) and are not built.  Every wait is
// bounded (device_sync.cuh); the epilogue warps wait with a sleep between
// tries so that they leave the issue slots to the TMA and MMA threads.
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

constexpr int BM = 128, BN = 128, BK = 64;
constexpr uint32_t A_TILE = BM * BK * 2u;             // 128 rows x 64 bf16 of K (16 KiB)
constexpr uint32_t RING_BYTES = 192u * 1024u;         // two 96 KiB BF16x3 stages, four 48 KiB Ozaki stages
constexpr int EPI_WARPS = 16;                         // 4 per TMEM lane quadrant, 32 columns each
constexpr int THREADS = (2 + EPI_WARPS) * 32;
constexpr int MAX_GROUPS = 64;
constexpr int MAX_STAGES = 16;
constexpr size_t SMEM_BYTES = 1024 + RING_BYTES + 1024;
constexpr int kSmallK = 2048;                         // BF16x3: K between small-product drains
constexpr uint32_t kSmallCol = 384;                   // BF16x3: TMEM column of the small-product accumulator

struct TcGroup {
    int8_t na, nb, np, pad0;
    int8_t aplane[4];
    int8_t bplane[4];
    int8_t pa[6];
    int8_t pb[6];
    int16_t scale_exp;   // weight of accumulator 0 (pair 0)
    int16_t scale_exp2;  // weight of accumulator 1 (pair 1, Ozaki)
    int16_t pad1[2];
};
static_assert(sizeof(TcGroup) == 32, "group record layout");

struct TcArgs {
    int M, N;
    int kblocks, chunk_kblocks, nchunks;
    int small_every;  // BF16x3: chunks between small-product drains
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
// that the tiles in flight at once span few rows and few columns and share
// their A and B plane tiles in L2.
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

// Exact FP32 integer x (1 <= |x| < 2^24, or 0) times 2^e as a double, built
// from the bit fields with 32-bit integer operations (no conversion or multiply
// on the FP64 pipe, few instructions on the warps that share the MMA thread's
// sub-partition): `bias_hi` = (1023 - 127 + e) << 20 moves the FP32 exponent
// field, shifted into the double's high word, to the double's bias and scale;
// the low 3 mantissa bits go to the top of the low word.  The exponent field
// e8 + 896 + e (127 <= e8 <= 150) stays inside 1..2046 and the bias inside its
// 11 bits for -896 <= e <= 1000; the digit weights -6 (s + t) are at least -66.
__device__ __forceinline__ double scaled_f32_to_f64(uint32_t xb, uint32_t bias_hi)
{
    const uint32_t mag = xb & 0x7FFFFFFFu;
    const uint32_t hi = ((mag >> 3) + bias_hi) | (xb & 0x80000000u);
    const uint32_t lo = xb << 29;
    return mag ? __hiloint2double((int)hi, (int)lo) : 0.0;
}

// Packed pairs of FP32 values (element 2j in the low half): Blackwell's f32x2
// arithmetic does two of the drain's additions per instruction.
__device__ __forceinline__ uint64_t f2add(uint64_t a, uint64_t b)
{
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t f2sub(uint64_t a, uint64_t b)
{
    uint64_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t pack2(uint32_t lo, uint32_t hi) { return ((uint64_t)hi << 32) | lo; }
__device__ __forceinline__ float unpack2(uint64_t v, int j) { return __uint_as_float((uint32_t)(v >> (32 * j))); }

// ring position: slot and pass parity, advanced without division
struct Ring {
    int s = 0;
    uint32_t ph = 0;
    __device__ __forceinline__ void next(int n)
    {
        if (++s == n) { s = 0; ph ^= 1u; }
    }
};

// 4 x 4 transpose inside each group of 4 lanes: lane 4g + r holds row r of its
// group's block in v[0..3] on entry and column r on exit.  Each butterfly stage
// m swaps the off-diagonal m x m sub-blocks: the lane without bit m trades its
// elements with bit m set for its partner's elements without it.
__device__ __forceinline__ void transpose4(double (&v)[4], int lane)
{
#pragma unroll
    for (int m = 2; m >= 1; m >>= 1) {
        const bool upper = (lane & m) != 0;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            if (e & m) continue;
            const double send = upper ? v[e] : v[e | m];
            const double got = __shfl_xor_sync(0xffffffffu, send, m);
            if (upper) v[e] = got;
            else v[e | m] = got;
        }
    }
}

// BF16x3 drains of the small-product accumulator: every `every` chunks (2048 of
// K) and at the last chunk of a tile (both the MMA issuer and the epilogue use this)
__device__ __forceinline__ bool small_drain_after(int c, int nchunks, int every)
{
    return c == nchunks - 1 || (c % every) == every - 1;
}

template <bool DF32>
__global__ void __launch_bounds__(THREADS, 1) tc_terms_kernel(const __grid_constant__ CUtensorMap tmA,
                                                              const __grid_constant__ CUtensorMap tmB,
                                                              const __grid_constant__ TcArgs p)
{
    constexpr uint32_t B_TILE = BN * BK * 2u;
    constexpr int NBUF = DF32 ? 3 : 2;                            // accumulator buffers in TMEM
    constexpr uint32_t BUF_COLS = DF32 ? BN : 2 * BN;
    constexpr uint32_t kTmemCols = 512;
    constexpr int NPMAX = DF32 ? 6 : 2;
    constexpr int KSTEPS = BK / 16;
    constexpr uint32_t kArrivals = EPI_WARPS;                     // epilogue warps releasing a buffer
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* ring = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                           ~uintptr_t(1023));
    uint64_t* full = reinterpret_cast<uint64_t*>(ring + RING_BYTES);
    uint64_t* empty = full + MAX_STAGES;
    uint64_t* acc_full = empty + MAX_STAGES;
    uint64_t* acc_empty = acc_full + 4;
    uint64_t* small_full = acc_empty + 4;
    uint64_t* small_empty = small_full + 1;
    uint64_t* drain = small_empty + 1;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 1) {
        tmem_alloc(tmem_slot, kTmemCols);
        tmem_relinquish();
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < p.nstages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < NBUF; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], kArrivals);
        }
        mbar_init(small_full, 1);
        mbar_init(small_empty, kArrivals);
        mbar_init(drain, 1);
        mbar_fence_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    const int64_t my_tiles =
        p.tiles > (int)blockIdx.x ? (p.tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

    if (warp == 0) {
        // ------------------------------------------------ TMA producer
        if (lane == 0) {
            tma_prefetch_desc(&tmA);
            tma_prefetch_desc(&tmB);
            Ring r;
            uint32_t issued = 0;
            bool ok = true;
            for (int64_t tl = 0; tl < my_tiles && ok; ++tl) {
                const int tile = (int)blockIdx.x + (int)tl * (int)gridDim.x;
                int tm, tn;
                tile_coords(tile, p.tiles_m, p.tiles_n, tm, tn);
                const int arow = tm * BM, brow = tn * BN;
                for (int c = 0; c < p.nchunks && ok; ++c) {
                    const int kb0 = c * p.chunk_kblocks, kb1 = min(p.kblocks, kb0 + p.chunk_kblocks);
                    for (int gi = 0; gi < p.ngroups && ok; ++gi) {
                        const TcGroup& g = p.g[gi];
                        const int na = g.na, nb = g.nb;
                        const uint32_t bytes = (uint32_t)na * A_TILE + (uint32_t)nb * B_TILE;
                        for (int kb = kb0; kb < kb1; ++kb) {
                            if (!mbar_wait(&empty[r.s], r.ph ^ 1u, p.err, kErrWaitEmpty)) { ok = false; break; }
                            unsigned char* st = ring + (size_t)r.s * p.stage_bytes;
                            mbar_arrive_expect_tx(&full[r.s], bytes);
                            for (int a = 0; a < na; ++a)
                                tma_load_3d(st + a * A_TILE, &tmA, &full[r.s], kb * BK, arow, g.aplane[a]);
                            for (int b = 0; b < nb; ++b)
                                tma_load_3d(st + na * A_TILE + b * B_TILE, &tmB, &full[r.s], kb * BK, brow,
                                            g.bplane[b]);
                            r.next(p.nstages);
                            ++issued;
                        }
                    }
                }
            }
            if (!ok) {
                // let the copies already issued land before the CTA exits
                const uint32_t n = min(issued, (uint32_t)p.nstages);
                for (uint32_t q = 0; q < n; ++q) {
                    int s = r.s - 1 - (int)q;
                    uint32_t ph = r.ph;
                    while (s < 0) { s += p.nstages; ph ^= 1u; }
                    const uint64_t t0 = globaltimer_ns();
                    while (!mbar_try_wait(smem_u32(&full[s]), ph) && globaltimer_ns() - t0 < kWaitLimitNs) {
                    }
                }
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16_f32(BM, BN);
            Ring r, b;
            uint32_t small_drains = 0;   // BF16x3: small-accumulator drains committed so far
            bool small_pending = false;  // a drain committed and not yet released by the epilogue
            bool ok = true;
            for (int64_t tl = 0; tl < my_tiles && ok; ++tl) {
                uint32_t small_acc = 0;  // BF16x3: accumulate flag of the small-product accumulator
                for (int c = 0; c < p.nchunks && ok; ++c) {
                    const int kb0 = c * p.chunk_kblocks, kb1 = min(p.kblocks, kb0 + p.chunk_kblocks);
                    for (int gi = 0; gi < p.ngroups && ok; ++gi) {
                        const TcGroup& g = p.g[gi];
                        // descriptor offsets of the group's pairs (16-byte units)
                        uint32_t aoff[NPMAX], boff[NPMAX];
                        const int np = g.np;
                        const uint32_t bbase = (uint32_t)g.na * A_TILE;
#pragma unroll
                        for (int q = 0; q < NPMAX; ++q) {
                            const int src = q < np ? q : 0;
                            aoff[q] = ((uint32_t)g.pa[src] * A_TILE) >> 4;
                            boff[q] = (bbase + (uint32_t)g.pb[src] * B_TILE) >> 4;
                        }
                        if (!mbar_wait(&acc_empty[b.s], b.ph ^ 1u, p.err, kErrWaitAcc)) { ok = false; break; }
                        tc_fence_after();
                        const uint32_t d0 = tmem_base + (uint32_t)b.s * BUF_COLS;
                        uint32_t acc0 = 0, acc1 = 0;
                        for (int kb = kb0; kb < kb1; ++kb) {
                            if (!mbar_wait(&full[r.s], r.ph, p.err, kErrWaitFull)) { ok = false; break; }
                            tc_fence_after();
                            const uint64_t dst = sw128_kmajor_desc(smem_u32(ring + (size_t)r.s * p.stage_bytes));
                            if constexpr (DF32) {
                                if (small_pending) {
                                    // the epilogue has read the small accumulator before it restarts
                                    if (!mbar_wait(small_empty, (small_drains - 1) & 1u, p.err, kErrWaitAcc)) {
                                        ok = false;
                                        break;
                                    }
                                    tc_fence_after();
                                    small_pending = false;
                                }
                            }
#pragma unroll
                            for (int q = 0; q < NPMAX; ++q) {
                                if (q < np) {
                                    // DF32: pair 0 (hh) into buffer d0, pairs 1.. into the small accumulator;
                                    // exact: pair q into accumulator q of the buffer
                                    const uint32_t d = DF32 ? (q == 0 ? d0 : tmem_base + kSmallCol)
                                                            : (q == 0 ? d0 : d0 + BN);
                                    uint32_t& flag = DF32 ? (q == 0 ? acc0 : small_acc) : (q == 0 ? acc0 : acc1);
                                    const uint64_t da = dst + aoff[q], db = dst + boff[q];
#pragma unroll
                                    for (int k = 0; k < KSTEPS; ++k) {
                                        const uint32_t f = k > 0 ? 1u : flag;
                                        tc_mma_bf16(d, da + 2 * k, db + 2 * k, idesc, f);
                                    }
                                    flag = 1u;
                                }
                            }
                            tc_commit(&empty[r.s]);
                            r.next(p.nstages);
                        }
                        if (!ok) break;
                        tc_commit(&acc_full[b.s]);
                        b.next(NBUF);
                        if constexpr (DF32) {
                            if (small_drain_after(c, p.nchunks, p.small_every)) {
                                tc_commit(small_full);
                                ++small_drains;
                                small_pending = true;
                                small_acc = 0;
                            }
                        }
                    }
                }
            }
            // every MMA issued so far has completed before TMEM is released
            tc_commit(drain);
            const uint64_t t0 = globaltimer_ns();
            while (!mbar_try_wait(smem_u32(drain), 0u) && globaltimer_ns() - t0 < kWaitLimitNs) {
            }
        }
    } else {
        // ------------------------------------------------ epilogue warps
        const int q4 = warp & 3;                 // TMEM lane quadrant this warp may access
        const int quarter = (warp - 2) >> 2;    // column quarter of the tile
        const int row_in_tile = q4 * 32 + lane;
        const uint32_t lane_off = (uint32_t)(q4 * 32) << 16;
        // DF32: a packed double-float (hi, lo) per output; exact: one double per output
        uint64_t hi2[DF32 ? 16 : 1], lo2[DF32 ? 16 : 1];
        double acc[DF32 ? 1 : 32];
#pragma unroll
        for (int j = 0; j < (DF32 ? 16 : 1); ++j) hi2[j] = lo2[j] = 0ull;
#pragma unroll
        for (int j = 0; j < (DF32 ? 1 : 32); ++j) acc[j] = 0.0;
        Ring b;
        uint32_t small_drains = 0;
        bool ok = true;
        for (int64_t tl = 0; tl < my_tiles && ok; ++tl) {
            const int tile = (int)blockIdx.x + (int)tl * (int)gridDim.x;
            int tm, tn;
            tile_coords(tile, p.tiles_m, p.tiles_n, tm, tn);
            for (int c = 0; c < p.nchunks && ok; ++c) {
                for (int gi = 0; gi < p.ngroups; ++gi) {
                    // every lane gives up together (the warp shuffles and syncs below need all 32)
                    if (!__all_sync(0xffffffffu, mbar_wait_backoff(&acc_full[b.s], b.ph, p.err, kErrWaitMma))) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t t0 = tmem_base + lane_off + (uint32_t)b.s * BUF_COLS + (uint32_t)(quarter * 32);
                    if constexpr (DF32) {
#pragma unroll
                        for (int cc = 0; cc < 4; ++cc) {
                            uint32_t v[8];
                            tmem_ld_32x32b_x8(t0 + cc * 8, v);
                            tmem_wait_ld();
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                // TwoSum on pairs: hi + x = sum + e exactly, e added into lo
                                uint64_t& h = hi2[cc * 4 + j];
                                const uint64_t x = pack2(v[2 * j], v[2 * j + 1]);
                                const uint64_t sum = f2add(h, x);
                                const uint64_t bp = f2sub(sum, h);
                                const uint64_t e = f2add(f2sub(h, f2sub(sum, bp)), f2sub(x, bp));
                                h = sum;
                                lo2[cc * 4 + j] = f2add(lo2[cc * 4 + j], e);
                            }
                        }
                    } else {
                        const uint32_t e0 = (uint32_t)(896 + p.g[gi].scale_exp) << 20;
                        const uint32_t e1 = (uint32_t)(896 + p.g[gi].scale_exp2) << 20;
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
                    if (lane == 0) mbar_arrive(&acc_empty[b.s]);
                    b.next(NBUF);
                    if constexpr (DF32) {
                        if (small_drain_after(c, p.nchunks, p.small_every)) {
                            // the small products (2^-8 of hh and below) go straight into lo
                            if (!__all_sync(0xffffffffu,
                                            mbar_wait_backoff(small_full, small_drains & 1u, p.err, kErrWaitMma))) {
                                ok = false;
                                break;
                            }
                            tc_fence_after();
                            const uint32_t ts = tmem_base + lane_off + kSmallCol + (uint32_t)(quarter * 32);
#pragma unroll
                            for (int cc = 0; cc < 4; ++cc) {
                                uint32_t v[8];
                                tmem_ld_32x32b_x8(ts + cc * 8, v);
                                tmem_wait_ld();
#pragma unroll
                                for (int j = 0; j < 4; ++j)
                                    lo2[cc * 4 + j] = f2add(lo2[cc * 4 + j], pack2(v[2 * j], v[2 * j + 1]));
                            }
                            tc_fence_before();
                            __syncwarp();
                            if (lane == 0) mbar_arrive(small_empty);
                            ++small_drains;
                        }
                    }
                }
            }
            if (!ok) break;
            // final epilogue of this tile, 4 columns at a time: each lane forms its own row's
            // values, transpose4 hands lane 4g + j column j of rows 4g .. 4g + 3, and each store
            // then covers 8 rows x 4 consecutive columns of C (whole 32-byte sectors for FP64)
            // BF16x3 forms alpha * (hi + lo) + beta * C_old in FP32 double-float steps (TwoSum,
            // products split with fma) and rounds once at the end: on this part the FP64 pipe
            // would take ~18 us per tile for it, holding the accumulators the MMAs wait for
            const float alpha_f = (float)p.alpha, beta_f = (float)p.beta;
            const int64_t row_me = (int64_t)tm * BM + row_in_tile;
            const int re = (!DF32 && p.row_exp && row_me < p.M) ? p.row_exp[row_me] : 0;
            const int64_t row0 = (int64_t)tm * BM + q4 * 32 + (lane & ~3);
#pragma unroll
            for (int pass = 0; pass < 8; ++pass) {
                const int64_t c0 = (int64_t)tn * BN + quarter * 32 + pass * 4;
                double v[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int jj = pass * 4 + j;
                    if constexpr (DF32) {
                        // no operand scaling in this form; (ph, pl) = alpha * (hi + lo), packed
                        const float hi = unpack2(hi2[jj >> 1], jj & 1), lo = unpack2(lo2[jj >> 1], jj & 1);
                        const float sh = __fadd_rn(hi, lo), bp = __fsub_rn(sh, hi);
                        const float sl = __fadd_rn(__fsub_rn(hi, __fsub_rn(sh, bp)), __fsub_rn(lo, bp));
                        const float ph = __fmul_rn(alpha_f, sh);
                        const float pl = __fmaf_rn(alpha_f, sl, __fmaf_rn(alpha_f, sh, -ph));
                        v[j] = __longlong_as_double((long long)pack2(__float_as_uint(ph), __float_as_uint(pl)));
                    } else {
                        const int ce = (p.col_exp && c0 + j < p.N) ? p.col_exp[c0 + j] : 0;
                        v[j] = p.alpha * ldexp(acc[jj], re + ce);
                    }
                }
                transpose4(v, lane);
                const int64_t col = c0 + (lane & 3);
                if (col < p.N) {
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int64_t row = row0 + i;
                        const bool keep =
                            p.tri == 0 || (p.tri == 1 ? col - row <= p.tri_off : col - row >= p.tri_off);
                        if (row < p.M && keep) {
                            const int64_t off = row * p.ldc + col;
                            if constexpr (DF32) {
                                const uint64_t b = (uint64_t)__double_as_longlong(v[i]);
                                const float ph = unpack2(b, 0), pl = unpack2(b, 1);
                                float* cp = static_cast<float*>(p.C) + off;
                                float w;
                                if (p.read_c) {
                                    // beta * c = qh + ql and ph + qh = th + tl exactly; one rounding left
                                    const float c = *cp;
                                    const float qh = __fmul_rn(beta_f, c), ql = __fmaf_rn(beta_f, c, -qh);
                                    const float th = __fadd_rn(ph, qh), bq = __fsub_rn(th, ph);
                                    const float tl = __fadd_rn(__fsub_rn(ph, __fsub_rn(th, bq)), __fsub_rn(qh, bq));
                                    w = __fadd_rn(th, __fadd_rn(tl, __fadd_rn(pl, ql)));
                                } else {
                                    w = __fadd_rn(ph, pl);
                                }
                                *cp = w;
                                continue;
                            }
                            double w = v[i];
                            if (p.c_fp32) {
                                float* cp = static_cast<float*>(p.C) + off;
                                if (p.read_c) w = fma(p.beta, (double)*cp, w);
                                *cp = (float)w;
                            } else {
                                double* cp = static_cast<double*>(p.C) + off;
                                if (p.read_c) w = fma(p.beta, *cp, w);
                                *cp = w;
                            }
                        }
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < (DF32 ? 16 : 1); ++j) hi2[j] = lo2[j] = 0ull;
#pragma unroll
            for (int j = 0; j < (DF32 ? 1 : 32); ++j) acc[j] = 0.0;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem_base, kTmemCols);
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

// The same split for a K-major source whose rows start on 16-byte boundaries
// (the A slots of row-major operands): thread (k8, row) splits 8 consecutive K
// with two 16-byte loads and one 16-byte store per piece plane; no staging.
// Grid: x over k_pad / 8 in blocks of 256 threads, y over rows_pad.
__device__ __forceinline__ uint32_t bf16_pair(float a, float b)
{
    return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(a)) |
           ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(b)) << 16);
}

__global__ void __launch_bounds__(256) split_bf16x3_rows_kernel(const float* __restrict__ X, int64_t sr, int rows,
                                                                int K, int rows_pad, int k_pad,
                                                                __nv_bfloat16* __restrict__ planes)
{
    const int r = blockIdx.y;
    const int k = (blockIdx.x * blockDim.x + threadIdx.x) * 8;
    if (k >= k_pad) return;
    float x[8];
    if (r < rows && k + 8 <= K) {
        const float4* src = reinterpret_cast<const float4*>(X + (int64_t)r * sr + k);
        const float4 a = __ldg(src), b = __ldg(src + 1);
        x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
        x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
    } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) x[j] = (r < rows && k + j < K) ? X[(int64_t)r * sr + k + j] : 0.f;
    }
    uint32_t hw[4], mw[4], lw[4];
#pragma unroll
    for (int j = 0; j < 8; j += 2) {
        float h2[2], r1[2], m2[2], r2[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            h2[q] = __bfloat162float(__float2bfloat16_rn(x[j + q]));
            r1[q] = x[j + q] - h2[q];
            m2[q] = __bfloat162float(__float2bfloat16_rn(r1[q]));
            r2[q] = r1[q] - m2[q];
        }
        hw[j / 2] = bf16_pair(h2[0], h2[1]);
        mw[j / 2] = bf16_pair(m2[0], m2[1]);
        lw[j / 2] = bf16_pair(r2[0], r2[1]);
    }
    const size_t plane = (size_t)rows_pad * k_pad, o = (size_t)r * k_pad + k;
    *reinterpret_cast<uint4*>(planes + o) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
    *reinterpret_cast<uint4*>(planes + plane + o) = make_uint4(mw[0], mw[1], mw[2], mw[3]);
    *reinterpret_cast<uint4*>(planes + 2 * plane + o) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
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

}  // namespace

int tc_max_groups() { return MAX_GROUPS; }

int launch_split_bf16x3(const float* X, int64_t sr, int64_t sk, int rows, int K, int rows_pad, int k_pad, void* planes,
                        void* stream, std::string& why)
{
    if (sk == 1 && sr % 4 == 0 && reinterpret_cast<uintptr_t>(X) % 16 == 0 && k_pad % 8 == 0 &&
        reinterpret_cast<uintptr_t>(planes) % 16 == 0 && rows_pad <= 65535) {
        dim3 grid((unsigned)((k_pad / 8 + 255) / 256), (unsigned)rows_pad);
        split_bf16x3_rows_kernel<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(
            X, sr, rows, K, rows_pad, k_pad, static_cast<__nv_bfloat16*>(planes));
    } else {
        dim3 grid((unsigned)((k_pad + ST - 1) / ST), (unsigned)((rows_pad + ST - 1) / ST));
        split_bf16x3_kernel<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(
            X, sr, sk, rows, K, rows_pad, k_pad, static_cast<__nv_bfloat16*>(planes));
    }
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
        cudaFuncSetAttribute(tc_terms_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
        cudaFuncSetAttribute(tc_terms_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
        g_sms = device_sm_count();
    });
    if (P.kblock != BK) { why = "only 64-wide K blocks are built"; return OOC_ERR_INVALID_ARG; }
    const uint32_t B_TILE = BN * BK * 2u;
    TcArgs a;
    std::memset(&a, 0, sizeof(a));
    a.M = (int)P.M; a.N = (int)P.N;
    if (P.k_pad % BK || P.chunk % BK) { why = "K padding / chunk not a multiple of the K block"; return OOC_ERR_INVALID_ARG; }
    a.kblocks = (int)(P.k_pad / BK);
    a.chunk_kblocks = std::max(1, P.chunk / BK);
    a.nchunks = (a.kblocks + a.chunk_kblocks - 1) / a.chunk_kblocks;
    a.small_every = std::max(1, kSmallK / (a.chunk_kblocks * BK));
    a.ngroups = P.ngroups;
    a.tiles_n = (int)((P.N + BN - 1) / BN);
    a.tiles_m = (int)((P.M + BM - 1) / BM);
    a.tiles = a.tiles_m * a.tiles_n;
    uint32_t max_stage = 0;
    for (int g = 0; g < P.ngroups; ++g) {
        const TcGroupSpec& s = P.groups[g];
        TcGroup& d = a.g[g];
        if (s.na < 1 || s.na > 4 || s.nb < 1 || s.nb > 4 || s.np < 1 || s.np > 6) {
            why = "bad group shape";
            return OOC_ERR_INVALID_ARG;
        }
        for (int q = 0; q < s.np; ++q)
            if (s.pa[q] < 0 || s.pa[q] >= s.na || s.pb[q] < 0 || s.pb[q] >= s.nb) {
                why = "group pair index outside its loaded planes";
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
        if (P.df32 && (!P.c_fp32 || (double)(float)P.alpha != P.alpha || (double)(float)P.beta != P.beta)) {
            why = "the BF16x3 form writes FP32 C with FP32 alpha and beta";
            return OOC_ERR_INVALID_ARG;
        }
        if (!P.df32 && (s.scale_exp < -896 || s.scale_exp > 1000 || s.scale_exp2 < -896 || s.scale_exp2 > 1000)) {
            why = "digit weight outside the drain's exponent range";
            return OOC_ERR_INVALID_ARG;
        }
        max_stage = std::max(max_stage, (uint32_t)s.na * A_TILE + (uint32_t)s.nb * B_TILE);
    }
    a.stage_bytes = max_stage;
    a.nstages = std::min<int>(MAX_STAGES, (int)(RING_BYTES / a.stage_bytes));
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
        int rc = encode_map_3d_bf16(&ma, P.a_planes, (uint64_t)P.k_pad, (uint64_t)P.a_rows_pad,
                                    (uint64_t)P.a_nplanes, BK, BM, why);
        if (rc) return rc;
        rc = encode_map_3d_bf16(&mb, P.b_planes, (uint64_t)P.k_pad, (uint64_t)P.b_rows_pad, (uint64_t)P.b_nplanes,
                                BK, BN, why);
        if (rc) return rc;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int grid = std::min(a.tiles, g_sms > 0 ? g_sms : 152);
    if (P.df32) tc_terms_kernel<true><<<grid, THREADS, SMEM_BYTES, st>>>(ma, mb, a);
    else tc_terms_kernel<false><<<grid, THREADS, SMEM_BYTES, st>>>(ma, mb, a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { why = std::string("tc_terms launch: ") + cudaGetErrorString(e); return OOC_ERR_CUDA; }
    return OOC_OK;
}

}  // namespace ooc
