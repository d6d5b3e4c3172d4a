// Device-side building blocks shared by the tile kernels: mbarrier waits with
// a time limit, TMA tile loads, and the global error flag they report to.
//
// Every spin-wait here is bounded: after kWaitLimitNs of wall time (read from
// %globaltimer) the waiting thread records a status in the launch's error
// word and returns false, so a lost arrival ends the kernel with an error the
// host reads instead of a hung GPU.
#pragma once
#include <cstdint>
#include <cuda.h>

namespace ooc {

constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s per wait

// status values written to the error word (host maps any nonzero to OOC_ERR_TIMEOUT)
constexpr int kErrWaitFull = 1;
constexpr int kErrWaitEmpty = 2;
constexpr int kErrWaitMma = 3;
constexpr int kErrWaitAcc = 4;
constexpr int kErrGridBarrier = 5;

__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait until the phase with the given parity has completed.  Returns false
// (after recording `code` in *err) when the limit passes or when another
// thread of the launch has already reported an error.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err, int code)
{
    const uint32_t a = smem_u32(bar);
#pragma unroll 1
    for (int i = 0; i < 128; ++i)
        if (mbar_try_wait(a, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
#pragma unroll 1
    while (true) {
        if (mbar_try_wait(a, parity)) return true;
        if (*reinterpret_cast<volatile int*>(err) != 0) return false;
        if (globaltimer_ns() - t0 > kWaitLimitNs) {
            atomicCAS(err, 0, code);
            return false;
        }
    }
}

// mbar_wait for threads that are not on the critical path (the epilogue warps
// of the tile kernels): between unsuccessful tries the warp sleeps, so that
// it does not take issue slots from the TMA and MMA threads of its SM while
// it waits.  Same limit and error reporting as mbar_wait.
__device__ __forceinline__ bool mbar_wait_backoff(uint64_t* bar, uint32_t parity, int* err, int code)
{
    const uint32_t a = smem_u32(bar);
    if (mbar_try_wait(a, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    uint32_t ns = 32;
#pragma unroll 1
    while (true) {
        __nanosleep(ns);
        if (mbar_try_wait(a, parity)) return true;
        if (ns < 256) ns <<= 1;
        if (*reinterpret_cast<volatile int*>(err) != 0) return false;
        if (globaltimer_ns() - t0 > kWaitLimitNs) {
            atomicCAS(err, 0, code);
            return false;
        }
    }
}

// 2-D TMA tile load into shared memory, completing on `bar` (transaction bytes).
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int32_t x, int32_t y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_prefetch_desc(const CUtensorMap* map)
{
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

__device__ __forceinline__ bool launch_failed(const int* err)
{
    return *reinterpret_cast<const volatile int*>(err) != 0;
}

}  // namespace ooc
