// Measured FP64 tensor-core peak of the current device (ooc_query_fp64_peak):
// the denominator of the plain form's roofline.  The paper quotes each
// device's FP64 peak beside its measured DGEMM rates (Section V); this
// measures the same quantity on the device the library runs on, with the same
// instruction the FP64 tile kernel uses (mma.sync m8n8k4 f64), fed from
// registers so that nothing but the FP64 pipe bounds it.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "ooc_internal.hpp"

namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;  // independent accumulators per warp (covers the MMA latency)

// Every warp runs `iters` rounds of kChains independent m8n8k4 FP64 MMAs
// (512 FLOP each); the sums are stored so that nothing is dead code.
__global__ void __launch_bounds__(kProbeThreads) dmma_probe_kernel(int iters, double* __restrict__ out)
{
    const double a = 1.0 + 1e-3 * (threadIdx.x & 31), b = 1.0 - 1e-3 * (threadIdx.x & 31);
    double d[kChains][2];
#pragma unroll
    for (int c = 0; c < kChains; ++c) d[c][0] = d[c][1] = 0.0;
#pragma unroll 1
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                         : "+d"(d[c][0]), "+d"(d[c][1])
                         : "d"(a), "d"(b));
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += d[c][0] + d[c][1];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int ooc_query_fp64_peak(double seconds, double* tflops)
{
    using namespace ooc;
    if (!tflops || !(seconds > 0.0) || seconds > 60.0) {
        set_error("ooc_query_fp64_peak: tflops must be non-null and seconds in (0, 60]");
        return OOC_ERR_INVALID_ARG;
    }
    std::string why;
    int rc = device_check(why);
    if (rc) {
        set_error(why);
        return rc;
    }
    const int sms = device_sm_count();
    const int grid = 2 * std::max(1, sms);
    double* out = nullptr;
    if (cudaMalloc(&out, sizeof(double) * (size_t)grid * kProbeThreads) != cudaSuccess) {
        cudaGetLastError();
        set_error("ooc_query_fp64_peak: probe output");
        return OOC_ERR_ALLOC;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaStream_t st = nullptr;
    double best = 0.0;
    rc = OOC_OK;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess) {
        rc = OOC_ERR_CUDA;
    } else {
        // size the launch from a short one, then take the best of the timed launches
        int iters = 1 << 12;
        const double flop_per_iter = (double)grid * (kProbeThreads / 32) * kChains * 512.0;
        double spent = 0.0;
        for (int rep = 0; rep < 64 && rc == OOC_OK; ++rep) {
            cudaEventRecord(e0, st);
            dmma_probe_kernel<<<grid, kProbeThreads, 0, st>>>(iters, out);
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                rc = OOC_ERR_CUDA;
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            const double s = ms * 1e-3;
            spent += s;
            if (s < 0.05 && iters < (1 << 26)) {  // too short to time well: grow, do not count it
                iters *= 4;
                continue;
            }
            best = std::max(best, flop_per_iter * iters / s / 1e12);
            if (spent >= seconds) break;
        }
        if (rc == OOC_OK && cudaGetLastError() != cudaSuccess) rc = OOC_ERR_CUDA;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    cudaFree(out);
    if (rc) {
        set_error("ooc_query_fp64_peak: probe launch failed");
        return rc;
    }
    *tflops = best;
    return OOC_OK;
}
