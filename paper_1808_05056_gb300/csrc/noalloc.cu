// ooc_dgemm_noalloc: the out-of-core FP64 GEMM for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc: a process whose device memory is
// entirely owned by another allocator (a framework's caching allocator that
// has reserved the pool, where an extra cudaMalloc fails or fragments it), or
// a latency-bound caller that cannot take the device-wide synchronisation a
// cudaFree implies.  This entry point needs no allocation of any kind: its
// operand slots live in one file-scope device array of fixed size, and all
// work is issued, in order, on the caller's stream (no streams or events are
// created, so copies do not overlap the tile kernels here).
//
// The array is kNoallocArenaBytes (32 MiB); every GPU that loads the library
// holds it until the process exits.  The device budget of a call must not
// exceed it (larger budgets are rejected with OOC_ERR_INVALID_ARG).
//
// Set-up: the first call on a device (with that device current) looks up the
// array's device address with cudaGetSymbolAddress and caches it; make that
// first call before any stream capture begins.  The cached address belongs to
// the device's primary context: after cudaDeviceReset (or any other reset of
// that context) the library must not be called again in the process.  All calls share the array and
// it keeps the last call's contents: the call clears the error word it needs
// at zero, and the plan never reads a slot before writing it.  Calls that
// overlap on the GPU (on different streams, or from several host threads)
// race on the array; serialise them.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "ooc_internal.hpp"

namespace {

constexpr size_t kNoallocArenaBytes = OOC_NOALLOC_MAX_BYTES;

static __device__ __align__(256) unsigned char g_noalloc_arena[kNoallocArenaBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_arena_ptr[kMaxDevices] = {nullptr};

int arena_for_current_device(char** out, std::string& why)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        why = "no current CUDA device";
        return OOC_ERR_NO_DEVICE;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_arena_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_arena);
        if (e != cudaSuccess || !p) {
            why = std::string("cudaGetSymbolAddress(no-alloc arena): ") + cudaGetErrorString(e);
            cudaGetLastError();
            return OOC_ERR_CUDA;
        }
        g_arena_ptr[dev] = p;
    }
    *out = static_cast<char*>(g_arena_ptr[dev]);
    return OOC_OK;
}

bool pinned_ptr(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

bool pinned_range(const void* base, int64_t rows, int64_t cols, int64_t ld)
{
    if (rows <= 0 || cols <= 0) return true;
    const char* b = static_cast<const char*>(base);
    return pinned_ptr(b) && pinned_ptr(b + ((rows - 1) * ld + cols - 1) * 8);
}

int noalloc_fail(int code, const std::string& msg)
{
    ooc::set_error(msg);
    return code;
}

}  // namespace

extern "C" int ooc_dgemm_noalloc(char transA, char transB, int64_t M, int64_t N, int64_t K, double alpha,
                                 const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
                                 double* C, int64_t ldc, size_t device_budget_bytes, void* stream)
{
    using namespace ooc;
    const bool ta = transA == 'T' || transA == 't', tb = transB == 'T' || transB == 't';
    if (!(ta || transA == 'N' || transA == 'n') || !(tb || transB == 'N' || transB == 'n'))
        return noalloc_fail(OOC_ERR_INVALID_ARG, "trans must be 'N' or 'T'");
    if (M < 0 || N < 0 || K < 0) return noalloc_fail(OOC_ERR_INVALID_ARG, "negative dimension");
    if (lda < std::max<int64_t>(1, ta ? M : K) || ldb < std::max<int64_t>(1, tb ? K : N) ||
        ldc < std::max<int64_t>(1, N))
        return noalloc_fail(OOC_ERR_INVALID_ARG, "leading dimension below the row width");
    if (device_budget_bytes > kNoallocArenaBytes)
        return noalloc_fail(OOC_ERR_INVALID_ARG,
                            "ooc_dgemm_noalloc: device budget " + std::to_string(device_budget_bytes) +
                                " exceeds the fixed no-alloc arena of " + std::to_string(kNoallocArenaBytes) +
                                " bytes");
    if (M == 0 || N == 0) return OOC_OK;
    if ((K > 0 && (!A || !B)) || !C) return noalloc_fail(OOC_ERR_INVALID_ARG, "null operand pointer");
    std::string why;
    int rc = device_check(why);
    if (rc) return noalloc_fail(rc, why);
    if (!pinned_range(A, ta ? K : M, ta ? M : K, lda) || !pinned_range(B, tb ? N : K, tb ? K : N, ldb) ||
        !pinned_range(C, M, N, ldc))
        return noalloc_fail(OOC_ERR_NOT_PINNED, "host operands must be page-locked");

    char* arena = nullptr;
    rc = arena_for_current_device(&arena, why);
    if (rc) return noalloc_fail(rc, why);

    ooc_opts opts;
    std::memset(&opts, 0, sizeof(opts));
    opts.form = OOC_FORM_FP64;
    PlanRequest rq{M, N, K, 8, beta != 0.0, ta, tb, device_budget_bytes, opts};
    rq.lda = lda; rq.ldb = ldb; rq.ldc = ldc;
    Plan p;
    rc = make_plan(rq, p, why);
    if (rc) return noalloc_fail(rc, why);
    if (p.device_bytes > kNoallocArenaBytes) return noalloc_fail(OOC_ERR_BUDGET, "plan exceeds the no-alloc arena");
    p.b_prefetch = false;  // one stream: copies cannot run ahead of the kernels anyway
    std::vector<Op> ops;
    build_schedule(p, ops);

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int* err = reinterpret_cast<int*>(arena);
    if (cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess)
        return noalloc_fail(OOC_ERR_CUDA, "clearing the error word");
    const char* hA = reinterpret_cast<const char*>(A);
    const char* hB = reinterpret_cast<const char*>(B);
    char* hC = reinterpret_cast<char*>(C);
    const int64_t es = 8;
    // One stream: issue order is execution order, so the schedule's event
    // records and waits are already satisfied and are skipped.
    for (const Op& op : ops) {
        cudaError_t e = cudaSuccess;
        if (op.kind == kH2D) {
            const Tag& t = op.wtag;
            char* dst = arena + slot_offset(p, op.wslot);
            const char* src;
            int64_t rows, width, spitch, dpitch;
            if (t.m == kMatA) {
                const int64_t r0 = t.r * p.mb, k0 = t.c * p.kb, mr = p.rows_of(t.r), kr = p.k_of(t.c);
                if (!p.ta) { src = hA + (r0 * lda + k0) * es; rows = mr; width = kr; }
                else { src = hA + (k0 * lda + r0) * es; rows = kr; width = mr; }
                spitch = lda * es; dpitch = p.lda_dev * es;
            } else if (t.m == kMatB) {
                const int64_t k0 = t.r * p.kb, c0 = t.c * p.nb, kr = p.k_of(t.r), nc = p.cols_of(t.c);
                if (!p.tb) { src = hB + (k0 * ldb + c0) * es; rows = kr; width = nc; }
                else { src = hB + (c0 * ldb + k0) * es; rows = nc; width = kr; }
                spitch = ldb * es; dpitch = p.ldb_dev * es;
            } else {
                src = hC + (t.r * p.mb * ldc + t.c * p.nb) * es;
                rows = p.rows_of(t.r); width = p.cols_of(t.c);
                spitch = ldc * es; dpitch = p.ldc_dev * es;
            }
            if (rows > 0 && width > 0)
                e = cudaMemcpy2DAsync(dst, dpitch, src, spitch, width * es, rows, cudaMemcpyHostToDevice, st);
        } else if (op.kind == kKernel) {
            int sa = -1, sb = -1;
            for (int r = 0; r < op.nr; ++r) {
                if (op.rslot[r] < p.nA) sa = op.rslot[r];
                else if (op.rslot[r] < p.nA + p.nB) sb = op.rslot[r];
            }
            const int64_t kk = p.K > 0 ? p.k_of(op.kc) : 0;
            const double* dA = sa >= 0 ? reinterpret_cast<const double*>(arena + slot_offset(p, sa)) : nullptr;
            const double* dB = sb >= 0 ? reinterpret_cast<const double*>(arena + slot_offset(p, sb)) : nullptr;
            double* dC = reinterpret_cast<double*>(arena + slot_offset(p, op.wslot));
            rc = launch_fp64_tile(!p.ta, p.tb, p.rows_of(op.i), p.cols_of(op.j), kk, alpha, dA, p.lda_dev, dB,
                                  p.ldb_dev, op.first ? beta : 1.0, !op.first || beta != 0.0, dC, p.ldc_dev, err, st,
                                  why);
            if (rc) {
                cudaStreamSynchronize(st);
                return noalloc_fail(rc, why);
            }
        } else if (op.kind == kD2H) {
            const int64_t rows = p.rows_of(op.i), width = p.cols_of(op.j);
            char* dst = hC + (op.i * p.mb * ldc + op.j * p.nb) * es;
            const char* src = arena + slot_offset(p, op.rslot[0]);
            e = cudaMemcpy2DAsync(dst, ldc * es, src, p.ldc_dev * es, width * es, rows, cudaMemcpyDeviceToHost, st);
        }
        if (e != cudaSuccess) {
            cudaStreamSynchronize(st);
            return noalloc_fail(OOC_ERR_CUDA, std::string("ooc_dgemm_noalloc copy: ") + cudaGetErrorString(e));
        }
    }
    // the error word is read on the caller's stream, behind the last kernel,
    // into pageable host memory (the copy completes before the synchronize returns)
    int herr = 0;
    if (cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) {
        cudaStreamSynchronize(st);
        return noalloc_fail(OOC_ERR_CUDA, "reading the error word");
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) return noalloc_fail(OOC_ERR_CUDA, "stream synchronize");
    if (herr) return noalloc_fail(OOC_ERR_TIMEOUT, "a device-side wait gave up");
    return OOC_OK;
}
