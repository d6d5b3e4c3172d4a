// Executor and C ABI of the pipeline-description language (pipe.cpp): binds
// host operands and variables, compiles the description, and issues the
// compiled copies, kernels and events on three streams in one device arena.
#include <cuda_runtime.h>

#include <chrono>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "ooc_internal.hpp"

struct ooc_pipe {
    std::shared_ptr<ooc::PipeSource> src;
    std::vector<ooc::PipeOperand> operands;
    std::map<std::string, double> vars;
};

namespace ooc {

namespace {

int fail(int code, const std::string& msg)
{
    set_error(msg);
    return code;
}

// Y = a X + b Y over a rows x cols tile (Y not read when it is fresh or b == 0)
__global__ void axpby_kernel(double* Y, int64_t ldy, const double* X, int64_t ldx, int64_t rows, int64_t cols,
                             double a, double b, int read_y)
{
    const int64_t n = rows * cols;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / cols, c = i % cols;
        double v = a * X[r * ldx + c];
        if (read_y) v += b * Y[r * ldy + c];
        Y[r * ldy + c] = v;
    }
}

double var(const std::map<std::string, double>& v, const char* name, double dflt)
{
    auto it = v.find(name);
    return it == v.end() ? dflt : it->second;
}

int compile(ooc_pipe* p, PipeProgram& prog)
{
    std::string why;
    const int rc = pipe_compile(*p->src, p->operands, p->vars, prog, why);
    if (rc) return fail(rc, why);
    return OOC_OK;
}

struct Run {
    char* arena = nullptr;
    cudaStream_t st[3] = {nullptr, nullptr, nullptr};
    std::vector<cudaEvent_t> ev, kev;
    cudaEvent_t t0 = nullptr, t1[3] = {nullptr, nullptr, nullptr};
    ~Run() { release(); }
    void release()
    {
        for (auto s : st)
            if (s) cudaStreamSynchronize(s);
        for (auto& e : ev) { if (e) cudaEventDestroy(e); e = nullptr; }
        for (auto& e : kev) { if (e) cudaEventDestroy(e); e = nullptr; }
        if (t0) cudaEventDestroy(t0);
        t0 = nullptr;
        for (auto& e : t1) { if (e) cudaEventDestroy(e); e = nullptr; }
        for (auto& s : st) { if (s) cudaStreamDestroy(s); s = nullptr; }
        if (arena) cudaFree(arena);
        arena = nullptr;
        cudaGetLastError();
    }
};

#define PCK(call)                                                                                          \
    do {                                                                                                   \
        cudaError_t e_ = (call);                                                                           \
        if (e_ != cudaSuccess) return fail(OOC_ERR_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
    } while (0)

}  // namespace

}  // namespace ooc

using namespace ooc;

int ooc_pipe_create(const char* spec, ooc_pipe** out)
{
    if (!spec || !out) return fail(OOC_ERR_INVALID_ARG, "null description or result pointer");
    *out = nullptr;
    std::unique_ptr<ooc_pipe> p(new ooc_pipe());
    std::vector<std::string> names;
    std::string why;
    const int rc = pipe_parse(spec, p->src, names, why);
    if (rc) return fail(rc, why);
    for (const auto& n : names) {
        PipeOperand o;
        o.name = n;
        p->operands.push_back(o);
    }
    *out = p.release();
    return OOC_OK;
}

int ooc_pipe_set(ooc_pipe* p, const char* name, double value)
{
    if (!p || !name || !*name) return fail(OOC_ERR_INVALID_ARG, "null pipeline or variable name");
    p->vars[name] = value;
    return OOC_OK;
}

int ooc_pipe_bind(ooc_pipe* p, const char* operand, void* host, int64_t rows, int64_t cols, int64_t ld,
                  int32_t elem_bytes)
{
    if (!p || !operand) return fail(OOC_ERR_INVALID_ARG, "null pipeline or operand name");
    if (rows < 1 || cols < 1 || ld < cols || (elem_bytes != 4 && elem_bytes != 8))
        return fail(OOC_ERR_INVALID_ARG, "bad operand dimensions, leading dimension or element size");
    for (auto& o : p->operands)
        if (o.name == operand) {
            o.host = host;
            o.rows = rows; o.cols = cols; o.ld = ld; o.es = elem_bytes;
            o.bound = true;
            return OOC_OK;
        }
    return fail(OOC_ERR_INVALID_ARG, std::string("the description declares no operand '") + operand + "'");
}

int ooc_pipe_schedule(ooc_pipe* p, size_t device_budget_bytes, ooc_stats* plan, ooc_sched_op* out, int64_t capacity,
                      int64_t* count)
{
    if (!p || !count) return fail(OOC_ERR_INVALID_ARG, "null pipeline or count");
    PipeProgram prog;
    int rc = compile(p, prog);
    if (rc) return rc;
    if (prog.device_bytes > device_budget_bytes)
        return fail(OOC_ERR_BUDGET, "the rings take " + std::to_string(prog.device_bytes) + " bytes");
    if (plan) {
        std::memset(plan, 0, sizeof(*plan));
        plan->device_bytes = (int64_t)prog.device_bytes;
        for (const Op& o : prog.ops) {
            plan->steps += o.kind == kKernel;
            if (o.kind == kH2D) {
                const PipeOperand& x = prog.operands[o.wtag.m];
                plan->h2d_bytes += (double)x.tile_rows(o.wtag.r) * x.tile_cols(o.wtag.c) * x.es;
            } else if (o.kind == kD2H) {
                const PipeOperand& x = prog.operands[o.rtag[0].m];
                plan->d2h_bytes += (double)x.tile_rows(o.rtag[0].r) * x.tile_cols(o.rtag[0].c) * x.es;
                ++plan->blocks;
            }
        }
    }
    *count = (int64_t)prog.ops.size();
    if (!out || capacity < *count) return fail(OOC_ERR_CAPACITY, "schedule needs more entries");
    for (size_t n = 0; n < prog.ops.size(); ++n) {
        const Op& o = prog.ops[n];
        ooc_sched_op& d = out[n];
        d.kind = o.kind; d.stream = o.stream; d.event = o.event; d.nreads = o.nr;
        d.write_slot = o.wslot;
        const int64_t wt[4] = {o.wtag.m, o.wtag.r, o.wtag.c, o.wtag.v};
        std::memcpy(d.write_tag, wt, sizeof(wt));
        for (int r = 0; r < 3; ++r) {
            d.read_slot[r] = o.rslot[r];
            const int64_t rt[4] = {o.rtag[r].m, o.rtag[r].r, o.rtag[r].c, o.rtag[r].v};
            std::memcpy(d.read_tag[r], rt, sizeof(rt));
        }
    }
    return OOC_OK;
}

int ooc_pipe_run(ooc_pipe* p, size_t device_budget_bytes, ooc_stats* stats)
{
    const auto th0 = std::chrono::steady_clock::now();
    if (stats) std::memset(stats, 0, sizeof(*stats));
    if (!p) return fail(OOC_ERR_INVALID_ARG, "null pipeline");
    std::string why;
    int rc = device_check(why);
    if (rc) return fail(rc, why);
    PipeProgram prog;
    if ((rc = compile(p, prog))) return rc;
    if (prog.device_bytes > device_budget_bytes)
        return fail(OOC_ERR_BUDGET, "the rings take " + std::to_string(prog.device_bytes) + " bytes");
    for (const PipeOperand& o : prog.operands)
        if (!o.host || !host_range_pinned(o.host, o.rows, o.cols, o.ld, o.es))
            return fail(OOC_ERR_NOT_PINNED, "operand " + o.name + " is not bound to page-locked host memory");
    const double alpha = var(p->vars, "alpha", 1.0), beta = var(p->vars, "beta", 0.0);
    const double a = var(p->vars, "a", 1.0), b = var(p->vars, "b", 1.0);
    Run x;
    if (cudaMalloc(&x.arena, prog.device_bytes) != cudaSuccess) {
        cudaGetLastError();
        x.arena = nullptr;
        return fail(OOC_ERR_ALLOC, "device arena of " + std::to_string(prog.device_bytes) + " bytes");
    }
    for (auto& s : x.st) PCK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    x.ev.assign(prog.events, nullptr);
    for (auto& e : x.ev) PCK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    int64_t nk = 0;
    for (const Op& o : prog.ops) nk += o.kind == kKernel;
    x.kev.assign(2 * nk, nullptr);
    for (auto& e : x.kev) PCK(cudaEventCreate(&e));
    PCK(cudaEventCreate(&x.t0));
    for (auto& e : x.t1) PCK(cudaEventCreate(&e));
    int* err = reinterpret_cast<int*>(x.arena);
    PCK(cudaEventRecord(x.t0, x.st[kStreamH2D]));
    PCK(cudaStreamWaitEvent(x.st[kStreamCompute], x.t0, 0));
    PCK(cudaStreamWaitEvent(x.st[kStreamD2H], x.t0, 0));
    PCK(cudaMemsetAsync(err, 0, sizeof(int), x.st[kStreamCompute]));
    double h2d = 0, d2h = 0;
    int64_t kn = 0, launches = 0;
    auto dev = [&](int slot) { return x.arena + prog.slot_off[slot]; };
    for (const Op& o : prog.ops) {
        cudaStream_t s = x.st[o.stream];
        switch (o.kind) {
        case kRecord: PCK(cudaEventRecord(x.ev[o.event], s)); break;
        case kWait: PCK(cudaStreamWaitEvent(s, x.ev[o.event], 0)); break;
        case kH2D:
        case kD2H: {
            const Tag& t = o.kind == kH2D ? o.wtag : o.rtag[0];
            const int slot = o.kind == kH2D ? o.wslot : o.rslot[0];
            const PipeOperand& op = prog.operands[t.m];
            const int64_t rows = op.tile_rows(t.r), cols = op.tile_cols(t.c);
            char* host = static_cast<char*>(op.host) + (t.r * op.tr * op.ld + t.c * op.tc) * op.es;
            if (o.kind == kH2D) {
                PCK(cudaMemcpy2DAsync(dev(slot), op.ld_dev * op.es, host, op.ld * op.es, cols * op.es, rows,
                                      cudaMemcpyHostToDevice, s));
                h2d += (double)rows * cols * op.es;
            } else {
                PCK(cudaMemcpy2DAsync(host, op.ld * op.es, dev(slot), op.ld_dev * op.es, cols * op.es, rows,
                                      cudaMemcpyDeviceToHost, s));
                d2h += (double)rows * cols * op.es;
            }
            break;
        }
        case kKernel: {
            PCK(cudaEventRecord(x.kev[2 * kn], s));
            const PipeOperand& Y = prog.operands[o.wtag.m];
            const int64_t rows = Y.tile_rows(o.wtag.r), cols = Y.tile_cols(o.wtag.c);
            // inputs follow the output in the read list unless the output is fresh
            const int in0 = o.mode == kPipeFresh ? 0 : 1;
            if (o.kernel == kPipeGemm) {
                const PipeOperand& A = prog.operands[o.rtag[in0].m];
                const PipeOperand& B = prog.operands[o.rtag[in0 + 1].m];
                const int64_t k = A.tile_cols(o.rtag[in0].c);
                const bool read_c = o.mode == kPipeAccumulate || (o.mode == kPipeLoaded && beta != 0.0);
                const double beta_eff = o.mode == kPipeAccumulate ? 1.0 : beta;
                rc = launch_fp64_tile(true, false, rows, cols, k, alpha,
                                      reinterpret_cast<const double*>(dev(o.rslot[in0])), A.ld_dev,
                                      reinterpret_cast<const double*>(dev(o.rslot[in0 + 1])), B.ld_dev, beta_eff,
                                      read_c, reinterpret_cast<double*>(dev(o.wslot)), Y.ld_dev, err, s, why);
                if (rc) return fail(rc, why);
            } else {
                const PipeOperand& X = prog.operands[o.rtag[in0].m];
                const int read_y = o.mode != kPipeFresh && b != 0.0;
                axpby_kernel<<<608, 256, 0, s>>>(reinterpret_cast<double*>(dev(o.wslot)), Y.ld_dev,
                                                 reinterpret_cast<const double*>(dev(o.rslot[in0])), X.ld_dev, rows,
                                                 cols, a, b, read_y);
                PCK(cudaGetLastError());
            }
            ++launches;
            PCK(cudaEventRecord(x.kev[2 * kn + 1], s));
            ++kn;
            break;
        }
        }
    }
    for (int i = 0; i < 3; ++i) PCK(cudaEventRecord(x.t1[i], x.st[i]));
    for (auto s : x.st) PCK(cudaStreamSynchronize(s));
    int herr = 0;
    PCK(cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost));
    if (herr) return fail(OOC_ERR_TIMEOUT, "a device-side wait gave up (status " + std::to_string(herr) + ")");
    if (stats) {
        float ms = 0, best = 0;
        for (auto e : x.t1) {
            PCK(cudaEventElapsedTime(&ms, x.t0, e));
            best = std::max(best, ms);
        }
        double ks = 0;
        for (int64_t k = 0; k < kn; ++k) {
            PCK(cudaEventElapsedTime(&ms, x.kev[2 * k], x.kev[2 * k + 1]));
            ks += ms;
        }
        stats->device_seconds = best * 1e-3;
        stats->kernel_seconds = ks * 1e-3;
        stats->h2d_bytes = h2d;
        stats->d2h_bytes = d2h;
        stats->steps = kn;
        stats->device_bytes = (int64_t)prog.device_bytes;
        stats->kernel_launches = launches;
    }
    x.release();  // the arena free is part of the call
    if (stats) stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - th0).count();
    return OOC_OK;
}

int ooc_pipe_free(ooc_pipe* p)
{
    delete p;
    return OOC_OK;
}
