// C ABI of libooc (declared in include/ooc.h): argument checks, the
// out-of-core executor that issues a planned schedule on three CUDA streams
// (H2D copy engine, compute, D2H copy engine) with events, and the in-core
// device entry point.
//
// The executor follows Section IV of the libhclooc paper: the stages S(b_j),
// S(a_i), S(c_ij), the block GEMM and R(c_ij) are asynchronous operations
// ordered only by recorded/waited events, so copies in both directions run
// on the copy engines while the tile kernels run.  Unlike the paper's two
// round-robin streams, each direction and the compute have their own stream,
// and the slot ring may be deeper than two.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "ooc_internal.hpp"

namespace ooc {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

int device_sm_count()
{
    static int sms = -1;
    static std::once_flag once;
    std::call_once(once, [] {
        int dev = 0, n = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && n > 0)
            sms = n;
        else {
            cudaGetLastError();
            sms = 152;  // GB300 (planning without a device)
        }
    });
    return sms;
}

// ------------------------------------------------------------ tensor maps --
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

int encode_map_2d(void* map_out, int dtype, const void* base, uint64_t inner, uint64_t outer, uint64_t ld_elems,
                  uint32_t box_inner, uint32_t box_outer, int swizzle128, std::string& why)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn) {
        why = "cuTensorMapEncodeTiled unavailable";
        return OOC_ERR_CUDA;
    }
    CUtensorMapDataType dt = dtype == 0   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                             : dtype == 1 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                          : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const uint64_t es = dtype == 0 ? 8 : dtype == 1 ? 2 : 4;
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {ld_elems * es};
    cuuint32_t box[2] = {box_inner, box_outer};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(reinterpret_cast<CUtensorMap*>(map_out), dt, 2, const_cast<void*>(base), dims, strides, box,
                    estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        why = "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")";
        return OOC_ERR_CUDA;
    }
    return OOC_OK;
}

// installed schedule cost model (ooc_costmodel_set)
static std::mutex g_model_mu;
static std::vector<float> g_model;

bool costmodel_get(std::vector<float>& params)
{
    std::lock_guard<std::mutex> lk(g_model_mu);
    if (g_model.empty()) return false;
    params = g_model;
    return true;
}

void costmodel_set(const float* params, int64_t n)
{
    std::lock_guard<std::mutex> lk(g_model_mu);
    if (!params || n <= 0) g_model.clear();
    else g_model.assign(params, params + n);
}

int encode_map_3d_bf16(void* map_out, const void* base, uint64_t inner, uint64_t rows, uint64_t planes,
                       uint32_t box_inner, uint32_t box_rows, std::string& why)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn) {
        why = "cuTensorMapEncodeTiled unavailable";
        return OOC_ERR_CUDA;
    }
    cuuint64_t dims[3] = {inner, rows, planes};
    cuuint64_t strides[2] = {inner * 2, inner * rows * 2};
    cuuint32_t box[3] = {box_inner, box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(reinterpret_cast<CUtensorMap*>(map_out), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3,
                    const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    box_inner * 2 == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        why = "cuTensorMapEncodeTiled (3-D bf16) failed (" + std::to_string((int)r) + ")";
        return OOC_ERR_CUDA;
    }
    return OOC_OK;
}

// The Ozaki groups of the tensor-core kernel: digit products (s, t) with
// s + t <= S + 1, two consecutive t per group so that the group loads the A
// plane s once; each product's exact FP32 sum is weighted 2^(-beta (s + t)).
// Groups sharing a pair of B planes run back to back (t outer, s inner): the
// tiles in flight then re-read those B planes from L2 rather than DRAM.
void ozaki_groups(TcProblem& P, int S)
{
    int n = 0;
    for (int t1 = 1; t1 <= S; t1 += 2)
        for (int s1 = 1; s1 <= S + 1 - t1; ++s1) {
            TcGroupSpec& g = P.groups[n++];
            const bool two = t1 + 1 <= S + 1 - s1;
            g.na = 1; g.nb = two ? 2 : 1; g.np = two ? 2 : 1;
            g.aplane[0] = s1 - 1;
            g.bplane[0] = t1 - 1; g.bplane[1] = two ? t1 : 0;
            g.pa[0] = 0; g.pb[0] = 0;
            g.pa[1] = 0; g.pb[1] = 1;
            g.scale_exp = -kOzakiBeta * (s1 + t1);
            g.scale_exp2 = -kOzakiBeta * (s1 + t1 + 1);
        }
    P.ngroups = n;
}

namespace {
size_t al256(size_t x) { return (x + 255) / 256 * 256; }
int64_t up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }
size_t side_bytes(int64_t rows, int64_t k_pad, int S)
{
    const int64_t rp = up(std::max<int64_t>(rows, 1), 128);
    return al256((size_t)S * rp * k_pad * 2) + al256((size_t)rp * 4) + al256((size_t)rp * 8);
}
}  // namespace

size_t ozaki_device_scratch(int64_t M, int64_t N, int64_t K, int S)
{
    const int64_t k_pad = up(std::max<int64_t>(K, 1), 64);
    return side_bytes(M, k_pad, S) + side_bytes(N, k_pad, S);
}

int ozaki_gemm_device(bool a_kmajor, bool b_kmajor, int64_t M, int64_t N, int64_t K, double alpha, const double* A,
                      int64_t lda, const double* B, int64_t ldb, double beta, bool read_c, double* C, int64_t ldc,
                      int S, void* scratch, size_t scratch_bytes, int* err, void* stream, std::string& why, int tri,
                      int64_t tri_off)
{
    if (M <= 0 || N <= 0) return OOC_OK;
    if (K <= 0) return launch_fp64_tile(a_kmajor, b_kmajor, M, N, K, alpha, A, lda, B, ldb, beta, read_c, C, ldc,
                                        err, stream, why, tri, tri_off);
    if (S < 2 || S > kOzakiMaxSlices) {
        why = "Ozaki slice count out of range";
        return OOC_ERR_INVALID_ARG;
    }
    if (ozaki_device_scratch(M, N, K, S) > scratch_bytes) {
        why = "Ozaki scratch too small";
        return OOC_ERR_BUDGET;
    }
    const int64_t k_pad = up(K, 64);
    char* base = static_cast<char*>(scratch);
    struct Side {
        const double* X;
        int64_t rows, sr, sk;
        char* planes;
        int* exps;
        unsigned long long* rowmax;
        int64_t rows_pad;
    } side[2];
    side[0] = {A, M, a_kmajor ? lda : 1, a_kmajor ? 1 : lda, nullptr, nullptr, nullptr, up(M, 128)};
    side[1] = {B, N, b_kmajor ? ldb : 1, b_kmajor ? 1 : ldb, nullptr, nullptr, nullptr, up(N, 128)};
    for (auto& sd : side) {
        sd.planes = base;
        base += al256((size_t)S * sd.rows_pad * k_pad * 2);
        sd.exps = reinterpret_cast<int*>(base);
        base += al256((size_t)sd.rows_pad * 4);
        sd.rowmax = reinterpret_cast<unsigned long long*>(base);
        base += al256((size_t)sd.rows_pad * 8);
        const int rc = launch_split_ozaki(sd.X, sd.sr, sd.sk, (int)sd.rows, (int)K, (int)sd.rows_pad, (int)k_pad,
                                          S, kOzakiBeta, sd.planes, sd.exps, sd.rowmax, stream, why);
        if (rc) return rc;
    }
    TcProblem P;
    P.M = M; P.N = N; P.k_pad = k_pad;
    P.chunk = kOzakiChunk;
    P.a_planes = side[0].planes; P.a_rows_pad = side[0].rows_pad; P.a_nplanes = S;
    P.b_planes = side[1].planes; P.b_rows_pad = side[1].rows_pad; P.b_nplanes = S;
    ozaki_groups(P, S);
    P.row_exp = side[0].exps;
    P.col_exp = side[1].exps;
    P.alpha = alpha;
    P.beta = beta;
    P.read_c = read_c;
    P.c_fp32 = false;
    P.C = C;
    P.ldc = ldc;
    P.err = err;
    P.kblock = 64;
    P.tri = tri;
    P.tri_off = tri_off;
    return launch_tc_terms(P, stream, why);
}

}  // namespace ooc

using namespace ooc;

namespace {

bool is_n(char t) { return t == 'N' || t == 'n'; }
bool is_t(char t) { return t == 'T' || t == 't'; }

int fail(int code, const std::string& msg)
{
    set_error(msg);
    return code;
}

int check_device(std::string& why)
{
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) {
        cudaGetLastError();
        why = "no CUDA device";
        return OOC_ERR_NO_DEVICE;
    }
    int dev = 0, maj = 0, min = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&maj, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&min, cudaDevAttrComputeCapabilityMinor, dev);
    if (maj != 10 || min != 3) {
        why = "device is sm_" + std::to_string(maj) + std::to_string(min) + ", library is built for sm_103a";
        return OOC_ERR_NO_DEVICE;
    }
    return OOC_OK;
}

int validate(char ta, char tb, int64_t M, int64_t N, int64_t K, const void* A, int64_t lda, const void* B,
             int64_t ldb, const void* C, int64_t ldc, bool beta_nz, std::string& why)
{
    if (!(is_n(ta) || is_t(ta)) || !(is_n(tb) || is_t(tb))) {
        why = "trans must be 'N' or 'T'";
        return OOC_ERR_INVALID_ARG;
    }
    if (M < 0 || N < 0 || K < 0) {
        why = "negative dimension";
        return OOC_ERR_INVALID_ARG;
    }
    const int64_t a_cols = is_t(ta) ? M : K, b_cols = is_t(tb) ? K : N;
    if (lda < std::max<int64_t>(1, a_cols) || ldb < std::max<int64_t>(1, b_cols) || ldc < std::max<int64_t>(1, N)) {
        why = "leading dimension below the row width";
        return OOC_ERR_INVALID_ARG;
    }
    if (M == 0 || N == 0) return OOC_OK;  // quick return: no operand is touched
    if ((K > 0 && !A) || (K > 0 && !B) || !C) {
        why = "null operand pointer";
        return OOC_ERR_INVALID_ARG;
    }
    (void)beta_nz;
    return OOC_OK;
}

bool pinned(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

bool range_pinned(const void* base, int64_t rows, int64_t cols, int64_t ld, int es)
{
    if (rows <= 0 || cols <= 0) return true;
    const char* b = static_cast<const char*>(base);
    const char* last = b + ((rows - 1) * ld + cols - 1) * es;
    return pinned(b) && pinned(last);
}

// OOC_FAULT_INJECT=alloc | copy:<n> | kernel:<n> | devword  (host-side failures
// for tests; devword: ooc_dgemm_device leaves its error word nonzero after its
// launch, as a wait that gave up would)
struct Inject {
    bool alloc = false, devword = false;
    long copy = -1, kernel = -1;
    Inject()
    {
        const char* e = std::getenv("OOC_FAULT_INJECT");
        if (!e) return;
        std::string s(e);
        if (s == "alloc") alloc = true;
        else if (s == "devword") devword = true;
        else if (s.rfind("copy:", 0) == 0) copy = std::atol(s.c_str() + 5);
        else if (s.rfind("kernel:", 0) == 0) kernel = std::atol(s.c_str() + 7);
    }
};

struct Operands {
    const void* A;
    int64_t lda;
    const void* B;
    int64_t ldb;
    void* C;
    int64_t ldc;
    double alpha, beta;
};

// OOC_TRACE=<file>: append one CSV line per copy/kernel of each call with its
// stream, block indices, bytes, host issue time and device start/end (ms from
// the call's first event) -- the pipeline timeline of Section IV's Fig. 3.
struct TraceRec {
    int kind, stream;
    int64_t i, j, kc;
    double bytes, host_ms;
    cudaEvent_t e0, e1;
};

// Resources of one call, released in the destructor after the streams drain.
struct Exec {
    Plan p;
    char* arena = nullptr;     // device arena; its first word is the launch error word
    char* base = nullptr;      // base of the current plan's slot region inside the arena
    bool own_arena = false;
    bool own_streams = true;   // false: the streams belong to a session and outlive this call
    cudaStream_t st[3] = {nullptr, nullptr, nullptr};
    cudaStream_t extra_compute = nullptr;  // second half's streams (batched calls): compute,
    cudaStream_t extra_h2d = nullptr;      // host-to-device
    cudaStream_t extra_d2h = nullptr;      // and device-to-host copies
    cudaStream_t smap[3] = {nullptr, nullptr, nullptr};  // schedule stream id -> stream for the current plan
    int ev_base = 0;           // offset of the current plan's events in ev
    bool time_kernels = true;  // record timing events around tile launches (not inside graph capture)
    uint32_t flags = 0;        // ooc_opts.flags of the call
    double h2d = 0, d2h = 0;
    long n_copy = 0, n_kern = 0;
    std::vector<cudaEvent_t> ev;
    std::vector<cudaEvent_t> kev;  // timing pairs around tile kernels
    std::vector<cudaEvent_t> sev;   // staged plans: timing pairs around split ops
    long n_split = 0;
    std::vector<TraceRec> trace;
    int64_t launches = 0;                 // kernels launched by this call
    cudaEvent_t t_begin = nullptr, t_end[3] = {nullptr, nullptr, nullptr};

    Exec() = default;
    Exec(const Exec&) = delete;
    Exec& operator=(const Exec&) = delete;
    ~Exec() { release(); }

    void release()
    {
        for (auto s : st)
            if (s) cudaStreamSynchronize(s);
        for (auto& e : ev) { if (e) cudaEventDestroy(e); e = nullptr; }
        for (auto& e : kev) { if (e) cudaEventDestroy(e); e = nullptr; }
        for (auto& e : sev) { if (e) cudaEventDestroy(e); e = nullptr; }
        for (auto& r : trace) { if (r.e0) cudaEventDestroy(r.e0); if (r.e1) cudaEventDestroy(r.e1); }
        trace.clear();
        if (t_begin) cudaEventDestroy(t_begin);
        t_begin = nullptr;
        for (auto& e : t_end) { if (e) cudaEventDestroy(e); e = nullptr; }
        for (auto* e : {&extra_compute, &extra_h2d, &extra_d2h})
            if (*e) cudaStreamSynchronize(*e);
        for (auto& s : st) { if (s && own_streams) cudaStreamDestroy(s); s = nullptr; }
        for (auto* e : {&extra_compute, &extra_h2d, &extra_d2h}) {
            if (*e) cudaStreamDestroy(*e);
            *e = nullptr;
        }
        if (own_arena && arena) cudaFree(arena);
        arena = nullptr;
        own_arena = false;
        cudaGetLastError();
    }
};

#define CK(call)                                                                           \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) return fail(OOC_ERR_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
    } while (0)

// Tensor-core forms: split each newly loaded A / B slot into bf16 planes (once
// per load), then run the split-product tile kernel on the C block.
// Split the raw data at src_slot (a slot, or a staged plan's staging area) of
// operand A or B into the bf16 planes (and Ozaki row exponents) of dst_slot,
// on the compute stream.
int split_slot(const Plan& p, Exec& x, int src_slot, int dst_slot, bool is_a, int64_t nrows, int64_t K,
               std::string& why)
{
    const bool ozaki = p.form == OOC_FORM_OZAKI;
    const int S = split_planes(p);
    const int64_t k_pad = split_k_pad(p);
    const int64_t rpad = split_rows_pad(is_a ? p.mb : p.nb);
    void* st = x.smap[kStreamCompute];
    char* planes = x.base + slot_aux_offset(p, dst_slot);
    int* exps = reinterpret_cast<int*>(planes + split_planes_bytes(p, is_a ? p.mb : p.nb));
    // element (r, k) of the slot: K-major rows or K down the stored rows
    const bool kmajor = is_a ? !p.ta : p.tb;
    const int64_t ld = is_a ? p.lda_dev : p.ldb_dev;
    const int64_t sr = kmajor ? ld : 1, sk = kmajor ? 1 : ld;
    const char* src = x.base + slot_offset(p, src_slot);
    x.launches += ozaki ? (K > 0 ? 3 : 2) : 1;
    if (ozaki) {
        auto* rowmax = reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(exps) + ((rpad * 4 + 255) / 256) * 256);
        return launch_split_ozaki(reinterpret_cast<const double*>(src), sr, sk, (int)nrows, (int)K, (int)rpad,
                                  (int)k_pad, S, kOzakiBeta, planes, exps, rowmax, st, why);
    }
    return launch_split_bf16x3(reinterpret_cast<const float*>(src), sr, sk, (int)nrows, (int)K, (int)rpad, (int)k_pad,
                               planes, st, why);
}

// A tile of a split form: the contraction of the slots' planes (written by the
// schedule's split ops; split-form plans are always staged) into C slot sc.
int launch_split_tile(const Plan& p, const Op& op, Exec& x, const Operands& o, int sa, int sb, int sc,
                      std::string& why)
{
    if (!p.staged) {
        why = "split-form plan without staging areas";
        return OOC_ERR_INVALID_ARG;
    }
    const bool ozaki = p.form == OOC_FORM_OZAKI;
    const int S = split_planes(p);
    const int64_t rows = p.rows_of(op.i), cols = p.cols_of(op.j), K = p.K > 0 ? p.k_of(op.kc) : 0;  // this chunk
    const int64_t k_pad = split_k_pad(p);
    const int64_t ra_pad = split_rows_pad(p.mb), rb_pad = split_rows_pad(p.nb);
    int* err = reinterpret_cast<int*>(x.arena);
    struct Side {
        int slot;
        bool is_a;
    } sides[2] = {{sa, true}, {sb, false}};
    int* exps[2] = {nullptr, nullptr};
    char* planes[2] = {nullptr, nullptr};
    for (int q = 0; q < 2; ++q) {
        const int s = sides[q].slot;
        if (s < 0) continue;
        char* aux = x.base + slot_aux_offset(p, s);
        planes[q] = aux;
        exps[q] = reinterpret_cast<int*>(aux + split_planes_bytes(p, sides[q].is_a ? p.mb : p.nb));
    }
    TcProblem P;
    P.M = rows; P.N = cols; P.k_pad = K > 0 ? k_pad : 0;
    P.chunk = ozaki ? kOzakiChunk : kBf16x3Chunk;
    P.a_planes = planes[0]; P.a_rows_pad = ra_pad; P.a_nplanes = S;
    P.b_planes = planes[1]; P.b_rows_pad = rb_pad; P.b_nplanes = S;
    if (ozaki) {
        ozaki_groups(P, S);
        P.row_exp = exps[0];
        P.col_exp = exps[1];
    } else {
        TcGroupSpec& g = P.groups[0];
        g.na = 3; g.nb = 3; g.np = 6;
        for (int i = 0; i < 3; ++i) { g.aplane[i] = i; g.bplane[i] = i; }
        const int pa[6] = {0, 0, 1, 0, 1, 2}, pb[6] = {0, 1, 0, 2, 1, 0};  // hh hm mh hl mm lh
        for (int i = 0; i < 6; ++i) { g.pa[i] = pa[i]; g.pb[i] = pb[i]; }
        P.ngroups = 1;
        P.df32 = true;
    }
    P.alpha = o.alpha;
    P.beta = op.first ? o.beta : 1.0;
    P.read_c = !op.first || o.beta != 0.0;
    P.c_fp32 = p.es == 4;
    P.C = x.base + slot_offset(p, sc);
    P.ldc = p.ldc_dev;
    P.err = err;
    P.kblock = 64;
    if (p.block_class(op.i, op.j) == 2) {
        P.tri = p.tri;
        P.tri_off = p.block_off(op.i, op.j);
    }
    ++x.launches;
    return launch_tc_terms(P, x.smap[kStreamCompute], why);
}

int launch_tile(const Plan& p, const Op& op, Exec& x, const Operands& o, std::string& why)
{
    const int sa = op.nr > 0 && op.rslot[0] < p.nA ? op.rslot[0] : -1;
    int sb = -1;
    for (int r = 0; r < op.nr; ++r)
        if (op.rslot[r] >= p.nA && op.rslot[r] < p.nA + p.nB) sb = op.rslot[r];
    const int sc = op.wslot;
    const int64_t rows = p.rows_of(op.i), cols = p.cols_of(op.j), kk = p.K > 0 ? p.k_of(op.kc) : 0;
    const double beta_eff = op.first ? o.beta : 1.0;
    const bool read_c = !op.first || o.beta != 0.0;
    int* err = reinterpret_cast<int*>(x.arena);
    if (p.form == OOC_FORM_BF16X3 || p.form == OOC_FORM_OZAKI) return launch_split_tile(p, op, x, o, sa, sb, sc, why);
    if (p.form == OOC_FORM_FP64) {
        const double* dA = sa >= 0 ? reinterpret_cast<const double*>(x.base + slot_offset(p, sa)) : nullptr;
        const double* dB = sb >= 0 ? reinterpret_cast<const double*>(x.base + slot_offset(p, sb)) : nullptr;
        double* dC = reinterpret_cast<double*>(x.base + slot_offset(p, sc));
        ++x.launches;
        const bool masked = p.block_class(op.i, op.j) == 2;
        return launch_fp64_tile(!p.ta, p.tb, rows, cols, kk, o.alpha, dA, p.lda_dev, dB, p.ldb_dev, beta_eff, read_c,
                                dC, p.ldc_dev, err, x.smap[kStreamCompute], why, masked ? p.tri : 0,
                                masked ? p.block_off(op.i, op.j) : 0);
    }
    why = "contraction form not available in this build";
    return OOC_ERR_UNSUPPORTED;
}

// Issue one plan's schedule: copies, tile launches and the events ordering
// them, on the streams x.smap, with the plan's slots at x.base and its events
// at x.ev[x.ev_base + id].
int issue_ops(Exec& x, const Plan& p, const std::vector<Op>& ops, const Operands& o, int es, const Inject& inj,
              std::string& why)
{
    int rc = 0;
    const char* hA = static_cast<const char*>(o.A);
    const char* hB = static_cast<const char*>(o.B);
    char* hC = static_cast<char*>(o.C);
    const char* trace_path = std::getenv("OOC_TRACE");
    const auto t_issue0 = std::chrono::steady_clock::now();
    for (const Op& op : ops) {
        cudaStream_t s = x.smap[op.stream];
        const bool traced = trace_path && (op.kind == kH2D || op.kind == kKernel || op.kind == kD2H || op.kind == kSplit);
        if (traced) {
            // a split is device work on the kernel stream: traced as a kernel
            TraceRec r{op.kind == kSplit ? (int)kKernel : op.kind, op.stream, op.i, op.j, op.kc, 0.0,
                       std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_issue0).count(),
                       nullptr, nullptr};
            CK(cudaEventCreate(&r.e0));
            CK(cudaEventCreate(&r.e1));
            CK(cudaEventRecord(r.e0, s));
            x.trace.push_back(r);
        }
        switch (op.kind) {
        case kRecord: CK(cudaEventRecord(x.ev[x.ev_base + op.event], s)); break;
        case kWait: CK(cudaStreamWaitEvent(s, x.ev[x.ev_base + op.event], 0)); break;
        case kH2D: {
            if (inj.copy >= 0 && x.n_copy++ == inj.copy) return fail(OOC_ERR_INJECTED, "injected copy failure");
            const Tag& t = op.wtag;
            char* dst = x.base + slot_offset(p, op.wslot);
            const char* src;
            int64_t rows, width, spitch, dpitch;
            if (t.m == kMatA) {
                const int64_t r0 = t.r * p.mb, k0 = t.c * p.kb, mr = p.rows_of(t.r), kr = p.k_of(t.c);
                if (!p.ta) { src = hA + (r0 * o.lda + k0) * es; rows = mr; width = kr; }
                else { src = hA + (k0 * o.lda + r0) * es; rows = kr; width = mr; }
                spitch = o.lda * es; dpitch = p.lda_dev * es;
            } else if (t.m == kMatB) {
                const int64_t k0 = t.r * p.kb, c0 = t.c * p.nb, kr = p.k_of(t.r), nc = p.cols_of(t.c);
                if (!p.tb) { src = hB + (k0 * o.ldb + c0) * es; rows = kr; width = nc; }
                else { src = hB + (c0 * o.ldb + k0) * es; rows = nc; width = kr; }
                spitch = o.ldb * es; dpitch = p.ldb_dev * es;
            } else {
                src = hC + (t.r * p.mb * o.ldc + t.c * p.nb) * es;
                rows = p.rows_of(t.r); width = p.cols_of(t.c);
                spitch = o.ldc * es; dpitch = p.ldc_dev * es;
            }
            if (op.nparts > 1) {  // one row range of the chunk (B prefetch pieces)
                const int64_t r0 = rows * op.part / op.nparts, r1 = rows * (op.part + 1) / op.nparts;
                src += r0 * spitch;
                dst += r0 * dpitch;
                rows = r1 - r0;
            }
            if (rows > 0 && width > 0) {
                if (spitch == width * es && dpitch == width * es)
                    CK(cudaMemcpyAsync(dst, src, rows * width * es, cudaMemcpyHostToDevice, s));
                else
                    CK(cudaMemcpy2DAsync(dst, dpitch, src, spitch, width * es, rows, cudaMemcpyHostToDevice, s));
                x.h2d += (double)rows * width * es;
            }
            break;
        }
        case kSplit: {
            // staged plans: the staging area's raw chunk into the planes of the slot it is for
            const Tag& t = op.wtag;
            const bool is_a = t.m == kMatA;
            const int64_t nrows = is_a ? p.rows_of(t.r) : p.cols_of(t.c);
            const int64_t K = p.K > 0 ? p.k_of(is_a ? t.c : t.r) : 0;
            const bool timed = x.time_kernels && 2 * x.n_split + 1 < (long)x.sev.size();
            if (timed) CK(cudaEventRecord(x.sev[2 * x.n_split], s));
            rc = split_slot(p, x, op.rslot[0], op.wslot, is_a, nrows, K, why);
            if (rc) return fail(rc, why);
            if (timed) CK(cudaEventRecord(x.sev[2 * x.n_split + 1], s));
            ++x.n_split;
            break;
        }
        case kKernel: {
            if (inj.kernel >= 0 && x.n_kern == inj.kernel) return fail(OOC_ERR_INJECTED, "injected kernel failure");
            if (x.time_kernels) CK(cudaEventRecord(x.kev[2 * x.n_kern], s));
            rc = launch_tile(p, op, x, o, why);
            if (rc) return fail(rc, why);
            if (x.time_kernels) CK(cudaEventRecord(x.kev[2 * x.n_kern + 1], s));
            ++x.n_kern;
            break;
        }
        case kD2H: {
            const int64_t rows = p.rows_of(op.i), width = p.cols_of(op.j);
            char* dst = hC + (op.i * p.mb * o.ldc + op.j * p.nb) * es;
            const char* src = x.base + slot_offset(p, op.rslot[0]);
            if (o.ldc == width && p.ldc_dev == width)
                CK(cudaMemcpyAsync(dst, src, rows * width * es, cudaMemcpyDeviceToHost, s));
            else
                CK(cudaMemcpy2DAsync(dst, o.ldc * es, src, p.ldc_dev * es, width * es, rows, cudaMemcpyDeviceToHost,
                                     s));
            x.d2h += (double)rows * width * es;
            break;
        }
        }
        if (traced) {
            CK(cudaEventRecord(x.trace.back().e1, s));
            x.trace.back().bytes = x.h2d + x.d2h;  // running total; differenced when written
        }
    }
    return OOC_OK;
}

// Issue a planned schedule on x's streams (already created) and arena, wait for
// it, check the device error word and fill the device-side statistics (the
// caller sets seconds / tflops after releasing its resources).
int execute(Exec& x, const std::vector<Op>& ops, const Operands& o, int es, const Inject& inj, ooc_stats* stats)
{
    const Plan& p = x.p;
    std::string why;
    int rc = OOC_OK;
    x.ev.resize(n_events(p), nullptr);
    for (auto& e : x.ev) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    int64_t nkern = 0, nsplit = 0;
    for (const Op& op : ops) {
        nkern += op.kind == kKernel;
        nsplit += op.kind == kSplit;
    }
    x.kev.resize(2 * nkern, nullptr);
    for (auto& e : x.kev) CK(cudaEventCreate(&e));
    x.sev.resize(2 * nsplit, nullptr);
    for (auto& e : x.sev) CK(cudaEventCreate(&e));
    CK(cudaEventCreate(&x.t_begin));
    for (auto& e : x.t_end) CK(cudaEventCreate(&e));

    int* err = reinterpret_cast<int*>(x.arena);
    CK(cudaEventRecord(x.t_begin, x.st[kStreamH2D]));
    CK(cudaStreamWaitEvent(x.st[kStreamCompute], x.t_begin, 0));
    CK(cudaStreamWaitEvent(x.st[kStreamD2H], x.t_begin, 0));
    CK(cudaMemsetAsync(err, 0, sizeof(int), x.st[kStreamCompute]));

    x.base = x.arena;
    x.smap[0] = x.st[0]; x.smap[1] = x.st[1]; x.smap[2] = x.st[2];
    x.ev_base = 0;
    rc = issue_ops(x, p, ops, o, es, inj, why);
    if (rc) return rc;
    const char* trace_path = std::getenv("OOC_TRACE");
    for (int i = 0; i < 3; ++i) CK(cudaEventRecord(x.t_end[i], x.st[i]));
    for (auto s : x.st) CK(cudaStreamSynchronize(s));
    int herr = 0;
    CK(cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost));
    if (herr != 0) return fail(OOC_ERR_TIMEOUT, "a device-side wait gave up (status " + std::to_string(herr) + ")");
    if (trace_path) {
        if (FILE* f = std::fopen(trace_path, "a")) {
            std::fprintf(f, "# call M=%lld N=%lld K=%lld mb=%lld nb=%lld kb=%lld nA=%d nB=%d nC=%d\n", (long long)p.M,
                         (long long)p.N, (long long)p.K, (long long)p.mb, (long long)p.nb, (long long)p.kb, p.nA, p.nB,
                         p.nC);
            double prev = 0;
            for (auto& r : x.trace) {
                float a = 0, b = 0;
                cudaEventElapsedTime(&a, x.t_begin, r.e0);
                cudaEventElapsedTime(&b, x.t_begin, r.e1);
                const char* k = r.kind == kH2D ? "h2d" : r.kind == kKernel ? "kernel" : "d2h";
                std::fprintf(f, "%s,%d,%lld,%lld,%lld,%.0f,%.3f,%.3f,%.3f\n", k, r.stream, (long long)r.i,
                             (long long)r.j, (long long)r.kc, r.bytes - prev, r.host_ms, a, b);
                prev = r.bytes;
            }
            std::fclose(f);
        }
    }

    if (stats) {
        float ms = 0, best = 0;
        for (auto e : x.t_end) {
            CK(cudaEventElapsedTime(&ms, x.t_begin, e));
            best = std::max(best, ms);
        }
        double ksum = 0, ssum = 0;
        for (int64_t k = 0; k < x.n_kern; ++k) {
            CK(cudaEventElapsedTime(&ms, x.kev[2 * k], x.kev[2 * k + 1]));
            ksum += ms;
        }
        for (long k = 0; 2 * k + 1 < (long)x.sev.size() && k < x.n_split; ++k) {
            CK(cudaEventElapsedTime(&ms, x.sev[2 * k], x.sev[2 * k + 1]));
            ksum += ms;
            ssum += ms;
        }
        stats->device_seconds = best * 1e-3;
        stats->kernel_seconds = ksum * 1e-3;
        stats->split_seconds = ssum * 1e-3;
        stats->h2d_bytes = x.h2d;
        stats->d2h_bytes = x.d2h;
        stats->mb = p.mb; stats->nb = p.nb; stats->kb = p.kb;
        stats->depth = p.nA; stats->c_buffers = p.nC; stats->b_buffers = p.nB; stats->form = p.form;
        int64_t nblk = 0;
        for (const Op& op : ops) nblk += op.kind == kD2H;
        stats->blocks = nblk; stats->steps = x.n_kern;
        stats->device_bytes = (int64_t)p.device_bytes;
        stats->slices = p.slices; stats->products = p.products;
        stats->kernel_launches = x.launches;
    }
    return OOC_OK;
}

// tri / tri_off: triangular update of C (Plan::tri); 0 updates all of C.
int run_ooc(char ta, char tb, int64_t M, int64_t N, int64_t K, const Operands& o, int es, size_t budget,
            const ooc_opts* opts_in, ooc_stats* stats, int tri = 0, int64_t tri_off = 0)
{
    const auto t_host0 = std::chrono::steady_clock::now();
    std::string why;
    int rc = validate(ta, tb, M, N, K, o.A, o.lda, o.B, o.ldb, o.C, o.ldc, o.beta != 0.0, why);
    if (rc) return fail(rc, why);
    if (stats) std::memset(stats, 0, sizeof(*stats));
    if (M == 0 || N == 0) return OOC_OK;
    rc = check_device(why);
    if (rc) return fail(rc, why);
    if (!range_pinned(o.A, is_t(ta) ? K : M, is_t(ta) ? M : K, o.lda, es) ||
        !range_pinned(o.B, is_t(tb) ? N : K, is_t(tb) ? K : N, o.ldb, es) || !range_pinned(o.C, M, N, o.ldc, es))
        return fail(OOC_ERR_NOT_PINNED, "host operands must be page-locked (cudaHostAlloc / cudaHostRegister)");

    ooc_opts opts;
    std::memset(&opts, 0, sizeof(opts));
    if (opts_in) opts = *opts_in;
    PlanRequest rq{M, N, K, es, o.beta != 0.0, is_t(ta), is_t(tb), budget, opts};
    rq.lda = o.lda; rq.ldb = o.ldb; rq.ldc = o.ldc;
    rq.tri = tri; rq.tri_off = tri_off;
    double hg = 0, dg = 0;
    if (ooc_query_device(nullptr, &hg, &dg) == OOC_OK && hg > 0 && dg > 0) {
        rq.h2d_gbps = hg;
        rq.d2h_gbps = dg;
    }
    Exec x;
    x.flags = opts.flags;
    rc = make_plan(rq, x.p, why);
    if (rc) return fail(rc, why);
    const Plan& p = x.p;
    std::vector<Op> ops;
    build_schedule(p, ops);

    Inject inj;
    if (opts.workspace) {
        if (opts.workspace_bytes < p.device_bytes)
            return fail(OOC_ERR_INVALID_ARG, "workspace smaller than the plan's device bytes");
        x.arena = static_cast<char*>(opts.workspace);
    } else {
        if (inj.alloc) return fail(OOC_ERR_INJECTED, "injected arena allocation failure");
        if (cudaMalloc(&x.arena, p.device_bytes) != cudaSuccess) {
            cudaGetLastError();
            x.arena = nullptr;
            return fail(OOC_ERR_ALLOC, "device arena of " + std::to_string(p.device_bytes) + " bytes");
        }
        x.own_arena = true;
    }
    for (auto& s : x.st) CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    // a triangular update of a square C counts N (N + 1) K flops (the level-3 BLAS convention for SYRK)
    const double flops = tri ? (double)M * (M + 1) * K : 2.0 * (double)M * N * K;
    rc = execute(x, ops, o, es, inj, stats);
    if (rc) return rc;
    // release before taking the wall time (the arena free is part of the call)
    x.release();
    if (stats) {
        stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_host0).count();
        stats->tflops = stats->seconds > 0 ? flops / stats->seconds / 1e12 : 0.0;
    }
    return OOC_OK;
}

}  // namespace

namespace ooc {
bool host_range_pinned(const void* base, int64_t rows, int64_t cols, int64_t ld, int es)
{
    return range_pinned(base, rows, cols, ld, es);
}
int device_check(std::string& why) { return check_device(why); }

int run_gemm_host(char ta, char tb, int64_t M, int64_t N, int64_t K, double alpha, const void* A, int64_t lda,
                  const void* B, int64_t ldb, double beta, void* C, int64_t ldc, int es, size_t budget,
                  const ooc_opts* opts, ooc_stats* stats, int tri, int64_t tri_off)
{
    Operands o{A, lda, B, ldb, C, ldc, alpha, beta};
    return run_ooc(ta, tb, M, N, K, o, es, budget, opts, stats, tri, tri_off);
}
}  // namespace ooc

namespace {

// ------------------------------------------------------------- grouped batch --
// Batched calls whose problems each fit in half of the budget: consecutive
// problems are packed whole into one arena half as a group (at most kGroupMax,
// one transpose pair), copied in with one copy per operand, multiplied by one
// persistent grouped launch over all their tiles, and copied out; groups
// alternate halves, each half on its own H2D / compute / D2H streams, so one
// group's copies overlap the other half's kernel.  Compared with one
// out-of-core pipeline per problem this pays a launch's tail and a pipeline
// fill once per group instead of once per problem (Section IV's pipeline with
// the group as its unit of work).
namespace {

struct DevMat {
    size_t off = 0;   // byte offset in the half
    int64_t ld = 0;   // device leading dimension (elements, even: TMA row pitch)
};

size_t mat_bytes(int64_t rows, int64_t ld) { return ((size_t)std::max<int64_t>(rows, 1) * ld * 8 + 255) / 256 * 256; }
int64_t even(int64_t x) { return std::max<int64_t>(2, (x + 1) / 2 * 2); }

// device bytes of problem d placed whole (A, B, C)
size_t whole_bytes(const ooc_gemm_desc& d)
{
    const bool ta = d.transA == 'T' || d.transA == 't', tb = d.transB == 'T' || d.transB == 't';
    const int64_t ar = ta ? d.K : d.M, ac = ta ? d.M : d.K, br = tb ? d.N : d.K, bc = tb ? d.K : d.N;
    return mat_bytes(ar, even(ac)) + mat_bytes(br, even(bc)) + mat_bytes(d.M, even(d.N));
}

int copy_h2d(char* dst, int64_t dld, const void* src, int64_t sld, int64_t rows, int64_t cols, cudaStream_t s,
             double& bytes)
{
    if (rows <= 0 || cols <= 0) return OOC_OK;
    cudaError_t e;
    if (sld == cols && dld == cols) e = cudaMemcpyAsync(dst, src, (size_t)rows * cols * 8, cudaMemcpyHostToDevice, s);
    else e = cudaMemcpy2DAsync(dst, dld * 8, src, sld * 8, cols * 8, rows, cudaMemcpyHostToDevice, s);
    bytes += (double)rows * cols * 8;
    return e == cudaSuccess ? OOC_OK : OOC_ERR_CUDA;
}

}  // namespace

int run_batched_grouped(int32_t count, const ooc_gemm_desc* d, size_t half, const ooc_opts& opts, bool use_graph,
                        ooc_stats* stats, std::chrono::steady_clock::time_point t_host0)
{
    std::string why;
    // groups: consecutive problems, same transposes, whole in one half, at most kGroupMax
    struct Group {
        int first = 0, n = 0;
        bool ta = false, tb = false;
    };
    std::vector<Group> groups;
    {
        size_t used = 0;
        for (int g = 0; g < count; ++g) {
            if (d[g].M == 0 || d[g].N == 0) continue;
            const bool ta = is_t(d[g].transA), tb = is_t(d[g].transB);
            const size_t b = whole_bytes(d[g]);
            if (groups.empty() || groups.back().ta != ta || groups.back().tb != tb || groups.back().n >= kGroupMax ||
                used + b > half) {
                groups.push_back(Group{g, 0, ta, tb});
                used = 0;
            }
            groups.back().n = g - groups.back().first + 1;
            used += b;
        }
    }
    double flops = 0;
    for (int g = 0; g < count; ++g) flops += 2.0 * (double)d[g].M * d[g].N * d[g].K;

    Inject inj;
    char* arena = nullptr;
    bool own = false;
    if (opts.workspace) {
        if (opts.workspace_bytes < 2 * half + 256) return fail(OOC_ERR_INVALID_ARG, "workspace smaller than the budget");
        arena = static_cast<char*>(opts.workspace);
    } else {
        if (inj.alloc) return fail(OOC_ERR_INJECTED, "injected arena allocation failure");
        if (cudaMalloc(&arena, 2 * half + 256) != cudaSuccess) {
            cudaGetLastError();
            return fail(OOC_ERR_ALLOC, "device arena of " + std::to_string(2 * half + 256) + " bytes");
        }
        own = true;
    }
    // resources, released on every return path
    struct Res {
        cudaStream_t s[7] = {};  // [0] fork/join, then per half: H2D, compute, D2H
        cudaEvent_t ev[7] = {};  // per half: in, done, out; [6] fork
        cudaEvent_t t0 = nullptr, t1 = nullptr;
        std::vector<cudaEvent_t> kev;
        char* arena = nullptr;
        bool own = false;
        void release()
        {
            for (auto& st : s)
                if (st) cudaStreamSynchronize(st);
            for (auto& st : s)
                if (st) { cudaStreamDestroy(st); st = nullptr; }
            for (auto& e : ev)
                if (e) { cudaEventDestroy(e); e = nullptr; }
            for (auto& e : kev)
                if (e) cudaEventDestroy(e);
            kev.clear();
            if (t0) { cudaEventDestroy(t0); t0 = nullptr; }
            if (t1) { cudaEventDestroy(t1); t1 = nullptr; }
            if (own && arena) cudaFree(arena);
            arena = nullptr;
            cudaGetLastError();
        }
        ~Res() { release(); }
    } r;
    r.arena = arena;
    r.own = own;
    for (auto& st : r.s) CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    for (auto& e : r.ev) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    CK(cudaEventCreate(&r.t0));
    CK(cudaEventCreate(&r.t1));
    if (!use_graph) {
        r.kev.resize(2 * groups.size(), nullptr);
        for (auto& e : r.kev) CK(cudaEventCreate(&e));
    }
    int* err = reinterpret_cast<int*>(arena);
    cudaStream_t s0 = r.s[0];
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    if (use_graph) CK(cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal));
    else CK(cudaEventRecord(r.t0, s0));
    CK(cudaMemsetAsync(err, 0, sizeof(int), s0));
    CK(cudaEventRecord(r.ev[6], s0));
    for (int k = 1; k < 7; ++k) CK(cudaStreamWaitEvent(r.s[k], r.ev[6], 0));
    double h2d = 0, d2h = 0;
    int launches = 0;
    int rc = OOC_OK;
    bool issued[2] = {false, false};
    std::vector<Fp64GroupSpec> spec;
    for (size_t G = 0; G < groups.size() && rc == OOC_OK; ++G) {
        const Group& gr = groups[G];
        const int h = (int)(G & 1);
        char* base = arena + 256 + (size_t)h * half;
        cudaStream_t sh = r.s[1 + 3 * h], sc = r.s[2 + 3 * h], sd = r.s[3 + 3 * h];
        cudaEvent_t ev_in = r.ev[3 * h], ev_done = r.ev[3 * h + 1], ev_out = r.ev[3 * h + 2];
        // the previous group of this half has copied its results out
        if (issued[h]) CK(cudaStreamWaitEvent(sh, ev_out, 0));
        spec.assign(gr.n, Fp64GroupSpec{});
        size_t off = 0;
        for (int q = 0; q < gr.n && rc == OOC_OK; ++q) {
            const ooc_gemm_desc& p = d[gr.first + q];
            Fp64GroupSpec& s = spec[q];
            s.M = p.M; s.N = p.N; s.K = p.K;
            s.alpha = p.alpha; s.beta = p.beta;
            s.read_c = p.beta != 0.0;
            if (p.M == 0 || p.N == 0) continue;
            const int64_t ar = gr.ta ? p.K : p.M, ac = gr.ta ? p.M : p.K;
            const int64_t br = gr.tb ? p.N : p.K, bc = gr.tb ? p.K : p.N;
            s.lda = even(ac); s.ldb = even(bc); s.ldc = even(p.N);
            char* dA = base + off;
            off += mat_bytes(ar, s.lda);
            char* dB = base + off;
            off += mat_bytes(br, s.ldb);
            char* dC = base + off;
            off += mat_bytes(p.M, s.ldc);
            s.A = reinterpret_cast<const double*>(dA);
            s.B = reinterpret_cast<const double*>(dB);
            s.C = reinterpret_cast<double*>(dC);
            if (inj.copy >= 0 && (int64_t)(G * 3 + q) == inj.copy) { rc = fail(OOC_ERR_INJECTED, "injected copy failure"); break; }
            if (p.K > 0) {
                if (copy_h2d(dA, s.lda, p.A, p.lda, ar, ac, sh, h2d) || copy_h2d(dB, s.ldb, p.B, p.ldb, br, bc, sh, h2d)) {
                    rc = fail(OOC_ERR_CUDA, "grouped batch: operand copy");
                    break;
                }
            }
            if (s.read_c && copy_h2d(dC, s.ldc, p.C, p.ldc, p.M, p.N, sh, h2d)) {
                rc = fail(OOC_ERR_CUDA, "grouped batch: C copy");
                break;
            }
        }
        if (rc) break;
        CK(cudaEventRecord(ev_in, sh));
        CK(cudaStreamWaitEvent(sc, ev_in, 0));
        if (inj.kernel >= 0 && (int64_t)G == inj.kernel) { rc = fail(OOC_ERR_INJECTED, "injected kernel failure"); break; }
        if (!use_graph) CK(cudaEventRecord(r.kev[2 * G], sc));
        rc = launch_fp64_group(!gr.ta, gr.tb, spec.data(), gr.n, err, sc, why);
        if (rc) { rc = fail(rc, why); break; }
        if (!use_graph) CK(cudaEventRecord(r.kev[2 * G + 1], sc));
        ++launches;
        CK(cudaEventRecord(ev_done, sc));
        CK(cudaStreamWaitEvent(sd, ev_done, 0));
        for (int q = 0; q < gr.n; ++q) {
            const ooc_gemm_desc& p = d[gr.first + q];
            const Fp64GroupSpec& s = spec[q];
            if (p.M == 0 || p.N == 0) continue;
            cudaError_t e;
            if (p.ldc == p.N && s.ldc == p.N)
                e = cudaMemcpyAsync(p.C, s.C, (size_t)p.M * p.N * 8, cudaMemcpyDeviceToHost, sd);
            else
                e = cudaMemcpy2DAsync(p.C, p.ldc * 8, s.C, s.ldc * 8, p.N * 8, p.M, cudaMemcpyDeviceToHost, sd);
            if (e != cudaSuccess) { rc = fail(OOC_ERR_CUDA, "grouped batch: C copy out"); break; }
            d2h += (double)p.M * p.N * 8;
        }
        CK(cudaEventRecord(ev_out, sd));
        issued[h] = true;
    }
    // join every stream into s0
    for (int k = 1; k < 7; ++k) {
        CK(cudaEventRecord(r.ev[6], r.s[k]));
        CK(cudaStreamWaitEvent(s0, r.ev[6], 0));
    }
    if (use_graph) {
        CK(cudaStreamEndCapture(s0, &graph));
        if (rc == OOC_OK) {
            cudaError_t e = cudaGraphInstantiate(&gexec, graph, 0);
            if (e == cudaSuccess) {
                CK(cudaEventRecord(r.t0, s0));
                e = cudaGraphLaunch(gexec, s0);
            }
            if (e != cudaSuccess) rc = fail(OOC_ERR_CUDA, std::string("grouped batch graph: ") + cudaGetErrorString(e));
        }
    }
    CK(cudaEventRecord(r.t1, s0));
    cudaError_t se = cudaStreamSynchronize(s0);
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);
    if (rc) return rc;
    if (se != cudaSuccess) return fail(OOC_ERR_CUDA, std::string("grouped batch: ") + cudaGetErrorString(se));
    int herr = 0;
    CK(cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost));
    if (herr != 0) return fail(OOC_ERR_TIMEOUT, "a device-side wait gave up (status " + std::to_string(herr) + ")");
    if (stats) {
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, r.t0, r.t1));
        stats->device_seconds = ms * 1e-3;
        double ksum = 0;
        for (size_t G = 0; !use_graph && G < groups.size(); ++G) {
            CK(cudaEventElapsedTime(&ms, r.kev[2 * G], r.kev[2 * G + 1]));
            ksum += ms;
        }
        stats->kernel_seconds = ksum * 1e-3;  // 0 in graph mode (not timed)
        stats->h2d_bytes = h2d;
        stats->d2h_bytes = d2h;
        for (int g = 0; g < count; ++g) stats->blocks += d[g].M > 0 && d[g].N > 0;
        stats->steps = (int64_t)groups.size();
        stats->device_bytes = (int64_t)(2 * half + 256);
        stats->form = OOC_FORM_FP64;
        stats->kernel_launches = launches;
    }
    r.release();  // the arena free is part of the call's wall time
    if (stats) {
        stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_host0).count();
        stats->tflops = stats->seconds > 0 ? flops / stats->seconds / 1e12 : 0.0;
    }
    return OOC_OK;
}

int run_batched(int32_t count, const ooc_gemm_desc* d, size_t budget, const ooc_opts* opts_in, ooc_stats* stats)
{
    const auto t_host0 = std::chrono::steady_clock::now();
    std::string why;
    if (count < 0 || (count > 0 && !d)) return fail(OOC_ERR_INVALID_ARG, "batched: bad count or descriptor array");
    if (stats) std::memset(stats, 0, sizeof(*stats));
    int rc;
    for (int g = 0; g < count; ++g) {
        rc = validate(d[g].transA, d[g].transB, d[g].M, d[g].N, d[g].K, d[g].A, d[g].lda, d[g].B, d[g].ldb, d[g].C,
                      d[g].ldc, d[g].beta != 0.0, why);
        if (rc) return fail(rc, "batched problem " + std::to_string(g) + ": " + why);
    }
    if (count == 0) return OOC_OK;
    rc = check_device(why);
    if (rc) return fail(rc, why);
    for (int g = 0; g < count; ++g) {
        if (d[g].M == 0 || d[g].N == 0) continue;
        const bool ta = is_t(d[g].transA), tb = is_t(d[g].transB);
        if (!range_pinned(d[g].A, ta ? d[g].K : d[g].M, ta ? d[g].M : d[g].K, d[g].lda, 8) ||
            !range_pinned(d[g].B, tb ? d[g].N : d[g].K, tb ? d[g].K : d[g].N, d[g].ldb, 8) ||
            !range_pinned(d[g].C, d[g].M, d[g].N, d[g].ldc, 8))
            return fail(OOC_ERR_NOT_PINNED, "batched problem " + std::to_string(g) + ": host operands must be page-locked");
    }
    ooc_opts opts;
    std::memset(&opts, 0, sizeof(opts));
    if (opts_in) opts = *opts_in;
    const bool use_graph = (opts.flags & OOC_BATCH_GRAPH) != 0;
    double hg = 0, dg = 0;
    const bool have_link = ooc_query_device(nullptr, &hg, &dg) == OOC_OK && hg > 0 && dg > 0;
    const size_t half = ((budget > 512 ? budget - 256 : 0) / 2) / 256 * 256;
    // FP64 problems that each fit whole in half the budget: the grouped path (one persistent launch
    // per group of problems) unless the caller asks for one out-of-core pipeline per problem
    if ((opts.form == OOC_FORM_AUTO || opts.form == OOC_FORM_FP64) && !(opts.flags & OOC_BATCH_STREAMED)) {
        bool all_fit = true;
        for (int g = 0; g < count && all_fit; ++g)
            if (d[g].M > 0 && d[g].N > 0) all_fit = whole_bytes(d[g]) <= half;
        if (all_fit) return run_batched_grouped(count, d, half, opts, use_graph, stats, t_host0);
    }

    // plans and schedules, each within half of the budget; the problems are planned in
    // parallel on host threads (planning is host work: candidate search, cost model)
    std::vector<Plan> plans(count);
    std::vector<std::vector<Op>> sched(count);
    std::vector<int> prc(count, OOC_OK);
    std::vector<std::string> pwhy(count);
    int cur_dev = 0;
    cudaGetDevice(&cur_dev);
    auto plan_some = [&](int t, int nt) {
        cudaSetDevice(cur_dev);  // the cost model runs on the caller's device
        for (int g = t; g < count; g += nt) {
            if (d[g].M == 0 || d[g].N == 0) continue;
            PlanRequest rq{d[g].M, d[g].N, d[g].K, 8, d[g].beta != 0.0, is_t(d[g].transA), is_t(d[g].transB), half,
                           opts};
            rq.lda = d[g].lda; rq.ldb = d[g].ldb; rq.ldc = d[g].ldc;
            if (have_link) { rq.h2d_gbps = hg; rq.d2h_gbps = dg; }
            prc[g] = make_plan(rq, plans[g], pwhy[g]);
            if (prc[g] == OOC_OK) build_schedule(plans[g], sched[g]);
        }
    };
    {
        const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
        const int nt = std::max(1, std::min({hw, 16, count}));
        std::vector<std::thread> th;
        int started = 1;
        try {
            for (int t = 1; t < nt; ++t, ++started) th.emplace_back(plan_some, t, nt);
        } catch (...) {
        }
        plan_some(0, nt);
        for (int t = started; t < nt; ++t) plan_some(t, nt);
        for (auto& x : th) x.join();
    }
    int E = 0;
    int64_t nkern = 0, nsplit = 0;
    double flops = 0;
    for (int g = 0; g < count; ++g) {
        if (d[g].M == 0 || d[g].N == 0) continue;
        if (prc[g]) return fail(prc[g], "batched problem " + std::to_string(g) + ": " + pwhy[g]);
        E = std::max(E, n_events(plans[g]));
        for (const Op& op : sched[g]) {
            nkern += op.kind == kKernel;
            nsplit += op.kind == kSplit;
        }
        flops += 2.0 * (double)d[g].M * d[g].N * d[g].K;
    }

    Inject inj;
    Exec x;
    x.flags = opts.flags;
    if (opts.workspace) {
        if (opts.workspace_bytes < 2 * half + 256) return fail(OOC_ERR_INVALID_ARG, "workspace smaller than the budget");
        x.arena = static_cast<char*>(opts.workspace);
    } else {
        if (inj.alloc) return fail(OOC_ERR_INJECTED, "injected arena allocation failure");
        if (cudaMalloc(&x.arena, 2 * half + 256) != cudaSuccess) {
            cudaGetLastError();
            x.arena = nullptr;
            return fail(OOC_ERR_ALLOC, "device arena of " + std::to_string(2 * half + 256) + " bytes");
        }
        x.own_arena = true;
    }
    for (auto& st : x.st) CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    // the second half runs on its own three streams: a problem waiting for its half's previous
    // problem never holds up the other half's copies
    CK(cudaStreamCreateWithFlags(&x.extra_compute, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&x.extra_h2d, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&x.extra_d2h, cudaStreamNonBlocking));
    x.ev.resize(2 * E + 2 + 6, nullptr);  // two event sets, two "half done" events, fork + five joins
    for (auto& e : x.ev) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    x.kev.resize(2 * nkern, nullptr);
    for (auto& e : x.kev) CK(cudaEventCreate(&e));
    x.sev.resize(2 * nsplit, nullptr);
    for (auto& e : x.sev) CK(cudaEventCreate(&e));
    CK(cudaEventCreate(&x.t_begin));
    for (auto& e : x.t_end) CK(cudaEventCreate(&e));
    const int ev_done0 = 2 * E, ev_fork = 2 * E + 2;

    cudaStream_t s0 = x.st[kStreamH2D];
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    // Timing events cannot be read back from inside a captured graph: in graph
    // mode the launch is timed from outside and tile launches are not timed.
    x.time_kernels = !use_graph;
    if (use_graph) CK(cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal));
    else CK(cudaEventRecord(x.t_begin, s0));
    CK(cudaEventRecord(x.ev[ev_fork], s0));
    cudaStream_t others[5] = {x.st[kStreamCompute], x.st[kStreamD2H], x.extra_compute, x.extra_h2d, x.extra_d2h};
    for (cudaStream_t o : others) CK(cudaStreamWaitEvent(o, x.ev[ev_fork], 0));
    CK(cudaMemsetAsync(x.arena, 0, sizeof(int), s0));
    bool issued_half[2] = {false, false};
    for (int g = 0; g < count; ++g) {
        if (d[g].M == 0 || d[g].N == 0) continue;
        const int h = g & 1;
        x.base = x.arena + 256 + (size_t)h * half;
        x.smap[kStreamH2D] = h ? x.extra_h2d : x.st[kStreamH2D];
        x.smap[kStreamCompute] = h ? x.extra_compute : x.st[kStreamCompute];
        x.smap[kStreamD2H] = h ? x.extra_d2h : x.st[kStreamD2H];
        x.ev_base = h * E;
        if (issued_half[h]) {
            // the previous problem in this half has copied its last block out
            CK(cudaStreamWaitEvent(x.smap[kStreamH2D], x.ev[ev_done0 + h], 0));
            CK(cudaStreamWaitEvent(x.smap[kStreamCompute], x.ev[ev_done0 + h], 0));
        }
        Operands o{d[g].A, d[g].lda, d[g].B, d[g].ldb, d[g].C, d[g].ldc, d[g].alpha, d[g].beta};
        rc = issue_ops(x, plans[g], sched[g], o, 8, inj, why);
        if (rc) {
            if (use_graph) {
                cudaGraph_t gg = nullptr;
                cudaStreamEndCapture(s0, &gg);
                if (gg) cudaGraphDestroy(gg);
                cudaGetLastError();
            }
            return rc;
        }
        CK(cudaEventRecord(x.ev[ev_done0 + h], x.smap[kStreamD2H]));
        issued_half[h] = true;
    }
    for (int k = 0; k < 5; ++k) {
        CK(cudaEventRecord(x.ev[ev_fork + 1 + k], others[k]));
        CK(cudaStreamWaitEvent(s0, x.ev[ev_fork + 1 + k], 0));
    }
    if (!use_graph) {
        for (auto& e : x.t_end) CK(cudaEventRecord(e, s0));
    } else {
        CK(cudaStreamEndCapture(s0, &graph));
        cudaError_t e = cudaGraphInstantiate(&gexec, graph, 0);
        if (e != cudaSuccess) {
            cudaGraphDestroy(graph);
            return fail(OOC_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
        }
        CK(cudaEventRecord(x.t_begin, s0));
        e = cudaGraphLaunch(gexec, s0);
        if (e != cudaSuccess) {
            cudaGraphExecDestroy(gexec);
            cudaGraphDestroy(graph);
            return fail(OOC_ERR_CUDA, std::string("cudaGraphLaunch: ") + cudaGetErrorString(e));
        }
        for (auto& ev : x.t_end) CK(cudaEventRecord(ev, s0));
    }
    cudaError_t se = cudaStreamSynchronize(s0);
    for (auto st : x.st) cudaStreamSynchronize(st);
    for (cudaStream_t o : others) cudaStreamSynchronize(o);
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);
    if (se != cudaSuccess) return fail(OOC_ERR_CUDA, std::string("batched pipeline: ") + cudaGetErrorString(se));
    int herr = 0;
    CK(cudaMemcpy(&herr, x.arena, sizeof(int), cudaMemcpyDeviceToHost));
    if (herr != 0) return fail(OOC_ERR_TIMEOUT, "a device-side wait gave up (status " + std::to_string(herr) + ")");
    if (stats) {
        float ms = 0, best = 0;
        for (auto e : x.t_end) {
            CK(cudaEventElapsedTime(&ms, x.t_begin, e));
            best = std::max(best, ms);
        }
        double ksum = 0, ssum = 0;
        for (int64_t k = 0; x.time_kernels && k < x.n_kern; ++k) {
            CK(cudaEventElapsedTime(&ms, x.kev[2 * k], x.kev[2 * k + 1]));
            ksum += ms;
        }
        for (long k = 0; x.time_kernels && 2 * k + 1 < (long)x.sev.size() && k < x.n_split; ++k) {
            CK(cudaEventElapsedTime(&ms, x.sev[2 * k], x.sev[2 * k + 1]));
            ksum += ms;
            ssum += ms;
        }
        stats->device_seconds = best * 1e-3;
        stats->kernel_seconds = ksum * 1e-3;  // 0 in graph mode (not timed)
        stats->split_seconds = ssum * 1e-3;
        stats->h2d_bytes = x.h2d;
        stats->d2h_bytes = x.d2h;
        for (int g = 0; g < count; ++g) {
            stats->blocks += plans[g].h * plans[g].w;
            stats->steps += plans[g].h * plans[g].w * plans[g].nkc;
        }
        stats->device_bytes = (int64_t)(2 * half + 256);
        stats->form = opts.form ? opts.form : OOC_FORM_FP64;
        stats->kernel_launches = x.launches;
    }
    x.release();
    if (stats) {
        stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_host0).count();
        stats->tflops = stats->seconds > 0 ? flops / stats->seconds / 1e12 : 0.0;
    }
    return OOC_OK;
}

}  // namespace

extern "C" {

int ooc_dgemm_batched(int32_t count, const ooc_gemm_desc* descs, size_t device_budget_bytes, const ooc_opts* opts,
                      ooc_stats* stats)
{
    return run_batched(count, descs, device_budget_bytes, opts, stats);
}

int ooc_plan_candidates(int64_t M, int64_t N, int64_t K, int32_t elem_bytes, int32_t beta_nonzero, size_t budget,
                        const ooc_opts* opts_in, ooc_plan_candidate* out, int32_t capacity, int32_t* count)
{
    if ((elem_bytes != 4 && elem_bytes != 8) || M <= 0 || N <= 0 || K < 0 || !count || capacity < 0 ||
        (capacity > 0 && !out))
        return fail(OOC_ERR_INVALID_ARG, "ooc_plan_candidates: bad arguments");
    ooc_opts opts;
    std::memset(&opts, 0, sizeof(opts));
    if (opts_in) opts = *opts_in;
    PlanRequest rq{M, N, K, elem_bytes, beta_nonzero != 0, false, false, budget, opts};
    double hg = 0, dg = 0;
    if (ooc_query_device(nullptr, &hg, &dg) == OOC_OK && hg > 0 && dg > 0) { rq.h2d_gbps = hg; rq.d2h_gbps = dg; }
    cudaGetLastError();
    std::vector<Plan> c;
    std::string why;
    int rc = plan_candidates(rq, std::max(capacity, 1), c, why);
    if (rc) return fail(rc, why);
    *count = (int32_t)std::min<size_t>(c.size(), (size_t)capacity);
    for (int32_t i = 0; i < *count; ++i) {
        ooc_plan_candidate& d = out[i];
        std::memset(&d, 0, sizeof(d));
        d.mb = c[i].mb; d.nb = c[i].nb; d.kb = c[i].kb;
        d.depth = c[i].nA; d.b_buffers = c[i].nB; d.c_buffers = c[i].nC;
        d.est_seconds = c[i].est_seconds;
        plan_features(c[i], rq, d.features);
    }
    return OOC_OK;
}

int ooc_autotune(const ooc_gemm_desc* d, int32_t elem_bytes, size_t budget, const ooc_opts* opts_in,
                 int32_t max_candidates, ooc_plan_candidate* out, double* seconds_out, int32_t* count)
{
    if (!d || !out || !seconds_out || !count || max_candidates <= 0 || (elem_bytes != 4 && elem_bytes != 8))
        return fail(OOC_ERR_INVALID_ARG, "ooc_autotune: bad arguments");
    ooc_opts opts;
    std::memset(&opts, 0, sizeof(opts));
    if (opts_in) opts = *opts_in;
    int32_t n = 0;
    int rc = ooc_plan_candidates(d->M, d->N, d->K, elem_bytes, d->beta != 0.0, budget, &opts, out, max_candidates, &n);
    if (rc) return rc;
    Operands o{d->A, d->lda, d->B, d->ldb, d->C, d->ldc, d->alpha, d->beta};
    for (int32_t i = -1; i < n; ++i) {  // i = -1: untimed warm-up with the first candidate
        const ooc_plan_candidate& c = out[std::max(i, 0)];
        ooc_opts oc = opts;
        oc.mb = c.mb; oc.nb = c.nb; oc.kb = c.kb;
        oc.depth = c.depth; oc.c_buffers = c.c_buffers; oc.b_buffers = c.b_buffers;
        oc.flags &= ~(OOC_PLAN_MODEL | OOC_PLAN_PAPER);
        ooc_stats st;
        rc = run_ooc(d->transA, d->transB, d->M, d->N, d->K, o, elem_bytes, budget, &oc, &st);
        if (rc) return rc;
        if (i >= 0) seconds_out[i] = st.device_seconds;
    }
    *count = n;
    return OOC_OK;
}

int ooc_mlp_forward(const float* params, const float* X, int64_t n, float* y)
{
    if (!params || (n > 0 && (!X || !y)) || n < 0) return fail(OOC_ERR_INVALID_ARG, "ooc_mlp_forward: bad arguments");
    std::string why;
    int rc = check_device(why);
    if (rc) return fail(rc, why);
    rc = mlp_forward_host(params, X, n, y, why);
    return rc ? fail(rc, why) : OOC_OK;
}

int ooc_mlp_loss_grad(const float* params, const float* X, const float* t, int64_t n, float* grad, float* loss)
{
    if (!params || !X || !t || !grad || !loss || n <= 0) return fail(OOC_ERR_INVALID_ARG, "ooc_mlp_loss_grad: bad arguments");
    std::string why;
    int rc = check_device(why);
    if (rc) return fail(rc, why);
    rc = mlp_loss_grad_host(params, X, t, n, grad, loss, why);
    return rc ? fail(rc, why) : OOC_OK;
}

int ooc_mlp_train(float* params, const float* X, const float* t, int64_t n, int32_t epochs, int32_t batch, float lr,
                  float weight_decay, uint64_t seed, float* final_loss)
{
    if (!params || !X || !t || n <= 0) return fail(OOC_ERR_INVALID_ARG, "ooc_mlp_train: bad arguments");
    std::string why;
    int rc = check_device(why);
    if (rc) return fail(rc, why);
    rc = mlp_train_host(params, X, t, n, epochs, batch, lr, weight_decay, seed, final_loss, why);
    return rc ? fail(rc, why) : OOC_OK;
}

int ooc_costmodel_set(const float* params, int64_t n)
{
    if (params && n != kMlpParams) return fail(OOC_ERR_INVALID_ARG, "cost model needs OOC_MLP_PARAMS floats");
    costmodel_set(params, n);
    return OOC_OK;
}

const char* ooc_strerror(int code)
{
    switch (code) {
    case OOC_OK: return "ok";
    case OOC_ERR_INVALID_ARG: return "invalid argument";
    case OOC_ERR_BUDGET: return "device budget too small for any plan";
    case OOC_ERR_NOT_PINNED: return "host operand not page-locked";
    case OOC_ERR_CUDA: return "CUDA call failed";
    case OOC_ERR_NO_DEVICE: return "no usable sm_103 device";
    case OOC_ERR_TIMEOUT: return "device-side wait timed out";
    case OOC_ERR_ALLOC: return "device allocation failed";
    case OOC_ERR_UNSUPPORTED: return "unsupported form or option";
    case OOC_ERR_INJECTED: return "injected failure";
    case OOC_ERR_CAPACITY: return "output array too small";
    default: return "unknown status";
    }
}

const char* ooc_last_error(void) { return g_last_error.c_str(); }

namespace {

void fill_plan_stats(const Plan& p, ooc_stats* out)
{
    std::memset(out, 0, sizeof(*out));
    out->mb = p.mb; out->nb = p.nb; out->kb = p.kb;
    out->depth = p.nA; out->c_buffers = p.nC; out->b_buffers = p.nB; out->form = p.form;
    int64_t nblk = 0;
    for (int64_t j = 0; j < p.w; ++j)
        for (int64_t i = 0; i < p.h; ++i) nblk += p.block_class(i, j) != 0;
    out->blocks = nblk; out->steps = nblk * p.nkc;
    out->device_bytes = (int64_t)p.device_bytes;
    out->h2d_bytes = p.h2d_bytes; out->d2h_bytes = p.d2h_bytes;
    out->slices = p.slices; out->products = p.products;
    out->seconds = p.est_seconds;
}

int export_schedule(const PlanRequest& rq, ooc_stats* plan_out, ooc_sched_op* out, int64_t capacity, int64_t* count)
{
    Plan p;
    std::string why;
    int rc = make_plan(rq, p, why);
    if (rc) return fail(rc, why);
    if (plan_out) fill_plan_stats(p, plan_out);
    std::vector<Op> ops;
    build_schedule(p, ops);
    *count = (int64_t)ops.size();
    if (!out || capacity < (int64_t)ops.size()) return fail(OOC_ERR_CAPACITY, "schedule needs more entries");
    for (size_t n = 0; n < ops.size(); ++n) {
        const Op& o = ops[n];
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

int uplo_code(char uplo) { return (uplo == 'L' || uplo == 'l') ? 1 : (uplo == 'U' || uplo == 'u') ? 2 : 0; }

}  // namespace

int ooc_plan(int64_t M, int64_t N, int64_t K, int32_t elem_bytes, int32_t beta_nonzero, size_t budget,
             const ooc_opts* opts_in, ooc_stats* out)
{
    if ((elem_bytes != 4 && elem_bytes != 8) || M <= 0 || N <= 0 || K < 0 || !out)
        return fail(OOC_ERR_INVALID_ARG, "ooc_plan: bad arguments");
    ooc_opts opts;
    std::memset(&opts, 0, sizeof(opts));
    if (opts_in) opts = *opts_in;
    PlanRequest rq{M, N, K, elem_bytes, beta_nonzero != 0, false, false, budget, opts};
    Plan p;
    std::string why;
    int rc = make_plan(rq, p, why);
    if (rc) return fail(rc, why);
    fill_plan_stats(p, out);
    return OOC_OK;
}

int ooc_schedule(int64_t M, int64_t N, int64_t K, int32_t elem_bytes, int32_t beta_nonzero, size_t budget,
                 const ooc_opts* opts_in, ooc_sched_op* out, int64_t capacity, int64_t* count)
{
    if ((elem_bytes != 4 && elem_bytes != 8) || M <= 0 || N <= 0 || K < 0 || !count)
        return fail(OOC_ERR_INVALID_ARG, "ooc_schedule: bad arguments");
    ooc_opts opts;
    std::memset(&opts, 0, sizeof(opts));
    if (opts_in) opts = *opts_in;
    PlanRequest rq{M, N, K, elem_bytes, beta_nonzero != 0, false, false, budget, opts};
    return export_schedule(rq, nullptr, out, capacity, count);
}

int ooc_schedule_gemmt(char uplo, int64_t N, int64_t K, int32_t elem_bytes, int32_t beta_nonzero, size_t budget,
                       const ooc_opts* opts_in, ooc_stats* plan, ooc_sched_op* out, int64_t capacity, int64_t* count)
{
    if ((elem_bytes != 4 && elem_bytes != 8) || N <= 0 || K < 0 || !count || !uplo_code(uplo))
        return fail(OOC_ERR_INVALID_ARG, "ooc_schedule_gemmt: bad arguments");
    ooc_opts opts;
    std::memset(&opts, 0, sizeof(opts));
    if (opts_in) opts = *opts_in;
    PlanRequest rq{N, N, K, elem_bytes, beta_nonzero != 0, false, false, budget, opts};
    rq.tri = uplo_code(uplo);
    return export_schedule(rq, plan, out, capacity, count);
}

int ooc_query_device(size_t* free_bytes, double* h2d_gbps, double* d2h_gbps)
{
    std::string why;
    int rc = check_device(why);
    if (rc) return fail(rc, why);
    if (free_bytes) {
        size_t f = 0, t = 0;
        if (cudaMemGetInfo(&f, &t) != cudaSuccess) return fail(OOC_ERR_CUDA, "cudaMemGetInfo");
        *free_bytes = f;
    }
    if (!h2d_gbps && !d2h_gbps) return OOC_OK;
    static double hg = 0, dg = 0;
    static int qrc = OOC_OK;
    static std::once_flag once;
    std::call_once(once, [] {
        const size_t bytes = 256ull << 20;
        void *h = nullptr, *d = nullptr;
        cudaStream_t s = nullptr;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (cudaHostAlloc(&h, bytes, cudaHostAllocDefault) != cudaSuccess || cudaMalloc(&d, bytes) != cudaSuccess ||
            cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
            cudaEventCreate(&e1) != cudaSuccess) {
            qrc = OOC_ERR_CUDA;
        } else {
            std::memset(h, 0, bytes);
            for (int dir = 0; dir < 2; ++dir) {
                float best = 1e30f;
                for (int r = 0; r < 4; ++r) {
                    cudaEventRecord(e0, s);
                    if (dir == 0) cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, s);
                    else cudaMemcpyAsync(h, d, bytes, cudaMemcpyDeviceToHost, s);
                    cudaEventRecord(e1, s);
                    cudaEventSynchronize(e1);
                    float ms = 0;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (r > 0) best = std::min(best, ms);
                }
                (dir == 0 ? hg : dg) = (double)bytes / (best * 1e-3) / 1e9;
            }
        }
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (s) cudaStreamDestroy(s);
        if (d) cudaFree(d);
        if (h) cudaFreeHost(h);
        cudaGetLastError();
    });
    if (qrc) return fail(qrc, "link bandwidth probe failed");
    if (h2d_gbps) *h2d_gbps = hg;
    if (d2h_gbps) *d2h_gbps = dg;
    return OOC_OK;
}

int ooc_dgemm(char transA, char transB, int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t lda,
              const double* B, int64_t ldb, double beta, double* C, int64_t ldc, size_t device_budget_bytes,
              const ooc_opts* opts, ooc_stats* stats)
{
    Operands o{A, lda, B, ldb, C, ldc, alpha, beta};
    return run_ooc(transA, transB, M, N, K, o, 8, device_budget_bytes, opts, stats);
}

int ooc_sgemm(char transA, char transB, int64_t M, int64_t N, int64_t K, float alpha, const float* A, int64_t lda,
              const float* B, int64_t ldb, float beta, float* C, int64_t ldc, size_t device_budget_bytes,
              const ooc_opts* opts, ooc_stats* stats)
{
    Operands o{A, lda, B, ldb, C, ldc, (double)alpha, (double)beta};
    return run_ooc(transA, transB, M, N, K, o, 4, device_budget_bytes, opts, stats);
}

int ooc_dgemmt(char uplo, char transA, char transB, int64_t N, int64_t K, double alpha, const double* A, int64_t lda,
               const double* B, int64_t ldb, double beta, double* C, int64_t ldc, size_t device_budget_bytes,
               const ooc_opts* opts, ooc_stats* stats)
{
    const int tri = uplo_code(uplo);
    if (!tri) return fail(OOC_ERR_INVALID_ARG, "uplo must be 'L' or 'U'");
    Operands o{A, lda, B, ldb, C, ldc, alpha, beta};
    return run_ooc(transA, transB, N, N, K, o, 8, device_budget_bytes, opts, stats, tri, 0);
}

int ooc_dsyrk(char uplo, char trans, int64_t N, int64_t K, double alpha, const double* A, int64_t lda, double beta,
              double* C, int64_t ldc, size_t device_budget_bytes, const ooc_opts* opts, ooc_stats* stats)
{
    const int tri = uplo_code(uplo);
    if (!tri) return fail(OOC_ERR_INVALID_ARG, "uplo must be 'L' or 'U'");
    if (!is_n(trans) && !is_t(trans)) return fail(OOC_ERR_INVALID_ARG, "trans must be 'N' or 'T'");
    // op(A) op(A)^T: the second operand is the same host matrix with the other transpose
    Operands o{A, lda, A, lda, C, ldc, alpha, beta};
    return run_ooc(trans, is_n(trans) ? 'T' : 'N', N, N, K, o, 8, device_budget_bytes, opts, stats, tri, 0);
}

int ooc_ssyrk(char uplo, char trans, int64_t N, int64_t K, float alpha, const float* A, int64_t lda, float beta,
              float* C, int64_t ldc, size_t device_budget_bytes, const ooc_opts* opts, ooc_stats* stats)
{
    const int tri = uplo_code(uplo);
    if (!tri) return fail(OOC_ERR_INVALID_ARG, "uplo must be 'L' or 'U'");
    if (!is_n(trans) && !is_t(trans)) return fail(OOC_ERR_INVALID_ARG, "trans must be 'N' or 'T'");
    Operands o{A, lda, A, lda, C, ldc, (double)alpha, (double)beta};
    return run_ooc(trans, is_n(trans) ? 'T' : 'N', N, N, K, o, 4, device_budget_bytes, opts, stats, tri, 0);
}

int ooc_dgemm_device(char transA, char transB, int64_t M, int64_t N, int64_t K, double alpha, const double* dA,
                     int64_t lda, const double* dB, int64_t ldb, double beta, double* dC, int64_t ldc, void* stream)
{
    std::string why;
    int rc = validate(transA, transB, M, N, K, dA, lda, dB, ldb, dC, ldc, beta != 0.0, why);
    if (rc) return fail(rc, why);
    if (M == 0 || N == 0) return OOC_OK;
    rc = check_device(why);
    if (rc) return fail(rc, why);
    // TMA needs 16-byte aligned bases and row pitches; the epilogue stores pairs
    if ((lda % 2) || (ldb % 2) || (ldc % 2) || (reinterpret_cast<uintptr_t>(dA) % 16) ||
        (reinterpret_cast<uintptr_t>(dB) % 16) || (reinterpret_cast<uintptr_t>(dC) % 16))
        return fail(OOC_ERR_UNSUPPORTED, "device operands need 16-byte aligned bases and even leading dimensions");
    // one error word per device, allocated by the first call on that device
    // and cleared on the caller's stream before every launch, so that a wait
    // that gave up in an earlier call cannot end this call's kernel early
    constexpr int kMaxDev = 64;
    static std::mutex mu;
    static int* words[kMaxDev] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) {
        cudaGetLastError();
        return fail(OOC_ERR_NO_DEVICE, "no current CUDA device");
    }
    int* err = nullptr;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (!words[dev]) {
            if (cudaMalloc(&words[dev], sizeof(int)) != cudaSuccess) {
                cudaGetLastError();
                words[dev] = nullptr;
                return fail(OOC_ERR_ALLOC, "error word");
            }
        }
        err = words[dev];
    }
    if (cudaMemsetAsync(err, 0, sizeof(int), static_cast<cudaStream_t>(stream)) != cudaSuccess)
        return fail(OOC_ERR_CUDA, "clearing the error word");
    rc = launch_fp64_tile(is_n(transA), is_t(transB), M, N, K, alpha, dA, lda, dB, ldb, beta, beta != 0.0, dC, ldc,
                          err, stream, why);
    if (rc) return fail(rc, why);
    if (Inject().devword && cudaMemsetAsync(err, 0x7F, sizeof(int), static_cast<cudaStream_t>(stream)) != cudaSuccess)
        return fail(OOC_ERR_CUDA, "injected error word");
    return OOC_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ session --
// Section IV's nsteps mode: the out-of-core GEMM called once per step of an
// outer algorithm (SUMMA and its hierarchical form), all calls adding into one
// C.  The session fixes the C blocking, keeps as many C blocks as the budget
// allows in HBM across the calls (the paper keeps the last two blocks of its
// pair of C buffers back between calls), and writes them back at the end.
struct ooc_session {
    int64_t M = 0, N = 0;
    double* C = nullptr;
    int64_t ldc = 0;
    double beta = 0.0;
    size_t budget = 0;
    ooc_opts opts{};
    int64_t mb = 0, nb = 0, h = 0, w = 0;
    int32_t nR = 0;
    int32_t calls = 0;
    char* arena = nullptr;
    bool own_arena = false;
    cudaStream_t st[3] = {nullptr, nullptr, nullptr};
    size_t c_slot = 0, header = 256;
    int64_t ldc_dev = 0;
    double h2d = 0, d2h = 0, kernel_s = 0, split_s = 0, device_s = 0, flops = 0;
    int64_t launches = 0, steps = 0;
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();

    ~ooc_session()
    {
        for (auto s : st)
            if (s) {
                cudaStreamSynchronize(s);
                cudaStreamDestroy(s);
            }
        if (own_arena && arena) cudaFree(arena);
        cudaGetLastError();
    }
};

namespace {

PlanRequest session_request(const ooc_session& s, char ta, char tb, int64_t K, int32_t nR, int32_t call)
{
    ooc_opts o = s.opts;
    o.mb = s.mb;
    o.nb = s.nb;
    o.workspace = nullptr;
    o.workspace_bytes = 0;
    o.flags &= ~(OOC_PLAN_MODEL | OOC_PLAN_PAPER);
    PlanRequest rq{s.M, s.N, K, 8, s.beta != 0.0, is_t(ta), is_t(tb), s.budget, o};
    rq.nR = nR;
    rq.session_step = call;
    rq.ldc = s.ldc;
    double hg = 0, dg = 0;
    if (ooc_query_device(nullptr, &hg, &dg) == OOC_OK && hg > 0 && dg > 0) {
        rq.h2d_gbps = hg;
        rq.d2h_gbps = dg;
    }
    return rq;
}

}  // namespace

int ooc_session_create(int64_t M, int64_t N, int64_t k_hint, double beta, double* C, int64_t ldc,
                       size_t device_budget_bytes, const ooc_opts* opts, ooc_session** out)
{
    if (!out) return fail(OOC_ERR_INVALID_ARG, "null session pointer");
    *out = nullptr;
    if (M <= 0 || N <= 0 || k_hint < 0 || !C || ldc < N) return fail(OOC_ERR_INVALID_ARG, "bad C or dimensions");
    std::string why;
    int rc = check_device(why);
    if (rc) return fail(rc, why);
    if (!range_pinned(C, M, N, ldc, 8))
        return fail(OOC_ERR_NOT_PINNED, "host operands must be page-locked (cudaHostAlloc / cudaHostRegister)");
    std::unique_ptr<ooc_session> s(new ooc_session());
    s->M = M; s->N = N; s->C = C; s->ldc = ldc; s->beta = beta; s->budget = device_budget_bytes;
    if (opts) s->opts = *opts;
    if (s->opts.form == OOC_FORM_AUTO) s->opts.form = OOC_FORM_FP64;
    if (s->opts.form != OOC_FORM_FP64 && s->opts.form != OOC_FORM_OZAKI)
        return fail(OOC_ERR_INVALID_ARG, "a session runs the FP64 or Ozaki form");
    if (s->opts.workspace && s->opts.workspace_bytes < device_budget_bytes)
        return fail(OOC_ERR_INVALID_ARG, "workspace smaller than the budget");
    const int64_t k = k_hint > 0 ? k_hint : 4096;
    // the C blocking: the planner's choice for one call of inner dimension k
    {
        ooc_opts o = s->opts;
        o.workspace = nullptr;
        o.workspace_bytes = 0;
        PlanRequest rq{M, N, k, 8, true, false, false, device_budget_bytes, o};
        rq.session_step = 1;
        Plan p;
        if ((rc = make_plan(rq, p, why))) return fail(rc, why);
        s->mb = p.mb; s->nb = p.nb;
    }
    s->h = (M + s->mb - 1) / s->mb;
    s->w = (N + s->nb - 1) / s->nb;
    // as many resident blocks as fit beside the streaming rings of a call with inner dimension k
    auto fits = [&](int64_t r) {
        Plan p;
        std::string w2;
        return make_plan(session_request(*s, 'N', 'N', k, (int32_t)r, 1), p, w2) == OOC_OK;
    };
    const int64_t blocks = s->h * s->w;
    int64_t nR = 0;
    if (blocks <= (1 << 30) && fits(blocks)) nR = blocks;
    else {
        int64_t lo = 0, hi = std::min<int64_t>(blocks - 1, 1 << 30);
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) / 2;
            if (fits(mid)) lo = mid;
            else hi = mid - 1;
        }
        nR = lo;
    }
    s->nR = (int32_t)nR;
    if (s->opts.workspace) {
        s->arena = static_cast<char*>(s->opts.workspace);
    } else {
        if (cudaMalloc(&s->arena, device_budget_bytes) != cudaSuccess) {
            cudaGetLastError();
            s->arena = nullptr;
            return fail(OOC_ERR_ALLOC, "device arena of " + std::to_string(device_budget_bytes) + " bytes");
        }
        s->own_arena = true;
    }
    for (auto& st : s->st)
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess)
            return fail(OOC_ERR_CUDA, "stream creation failed");
    *out = s.release();
    return OOC_OK;
}

int ooc_session_step(ooc_session* s, char transA, char transB, int64_t K, double alpha, const double* A, int64_t lda,
                     const double* B, int64_t ldb, ooc_stats* stats)
{
    if (stats) std::memset(stats, 0, sizeof(*stats));
    if (!s) return fail(OOC_ERR_INVALID_ARG, "null session");
    const auto t_host0 = std::chrono::steady_clock::now();
    std::string why;
    int rc = validate(transA, transB, s->M, s->N, K, A, lda, B, ldb, s->C, s->ldc, true, why);
    if (rc) return fail(rc, why);
    if (K == 0 && s->calls > 0) return OOC_OK;  // adds nothing
    if (K > 0 && (!range_pinned(A, is_t(transA) ? K : s->M, is_t(transA) ? s->M : K, lda, 8) ||
                  !range_pinned(B, is_t(transB) ? s->N : K, is_t(transB) ? K : s->N, ldb, 8)))
        return fail(OOC_ERR_NOT_PINNED, "host operands must be page-locked (cudaHostAlloc / cudaHostRegister)");
    PlanRequest rq = session_request(*s, transA, transB, K, s->nR, s->calls);
    rq.lda = lda;
    rq.ldb = ldb;
    Exec x;
    x.flags = s->opts.flags;
    if ((rc = make_plan(rq, x.p, why))) return fail(rc, why);
    const Plan& p = x.p;
    if (p.mb != s->mb || p.nb != s->nb || p.nR != s->nR || p.device_bytes > s->budget)
        return fail(OOC_ERR_BUDGET, "this call's operand rings do not fit beside the resident C blocks");
    std::vector<Op> ops;
    build_schedule(p, ops);
    x.arena = s->arena;
    x.own_arena = false;
    x.own_streams = false;
    for (int i = 0; i < 3; ++i) x.st[i] = s->st[i];
    Inject inj;
    Operands o{A, lda, B, ldb, s->C, s->ldc, alpha, s->beta};
    ooc_stats st;
    std::memset(&st, 0, sizeof(st));
    if ((rc = execute(x, ops, o, 8, inj, &st))) return rc;
    x.release();
    s->c_slot = p.c_slot + p.c_aux;
    s->header = p.header;
    s->ldc_dev = p.ldc_dev;
    s->h2d += st.h2d_bytes;
    s->d2h += st.d2h_bytes;
    s->kernel_s += st.kernel_seconds;
    s->split_s += st.split_seconds;
    s->device_s += st.device_seconds;
    s->launches += st.kernel_launches;
    s->steps += st.steps;
    s->flops += 2.0 * (double)s->M * s->N * K;
    ++s->calls;
    if (stats) {
        *stats = st;
        stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_host0).count();
        stats->tflops = stats->seconds > 0 ? 2.0 * (double)s->M * s->N * K / stats->seconds / 1e12 : 0.0;
    }
    return OOC_OK;
}

int ooc_session_query(const ooc_session* s, int64_t* mb, int64_t* nb, int64_t* resident_blocks, int64_t* blocks,
                      int32_t* calls)
{
    if (!s) return fail(OOC_ERR_INVALID_ARG, "null session");
    if (mb) *mb = s->mb;
    if (nb) *nb = s->nb;
    if (resident_blocks) *resident_blocks = s->nR;
    if (blocks) *blocks = s->h * s->w;
    if (calls) *calls = s->calls;
    return OOC_OK;
}

int ooc_session_finish(ooc_session* s, ooc_stats* stats)
{
    if (stats) std::memset(stats, 0, sizeof(*stats));
    if (!s) return fail(OOC_ERR_INVALID_ARG, "null session");
    std::unique_ptr<ooc_session> own(s);
    int rc;
    if (s->calls == 0) {
        // no product was added: C = beta * C
        if ((rc = ooc_session_step(s, 'N', 'N', 0, 0.0, nullptr, 1, nullptr, s->N, nullptr))) return rc;
    }
    // the resident blocks go back to the host (schedule order: block column j outer, row i inner)
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    CK(cudaEventRecord(e0, s->st[kStreamD2H]));
    for (int64_t r = 0; r < s->nR; ++r) {
        const int64_t j = r / s->h, i = r % s->h;
        const int64_t rows = std::min(s->mb, s->M - i * s->mb), cols = std::min(s->nb, s->N - j * s->nb);
        const char* src = s->arena + s->header + (size_t)r * s->c_slot;
        double* dst = s->C + i * s->mb * s->ldc + j * s->nb;
        CK(cudaMemcpy2DAsync(dst, s->ldc * 8, src, s->ldc_dev * 8, cols * 8, rows, cudaMemcpyDeviceToHost,
                             s->st[kStreamD2H]));
        s->d2h += (double)rows * cols * 8;
    }
    CK(cudaEventRecord(e1, s->st[kStreamD2H]));
    CK(cudaStreamSynchronize(s->st[kStreamD2H]));
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    s->device_s += ms * 1e-3;
    if (stats) {
        stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - s->t0).count();
        stats->device_seconds = s->device_s;
        stats->kernel_seconds = s->kernel_s;
        stats->split_seconds = s->split_s;
        stats->tflops = stats->seconds > 0 ? s->flops / stats->seconds / 1e12 : 0.0;
        stats->h2d_bytes = s->h2d;
        stats->d2h_bytes = s->d2h;
        stats->mb = s->mb; stats->nb = s->nb;
        stats->form = s->opts.form;
        stats->blocks = s->h * s->w;
        stats->steps = s->steps;
        stats->device_bytes = (int64_t)s->budget;
        stats->kernel_launches = s->launches;
    }
    return OOC_OK;
}

int ooc_session_free(ooc_session* s)
{
    delete s;
    return OOC_OK;
}

int ooc_schedule_session(int64_t M, int64_t N, int64_t K, int32_t beta_nonzero, size_t budget, const ooc_opts* opts_in,
                         int32_t resident_blocks, int32_t call, ooc_stats* plan, ooc_sched_op* out, int64_t capacity,
                         int64_t* count)
{
    if (M <= 0 || N <= 0 || K < 0 || !count || resident_blocks < 0 || call < 0)
        return fail(OOC_ERR_INVALID_ARG, "ooc_schedule_session: bad arguments");
    ooc_opts opts;
    std::memset(&opts, 0, sizeof(opts));
    if (opts_in) opts = *opts_in;
    PlanRequest rq{M, N, K, 8, beta_nonzero != 0, false, false, budget, opts};
    rq.nR = resident_blocks;
    rq.session_step = call;
    return export_schedule(rq, plan, out, capacity, count);
}
