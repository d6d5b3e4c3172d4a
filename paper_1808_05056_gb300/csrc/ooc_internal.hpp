// Internal interfaces of libooc: the plan, the issued schedule and the kernel
// launchers.  Host-only declarations; nothing here is exported.
#pragma once
#include <algorithm>
#include <cstddef>
#include <cstdint>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "../../include/ooc.h"

namespace ooc {

// ---------------------------------------------------------------- plan ----
// One out-of-core plan: C is cut into h x w blocks of mb x nb, K into nkc
// chunks of kb (Section IV partitioner, generalised with K-chunks and
// ragged edges); A chunks (mb x kb), B chunks (kb x nb) and C blocks live in
// rings of device slots.
struct Plan {
    int64_t M = 0, N = 0, K = 0;
    int32_t es = 8;          // host element bytes (8 FP64, 4 FP32)
    int32_t form = OOC_FORM_FP64;
    bool beta_nz = false;
    bool ta = false, tb = false;
    bool paper = false;
    int64_t lda_host = 0, ldb_host = 0, ldc_host = 0;  // 0: assume contiguous host rows
    int64_t mb = 0, nb = 0, kb = 0;
    int64_t h = 0, w = 0, nkc = 0;
    int32_t nA = 0, nB = 0, nC = 0;
    int32_t slices = 0, products = 0;
    // device layout (bytes); each slot is 256-byte aligned
    size_t a_slot = 0, b_slot = 0, c_slot = 0;      // raw operand slots
    size_t a_aux = 0, b_aux = 0, c_aux = 0;         // per-slot form scratch (split planes, FP64 acc)
    size_t header = 256;                            // error word etc.
    size_t device_bytes = 0;
    double h2d_bytes = 0, d2h_bytes = 0;
    double est_seconds = 0;
    // device leading dimensions (elements) of the slots, per stored layout
    int64_t lda_dev = 0, ldb_dev = 0, ldc_dev = 0;
    // Triangular update (GEMMT / SYRK): only elements with col - row <= tri_off
    // (tri 1, lower) or col - row >= tri_off (tri 2, upper) of C are updated.
    int32_t tri = 0;
    int64_t tri_off = 0;
    // Session mode (Section IV's nsteps invocations): the first nR updated
    // blocks in schedule order keep a dedicated device slot for the whole
    // session (slots nA + nB + nC ..), placed first in the arena so that every
    // call of the session finds them at the same address.  session_step is -1
    // for a single call, 0 for a session's first call, > 0 for later calls
    // (which accumulate onto the partial sums instead of applying beta).
    int32_t nR = 0;
    int32_t session_step = -1;
    // Whole-K B slices of the next block column are copied ahead, in row ranges
    // between the A loads of the current column (schedule generator, plan.cpp)
    bool b_prefetch = true;
    // Split forms: A and B loads land in raw staging areas (nSA for A, nSB for B,
    // used in turn), and a split op on the compute stream turns the staged data
    // into the bf16 planes of the operand's slot; the slots hold planes only
    // (layout in plan.cpp).  Two A areas let the next block's A copy run while
    // the current one waits for its split; one B area suffices when each whole-K
    // B slice is loaded once per block column.
    bool staged = false;
    int32_t nSA = 0, nSB = 0;

    int64_t rows_of(int64_t i) const { return (i + 1) * mb <= M ? mb : M - i * mb; }
    int64_t cols_of(int64_t j) const { return (j + 1) * nb <= N ? nb : N - j * nb; }
    int64_t k_of(int64_t c) const { return (c + 1) * kb <= K ? kb : K - c * kb; }
    int32_t slots() const { return nA + nB + nC + nR; }
    // staged plans: staging area k of operand mat (kMatA, kMatB) as a slot id past the slots
    int32_t stage_slot(int mat, int k) const { return slots() + 2 * mat + k; }
    // 0: block (i, j) holds no updated element (skipped); 1: all of it is
    // updated; 2: it straddles the edge of the updated part (masked epilogue,
    // and the block is loaded so that its other elements go back unchanged)
    int block_class(int64_t i, int64_t j) const
    {
        if (!tri) return 1;
        const int64_t r0 = i * mb, c0 = j * nb;
        const int64_t lo = c0 - (r0 + rows_of(i) - 1), hi = c0 + cols_of(j) - 1 - r0;  // min / max of col - row
        if (tri == 1) return lo > tri_off ? 0 : (hi <= tri_off ? 1 : 2);
        return hi < tri_off ? 0 : (lo >= tri_off ? 1 : 2);
    }
    // the diagonal offset in block (i, j)'s own coordinates
    int64_t block_off(int64_t i, int64_t j) const { return tri_off + i * mb - j * nb; }
};

struct PlanRequest {
    int64_t M, N, K;
    int32_t es;
    bool beta_nz, ta, tb;
    size_t budget;
    ooc_opts opts;
    double h2d_gbps = 200.0, d2h_gbps = 190.0;  // link model for the estimate
    int64_t lda = 0, ldb = 0, ldc = 0;          // host leading dimensions (0: rows are contiguous)
    int32_t tri = 0;                            // triangular update of C (Plan::tri)
    int64_t tri_off = 0;
    int32_t nR = 0;                             // resident C blocks (Plan::nR)
    int32_t session_step = -1;
};

// Returns OOC_OK and fills `plan`, or an error code with a message in `why`.
// With OOC_PLAN_MODEL in rq.opts.flags and a cost model installed, the plan is
// the candidate with the smallest predicted time; otherwise the heuristic best.
int make_plan(const PlanRequest& rq, Plan& plan, std::string& why);

// The best `max_n` distinct candidate plans by the heuristic estimate (fitting the budget).
int plan_candidates(const PlanRequest& rq, int max_n, std::vector<Plan>& out, std::string& why);

// --- schedule cost model (mlp.cu, plan.cpp) ---------------------------------
constexpr int kMlpIn = 16;
constexpr int kMlpParams = 64 * 16 + 64 + 64 * 64 + 64 + 64 + 1;
void plan_features(const Plan& p, const PlanRequest& rq, float* f);
int mlp_forward_host(const float* params, const float* X, int64_t n, float* y, std::string& why);
int mlp_loss_grad_host(const float* params, const float* X, const float* t, int64_t n, float* grad, float* loss,
                       std::string& why);
int mlp_train_host(float* params, const float* X, const float* t, int64_t n, int epochs, int batch, float lr,
                   float wd, uint64_t seed, float* final_loss, std::string& why);
bool costmodel_get(std::vector<float>& params);
void costmodel_set(const float* params, int64_t n);

// -------------------------------------------------------------- schedule --
enum OpKind { kH2D = 0, kKernel = 1, kD2H = 2, kRecord = 3, kWait = 4, kSplit = 5 };
enum StreamId { kStreamH2D = 0, kStreamCompute = 1, kStreamD2H = 2 };
enum MatId { kMatA = 0, kMatB = 1, kMatC = 2 };

struct Tag {
    int64_t m = -1, r = -1, c = -1, v = -1;
    bool operator==(const Tag& o) const { return m == o.m && r == o.r && c == o.c && v == o.v; }
};

struct Op {
    int32_t kind = 0, stream = 0, event = -1;
    int32_t wslot = -1;
    Tag wtag;
    int32_t nr = 0;
    int32_t rslot[3] = {-1, -1, -1};
    Tag rtag[3];
    // execution detail
    int64_t i = 0, j = 0, kc = 0;  // block row, block column, K chunk
    bool first = false, last = false;
    int32_t kernel = -1;           // pipeline-language kernels: which built-in
    int32_t mode = 0;              // and how its output tile starts (pipe.cpp)
    int32_t part = 0, nparts = 1;  // H2D: rows [part, part + 1) * rows / nparts of the operand chunk
};

// Events: ready(s) after a load into slot s, free(s) after a kernel read s,
// out(s) after the D2H of C slot s, done(s) after the last kernel of C slot s;
// staged plans: sready(a) after a load into staging area a (a = stage_slot id),
// staged(a) after the split that emptied it.
inline int32_t ev_ready(const Plan&, int32_t s) { return s; }
inline int32_t ev_free(const Plan& p, int32_t s) { return p.slots() + s; }
inline int32_t ev_out(const Plan& p, int32_t s) { return 2 * p.slots() + s; }
inline int32_t ev_done(const Plan& p, int32_t s) { return 3 * p.slots() + s; }
inline int32_t ev_staged(const Plan& p, int32_t a) { return 4 * p.slots() + (a - p.slots()); }
inline int32_t ev_sready(const Plan& p, int32_t a) { return 4 * p.slots() + 4 + (a - p.slots()); }
inline int32_t n_events(const Plan& p) { return 4 * p.slots() + 8; }

void build_schedule(const Plan& plan, std::vector<Op>& ops);

// split-form scratch of a slot (bf16 planes, Ozaki exponents) -- plan.cpp
int split_planes(const Plan& p);
int64_t split_rows_pad(int64_t rows);
int64_t split_k_pad(const Plan& p);
size_t split_planes_bytes(const Plan& p, int64_t rows);
size_t split_aux_bytes(const Plan& p, int64_t rows);

// slot byte offsets inside the arena
size_t slot_offset(const Plan& p, int32_t slot);
size_t slot_aux_offset(const Plan& p, int32_t slot);

// ------------------------------------------------- pipeline language --
// A compiled pipeline description (pipe.cpp): the operands' tiles and rings,
// and the schedule with its events, ready for the executor (pipe_exec.cu).
struct PipeOperand {
    std::string name;
    void* host = nullptr;
    int64_t rows = 0, cols = 0, ld = 0;
    int32_t es = 8;
    int64_t tr = 0, tc = 0;      // tile rows / columns
    int32_t ring = 0;            // device slots
    int32_t slot0 = 0;           // its first slot (global slot numbering)
    int64_t ld_dev = 0;          // slot leading dimension (elements)
    size_t slot_bytes = 0;
    bool bound = false;
    int64_t tile_rows(int64_t r) const { return std::min(tr, rows - r * tr); }
    int64_t tile_cols(int64_t c) const { return std::min(tc, cols - c * tc); }
};

struct PipeProgram {
    std::vector<PipeOperand> operands;
    std::vector<Op> ops;
    int32_t slots = 0, events = 0;
    size_t header = 256, device_bytes = 0;
    std::vector<size_t> slot_off;            // byte offset of each slot in the arena
};

enum PipeKernel { kPipeGemm = 0, kPipeAxpby = 1 };
// how the output tile of a kernel op starts: loaded from the host (apply the
// beta-like parameter), claimed without data (overwrite), or already written
// by an earlier kernel op (accumulate)
enum PipeMode { kPipeLoaded = 0, kPipeFresh = 1, kPipeAccumulate = 2 };

struct PipeSource;  // a parsed description
int pipe_parse(const std::string& text, std::shared_ptr<PipeSource>& out, std::vector<std::string>& operand_names,
               std::string& why);
int pipe_compile(const PipeSource& src, std::vector<PipeOperand> operands, const std::map<std::string, double>& vars,
                 PipeProgram& prog, std::string& why);

// ---------------------------------------------------------- kernel side --
// Tensor-map encoder (driver entry point fetched at first use).
int encode_map_2d(void* map_out, int dtype /*0 f64, 1 bf16, 2 f32*/, const void* base,
                  uint64_t inner, uint64_t outer, uint64_t ld_elems, uint32_t box_inner,
                  uint32_t box_outer, int swizzle128, std::string& why);

// FP64 tile GEMM on device operands (one C block, one K chunk):
// C = alpha*op(A)*op(B) + (read_c ? beta*C : 0).
// a_kmajor: A stored rows x K (else K x rows); b_kmajor: B stored cols x K (else K x cols).
// tri (1 lower, 2 upper) limits the update to elements with col - row <= / >=
// tri_off; tiles holding no such element are not computed.
int launch_fp64_tile(bool a_kmajor, bool b_kmajor, int64_t M, int64_t N, int64_t K, double alpha,
                     const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
                     bool read_c, double* C, int64_t ldc, int* err, void* stream,
                     std::string& why, int tri = 0, int64_t tri_off = 0);

// Grouped FP64 tile GEMM: the problems' tiles in one persistent launch, each
// problem's operands already on the device (conventions as launch_fp64_tile,
// full updates only); at most kGroupMax problems.  *tiles_out (nullable)
// receives the launch's work items.
struct Fp64GroupSpec {
    const double* A = nullptr;
    int64_t lda = 0;
    const double* B = nullptr;
    int64_t ldb = 0;
    double* C = nullptr;
    int64_t ldc = 0;
    int64_t M = 0, N = 0, K = 0;
    double alpha = 1.0, beta = 0.0;
    bool read_c = false;
};
constexpr int kGroupMax = 64;
int launch_fp64_group(bool a_kmajor, bool b_kmajor, const Fp64GroupSpec* probs, int count, int* err, void* stream,
                      std::string& why, int64_t* tiles_out = nullptr);

// --- tensor-core split-product forms (tc_gemm.cu) -------------------------
// A group: pairs (A plane, B plane) accumulated into one FP32 TMEM accumulator
// and added into FP64 with weight 2^scale_exp after every K chunk.
struct TcGroupSpec {
    int na = 0, nb = 0, np = 0;
    int aplane[4] = {0, 0, 0, 0}, bplane[4] = {0, 0, 0, 0};  // planes loaded per K block
    int pa[6] = {0, 0, 0, 0, 0, 0}, pb[6] = {0, 0, 0, 0, 0, 0};  // pair -> loaded A / B index
    int scale_exp = 0;   // weight of pair 0's accumulator
    int scale_exp2 = 0;  // weight of the second accumulator (exact form: pair 1)
};

struct TcProblem {
    int64_t M = 0, N = 0, k_pad = 0;  // C block rows / cols, padded K (multiple of 64)
    int chunk = 0;                     // K elements per FP64 flush (multiple of 64)
    const void* a_planes = nullptr;    // [a_nplanes][a_rows_pad][k_pad] bf16
    int64_t a_rows_pad = 0;
    int a_nplanes = 0;
    const void* b_planes = nullptr;    // [b_nplanes][b_rows_pad][k_pad] bf16 (rows = C columns)
    int64_t b_rows_pad = 0;
    int b_nplanes = 0;
    int ngroups = 0;
    TcGroupSpec groups[64];
    double alpha = 1.0, beta = 0.0;
    bool read_c = false, c_fp32 = false;
    void* C = nullptr;
    int64_t ldc = 0;
    const int* row_exp = nullptr;      // per-row power-of-two scale (Ozaki), nullable
    const int* col_exp = nullptr;
    int* err = nullptr;
    bool df32 = false;                 // two accumulators per group, double-float drain (BF16x3)
    int kblock = 64;                   // K block per pipeline stage: 64 or 32
    int tri = 0;                       // epilogue mask as in launch_fp64_tile
    int64_t tri_off = 0;
};

int tc_max_groups();
void ozaki_groups(TcProblem& P, int S);
// C = alpha op(A) op(B) + beta C on device FP64 operands in the Ozaki form (S
// digit planes per operand in `scratch`, at least ozaki_device_scratch bytes);
// operand conventions as launch_fp64_tile.
size_t ozaki_device_scratch(int64_t M, int64_t N, int64_t K, int S);
int ozaki_gemm_device(bool a_kmajor, bool b_kmajor, int64_t M, int64_t N, int64_t K, double alpha, const double* A,
                      int64_t lda, const double* B, int64_t ldb, double beta, bool read_c, double* C, int64_t ldc,
                      int S, void* scratch, size_t scratch_bytes, int* err, void* stream, std::string& why, int tri = 0,
                      int64_t tri_off = 0);
int launch_tc_terms(const TcProblem& P, void* stream, std::string& why);
int launch_split_bf16x3(const float* X, int64_t sr, int64_t sk, int rows, int K, int rows_pad, int k_pad,
                        void* planes, void* stream, std::string& why);
int launch_split_ozaki(const double* X, int64_t sr, int64_t sk, int rows, int K, int rows_pad, int k_pad, int S,
                       int beta, void* planes, int* rowexp, unsigned long long* rowmax, void* stream,
                       std::string& why);
int encode_map_3d_bf16(void* map_out, const void* base, uint64_t inner, uint64_t rows, uint64_t planes,
                       uint32_t box_inner, uint32_t box_rows, std::string& why);

// Ozaki digit width and the largest K chunk whose digit products sum exactly in FP32
constexpr int kOzakiBeta = 6;
// digits per operand: 8 (48 bits) for the GEMM entry points unless opts->slices
// asks otherwise; 9 (54 bits, FP64's 53-bit significand covered) for the
// updates inside the factorizations, whose factors must track FP64's
constexpr int kOzakiSlicesGemm = 8;
constexpr int kOzakiSlicesFactor = 9;
constexpr int kOzakiMaxSlices = 10;
constexpr int kOzakiChunk = 4096;
// BF16x3: K between drains of the leading product's round-toward-zero FP32
// accumulator (32 accumulations of up to one ulp each: 2^-18 of sum |x||y|)
constexpr int kBf16x3Chunk = 512;

int device_sm_count();
void set_error(const std::string& msg);

bool host_range_pinned(const void* base, int64_t rows, int64_t cols, int64_t ld, int es);
int device_check(std::string& why);  // OOC_OK when an sm_103 device is current

// The whole out-of-core pipeline on host operands (ooc_dgemm / ooc_sgemm /
// ooc_dgemmt), for the drivers built on it (TRSM, Cholesky).
int run_gemm_host(char ta, char tb, int64_t M, int64_t N, int64_t K, double alpha, const void* A, int64_t lda,
                  const void* B, int64_t ldb, double beta, void* C, int64_t ldc, int es, size_t budget,
                  const ooc_opts* opts, ooc_stats* stats, int tri, int64_t tri_off);

}  // namespace ooc
