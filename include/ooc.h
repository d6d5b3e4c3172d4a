/*
 * ooc.h — C ABI of the GB300 out-of-core GEMM library (libooc.so).
 *
 * The problem is the one stated in Section IV of the libhclooc paper
 * (arXiv:1808.05056): C = alpha * A * B + beta * C with A of M x K, B of K x N
 * and C of M x N, where the matrices live in host memory and together exceed
 * the device memory the caller grants.  The library partitions A into
 * horizontal slices, B into vertical slices and C into blocks (Section IV,
 * partitioner paragraph and Fig. 2), streams them through a budget-sized set of
 * device buffers (the five pipeline stages S(b_j), S(a_i), S(c_ij), GEMM,
 * R(c_ij) of Section IV) and runs the per-block product with its own sm_103a
 * kernels.
 *
 * Conventions for every call below
 *   - Storage is row-major: element (r, c) of a stored matrix X with leading
 *     dimension ldX is X[r * ldX + c].  trans is 'N' (op(X) = X) or 'T'
 *     (op(X) = X^T); for transA == 'N' A is stored M x K (lda >= K), for 'T'
 *     it is stored K x M (lda >= M); likewise B is K x N (ldb >= N) or N x K
 *     (ldb >= K); C is M x N (ldc >= N).
 *   - Host pointers must point to page-locked memory (cudaHostAlloc or
 *     cudaHostRegister'ed by the caller): the call checks and returns
 *     OOC_ERR_NOT_PINNED instead of staging through pageable memory.
 *   - The caller owns every host buffer; the library never frees or keeps
 *     them.  The call is synchronous: it returns when C is back on the host.
 *   - beta == 0 never reads C (NaN in C is ignored); K == 0 gives C = beta*C;
 *     M == 0 or N == 0 is a no-op returning OOC_OK.
 *   - Device memory: at most device_budget_bytes are used for the operand
 *     buffers.  If opts->workspace is non-NULL the buffers are carved from
 *     that caller-owned device allocation (which must hold
 *     device_budget_bytes) and nothing is allocated; otherwise one arena of
 *     at most device_budget_bytes is allocated and freed before return.
 *   - Errors: every call returns OOC_OK (0) or a negative OOC_ERR_* code and
 *     never aborts the process.  ooc_strerror() names a code; ooc_last_error()
 *     gives a one-line detail of the last failure on the calling thread.
 */
#ifndef OOC_H
#define OOC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define OOC_OK 0
#define OOC_ERR_INVALID_ARG (-1)    /* bad trans, dims, leading dimensions or options   */
#define OOC_ERR_BUDGET (-2)         /* budget below the smallest plan for this problem  */
#define OOC_ERR_NOT_PINNED (-3)     /* a host operand is not page-locked                */
#define OOC_ERR_CUDA (-4)           /* a CUDA runtime/driver call failed                */
#define OOC_ERR_NO_DEVICE (-5)      /* no usable sm_103 device                          */
#define OOC_ERR_TIMEOUT (-6)        /* a bounded device-side wait gave up               */
#define OOC_ERR_ALLOC (-7)          /* device arena allocation failed                   */
#define OOC_ERR_UNSUPPORTED (-8)    /* form/option not available for this call          */
#define OOC_ERR_INJECTED (-9)       /* failure injected by OOC_FAULT_INJECT (testing)   */
#define OOC_ERR_CAPACITY (-10)      /* output array too small (schedule export)         */

/* ---- contraction forms ----------------------------------------------- */
#define OOC_FORM_AUTO 0    /* dgemm: FP64; sgemm: BF16x3                                 */
#define OOC_FORM_FP64 1    /* plain FP64 tiles (FP64 tensor-core MMA)                    */
#define OOC_FORM_OZAKI 2   /* FP64-accurate: Ozaki bf16 slice products, FP64 accumulate  */
#define OOC_FORM_BF16X3 3  /* FP32-accurate: three-piece bf16 split, six products        */

/* ---- plan selection flags (ooc_opts.flags) --------------------------- */
#define OOC_PLAN_PAPER 1u  /* Section IV partitioner: equal h x w split, 2A + 1B + 2C buffers */
#define OOC_PLAN_MODEL 4u  /* choose among candidates with the installed cost model (ooc_costmodel_set) */

/*
 * Options; a zero-initialised struct means "choose automatically".
 * mb, nb, kb: C block rows, C block columns and K-chunk length.
 * depth: A-slice buffers (2 or 3); c_buffers: C-block buffers; b_buffers:
 * B-chunk buffers (a whole column of B chunks keeps B resident per column).
 * slices: Ozaki slice count (0 = chosen from the input exponent spread).
 * workspace/workspace_bytes: optional caller-owned device memory for the
 * buffers (see the conventions above).
 */
typedef struct {
    int32_t form;
    int32_t depth;
    int32_t c_buffers;
    int32_t slices;
    int64_t mb, nb, kb;
    uint32_t flags;
    int32_t b_buffers;   /* B-slot ring size (0 = automatic)                       */
    void* workspace;
    size_t workspace_bytes;
} ooc_opts;

/* What a call did; every field is filled on OOC_OK. */
typedef struct {
    double seconds;          /* host wall time of the call                          */
    double device_seconds;   /* first H2D start to last D2H end (CUDA events)       */
    double kernel_seconds;   /* summed duration of the tile-contraction launches
                                and the split forms' splitting kernels              */
    double tflops;           /* 2*M*N*K / seconds / 1e12 (transfers included)       */
    double h2d_bytes;        /* bytes copied host -> device                          */
    double d2h_bytes;        /* bytes copied device -> host                          */
    int64_t mb, nb, kb;      /* plan used                                            */
    int32_t depth, c_buffers, b_buffers, form;
    int64_t blocks;          /* C blocks (h * w)                                     */
    int64_t steps;           /* block x K-chunk steps (tile launches)                */
    int64_t device_bytes;    /* device buffer bytes the plan uses                    */
    int32_t slices;          /* Ozaki slices / BF16x3 pieces used                    */
    int32_t products;        /* slice products per tile                              */
    int64_t kernel_launches; /* kernels the call launched (tile + split kernels)    */
    double split_seconds;    /* share of kernel_seconds spent in the split forms'
                                splitting kernels (0 for FP64 and in graph mode)    */
} ooc_stats;

/*
 * Out-of-core DGEMM: C = alpha * op(A) * op(B) + beta * C, FP64 host
 * operands (Section IV problem statement; per-block update c_ij =
 * alpha a_i b_j + beta c_ij of the DGEMM stage).  opts->form selects plain
 * FP64 tiles (default) or the FP64-accurate Ozaki form.  opts and stats may
 * be NULL.
 */
int ooc_dgemm(char transA, char transB, int64_t M, int64_t N, int64_t K, double alpha,
              const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
              double* C, int64_t ldc, size_t device_budget_bytes, const ooc_opts* opts,
              ooc_stats* stats);

/*
 * Out-of-core SGEMM with FP32-accurate BF16x3 tiles: FP32 host operands and
 * result, the same problem statement as ooc_dgemm.  alpha and beta are
 * applied in FP64 before the result is rounded to FP32.
 */
int ooc_sgemm(char transA, char transB, int64_t M, int64_t N, int64_t K, float alpha,
              const float* A, int64_t lda, const float* B, int64_t ldb, float beta,
              float* C, int64_t ldc, size_t device_budget_bytes, const ooc_opts* opts,
              ooc_stats* stats);

/* One GEMM of a batch: the arguments of ooc_dgemm for one problem. */
typedef struct {
    char transA, transB;
    char reserved[6];
    int64_t M, N, K;
    double alpha, beta;
    const double* A;
    int64_t lda;
    const double* B;
    int64_t ldb;
    double* C;
    int64_t ldc;
} ooc_gemm_desc;

#define OOC_BATCH_GRAPH 2u     /* capture the whole batched pipeline as one CUDA graph, then launch it */
#define OOC_BATCH_STREAMED 16u /* run every batched problem through its own out-of-core pipeline */

/*
 * A stream of uneven out-of-core DGEMMs in one call (each one the Section IV
 * problem on its own operands; problems must not share output memory).  The
 * device budget is split into two halves.  FP64 batches whose problems each
 * fit whole in half the budget (A, B and C, rows padded to an even length)
 * run grouped, unless OOC_BATCH_STREAMED is set: consecutive problems with
 * the same transposes are packed into one half (at most 64 per group), copied
 * in with one copy per operand, multiplied by one persistent launch over all
 * their tiles and copied out, groups alternating halves so that one group's
 * copies overlap the other's kernel; stats->steps then counts groups,
 * stats->blocks problems, and stats->mb / nb / kb stay 0: grouped problems are
 * not planned, so opts' planner flags (OOC_PLAN_MODEL) have no effect there.
 * Otherwise consecutive problems alternate halves
 * and compute streams, so the copies and kernels of problem g + 1 overlap
 * problem g, while problem g + 2 waits for problem g to finish; each problem
 * is planned for half the budget with opts (form: FP64 or Ozaki).
 * With OOC_BATCH_GRAPH in opts->flags the issued copies, kernels and events
 * are captured into one CUDA graph and launched as a single graph.  stats
 * (nullable) receives totals: seconds, device_seconds, kernel_seconds (0 in
 * graph mode, where launches inside the graph are not timed), tflops (sum of
 * 2MNK over the call's wall time), bytes, blocks, steps, kernel_launches and
 * the arena size in device_bytes.  Synchronous.
 */
int ooc_dgemm_batched(int32_t count, const ooc_gemm_desc* descs, size_t device_budget_bytes,
                      const ooc_opts* opts, ooc_stats* stats);

/*
 * In-core device GEMM (the paper's runtime DGEMM call of the pipeline's
 * compute stage): C = alpha * op(A) * op(B) + beta * C on device pointers,
 * FP64, enqueued on `stream` (a cudaStream_t, NULL = legacy default stream)
 * and not synchronised.  Same layout rules as ooc_dgemm, plus 16-byte aligned
 * device bases and even leading dimensions (else OOC_ERR_UNSUPPORTED).  The
 * first call on each device allocates a 4-byte device error word kept for the
 * process; every call clears it on `stream` before its launch.  The call does
 * not wait for the kernel, so it cannot report a device-side wait that gave up
 * (the kernel's bounded waits end it early in that case and C is left
 * incomplete); callers that need that status use ooc_dgemm.
 */
int ooc_dgemm_device(char transA, char transB, int64_t M, int64_t N, int64_t K, double alpha,
                     const double* dA, int64_t lda, const double* dB, int64_t ldb, double beta,
                     double* dC, int64_t ldc, void* stream);

/*
 * No-allocation variant of ooc_dgemm.  The paper has no counterpart: this entry
 * point is for callers that cannot call cudaMalloc -- a process whose device
 * memory is owned by another allocator (for example a framework's caching
 * allocator that has reserved the pool), or a latency-bound caller that cannot
 * take the device-wide synchronisation of cudaFree.  It allocates nothing: the
 * device buffers are carved from one fixed array of OOC_NOALLOC_MAX_BYTES
 * (32 MiB) in the library's device memory, which every GPU that loads the
 * library holds until the process exits; it creates no streams or events and
 * issues all copies and tile kernels, in order, on `stream` (a cudaStream_t,
 * NULL = legacy default stream), so copies do not overlap the kernels.
 * Arguments are those of ooc_dgemm (FP64, plain FP64 form, pinned host
 * operands) with device_budget_bytes <= OOC_NOALLOC_MAX_BYTES, else
 * OOC_ERR_INVALID_ARG.  The call is synchronous.  The first call on a device
 * (that device current) looks up the array's address; make it before any
 * stream capture.  The address is kept for the process: do not call this
 * entry point again after cudaDeviceReset.  All calls share the array and it keeps the last call's
 * contents; calls that overlap on the GPU race, so serialise them.
 */
#define OOC_NOALLOC_MAX_BYTES (32u << 20)
int ooc_dgemm_noalloc(char transA, char transB, int64_t M, int64_t N, int64_t K, double alpha,
                      const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
                      double* C, int64_t ldc, size_t device_budget_bytes, void* stream);

/* ---- level-3 operations beyond GEMM ------------------------------------ */
/* Section VII of the paper names the rest of level-3 BLAS as the next step
 * for the out-of-core pipeline; these run through the same planner, schedule
 * and tile kernels as ooc_dgemm. */

/*
 * GEMMT: C = alpha * op(A) * op(B) + beta * C on one triangle of the N x N
 * matrix C only: uplo 'L' updates the elements with column <= row, 'U' those
 * with column >= row.  op(A) is N x K and op(B) is K x N (layouts as for
 * ooc_dgemm with M = N).  Elements of the other triangle keep their values:
 * blocks of C that hold no updated element are never copied, and blocks that
 * straddle the diagonal are copied to the device and back whole (so the host
 * memory of the other triangle must not change during the call).  beta == 0
 * never reads the updated triangle.  opts->form: FP64 (default) or Ozaki.
 * stats->tflops counts N (N + 1) K flops.
 */
int ooc_dgemmt(char uplo, char transA, char transB, int64_t N, int64_t K, double alpha,
               const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
               double* C, int64_t ldc, size_t device_budget_bytes, const ooc_opts* opts,
               ooc_stats* stats);

/*
 * SYRK: C = alpha * op(A) * op(A)^T + beta * C on the uplo triangle of the
 * N x N matrix C; trans 'N': A is stored N x K (lda >= K) and the update is
 * A A^T; 'T': A is stored K x N (lda >= N) and the update is A^T A.  Same
 * rules as ooc_dgemmt.  ooc_ssyrk takes FP32 operands and runs the BF16x3
 * form (alpha and beta applied in FP64 before rounding to FP32).
 */
int ooc_dsyrk(char uplo, char trans, int64_t N, int64_t K, double alpha, const double* A,
              int64_t lda, double beta, double* C, int64_t ldc, size_t device_budget_bytes,
              const ooc_opts* opts, ooc_stats* stats);
int ooc_ssyrk(char uplo, char trans, int64_t N, int64_t K, float alpha, const float* A,
              int64_t lda, float beta, float* C, int64_t ldc, size_t device_budget_bytes,
              const ooc_opts* opts, ooc_stats* stats);

/*
 * TRSM: solve op(A) X = alpha B (side 'L', A of order M) or X op(A) = alpha B
 * (side 'R', A of order N) for X, which overwrites the M x N matrix B.  A is
 * triangular: uplo 'L' or 'U' names the stored triangle (the other one is not
 * read); transA 'N' or 'T' gives op(A); diag 'U' takes the diagonal as ones
 * (not read), 'N' reads it.  Left-looking over panels of X: each panel is
 * updated with one out-of-core GEMM over the panels already solved (opts->form
 * FP64 or Ozaki) and then solved in device memory.  alpha == 0 sets B to zero
 * without reading it.  No check for a singular A: a zero diagonal element
 * gives infinities or NaN, as in BLAS.  The call allocates one device arena of
 * device_budget_bytes (opts->workspace must be NULL).  stats: seconds, tflops
 * (M^2 N flops for side 'L', M N^2 for 'R'), bytes moved, GEMM calls in steps.
 */
int ooc_dtrsm(char side, char uplo, char transA, char diag, int64_t M, int64_t N, double alpha,
              const double* A, int64_t lda, double* B, int64_t ldb, size_t device_budget_bytes,
              const ooc_opts* opts, ooc_stats* stats);

/*
 * POTRF: Cholesky factorisation of the symmetric positive definite N x N
 * matrix A in place: uplo 'L' gives A = L L^T with L in the lower triangle,
 * 'U' gives A = U^T U with U in the upper triangle; the other triangle is
 * neither used nor changed.  Left-looking over panels: each panel is updated
 * with one out-of-core GEMMT (opts->form FP64 or Ozaki) and factored in device
 * memory.  *info is 0 on success, or j + 1 when the leading minor of order
 * j + 1 is not positive definite (the status is still OOC_OK; panels before
 * the one holding column j are final, the rest of A is unspecified).  Same
 * arena rule as ooc_dtrsm; stats->tflops counts N^3 / 3 flops.
 */
int ooc_dpotrf(char uplo, int64_t N, double* A, int64_t lda, size_t device_budget_bytes,
               const ooc_opts* opts, ooc_stats* stats, int64_t* info);

/*
 * GETRF: LU factorisation with partial pivoting of the N x N matrix A in
 * place, A = P L U: L unit lower triangular (stored below the diagonal), U
 * upper triangular (on and above it).  ipiv (host, N entries, 0-based): at
 * step j row j was exchanged with row ipiv[j] >= j, applied in order j = 0, 1,
 * ...; the pivot is the first row with the largest |a| in the column (a NaN
 * is never chosen while a number remains; a column with no comparable entry
 * keeps row j).  Right-
 * looking over panels of t columns: the (N - c0) x t panel is factored in
 * device memory (recursive halving; 64-column panels by one cooperative kernel
 * with a bounded grid barrier per pivot), its interchanges are applied to the
 * other columns on the host, U12 = L11^{-1} A12 is solved in device memory,
 * and the trailing matrix is updated with one out-of-core GEMM.  *info is 0, or j + 1
 * for the first exactly zero pivot (the factorisation still completes, as in
 * LAPACK).  The budget must hold one N x 64 panel.  opts->form: FP64 or Ozaki
 * for the out-of-core updates; same arena rule as ooc_dtrsm.  stats->tflops
 * counts 2 N^3 / 3 flops.
 */
int ooc_dgetrf(int64_t N, double* A, int64_t lda, int64_t* ipiv, size_t device_budget_bytes,
               const ooc_opts* opts, ooc_stats* stats, int64_t* info);

/* ---- sessions: one C over several calls (Section IV's nsteps) ------------ */
/*
 * Section IV gives the out-of-core DGEMM an nsteps parameter: it can be the
 * per-step update of SUMMA or hierarchical SUMMA, called once per main step
 * with that step's panels, all steps adding into one C (the paper keeps the
 * C blocks of its two C buffers on the device between calls).  A session does
 * this for an M x N C: it fixes the C blocking and keeps as many C blocks as
 * fit in HBM across the calls; the other blocks travel to the host and back in
 * every call.  On GB300 a 32 GiB C fits whole.
 *
 * ooc_session_create: C (pinned, M x N, ldc >= N) is the result matrix and the
 *   initial value; the final result is beta * C + sum of the calls' products.
 *   k_hint (0: 4096) is the largest inner dimension a call is planned for: the
 *   resident blocks are chosen so that a call of that K still streams its
 *   operands beside them (a call with a larger K streams it in chunks).  opts->form: FP64 or Ozaki;
 *   opts->workspace (holding the budget) makes the session allocate nothing.
 *   The session owns one arena of device_budget_bytes and three streams.
 * ooc_session_step: adds alpha * op(A) * op(B) (op(A) M x K, op(B) K x N,
 *   layouts as for ooc_dgemm) into the session's C; synchronous, A and B may
 *   be reused when it returns.  The first call also applies beta (beta == 0
 *   never reads C).  Until ooc_session_finish the host C holds partial sums
 *   for streamed blocks and stale values for resident ones, and must not be
 *   changed by the caller.
 * ooc_session_finish: writes the resident blocks back (after a call with
 *   K = 0 when no step was made, so C = beta * C) and destroys the session;
 *   stats (nullable): totals since creation, tflops over 2 M N sum(K).
 * ooc_session_free: destroys a session without writing anything back.
 * ooc_session_query: the blocking, how many of its blocks are resident, calls.
 */
typedef struct ooc_session ooc_session;
int ooc_session_create(int64_t M, int64_t N, int64_t k_hint, double beta, double* C, int64_t ldc,
                       size_t device_budget_bytes, const ooc_opts* opts, ooc_session** session);
int ooc_session_step(ooc_session* session, char transA, char transB, int64_t K, double alpha,
                     const double* A, int64_t lda, const double* B, int64_t ldb, ooc_stats* stats);
int ooc_session_finish(ooc_session* session, ooc_stats* stats);
int ooc_session_free(ooc_session* session);
int ooc_session_query(const ooc_session* session, int64_t* mb, int64_t* nb, int64_t* resident_blocks,
                      int64_t* blocks, int32_t* calls);

/*
 * Plan only (host, no device needed): the block/chunk/buffer plan the call
 * with these arguments would use.  elem_bytes is 8 for ooc_dgemm, 4 for
 * ooc_sgemm.  Fills stats' plan fields (mb, nb, kb, depth, c_buffers,
 * b_buffers, form, blocks, steps, device_bytes, h2d_bytes, d2h_bytes).
 * Section IV partitioner paragraph; worked example of Fig. 2.
 */
int ooc_plan(int64_t M, int64_t N, int64_t K, int32_t elem_bytes, int32_t beta_nonzero,
             size_t device_budget_bytes, const ooc_opts* opts, ooc_stats* plan);

/*
 * One operation of an issued pipeline schedule (host issue order), for
 * checking the Section IV buffer-hazard rule without a GPU.
 * kind: 0 H2D copy, 1 tile kernel, 2 D2H copy, 3 event record, 4 event wait,
 * 5 split (the split forms: the raw chunk in read_slot[0] into the bf16
 * planes of write_slot).
 * stream: 0 H2D stream, 1 compute stream, 2 D2H stream.
 * A tag names the datum in a device slot: {matrix (0 A, 1 B, 2 C),
 * row chunk, column chunk, version}; a C block's version counts the K-chunks
 * folded into it.  Unused slots are -1.  Plans of the split forms load A and B
 * into raw staging areas, used in turn, and split them from there into the
 * slots' planes: after the plan's S slots, ids S and S + 1 are A's areas and
 * S + 2 (and S + 3 when B is loaded in K chunks) B's.
 */
typedef struct {
    int32_t kind, stream, event, nreads;
    int32_t write_slot;
    int32_t read_slot[3];
    int64_t write_tag[4];
    int64_t read_tag[3][4];
} ooc_sched_op;

/*
 * Export the schedule ooc_dgemm (elem_bytes 8) or ooc_sgemm (4) would issue.
 * Writes at most capacity ops to out; *count receives the total.  Returns
 * OOC_ERR_CAPACITY (with *count set) when out is too small.
 */
int ooc_schedule(int64_t M, int64_t N, int64_t K, int32_t elem_bytes, int32_t beta_nonzero,
                 size_t device_budget_bytes, const ooc_opts* opts, ooc_sched_op* out,
                 int64_t capacity, int64_t* count);

/*
 * Export the schedule of ooc_dgemmt / ooc_dsyrk (elem_bytes 8) or ooc_ssyrk
 * (4) for an N x N C and inner dimension K, as ooc_schedule does; plan
 * (nullable) receives the plan fields as ooc_plan fills them, with blocks and
 * steps counting the updated blocks only.
 */
int ooc_schedule_gemmt(char uplo, int64_t N, int64_t K, int32_t elem_bytes, int32_t beta_nonzero,
                       size_t device_budget_bytes, const ooc_opts* opts, ooc_stats* plan,
                       ooc_sched_op* out, int64_t capacity, int64_t* count);

/*
 * Export the schedule of one session call (host only): FP64 operands, the
 * blocking forced by opts->mb / opts->nb, the first resident_blocks updated
 * blocks resident, call 0 (applies beta) or a later call (call > 0: resident
 * blocks start from their slot contents and are not copied back; streamed
 * blocks bring their partial sums from the host).  As ooc_schedule_gemmt.
 */
int ooc_schedule_session(int64_t M, int64_t N, int64_t K, int32_t beta_nonzero,
                         size_t device_budget_bytes, const ooc_opts* opts, int32_t resident_blocks,
                         int32_t call, ooc_stats* plan, ooc_sched_op* out, int64_t capacity,
                         int64_t* count);

/* ---- pipeline-description language (end of Section IV) ------------------ */
/*
 * Section IV closes by noting that the event synchronisation of its pipeline
 * is a pattern shared by out-of-core data-parallel kernels, and proposes a
 * pattern language from which a compiler writes that code.  A description
 * (text, one statement per line, '#' starts a comment):
 *
 *   operand NAME tile ROWS COLS ring SLOTS    host matrix cut into tiles; SLOTS device slots
 *   for VAR in LO .. HI   ...   end           loop (HI exclusive)
 *   load  NAME[ROW, COL]  [if VAR | unless VAR]   tile to the device (no copy when resident)
 *   alloc NAME[ROW, COL]  [if VAR | unless VAR]   slot for a tile written without being read
 *   run   KERNEL OUT[..] IN[..] ...               OUT is written, the rest are read
 *   store NAME[ROW, COL]  [if VAR | unless VAR]   tile back to the host
 *
 * Integer expressions: + - * / ( ), numbers, variables (ooc_pipe_set), loop
 * variables, trows(NAME) / tcols(NAME) = tile rows / columns of an operand.
 * Kernels (FP64 operands): gemm C A B -- C = alpha A B + beta C when C was
 * loaded, alpha A B when allocated, C + alpha A B when already written by an
 * earlier run; axpby Y X -- Y = a X + b Y (a X when Y was allocated); alpha,
 * beta, a, b are variables (defaults 1, 0, 1, 1).
 *
 * The compiler runs the loop nest on the host and emits copies and kernels
 * on an H2D, a compute and a D2H stream with exactly the events the Section IV
 * hazard rule requires (slots reused least recently used first).  A tile
 * written and never stored, a kernel on a tile that is not resident, tile
 * shapes a kernel cannot take, or an unknown name are errors
 * (OOC_ERR_INVALID_ARG; ooc_last_error() names the line).
 *
 * ooc_pipe_create parses; ooc_pipe_set sets a variable; ooc_pipe_bind gives
 * an operand its host matrix (row-major rows x cols, leading dimension ld,
 * elem_bytes 8 for the kernels; host may be NULL for ooc_pipe_schedule);
 * ooc_pipe_schedule compiles and exports the schedule (as ooc_schedule;
 * plan: device_bytes, bytes moved, steps = kernels, blocks = stores);
 * ooc_pipe_run compiles and executes synchronously in one arena of at most
 * device_budget_bytes (pinned host operands); ooc_pipe_free releases.
 */
typedef struct ooc_pipe ooc_pipe;
int ooc_pipe_create(const char* description, ooc_pipe** pipe);
int ooc_pipe_set(ooc_pipe* pipe, const char* name, double value);
int ooc_pipe_bind(ooc_pipe* pipe, const char* operand, void* host, int64_t rows, int64_t cols,
                  int64_t ld, int32_t elem_bytes);
int ooc_pipe_schedule(ooc_pipe* pipe, size_t device_budget_bytes, ooc_stats* plan, ooc_sched_op* out,
                      int64_t capacity, int64_t* count);
int ooc_pipe_run(ooc_pipe* pipe, size_t device_budget_bytes, ooc_stats* stats);
int ooc_pipe_free(ooc_pipe* pipe);

/* ---- plan search: candidates, autotuner, learned cost model ------------ */
/* The paper has no plan search beyond its partitioner (Section IV); these
 * calls pick block/chunk/ring sizes for this hardware. */
#define OOC_MLP_INPUTS 16
#define OOC_MLP_PARAMS 5313

/* One candidate plan and its cost-model features (see ooc_plan_candidates). */
typedef struct {
    int64_t mb, nb, kb;
    int32_t depth, b_buffers, c_buffers, reserved;
    double est_seconds;                 /* the planner's analytic estimate      */
    float features[OOC_MLP_INPUTS];     /* inputs of the cost model             */
} ooc_plan_candidate;

/*
 * The best `capacity` distinct plans for a problem by the planner's analytic
 * estimate (host only).  Problem arguments as in ooc_plan; opts->form picks
 * the form.  *count receives the number written.
 */
int ooc_plan_candidates(int64_t M, int64_t N, int64_t K, int32_t elem_bytes, int32_t beta_nonzero,
                        size_t device_budget_bytes, const ooc_opts* opts, ooc_plan_candidate* out,
                        int32_t capacity, int32_t* count);

/*
 * Exhaustive autotuner: run the problem once with each of the best
 * `max_candidates` candidate plans (after one untimed warm-up run) and report
 * each candidate's device time in seconds_out (same order as out).  The
 * problem's C is overwritten by every run, so tune on scratch operands of the
 * right shape.  elem_bytes 8 runs ooc_dgemm (desc pointers are double*),
 * 4 runs ooc_sgemm (desc pointers are float*); opts->form picks the form.
 */
int ooc_autotune(const ooc_gemm_desc* desc, int32_t elem_bytes, size_t device_budget_bytes,
                 const ooc_opts* opts, int32_t max_candidates, ooc_plan_candidate* out,
                 double* seconds_out, int32_t* count);

/*
 * Cost-model MLP (16 -> 64 -> 64 -> 1, ReLU), parameters packed W1[64][16],
 * b1[64], W2[64][64], b2[64], W3[64], b3 (OOC_MLP_PARAMS floats), all host
 * arrays, computed on the GPU.  Predicts log2(seconds) of a candidate.
 *   ooc_mlp_forward:   y[i] = f(X[i]) for n rows of OOC_MLP_INPUTS features
 *   ooc_mlp_loss_grad: loss = mean of 0.5 (f(X[i]) - t[i])^2 and its gradient
 *   ooc_mlp_train:     Adam (lr, betas 0.9/0.999, L2 weight decay added to the
 *                      gradient) over seeded shuffled mini-batches; params are
 *                      updated in place; final_loss (nullable) = loss of the
 *                      result over all samples
 *   ooc_costmodel_set: install params for OOC_PLAN_MODEL (NULL clears)
 */
int ooc_mlp_forward(const float* params, const float* X, int64_t n, float* y);
int ooc_mlp_loss_grad(const float* params, const float* X, const float* t, int64_t n, float* grad,
                      float* loss);
int ooc_mlp_train(float* params, const float* X, const float* t, int64_t n, int32_t epochs,
                  int32_t batch, float lr, float weight_decay, uint64_t seed, float* final_loss);
int ooc_costmodel_set(const float* params, int64_t n);

/*
 * hclGetMemSize analogue (Section III runtime methods): free device memory,
 * and host-link bandwidth in GB/s measured once per process with pinned
 * 256 MiB copies (H2D, D2H).  Any pointer may be NULL.
 */
int ooc_query_device(size_t* free_bytes, double* h2d_gbps, double* d2h_gbps);

/*
 * Measured FP64 peak of the current device in TFLOP/s: the paper quotes each
 * device's FP64 peak beside its DGEMM results (Section V); this measures it
 * with the instruction the FP64 tile kernel runs (mma.sync m8n8k4 f64, operands
 * in registers, so only the FP64 pipe bounds it), the best of repeated
 * launches over about `seconds` (0 < seconds <= 60; else OOC_ERR_INVALID_ARG).
 * Allocates and frees a small output buffer; synchronous.  OOC_ERR_NO_DEVICE
 * without an sm_103 device.
 */
int ooc_query_fp64_peak(double seconds, double* tflops);

/* Name of a status code (static string). */
const char* ooc_strerror(int code);

/* One-line detail of the last failure on the calling thread (static per thread). */
const char* ooc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* OOC_H */
