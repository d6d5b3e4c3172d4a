// Host planner and schedule generator of the out-of-core GEMM.
//
// Planner (Section IV, partitioner paragraph): A is cut into horizontal
// slices, B into vertical slices and C into blocks so that the buffers of the
// pipeline fit the device budget.  Two modes:
//   * paper mode reproduces the Section IV partitioner: h | M, w | N equal
//     slices, whole-K slices, buffers for two A slices, one B slice and two C
//     blocks (enough to update two C blocks of one block column), fewest
//     blocks first, then the smaller footprint, then the larger h (the worked
//     example's 4 x 2 split of Fig. 2);
//   * auto mode searches block rows/columns, an optional K chunk and the
//     buffer counts, scoring each candidate with a time estimate built from
//     the device's compute rate, tile-wave quantisation and the measured host
//     link, and keeps the fastest that fits.
//
// Schedule (Section IV, five pipeline stages and the event rule that device
// data is not overwritten until the kernels using it have completed): steps
// run column-major over C blocks (j outer, i inner, the B slice of a column
// stays resident as in Fig. 1's loop order), K chunks innermost.  Every load
// takes an empty slot, else the least recently used one; it waits on
// the event recorded after the slot's last reader, and records a ready event
// that the compute stream waits on.  H2D, compute and D2H each have a stream.
#include <algorithm>
#include <cstdlib>
#include <cmath>
#include <cstring>
#include <limits>
#include <string>
#include <vector>

#include "ooc_internal.hpp"

namespace ooc {

namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }
int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }
int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

struct FormModel {
    int64_t tile_m, tile_n;  // CTA tile of the contraction kernel
    double rate;             // sustained tile throughput, logical FLOP/s of the whole device
    int ctas_per_sm;
    int products;            // slice products per logical product
    int slices;
    double overlap_cost;     // share of the hidden copy time a step still loses (measured)
};

FormModel form_model(int form, int es, int64_t K, int slices_opt)
{
    FormModel f{};
    if (form == OOC_FORM_FP64) {
        f.tile_m = 64; f.tile_n = 64; f.rate = 1.0e12; f.ctas_per_sm = 3;
        f.products = 1; f.slices = 1;
        // no measurable cost: 32768^3 with 180 GB of copies (0.85 s at the link rate) ran 64.16 s
        // steps on 64.13 s of kernels
        f.overlap_cost = 0.0;
    } else if (form == OOC_FORM_BF16X3) {
        // measured bf16 rate of the tensor-core kernel on whole-K blocks (1.42-1.64 PFLOP/s)
        f.tile_m = 128; f.tile_n = 128; f.ctas_per_sm = 1;
        f.products = 6; f.slices = 3;
        f.rate = 1.4e15 / 6.0;
        // copies beside tensor-core kernels share HBM and the power budget: 65536^3 with 309 GB
        // H2D (1.46 s at the link rate) ran 2.84 s steps on 2.45 s of kernel-stream time
        f.overlap_cost = 0.27;
    } else {  // Ozaki (measured 1.39-1.40 PFLOP/s bf16)
        int s = slices_opt > 0 ? slices_opt : kOzakiSlicesGemm;
        f.tile_m = 128; f.tile_n = 128; f.ctas_per_sm = 1;
        f.slices = s; f.products = s * (s + 1) / 2;
        f.rate = 1.38e15 / f.products;
        f.overlap_cost = 0.27;
    }
    (void)es; (void)K;
    return f;
}

}  // namespace

int split_planes(const Plan& p) { return p.form == OOC_FORM_BF16X3 ? 3 : p.slices; }
int64_t split_rows_pad(int64_t rows) { return round_up(std::max<int64_t>(rows, 1), 128); }
int64_t split_k_pad(const Plan& p) { return round_up(p.kb, 64); }
size_t split_planes_bytes(const Plan& p, int64_t rows)
{
    return align_up((size_t)split_planes(p) * split_rows_pad(rows) * split_k_pad(p) * 2, kAlign);
}
size_t split_aux_bytes(const Plan& p, int64_t rows)
{
    size_t b = split_planes_bytes(p, rows);
    if (p.form == OOC_FORM_OZAKI)
        b += align_up((size_t)split_rows_pad(rows) * 4, kAlign) + align_up((size_t)split_rows_pad(rows) * 8, kAlign);
    return b;
}

namespace {

void layout(Plan& p, const FormModel& f)
{
    const int64_t ald = 16;  // 16 elements: 128-byte rows for FP64, 64 for FP32
    const int64_t a_rows = p.ta ? p.kb : p.mb, a_cols = p.ta ? p.mb : p.kb;
    const int64_t b_rows = p.tb ? p.nb : p.kb, b_cols = p.tb ? p.kb : p.nb;
    p.lda_dev = round_up(std::max<int64_t>(a_cols, 1), ald);
    p.ldb_dev = round_up(std::max<int64_t>(b_cols, 1), ald);
    p.ldc_dev = round_up(std::max<int64_t>(p.nb, 1), ald);
    p.a_slot = align_up((size_t)std::max<int64_t>(a_rows, 1) * p.lda_dev * p.es, kAlign);
    p.b_slot = align_up((size_t)std::max<int64_t>(b_rows, 1) * p.ldb_dev * p.es, kAlign);
    const int es_c = p.es;  // C slot holds the host element type
    p.c_slot = align_up((size_t)p.mb * p.ldc_dev * es_c, kAlign);
    p.a_aux = p.b_aux = p.c_aux = 0;
    if (p.form != OOC_FORM_FP64) {
        // bf16 planes [planes][rows_pad][k_pad], plus per-row exponent and max (Ozaki)
        p.a_aux = split_aux_bytes(p, p.mb);
        p.b_aux = split_aux_bytes(p, p.nb);
    }
    (void)f;
    // split forms keep raw staging areas (two for A; one for B when whole-K B slices are
    // loaded once per block column, else two) and planes per slot
    p.staged = p.form != OOC_FORM_FP64;
    p.nSA = p.staged ? 2 : 0;
    p.nSB = p.staged ? (p.nkc <= 1 ? 1 : 2) : 0;
    if (p.staged)
        p.device_bytes = p.header + (size_t)p.nSA * p.a_slot + (size_t)p.nA * p.a_aux + (size_t)p.nSB * p.b_slot +
                         (size_t)p.nB * p.b_aux + (size_t)(p.nC + p.nR) * (p.c_slot + p.c_aux);
    else
        p.device_bytes = p.header + (size_t)p.nA * (p.a_slot + p.a_aux) + (size_t)p.nB * (p.b_slot + p.b_aux) +
                         (size_t)(p.nC + p.nR) * (p.c_slot + p.c_aux);
}

// The updated blocks of block column j: block rows [lo, hi) are updated, of
// which those outside [in_lo, in_hi) straddle the edge of a triangular
// update.  For the lower part both ranges end at the last block row, for the
// upper part both start at row 0 (min and max of col - row over a block fall
// as i grows).
struct ColumnBlocks {
    int64_t lo, hi, in_lo, in_hi;
};

ColumnBlocks column_blocks(const Plan& p, int64_t j)
{
    if (!p.tri) return {0, p.h, 0, p.h};
    // first block row at which pred(i) holds (pred turns true once and stays true)
    auto first = [&](auto pred) {
        int64_t a = 0, b = p.h;
        while (a < b) {
            const int64_t m = (a + b) / 2;
            if (pred(m)) b = m;
            else a = m + 1;
        }
        return a;
    };
    if (p.tri == 1) {
        const int64_t lo = first([&](int64_t i) { return p.block_class(i, j) != 0; });
        const int64_t in = first([&](int64_t i) { return p.block_class(i, j) == 1; });
        return {lo, p.h, std::max(in, lo), p.h};
    }
    const int64_t hi = first([&](int64_t i) { return p.block_class(i, j) == 0; });
    const int64_t in = first([&](int64_t i) { return p.block_class(i, j) != 1; });
    return {0, hi, 0, std::min(in, hi)};
}

// rows of block rows [a, b)
int64_t rows_in(const Plan& p, int64_t a, int64_t b)
{
    if (b <= a) return 0;
    return b == p.h ? p.M - a * p.mb : (b - a) * p.mb;
}

int64_t active_blocks(const Plan& p)
{
    if (!p.tri) return p.h * p.w;
    int64_t n = 0;
    for (int64_t j = 0; j < p.w; ++j) {
        const ColumnBlocks cb = column_blocks(p, j);
        n += std::max<int64_t>(0, cb.hi - cb.lo);
    }
    return n;
}

// Closed-form traffic of the schedule for this plan.
void traffic(Plan& p)
{
    const double es = p.es;
    const double A = (double)p.M * p.K * es, B = (double)p.K * p.N * es, C = (double)p.M * p.N * es;
    if (!p.tri) {
        // A chunks are re-sent for every block column unless one column's worth stays resident
        double a_loads = (p.h == 1 && p.nkc <= p.nA) ? A : A * p.w;
        double b_loads = (p.nkc <= p.nB) ? B : B * p.h;
        if (p.K == 0) a_loads = b_loads = 0;
        // resident blocks of a session move only on the first call (beta != 0) and at its end
        const double streamed = 1.0 - (double)p.nR / (double)std::max<int64_t>(1, p.h * p.w);
        const bool later = p.session_step > 0;
        p.h2d_bytes = a_loads + b_loads + (later ? C * streamed : (p.beta_nz ? C : 0.0));
        p.d2h_bytes = C * streamed;
        return;
    }
    double a_loads = 0, b_loads = 0, c_in = 0, c_out = 0;
    for (int64_t j = 0; j < p.w; ++j) {
        const ColumnBlocks cb = column_blocks(p, j);
        if (cb.hi <= cb.lo) continue;
        const double cols = (double)p.cols_of(j);
        const double rows = (double)rows_in(p, cb.lo, cb.hi);
        const double straddle = rows - (double)rows_in(p, cb.in_lo, cb.in_hi);
        a_loads += rows * p.K * es;
        b_loads += (p.nkc <= p.nB ? 1.0 : (double)(cb.hi - cb.lo)) * p.K * cols * es;
        c_out += rows * cols * es;
        c_in += (p.beta_nz ? rows : straddle) * cols * es;
    }
    if (p.h == 1 && p.nkc <= p.nA) a_loads = std::min(a_loads, A);
    if (p.K == 0) a_loads = b_loads = 0;
    (void)B; (void)C;
    p.h2d_bytes = a_loads + b_loads + c_in;
    p.d2h_bytes = c_out;
}

// Host rows of one copy of `mat` are short and not contiguous.
bool narrow_rows(const Plan& p, int mat)
{
    int64_t width, full, ld;
    if (mat == kMatA) {
        width = p.ta ? p.mb : p.kb; full = p.ta ? p.M : p.K; ld = p.lda_host;
    } else if (mat == kMatB) {
        width = p.tb ? p.kb : p.nb; full = p.tb ? p.K : p.N; ld = p.ldb_host;
    } else {
        width = p.nb; full = p.N; ld = p.ldc_host;
    }
    const bool contiguous = width == full && (ld == 0 || ld == full);
    return !contiguous && width * p.es < 64 * 1024;
}

double estimate(const Plan& p, const FormModel& f, int sms, double h2d_gbps, double d2h_gbps)
{
    const double slots_total = (double)sms * f.ctas_per_sm;
    // compute: per step waves x per-tile time, summed over full / ragged blocks
    double t_comp = 0;
    const int64_t hf = p.M / p.mb, wf = p.N / p.nb;
    const int64_t mr = p.M - hf * p.mb, nr = p.N - wf * p.nb;
    struct Part { int64_t rows, cols, count; };
    Part parts[4] = {{p.mb, p.nb, hf * wf}, {mr, p.nb, (mr ? 1 : 0) * wf},
                     {p.mb, nr, hf * (nr ? 1 : 0)}, {mr, nr, (mr && nr) ? 1 : 0}};
    if (p.tri) {  // count only the updated blocks (straddling ones as whole blocks)
        for (auto& pt : parts) pt.count = 0;
        for (int64_t j = 0; j < p.w; ++j) {
            const ColumnBlocks cb = column_blocks(p, j);
            if (cb.hi <= cb.lo) continue;
            const bool rag_col = p.cols_of(j) != p.nb;
            const bool rag_row = cb.hi == p.h && mr != 0;
            const int64_t full_rows = cb.hi - cb.lo - (rag_row ? 1 : 0);
            parts[rag_col ? 2 : 0].count += full_rows;
            if (rag_row) parts[rag_col ? 3 : 1].count += 1;
        }
    }
    const double tile_time_per_k = 2.0 * f.tile_m * f.tile_n * slots_total / f.rate;
    for (auto& pt : parts) {
        if (pt.count == 0 || pt.rows == 0 || pt.cols == 0) continue;
        const double tiles = (double)cdiv(pt.rows, f.tile_m) * cdiv(pt.cols, f.tile_n);
        const double waves = std::ceil(tiles / slots_total);
        t_comp += pt.count * waves * tile_time_per_k * (double)p.K;
    }
    const double bw_h = h2d_gbps * 1e9, bw_d = d2h_gbps * 1e9;
    const double t_link = std::max({p.h2d_bytes / bw_h, p.d2h_bytes / bw_d,
                                    (p.h2d_bytes + p.d2h_bytes) / (0.85 * (bw_h + bw_d))});
    const double es = p.es;
    const double fill = ((double)p.mb * p.kb + (double)p.kb * p.nb * std::min<int64_t>(p.nkc, p.nB)) * es / bw_h;
    const double drain = (double)p.mb * p.nb * es / bw_d;
    double bubbles = 0;
    // one B slot: each column switch waits for the next slice, unless a staged plan streams it
    // into the staging area during the previous column (the B prefetch)
    const bool staged_prefetch = p.staged && p.b_prefetch && p.nkc == 1 && p.h >= 2;
    if (p.nB < 2 * p.nkc && p.nkc <= p.nB && !staged_prefetch) bubbles = (double)(p.w - 1) * p.K * p.nb * es / bw_h;
    const double steps = (double)active_blocks(p) * p.nkc;
    // Strided host copies with short rows (< 64 KiB) run far below the link
    // rate on this host link and were seen to slow down further as more host
    // memory is touched; charge them at a quarter of the link rate, outside
    // the overlap.
    double narrow = 0;
    const double A = (double)p.M * p.K * es, B = (double)p.K * p.N * es, C = (double)p.M * p.N * es;
    double a_loads = (p.h == 1 && p.nkc <= p.nA) ? A : A * p.w;
    double b_loads = (p.nkc <= p.nB) ? B : B * p.h;
    double c_moved = C * (p.beta_nz ? 2.0 : 1.0);
    if (p.tri) {  // the traffic model already counts the updated blocks only
        const double c_frac = p.d2h_bytes / std::max(C, 1.0);
        a_loads *= c_frac;
        b_loads *= c_frac;
        c_moved = p.d2h_bytes * (p.beta_nz ? 2.0 : 1.0);
    }
    if (narrow_rows(p, kMatA)) narrow += a_loads;
    if (narrow_rows(p, kMatB)) narrow += b_loads;
    if (narrow_rows(p, kMatC)) narrow += c_moved;
    return std::max(t_comp, t_link) + f.overlap_cost * std::min(t_comp, t_link) + fill + drain + bubbles +
           steps * 8e-6 + narrow / (0.25 * bw_h);
}

bool paper_plan(const PlanRequest& rq, Plan& best, std::string& why)
{
    const int64_t M = rq.M, N = rq.N, K = rq.K;
    const double mem = (double)rq.budget / rq.es;  // elements, as Section IV counts them
    bool found = false;
    int64_t bh = 0, bw = 0;
    double bkey0 = 0, bkey1 = 0;
    for (int64_t h = 1; h <= M; ++h) {
        if (M % h) continue;
        for (int64_t w = 1; w <= N; ++w) {
            if (N % w) continue;
            const double mb = (double)(M / h), nb = (double)(N / w);
            const double fp = 2 * mb * K + K * nb + 2 * mb * nb;
            if (fp > mem) continue;
            const double k0 = (double)h * w, k1 = fp;
            bool better = !found || k0 < bkey0 || (k0 == bkey0 && (k1 < bkey1 || (k1 == bkey1 && h > bh)));
            if (better) { found = true; bh = h; bw = w; bkey0 = k0; bkey1 = k1; }
        }
    }
    if (!found) {
        why = "no equal h x w split fits 2A + 1B + 2C in the budget";
        return false;
    }
    best.mb = M / bh; best.nb = N / bw; best.kb = std::max<int64_t>(K, 1);
    best.nA = 2; best.nB = 1; best.nC = 2;
    return true;
}

}  // namespace

static thread_local std::vector<Plan>* collect_ = nullptr;

int make_plan(const PlanRequest& rq, Plan& p, std::string& why)
{
    p = Plan{};
    p.M = rq.M; p.N = rq.N; p.K = rq.K; p.es = rq.es;
    p.beta_nz = rq.beta_nz; p.ta = rq.ta; p.tb = rq.tb;
    p.tri = rq.tri; p.tri_off = rq.tri_off;
    p.nR = rq.nR; p.session_step = rq.session_step;
    p.lda_host = rq.lda; p.ldb_host = rq.ldb; p.ldc_host = rq.ldc;
    // OOC_B_PREFETCH=0 issues each B slice at its column switch (the schedule without the prefetch)
    if (const char* e = std::getenv("OOC_B_PREFETCH")) p.b_prefetch = std::atoi(e) != 0;
    int form = rq.opts.form;
    if (form == OOC_FORM_AUTO) form = (rq.es == 8) ? OOC_FORM_FP64 : OOC_FORM_BF16X3;
    if (rq.es == 8 && form != OOC_FORM_FP64 && form != OOC_FORM_OZAKI) {
        why = "ooc_dgemm supports the FP64 and Ozaki forms";
        return OOC_ERR_INVALID_ARG;
    }
    if (rq.es == 4 && form != OOC_FORM_BF16X3) {
        why = "ooc_sgemm supports the BF16x3 form";
        return OOC_ERR_INVALID_ARG;
    }
    p.form = form;
    if (form == OOC_FORM_OZAKI && rq.opts.slices != 0 && (rq.opts.slices < 2 || rq.opts.slices > kOzakiMaxSlices)) {
        why = "opts->slices must be 0 or 2.." + std::to_string(kOzakiMaxSlices);
        return OOC_ERR_INVALID_ARG;
    }
    const FormModel f = form_model(form, rq.es, rq.K, rq.opts.slices);
    p.slices = f.slices; p.products = f.products;
    const int sms = device_sm_count();
    if (rq.M <= 0 || rq.N <= 0) {
        why = "empty problem";
        return OOC_ERR_INVALID_ARG;
    }

    if (rq.opts.flags & OOC_PLAN_PAPER) {
        if (!paper_plan(rq, p, why)) return OOC_ERR_BUDGET;
        p.paper = true;
        p.h = rq.M / p.mb; p.w = rq.N / p.nb; p.nkc = 1;
        layout(p, f);
        traffic(p);
        p.est_seconds = estimate(p, f, sms, rq.h2d_gbps, rq.d2h_gbps);
        return OOC_OK;
    }

    // candidate block sizes: equal splits rounded up to the kernel tile
    auto sizes = [](int64_t X, int64_t g, int64_t forced) {
        std::vector<int64_t> v;
        if (forced > 0) { v.push_back(std::min(forced, X)); return v; }
        for (int64_t parts = 1; parts <= 4096; parts = parts < 16 ? parts + 1 : parts * 5 / 4) {
            int64_t s = round_up(cdiv(X, parts), g);
            if (s > X) s = X;
            if (s < 1) continue;
            if (std::find(v.begin(), v.end(), s) == v.end()) v.push_back(s);
            if (s <= g) break;
        }
        // below one kernel tile, for very small budgets
        for (int64_t s = g / 2; s >= 8; s /= 2)
            if (s < X && std::find(v.begin(), v.end(), s) == v.end()) v.push_back(s);
        return v;
    };
    const std::vector<int64_t> mbs = sizes(rq.M, f.tile_m, rq.opts.mb);
    const std::vector<int64_t> nbs = sizes(rq.N, f.tile_n, rq.opts.nb);
    std::vector<int64_t> kbs, split_chunks;
    if (form != OOC_FORM_FP64) {
        // split forms: whole-K slices (measured fastest on GB300 whenever they fit), else up to 16 K
        // chunks (each chunk is split into digit planes on its own; BF16x3 rounds C to FP32 once
        // per chunk, so few chunks) -- tried only when no whole-K plan fits the budget
        if (rq.opts.kb > 0) kbs.push_back(std::min<int64_t>(rq.opts.kb, std::max<int64_t>(rq.K, 1)));
        else {
            kbs.push_back(std::max<int64_t>(rq.K, 1));
            for (int64_t c : {2, 4, 8, 16}) {
                const int64_t kb = round_up(cdiv(rq.K, c), 64);
                if (kb < rq.K && kb >= 256 && std::find(split_chunks.begin(), split_chunks.end(), kb) ==
                                                  split_chunks.end())
                    split_chunks.push_back(kb);
            }
        }
    } else if (rq.opts.kb > 0) kbs.push_back(std::min<int64_t>(rq.opts.kb, std::max<int64_t>(rq.K, 1)));
    else {
        kbs.push_back(std::max<int64_t>(rq.K, 1));
        for (int64_t c = 2; c <= 1024 && rq.K > 64; c = c < 8 ? c + 1 : c * 2) {
            int64_t kb = round_up(cdiv(rq.K, c), 64);
            if (kb >= rq.K) continue;
            if (std::find(kbs.begin(), kbs.end(), kb) == kbs.end()) kbs.push_back(kb);
            if (kb <= 64) break;
        }
        for (int64_t kb = 32; kb >= 16; kb /= 2)
            if (kb < rq.K) kbs.push_back(kb);
    }
    const std::vector<int> nAs = rq.opts.depth > 0 ? std::vector<int>{rq.opts.depth} : std::vector<int>{2, 3};
    const std::vector<int> nCs = rq.opts.c_buffers > 0 ? std::vector<int>{rq.opts.c_buffers} : std::vector<int>{2, 3};

    bool found = false;
    Plan best;
    double best_t = std::numeric_limits<double>::infinity();
    std::vector<Plan>* keep = collect_;  // candidate collection (plan_candidates)
    std::vector<Plan> tri_pool;          // triangular updates: candidates awaiting the exact estimate
    for (int pass = 0; pass < 2; ++pass) {
    if (pass == 1) {
        if (found || !tri_pool.empty() || split_chunks.empty()) break;
        kbs = split_chunks;  // no whole-K split plan fits: stream K in chunks
    }
    for (int64_t kb : kbs) {
        const int64_t nkc = rq.K == 0 ? 1 : cdiv(rq.K, kb);
        std::vector<int> nBs = {(int)std::min<int64_t>(2 * nkc, 1 << 20), (int)nkc};
        if (nkc > 2) nBs.push_back(2);
        if (rq.opts.b_buffers > 0) nBs = {rq.opts.b_buffers};
        for (int64_t mb : mbs)
            for (int64_t nb : nbs)
                for (int nA : nAs)
                    for (int nC : nCs)
                        for (int nB : nBs) {
                            Plan c = p;
                            c.mb = mb; c.nb = nb; c.kb = kb;
                            c.h = cdiv(rq.M, mb); c.w = cdiv(rq.N, nb); c.nkc = nkc;
                            c.nA = nA; c.nB = nB; c.nC = nC;
                            if (c.nR > c.h * c.w) continue;        // resident blocks need this blocking
                            if (c.nR == c.h * c.w) c.nC = 0;       // every block resident: no C ring
                            layout(c, f);
                            if (c.device_bytes > rq.budget) continue;
                            if (c.tri) {
                                // triangular updates: rank by the full-update estimate first (the exact
                                // one walks every block column); the best of these are re-ranked below
                                Plan full = c;
                                full.tri = 0;
                                traffic(full);
                                full.est_seconds = estimate(full, f, sms, rq.h2d_gbps, rq.d2h_gbps);
                                c.est_seconds = full.est_seconds;
                                tri_pool.push_back(c);
                                continue;
                            }
                            traffic(c);
                            c.est_seconds = estimate(c, f, sms, rq.h2d_gbps, rq.d2h_gbps);
                            if (keep) keep->push_back(c);
                            // prefer faster; near-ties go to fewer device bytes
                            if (!found || c.est_seconds < best_t * (1 - 1e-9) ||
                                (c.est_seconds <= best_t * (1 + 1e-9) && c.device_bytes < best.device_bytes)) {
                                best = c; best_t = c.est_seconds; found = true;
                            }
                        }
    }
    }
    if (!tri_pool.empty()) {
        const size_t top = std::min<size_t>(tri_pool.size(), 48);
        std::partial_sort(tri_pool.begin(), tri_pool.begin() + top, tri_pool.end(),
                          [](const Plan& a, const Plan& b) { return a.est_seconds < b.est_seconds; });
        for (size_t q = 0; q < top; ++q) {
            Plan c = tri_pool[q];
            traffic(c);
            c.est_seconds = estimate(c, f, sms, rq.h2d_gbps, rq.d2h_gbps);
            if (keep) keep->push_back(c);
            if (!found || c.est_seconds < best_t * (1 - 1e-9) ||
                (c.est_seconds <= best_t * (1 + 1e-9) && c.device_bytes < best.device_bytes)) {
                best = c; best_t = c.est_seconds; found = true;
            }
        }
    }
    if (!found) {
        why = "budget of " + std::to_string(rq.budget) + " bytes is below the smallest plan";
        return OOC_ERR_BUDGET;
    }
    p = best;
    if (!keep && (rq.opts.flags & OOC_PLAN_MODEL) && !rq.tri) {  // the model is trained on full updates
        std::vector<float> params;
        if (costmodel_get(params)) {
            std::vector<Plan> cands;
            std::string w2;
            if (plan_candidates(rq, 64, cands, w2) == OOC_OK && !cands.empty()) {
                std::vector<float> X(cands.size() * kMlpIn), y(cands.size());
                for (size_t i = 0; i < cands.size(); ++i) plan_features(cands[i], rq, &X[i * kMlpIn]);
                if (mlp_forward_host(params.data(), X.data(), (int64_t)cands.size(), y.data(), w2) == OOC_OK) {
                    size_t bi = 0;
                    for (size_t i = 1; i < cands.size(); ++i)
                        if (y[i] < y[bi]) bi = i;
                    p = cands[bi];
                }
            }
        }
    }
    return OOC_OK;
}

int plan_candidates(const PlanRequest& rq, int max_n, std::vector<Plan>& out, std::string& why)
{
    std::vector<Plan> all;
    collect_ = &all;
    Plan best;
    PlanRequest r2 = rq;
    r2.opts.flags &= ~OOC_PLAN_MODEL;
    const int rc = make_plan(r2, best, why);
    collect_ = nullptr;
    if (rc) return rc;
    std::stable_sort(all.begin(), all.end(), [](const Plan& a, const Plan& b) { return a.est_seconds < b.est_seconds; });
    out.clear();
    for (const Plan& c : all) {
        bool dup = false;
        for (const Plan& o : out)
            if (o.mb == c.mb && o.nb == c.nb && o.kb == c.kb && o.nA == c.nA && o.nB == c.nB && o.nC == c.nC) dup = true;
        if (!dup) out.push_back(c);
        if ((int)out.size() >= max_n) break;
    }
    if (out.empty()) out.push_back(best);
    return OOC_OK;
}

// Cost-model inputs: problem scale and form, the plan's block / chunk / ring
// sizes, and three quantities the analytic estimate models coarsely: the wave
// efficiency of a full block's tiles on the device, the share of operand
// copies that are narrow strided rows, and the estimate itself.
void plan_features(const Plan& p, const PlanRequest& rq, float* f)
{
    auto lg = [](double x) { return (float)std::log2(std::max(x, 1.0)); };
    const FormModel fm = form_model(p.form, p.es, p.K, p.slices);
    const double slots = (double)device_sm_count() * fm.ctas_per_sm;
    const double tiles = (double)cdiv(p.mb, fm.tile_m) * cdiv(p.nb, fm.tile_n);
    const double waves = std::ceil(tiles / slots);
    f[0] = lg((double)p.M) / 16; f[1] = lg((double)p.N) / 16; f[2] = lg((double)std::max<int64_t>(p.K, 1)) / 16;
    f[3] = p.form == OOC_FORM_FP64; f[4] = p.form == OOC_FORM_OZAKI; f[5] = p.form == OOC_FORM_BF16X3;
    f[6] = lg((double)rq.budget) / 40;
    f[7] = (float)(tiles / (waves * slots));
    f[8] = lg((double)p.mb) / 16; f[9] = lg((double)p.nb) / 16; f[10] = lg((double)p.kb) / 16;
    f[11] = p.nA / 3.0f; f[12] = lg((double)p.nB + 1) / 8;
    f[13] = (narrow_rows(p, kMatA) + narrow_rows(p, kMatB) + narrow_rows(p, kMatC)) / 3.0f;
    f[14] = lg((double)(p.h * p.w * p.nkc)) / 16;
    f[15] = (float)(std::log2(std::max(p.est_seconds, 1e-9)) / 10.0);
}

// Arena: header, resident C slots (sessions), the A ring, the B ring, the C
// ring.  Each A / B slot is its raw data then its split scratch; in a staged
// plan the ring is its raw staging areas then the slots' scratch (planes) only,
// and a slot's raw data is the first staging area (the schedule names the
// staging areas by their own ids).
namespace {
size_t ring_a_offset(const Plan& p) { return p.header + (size_t)p.nR * (p.c_slot + p.c_aux); }
size_t ring_b_offset(const Plan& p)
{
    return ring_a_offset(p) +
           (p.staged ? (size_t)p.nSA * p.a_slot + (size_t)p.nA * p.a_aux : (size_t)p.nA * (p.a_slot + p.a_aux));
}
size_t ring_c_offset(const Plan& p)
{
    return ring_b_offset(p) +
           (p.staged ? (size_t)p.nSB * p.b_slot + (size_t)p.nB * p.b_aux : (size_t)p.nB * (p.b_slot + p.b_aux));
}
}  // namespace

size_t slot_offset(const Plan& p, int32_t s)
{
    const int32_t ring = p.nA + p.nB + p.nC;
    if (s >= p.slots()) {  // staging areas: two per operand at most
        const int a = s - p.slots();
        return a < 2 ? ring_a_offset(p) + (size_t)a * p.a_slot : ring_b_offset(p) + (size_t)(a - 2) * p.b_slot;
    }
    if (s >= ring) return p.header + (size_t)(s - ring) * (p.c_slot + p.c_aux);  // resident C slots come first
    if (s < p.nA) return ring_a_offset(p) + (p.staged ? 0 : (size_t)s * (p.a_slot + p.a_aux));
    if (s < p.nA + p.nB) return ring_b_offset(p) + (p.staged ? 0 : (size_t)(s - p.nA) * (p.b_slot + p.b_aux));
    return ring_c_offset(p) + (size_t)(s - p.nA - p.nB) * (p.c_slot + p.c_aux);
}

size_t slot_aux_offset(const Plan& p, int32_t s)
{
    if (p.staged && s < p.nA) return ring_a_offset(p) + (size_t)p.nSA * p.a_slot + (size_t)s * p.a_aux;
    if (p.staged && s < p.nA + p.nB)
        return ring_b_offset(p) + (size_t)p.nSB * p.b_slot + (size_t)(s - p.nA) * p.b_aux;
    const size_t base = slot_offset(p, s);
    if (s < p.nA) return base + p.a_slot;
    if (s < p.nA + p.nB) return base + p.b_slot;
    return base + p.c_slot;
}

// ------------------------------------------------------------- schedule --
namespace {

struct Gen {
    const Plan& p;
    std::vector<Op>& ops;
    std::vector<Tag> content;
    std::vector<int64_t> last_use;
    std::vector<bool> read_since_load, compute_synced, d2h_pending;

    Gen(const Plan& plan, std::vector<Op>& o) : p(plan), ops(o)
    {
        const int S = p.slots();
        content.assign(S, Tag{});
        last_use.assign(S, -1);
        read_since_load.assign(S, false);
        compute_synced.assign(S, true);
        d2h_pending.assign(S, false);
        rec.assign(n_events(p), {0, 0});
    }

    int64_t step_index(int64_t i, int64_t j, int64_t kc) const { return (j * p.h + i) * p.nkc + kc; }

    // Stream-order bookkeeping: pos[s] counts copies/kernels issued on stream s;
    // rec[e] is (stream, position) of event e's latest record; synced[a][b]
    // is the last position of stream b that stream a is already ordered
    // after.  A wait that adds no ordering is not issued.
    int64_t pos[3] = {0, 0, 0};
    std::vector<std::pair<int, int64_t>> rec;
    int64_t synced[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};

    void push(const Op& o)
    {
        ops.push_back(o);
        if (o.kind == kH2D || o.kind == kKernel || o.kind == kD2H || o.kind == kSplit) ++pos[o.stream];  // work
    }
    void emit_wait(int stream, int ev)
    {
        const auto r = rec[ev];
        if (r.first == stream || synced[stream][r.first] >= r.second) return;
        Op o; o.kind = kWait; o.stream = stream; o.event = ev; push(o);
        synced[stream][r.first] = r.second;
    }
    void emit_record(int stream, int ev)
    {
        Op o; o.kind = kRecord; o.stream = stream; o.event = ev; push(o);
        rec[ev] = {stream, pos[stream]};
    }

    // Staged plans: what each staging area holds and whether it is still to be
    // split (a prefetched B slice waits there for its column); the areas of an
    // operand are used in turn.
    Tag stage_tag[4];
    bool stage_pending[4] = {false, false, false, false};
    int stage_next[2] = {0, 0};
    int pf_area = -1;

    int next_area(int mat)
    {
        const int n = mat == kMatA ? p.nSA : p.nSB;
        const int a = p.stage_slot(mat, stage_next[mat]);
        stage_next[mat] = (stage_next[mat] + 1) % n;
        return a;
    }

    int ensure(int mat, const Tag& tg, int64_t t, int lo, int n, int64_t i, int64_t j, int64_t kc)
    {
        for (int s = lo; s < lo + n; ++s)
            if (content[s] == tg) { last_use[s] = t; return s; }
        // victim: an empty slot, else the least recently used one.  LRU keeps
        // the victim's last reader as old as possible, so the load overlaps the
        // kernels in between; cyclic reuse longer than the ring is reloaded,
        // which is what the planner's traffic model counts.
        int victim = -1;
        for (int s = lo; s < lo + n; ++s)
            if (content[s].m < 0) { victim = s; break; }
        if (victim < 0) {
            victim = lo;
            for (int s = lo + 1; s < lo + n; ++s)
                if (last_use[s] < last_use[victim]) victim = s;
        }
        if (p.staged) {
            // the raw data goes to a staging area once the area's previous content is split;
            // the split writes the victim's planes on the compute stream, after the victim's
            // earlier readers there
            int area = -1;
            for (int k = 0; k < (mat == kMatA ? p.nSA : p.nSB); ++k) {
                const int a = p.stage_slot(mat, k);
                if (stage_pending[a - p.slots()] && stage_tag[a - p.slots()] == tg) area = a;
            }
            if (area < 0) {
                area = next_area(mat);
                emit_wait(kStreamH2D, ev_staged(p, area));
                Op o; o.kind = kH2D; o.stream = kStreamH2D; o.wslot = area; o.wtag = tg;
                o.i = i; o.j = j; o.kc = kc;
                push(o);
                emit_record(kStreamH2D, ev_sready(p, area));
                stage_tag[area - p.slots()] = tg;
                stage_pending[area - p.slots()] = true;
            }
            emit_wait(kStreamCompute, ev_sready(p, area));
            Op sp; sp.kind = kSplit; sp.stream = kStreamCompute; sp.nr = 1;
            sp.rslot[0] = area; sp.rtag[0] = tg;
            sp.wslot = victim; sp.wtag = tg;
            sp.i = i; sp.j = j; sp.kc = kc;
            push(sp);
            emit_record(kStreamCompute, ev_staged(p, area));
            stage_pending[area - p.slots()] = false;
            content[victim] = tg;
            last_use[victim] = t;
            read_since_load[victim] = false;
            compute_synced[victim] = true;
            return victim;
        }
        if (read_since_load[victim]) emit_wait(kStreamH2D, ev_free(p, victim));
        Op o; o.kind = kH2D; o.stream = kStreamH2D; o.wslot = victim; o.wtag = tg;
        o.i = i; o.j = j; o.kc = kc;
        (void)mat;
        push(o);
        emit_record(kStreamH2D, ev_ready(p, victim));
        content[victim] = tg;
        last_use[victim] = t;
        read_since_load[victim] = false;
        compute_synced[victim] = false;
        return victim;
    }

    // Piece `part` of the next column's whole-K B slice (B prefetch): the first
    // piece takes the least recently used B slot, after its last readers.
    int pf_slot = -1;
    void prefetch_piece(const Tag& tg, int part, int nparts, int64_t t, int64_t jn)
    {
        if (p.staged) {  // into a staging area, once the slice it last held has been split
            if (part == 0) {
                pf_area = next_area(kMatB);
                emit_wait(kStreamH2D, ev_staged(p, pf_area));
            }
            Op o; o.kind = kH2D; o.stream = kStreamH2D; o.wslot = pf_area; o.wtag = tg;
            o.i = 0; o.j = jn; o.kc = 0; o.part = part; o.nparts = nparts;
            push(o);
            emit_record(kStreamH2D, ev_sready(p, pf_area));
            stage_tag[pf_area - p.slots()] = tg;
            stage_pending[pf_area - p.slots()] = true;
            return;
        }
        const int lo = p.nA, n = p.nB;
        if (part == 0) {
            int victim = -1;
            for (int s = lo; s < lo + n; ++s)
                if (content[s].m < 0) { victim = s; break; }
            if (victim < 0) {
                victim = lo;
                for (int s = lo + 1; s < lo + n; ++s)
                    if (last_use[s] < last_use[victim]) victim = s;
            }
            if (read_since_load[victim]) emit_wait(kStreamH2D, ev_free(p, victim));
            pf_slot = victim;
            content[victim] = tg;
            last_use[victim] = t;
            read_since_load[victim] = false;
            compute_synced[victim] = false;
        }
        Op o; o.kind = kH2D; o.stream = kStreamH2D; o.wslot = pf_slot; o.wtag = tg;
        o.i = 0; o.j = jn; o.kc = 0; o.part = part; o.nparts = nparts;
        push(o);
        emit_record(kStreamH2D, ev_ready(p, pf_slot));
    }

    int64_t updated_blocks(int64_t j) const
    {
        int64_t n = 0;
        for (int64_t i = 0; i < p.h; ++i) n += p.block_class(i, j) != 0;
        return n;
    }

    void run()
    {
        const int a0 = 0, b0 = p.nA, c0 = p.nA + p.nB;
        const bool have_k = p.K > 0;
        int64_t nblk = 0;  // blocks issued so far: C blocks take the C slots in turn
        constexpr int kMaxPieces = 8;
        for (int64_t j = 0; j < p.w; ++j) {
            // B prefetch: with whole-K B slices and a spare B slot, the next column's slice is
            // copied in row ranges after the A loads of this column's 2nd, 3rd, ... updated blocks,
            // so the column switch finds it resident instead of waiting for the whole slice
            const int64_t ublk = updated_blocks(j);
            const int npieces = (p.b_prefetch && have_k && p.nkc == 1 && (p.nB >= 2 || p.staged) && j + 1 < p.w &&
                                 ublk >= 2 &&
                                 updated_blocks(j + 1) > 0)
                                    ? (int)std::min<int64_t>(kMaxPieces, ublk - 1)
                                    : 0;
            int64_t u = 0;  // updated blocks of this column so far
            for (int64_t i = 0; i < p.h; ++i) {
                const int cls = p.block_class(i, j);
                if (cls == 0) continue;  // no element of this block is updated
                // session: the first nR blocks keep their own slot across the session's calls
                const bool resident = nblk < p.nR;
                const int sc = resident ? c0 + p.nC + (int)nblk : c0 + (int)((nblk - p.nR) % p.nC);
                ++nblk;
                // a later session call adds onto partial sums: a resident block's are in its slot,
                // a streamed block's come back from the host.  A block straddling a triangular
                // update's edge goes back whole, so it is loaded even for beta == 0.
                const bool later = p.session_step > 0;
                const bool load_c = later ? !resident : (p.beta_nz || cls == 2);
                for (int64_t kc = 0; kc < p.nkc; ++kc) {
                    const int64_t t = step_index(i, j, kc);
                    int sa = -1, sb = -1;
                    if (have_k) {
                        sa = ensure(kMatA, Tag{kMatA, i, kc, 0}, t, a0, p.nA, i, j, kc);
                        sb = ensure(kMatB, Tag{kMatB, kc, j, 0}, t, b0, p.nB, i, j, kc);
                        if (u >= 1 && u <= npieces) prefetch_piece(Tag{kMatB, 0, j + 1, 0}, (int)(u - 1), npieces, t, j + 1);
                    }
                    if (kc == 0) {
                        const Tag ct{kMatC, i, j, 0};
                        if (load_c) {
                            if (d2h_pending[sc]) emit_wait(kStreamH2D, ev_out(p, sc));
                            Op o; o.kind = kH2D; o.stream = kStreamH2D; o.wslot = sc; o.wtag = ct;
                            o.i = i; o.j = j; o.kc = 0;
                            push(o);
                            emit_record(kStreamH2D, ev_ready(p, sc));
                            compute_synced[sc] = false;
                        } else if (d2h_pending[sc]) {
                            emit_wait(kStreamCompute, ev_out(p, sc));
                        }
                        d2h_pending[sc] = false;
                        content[sc] = ct;
                    }
                    // wait for the inputs' loads, latest-issued first (it covers the earlier ones)
                    std::vector<int> need;
                    for (int s : {sa, sb, sc})
                        if (s >= 0 && !compute_synced[s]) need.push_back(s);
                    std::sort(need.begin(), need.end(), [&](int x, int y) {
                        return rec[ev_ready(p, x)].second > rec[ev_ready(p, y)].second;
                    });
                    for (int s : need) {
                        emit_wait(kStreamCompute, ev_ready(p, s));
                        compute_synced[s] = true;
                    }
                    Op k; k.kind = kKernel; k.stream = kStreamCompute;
                    k.i = i; k.j = j; k.kc = kc;
                    k.first = (kc == 0) && !later; k.last = (kc == p.nkc - 1);
                    if (sa >= 0) { k.rslot[k.nr] = sa; k.rtag[k.nr] = content[sa]; ++k.nr; }
                    if (sb >= 0) { k.rslot[k.nr] = sb; k.rtag[k.nr] = content[sb]; ++k.nr; }
                    if (kc > 0 || load_c || later) { k.rslot[k.nr] = sc; k.rtag[k.nr] = content[sc]; ++k.nr; }
                    k.wslot = sc;
                    k.wtag = Tag{kMatC, i, j, kc + 1};
                    push(k);
                    content[sc] = k.wtag;
                    for (int s : {sa, sb}) {
                        if (s < 0 || p.staged) continue;  // staged slots are rewritten on this stream only
                        read_since_load[s] = true;
                        emit_record(kStreamCompute, ev_free(p, s));
                    }
                    if (kc == p.nkc - 1 && !resident) {
                        emit_record(kStreamCompute, ev_done(p, sc));
                        emit_wait(kStreamD2H, ev_done(p, sc));
                        Op d; d.kind = kD2H; d.stream = kStreamD2H; d.nr = 1;
                        d.rslot[0] = sc; d.rtag[0] = content[sc];
                        d.i = i; d.j = j; d.kc = kc;
                        push(d);
                        emit_record(kStreamD2H, ev_out(p, sc));
                        d2h_pending[sc] = true;
                    }
                }
                ++u;
            }
        }
    }
};

}  // namespace

void build_schedule(const Plan& plan, std::vector<Op>& ops)
{
    ops.clear();
    ops.reserve((size_t)(plan.h * plan.w * plan.nkc * 12 + 16));
    Gen g(plan, ops);
    g.run();
}

}  // namespace ooc
