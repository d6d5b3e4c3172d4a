// Pipeline-description language: the end of Section IV observes that the
// event synchronisation of its out-of-core DGEMM follows a pattern common to
// out-of-core data-parallel kernels, and proposes a pattern language in which
// a programmer states the software pipeline and a compiler writes the
// synchronisation code.  This file is that compiler (the executor is
// pipe_exec.cu).
//
// A description names operands (matrices in host memory cut into tiles, each
// with a ring of device slots) and a loop nest of four statements:
//
//   operand NAME tile ROWS COLS ring SLOTS
//   for VAR in LO .. HI          (HI exclusive)       ...  end
//   load  NAME[ROW, COL]   bring a tile into a slot of NAME's ring (no copy when resident)
//   alloc NAME[ROW, COL]   claim a slot for a tile a kernel will write without reading
//   run   KERNEL OUT[..] IN[..] ...   OUT is written, the inputs are read
//   store NAME[ROW, COL]   copy a tile back to the host
//
// load, alloc and store take an optional "if VAR" / "unless VAR".  Integer
// expressions use + - * / ( ), variables set by the host, loop variables and
// trows(NAME) / tcols(NAME) (tile rows / columns of an operand).  Kernels:
//   gemm  C A B   C = alpha A B + beta C (C loaded), alpha A B (C allocated),
//                 C + alpha A B (C already written by an earlier run)
//   axpby Y X     Y = a X + b Y (Y loaded or written), a X (Y allocated)
// with alpha, beta, a, b host variables (FP64 operands).
//
// Compilation executes the loop nest on the host and emits the copies and
// kernel launches of three streams (H2D, compute, D2H) with the events the
// Section IV hazard rule needs, and no others: a slot is refilled only after
// the kernels that read it and the copy that stored it have finished, a
// kernel starts after its tiles arrived, a store after the kernel that wrote
// the tile.  Slots are reused least-recently-used first.  A tile written and
// not stored is never evicted (that is a compile error), and so is a kernel
// whose tile is not resident (a ring too small for one step).
#include <cctype>
#include <cmath>
#include <functional>
#include <map>
#include <memory>
#include <sstream>

#include "ooc_internal.hpp"

namespace ooc {

namespace {

// ------------------------------------------------------------- parsing --
struct Expr {
    // a tiny expression tree: number, variable, tile count, or binary op
    enum Kind { Num, Var, TRows, TCols, Bin } kind = Num;
    int64_t num = 0;
    std::string name;
    char op = 0;
    std::shared_ptr<Expr> a, b;
};

struct TileRef {
    std::string operand;
    std::shared_ptr<Expr> r, c;
};

struct Stmt {
    enum Kind { Operand, For, Load, Alloc, Store, Run } kind = Load;
    int line = 0;
    std::string name;                   // operand / loop variable / kernel
    std::shared_ptr<Expr> e0, e1, e2;   // operand tile sizes and ring / loop bounds
    std::vector<TileRef> tiles;         // load/alloc/store: one; run: output then inputs
    std::string cond;                   // if / unless variable
    bool negate = false;
    std::vector<Stmt> body;             // for
};

struct Lexer {
    std::string s;
    size_t p = 0;
    explicit Lexer(const std::string& line) : s(line) {}
    void ws()
    {
        while (p < s.size() && std::isspace((unsigned char)s[p])) ++p;
    }
    bool end()
    {
        ws();
        return p >= s.size();
    }
    bool eat(const std::string& t)
    {
        ws();
        if (s.compare(p, t.size(), t) == 0) {
            p += t.size();
            return true;
        }
        return false;
    }
    std::string ident()
    {
        ws();
        size_t q = p;
        while (q < s.size() && (std::isalnum((unsigned char)s[q]) || s[q] == '_')) ++q;
        std::string r = s.substr(p, q - p);
        p = q;
        return r;
    }
    bool peek_ident() { ws(); return p < s.size() && (std::isalpha((unsigned char)s[p]) || s[p] == '_'); }
};

struct ParseError {
    std::string msg;
};

std::shared_ptr<Expr> parse_expr(Lexer& L);

std::shared_ptr<Expr> parse_atom(Lexer& L)
{
    L.ws();
    auto e = std::make_shared<Expr>();
    if (L.eat("(")) {
        e = parse_expr(L);
        if (!L.eat(")")) throw ParseError{"expected ')'"};
        return e;
    }
    if (L.p < L.s.size() && std::isdigit((unsigned char)L.s[L.p])) {
        size_t q = L.p;
        while (q < L.s.size() && std::isdigit((unsigned char)L.s[q])) ++q;
        e->kind = Expr::Num;
        e->num = std::stoll(L.s.substr(L.p, q - L.p));
        L.p = q;
        return e;
    }
    if (!L.peek_ident()) throw ParseError{"expected a number, a variable or '('"};
    const std::string id = L.ident();
    if ((id == "trows" || id == "tcols") && L.eat("(")) {
        e->kind = id == "trows" ? Expr::TRows : Expr::TCols;
        e->name = L.ident();
        if (e->name.empty() || !L.eat(")")) throw ParseError{"expected " + id + "(OPERAND)"};
        return e;
    }
    e->kind = Expr::Var;
    e->name = id;
    return e;
}

std::shared_ptr<Expr> parse_term(Lexer& L)
{
    auto a = parse_atom(L);
    for (;;) {
        L.ws();
        char op = 0;
        if (L.eat("*")) op = '*';
        else if (L.eat("/")) op = '/';
        else return a;
        auto e = std::make_shared<Expr>();
        e->kind = Expr::Bin; e->op = op; e->a = a; e->b = parse_atom(L);
        a = e;
    }
}

std::shared_ptr<Expr> parse_expr(Lexer& L)
{
    auto a = parse_term(L);
    for (;;) {
        L.ws();
        char op = 0;
        if (L.s.compare(L.p, 2, "..") == 0) return a;  // range separator, not an operator
        if (L.eat("+")) op = '+';
        else if (L.eat("-")) op = '-';
        else return a;
        auto e = std::make_shared<Expr>();
        e->kind = Expr::Bin; e->op = op; e->a = a; e->b = parse_term(L);
        a = e;
    }
}

TileRef parse_tile(Lexer& L)
{
    TileRef t;
    t.operand = L.ident();
    if (t.operand.empty() || !L.eat("[")) throw ParseError{"expected OPERAND[ROW, COL]"};
    t.r = parse_expr(L);
    if (!L.eat(",")) throw ParseError{"expected ',' between tile indices"};
    t.c = parse_expr(L);
    if (!L.eat("]")) throw ParseError{"expected ']'"};
    return t;
}

void parse_cond(Lexer& L, Stmt& st)
{
    if (L.end()) return;
    if (L.eat("if")) st.negate = false;
    else if (L.eat("unless")) st.negate = true;
    else throw ParseError{"unexpected text after the statement"};
    st.cond = L.ident();
    if (st.cond.empty()) throw ParseError{"expected a variable after if / unless"};
}

// Parse lines [i, end) into `out` until an "end" line (nested) or the end of input.
void parse_block(const std::vector<std::string>& lines, size_t& i, std::vector<Stmt>& out, bool nested)
{
    while (i < lines.size()) {
        std::string text = lines[i];
        const size_t hash = text.find('#');
        if (hash != std::string::npos) text = text.substr(0, hash);
        Lexer L(text);
        const int line = (int)i + 1;
        ++i;
        if (L.end()) continue;
        try {
            const std::string kw = L.ident();
            Stmt st;
            st.line = line;
            if (kw == "end") {
                if (!L.end()) throw ParseError{"unexpected text after end"};
                if (!nested) throw ParseError{"'end' without 'for'"};
                return;
            } else if (kw == "operand") {
                st.kind = Stmt::Operand;
                st.name = L.ident();
                if (st.name.empty() || !L.eat("tile")) throw ParseError{"expected: operand NAME tile ROWS COLS ring N"};
                st.e0 = parse_expr(L);
                st.e1 = parse_expr(L);
                if (!L.eat("ring")) throw ParseError{"expected 'ring'"};
                st.e2 = parse_expr(L);
                if (!L.end()) throw ParseError{"unexpected text after the ring size"};
            } else if (kw == "for") {
                st.kind = Stmt::For;
                st.name = L.ident();
                if (st.name.empty() || !L.eat("in")) throw ParseError{"expected: for VAR in LO .. HI"};
                st.e0 = parse_expr(L);
                if (!L.eat("..")) throw ParseError{"expected '..'"};
                st.e1 = parse_expr(L);
                if (!L.end()) throw ParseError{"unexpected text after the loop range"};
                parse_block(lines, i, st.body, true);
            } else if (kw == "load" || kw == "alloc" || kw == "store") {
                st.kind = kw == "load" ? Stmt::Load : kw == "alloc" ? Stmt::Alloc : Stmt::Store;
                st.tiles.push_back(parse_tile(L));
                parse_cond(L, st);
            } else if (kw == "run") {
                st.kind = Stmt::Run;
                st.name = L.ident();
                if (st.name.empty()) throw ParseError{"expected a kernel name"};
                while (!L.end()) st.tiles.push_back(parse_tile(L));
                if (st.tiles.empty()) throw ParseError{"run needs an output tile"};
            } else {
                throw ParseError{"unknown statement '" + kw + "'"};
            }
            out.push_back(std::move(st));
        } catch (const ParseError& e) {
            if (e.msg.rfind("line ", 0) == 0) throw;  // from a nested block: already located
            throw ParseError{"line " + std::to_string(line) + ": " + e.msg};
        }
    }
    if (nested) throw ParseError{"'for' without 'end'"};
}

// ----------------------------------------------------------- compiling --
struct SlotState {
    Tag content;
    bool fresh = false;          // claimed by alloc, no data yet
    bool dirty = false;          // written by a kernel since the last store
    bool read_since_fill = false;
    bool compute_synced = true;
    bool d2h_pending = false;
    int64_t last_use = -1;
};

struct Compiler {
    PipeProgram& prog;
    const std::map<std::string, double>& vars;
    std::map<std::string, int64_t> env;   // loop variables
    std::vector<SlotState> slot;
    int64_t clock = 0;
    // Stream order bookkeeping: pos[s] counts the copies / kernels issued on
    // stream s; synced[a] is a vector clock -- synced[a][b] is the last
    // position of stream b that stream a is already ordered after, directly
    // or through other streams; rec[e] is the clock of event e's latest
    // record.  A wait that adds no ordering is not issued.
    struct Clock {
        int stream = -1;
        int64_t vc[3] = {0, 0, 0};
    };
    int64_t pos[3] = {0, 0, 0};
    std::vector<Clock> rec;
    int64_t synced[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};

    Compiler(PipeProgram& p, const std::map<std::string, double>& v) : prog(p), vars(v) {}

    int ev_ready(int s) const { return s; }
    int ev_free(int s) const { return prog.slots + s; }
    int ev_out(int s) const { return 2 * prog.slots + s; }
    int ev_done(int s) const { return 3 * prog.slots + s; }

    void push(const Op& o)
    {
        prog.ops.push_back(o);
        if (o.kind == kH2D || o.kind == kKernel || o.kind == kD2H) ++pos[o.stream];
    }
    void wait(int stream, int ev)
    {
        const Clock& r = rec[ev];
        if (r.stream < 0) return;  // never recorded: nothing to wait for
        if (r.stream == stream || synced[stream][r.stream] >= r.vc[r.stream]) return;
        Op o; o.kind = kWait; o.stream = stream; o.event = ev;
        push(o);
        for (int x = 0; x < 3; ++x) synced[stream][x] = std::max(synced[stream][x], r.vc[x]);
    }
    void record(int stream, int ev)
    {
        Op o; o.kind = kRecord; o.stream = stream; o.event = ev;
        push(o);
        Clock c;
        c.stream = stream;
        for (int x = 0; x < 3; ++x) c.vc[x] = synced[stream][x];
        c.vc[stream] = pos[stream];
        rec[ev] = c;
    }

    int op_index(const std::string& name, int line) const
    {
        for (size_t i = 0; i < prog.operands.size(); ++i)
            if (prog.operands[i].name == name) return (int)i;
        throw ParseError{"line " + std::to_string(line) + ": unknown operand '" + name + "'"};
    }

    int64_t eval(const Expr& e, int line) const
    {
        switch (e.kind) {
        case Expr::Num: return e.num;
        case Expr::Var: {
            auto it = env.find(e.name);
            if (it != env.end()) return it->second;
            auto jt = vars.find(e.name);
            if (jt != vars.end()) return (int64_t)std::llround(jt->second);
            throw ParseError{"line " + std::to_string(line) + ": unknown variable '" + e.name + "'"};
        }
        case Expr::TRows:
        case Expr::TCols: {
            const PipeOperand& o = prog.operands[op_index(e.name, line)];
            if (o.tr <= 0 || o.tc <= 0) throw ParseError{"line " + std::to_string(line) + ": operand not ready"};
            return e.kind == Expr::TRows ? (o.rows + o.tr - 1) / o.tr : (o.cols + o.tc - 1) / o.tc;
        }
        case Expr::Bin: {
            const int64_t a = eval(*e.a, line), b = eval(*e.b, line);
            switch (e.op) {
            case '+': return a + b;
            case '-': return a - b;
            case '*': return a * b;
            default:
                if (b == 0) throw ParseError{"line " + std::to_string(line) + ": division by zero"};
                return a / b;
            }
        }
        }
        return 0;
    }

    bool cond_true(const Stmt& st) const
    {
        if (st.cond.empty()) return true;
        auto it = vars.find(st.cond);
        const bool v = it != vars.end() && it->second != 0.0;
        return st.negate ? !v : v;
    }

    struct Ref {
        int op;
        int64_t r, c;
    };
    Ref tile(const TileRef& t, int line)
    {
        Ref x{op_index(t.operand, line), eval(*t.r, line), eval(*t.c, line)};
        const PipeOperand& o = prog.operands[x.op];
        const int64_t nr = (o.rows + o.tr - 1) / o.tr, nc = (o.cols + o.tc - 1) / o.tc;
        if (x.r < 0 || x.c < 0 || x.r >= nr || x.c >= nc)
            throw ParseError{"line " + std::to_string(line) + ": tile " + t.operand + "[" + std::to_string(x.r) +
                             ", " + std::to_string(x.c) + "] is outside the operand"};
        return x;
    }

    int find(const Ref& x) const
    {
        const PipeOperand& o = prog.operands[x.op];
        for (int s = o.slot0; s < o.slot0 + o.ring; ++s)
            if (slot[s].content.m == x.op && slot[s].content.r == x.r && slot[s].content.c == x.c) return s;
        return -1;
    }

    int victim(const Ref& x, int line)
    {
        const PipeOperand& o = prog.operands[x.op];
        int v = -1;
        for (int s = o.slot0; s < o.slot0 + o.ring; ++s)
            if (slot[s].content.m < 0) return s;
        for (int s = o.slot0; s < o.slot0 + o.ring; ++s)
            if (v < 0 || slot[s].last_use < slot[v].last_use) v = s;
        if (slot[v].dirty)
            throw ParseError{"line " + std::to_string(line) + ": the ring of " + o.name +
                             " is full and would evict a tile written but not stored"};
        return v;
    }

    void do_load(const Stmt& st, bool alloc)
    {
        const Ref x = tile(st.tiles[0], st.line);
        int s = find(x);
        if (s >= 0) {
            slot[s].last_use = clock;
            return;
        }
        s = victim(x, st.line);
        SlotState& S = slot[s];
        const Tag tg{x.op, x.r, x.c, 0};
        if (!alloc) {
            if (S.read_since_fill) wait(kStreamH2D, ev_free(s));
            if (S.d2h_pending) wait(kStreamH2D, ev_out(s));
            Op o; o.kind = kH2D; o.stream = kStreamH2D; o.wslot = s; o.wtag = tg;
            push(o);
            record(kStreamH2D, ev_ready(s));
            S.compute_synced = false;
        } else {
            // the next writer is a kernel on the compute stream
            if (S.read_since_fill) wait(kStreamCompute, ev_free(s));
            if (S.d2h_pending) wait(kStreamCompute, ev_out(s));
            S.compute_synced = true;
        }
        S.content = tg;
        S.fresh = alloc;
        S.dirty = false;
        S.read_since_fill = false;
        S.d2h_pending = false;
        S.last_use = clock;
    }

    void do_run(const Stmt& st)
    {
        int kernel;
        if (st.name == "gemm") kernel = kPipeGemm;
        else if (st.name == "axpby") kernel = kPipeAxpby;
        else throw ParseError{"line " + std::to_string(st.line) + ": unknown kernel '" + st.name + "'"};
        const size_t want = kernel == kPipeGemm ? 3 : 2;
        if (st.tiles.size() != want)
            throw ParseError{"line " + std::to_string(st.line) + ": " + st.name + " takes " + std::to_string(want) +
                             " tiles"};
        std::vector<Ref> t;
        std::vector<int> sl;
        for (const TileRef& tr : st.tiles) {
            t.push_back(tile(tr, st.line));
            const int s = find(t.back());
            if (s < 0)
                throw ParseError{"line " + std::to_string(st.line) + ": tile " + tr.operand +
                                 " is not resident (load or alloc it first; is its ring large enough?)"};
            sl.push_back(s);
        }
        for (size_t a = 0; a < sl.size(); ++a)
            for (size_t b = a + 1; b < sl.size(); ++b)
                if (sl[a] == sl[b])
                    throw ParseError{"line " + std::to_string(st.line) + ": a tile is both read and written"};
        // shapes
        auto dims = [&](const Ref& x) {
            const PipeOperand& o = prog.operands[x.op];
            return std::make_pair(o.tile_rows(x.r), o.tile_cols(x.c));
        };
        const auto d0 = dims(t[0]), d1 = dims(t[1]);
        if (kernel == kPipeGemm) {
            const auto d2 = dims(t[2]);
            if (d1.first != d0.first || d2.second != d0.second || d1.second != d2.first)
                throw ParseError{"line " + std::to_string(st.line) + ": gemm tile shapes do not match"};
        } else if (d0 != d1) {
            throw ParseError{"line " + std::to_string(st.line) + ": axpby tiles differ in shape"};
        }
        for (const Ref& x : t)
            if (prog.operands[x.op].es != 8)
                throw ParseError{"line " + std::to_string(st.line) + ": kernels take FP64 operands"};
        // inputs' (and a loaded output's) data must have arrived
        std::vector<int> need;
        for (size_t a = 0; a < sl.size(); ++a)
            if (!slot[sl[a]].compute_synced) need.push_back(sl[a]);
        std::sort(need.begin(), need.end(), [&](int x, int y) {
            return rec[ev_ready(x)].vc[kStreamH2D] > rec[ev_ready(y)].vc[kStreamH2D];
        });
        for (int s : need) {
            wait(kStreamCompute, ev_ready(s));
            slot[s].compute_synced = true;
        }
        SlotState& out = slot[sl[0]];
        Op k; k.kind = kKernel; k.stream = kStreamCompute; k.kernel = kernel;
        k.mode = out.fresh ? kPipeFresh : (out.content.v == 0 ? kPipeLoaded : kPipeAccumulate);
        if (k.mode != kPipeFresh) { k.rslot[k.nr] = sl[0]; k.rtag[k.nr] = out.content; ++k.nr; }
        for (size_t a = 1; a < sl.size(); ++a) { k.rslot[k.nr] = sl[a]; k.rtag[k.nr] = slot[sl[a]].content; ++k.nr; }
        k.wslot = sl[0];
        k.wtag = out.content;
        k.wtag.v = out.content.v + 1;
        push(k);
        out.content = k.wtag;
        out.fresh = false;
        out.dirty = true;
        for (size_t a = 1; a < sl.size(); ++a) {
            slot[sl[a]].read_since_fill = true;
            slot[sl[a]].last_use = clock;
            record(kStreamCompute, ev_free(sl[a]));
        }
        out.last_use = clock;
        record(kStreamCompute, ev_done(sl[0]));
    }

    void do_store(const Stmt& st)
    {
        const Ref x = tile(st.tiles[0], st.line);
        const int s = find(x);
        if (s < 0 || slot[s].fresh)
            throw ParseError{"line " + std::to_string(st.line) + ": store of a tile that is not resident"};
        SlotState& S = slot[s];
        wait(kStreamD2H, S.content.v > 0 ? ev_done(s) : ev_ready(s));
        Op d; d.kind = kD2H; d.stream = kStreamD2H; d.nr = 1; d.rslot[0] = s; d.rtag[0] = S.content;
        push(d);
        record(kStreamD2H, ev_out(s));
        S.d2h_pending = true;
        S.dirty = false;
        S.last_use = clock;
    }

    void exec(const std::vector<Stmt>& body)
    {
        for (const Stmt& st : body) {
            ++clock;
            switch (st.kind) {
            case Stmt::Operand: break;
            case Stmt::For: {
                const int64_t lo = eval(*st.e0, st.line), hi = eval(*st.e1, st.line);
                if (env.count(st.name)) throw ParseError{"line " + std::to_string(st.line) + ": loop variable reused"};
                for (int64_t v = lo; v < hi; ++v) {
                    env[st.name] = v;
                    exec(st.body);
                    if (prog.ops.size() > (size_t)50000000)
                        throw ParseError{"the pipeline issues more than 50 million operations"};
                }
                env.erase(st.name);
                break;
            }
            case Stmt::Load:
                if (cond_true(st)) do_load(st, false);
                break;
            case Stmt::Alloc:
                if (cond_true(st)) do_load(st, true);
                break;
            case Stmt::Store:
                if (cond_true(st)) do_store(st);
                break;
            case Stmt::Run: do_run(st); break;
            }
        }
    }
};

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

struct PipeSource {
    std::vector<Stmt> stmts;
};

// Parse the description; returns OOC_OK or OOC_ERR_INVALID_ARG with a message.
int pipe_parse(const std::string& text, std::shared_ptr<PipeSource>& out, std::vector<std::string>& operand_names,
               std::string& why)
{
    std::vector<std::string> lines;
    std::stringstream ss(text);
    std::string l;
    while (std::getline(ss, l)) lines.push_back(l);
    auto src = std::make_shared<PipeSource>();
    try {
        size_t i = 0;
        parse_block(lines, i, src->stmts, false);
        operand_names.clear();
        for (const Stmt& st : src->stmts) {
            if (st.kind != Stmt::Operand) continue;
            for (const auto& n : operand_names)
                if (n == st.name) throw ParseError{"line " + std::to_string(st.line) + ": operand declared twice"};
            operand_names.push_back(st.name);
        }
        std::function<void(const std::vector<Stmt>&, bool)> check = [&](const std::vector<Stmt>& b, bool top) {
            for (const Stmt& st : b) {
                if (st.kind == Stmt::Operand && !top)
                    throw ParseError{"line " + std::to_string(st.line) + ": operands are declared at the top level"};
                if (st.kind == Stmt::For) check(st.body, false);
            }
        };
        check(src->stmts, true);
    } catch (const ParseError& e) {
        why = e.msg;
        return OOC_ERR_INVALID_ARG;
    }
    out = src;
    return OOC_OK;
}

// Compile for the bound operands and variables: tile sizes, slot layout and
// the schedule.  Operand dimensions must be set (host pointers may be null
// when only the schedule is wanted).
int pipe_compile(const PipeSource& src, std::vector<PipeOperand> operands, const std::map<std::string, double>& vars,
                 PipeProgram& prog, std::string& why)
{
    prog = PipeProgram{};
    prog.operands = std::move(operands);
    try {
        Compiler c(prog, vars);
        // tile sizes and rings in declaration order
        size_t k = 0;
        int32_t slots = 0;
        for (const Stmt& st : src.stmts) {
            if (st.kind != Stmt::Operand) continue;
            PipeOperand& o = prog.operands[k++];
            if (!o.bound) throw ParseError{"operand " + o.name + " is not bound"};
            o.tr = c.eval(*st.e0, st.line);
            o.tc = c.eval(*st.e1, st.line);
            if (o.tr < 1 || o.tc < 1)
                throw ParseError{"line " + std::to_string(st.line) + ": tile sizes must be positive"};
            o.tr = std::min(o.tr, o.rows);
            o.tc = std::min(o.tc, o.cols);
            const int64_t ring = c.eval(*st.e2, st.line);
            if (ring < 1 || ring > 4096)
                throw ParseError{"line " + std::to_string(st.line) + ": a ring needs 1 to 4096 slots"};
            o.ring = (int32_t)ring;
            o.slot0 = slots;
            slots += o.ring;
            o.ld_dev = (o.tc + 15) / 16 * 16;
            o.slot_bytes = align256((size_t)o.tr * o.ld_dev * o.es);
        }
        prog.slots = slots;
        prog.events = 4 * slots;
        size_t off = prog.header;
        for (const PipeOperand& o : prog.operands)
            for (int r = 0; r < o.ring; ++r) {
                prog.slot_off.push_back(off);
                off += o.slot_bytes;
            }
        prog.device_bytes = off;
        c.slot.assign(slots, SlotState{});
        c.rec.assign(prog.events, Compiler::Clock{});
        c.exec(src.stmts);
        for (int s = 0; s < slots; ++s)
            if (c.slot[s].dirty) {
                const PipeOperand& o = prog.operands[c.slot[s].content.m];
                throw ParseError{"tile " + o.name + "[" + std::to_string(c.slot[s].content.r) + ", " +
                                 std::to_string(c.slot[s].content.c) + "] is written but never stored"};
            }
    } catch (const ParseError& e) {
        why = e.msg;
        return OOC_ERR_INVALID_ARG;
    }
    return OOC_OK;
}

}  // namespace ooc
