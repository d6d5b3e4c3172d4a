"""Host-side logic of the library, checked without a GPU.

* the shared library loads and exports every function include/ooc.h declares;
* the planner's paper mode equals the oracle's reading of the Section IV
  partitioner (bit-exact integers), and every plan fits its budget;
* every issued schedule satisfies the Section IV buffer-hazard rule, checked by
  the oracle's timeline checker, and returns each C block exactly once.
"""
import itertools
import os
import re

import pytest

import paper_1808_05056_gb300 as P
from oracle import partition, pipeline

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "ooc.h")


@pytest.fixture(scope="module", autouse=True)
def built():
    P.build()
    P.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ooc_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported():
    lib = P.load()
    names = declared_functions()
    assert "ooc_dgemm" in names and "ooc_plan" in names
    for n in names:
        assert hasattr(lib, n), n
    assert set(P.EXPORTS) <= set(names)


def test_errors_are_named():
    for code in range(0, -11, -1):
        assert P.ooc_strerror(code) != "unknown status"


def test_invalid_arguments_rejected_before_device():
    assert P.ooc_dgemm("X", "N", 2, 2, 2, 1.0, 1, 2, 1, 2, 0.0, 1, 2, 1 << 20) == P.OOC_ERR_INVALID_ARG
    assert P.ooc_dgemm("N", "N", 2, 2, 4, 1.0, 1, 3, 1, 2, 0.0, 1, 2, 1 << 20) == P.OOC_ERR_INVALID_ARG
    assert P.ooc_dgemm("N", "N", -1, 2, 2, 1.0, 1, 2, 1, 2, 0.0, 1, 2, 1 << 20) == P.OOC_ERR_INVALID_ARG
    assert P.ooc_dgemm("N", "N", 2, 2, 2, 1.0, None, 2, 1, 2, 0.0, 1, 2, 1 << 20) == P.OOC_ERR_INVALID_ARG
    # empty problems are a no-op
    assert P.ooc_dgemm("N", "N", 0, 5, 5, 1.0, None, 5, None, 5, 0.0, None, 5, 1 << 20) == P.OOC_OK


def test_missing_library_fails_loudly(tmp_path):
    with pytest.raises(RuntimeError, match="not built"):
        P.load(str(tmp_path / "libooc.so"))


@pytest.mark.skipif(__import__("torch").cuda.is_available(), reason="needs a machine without a GPU")
def test_no_cpu_fallback_without_a_device():
    """Every compute entry point returns an error on a machine with no sm_103 device and leaves
    the host data untouched: there is no CPU path behind the C ABI."""
    import numpy as np
    A, B = np.ones((4, 4)), np.ones((4, 4))
    C = np.full((4, 4), 7.0)
    A4, C4 = np.ones((4, 4), dtype=np.float32), np.full((4, 4), 7.0, dtype=np.float32)
    ipiv = np.zeros(4, dtype=np.int64)
    nd = P.OOC_ERR_NO_DEVICE
    assert P.ooc_dgemm("N", "N", 4, 4, 4, 1.0, A, 4, B, 4, 0.0, C, 4, 1 << 20) == nd
    assert P.ooc_sgemm("N", "N", 4, 4, 4, 1.0, A4, 4, A4, 4, 0.0, C4, 4, 1 << 20) == nd
    assert P.ooc_dgemmt("L", "N", "N", 4, 4, 1.0, A, 4, B, 4, 0.0, C, 4, 1 << 20) == nd
    assert P.ooc_dsyrk("L", "N", 4, 4, 1.0, A, 4, 0.0, C, 4, 1 << 20) == nd
    assert P.ooc_ssyrk("L", "N", 4, 4, 1.0, A4, 4, 0.0, C4, 4, 1 << 20) == nd
    assert P.ooc_dtrsm("L", "L", "N", "N", 4, 4, 1.0, A, 4, C, 4, 1 << 20) == nd
    assert P.ooc_dpotrf("L", 4, C, 4, 1 << 20)[0] == nd
    assert P.ooc_dgetrf(4, C, 4, ipiv, 1 << 20)[0] == nd
    assert P.ooc_dgemm_batched([P.gemm_desc("N", "N", A, B, C)], 1 << 20) == nd
    assert P.ooc_dgemm_device("N", "N", 4, 4, 4, 1.0, 1, 4, 1, 4, 0.0, 1, 4) == nd
    assert P.ooc_dgemm_noalloc("N", "N", 4, 4, 4, 1.0, A, 4, B, 4, 0.0, C, 4, 1 << 20) == nd
    with pytest.raises(RuntimeError):
        P.ooc_query_fp64_peak(0.1)
    assert P.Session(4, 4, C, 4, 0.0, 1 << 20).rc == nd
    pipe = P.Pipe(P.MMOOC_PIPELINE)
    for name, v in dict(mb=4, nb=4, kb=4, ra=2, rb=2, rc=2, alpha=1.0, beta=0.0, beta_nz=0).items():
        pipe.set(name, v)
    for name, t in (("A", A), ("B", B), ("C", C)):
        pipe.bind(name, t)
    assert pipe.run(1 << 20) == nd
    assert (C == 7.0).all() and (C4 == 7.0).all() and (ipiv == 0).all()


def test_leading_dimension_of_row_major_views():
    """The binding passes views whose rows are contiguous (padding between rows is fine) and
    rejects views with strided rows, which the C ABI's (pointer, ld) pair cannot describe."""
    import numpy as np
    import torch
    t = torch.zeros(8, 16, dtype=torch.float64)
    assert P._ld(t) == 16
    assert P._ld(t[:, :10]) == 16          # padded rows: ld 16 for 10 columns
    assert P._ld(t[:, 3:4]) == 16          # one column: no stride within a row
    assert P._ld(t[2:3, :]) == 16          # one row
    for bad in (t[:, ::2], t.t()):
        with pytest.raises(ValueError):
            P._ld(bad)
    a = np.zeros((8, 16))
    assert P._ld(a) == 16 and P._ld(a[:, :10]) == 16
    for bad in (a[:, ::2], a.T):
        with pytest.raises(ValueError):
            P._ld(bad)


def test_gemm_helpers_check_shapes_and_types():
    import torch
    f8 = lambda r, c: torch.zeros(r, c, dtype=torch.float64)
    f4 = lambda r, c: torch.zeros(r, c, dtype=torch.float32)
    assert P._shape_args("N", "N", f8(5, 3), f8(3, 4), f8(5, 4), 8) == (5, 4, 3)
    assert P._shape_args("T", "T", f8(3, 5), f8(4, 3), f8(5, 4), 8) == (5, 4, 3)
    assert P._shape_args("N", "N", f4(5, 3), f4(3, 4), f4(5, 4)) == (5, 4, 3)
    bad = [
        (("N", "N", f8(5, 3), f8(2, 4), f8(5, 4), 8), "chain"),        # inner dimensions differ
        (("N", "T", f8(5, 3), f8(3, 4), f8(5, 4), 8), "chain"),        # op(B) is 4 x 3
        (("N", "N", f8(5, 3), f8(3, 4), f8(4, 5), 8), "chain"),        # C the wrong shape
        (("N", "N", f4(5, 3), f4(3, 4), f4(5, 4), 8), "bytes"),        # float32 into dgemm
        (("N", "N", f8(5, 3), f8(3, 4), f8(5, 4), 4), "bytes"),        # float64 into sgemm
        (("N", "N", f8(5, 3), f4(3, 4), f8(5, 4)), "one element type"),
        (("N", "N", torch.zeros(5, 3, dtype=torch.int64), f8(3, 4), f8(5, 4), 8), "bytes"),
        (("N", "N", f8(5, 3)[0], f8(3, 4), f8(5, 4), 8), "2-D"),
    ]
    for args, msg in bad:
        with pytest.raises(ValueError, match=msg):
            P._shape_args(*args)


def test_paper_mode_worked_example():
    plan = P.ooc_plan(4, 4, 8, 8, 1, 44 * 8, P.make_opts(flags=P.OOC_PLAN_PAPER))
    assert plan["blocks"] == 8 and (plan["mb"], plan["nb"], plan["kb"]) == (1, 2, 8)
    assert (plan["depth"], plan["b_buffers"], plan["c_buffers"]) == (2, 1, 2)


@pytest.mark.parametrize("M,N,K,mem", [(4, 4, 8, 44), (16, 16, 16, 200), (12, 18, 10, 150),
                                       (32, 8, 64, 1000), (6, 6, 6, 108), (24, 36, 5, 300),
                                       (30, 20, 7, 199), (9, 27, 81, 2000)])
def test_paper_mode_matches_oracle_partitioner(M, N, K, mem):
    hw = partition.partition(M, N, K, mem)
    opts = P.make_opts(flags=P.OOC_PLAN_PAPER)
    if hw is None:
        with pytest.raises(P.OocError):
            P.ooc_plan(M, N, K, 8, 1, mem * 8, opts)
        return
    plan = P.ooc_plan(M, N, K, 8, 1, mem * 8, opts)
    assert (M // plan["mb"], N // plan["nb"]) == hw


@pytest.mark.parametrize("M,N,K,es,budget,beta", [
    (1024, 1024, 1024, 8, 4 << 20, 0), (1000, 700, 300, 8, 1 << 20, 1), (64, 64, 64, 8, 1 << 16, 1),
    (32768, 32768, 32768, 8, 4 << 30, 1), (65536, 65536, 16384, 8, 16 << 30, 0),
    (65536, 65536, 65536, 4, 8 << 30, 1), (5000, 3, 7000, 8, 2 << 20, 0), (3, 5000, 7000, 8, 2 << 20, 1)])
def test_auto_plans_fit_and_count_traffic(M, N, K, es, budget, beta):
    plan = P.ooc_plan(M, N, K, es, beta, budget)
    assert 0 < plan["device_bytes"] <= budget
    assert plan["mb"] >= 1 and plan["nb"] >= 1 and plan["kb"] >= 1
    # traffic lower bounds: every operand crosses at least once, C comes back once
    assert plan["h2d_bytes"] >= (M * K + K * N + (M * N if beta else 0)) * es
    assert plan["d2h_bytes"] == M * N * es


def test_budget_too_small():
    with pytest.raises(P.OocError) as e:
        P.ooc_plan(1024, 1024, 1024, 8, 0, 4096)
    assert e.value.code == P.OOC_ERR_BUDGET


def to_checker(ops):
    """Library schedule entries -> the oracle checker's operation dicts."""
    kinds = {0: "h2d", 1: "kernel", 2: "d2h", 3: "record", 4: "wait", 5: "split"}
    out = []
    for o in ops:
        d = dict(kind=kinds[o["kind"]], stream=o["stream"])
        if o["kind"] in (3, 4):
            d["event"] = o["event"]
        if o["write_slot"] >= 0:
            d["writes"] = [(o["write_slot"], o["write_tag"])]
        d["reads"] = list(zip(o["read_slot"], o["read_tag"]))
        out.append(d)
    return out


def _expected_blocks(M, N, plan):
    h = -(-M // plan["mb"])
    w = -(-N // plan["nb"])
    nkc = plan["steps"] // (h * w)
    return h, w, nkc


CASES = [
    # (M, N, K, es, beta, budget, opts kwargs)
    (4, 4, 8, 8, 1, 44 * 8, dict(flags=1)),
    (4, 4, 8, 8, 0, 44 * 8, dict(flags=1)),
    (12, 18, 10, 8, 1, 150 * 8, dict(flags=1)),
    (1024, 1024, 1024, 8, 0, 4 << 20, {}),
    (1000, 700, 300, 8, 1, 1 << 20, {}),
    (300, 200, 170, 8, 1, 0, dict(mb=64, nb=64, kb=64, depth=2, c_buffers=2)),
    (300, 200, 170, 8, 0, 0, dict(mb=128, nb=64, kb=64, depth=3, c_buffers=3)),
    (256, 256, 512, 8, 1, 0, dict(mb=64, nb=128, kb=128, depth=2, c_buffers=2)),
    (200, 130, 0, 8, 1, 1 << 20, {}),
    (640, 64, 640, 8, 1, 0, dict(mb=64, nb=64, kb=640, depth=2, c_buffers=2)),
    # whole-K B slices, two B slots, several blocks per column: the next column's B slice is
    # prefetched in row ranges between this column's A loads
    (1000, 700, 300, 8, 1, 0, dict(mb=128, nb=128, kb=300, depth=2, c_buffers=2, b_buffers=2)),
    (1024, 1024, 512, 4, 1, 0, dict(form=3, mb=256, nb=256, depth=3, b_buffers=2)),
    # split forms (staged: raw A / B chunks land in one staging area per operand and are split from
    # there into the slots' planes): one B slot with the next slice streamed into the staging area,
    # K chunks, ragged edges, Ozaki and BF16x3
    (1000, 700, 300, 4, 1, 0, dict(form=3, mb=128, nb=128, kb=300, depth=2, c_buffers=2, b_buffers=1)),
    (1000, 700, 300, 8, 0, 0, dict(form=2, mb=256, nb=128, kb=300, depth=2, c_buffers=2, b_buffers=1)),
    (600, 520, 700, 8, 1, 0, dict(form=2, mb=128, nb=256, kb=256, depth=2, c_buffers=2, b_buffers=2)),
    (600, 520, 700, 4, 0, 0, dict(form=3, mb=256, nb=128, kb=192, depth=3, c_buffers=3, b_buffers=1)),
    (65536, 65536, 65536, 4, 1, 8 << 30, dict(form=3)),
]


def test_next_b_slice_is_prefetched_in_pieces_before_the_column_switch():
    """Whole-K B slices with a spare B slot: the next column's slice is copied as row-range pieces
    issued between the current column's kernels, all of them before the next column's first
    kernel, and the first of them after the current column's second A load (so it never waits
    for the kernel issued just before it)."""
    M, N, K = 1000, 700, 300
    opts = P.make_opts(mb=128, nb=128, kb=300, depth=2, c_buffers=2, b_buffers=2)
    plan = P.ooc_plan(M, N, K, 8, 1, 1 << 40, opts)
    assert plan["kb"] == K and plan["b_buffers"] == 2
    ops = P.ooc_schedule(M, N, K, 8, 1, 1 << 40, opts)
    h, w = -(-M // 128), -(-N // 128)
    kernel_pos = {}
    b_writes = {}
    for n, o in enumerate(ops):
        if o["kind"] == 1:
            kernel_pos.setdefault(o["write_tag"][2], []).append(n)
        elif o["kind"] == 0 and o["write_tag"][0] == 1:
            b_writes.setdefault(o["write_tag"][2], []).append(n)
    assert len(b_writes[0]) == 1                       # the first column's slice: one copy
    for j in range(1, w):
        pieces = b_writes[j]
        assert len(pieces) == min(8, h - 1)            # the others: pieces
        assert max(pieces) < kernel_pos[j][0]          # all before the column's first kernel
        assert min(pieces) > kernel_pos[j - 1][0]      # the first after the previous column's first kernel
        assert min(pieces) < kernel_pos[j - 1][-1]     # issued while that column still runs


@pytest.mark.parametrize("case", range(len(CASES)))
def test_issued_schedule_respects_the_hazard_rule(case):
    M, N, K, es, beta, budget, kw = CASES[case]
    opts = P.make_opts(**kw)
    if budget == 0:
        budget = 1 << 40
    plan = P.ooc_plan(M, N, K, es, beta, budget, opts)
    ops = P.ooc_schedule(M, N, K, es, beta, budget, opts)
    chk = to_checker(ops)
    assert pipeline.check(chk) == []
    h, w, nkc = _expected_blocks(M, N, plan)
    finals = sorted(t for _, t in pipeline.final_host_writes(chk))
    assert finals == sorted((2, i, j, nkc) for i in range(h) for j in range(w))
    # every kernel of block (i, j, kc) reads its own A and B chunks (when K > 0)
    for o in ops:
        if o["kind"] != 1:
            continue
        _, i, j, v = o["write_tag"]
        kc = v - 1
        tags = o["read_tag"]
        if K > 0:
            assert (0, i, kc, 0) in tags and (1, kc, j, 0) in tags
        if kc > 0 or beta:
            assert (2, i, j, kc) in tags


@pytest.mark.parametrize("form,es,b_buffers", [(3, 4, 1), (2, 8, 2)])
def test_staged_schedule_splits_each_load_once_and_every_wait_is_needed(form, es, b_buffers):
    """Split forms: every A / B copy writes the operand's staging area (slot ids just past the
    plan's slots), every such datum is split exactly once into a slot before a kernel reads it,
    and removing any wait the library issues breaks the hazard rule."""
    M, N, K = 1000, 700, 300
    opts = P.make_opts(form=form, mb=128, nb=128, kb=300, depth=2, c_buffers=2, b_buffers=b_buffers)
    ops = P.ooc_schedule(M, N, K, es, 1, 1 << 40, opts)
    plan = P.ooc_plan(M, N, K, es, 1, 1 << 40, opts)
    nslots = plan["depth"] + plan["b_buffers"] + plan["c_buffers"]
    staged_copies, splits = [], []
    for o in ops:
        if o["kind"] == 0 and o["write_tag"][0] in (0, 1):
            assert o["write_slot"] - nslots - 2 * o["write_tag"][0] in (0, 1)
            staged_copies.append(tuple(o["write_tag"]))
        elif o["kind"] == 5:
            assert o["stream"] == 1 and o["read_slot"][0] - nslots - 2 * o["read_tag"][0][0] in (0, 1)
            assert tuple(o["read_tag"][0]) == tuple(o["write_tag"]) and o["write_slot"] < nslots
            splits.append(tuple(o["write_tag"]))
    # per operand, the staged data in copy order (the row-range pieces of one B slice collapse to
    # one) is exactly the split order
    for m in (0, 1):
        copies = [t for t in staged_copies if t[0] == m]
        collapsed = [t for k, t in enumerate(copies) if k == 0 or copies[k - 1] != t]
        assert collapsed == [t for t in splits if t[0] == m] and collapsed
    chk = to_checker(ops)
    assert pipeline.check(chk) == []
    waits = [k for k, o in enumerate(chk) if o["kind"] == "wait"]
    assert waits
    assert all(pipeline.check(chk[:k] + chk[k + 1:]) for k in waits)


@pytest.mark.parametrize("form,es", [(3, 4), (2, 8)])
def test_staged_a_loads_run_a_block_ahead(form, es):
    """Split forms: an A copy waits only for the split of the A chunk two blocks back (two staging
    areas), so the copy for block i + 1 overlaps kernel i and the kernel before it."""
    M, N, K = 2000, 700, 300
    opts = P.make_opts(form=form, mb=128, nb=128, kb=300, depth=2, c_buffers=2, b_buffers=1)
    ops = P.ooc_schedule(M, N, K, es, 1, 1 << 40, opts)
    kernels_issued, recorded_after, pending = 0, {}, None
    checked = 0
    for o in ops:
        if o["kind"] == 1:
            kernels_issued += 1
        elif o["kind"] == 3 and o["stream"] == 1:
            recorded_after[o["event"]] = kernels_issued
        elif o["kind"] == 4 and o["stream"] == 0:
            pending = o["event"]
        elif o["kind"] == 0:
            if pending is not None and o["write_tag"][0] == 0 and pending in recorded_after:
                assert recorded_after[pending] <= kernels_issued - 2, (o["write_tag"], kernels_issued)
                checked += 1
            pending = None
    assert checked > 10


def test_staged_plan_streams_the_next_b_slice_with_one_b_slot():
    """One B slot in a split-form plan: the next column's slice is copied in pieces into the
    staging area while the current column runs, and split into the slot at the column switch."""
    M, N, K = 1000, 700, 300
    opts = P.make_opts(form=3, mb=128, nb=128, kb=300, depth=2, c_buffers=2, b_buffers=1)
    ops = P.ooc_schedule(M, N, K, 4, 1, 1 << 40, opts)
    h, w = -(-M // 128), -(-N // 128)
    kernel_pos, b_pieces, b_split = {}, {}, {}
    for n, o in enumerate(ops):
        if o["kind"] == 1:
            kernel_pos.setdefault(o["write_tag"][2], []).append(n)
        elif o["kind"] == 0 and o["write_tag"][0] == 1:
            b_pieces.setdefault(o["write_tag"][2], []).append(n)
        elif o["kind"] == 5 and o["write_tag"][0] == 1:
            b_split[o["write_tag"][2]] = n
    for j in range(1, w):
        assert len(b_pieces[j]) == min(8, h - 1)
        assert kernel_pos[j - 1][0] < min(b_pieces[j]) and max(b_pieces[j]) < kernel_pos[j - 1][-1]
        assert kernel_pos[j - 1][-1] < b_split[j] < kernel_pos[j][0]


def test_checker_catches_a_dropped_library_wait():
    ops = P.ooc_schedule(300, 200, 170, 8, 1, 1 << 40,
                         P.make_opts(mb=64, nb=64, kb=64, depth=2, c_buffers=2))
    chk = to_checker(ops)
    waits = [k for k, o in enumerate(chk) if o["kind"] == "wait"]
    assert waits
    caught = 0
    for k in waits:
        if pipeline.check(chk[:k] + chk[k + 1:]):
            caught += 1
    # every wait the library issues is needed
    assert caught == len(waits)


@pytest.mark.parametrize("M,N,K,es,beta,budget,kw", [
    (32768, 32768, 32768, 8, 1, 4 << 30, {}),
    (1000, 700, 300, 8, 1, 0, dict(mb=64, nb=64, kb=64, depth=2, c_buffers=2)),
    (4096, 4096, 4096, 8, 0, 0, dict(mb=1024, nb=1024, kb=1024, depth=3, c_buffers=2)),
])
def test_operand_loads_never_wait_for_the_kernel_just_issued(M, N, K, es, beta, budget, kw):
    """With rings of >= 2 slots, a refill waits at most for the kernel two steps back,
    so every copy overlaps the kernel issued just before it."""
    budget = budget or 1 << 40
    opts = P.make_opts(**kw)
    plan = P.ooc_plan(M, N, K, es, beta, budget, opts)
    assert plan["depth"] >= 2
    ops = P.ooc_schedule(M, N, K, es, beta, budget, opts)
    kernels_issued = 0
    recorded_after = {}      # event -> kernels issued when it was last recorded (compute stream)
    pending_wait = None
    for o in ops:
        if o["kind"] == 1:
            kernels_issued += 1
        elif o["kind"] == 3 and o["stream"] == 1:
            recorded_after[o["event"]] = kernels_issued
        elif o["kind"] == 4 and o["stream"] == 0:
            pending_wait = o["event"]
        elif o["kind"] == 0:
            if pending_wait is not None and pending_wait in recorded_after and o["write_tag"][0] in (0, 1):
                waited_kernel = recorded_after[pending_wait] - 1
                assert waited_kernel <= kernels_issued - 2, (o["write_tag"], waited_kernel, kernels_issued)
            pending_wait = None


# ---- triangular updates (GEMMT / SYRK) -----------------------------------
def _classify(N, mb, nb, i, j, uplo):
    """0: no element of block (i, j) is updated, 1: all are, 2: some are."""
    rows = range(i * mb, min(N, (i + 1) * mb))
    cols = range(j * nb, min(N, (j + 1) * nb))
    # the updated set of a rectangle is decided by its extreme values of col - row
    lo, hi = cols[0] - rows[-1], cols[-1] - rows[0]
    if uplo == "L":
        return 0 if lo > 0 else (1 if hi <= 0 else 2)
    return 0 if hi < 0 else (1 if lo >= 0 else 2)


TRI_CASES = [
    # (uplo, N, K, beta, opts)
    ("L", 300, 170, 0, dict(mb=64, nb=64, kb=64, depth=2, c_buffers=2)),
    ("U", 300, 170, 1, dict(mb=64, nb=64, kb=64, depth=2, c_buffers=2)),
    ("L", 333, 90, 0, dict(mb=96, nb=160, kb=90, depth=3, c_buffers=3)),
    ("U", 333, 90, 0, dict(mb=160, nb=96, kb=32, depth=2, c_buffers=2)),
    ("L", 1000, 500, 1, {}),
    ("U", 4096, 1024, 0, {}),
]


@pytest.mark.parametrize("case", range(len(TRI_CASES)))
def test_triangular_schedule_updates_exactly_the_triangle(case):
    uplo, N, K, beta, kw = TRI_CASES[case]
    budget = (1 << 40) if kw else (8 << 20)
    plan, ops = P.ooc_schedule_gemmt(uplo, N, K, 8, beta, budget, P.make_opts(**kw))
    mb, nb = plan["mb"], plan["nb"]
    h, w = -(-N // mb), -(-N // nb)
    cls = {(i, j): _classify(N, mb, nb, i, j, uplo) for i in range(h) for j in range(w)}
    active = {b for b, c in cls.items() if c}
    chk = to_checker(ops)
    assert pipeline.check(chk) == []
    nkc = plan["steps"] // plan["blocks"]
    finals = sorted(t for _, t in pipeline.final_host_writes(chk))
    assert finals == sorted((2, i, j, nkc) for i, j in active)
    assert plan["blocks"] == len(active)
    loaded_c = {(o["write_tag"][1], o["write_tag"][2]) for o in ops if o["kind"] == 0 and o["write_tag"][0] == 2}
    straddling = {b for b, c in cls.items() if c == 2}
    assert loaded_c == (active if beta else straddling)
    # blocks with no updated element are never touched
    touched = {(o["write_tag"][1], o["write_tag"][2]) for o in ops if o["write_tag"][0] == 2}
    assert touched <= active
    if any(c == 0 for c in cls.values()):
        assert len(active) < h * w


def test_triangular_schedule_waits_are_all_needed():
    _, ops = P.ooc_schedule_gemmt("L", 333, 90, 8, 0, 1 << 40,
                                  P.make_opts(mb=96, nb=160, kb=32, depth=2, c_buffers=2))
    chk = to_checker(ops)
    waits = [k for k, o in enumerate(chk) if o["kind"] == "wait"]
    assert waits and all(pipeline.check(chk[:k] + chk[k + 1:]) for k in waits)


def test_triangular_plan_moves_about_half_the_bytes():
    full = P.ooc_plan(16384, 16384, 4096, 8, 0, 1 << 30, P.make_opts(mb=2048, nb=2048, kb=4096))
    tri, _ = P.ooc_schedule_gemmt("L", 16384, 4096, 8, 0, 1 << 30, P.make_opts(mb=2048, nb=2048, kb=4096))
    assert tri["blocks"] == 8 * 9 // 2 and full["blocks"] == 64
    assert tri["d2h_bytes"] == pytest.approx(full["d2h_bytes"] * 36 / 64)
    assert tri["seconds"] < 0.7 * full["seconds"]


# ---- sessions (Section IV nsteps: one C over several calls) ----------------------
SESSION_CASES = [
    # (M, N, K, beta, mb, nb, resident blocks, call)
    (300, 200, 170, 1, 64, 64, 0, 0),
    (300, 200, 170, 1, 64, 64, 5, 0),
    (300, 200, 170, 0, 64, 64, 5, 1),
    (300, 200, 170, 1, 64, 64, 20, 2),     # every block resident: no C ring, no C copies
    (300, 200, 170, 0, 128, 64, 3, 0),
    (1000, 700, 300, 1, 256, 128, 7, 3),
]


@pytest.mark.parametrize("case", range(len(SESSION_CASES)))
def test_session_call_schedule(case):
    M, N, K, beta, mb, nb, nres, call = SESSION_CASES[case]
    opts = P.make_opts(mb=mb, nb=nb, kb=64, depth=2)
    plan, ops = P.ooc_schedule_session(M, N, K, beta, 1 << 40, opts, nres, call)
    h, w = -(-M // mb), -(-N // nb)
    order = [(i, j) for j in range(w) for i in range(h)]       # schedule order of the blocks
    resident = set(order[:nres])
    ring = plan["depth"] + plan["b_buffers"] + plan["c_buffers"]
    res_slot = {b: ring + r for r, b in enumerate(order[:nres])}
    initial = [(res_slot[b], (2, b[0], b[1], 0)) for b in resident] if call > 0 else []
    chk = to_checker(ops)
    assert pipeline.check(chk, initial=initial) == []
    if call > 0 and resident:
        assert pipeline.check(chk)          # without the carried-over contents the reads are unfed
    # resident blocks never leave the device; every other block goes back exactly once
    nkc = plan["steps"] // (h * w)
    finals = sorted(t for _, t in pipeline.final_host_writes(chk))
    assert finals == sorted((2, i, j, nkc) for i, j in order if (i, j) not in resident)
    loads = {(o["write_tag"][1], o["write_tag"][2]) for o in ops if o["kind"] == 0 and o["write_tag"][0] == 2}
    if call == 0:
        assert loads == (set(order) if beta else set())
    else:
        assert loads == set(order) - resident           # partial sums come back from the host
    # resident blocks live in their own slots; the kernels of a later call accumulate
    for o in ops:
        if o["kind"] == 1:
            _, i, j, v = o["write_tag"]
            if (i, j) in resident:
                assert o["write_slot"] == res_slot[(i, j)]
            if call > 0:
                assert (2, i, j, v - 1) in o["read_tag"]
    if nres == h * w:
        assert plan["c_buffers"] == 0


def test_planner_keeps_the_fp64_benchmark_plan():
    """FP64 32768^3 in 4 GiB: the plan the FP64 tile kernel was measured on (0.996 of its peak);
    the planner's overlap cost is zero for FP64, so copies hidden under FP64 kernels do not move it."""
    p = P.ooc_plan(32768, 32768, 32768, 8, 1, 4 << 30, P.make_opts(form=P.OOC_FORM_FP64))
    assert (p["mb"], p["nb"], p["kb"]) == (2048, 8192, 8192)


@pytest.mark.parametrize("form,es,K,beta,budget,max_h2d", [
    (3, 4, 65536, 1, 8 << 30, 200e9),    # BF16x3 65536^3, 8 GiB: was 309 GB per call before staging
    (2, 8, 16384, 0, 16 << 30, 40e9),    # Ozaki 65536^2 x 16384, 16 GiB: was 77 GB
])
def test_planner_prefers_fewer_bytes_for_the_split_forms(form, es, K, beta, budget, max_h2d):
    """The split forms' staged layout fits wider blocks in the budget, and the overlap cost makes
    the planner use that room to send fewer bytes; the plan still fits the budget."""
    p = P.ooc_plan(65536, 65536, K, es, beta, budget, P.make_opts(form=form))
    assert p["h2d_bytes"] <= max_h2d
    assert p["device_bytes"] <= budget
