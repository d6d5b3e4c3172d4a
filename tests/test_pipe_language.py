"""The pipeline-description language (end of Section IV): descriptions compile
to schedules that satisfy the Section IV hazard rule (checked by the oracle's
checker), carry the same work as the library's own GEMM schedule, and name the
line of every mistake.  Host only: the compiler needs no GPU.
"""
import pytest

import paper_1808_05056_gb300 as P
from oracle import pipeline
from test_host_logic import to_checker

AXPBY = """
operand X tile tr tc ring 2
operand Y tile tr tc ring 2
for i in 0 .. trows(Y)
  for j in 0 .. tcols(Y)
    load X[i, j]
    load Y[i, j]
    run axpby Y[i, j] X[i, j]
    store Y[i, j]
  end
end
"""


def mmooc(M, N, K, mb, nb, kb, ra=2, rb=2, rc=2, beta_nz=1):
    p = P.Pipe(P.MMOOC_PIPELINE)
    assert p.rc == 0, P.ooc_last_error()
    for name, v in dict(mb=mb, nb=nb, kb=kb, ra=ra, rb=rb, rc=rc, beta_nz=beta_nz).items():
        assert p.set(name, v) == 0
    p.bind("A", rows=M, cols=K, ld=K)
    p.bind("B", rows=K, cols=N, ld=N)
    p.bind("C", rows=M, cols=N, ld=N)
    return p


@pytest.mark.parametrize("M,N,K,mb,nb,kb,ra,rb,rc,beta", [
    (300, 200, 170, 64, 64, 64, 2, 2, 2, 1),
    (300, 200, 170, 64, 64, 64, 2, 3, 2, 0),      # B column resident across the block rows
    (1000, 700, 300, 256, 128, 300, 3, 1, 3, 1),
    (64, 64, 64, 64, 64, 64, 1, 1, 1, 0),          # one slot each: fully serial, still correct
])
def test_mmooc_description_is_hazard_free_and_complete(M, N, K, mb, nb, kb, ra, rb, rc, beta):
    p = mmooc(M, N, K, mb, nb, kb, ra, rb, rc, beta)
    plan, ops = p.schedule(1 << 40)
    chk = to_checker(ops)
    assert pipeline.check(chk) == []
    h, w, nk = -(-M // mb), -(-N // nb), -(-K // kb)
    finals = sorted(t for _, t in pipeline.final_host_writes(chk))
    assert finals == sorted((2, i, j, nk) for i in range(h) for j in range(w))
    assert plan["steps"] == h * w * nk
    # every wait the compiler emitted is needed
    waits = [k for k, o in enumerate(chk) if o["kind"] == "wait"]
    assert all(pipeline.check(chk[:k] + chk[k + 1:]) for k in waits)
    # C copied in only when beta != 0
    c_loads = [o for o in ops if o["kind"] == 0 and o["write_tag"][0] == 2]
    assert len(c_loads) == (h * w if beta else 0)


def test_mmooc_description_matches_the_library_schedule_work():
    """Same plan, same work: the description and the built-in generator copy the same bytes."""
    M, N, K, mb, nb, kb = 1000, 700, 300, 256, 128, 64
    lib_plan = P.ooc_plan(M, N, K, 8, 1, 1 << 40, P.make_opts(mb=mb, nb=nb, kb=kb, depth=2, c_buffers=2,
                                                               b_buffers=2))
    p = mmooc(M, N, K, mb, nb, kb, 2, 2, 2, 1)
    plan, ops = p.schedule(1 << 40)
    lib_ops = P.ooc_schedule(M, N, K, 8, 1, 1 << 40, P.make_opts(mb=mb, nb=nb, kb=kb, depth=2, c_buffers=2,
                                                                  b_buffers=2))
    count = lambda o, k: sum(1 for x in o if x["kind"] == k)
    for k in (0, 1, 2):
        assert count(ops, k) == count(lib_ops, k)
    assert plan["h2d_bytes"] == lib_plan["h2d_bytes"]
    assert plan["d2h_bytes"] == lib_plan["d2h_bytes"]


def test_axpby_description():
    p = P.Pipe(AXPBY)
    assert p.rc == 0
    p.set("tr", 100)
    p.set("tc", 64)
    p.bind("X", rows=250, cols=130, ld=130)
    p.bind("Y", rows=250, cols=130, ld=130)
    plan, ops = p.schedule(1 << 30)
    chk = to_checker(ops)
    assert pipeline.check(chk) == []
    assert plan["blocks"] == 3 * 3 and plan["steps"] == 9
    assert plan["h2d_bytes"] == 2 * 250 * 130 * 8 and plan["d2h_bytes"] == 250 * 130 * 8


@pytest.mark.parametrize("text,needle", [
    ("operand A tile 4 4 ring 1\nfoo A[0, 0]\n", "line 2: unknown statement"),
    ("operand A tile 4 4 ring 1\nfor i in 0 .. 2\nload A[i, 0]\n", "without 'end'"),
    ("operand A tile 4 4 ring 1\nend\n", "line 2: 'end' without 'for'"),
    ("operand A tile 4 4 ring 1\nload A[0 0]\n", "line 2: expected ','"),
    ("operand A tile 4 4 ring 1\noperand A tile 4 4 ring 1\n", "declared twice"),
])
def test_parse_errors_name_the_line(text, needle):
    p = P.Pipe(text)
    assert p.rc == P.OOC_ERR_INVALID_ARG
    assert needle in P.ooc_last_error(), P.ooc_last_error()


@pytest.mark.parametrize("body,needle", [
    ("run gemm C[0, 0] A[0, 0] B[0, 0]\n", "not resident"),
    ("alloc C[0, 0]\nload A[0, 0]\nload B[0, 0]\nrun gemm C[0, 0] A[0, 0] B[0, 0]\n", "never stored"),
    ("alloc C[0, 0]\nload A[0, 0]\nload B[0, 0]\nrun gemm C[0, 0] A[0, 0] B[0, 0]\nalloc C[1, 0]\n",
     "not stored"),
    ("load A[9, 0]\n", "outside the operand"),
    ("load Q[0, 0]\n", "unknown operand"),
    ("load A[zz, 0]\n", "unknown variable"),
    ("alloc C[0, 0]\nload A[0, 0]\nload B[0, 0]\nrun fft C[0, 0] A[0, 0] B[0, 0]\n", "unknown kernel"),
    ("alloc C[0, 0]\nload A[0, 0]\nload B[0, 1]\nrun gemm C[0, 0] A[0, 0] B[0, 1]\nstore C[0, 0]\n", None),
])
def test_compile_errors(body, needle):
    head = "operand A tile 4 8 ring 1\noperand B tile 8 4 ring 1\noperand C tile 4 4 ring 1\n"
    p = P.Pipe(head + body)
    assert p.rc == 0, P.ooc_last_error()
    p.bind("A", rows=8, cols=8, ld=8)
    p.bind("B", rows=8, cols=8, ld=8)
    p.bind("C", rows=8, cols=8, ld=8)
    if needle is None:
        p.schedule(1 << 30)
        return
    with pytest.raises(P.OocError):
        p.schedule(1 << 30)
    assert needle in P.ooc_last_error(), P.ooc_last_error()


def test_ring_size_is_checked():
    p = P.Pipe("operand A tile 4 4 ring r\nload A[0, 0]\nstore A[0, 0]\n")
    assert p.rc == 0
    p.set("r", 0)
    p.bind("A", rows=8, cols=8, ld=8)
    with pytest.raises(P.OocError):
        p.schedule(1 << 20)
    assert "line 1: a ring needs" in P.ooc_last_error()


def test_budget_is_checked():
    p = mmooc(1000, 700, 300, 256, 128, 300)
    with pytest.raises(P.OocError):
        p.schedule(1 << 20)
    assert P.ooc_last_error().startswith("the rings take")
