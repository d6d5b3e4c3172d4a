"""Pins of the partitioner reading and of the buffer-hazard checker (oracle side)."""
import json
import os

import pytest

from oracle import partition, pipeline

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "partition_example.json")


def test_paper_worked_example():
    g = json.load(open(GOLDEN))
    assert g["M"] * g["K"] + g["K"] * g["N"] + g["M"] * g["N"] == g["total_elems"]
    h, w = partition.partition(g["M"], g["N"], g["K"], g["dmem_elems"])
    assert (h, w) == (g["h"], g["w"]) and h * w == g["blocks"]
    assert partition.footprint(g["M"], g["N"], g["K"], h, w) <= g["dmem_elems"]


def test_partition_fits_and_is_minimal():
    for (M, N, K, mem) in [(16, 16, 16, 200), (12, 18, 10, 150), (32, 8, 64, 1000), (6, 6, 6, 108)]:
        hw = partition.partition(M, N, K, mem)
        assert hw is not None
        h, w = hw
        assert partition.footprint(M, N, K, h, w) <= mem
        for hh in range(1, M + 1):
            for ww in range(1, N + 1):
                if M % hh == 0 and N % ww == 0 and hh * ww < h * w:
                    assert partition.footprint(M, N, K, hh, ww) > mem


def test_whole_problem_in_core_when_it_fits():
    # with room for 2A + B + 2C of the whole problem, one block (in-core)
    assert partition.partition(8, 8, 8, 2 * 64 + 64 + 2 * 64) == (1, 1)
    assert partition.partition(8, 8, 8, 10) is None


def _two_stream_schedule(h, w, drop=None):
    """A correct two-stream round-robin schedule over the paper's 2A + 1B + 2C buffers.

    Step idx = i + j*h runs on stream idx % 2 and uses A/C slot idx % 2 (stream
    order protects slot reuse two steps later).  The single B slot is shared:
    its refill waits for the other stream's last kernel, and the other stream's
    next kernel waits for the refill.
    """
    ops = []
    for j in range(w):
        for i in range(h):
            idx = i + j * h
            s = idx % 2
            if i == 0:
                if j > 0 and drop != "wait_kernels_before_b":
                    ops.append(dict(kind="wait", stream=s, event=("k", idx - 1)))
                ops.append(dict(kind="h2d", stream=s, writes=[("B", ("b", j))]))
                ops.append(dict(kind="record", stream=s, event=("b", j)))
            elif i == 1 and drop != "wait_b_ready":
                ops.append(dict(kind="wait", stream=s, event=("b", j)))
            ops.append(dict(kind="h2d", stream=s, writes=[("A%d" % s, ("a", i))]))
            ops.append(dict(kind="h2d", stream=s, writes=[("C%d" % s, ("c", i, j))]))
            ops.append(dict(kind="kernel", stream=s,
                            reads=[("A%d" % s, ("a", i)), ("B", ("b", j)), ("C%d" % s, ("c", i, j))],
                            writes=[("C%d" % s, ("c'", i, j))]))
            ops.append(dict(kind="record", stream=s, event=("k", idx)))
            ops.append(dict(kind="d2h", stream=s, reads=[("C%d" % s, ("c'", i, j))]))
    return ops


def test_checker_accepts_a_correct_pipeline():
    ops = _two_stream_schedule(4, 2)
    assert pipeline.check(ops) == []
    outs = pipeline.final_host_writes(ops)
    assert sorted(t for _, t in outs) == sorted(("c'", i, j) for i in range(4) for j in range(2))


@pytest.mark.parametrize("drop", ["wait_kernels_before_b", "wait_b_ready"])
def test_checker_rejects_a_missing_wait(drop):
    assert pipeline.check(_two_stream_schedule(4, 2, drop=drop))


def test_checker_single_stream_is_always_ordered():
    ops = [dict(kind="h2d", stream=0, writes=[("X", 1)]),
           dict(kind="kernel", stream=0, reads=[("X", 1)], writes=[("Y", 2)]),
           dict(kind="h2d", stream=0, writes=[("X", 3)]),
           dict(kind="kernel", stream=0, reads=[("X", 3), ("Y", 2)], writes=[("Y", 4)]),
           dict(kind="d2h", stream=0, reads=[("Y", 4)])]
    assert pipeline.check(ops) == []


def test_checker_unordered_streams_and_stale_event():
    ops = [dict(kind="h2d", stream=0, writes=[("X", 1)]),
           dict(kind="kernel", stream=1, reads=[("X", 1)])]
    assert pipeline.check(ops)
    # a wait sees the most recent record issued before it, not a later one
    ops = [dict(kind="h2d", stream=0, writes=[("X", 1)]),
           dict(kind="record", stream=0, event="e"),
           dict(kind="h2d", stream=0, writes=[("X", 2)]),
           dict(kind="wait", stream=1, event="e"),
           dict(kind="kernel", stream=1, reads=[("X", 2)]),
           dict(kind="record", stream=0, event="e")]
    assert pipeline.check(ops)


def test_resident_content_from_an_earlier_call():
    """A slot left on the device by an earlier call (nsteps mode) may be read without a
    load in this call only when declared as initial content with the matching tag."""
    sched = [
        dict(kind="h2d", stream=0, writes=[(0, ("A", 0))], reads=[]),
        dict(kind="record", stream=0, event=0),
        dict(kind="wait", stream=1, event=0),
        dict(kind="kernel", stream=1, reads=[(0, ("A", 0)), (5, ("C", 0, 0, 1))], writes=[(5, ("C", 0, 0, 2))]),
    ]
    assert pipeline.check(sched)                                   # nothing wrote slot 5
    assert pipeline.check(sched, initial=[(5, ("C", 0, 0, 1))]) == []
    assert pipeline.check(sched, initial=[(5, ("C", 0, 0, 0))])    # stale version
    # a later load into the resident slot must still be ordered after the kernel's read
    bad = sched + [dict(kind="h2d", stream=0, writes=[(5, ("C", 1, 0, 0))], reads=[])]
    assert pipeline.check(bad, initial=[(5, ("C", 0, 0, 1))])
