"""The OOC_TRACE timeline summariser on hand-made traces with known overlaps."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_1808_05056_gb300 import trace  # noqa: E402

# kind,stream,i,j,kc,bytes,host_ms,start_ms,end_ms
TRACE = """\
# getrf N=64 t=64: c0,panel,laswp,u12,gemm
0,1.0,2.0,3.0,4.0
# call M=8 N=8 K=8 mb=4 nb=4 kb=8 nA=2 nB=2 nC=2
h2d,0,0,0,0,1000000,0.0,0.0,2.0
h2d,0,1,0,0,1000000,0.0,2.0,4.0
kernel,1,0,0,0,0,0.0,2.0,5.0
kernel,1,1,0,0,0,0.0,6.0,9.0
d2h,2,0,0,0,500000,0.0,5.0,6.0
d2h,2,1,0,0,500000,0.0,9.0,10.0
# call M=4 N=4 K=4 mb=4 nb=4 kb=4 nA=2 nB=2 nC=2
h2d,0,0,0,0,64,0.0,0.0,1.0
kernel,1,0,0,0,0,0.0,1.0,3.0
d2h,2,0,0,0,64,0.0,3.0,4.0
"""


@pytest.fixture
def calls(tmp_path):
    p = tmp_path / "t.csv"
    p.write_text(TRACE)
    return trace.parse(str(p))


def test_parse_skips_other_lines(calls):
    assert len(calls) == 2
    assert calls[0]["header"] == {"M": 8, "N": 8, "K": 8, "mb": 4, "nb": 4, "kb": 8, "nA": 2, "nB": 2, "nC": 2}
    assert [o[0] for o in calls[0]["ops"]] == ["h2d", "h2d", "kernel", "kernel", "d2h", "d2h"]


def test_interval_arithmetic():
    u = trace.union([(3, 5), (0, 1), (4, 6), (1, 2), (7, 7)])
    assert u == [(0, 2), (3, 6)]
    assert trace.length(u) == 5
    assert trace.intersect_length(u, trace.union([(1, 4), (5, 9)])) == 1 + 1 + 1


def test_summary_of_a_known_timeline(calls):
    s = trace.summarize(calls[0])
    assert s["span_ms"] == 10.0
    assert s["busy_ms"] == {"h2d": 4.0, "kernel": 6.0, "d2h": 2.0}
    # kernels [2,5) and [6,9): fill 2, one gap of 1, drain 1
    assert s["kernel_idle_ms"] == {"fill": 2.0, "gaps": 1.0, "drain": 1.0}
    # h2d [0,4): [2,4) under a kernel; d2h [5,6) and [9,10): none
    assert s["h2d"]["under_kernels_ms"] == 2.0 and s["h2d"]["under_kernels_frac"] == 0.5
    assert s["d2h"]["under_kernels_ms"] == 0.0
    # 2 MB in 4 ms = 0.5 GB/s; 1 MB in 2 ms = 0.5 GB/s
    assert s["h2d"]["gbps_while_busy"] == pytest.approx(0.5)
    assert s["d2h"]["gbps_while_busy"] == pytest.approx(0.5)
    assert s["kernel_busy_frac"] == pytest.approx(0.6)


def test_cli_prints_every_call(calls, tmp_path, capsys):
    p = tmp_path / "t.csv"
    p.write_text(TRACE)
    assert trace.main([str(p)]) == 0
    out = capsys.readouterr().out
    assert out.count("call ") == 2 and "60.0 % of the span" in out
    assert trace.main([str(p), "--call", "1", "--json"]) == 0
    assert '"call": 1' in capsys.readouterr().out
