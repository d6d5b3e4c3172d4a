"""GPU runs of pipeline descriptions (end of Section IV's pattern language):
the out-of-core GEMM written in the language against the CPU oracle, and a
non-GEMM data-parallel pipeline (tiled axpby) against its definition."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import np64, pinned, pinned_from

pytestmark = pytest.mark.gpu

AXPBY = """
operand X tile tr tc ring 2
operand Y tile tr tc ring 2
for i in 0 .. trows(Y)
  for j in 0 .. tcols(Y)
    load X[i, j]
    load Y[i, j] if b_nz
    alloc Y[i, j] unless b_nz
    run axpby Y[i, j] X[i, j]
    store Y[i, j]
  end
end
"""


def _mmooc(ooc, A, B, C, mb, nb, kb, alpha, beta, rings=(2, 2, 2)):
    p = ooc.Pipe(ooc.MMOOC_PIPELINE)
    assert p.rc == 0, ooc.ooc_last_error()
    for name, v in dict(mb=mb, nb=nb, kb=kb, ra=rings[0], rb=rings[1], rc=rings[2], alpha=alpha, beta=beta,
                        beta_nz=int(beta != 0.0)).items():
        assert p.set(name, v) == 0
    for name, t in (("A", A), ("B", B), ("C", C)):
        assert p.bind(name, t) == 0, ooc.ooc_last_error()
    return p


@pytest.mark.parametrize("M,N,K,mb,nb,kb,beta,rings", [
    (300, 200, 170, 64, 64, 64, 0.5, (2, 2, 2)),
    (300, 200, 170, 96, 160, 64, 0.0, (2, 3, 2)),
    (1000, 700, 300, 256, 128, 300, -1.0, (3, 1, 3)),
    (129, 65, 33, 64, 64, 16, 2.0, (1, 1, 1)),
])
def test_mmooc_description_matches_oracle(ooc, M, N, K, mb, nb, kb, beta, rings):
    A = pinned_from(150, 0, M, K, synth.NORMAL)
    B = pinned_from(150, 1, K, N, synth.NORMAL)
    C = pinned(M, N, fill=float("nan")) if beta == 0.0 else pinned_from(150, 2, M, N, synth.NORMAL)
    C0 = np64(C)
    p = _mmooc(ooc, A, B, C, mb, nb, kb, 1.5, beta, rings)
    st = ooc.ooc_stats()
    assert p.run(1 << 30, st) == 0, ooc.ooc_last_error()
    ref = oracle.gemm("N", "N", 1.5, np64(A), np64(B), beta, None if beta == 0.0 else C0)
    assert oracle.rel_fro(np64(C), ref) <= 1e-13
    assert st.steps == -(-M // mb) * -(-N // nb) * -(-K // kb)


def test_mmooc_description_integers_exact(ooc):
    M, N, K = 256, 192, 300
    A = pinned_from(151, 0, M, K, synth.INTEGER, 512)
    B = pinned_from(151, 1, K, N, synth.INTEGER, 512)
    C = pinned_from(151, 2, M, N, synth.INTEGER, 512)
    C0 = np64(C)
    p = _mmooc(ooc, A, B, C, 64, 128, 64, 1.0, 1.0)
    assert p.run(1 << 30) == 0, ooc.ooc_last_error()
    assert np.array_equal(np64(C), oracle.gemm("N", "N", 1.0, np64(A), np64(B), 1.0, C0))


@pytest.mark.parametrize("b", [0.25, 0.0])
def test_axpby_description(ooc, b):
    rows, cols = 1000, 777
    X = pinned_from(152, 0, rows, cols, synth.NORMAL)
    Y = pinned(rows, cols, fill=float("nan")) if b == 0.0 else pinned_from(152, 1, rows, cols, synth.NORMAL)
    Y0 = np64(Y)
    p = ooc.Pipe(AXPBY)
    assert p.rc == 0, ooc.ooc_last_error()
    for name, v in dict(tr=256, tc=200, a=-2.0, b=b, b_nz=int(b != 0.0)).items():
        p.set(name, v)
    p.bind("X", X)
    p.bind("Y", Y)
    st = ooc.ooc_stats()
    assert p.run(64 << 20, st) == 0, ooc.ooc_last_error()
    want = -2.0 * np64(X) + (b * Y0 if b != 0.0 else 0.0)
    assert np.array_equal(np64(Y), want)   # one multiply-add per element on both sides
    assert st.d2h_bytes == rows * cols * 8


def test_pipe_run_rejects_unpinned_and_budget(ooc):
    A = pinned_from(153, 0, 64, 64, synth.NORMAL)
    B = pinned_from(153, 1, 64, 64, synth.NORMAL)
    C = np.zeros((64, 64))
    p = _mmooc(ooc, A, B, C, 64, 64, 64, 1.0, 0.0)
    assert p.run(1 << 30) == ooc.OOC_ERR_NOT_PINNED
    C2 = pinned(64, 64)
    p = _mmooc(ooc, A, B, C2, 64, 64, 64, 1.0, 0.0)
    assert p.run(1024) == ooc.OOC_ERR_BUDGET
