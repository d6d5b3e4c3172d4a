"""GPU parity of ooc_dgemm_batched (uneven problems through one call) against the CPU oracle."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import np64, pinned, pinned_from

pytestmark = pytest.mark.gpu

SHAPES = [  # (transA, transB, M, N, K, alpha, beta)
    ("N", "N", 300, 200, 170, 1.5, 0.5),
    ("T", "N", 64, 513, 129, 1.0, 0.0),
    ("N", "T", 777, 65, 300, -1.0, 2.0),
    ("T", "T", 128, 128, 1024, 0.5, 0.0),
    ("N", "N", 1000, 700, 64, 1.0, 1.0),
    ("N", "N", 45, 77, 0, 1.0, -2.0),
    ("N", "T", 512, 384, 256, 2.0, 0.25),
]


def _problems(seed, kind=synth.NORMAL):
    probs = []
    for n, (ta, tb, M, N, K, al, be) in enumerate(SHAPES):
        sa = (M, K) if ta == "N" else (K, M)
        sb = (K, N) if tb == "N" else (N, K)
        A = pinned_from(seed + n, 0, *sa, kind) if K else pinned(*((M, 1) if ta == "N" else (1, M)))
        B = pinned_from(seed + n, 1, *sb, kind) if K else pinned(*((1, N) if tb == "N" else (N, 1)))
        C = pinned_from(seed + n, 2, M, N, kind)
        probs.append((ta, tb, M, N, K, al, be, A, B, C, np64(C)))
    return probs


def _descs(ooc, probs):
    out = []
    for ta, tb, M, N, K, al, be, A, B, C, _ in probs:
        d = ooc.ooc_gemm_desc()
        d.transA, d.transB = ta.encode(), tb.encode()
        d.M, d.N, d.K, d.alpha, d.beta = M, N, K, al, be
        d.A, d.lda = A.data_ptr(), (A.stride(0) if A.shape[0] > 1 else A.shape[1])
        d.B, d.ldb = B.data_ptr(), (B.stride(0) if B.shape[0] > 1 else B.shape[1])
        d.C, d.ldc = C.data_ptr(), N
        out.append(d)
    return out


@pytest.mark.parametrize("flags", [0, 2])
def test_batched_fp64_uneven(ooc, flags):
    probs = _problems(60)
    st = ooc.ooc_stats()
    rc = ooc.ooc_dgemm_batched(_descs(ooc, probs), 6 << 20, ooc.make_opts(flags=flags), st)
    assert rc == 0, ooc.ooc_last_error()
    assert st.steps >= len(SHAPES) and st.kernel_launches >= st.steps - 1
    for ta, tb, M, N, K, al, be, A, B, C, C0 in probs:
        ref = oracle.gemm(ta, tb, al, np64(A), np64(B), be, C0) if K else be * C0
        assert oracle.rel_fro(np64(C), ref) <= 1e-13, (ta, tb, M, N, K)


def test_batched_ozaki(ooc):
    probs = _problems(70, synth.LOGSPREAD)[:4]
    st = ooc.ooc_stats()
    rc = ooc.ooc_dgemm_batched(_descs(ooc, probs), 64 << 20, ooc.make_opts(form=ooc.OOC_FORM_OZAKI), st)
    assert rc == 0, ooc.ooc_last_error()
    for ta, tb, M, N, K, al, be, A, B, C, C0 in probs:
        ref = oracle.gemm(ta, tb, al, np64(A), np64(B), be, C0)
        assert oracle.rel_fro(np64(C), ref) <= 1e-12


def test_batched_empty_and_errors(ooc):
    assert ooc.ooc_dgemm_batched([], 1 << 20) == 0
    A = np.ones((8, 8))  # not pinned
    d = ooc.ooc_gemm_desc()
    d.transA = d.transB = b"N"
    d.M = d.N = d.K = 8
    d.alpha = 1.0
    d.A = d.B = d.C = A.ctypes.data
    d.lda = d.ldb = d.ldc = 8
    assert ooc.ooc_dgemm_batched([d], 1 << 20) == ooc.OOC_ERR_NOT_PINNED


@pytest.mark.parametrize("flags", [0, 2])
def test_batched_grouped_path(ooc, flags):
    """Every problem fits whole in half the budget: the grouped path (one persistent launch per
    group of problems, whole-matrix copies), with and without CUDA-graph capture; all transpose
    pairs (a group per change of pair), K = 0, beta = 0 with NaN in C, ragged tiles."""
    probs = _problems(80)
    for n in (1, 3):   # beta = 0 problems: C is never read
        probs[n][9].fill_(float("nan"))
    st = ooc.ooc_stats()
    rc = ooc.ooc_dgemm_batched(_descs(ooc, probs), 256 << 20, ooc.make_opts(flags=flags), st)
    assert rc == 0, ooc.ooc_last_error()
    assert st.blocks == len(SHAPES)
    assert 1 <= st.steps < len(SHAPES)          # groups, not problems
    assert st.kernel_launches == st.steps
    for ta, tb, M, N, K, al, be, A, B, C, C0 in probs:
        ref = oracle.gemm(ta, tb, al, np64(A), np64(B), be, None if be == 0 else C0) if K else be * C0
        assert oracle.rel_fro(np64(C), ref) <= 1e-13, (ta, tb, M, N, K)


def test_batched_grouped_matches_streamed(ooc):
    """The same batch through the grouped path and through one pipeline per problem."""
    shapes = [("N", "N", 520 + 37 * q, 300 + 53 * q, 64 + 91 * q, 1.0, 0.5) for q in range(12)]
    outs = []
    for flags in (0, ooc.OOC_BATCH_STREAMED):
        probs = []
        for n, (ta, tb, M, N, K, al, be) in enumerate(shapes):
            A = pinned_from(90 + n, 0, M, K, synth.INTEGER, 30)
            B = pinned_from(90 + n, 1, K, N, synth.INTEGER, 30)
            C = pinned_from(90 + n, 2, M, N, synth.INTEGER, 30)
            probs.append((ta, tb, M, N, K, al, be, A, B, C, np64(C)))
        st = ooc.ooc_stats()
        rc = ooc.ooc_dgemm_batched(_descs(ooc, probs), 64 << 20, ooc.make_opts(flags=flags), st)
        assert rc == 0, ooc.ooc_last_error()
        outs.append([np64(p[9]) for p in probs])
        for ta, tb, M, N, K, al, be, A, B, C, C0 in probs:
            assert np.array_equal(np64(C), oracle.gemm(ta, tb, al, np64(A), np64(B), be, C0))  # integers: exact
    for a, b in zip(*outs):
        assert np.array_equal(a, b)
