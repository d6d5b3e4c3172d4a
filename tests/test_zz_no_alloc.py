"""GPU test of ooc_dgemm_noalloc, the entry point for callers that cannot allocate
device memory (its buffers live in a fixed device array inside the library).

It is checked against ooc_dgemm, the allocating entry point, on the same pinned
inputs, within the plain FP64 tolerance of the other GPU tests, on two calls in a
row (the second reuses the array the first call left behind).  This file is
collected last so that a run stopping at the first failure has run every other
test first.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import np64, pinned, pinned_from

pytestmark = pytest.mark.gpu
TOL = 1e-13


def _pair(ooc, seed, ta, tb, M, N, K, alpha, beta, budget, stream=None):
    sa = (M, K) if ta == "N" else (K, M)
    sb = (K, N) if tb == "N" else (N, K)
    A = pinned_from(seed, 0, *sa, synth.NORMAL)
    B = pinned_from(seed, 1, *sb, synth.NORMAL)
    C1 = pinned_from(seed, 2, M, N, synth.NORMAL)
    C2 = pinned(M, N)
    C2.copy_(C1)
    C0 = np64(C1)
    rc = ooc.ooc_dgemm(ta, tb, M, N, K, alpha, A, sa[1], B, sb[1], beta, C1, N, budget)
    assert rc == 0, ooc.ooc_last_error()
    rc = ooc.ooc_dgemm_noalloc(ta, tb, M, N, K, alpha, A, sa[1], B, sb[1], beta, C2, N, budget, stream)
    assert rc == 0, ooc.ooc_last_error()
    return np64(C1), np64(C2), oracle.gemm(ta, tb, alpha, np64(A), np64(B), beta, C0)


def test_noalloc_matches_allocating_entry_on_two_calls_in_a_row(ooc):
    # first call: beta != 0, transposed B, a budget far below the problem
    ref1, got1, ora1 = _pair(ooc, 31, "N", "T", 700, 520, 390, 1.5, 0.5, 1 << 20)
    assert oracle.rel_fro(got1, ref1) <= TOL
    assert oracle.rel_fro(got1, ora1) <= TOL
    # second call right after: different shape, beta == 0, larger budget
    ref2, got2, ora2 = _pair(ooc, 32, "T", "N", 1024, 1024, 1024, -1.0, 0.0, 8 << 20)
    assert oracle.rel_fro(got2, ref2) <= TOL
    assert oracle.rel_fro(got2, ora2) <= TOL


def test_noalloc_rejects_budget_above_its_array(ooc):
    A = pinned(8, 8, fill=1.0)
    B = pinned(8, 8, fill=1.0)
    C = pinned(8, 8, fill=0.0)
    rc = ooc.ooc_dgemm_noalloc("N", "N", 8, 8, 8, 1.0, A, 8, B, 8, 0.0, C, 8,
                               ooc.OOC_NOALLOC_MAX_BYTES + 1, None)
    assert rc == ooc.OOC_ERR_INVALID_ARG
    assert "exceeds" in ooc.ooc_last_error()


def test_noalloc_on_a_non_blocking_stream(ooc):
    """The stream argument is what sets this entry point apart: all its copies, kernels and
    the read of its error word run on the caller's stream.  Two calls in a row on a
    non-blocking stream (which does not synchronise with the legacy default stream); the
    error word the first call used must be cleared again for the second."""
    import torch
    s = torch.cuda.Stream()
    ref1, got1, ora1 = _pair(ooc, 33, "T", "T", 600, 300, 700, 0.5, -2.0, 2 << 20, stream=s.cuda_stream)
    assert oracle.rel_fro(got1, ref1) <= TOL
    assert oracle.rel_fro(got1, ora1) <= TOL
    ref2, got2, ora2 = _pair(ooc, 34, "N", "N", 257, 513, 1000, 1.0, 0.0, 4 << 20, stream=s.cuda_stream)
    assert oracle.rel_fro(got2, ref2) <= TOL
    assert oracle.rel_fro(got2, ora2) <= TOL
