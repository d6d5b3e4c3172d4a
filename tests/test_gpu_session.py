"""GPU parity of sessions (Section IV's nsteps mode: one C over several calls,
as in the steps of SUMMA) against the CPU oracle applied step by step:
C_1 = alpha_0 op(A_0) op(B_0) + beta C_0, C_{s+1} = alpha_s op(A_s) op(B_s) + C_s.

Budgets are chosen so that every C block, some of them, or none stays
resident in HBM between calls; the result must not depend on it.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import np64, pinned, pinned_from

pytestmark = pytest.mark.gpu
TOL = 1e-13

STEPS = [("N", "N", 100, 1.0), ("T", "N", 64, -0.5), ("N", "T", 130, 2.0), ("T", "T", 1, 1.0)]


def _panels(M, N, steps, seed):
    out = []
    for s, (ta, tb, K, alpha) in enumerate(steps):
        sa = (M, K) if ta == "N" else (K, M)
        sb = (K, N) if tb == "N" else (N, K)
        A = pinned_from(seed + s, 0, *sa, synth.NORMAL)
        B = pinned_from(seed + s, 1, *sb, synth.NORMAL)
        out.append((ta, tb, K, alpha, A, sa[1], B, sb[1]))
    return out


def _reference(C0, beta, panels):
    C = C0
    for s, (ta, tb, K, alpha, A, lda, B, ldb) in enumerate(panels):
        b = beta if s == 0 else 1.0
        C = oracle.gemm(ta, tb, alpha, np64(A), np64(B), b, None if b == 0.0 else C)
    return C


def _run(ooc, M, N, budget, beta=0.5, k_hint=256, opts=None, seed=110, c_nan=False):
    panels = _panels(M, N, STEPS, seed)
    C = pinned(M, N, fill=float("nan")) if c_nan else pinned_from(seed, 2, M, N, synth.NORMAL)
    C0 = np64(C)
    s = ooc.Session(M, N, C, N, beta, budget, k_hint=k_hint, opts=opts)
    assert s.rc == 0, ooc.ooc_last_error()
    info = s.query()
    for ta, tb, K, alpha, A, lda, B, ldb in panels:
        rc = s.step(ta, tb, K, alpha, A, lda, B, ldb)
        assert rc == 0, ooc.ooc_last_error()
    st = ooc.ooc_stats()
    assert s.finish(st) == 0, ooc.ooc_last_error()
    ref = _reference(C0, beta, panels)
    return np64(C), ref, info, st


@pytest.mark.parametrize("budget,blocking,resident", [(1 << 30, {}, "all"), (1 << 20, dict(mb=64, nb=64), "some"),
                                                       (700 << 10, {}, "none")])
def test_session_matches_stepwise_oracle(ooc, budget, blocking, resident):
    M, N = 500, 460
    got, ref, info, st = _run(ooc, M, N, budget, opts=ooc.make_opts(**blocking))
    if resident == "all":
        assert info["resident_blocks"] == info["blocks"]
    elif resident == "some":
        assert 0 < info["resident_blocks"] < info["blocks"]
    else:
        assert info["resident_blocks"] == 0
    assert oracle.rel_fro(got, ref) <= TOL
    # resident blocks cross the link twice at most (in once for beta, out once at the end)
    c_bytes = 8.0 * M * N
    if resident == "all":
        assert st.d2h_bytes == c_bytes


def test_session_beta_zero_ignores_nan(ooc):
    got, ref, _, _ = _run(ooc, 300, 200, 1 << 30, beta=0.0, c_nan=True)
    assert not np.isnan(got).any()
    assert oracle.rel_fro(got, ref) <= TOL


def test_session_without_steps_scales_c(ooc):
    M, N = 200, 150
    C = pinned_from(120, 2, M, N, synth.NORMAL)
    C0 = np64(C)
    s = ooc.Session(M, N, C, N, -2.0, 1 << 30)
    assert s.rc == 0
    assert s.finish() == 0, ooc.ooc_last_error()
    assert np.array_equal(np64(C), -2.0 * C0)


def test_session_ozaki_form(ooc):
    got, ref, info, st = _run(ooc, 400, 300, 64 << 20, opts=ooc.make_opts(form=ooc.OOC_FORM_OZAKI), seed=130)
    assert info["resident_blocks"] > 0
    assert oracle.rel_fro(got, ref) <= 1e-12


def test_session_integer_panels_exact(ooc):
    M, N = 256, 192
    panels = []
    for s in range(5):
        A = pinned_from(140 + s, 0, M, 96, synth.INTEGER, 256)
        B = pinned_from(140 + s, 1, 96, N, synth.INTEGER, 256)
        panels.append(("N", "N", 96, 1.0, A, 96, B, N))
    C = pinned_from(140, 2, M, N, synth.INTEGER, 256)
    C0 = np64(C)
    s = ooc.Session(M, N, C, N, 1.0, 2 << 20, k_hint=96)
    assert s.rc == 0
    for ta, tb, K, alpha, A, lda, B, ldb in panels:
        assert s.step(ta, tb, K, alpha, A, lda, B, ldb) == 0, ooc.ooc_last_error()
    assert s.finish() == 0
    assert np.array_equal(np64(C), _reference(C0, 1.0, panels))


def test_session_bad_arguments(ooc):
    C = pinned(8, 8)
    s = ooc.Session(8, 8, C, 4, 0.0, 1 << 20)
    assert s.rc == ooc.OOC_ERR_INVALID_ARG
    s = ooc.Session(8, 8, C, 8, 0.0, 1 << 20, opts=ooc.make_opts(form=ooc.OOC_FORM_BF16X3))
    assert s.rc == ooc.OOC_ERR_INVALID_ARG
    s = ooc.Session(8, 8, C, 8, 0.0, 1 << 20)
    assert s.rc == 0
    A = pinned(8, 8)
    assert s.step("X", "N", 8, 1.0, A, 8, A, 8) == ooc.OOC_ERR_INVALID_ARG
    s.free()
