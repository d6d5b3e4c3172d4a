"""GPU parity of the two tensor-core forms against the CPU FP64 oracle.

BF16x3 (ooc_sgemm): FP32 operands, FP32-accurate: relative Frobenius error
<= 1e-6 against the FP64 product of the FP32 inputs.  Inputs exactly
representable in bf16 with small integer values are reproduced exactly.

Ozaki (ooc_dgemm, OOC_FORM_OZAKI): FP64 operands, FP64-accurate: relative
Frobenius error <= 1e-12 against the FP64 oracle, on inputs with a 10^8
exponent spread (sign * 10^U(-4,4)).  Small-integer inputs are exact (their
digits are exact and every digit product sums exactly in FP32).

Besides the norm, every result is checked element by element against the bound each form's
arithmetic gives (tests/bounds.py): BF16x3 relative to (|A||B|)_ij, Ozaki relative to the
operand rows' and columns' largest entries (its digits are cut from each row's fixed-point
value), so a wrong small entry cannot hide behind the large ones that dominate the norm.
"""
import itertools

import numpy as np
import pytest
import torch

import oracle
import synth
from bounds import bf16x3_bound, op, ozaki_bound, worst_ratio
from gpu_util import np64, pinned, pinned_from

pytestmark = pytest.mark.gpu
TOL_BF16X3 = 1e-6
TOL_OZAKI = 1e-12
OZAKI_DIGITS = 8   # the GEMM entry points' default digit count


def _elementwise(ooc, form, got, ref, A, B, ta, tb, alpha, beta, C0, kchunks=1, S=OZAKI_DIGITS):
    Aop, Bop = op(np64(A), ta), op(np64(B), tb)
    if form == ooc.OOC_FORM_BF16X3:
        bound = bf16x3_bound(Aop, Bop, alpha, beta, C0, kchunks)
    else:
        bound = ozaki_bound(Aop, Bop, alpha, beta, C0, S, kchunks)
    r = worst_ratio(got, ref, bound)
    assert r <= 1.0, "elementwise error %.3g x its bound" % r


def _run(ooc, form, ta, tb, M, N, K, alpha, beta, kind, param=0.0, budget=1 << 30, seed=40, c_nan=False):
    fp32 = form == ooc.OOC_FORM_BF16X3
    dt = torch.float32 if fp32 else torch.float64
    sa = (M, K) if ta == "N" else (K, M)
    sb = (K, N) if tb == "N" else (N, K)
    A = pinned_from(seed, 0, *sa, kind, param, dtype=dt)
    B = pinned_from(seed, 1, *sb, kind, param, dtype=dt)
    if c_nan:
        C = pinned(M, N, dtype=dt, fill=float("nan"))
    else:
        C = pinned_from(seed, 2, M, N, kind, param, dtype=dt)
    C0 = np64(C)
    st = ooc.ooc_stats()
    opts = ooc.make_opts(form=form)
    f = ooc.ooc_sgemm if fp32 else ooc.ooc_dgemm
    rc = f(ta, tb, M, N, K, alpha, A, sa[1], B, sb[1], beta, C, N, budget, opts, st)
    assert rc == 0, ooc.ooc_last_error()
    ref = oracle.gemm(ta, tb, alpha, np64(A), np64(B), beta, None if beta == 0 else C0)
    got = np64(C)
    if kind != synth.INTEGER:
        _elementwise(ooc, form, got, ref, A, B, ta, tb, alpha, beta, None if beta == 0 else C0,
                     kchunks=max(1, -(-K // st.kb)) if st.kb else 1)
    return got, ref, st


@pytest.mark.parametrize("ta,tb", list(itertools.product("NT", "NT")))
def test_bf16x3_transposes_ragged(ooc, ta, tb):
    got, ref, _ = _run(ooc, ooc.OOC_FORM_BF16X3, ta, tb, 300, 200, 170, 1.5, 0.5, synth.UNIFORM)
    assert oracle.rel_fro(got, ref) <= TOL_BF16X3


def test_bf16x3_small_config_many_blocks(ooc):
    # 1024^3, U[-1,1], alpha 1 beta 1, budget forcing several blocks
    got, ref, st = _run(ooc, ooc.OOC_FORM_BF16X3, "N", "N", 1024, 1024, 1024, 1.0, 1.0, synth.UNIFORM,
                        budget=8 << 20)
    assert st.blocks > 1 and st.products == 6
    assert oracle.rel_fro(got, ref) <= TOL_BF16X3


def test_bf16x3_long_k(ooc):
    got, ref, _ = _run(ooc, ooc.OOC_FORM_BF16X3, "N", "N", 256, 256, 20000, 1.0, 0.0, synth.UNIFORM)
    assert oracle.rel_fro(got, ref) <= TOL_BF16X3


def test_bf16x3_integers_exact(ooc):
    got, ref, _ = _run(ooc, ooc.OOC_FORM_BF16X3, "N", "T", 257, 129, 300, 1.0, 1.0, synth.INTEGER, 100)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("ta,tb", list(itertools.product("NT", "NT")))
def test_ozaki_transposes_ragged_spread(ooc, ta, tb):
    got, ref, st = _run(ooc, ooc.OOC_FORM_OZAKI, ta, tb, 300, 200, 170, 1.5, 0.5, synth.LOGSPREAD)
    assert st.form == ooc.OOC_FORM_OZAKI
    assert oracle.rel_fro(got, ref) <= TOL_OZAKI


def test_ozaki_spread_many_blocks_long_k(ooc):
    got, ref, st = _run(ooc, ooc.OOC_FORM_OZAKI, "N", "N", 700, 600, 9000, 1.0, 0.0, synth.LOGSPREAD,
                        budget=64 << 20)
    assert st.steps > 1   # several C blocks or K chunks stream through the budget
    assert oracle.rel_fro(got, ref) <= TOL_OZAKI


def test_ozaki_normal_inputs(ooc):
    got, ref, _ = _run(ooc, ooc.OOC_FORM_OZAKI, "N", "N", 512, 384, 2048, 1.5, 0.5, synth.NORMAL)
    assert oracle.rel_fro(got, ref) <= TOL_OZAKI


def test_ozaki_integers_exact(ooc):
    got, ref, _ = _run(ooc, ooc.OOC_FORM_OZAKI, "T", "N", 200, 300, 1000, 2.0, -1.0, synth.INTEGER, 1000)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("form", [3, 2])
def test_forms_beta_zero_ignores_nan(ooc, form):
    got, ref, _ = _run(ooc, form, "N", "N", 130, 250, 90, 1.0, 0.0, synth.UNIFORM, c_nan=True)
    assert np.isfinite(got).all()
    assert oracle.rel_fro(got, ref) <= (TOL_BF16X3 if form == 3 else TOL_OZAKI)


@pytest.mark.parametrize("form", [3, 2])
def test_forms_k_zero(ooc, form):
    fp32 = form == 3
    dt = torch.float32 if fp32 else torch.float64
    M, N = 77, 45
    A = pinned(M, 1, dtype=dt)
    B = pinned(1, N, dtype=dt)
    C = pinned_from(6, 2, M, N, synth.INTEGER, 50, dtype=dt)
    C0 = np64(C)
    f = ooc.ooc_sgemm if fp32 else ooc.ooc_dgemm
    rc = f("N", "N", M, N, 0, 1.0, A, 1, B, N, -2.0, C, N, 1 << 20, ooc.make_opts(form=form), None)
    assert rc == 0, ooc.ooc_last_error()
    assert np.array_equal(np64(C), -2.0 * C0)


@pytest.mark.parametrize("form", [3, 2])
def test_forms_with_k_chunks(ooc, form):
    """K streamed in chunks (the last one ragged): each chunk is split on its own and the partial
    results accumulate in C (FP32 for BF16x3, FP64 for Ozaki)."""
    fp32 = form == 3
    dt = torch.float32 if fp32 else torch.float64
    M, N, K = 300, 260, 1000
    kind = synth.UNIFORM if fp32 else synth.LOGSPREAD
    A = pinned_from(45, 0, M, K, kind, dtype=dt)
    B = pinned_from(45, 1, K, N, kind, dtype=dt)
    C = pinned_from(45, 2, M, N, kind, dtype=dt)
    C0 = np64(C)
    st = ooc.ooc_stats()
    f = ooc.ooc_sgemm if fp32 else ooc.ooc_dgemm
    rc = f("N", "N", M, N, K, 1.25, A, K, B, N, 0.5, C, N, 1 << 30, ooc.make_opts(form=form, kb=256, mb=128, nb=128),
           st)
    assert rc == 0, ooc.ooc_last_error()
    assert st.kb == 256 and st.steps == 3 * 3 * 4
    ref = oracle.gemm("N", "N", 1.25, np64(A), np64(B), 0.5, C0)
    assert oracle.rel_fro(np64(C), ref) <= (TOL_BF16X3 if fp32 else TOL_OZAKI)
    _elementwise(ooc, form, np64(C), ref, A, B, "N", "N", 1.25, 0.5, C0, kchunks=4)


@pytest.mark.parametrize("S", [9, 10])
def test_ozaki_more_digits(ooc, S):
    """opts->slices above the default: more digit planes and products, the bound shrinks by
    2^-6 per digit, and both checks still hold with it."""
    M, N, K = 260, 200, 300
    A = pinned_from(46, 0, M, K, synth.LOGSPREAD)
    B = pinned_from(46, 1, K, N, synth.LOGSPREAD)
    C = pinned_from(46, 2, M, N, synth.LOGSPREAD)
    C0 = np64(C)
    st = ooc.ooc_stats()
    rc = ooc.ooc_dgemm("N", "N", M, N, K, 1.0, A, K, B, N, -1.0, C, N, 1 << 30,
                       ooc.make_opts(form=ooc.OOC_FORM_OZAKI, slices=S), st)
    assert rc == 0, ooc.ooc_last_error()
    assert st.slices == S and st.products == S * (S + 1) // 2
    ref = oracle.gemm("N", "N", 1.0, np64(A), np64(B), -1.0, C0)
    assert oracle.rel_fro(np64(C), ref) <= TOL_OZAKI
    _elementwise(ooc, ooc.OOC_FORM_OZAKI, np64(C), ref, A, B, "N", "N", 1.0, -1.0, C0, S=S)


def test_ozaki_bad_digit_count(ooc):
    A = pinned(8, 8, fill=1.0)
    C = pinned(8, 8, fill=0.0)
    for S in (1, 11):
        rc = ooc.ooc_dgemm("N", "N", 8, 8, 8, 1.0, A, 8, A, 8, 0.0, C, 8, 1 << 20,
                           ooc.make_opts(form=ooc.OOC_FORM_OZAKI, slices=S), None)
        assert rc == ooc.OOC_ERR_INVALID_ARG


@pytest.mark.parametrize("form", ["bf16x3", "ozaki", "fp64"])
def test_split_kernel_time_reported(ooc, form):
    """stats.split_seconds is the split kernels' share of kernel_seconds: positive and below
    it for the split forms, zero for FP64 (no split kernels)."""
    f = {"bf16x3": ooc.OOC_FORM_BF16X3, "ozaki": ooc.OOC_FORM_OZAKI, "fp64": ooc.OOC_FORM_FP64}[form]
    _, _, st = _run(ooc, f, "N", "N", 700, 600, 900, 1.0, 0.0, synth.UNIFORM, budget=8 << 20)
    assert st.kernel_seconds > 0
    if form == "fp64":
        assert st.split_seconds == 0.0
    else:
        assert 0.0 < st.split_seconds < st.kernel_seconds
