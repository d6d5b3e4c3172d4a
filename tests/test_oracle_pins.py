"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Section IV fixes what is computed: C = alpha*A*B + beta*C.  The checks below do
not re-type the oracle's loop: they use exact rational arithmetic, closed forms
(identity, rank-1, diagonal scaling), the alpha/beta invariants, and numpy's
BLAS product as an independent library routine.
"""
from fractions import Fraction
import itertools

import numpy as np
import pytest

import oracle
import synth

TRANS = list(itertools.product("NT", "NT"))


def _stored(x, t):
    """The stored operand whose op(.) is x (row-major copy)."""
    return np.ascontiguousarray(x.T if t == "T" else x)


def _exact(alpha, A, B, beta, C):
    M, K = A.shape
    N = B.shape[1]
    out = []
    for i in range(M):
        row = []
        for j in range(N):
            s = sum((Fraction(float(A[i, k])) * Fraction(float(B[k, j])) for k in range(K)),
                    Fraction(0))
            v = Fraction(alpha) * s
            if beta != 0:
                v += Fraction(beta) * Fraction(float(C[i, j]))
            row.append(v)
        out.append(row)
    return out


@pytest.mark.parametrize("ta,tb", TRANS)
@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (3, 5, 2), (6, 4, 7), (5, 6, 6), (2, 7, 1)])
def test_exact_rationals_tiny(ta, tb, M, N, K):
    # dyadic entries k/256 with |k| <= 64: every product and partial sum is exact in FP64
    A = synth.matrix(M, K, 7, 0, synth.DYADIC, 64)
    B = synth.matrix(K, N, 7, 1, synth.DYADIC, 64)
    C = synth.matrix(M, N, 7, 2, synth.DYADIC, 64)
    alpha, beta = 1.5, -0.75
    got = oracle.gemm(ta, tb, alpha, _stored(A, ta), _stored(B, tb), beta, C)
    ref = _exact(alpha, A, B, beta, C)
    for i in range(M):
        for j in range(N):
            assert Fraction(float(got[i, j])) == ref[i][j], (i, j)


def test_identity_closed_form():
    n, N = 9, 11
    I = np.eye(n)
    B = synth.matrix(n, N, 3, 1, synth.DYADIC, 100)
    C = synth.matrix(n, N, 3, 2, synth.DYADIC, 100)
    got = oracle.gemm("N", "N", 2.0, I, B, 0.5, C)
    assert np.array_equal(got, 2.0 * B + 0.5 * C)
    # identity on the right
    A = synth.matrix(N, n, 3, 3, synth.DYADIC, 100)
    C2 = synth.matrix(N, n, 3, 4, synth.DYADIC, 100)
    got = oracle.gemm("N", "N", -1.0, A, I, 0.25, C2)
    assert np.array_equal(got, -A + 0.25 * C2)


@pytest.mark.parametrize("ta,tb", TRANS)
def test_rank1_closed_form(ta, tb):
    M, N = 13, 9
    u = synth.matrix(M, 1, 4, 0, synth.DYADIC, 50)
    v = synth.matrix(1, N, 4, 1, synth.DYADIC, 50)
    C = synth.matrix(M, N, 4, 2, synth.DYADIC, 50)
    got = oracle.gemm(ta, tb, 3.0, _stored(u, ta), _stored(v, tb), -2.0, C)
    assert np.array_equal(got, 3.0 * np.multiply.outer(u[:, 0], v[0, :]) - 2.0 * C)


def test_diagonal_scaling_invariant():
    # (D1 A)(B D2) = D1 (A B) D2 exactly when D1, D2 hold powers of two
    M, N, K = 10, 12, 8
    A = synth.matrix(M, K, 5, 0, synth.NORMAL)
    B = synth.matrix(K, N, 5, 1, synth.NORMAL)
    d1 = 2.0 ** np.arange(-4, M - 4)
    d2 = 2.0 ** np.arange(3, 3 - N, -1)
    base = oracle.gemm("N", "N", 1.0, A, B, 0.0, None)
    got = oracle.gemm("N", "N", 1.0, d1[:, None] * A, B * d2[None, :], 0.0, None)
    assert np.array_equal(got, d1[:, None] * base * d2[None, :])


def test_beta_zero_ignores_nan_c():
    M, N, K = 7, 5, 6
    A = synth.matrix(M, K, 6, 0, synth.UNIFORM)
    B = synth.matrix(K, N, 6, 1, synth.UNIFORM)
    C = np.full((M, N), np.nan)
    got = oracle.gemm("N", "N", 1.0, A, B, 0.0, C)
    assert np.isfinite(got).all()
    np.testing.assert_allclose(got, A @ B, rtol=1e-14, atol=1e-15)


def test_alpha_zero_gives_beta_c():
    M, N, K = 6, 8, 5
    A = synth.matrix(M, K, 8, 0, synth.NORMAL)
    B = synth.matrix(K, N, 8, 1, synth.NORMAL)
    C = synth.matrix(M, N, 8, 2, synth.NORMAL)
    assert np.array_equal(oracle.gemm("N", "N", 0.0, A, B, 0.5, C), 0.5 * C)


def test_linear_in_alpha():
    M, N, K = 9, 7, 11
    A = synth.matrix(M, K, 9, 0, synth.NORMAL)
    B = synth.matrix(K, N, 9, 1, synth.NORMAL)
    r1 = oracle.gemm("N", "N", 1.0, A, B, 0.0, None)
    r4 = oracle.gemm("N", "N", 4.0, A, B, 0.0, None)
    rm = oracle.gemm("N", "N", -0.5, A, B, 0.0, None)
    assert np.array_equal(r4, 4.0 * r1)
    assert np.array_equal(rm, -0.5 * r1)


def test_k_zero_gives_beta_c():
    C = synth.matrix(4, 3, 10, 2, synth.NORMAL)
    got = oracle.gemm("N", "N", 2.0, np.zeros((4, 0)), np.zeros((0, 3)), -3.0, C)
    assert np.array_equal(got, -3.0 * C)


@pytest.mark.parametrize("ta,tb", TRANS)
def test_matches_blas_random(ta, tb):
    M, N, K = 67, 45, 130
    A = synth.matrix(M, K, 11, 0, synth.NORMAL)
    B = synth.matrix(K, N, 11, 1, synth.NORMAL)
    C = synth.matrix(M, N, 11, 2, synth.NORMAL)
    got = oracle.gemm(ta, tb, 1.5, _stored(A, ta), _stored(B, tb), 0.5, C)
    ref = 1.5 * (A @ B) + 0.5 * C
    assert oracle.rel_fro(got, ref) < 1e-14


def test_leading_dimension_padding_not_read():
    M, N, K = 8, 6, 5
    A = synth.matrix(M, K, 12, 0, synth.UNIFORM)
    B = synth.matrix(K, N, 12, 1, synth.UNIFORM)
    Ap = np.full((M, K + 3), np.nan); Ap[:, :K] = A
    Bp = np.full((K, N + 5), np.nan); Bp[:, :N] = B
    got, _ = oracle.gemm_block("N", "N", 0, 0, M, N, K, 1.0, Ap[:, :K], Bp[:, :N], 0.0, None)
    assert np.array_equal(got, oracle.gemm("N", "N", 1.0, A, B, 0.0, None))


def test_fp32_inputs_are_widened():
    M, N, K = 20, 30, 40
    A = synth.matrix(M, K, 13, 0, synth.UNIFORM, dtype=np.float32)
    B = synth.matrix(K, N, 13, 1, synth.UNIFORM, dtype=np.float32)
    C = synth.matrix(M, N, 13, 2, synth.UNIFORM)
    got = oracle.gemm("N", "N", 1.0, A, B, 1.0, C)
    ref = A.astype(np.float64) @ B.astype(np.float64) + C
    assert oracle.rel_fro(got, ref) < 1e-14


def test_block_mode_matches_whole_and_threads_do_not_change_bits():
    M, N, K = 40, 33, 21
    A = synth.matrix(M, K, 14, 0, synth.NORMAL)
    B = synth.matrix(K, N, 14, 1, synth.NORMAL)
    C = synth.matrix(M, N, 14, 2, synth.NORMAL)
    whole = oracle.gemm("N", "N", 1.5, A, B, 0.5, C, nthreads=1)
    whole7 = oracle.gemm("N", "N", 1.5, A, B, 0.5, C, nthreads=7)
    assert np.array_equal(whole, whole7)
    blk, _ = oracle.gemm_block("N", "N", 9, 4, 17, 20, K, 1.5, A, B, 0.5, C[9:26, 4:24])
    assert np.array_equal(blk, whole[9:26, 4:24])


def test_generator_known_answers():
    # Philox4x32-10 known-answer vectors published with the Random123 library (Salmon et al. 2011)
    assert synth.philox4x32_10([0, 0, 0, 0], [0, 0]) == [0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8]
    assert synth.philox4x32_10([0xffffffff] * 4, [0xffffffff] * 2) == [
        0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd]
    assert synth.philox4x32_10([0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344],
                               [0xa4093822, 0x299f31d0]) == [0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1]


def test_generator_distributions_and_ld_independence():
    a = synth.matrix(400, 500, 1, 0, synth.NORMAL)
    assert abs(a.mean()) < 0.01 and abs(a.std() - 1.0) < 0.01
    u = synth.matrix(400, 500, 1, 0, synth.UNIFORM)
    assert u.min() >= -1.0 and u.max() < 1.0 and abs(u.mean()) < 0.01
    g = synth.matrix(400, 500, 1, 0, synth.LOGSPREAD)
    lg = np.log10(np.abs(g))
    assert lg.min() >= -4.0 and lg.max() <= 4.0 and abs(lg.mean()) < 0.05
    assert 0.45 < (g > 0).mean() < 0.55
    wide = np.zeros((400, 512))
    synth.fill(wide[:, :500], 1, 0, synth.NORMAL)
    assert np.array_equal(wide[:, :500], a)
