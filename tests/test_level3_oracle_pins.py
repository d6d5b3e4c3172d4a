"""Pins of the level-3 oracle (oracle/level3.py, oracle/factor.c) against
exact arithmetic, closed forms and invariants -- nothing here re-calls the
oracle's own arithmetic as the expected value.

SYRK/GEMMT: brute force in exact rationals on dyadic inputs (FP64 exact).
TRSM: integer solutions X with power-of-two diagonals, B = op(A) X formed
with Python integers, so the substitution must return X exactly; NaN planted
in the unread triangle (and on a unit diagonal) must not reach the result.
POTRF: A = L L^T from an integer L with positive integer diagonal, formed with
Python integers, must give back L exactly; non-positive pivots give info.
"""
import itertools
import zlib
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import level3


def dyadic(rng, shape, lo=-8, hi=8, den=4):
    return rng.integers(lo, hi + 1, size=shape).astype(np.float64) / den


@pytest.mark.parametrize("uplo,trans", list(itertools.product("LU", "NT")))
def test_syrk_brute_force_rationals(uplo, trans):
    rng = np.random.default_rng(7)
    N, K = 5, 4
    A = dyadic(rng, (N, K) if trans == "N" else (K, N))
    C = dyadic(rng, (N, N))
    alpha, beta = 0.75, -1.5
    got = level3.syrk(uplo, trans, alpha, A, beta, C)
    opA = [[Fraction(A[i, k] if trans == "N" else A[k, i]) for k in range(K)] for i in range(N)]
    for i in range(N):
        for j in range(N):
            upd = (j <= i) if uplo == "L" else (j >= i)
            if upd:
                s = sum(opA[i][k] * opA[j][k] for k in range(K))
                want = Fraction(alpha) * s + Fraction(beta) * Fraction(C[i, j])
                assert Fraction(got[i, j]) == want
            else:
                assert got[i, j] == C[i, j]


def test_gemmt_brute_force_and_untouched_triangle():
    rng = np.random.default_rng(8)
    N, K = 6, 3
    A = dyadic(rng, (K, N))    # transA 'T'
    B = dyadic(rng, (K, N))    # transB 'N'
    C = dyadic(rng, (N, N))
    C[np.triu_indices(N, 1)] = np.nan   # never read by uplo 'L'
    got = level3.gemmt("L", "T", "N", 2.0, A, B, 0.5, C)
    for i in range(N):
        for j in range(N):
            if j <= i:
                s = sum(Fraction(A[k, i]) * Fraction(B[k, j]) for k in range(K))
                assert Fraction(got[i, j]) == 2 * s + Fraction(1, 2) * Fraction(C[i, j])
            else:
                assert np.isnan(got[i, j])


def test_syrk_beta_zero_ignores_nan_and_identity_closed_form():
    N = 7
    C = np.full((N, N), np.nan)
    got = level3.syrk("U", "N", 3.0, np.eye(N), 0.0, C)
    assert np.array_equal(np.triu(got), 3.0 * np.eye(N))     # A = I: alpha I on the updated triangle
    assert np.isnan(got[np.tril_indices(N, -1)]).all()       # the other triangle is kept (NaN stays)


def test_syrk_lower_is_transposed_upper():
    rng = np.random.default_rng(9)
    A = rng.standard_normal((40, 23))
    S = rng.standard_normal((40, 40))
    S = S + S.T
    lo = level3.syrk("L", "N", 1.25, A, 0.5, S)
    up = level3.syrk("U", "N", 1.25, A, 0.5, S)
    assert np.array_equal(np.tril(lo), np.tril(up.T))


def test_syrk_block_matches_whole_syrk_on_a_straddling_block():
    rng = np.random.default_rng(10)
    A = rng.standard_normal((50, 17))
    C = rng.standard_normal((50, 50))
    whole = level3.syrk("L", "N", 1.0, A, 2.0, C)
    blk = level3.syrk_block("L", "N", 10, 20, 15, 12, 1.0, A, 2.0, C[10:25, 20:32])
    assert np.array_equal(blk, whole[10:25, 20:32])


def _tri_int(rng, n, uplo, unit, nan_other):
    """Integer triangular A (stored), power-of-two diagonal (or NaN when unit)."""
    A = rng.integers(-3, 4, size=(n, n)).astype(np.float64)
    d = rng.choice([-4.0, -2.0, -1.0, 1.0, 2.0, 4.0], size=n)
    A[np.diag_indices(n)] = np.nan if unit else d
    other = np.triu_indices(n, 1) if uplo == "L" else np.tril_indices(n, -1)
    A[other] = np.nan if nan_other else 0.0
    return A


@pytest.mark.parametrize("side,uplo,ta,diag", list(itertools.product("LR", "LU", "NT", "NU")))
def test_trsm_recovers_integer_solutions_exactly(side, uplo, ta, diag):
    rng = np.random.default_rng(zlib.crc32((side + uplo + ta + diag).encode()))
    M, N = (9, 5) if side == "L" else (5, 9)
    n = M if side == "L" else N
    A = _tri_int(rng, n, uplo, diag == "U", nan_other=True)
    # the triangular matrix the solve sees, as Python integers
    T = [[0] * n for _ in range(n)]
    for r in range(n):
        for c in range(n):
            if r == c:
                T[r][c] = 1 if diag == "U" else int(A[r, c])
            elif (c < r) if uplo == "L" else (c > r):
                T[r][c] = int(A[r, c])
    opT = T if ta == "N" else [list(x) for x in zip(*T)]
    X = rng.integers(-5, 6, size=(M, N))
    # solution X scaled so that every division by the power-of-two diagonal stays exact
    X = X * 64
    if side == "L":
        Bi = [[sum(opT[i][k] * int(X[k, j]) for k in range(n)) for j in range(N)] for i in range(M)]
    else:
        Bi = [[sum(int(X[i, k]) * opT[k][j] for k in range(n)) for j in range(N)] for i in range(M)]
    B = np.array(Bi, dtype=np.float64) * 2.0       # alpha = 0.5 below
    got = level3.trsm(side, uplo, ta, diag, 0.5, A, B)
    assert np.array_equal(got, X.astype(np.float64))


def test_trsm_identity_and_diagonal_closed_forms():
    rng = np.random.default_rng(3)
    B = rng.standard_normal((6, 4))
    assert np.array_equal(level3.trsm("L", "L", "N", "N", 1.5, np.eye(6), B), 1.5 * B)
    D = np.diag([2.0, 4.0, 0.5, 8.0])
    assert np.array_equal(level3.trsm("R", "U", "T", "N", 1.0, D, B), B / np.diag(D)[None, :])


def _spd_from_int_factor(rng, n):
    L = np.tril(rng.integers(-3, 4, size=(n, n))).astype(np.int64)
    L[np.diag_indices(n)] = rng.integers(1, 4, size=n)
    Li = [[int(x) for x in row] for row in L]
    A = [[sum(Li[i][k] * Li[j][k] for k in range(n)) for j in range(n)] for i in range(n)]
    return np.array(A, dtype=np.float64), L.astype(np.float64)


@pytest.mark.parametrize("uplo", "LU")
def test_potrf_recovers_integer_factor_exactly(uplo):
    rng = np.random.default_rng(11)
    n = 12
    A, L = _spd_from_int_factor(rng, n)
    A_in = A.copy()
    other = np.triu_indices(n, 1) if uplo == "L" else np.tril_indices(n, -1)
    A_in[other] = np.nan
    F, info = level3.potrf(uplo, A_in)
    assert info == 0
    if uplo == "L":
        assert np.array_equal(np.tril(np.nan_to_num(F)), L)
    else:
        assert np.array_equal(np.triu(np.nan_to_num(F)), L.T)
    assert np.isnan(F[other]).all()


def test_potrf_two_by_two_closed_form_and_info():
    F, info = level3.potrf("L", np.array([[4.0, 2.0], [2.0, 5.0]]))
    assert info == 0 and np.array_equal(np.tril(F), [[2.0, 0.0], [1.0, 2.0]])
    _, info = level3.potrf("L", np.diag([1.0, -1.0, 1.0]))
    assert info == 2
    _, info = level3.potrf("U", np.array([[1.0, 2.0], [2.0, 4.0]]))  # singular: second pivot 0
    assert info == 2


def test_potrf_residual_on_a_random_spd_matrix():
    rng = np.random.default_rng(12)
    n = 200
    G = rng.standard_normal((n, n))
    A = G @ G.T + n * np.eye(n)
    F, info = level3.potrf("L", A)
    L = np.tril(F)
    assert info == 0
    assert np.linalg.norm(L @ L.T - A) / np.linalg.norm(A) < 1e-14
    assert (np.diag(L) > 0).all()


# ---- GETRF (LU with partial pivoting) ------------------------------------
def _lu_from_factors(rng, n):
    """A = P L U with dyadic |l| <= 1/2 (unit diagonal) and integer U with a large
    diagonal: each step's pivot is unique (the row whose l is 1) and every
    operation is exact in FP64.  Returns A, L, U, the row order of A."""
    L = np.tril(rng.choice([-0.5, -0.25, 0.0, 0.25, 0.5], size=(n, n)), -1) + np.eye(n)
    U = np.triu(rng.integers(-3, 4, size=(n, n))).astype(np.float64)
    U[np.diag_indices(n)] = rng.choice([-8.0, -6.0, 6.0, 8.0], size=n)
    LU = [[sum(Fraction(L[i, k]) * Fraction(U[k, j]) for k in range(n)) for j in range(n)] for i in range(n)]
    order = rng.permutation(n)
    A = np.empty((n, n))
    for i in range(n):
        A[order[i]] = [float(x) for x in LU[i]]   # row i of L U sits at row order[i] of A
    return A, L, U


def test_getrf_recovers_exact_factors():
    rng = np.random.default_rng(21)
    n = 14
    A, L, U = _lu_from_factors(rng, n)
    F, ipiv, info = level3.getrf(A)
    assert info == 0
    assert np.array_equal(np.tril(F, -1) + np.eye(n), L)
    assert np.array_equal(np.triu(F), U)
    # the exchanges put the rows of A in the order of L U
    assert np.array_equal(level3.apply_pivots(A, ipiv), L @ U)


def test_getrf_closed_forms_ties_and_zero_pivots():
    F, ipiv, info = level3.getrf(np.array([[1.0, 2.0], [4.0, 4.0]]))
    assert info == 0 and list(ipiv) == [1, 1]
    assert np.array_equal(F, [[4.0, 4.0], [0.25, 1.0]])       # l = 1/4, u22 = 2 - 4/4
    F, ipiv, _ = level3.getrf(np.array([[2.0, 1.0], [-2.0, 3.0]]))
    assert list(ipiv) == [0, 1]                                # ties go to the first row
    _, ipiv, info = level3.getrf(np.array([[0.0, 0.0], [0.0, 1.0]]))
    assert info == 1 and list(ipiv) == [0, 1]                  # zero column: no exchange, info set


def test_getrf_residual_and_multiplier_bound_on_random_input():
    rng = np.random.default_rng(22)
    n = 300
    A = rng.standard_normal((n, n))
    F, ipiv, info = level3.getrf(A)
    L = np.tril(F, -1) + np.eye(n)
    U = np.triu(F)
    assert info == 0
    assert np.abs(np.tril(F, -1)).max() <= 1.0                  # partial pivoting: |l| <= 1
    assert np.linalg.norm(level3.apply_pivots(A, ipiv) - L @ U) / np.linalg.norm(A) < 1e-13
