"""Planted mistakes in the TRSM / POTRF oracle (oracle/factor.c): each plausible
slip must fail at least one pin of tests/test_level3_oracle_pins.py's kind.

The mistake is planted in a copy of factor.c, built with oracle.c into a
temporary library on the CPU; the committed oracle is never modified.
"""
import itertools
import os
import shutil
import subprocess
import zlib

import numpy as np
import pytest

import oracle
from oracle import level3

HERE = os.path.dirname(oracle.__file__)
FACTOR = os.path.join(HERE, "factor.c")

MUTANTS = {
    "trsm_order_swapped": ("const int forward = is_l(j->side) ? op_lower : !op_lower;",
                           "const int forward = is_l(j->side) ? !op_lower : op_lower;"),
    "trsm_alpha_dropped": ("const double rhs = j->alpha * base[t * step] - s;",
                           "const double rhs = base[t * step] - s;"),
    "trsm_unit_diagonal_ignored": ("base[t * step] = is_u(j->diag) ? rhs : rhs / opa(j, t, t);",
                                   "base[t * step] = rhs / j->A[t * j->lda + t];"),
    "trsm_coefficient_transposed": ("(is_l(j->side) ? opa(j, t, k) : opa(j, k, t))",
                                    "(is_l(j->side) ? opa(j, k, t) : opa(j, t, k))"),
    "trsm_sum_includes_diagonal": ("for (int64_t k = 0; k < t; ++k)", "for (int64_t k = 0; k <= t; ++k)"),
    "potrf_no_sqrt": ("*fac(&base, j, j) = sqrt(piv);", "*fac(&base, j, j) = piv;"),
    "potrf_wrong_update_row": ("s += *fac(p, i, k) * *fac(p, j, k);", "s += *fac(p, i, k) * *fac(p, i, k);"),
    "potrf_missing_division": ("*fac(p, i, j) = (*fac(p, i, j) - s) / d;", "*fac(p, i, j) = (*fac(p, i, j) - s);"),
    "potrf_info_off_by_one": ("info = j + 1;", "info = j;"),
    "potrf_upper_reads_lower": ("return p->lower ? &p->A[r * p->lda + c] : &p->A[c * p->lda + r];",
                                "return &p->A[r * p->lda + c];"),
}


def _build_variant(tmp_path, name, old, new):
    src = open(FACTOR).read()
    assert src.count(old) >= 1, name
    src = src.replace(old, new)
    d = tmp_path / name
    d.mkdir()
    (d / "f.c").write_text(src)
    lib = str(d / "libo.so")
    subprocess.check_call(["gcc", "-O1", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off",
                           os.path.join(HERE, "oracle.c"), str(d / "f.c"), "-o", lib, "-lpthread", "-lm"])
    return oracle.load(lib)


def _trsm_case(lib, side, uplo, ta, diag):
    rng = np.random.default_rng(zlib.crc32((side + uplo + ta + diag).encode()))
    M, N = (7, 4) if side == "L" else (4, 7)
    n = M if side == "L" else N
    A = rng.integers(-3, 4, size=(n, n)).astype(np.float64)
    A[np.diag_indices(n)] = np.nan if diag == "U" else rng.choice([-2.0, 2.0, 4.0], size=n)
    A[np.triu_indices(n, 1) if uplo == "L" else np.tril_indices(n, -1)] = np.nan
    T = np.where(np.isnan(A), 0.0, A)
    if diag == "U":
        T[np.diag_indices(n)] = 1.0
    opT = T if ta == "N" else T.T
    X = rng.integers(-5, 6, size=(M, N)).astype(np.float64) * 64
    B = (opT @ X if side == "L" else X @ opT) * 2.0    # small integers: exact in FP64
    got = level3.trsm(side, uplo, ta, diag, 0.5, A, B, lib=lib)
    return np.array_equal(got, X)


def _pins(lib):
    failures = []
    for side, uplo, ta, diag in itertools.product("LR", "LU", "NT", "NU"):
        if not _trsm_case(lib, side, uplo, ta, diag):
            failures.append("trsm %s%s%s%s" % (side, uplo, ta, diag))
    rng = np.random.default_rng(11)
    n = 9
    L = np.tril(rng.integers(-3, 4, size=(n, n))).astype(np.float64)
    L[np.diag_indices(n)] = rng.integers(1, 4, size=n)
    A = L @ L.T                                          # small integers: exact
    for uplo in "LU":
        A_in = A.copy()
        A_in[np.triu_indices(n, 1) if uplo == "L" else np.tril_indices(n, -1)] = np.nan
        F, info = level3.potrf(uplo, A_in, lib=lib)
        want = L if uplo == "L" else L.T
        got = np.tril(np.nan_to_num(F)) if uplo == "L" else np.triu(np.nan_to_num(F))
        if info != 0 or not np.array_equal(got, want):
            failures.append("potrf %s" % uplo)
    _, info = level3.potrf("L", np.diag([1.0, 4.0, -1.0]), lib=lib)
    if info != 3:
        failures.append("potrf info")
    return failures


def test_committed_factor_oracle_passes_the_pins():
    assert _pins(oracle.load()) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(tmp_path, name):
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    old, new = MUTANTS[name]
    lib = _build_variant(tmp_path, name, old, new)
    assert _pins(lib), "mutant %s passed every pin" % name


GETRF_MUTANTS = {
    "getrf_signed_pivot": ("const double v = fabs(A[i * lda + j]);", "const double v = A[i * lda + j];"),
    "getrf_last_of_ties": ("if (v > best) {", "if (v >= best) {"),
    "getrf_swap_right_part_only": ("for (int64_t k = 0; k < n; ++k) {\n                const double t = A[j * lda + k];",
                                   "for (int64_t k = j; k < n; ++k) {\n                const double t = A[j * lda + k];"),
    "getrf_no_scaling": ("const double l = A[i * lda + j] / d;", "const double l = A[i * lda + j];"),
    "getrf_update_from_wrong_row": ("A[i * lda + k] -= l * A[j * lda + k];", "A[i * lda + k] -= l * A[i * lda + k];"),
}


def _getrf_pins(lib):
    rng = np.random.default_rng(21)
    n = 10
    L = np.tril(rng.choice([-0.5, -0.25, 0.0, 0.25, 0.5], size=(n, n)), -1) + np.eye(n)
    U = np.triu(rng.integers(-3, 4, size=(n, n))).astype(np.float64)
    U[np.diag_indices(n)] = rng.choice([-8.0, -6.0, 6.0, 8.0], size=n)
    order = rng.permutation(n)
    A = np.empty((n, n))
    A[order] = L @ U                                     # exact: dyadic products of small integers
    F, ipiv, info = level3.getrf(A, lib=lib)
    ok = (info == 0 and np.array_equal(np.tril(F, -1) + np.eye(n), L) and np.array_equal(np.triu(F), U)
          and np.array_equal(level3.apply_pivots(A, ipiv), L @ U))
    _, ipiv2, _ = level3.getrf(np.array([[2.0, 1.0], [-2.0, 3.0]]), lib=lib)
    return [] if ok and list(ipiv2) == [0, 1] else ["getrf"]


@pytest.mark.parametrize("name", sorted(GETRF_MUTANTS))
def test_planted_getrf_mistake_is_caught(tmp_path, name):
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    old, new = GETRF_MUTANTS[name]
    lib = _build_variant(tmp_path, name, old, new)
    assert _getrf_pins(lib), "mutant %s passed every pin" % name


def test_committed_getrf_oracle_passes_the_pins():
    assert _getrf_pins(oracle.load()) == []
