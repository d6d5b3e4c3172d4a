"""Planted mistakes: each plausible slip in the oracle must fail at least one pin.

The mistake is planted in a copy of the oracle's C source, built into a temporary
library on the CPU; the committed oracle is never modified.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
import synth

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")

MUTANTS = {
    "dropped_beta_term": ("if (beta != 0.0) r += beta * cold;", "if (beta != 0.0) r += 0.0 * cold;"),
    "wrong_beta_sign": ("if (beta != 0.0) r += beta * cold;", "if (beta != 0.0) r -= beta * cold;"),
    "alpha_not_applied": ("double r = alpha * acc;", "double r = acc;"),
    "c_read_when_beta_zero": ("double cold = (jb->beta != 0.0) ? jb->Cold[r * jb->ldco + c] : 0.0;",
                              "double cold = jb->Cold[r * jb->ldco + c];"),
    "transposed_a_index": ("return is_t(ta) ? A[k * lda + i] : A[i * lda + k];",
                           "return is_t(ta) ? A[i * lda + k] : A[k * lda + i];"),
    "transposed_b_index": ("return is_t(tb) ? B[j * ldb + k] : B[k * ldb + j];",
                           "return is_t(tb) ? B[k * ldb + j] : B[j * ldb + k];"),
    "dropped_last_k": ("for (int64_t k = 0; k < K; ++k)\n        acc += elem_a(",
                       "for (int64_t k = 0; k + 1 < K; ++k)\n        acc += elem_a("),
    "ld_ignored_for_a": ("A[i * lda + k];\n}", "A[i * K_ + k];\n}"),
    "sign_flip_product": ("acc += elem_a(A, lda, ta, i, k) * elem_b(B, ldb, tb, k, j);",
                          "acc -= elem_a(A, lda, ta, i, k) * elem_b(B, ldb, tb, k, j);"),
    "wrong_block_column_offset": ("jb->i0 + r, jb->j0 + c);\n            jb->out",
                                  "jb->i0 + r, c);\n            jb->out"),
}


def _build_variant(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) >= 1, name
    if name == "ld_ignored_for_a":
        # the A leading dimension replaced by the row width of a padded-free layout
        src = src.replace("static double elem_a(const double* A, int64_t lda, char ta, int64_t i, int64_t k)\n{",
                          "static double elem_a(const double* A, int64_t lda, char ta, int64_t i, int64_t k)\n{\n    const int64_t K_ = 5; (void)K_;")
    src = src.replace(old, new, 1)
    if name == "c_read_when_beta_zero":
        src = src.replace("if (beta != 0.0) r += beta * cold;", "r += beta * cold;")
    d = tmp_path / name
    d.mkdir()
    (d / "o.c").write_text(src)
    lib = str(d / "libo.so")
    factor = os.path.join(os.path.dirname(SRC), "factor.c")
    subprocess.check_call(["gcc", "-O1", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off",
                           str(d / "o.c"), factor, "-o", lib, "-lpthread", "-lm"])
    return oracle.load(lib)


def _pins(lib):
    """Independent pins: exact rationals (all transposes), NaN C with beta=0, padding, BLAS."""
    failures = []
    A = synth.matrix(5, 7, 21, 0, synth.DYADIC, 64)
    B = synth.matrix(7, 6, 21, 1, synth.DYADIC, 64)
    C = synth.matrix(5, 6, 21, 2, synth.DYADIC, 64)
    ref = 1.5 * (A @ B) - 0.75 * C   # exact: dyadic inputs, K=7
    for ta in "NT":
        for tb in "NT":
            a = np.ascontiguousarray(A.T if ta == "T" else A)
            b = np.ascontiguousarray(B.T if tb == "T" else B)
            got, _ = oracle.gemm_block(ta, tb, 0, 0, 5, 6, 7, 1.5, a, b, -0.75, C, lib=lib)
            if not np.array_equal(got, ref):
                failures.append("exact %s%s" % (ta, tb))
    got, _ = oracle.gemm_block("N", "N", 0, 0, 5, 6, 7, 1.0, A, B, 0.0, np.full((5, 6), np.nan),
                               lib=lib)
    if not np.array_equal(got, A @ B):
        failures.append("beta=0 NaN")
    Ap = np.full((5, 7 + 4), np.nan); Ap[:, :7] = A
    got, _ = oracle.gemm_block("N", "N", 0, 0, 5, 6, 7, 1.0, Ap[:, :7], B, 0.0, np.zeros((5, 6)),
                               lib=lib)
    if not np.array_equal(got, A @ B):
        failures.append("padding")
    blk, _ = oracle.gemm_block("N", "N", 1, 2, 3, 3, 7, 1.5, A, B, -0.75, C[1:4, 2:5], lib=lib)
    if not np.array_equal(blk, ref[1:4, 2:5]):
        failures.append("block")
    return failures


def test_committed_oracle_passes_the_pins():
    assert _pins(oracle.load()) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(tmp_path, name):
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    old, new = MUTANTS[name]
    lib = _build_variant(tmp_path, name, old, new)
    assert _pins(lib), "mutant %s passed every pin" % name
