"""GPU parity of the triangular updates (ooc_dgemmt, ooc_dsyrk, ooc_ssyrk)
against the CPU oracle (oracle/level3.py).

Updated triangle: within the form's tolerance of the oracle (FP64 1e-13,
Ozaki 1e-12, BF16x3 1e-6 relative Frobenius over the triangle).  The other
triangle must come back bit-identical, NaN included.  Blocks are forced small
and uneven (mb != nb, neither a multiple of the kernel tile) so that blocks
straddle the diagonal at every offset.
"""
import itertools

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import np64, pinned, pinned_from
from oracle import level3

pytestmark = pytest.mark.gpu
TOL = {1: 1e-13, 2: 1e-12, 3: 1e-6}


def _check(got, C0, ref, uplo, tol):
    m = level3.tri_mask(*got.shape, uplo)
    assert oracle.rel_fro(got[m], ref[m]) <= tol
    keep = ~m
    assert np.array_equal(got[keep], C0[keep], equal_nan=True)


def _syrk(ooc, uplo, trans, N, K, alpha, beta, form=1, kw=None, budget=1 << 30, seed=70, other_nan=True,
          kind=synth.NORMAL, param=0.0):
    fp32 = form == 3
    dt = torch.float32 if fp32 else torch.float64
    sa = (N, K) if trans == "N" else (K, N)
    A = pinned_from(seed, 0, *sa, kind, param, dtype=dt)
    C = pinned_from(seed, 2, N, N, kind, param, dtype=dt)
    if other_nan:
        C.numpy()[~level3.tri_mask(N, N, uplo)] = np.nan
    C0 = np64(C)
    st = ooc.ooc_stats()
    opts = ooc.make_opts(form=form, **(kw or {}))
    f = ooc.ooc_ssyrk if fp32 else ooc.ooc_dsyrk
    rc = f(uplo, trans, N, K, alpha, A, sa[1], beta, C, N, budget, opts, st)
    assert rc == 0, ooc.ooc_last_error()
    ref = level3.syrk(uplo, trans, alpha, np64(A), beta, np.nan_to_num(C0) if beta != 0 else C0)
    return np64(C), C0, ref, st


@pytest.mark.parametrize("uplo,trans", list(itertools.product("LU", "NT")))
def test_dsyrk_uneven_blocks(ooc, uplo, trans):
    got, C0, ref, st = _syrk(ooc, uplo, trans, 333, 170, 1.5, 0.5,
                             kw=dict(mb=96, nb=160, kb=64, depth=2, c_buffers=2))
    _check(got, C0, ref, uplo, TOL[1])
    assert st.blocks < 4 * 3  # blocks wholly outside the triangle were skipped


@pytest.mark.parametrize("uplo", "LU")
def test_dsyrk_auto_plan_small_budget(ooc, uplo):
    got, C0, ref, st = _syrk(ooc, uplo, "N", 1000, 300, 1.0, 1.0, budget=3 << 20)
    assert st.blocks > 2
    _check(got, C0, ref, uplo, TOL[1])


def test_dsyrk_beta_zero_ignores_nan_in_the_updated_triangle(ooc):
    N, K = 257, 65
    A = pinned_from(71, 0, N, K, synth.NORMAL)
    C = pinned(N, N, fill=float("nan"))
    C0 = np64(C)
    rc = ooc.ooc_dsyrk("L", "N", N, K, 2.0, A, K, 0.0, C, N, 1 << 30,
                       ooc.make_opts(mb=64, nb=96, kb=K), None)
    assert rc == 0, ooc.ooc_last_error()
    got = np64(C)
    ref = level3.syrk("L", "N", 2.0, np64(A), 0.0, C0)
    _check(got, C0, ref, "L", TOL[1])
    assert not np.isnan(got[level3.tri_mask(N, N, "L")]).any()


def test_dsyrk_integers_exact(ooc):
    N, K = 200, 400
    A = pinned_from(72, 0, N, K, synth.INTEGER, 64)
    C = pinned_from(72, 2, N, N, synth.INTEGER, 64)
    C0 = np64(C)
    rc = ooc.ooc_dsyrk("U", "N", N, K, 1.0, A, K, -1.0, C, N, 1 << 30, ooc.make_opts(mb=64, nb=64, kb=128), None)
    assert rc == 0, ooc.ooc_last_error()
    got = np64(C)
    ref = level3.syrk("U", "N", 1.0, np64(A), -1.0, C0)
    assert np.array_equal(got, ref)


def test_dsyrk_k_zero_scales_the_triangle(ooc):
    N = 150
    C = pinned_from(73, 2, N, N, synth.NORMAL)
    C0 = np64(C)
    A = pinned(N, 1)
    rc = ooc.ooc_dsyrk("L", "N", N, 0, 1.0, A, 1, 3.0, C, N, 1 << 30, None, None)
    assert rc == 0, ooc.ooc_last_error()
    m = level3.tri_mask(N, N, "L")
    got = np64(C)
    assert np.array_equal(got[m], 3.0 * C0[m]) and np.array_equal(got[~m], C0[~m])


@pytest.mark.parametrize("uplo", "LU")
def test_dsyrk_ozaki_form(ooc, uplo):
    got, C0, ref, st = _syrk(ooc, uplo, "T", 300, 200, 1.0, 0.5, form=2, kind=synth.LOGSPREAD,
                             kw=dict(mb=128, nb=256))
    assert st.products > 1
    _check(got, C0, ref, uplo, TOL[2])


@pytest.mark.parametrize("uplo", "LU")
def test_ssyrk_bf16x3_form(ooc, uplo):
    got, C0, ref, st = _syrk(ooc, uplo, "N", 300, 170, 1.5, 0.5, form=3, kind=synth.UNIFORM,
                             kw=dict(mb=128, nb=256))
    _check(got, C0, ref, uplo, TOL[3])


@pytest.mark.parametrize("ta,tb", list(itertools.product("NT", "NT")))
def test_dgemmt_distinct_operands(ooc, ta, tb):
    N, K = 290, 130
    sa = (N, K) if ta == "N" else (K, N)
    sb = (K, N) if tb == "N" else (N, K)
    A = pinned_from(74, 0, *sa, synth.NORMAL)
    B = pinned_from(74, 1, *sb, synth.NORMAL)
    C = pinned_from(74, 2, N, N, synth.NORMAL)
    C0 = np64(C)
    rc = ooc.ooc_dgemmt("U", ta, tb, N, K, 0.5, A, sa[1], B, sb[1], 2.0, C, N, 1 << 30,
                        ooc.make_opts(mb=64, nb=128, kb=64), None)
    assert rc == 0, ooc.ooc_last_error()
    ref = level3.gemmt("U", ta, tb, 0.5, np64(A), np64(B), 2.0, C0)
    _check(np64(C), C0, ref, "U", TOL[1])


def test_level3_bad_arguments(ooc):
    A = pinned(8, 8)
    C = pinned(8, 8)
    assert ooc.ooc_dsyrk("X", "N", 8, 8, 1.0, A, 8, 0.0, C, 8, 1 << 20, None, None) == ooc.OOC_ERR_INVALID_ARG
    assert ooc.ooc_dsyrk("L", "Q", 8, 8, 1.0, A, 8, 0.0, C, 8, 1 << 20, None, None) == ooc.OOC_ERR_INVALID_ARG
    assert ooc.ooc_dsyrk("L", "N", 8, 8, 1.0, A, 4, 0.0, C, 8, 1 << 20, None, None) == ooc.OOC_ERR_INVALID_ARG


# ---- TRSM ------------------------------------------------------------------
def _tri_operand(seed, n, uplo, diag, nan_other=True):
    """A well-conditioned triangular A (stored n x n): N(0,1) / sqrt(n) off the
    diagonal, diagonal 1 + |N(0,1)| (NaN when unit), NaN in the unread triangle."""
    A = pinned_from(seed, 0, n, n, synth.NORMAL)
    a = A.numpy()
    a *= 1.0 / np.sqrt(n)
    d = np.abs(np.diag(a)) * np.sqrt(n) + 1.0
    a[np.diag_indices(n)] = np.nan if diag == "U" else d
    if nan_other:
        a[np.triu_indices(n, 1) if uplo == "L" else np.tril_indices(n, -1)] = np.nan
    return A


def _trsm(ooc, side, uplo, ta, diag, M, N, alpha, budget, seed=80, opts=None):
    n = M if side == "L" else N
    A = _tri_operand(seed, n, uplo, diag)
    B = pinned_from(seed, 1, M, N, synth.NORMAL)
    B0 = np64(B)
    st = ooc.ooc_stats()
    rc = ooc.ooc_dtrsm(side, uplo, ta, diag, M, N, alpha, A, n, B, N, budget, opts, st)
    assert rc == 0, ooc.ooc_last_error()
    ref = level3.trsm(side, uplo, ta, diag, alpha, np64(A), B0)
    return np64(B), ref, st


@pytest.mark.parametrize("side,uplo,ta,diag", list(itertools.product("LR", "LU", "NT", "NU")))
def test_dtrsm_all_variants_several_panels(ooc, side, uplo, ta, diag):
    # a 256 KiB budget gives 64-wide panels: 5 panels of the 300-order triangle, ragged last one
    M, N = (300, 170) if side == "L" else (170, 300)
    got, ref, st = _trsm(ooc, side, uplo, ta, diag, M, N, 1.5, 256 << 10)
    assert st.steps >= 4  # one out-of-core GEMM per panel after the first
    assert oracle.rel_fro(got, ref) <= 1e-12


@pytest.mark.parametrize("side", "LR")
def test_dtrsm_large_panels_recursive_solve(ooc, side):
    # panels of 1024 -> the in-device solve recurses down to 64 blocks with tile-kernel updates
    M, N = (1100, 700) if side == "L" else (700, 1100)
    got, ref, _ = _trsm(ooc, side, "L", "N", "N", M, N, -0.5, 64 << 20, seed=81)
    assert oracle.rel_fro(got, ref) <= 1e-12


def test_dtrsm_ozaki_updates(ooc):
    got, ref, st = _trsm(ooc, "L", "U", "T", "N", 1500, 300, 1.0, 16 << 20, seed=82,
                         opts=ooc.make_opts(form=ooc.OOC_FORM_OZAKI))
    assert st.form == ooc.OOC_FORM_OZAKI
    assert oracle.rel_fro(got, ref) <= 1e-12


def test_dtrsm_integer_solution_exact(ooc):
    n, N = 256, 96
    rng = np.random.default_rng(5)
    A = pinned(n, n)
    a = A.numpy()
    a[:] = np.tril(rng.integers(-2, 3, size=(n, n))).astype(np.float64)
    a[np.diag_indices(n)] = 1.0
    X = rng.integers(-3, 4, size=(n, N)).astype(np.float64)
    B = pinned(n, N)
    B.numpy()[:] = np.tril(a) @ X  # small integers, exact (entries far below 2^53)
    assert np.abs(B.numpy()).max() < 2.0 ** 40
    rc = ooc.ooc_dtrsm("L", "L", "N", "U", n, N, 1.0, A, n, B, N, 256 << 10, None, None)
    assert rc == 0, ooc.ooc_last_error()
    assert np.array_equal(np64(B), X)


def test_dtrsm_alpha_zero_and_bad_arguments(ooc):
    A = pinned(8, 8, fill=1.0)
    B = pinned(8, 4, fill=float("nan"))
    assert ooc.ooc_dtrsm("L", "L", "N", "N", 8, 4, 0.0, A, 8, B, 4, 1 << 20, None, None) == 0
    assert np.array_equal(np64(B), np.zeros((8, 4)))
    assert ooc.ooc_dtrsm("X", "L", "N", "N", 8, 4, 1.0, A, 8, B, 4, 1 << 20, None, None) == ooc.OOC_ERR_INVALID_ARG
    assert ooc.ooc_dtrsm("L", "L", "N", "N", 8, 4, 1.0, A, 4, B, 4, 1 << 20, None, None) == ooc.OOC_ERR_INVALID_ARG
    assert ooc.ooc_dtrsm("L", "L", "N", "N", 8, 4, 1.0, A, 8, B, 4, 4096, None, None) == ooc.OOC_ERR_BUDGET


# ---- Cholesky ----------------------------------------------------------------
def _spd(seed, n, nan_other=None):
    """SPD A = G G^T / n + I (G N(0,1)), formed in FP64 on the host; NaN in the unread triangle."""
    G = synth.matrix(n, n, seed, 0, synth.NORMAL)
    S = G @ G.T / n + np.eye(n)
    A = pinned(n, n)
    A.numpy()[:] = S
    if nan_other:
        A.numpy()[np.triu_indices(n, 1) if nan_other == "L" else np.tril_indices(n, -1)] = np.nan
    return A, S


@pytest.mark.parametrize("uplo", "LU")
@pytest.mark.parametrize("n,budget", [(300, 256 << 10), (1000, 16 << 20), (1300, 64 << 20)])
def test_dpotrf_matches_oracle(ooc, uplo, n, budget):
    A, S = _spd(90 + n, n, nan_other=uplo)
    A0 = np64(A)
    st = ooc.ooc_stats()
    rc, info = ooc.ooc_dpotrf(uplo, n, A, n, budget, None, st)
    assert rc == 0 and info == 0, ooc.ooc_last_error()
    ref, rinfo = level3.potrf(uplo, A0)
    assert rinfo == 0
    got = np64(A)
    m = level3.tri_mask(n, n, "L" if uplo == "L" else "U")
    assert oracle.rel_fro(got[m], ref[m]) <= 1e-12
    assert np.isnan(got[~m]).all()  # the other triangle is neither used nor changed
    F = np.tril(np.nan_to_num(got)) if uplo == "L" else np.triu(np.nan_to_num(got)).T
    assert oracle.rel_fro(F @ F.T, S) <= 1e-14


def test_dpotrf_ozaki_updates(ooc):
    n = 900
    A, S = _spd(95, n, nan_other="L")
    A0 = np64(A)
    rc, info = ooc.ooc_dpotrf("L", n, A, n, 8 << 20, ooc.make_opts(form=ooc.OOC_FORM_OZAKI), None)
    assert rc == 0 and info == 0, ooc.ooc_last_error()
    ref, _ = level3.potrf("L", A0)
    m = level3.tri_mask(n, n, "L")
    assert oracle.rel_fro(np64(A)[m], ref[m]) <= 1e-12


def test_dpotrf_integer_factor_exact(ooc):
    n = 200
    rng = np.random.default_rng(6)
    L = np.tril(rng.integers(-2, 3, size=(n, n))).astype(np.float64)
    L[np.diag_indices(n)] = 1.0
    A = pinned(n, n)
    A.numpy()[:] = L @ L.T   # integers below 2^53: exact
    rc, info = ooc.ooc_dpotrf("L", n, A, n, 256 << 10, None, None)
    assert rc == 0 and info == 0, ooc.ooc_last_error()
    assert np.array_equal(np.tril(np64(A)), L)


@pytest.mark.parametrize("bad", [37, 130, 299])
def test_dpotrf_reports_the_first_bad_pivot(ooc, bad):
    n = 300
    A, S = _spd(96, n)
    a = A.numpy()
    a[bad, bad] = -1.0      # leading minors up to bad stay positive definite, order bad + 1 is not
    A0 = np64(A)
    rc, info = ooc.ooc_dpotrf("L", n, A, n, 256 << 10, None, None)
    assert rc == 0, ooc.ooc_last_error()
    _, rinfo = level3.potrf("L", A0)
    assert info == rinfo == bad + 1


# ---- LU with partial pivoting ------------------------------------------------------
def _getrf(ooc, A, budget, opts=None):
    n = A.shape[0]
    ipiv = np.zeros(n, dtype=np.int64)
    st = ooc.ooc_stats()
    rc, info = ooc.ooc_dgetrf(n, A, n, ipiv, budget, opts, st)
    assert rc == 0, ooc.ooc_last_error()
    return ipiv, info, st


def test_dgetrf_exact_factors_several_panels(ooc):
    """A = P L U with dyadic |l| <= 1/2 and an integer U: unique pivots, exact arithmetic."""
    rng = np.random.default_rng(31)
    n = 300
    L = np.tril(rng.choice([-0.5, -0.25, 0.0, 0.25, 0.5], size=(n, n)), -1) + np.eye(n)
    U = np.triu(rng.integers(-3, 4, size=(n, n))).astype(np.float64)
    U[np.diag_indices(n)] = rng.choice([-8.0, -6.0, 6.0, 8.0], size=n)
    A = pinned(n, n)
    A.numpy()[rng.permutation(n)] = L @ U      # dyadic products of small integers: exact
    A0 = np64(A)
    ipiv, info, st = _getrf(ooc, A, 256 << 10)   # 64-column panels
    assert info == 0 and st.steps >= 4
    F, rpiv, rinfo = level3.getrf(A0)
    assert list(ipiv) == list(rpiv)
    assert np.array_equal(np64(A), F)
    assert np.array_equal(np.triu(np64(A)), U)


@pytest.mark.parametrize("n,budget", [(500, 512 << 10), (1500, 4 << 20), (1100, 64 << 20)])
def test_dgetrf_matches_oracle(ooc, n, budget):
    A = pinned_from(160 + n, 0, n, n, synth.NORMAL)
    A0 = np64(A)
    ipiv, info, _ = _getrf(ooc, A, budget)
    F, rpiv, rinfo = level3.getrf(A0)
    assert info == rinfo == 0
    assert list(ipiv) == list(rpiv)              # clear-cut pivots on these seeded inputs
    assert oracle.rel_fro(np64(A), F) <= 1e-12
    got = np64(A)
    Lg = np.tril(got, -1) + np.eye(n)
    assert np.abs(np.tril(got, -1)).max() <= 1.0
    assert oracle.rel_fro(Lg @ np.triu(got), level3.apply_pivots(A0, ipiv)) <= 1e-14


def test_dgetrf_ozaki_updates(ooc):
    n = 1500
    A = pinned_from(170, 0, n, n, synth.NORMAL)
    A0 = np64(A)
    # Ozaki operand slots hold whole-K bf16 digit planes: a budget with room for them
    ipiv, info, st = _getrf(ooc, A, 64 << 20, ooc.make_opts(form=ooc.OOC_FORM_OZAKI))
    # the factorizations' Ozaki updates carry 9 digits of 6 bits (54 bits, FP64's 53-bit
    # significand covered), so the factors are held to the FP64-accurate tolerance
    assert st.slices == 9 and st.products == 45
    F, rpiv, _ = level3.getrf(A0)
    assert list(ipiv) == list(rpiv)
    got = np64(A)
    assert oracle.rel_fro(got, F) <= 1e-12
    # Gaussian elimination's backward error bound ||P A - L U|| <= n u || |L| |U| || at FP64's u
    Lg, Ug = np.tril(got, -1) + np.eye(n), np.triu(got)
    resid = oracle.rel_fro(Lg @ Ug, level3.apply_pivots(A0, ipiv))
    growth = np.linalg.norm(np.abs(Lg) @ np.abs(Ug)) / np.linalg.norm(A0)
    assert resid <= n * 2.0 ** -53 * growth


def test_dgetrf_ozaki_eight_digits_on_request(ooc):
    """opts->slices = 8 gives the GEMM entry points' 48-bit digits inside the factorization:
    each update is then rounded at u = 2^-48 relative to the operand rows' maxima, so Gaussian
    elimination's backward error bound n u || |L| |U| || applies with that u."""
    n = 1500
    A = pinned_from(170, 0, n, n, synth.NORMAL)
    A0 = np64(A)
    ipiv, info, st = _getrf(ooc, A, 64 << 20, ooc.make_opts(form=ooc.OOC_FORM_OZAKI, slices=8))
    assert st.slices == 8
    got = np64(A)
    Lg, Ug = np.tril(got, -1) + np.eye(n), np.triu(got)
    resid = oracle.rel_fro(Lg @ Ug, level3.apply_pivots(A0, ipiv))
    growth = np.linalg.norm(np.abs(Lg) @ np.abs(Ug)) / np.linalg.norm(A0)
    assert resid <= n * 2.0 ** -48 * growth


@pytest.mark.parametrize("zero_col", [5, 70, 299])
def test_dgetrf_zero_pivot_sets_info(ooc, zero_col):
    n = 300
    A = pinned_from(171, 0, n, n, synth.NORMAL)
    A.numpy()[:, zero_col] = 0.0   # a zero column stays exactly zero through the elimination
    A0 = np64(A)
    ipiv, info, _ = _getrf(ooc, A, 256 << 10)
    F, rpiv, rinfo = level3.getrf(A0)
    assert info == rinfo == zero_col + 1
    assert list(ipiv) == list(rpiv)
    assert oracle.rel_fro(np64(A), F) <= 1e-12


@pytest.mark.parametrize("n,budget,zero_col", [(500, 512 << 10, None), (1100, 64 << 20, None), (300, 256 << 10, 70)])
def test_dgetrf_panel_rows_in_global_memory(ooc, n, budget, zero_col, monkeypatch):
    """The panel kernel's other path (rows kept in global memory, taken when a co-resident
    grid's row slices do not fit shared memory), forced here on panels that would fit."""
    monkeypatch.setenv("OOC_LU_ROWS_GLOBAL", "1")
    A = pinned_from(180 + n, 0, n, n, synth.NORMAL)
    if zero_col is not None:
        A.numpy()[:, zero_col] = 0.0
    A0 = np64(A)
    ipiv, info, _ = _getrf(ooc, A, budget)
    F, rpiv, rinfo = level3.getrf(A0)
    assert info == rinfo == (0 if zero_col is None else zero_col + 1)
    assert list(ipiv) == list(rpiv)
    assert oracle.rel_fro(np64(A), F) <= 1e-12


def test_dgetrf_bad_arguments(ooc):
    A = pinned(8, 8)
    ipiv = np.zeros(8, dtype=np.int64)
    assert ooc.ooc_dgetrf(8, A, 4, ipiv, 1 << 20)[0] == ooc.OOC_ERR_INVALID_ARG
    assert ooc.ooc_dgetrf(8, A, 8, ipiv, 1024)[0] == ooc.OOC_ERR_BUDGET
