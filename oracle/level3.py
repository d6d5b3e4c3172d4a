"""Oracle of the level-3 operations beyond GEMM (Section VII's next step).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper defines none of these operations; each function is the textbook
definition:

  gemmt(uplo, ...)  C <- alpha op(A) op(B) + beta C on one triangle of the
                    square C (uplo 'L': column <= row, 'U': column >= row),
                    other elements unchanged.  The updated elements are the
                    GEMM oracle's values (oracle.c), so their sums run in the
                    same order as there.
  syrk(uplo, ...)   gemmt with op(B) = op(A)^T.
  trsm(...)         factor.c: substitution for each right-hand side.
  potrf(...)        factor.c: column-by-column Cholesky.
  getrf(...)        factor.c: right-looking LU with partial pivoting.

Operands are numpy arrays (row-major, float64; float32 is widened for the
triangle values of gemmt/syrk).  Each function returns a new array.
"""
import numpy as np

from . import _ld, _ptr, _threads, gemm_block, load


def tri_mask(n_rows, n_cols, uplo, off=0, r0=0, c0=0):
    """Boolean mask of the updated elements of rows r0.. and columns c0..:
    column - row <= off for 'L', >= off for 'U'."""
    r = np.arange(r0, r0 + n_rows)[:, None]
    c = np.arange(c0, c0 + n_cols)[None, :]
    return (c - r <= off) if uplo in "Ll" else (c - r >= off)


def gemmt(uplo, ta, tb, alpha, A, B, beta, C, nthreads=None):
    """C <- alpha op(A) op(B) + beta C on the uplo triangle of the N x N C."""
    N = C.shape[0]
    K = A.shape[1] if ta in "Nn" else A.shape[0]
    full, _ = gemm_block(ta, tb, 0, 0, N, N, K, alpha, A, B, beta,
                         None if beta == 0.0 else np.asarray(C, dtype=np.float64), nthreads=nthreads)
    out = np.array(C, dtype=np.float64, copy=True)
    m = tri_mask(N, N, uplo)
    out[m] = full[m]
    return out


def syrk(uplo, trans, alpha, A, beta, C, nthreads=None):
    """C <- alpha op(A) op(A)^T + beta C on the uplo triangle; trans 'N': A A^T, 'T': A^T A."""
    return gemmt(uplo, trans, "T" if trans in "Nn" else "N", alpha, A, A, beta, C, nthreads=nthreads)


def syrk_block(uplo, trans, i0, j0, rows, cols, alpha, A, beta, Cold, nthreads=None):
    """Rows i0.. and columns j0.. of syrk's result, given that block of the old C (float64)."""
    K = A.shape[1] if trans in "Nn" else A.shape[0]
    full, _ = gemm_block(trans, "T" if trans in "Nn" else "N", i0, j0, rows, cols, K, alpha, A, A, beta,
                         None if beta == 0.0 else Cold, nthreads=nthreads)
    out = np.array(Cold, dtype=np.float64, copy=True)
    m = tri_mask(rows, cols, uplo, 0, i0, j0)
    out[m] = full[m]
    return out


def trsm(side, uplo, ta, diag, alpha, A, B, nthreads=None, lib=None):
    """X with op(A) X = alpha B (side 'L') or X op(A) = alpha B (side 'R'); A triangular."""
    lib = lib or load()
    X = np.array(B, dtype=np.float64, copy=True, order="C")
    A = np.ascontiguousarray(A, dtype=np.float64)
    M, N = X.shape
    if M and N:
        lib.oracle_dtrsm(side.encode(), uplo.encode(), ta.encode(), diag.encode(), M, N, float(alpha),
                         _ptr(A), _ld(A), _ptr(X), _ld(X), _threads(nthreads))
    return X


def potrf(uplo, A, nthreads=None, lib=None):
    """(factor, info): the Cholesky factor in the uplo triangle of a copy of A
    (the other triangle copied unchanged); info 0, or j + 1 at a non-positive pivot j."""
    lib = lib or load()
    F = np.array(A, dtype=np.float64, copy=True, order="C")
    n = F.shape[0]
    info = lib.oracle_dpotrf(uplo.encode(), n, _ptr(F), _ld(F), _threads(nthreads)) if n else 0
    return F, int(info)


def getrf(A, nthreads=None, lib=None):
    """(factors, ipiv, info): L (unit, below the diagonal) and U (on and above it) of a copy of
    the square A with A = P L U; ipiv[j] = the row exchanged with row j at step j (0-based)."""
    lib = lib or load()
    F = np.array(A, dtype=np.float64, copy=True, order="C")
    n = F.shape[0]
    ipiv = np.zeros(max(n, 1), dtype=np.int64)
    info = lib.oracle_dgetrf(n, _ptr(F), _ld(F), ipiv.ctypes.data, _threads(nthreads)) if n else 0
    return F, ipiv[:n], int(info)


def apply_pivots(X, ipiv):
    """Rows of X exchanged in order: row j with row ipiv[j] (a copy)."""
    Y = np.array(X, copy=True)
    for j, p in enumerate(ipiv):
        if p != j:
            Y[[j, p]] = Y[[p, j]]
    return Y
