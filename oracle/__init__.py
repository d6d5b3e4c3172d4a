"""CPU oracle for the out-of-core GEMM path.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this package; the
product library never does, and it shares no code with it.

Contents
  oracle.c        plain FP64 triple-loop GEMM (Section IV problem statement)
  factor.c        plain FP64 triangular solve and Cholesky (Section VII's next step)
  level3.py       SYRK / GEMMT / TRSM / POTRF on numpy operands
  partition.py    the paper's matrix partitioner, read from Section IV
  pipeline.py     the Section IV buffer-hazard rule, as a timeline checker
  costmodel.py    FP64 reference of the schedule cost-model MLP
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "factor.c")]
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force=False):
    """Compile oracle.c and factor.c with the host C compiler (no FMA contraction)."""
    if (not force and os.path.exists(_LIB)
            and all(os.path.getmtime(_LIB) >= os.path.getmtime(f) for f in _SRCS)):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off"] + _SRCS +
                          ["-o", tmp, "-lpthread", "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def load(path=None):
    """Load the compiled oracle (``path`` lets a test load a variant build)."""
    global _lib
    if path is None and _lib is not None:
        return _lib
    if path is None:
        build()
    lib = ctypes.CDLL(path or _LIB)
    i64, dbl, vp = ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
    blk = [ctypes.c_char, ctypes.c_char, i64, i64, i64, i64, i64, dbl, vp, i64, vp, i64, dbl,
           vp, i64, vp, i64, ctypes.c_int]
    for name in ("oracle_dgemm_block", "oracle_sgemm_block"):
        f = getattr(lib, name)
        f.restype = ctypes.c_int
        f.argtypes = blk
    lib.oracle_dtrsm.restype = ctypes.c_int
    lib.oracle_dtrsm.argtypes = [ctypes.c_char] * 4 + [i64, i64, dbl, vp, i64, vp, i64, ctypes.c_int]
    lib.oracle_dgetrf.restype = i64
    lib.oracle_dgetrf.argtypes = [i64, vp, i64, vp, ctypes.c_int]
    lib.oracle_dpotrf.restype = i64
    lib.oracle_dpotrf.argtypes = [ctypes.c_char, i64, vp, i64, ctypes.c_int]
    lib.oracle_dgemm.restype = ctypes.c_int
    lib.oracle_dgemm.argtypes = [ctypes.c_char, ctypes.c_char, i64, i64, i64, dbl, vp, i64, vp,
                                 i64, dbl, vp, i64, ctypes.c_int]
    if path is None:
        _lib = lib
    return lib


def _threads(n):
    if n is not None:
        return n
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def _ptr(x):
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return x.ctypes.data


def _ld(x):
    """Leading dimension (elements) of a 2-D array whose rows are contiguous."""
    if (x.numel() if hasattr(x, "numel") else x.size) == 0:
        return max(1, x.shape[1])
    if hasattr(x, "data_ptr"):
        assert x.shape[1] <= 1 or x.stride(1) == 1
        return x.stride(0) if x.shape[0] > 1 else max(1, x.shape[1])
    assert x.shape[1] <= 1 or x.strides[1] == x.itemsize
    return x.strides[0] // x.itemsize if x.shape[0] > 1 else max(1, x.shape[1])


def gemm_block(ta, tb, i0, j0, rows, cols, K, alpha, A, B, beta, Cold, nthreads=None, lib=None):
    """Rows i0.. and columns j0.. of alpha*op(A)*op(B) + beta*Cold as a new FP64 array.

    A and B are whole row-major operands (float64 or float32; float32 is
    widened).  Cold is the rows x cols block of the old C (float64), or None
    when beta == 0.  Returns (out, threads_used).
    """
    lib = lib or load()
    fp32 = (str(A.dtype) in ("float32", "torch.float32"))
    out = np.empty((rows, cols), dtype=np.float64)
    if Cold is not None:
        Cold = np.ascontiguousarray(Cold, dtype=np.float64)
    f = lib.oracle_sgemm_block if fp32 else lib.oracle_dgemm_block
    t = f(ta.encode(), tb.encode(), i0, j0, rows, cols, K, float(alpha), _ptr(A), _ld(A),
          _ptr(B), _ld(B), float(beta), _ptr(Cold), cols if Cold is not None else 0,
          out.ctypes.data, cols, _threads(nthreads))
    return out, t


def gemm(ta, tb, alpha, A, B, beta, C, nthreads=None, lib=None):
    """alpha*op(A)*op(B) + beta*C for whole numpy operands; returns a new FP64 array.

    Shapes follow the stored operands: for ta == 'N' A is M x K, else K x M;
    for tb == 'N' B is K x N, else N x K.  C (M x N) may be None when beta == 0.
    """
    M = A.shape[0] if ta in "Nn" else A.shape[1]
    K = A.shape[1] if ta in "Nn" else A.shape[0]
    N = B.shape[1] if tb in "Nn" else B.shape[0]
    out, _ = gemm_block(ta, tb, 0, 0, M, N, K, alpha, A, B, beta,
                        None if beta == 0.0 else C, nthreads=nthreads, lib=lib)
    return out


def rel_fro(x, ref):
    """||x - ref||_F / ||ref||_F in FP64 (0 when both are zero)."""
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    num = np.linalg.norm((x - ref).ravel())
    den = np.linalg.norm(ref.ravel())
    if den == 0.0:
        return 0.0 if num == 0.0 else float("inf")
    return float(num / den)
