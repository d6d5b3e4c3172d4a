"""Seeded synthetic inputs (Philox4x32-10), shared by tests, benchmark and oracle callers.

This module holds none of the GEMM method's arithmetic: it only fills host
buffers with reproducible numbers.  The C source is ``gen.c`` beside this file;
it is compiled on first use with the host C compiler (no CUDA involved).
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "libsynth.so")
_lib = None

UNIFORM, NORMAL, LOGSPREAD, INTEGER, DYADIC = 0, 1, 2, 3, 4


def build(force=False):
    """Compile gen.c into libsynth.so (skipped when the library is newer)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off",
                           _SRC, "-o", tmp, "-lm", "-lpthread"])
    os.replace(tmp, _LIB)
    return _LIB


def _get():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        lib.synth_fill.restype = ctypes.c_int
        lib.synth_fill.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_int64,
                                   ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int,
                                   ctypes.c_double, ctypes.c_int]
        lib.synth_philox4x32_10.restype = None
        lib.synth_philox4x32_10.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        _lib = lib
    return _lib


def default_threads():
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def fill_ptr(ptr, fp32, rows, cols, ld, seed, stream, kind, param=0.0, nthreads=None):
    """Fill raw host memory at ``ptr`` (row-major, leading dimension ``ld``)."""
    n = default_threads() if nthreads is None else nthreads
    return _get().synth_fill(ctypes.c_void_p(ptr), int(bool(fp32)), int(rows), int(cols), int(ld),
                             int(seed), int(stream), int(kind), float(param), int(n))


def fill(arr, seed, stream, kind, param=0.0, nthreads=None):
    """Fill a 2-D C-contiguous-rows float32/float64 numpy array or CPU torch tensor in place."""
    if hasattr(arr, "data_ptr"):  # torch tensor (e.g. pinned host memory)
        assert arr.dim() == 2 and arr.stride(1) == 1 and not arr.is_cuda
        fp32 = str(arr.dtype) == "torch.float32"
        assert fp32 or str(arr.dtype) == "torch.float64"
        return fill_ptr(arr.data_ptr(), fp32, arr.shape[0], arr.shape[1], arr.stride(0),
                        seed, stream, kind, param, nthreads)
    assert arr.ndim == 2 and arr.strides[1] == arr.itemsize
    assert arr.dtype in (np.float32, np.float64)
    return fill_ptr(arr.ctypes.data, arr.dtype == np.float32, arr.shape[0], arr.shape[1],
                    arr.strides[0] // arr.itemsize, seed, stream, kind, param, nthreads)


def matrix(rows, cols, seed, stream, kind, param=0.0, dtype=np.float64):
    """A new rows x cols numpy array drawn from the given stream."""
    a = np.empty((rows, cols), dtype=dtype)
    fill(a, seed, stream, kind, param)
    return a


def philox4x32_10(ctr, key):
    """The raw generator block, for known-answer checks."""
    c = (ctypes.c_uint32 * 4)(*ctr)
    k = (ctypes.c_uint32 * 2)(*key)
    o = (ctypes.c_uint32 * 4)()
    _get().synth_philox4x32_10(c, k, o)
    return list(o)
