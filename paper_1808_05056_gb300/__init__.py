"""Python binding of libooc, the GB300 out-of-core GEMM (C ABI in include/ooc.h).

Every function here only marshals arguments into the C ABI of the same name;
all work runs in the library's CUDA kernels and copy streams.  There is no
CPU path: if the compiled library is missing, ``load()`` raises.

Host operands must be page-locked (e.g. ``torch.empty(..., pin_memory=True)``);
tensors are passed as row-major 2-D arrays whose rows are contiguous.
"""
import ctypes
import os

from . import _build

LIB_PATH = _build.LIB

OOC_OK = 0
OOC_ERR_INVALID_ARG = -1
OOC_ERR_BUDGET = -2
OOC_ERR_NOT_PINNED = -3
OOC_ERR_CUDA = -4
OOC_ERR_NO_DEVICE = -5
OOC_ERR_TIMEOUT = -6
OOC_ERR_ALLOC = -7
OOC_ERR_UNSUPPORTED = -8
OOC_ERR_INJECTED = -9
OOC_ERR_CAPACITY = -10

OOC_FORM_AUTO, OOC_FORM_FP64, OOC_FORM_OZAKI, OOC_FORM_BF16X3 = 0, 1, 2, 3
OOC_PLAN_PAPER = 1


class ooc_opts(ctypes.Structure):
    _fields_ = [("form", ctypes.c_int32), ("depth", ctypes.c_int32), ("c_buffers", ctypes.c_int32),
                ("slices", ctypes.c_int32), ("mb", ctypes.c_int64), ("nb", ctypes.c_int64),
                ("kb", ctypes.c_int64), ("flags", ctypes.c_uint32), ("b_buffers", ctypes.c_int32),
                ("workspace", ctypes.c_void_p), ("workspace_bytes", ctypes.c_size_t)]


class ooc_stats(ctypes.Structure):
    _fields_ = [("seconds", ctypes.c_double), ("device_seconds", ctypes.c_double),
                ("kernel_seconds", ctypes.c_double), ("tflops", ctypes.c_double),
                ("h2d_bytes", ctypes.c_double), ("d2h_bytes", ctypes.c_double),
                ("mb", ctypes.c_int64), ("nb", ctypes.c_int64), ("kb", ctypes.c_int64),
                ("depth", ctypes.c_int32), ("c_buffers", ctypes.c_int32), ("b_buffers", ctypes.c_int32),
                ("form", ctypes.c_int32), ("blocks", ctypes.c_int64), ("steps", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("slices", ctypes.c_int32), ("products", ctypes.c_int32),
                ("kernel_launches", ctypes.c_int64), ("split_seconds", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ooc_sched_op(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("stream", ctypes.c_int32), ("event", ctypes.c_int32),
                ("nreads", ctypes.c_int32), ("write_slot", ctypes.c_int32),
                ("read_slot", ctypes.c_int32 * 3), ("write_tag", ctypes.c_int64 * 4),
                ("read_tag", (ctypes.c_int64 * 4) * 3)]


class ooc_gemm_desc(ctypes.Structure):
    _fields_ = [("transA", ctypes.c_char), ("transB", ctypes.c_char), ("reserved", ctypes.c_char * 6),
                ("M", ctypes.c_int64), ("N", ctypes.c_int64), ("K", ctypes.c_int64),
                ("alpha", ctypes.c_double), ("beta", ctypes.c_double),
                ("A", ctypes.c_void_p), ("lda", ctypes.c_int64), ("B", ctypes.c_void_p), ("ldb", ctypes.c_int64),
                ("C", ctypes.c_void_p), ("ldc", ctypes.c_int64)]


OOC_BATCH_GRAPH = 2
OOC_BATCH_STREAMED = 16
OOC_PLAN_MODEL = 4
OOC_MLP_INPUTS = 16
OOC_MLP_PARAMS = 5313


class ooc_plan_candidate(ctypes.Structure):
    _fields_ = [("mb", ctypes.c_int64), ("nb", ctypes.c_int64), ("kb", ctypes.c_int64),
                ("depth", ctypes.c_int32), ("b_buffers", ctypes.c_int32), ("c_buffers", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("est_seconds", ctypes.c_double),
                ("features", ctypes.c_float * OOC_MLP_INPUTS)]

EXPORTS = ("ooc_dgemm", "ooc_sgemm", "ooc_dgemm_batched", "ooc_dgemm_device", "ooc_plan", "ooc_schedule",
           "ooc_plan_candidates", "ooc_autotune", "ooc_mlp_forward", "ooc_mlp_loss_grad", "ooc_mlp_train",
           "ooc_costmodel_set",
           "ooc_query_device", "ooc_strerror", "ooc_last_error")

_lib = None


class OocError(RuntimeError):
    def __init__(self, code, fn):
        self.code = code
        lib = load()
        super().__init__("%s: %s (%d): %s" % (fn, lib.ooc_strerror(code).decode(), code,
                                              lib.ooc_last_error().decode()))


def build(force=False):
    """Compile libooc.so for sm_103a (in-tree)."""
    return _build.build(force=force)


def load(path=None):
    """Load libooc.so and declare its signatures; raises if it is not built."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError("libooc.so is not built (%s); run paper_1808_05056_gb300.build()" % p)
    lib = ctypes.CDLL(p)
    i64, i32, dbl, flt, vp, ch = (ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_float,
                                  ctypes.c_void_p, ctypes.c_char)
    sz = ctypes.c_size_t
    po, ps = ctypes.POINTER(ooc_opts), ctypes.POINTER(ooc_stats)
    lib.ooc_dgemm.argtypes = [ch, ch, i64, i64, i64, dbl, vp, i64, vp, i64, dbl, vp, i64, sz, po, ps]
    lib.ooc_sgemm.argtypes = [ch, ch, i64, i64, i64, flt, vp, i64, vp, i64, flt, vp, i64, sz, po, ps]
    lib.ooc_dgemm_device.argtypes = [ch, ch, i64, i64, i64, dbl, vp, i64, vp, i64, dbl, vp, i64, vp]
    lib.ooc_plan.argtypes = [i64, i64, i64, i32, i32, sz, po, ps]
    lib.ooc_schedule.argtypes = [i64, i64, i64, i32, i32, sz, po, ctypes.POINTER(ooc_sched_op), i64,
                                 ctypes.POINTER(i64)]
    lib.ooc_dgemmt.argtypes = [ch, ch, ch, i64, i64, dbl, vp, i64, vp, i64, dbl, vp, i64, sz, po, ps]
    lib.ooc_dsyrk.argtypes = [ch, ch, i64, i64, dbl, vp, i64, dbl, vp, i64, sz, po, ps]
    lib.ooc_ssyrk.argtypes = [ch, ch, i64, i64, flt, vp, i64, flt, vp, i64, sz, po, ps]
    lib.ooc_schedule_gemmt.argtypes = [ch, i64, i64, i32, i32, sz, po, ps, ctypes.POINTER(ooc_sched_op), i64,
                                       ctypes.POINTER(i64)]
    lib.ooc_dtrsm.argtypes = [ch, ch, ch, ch, i64, i64, dbl, vp, i64, vp, i64, sz, po, ps]
    lib.ooc_dpotrf.argtypes = [ch, i64, vp, i64, sz, po, ps, ctypes.POINTER(i64)]
    lib.ooc_dgetrf.argtypes = [i64, vp, i64, vp, sz, po, ps, ctypes.POINTER(i64)]
    sp = ctypes.c_void_p
    lib.ooc_session_create.argtypes = [i64, i64, i64, dbl, vp, i64, sz, po, ctypes.POINTER(sp)]
    lib.ooc_session_step.argtypes = [sp, ch, ch, i64, dbl, vp, i64, vp, i64, ps]
    lib.ooc_session_finish.argtypes = [sp, ps]
    lib.ooc_session_free.argtypes = [sp]
    lib.ooc_session_query.argtypes = [sp] + [ctypes.POINTER(i64)] * 4 + [ctypes.POINTER(i32)]
    lib.ooc_schedule_session.argtypes = [i64, i64, i64, i32, sz, po, i32, i32, ps, ctypes.POINTER(ooc_sched_op),
                                         i64, ctypes.POINTER(i64)]
    lib.ooc_pipe_create.argtypes = [ctypes.c_char_p, ctypes.POINTER(sp)]
    lib.ooc_pipe_set.argtypes = [sp, ctypes.c_char_p, dbl]
    lib.ooc_pipe_bind.argtypes = [sp, ctypes.c_char_p, vp, i64, i64, i64, i32]
    lib.ooc_pipe_schedule.argtypes = [sp, sz, ps, ctypes.POINTER(ooc_sched_op), i64, ctypes.POINTER(i64)]
    lib.ooc_pipe_run.argtypes = [sp, sz, ps]
    lib.ooc_pipe_free.argtypes = [sp]
    lib.ooc_query_device.argtypes = [ctypes.POINTER(sz), ctypes.POINTER(dbl), ctypes.POINTER(dbl)]
    lib.ooc_strerror.argtypes = [ctypes.c_int]
    lib.ooc_strerror.restype = ctypes.c_char_p
    lib.ooc_last_error.argtypes = []
    lib.ooc_last_error.restype = ctypes.c_char_p
    for f in ("ooc_dgemm", "ooc_sgemm", "ooc_dgemm_device", "ooc_plan", "ooc_schedule", "ooc_query_device",
              "ooc_dgemmt", "ooc_dsyrk", "ooc_ssyrk", "ooc_schedule_gemmt", "ooc_dtrsm", "ooc_dpotrf", "ooc_dgetrf",
              "ooc_session_create", "ooc_session_step", "ooc_session_finish", "ooc_session_free",
              "ooc_session_query", "ooc_schedule_session", "ooc_pipe_create", "ooc_pipe_set", "ooc_pipe_bind",
              "ooc_pipe_schedule", "ooc_pipe_run", "ooc_pipe_free"):
        getattr(lib, f).restype = ctypes.c_int
    if path is None:
        _lib = lib
    return lib


def _opts(form=0, depth=0, c_buffers=0, slices=0, mb=0, nb=0, kb=0, flags=0, workspace=None,
          workspace_bytes=0, b_buffers=0):
    o = ooc_opts()
    o.form, o.depth, o.c_buffers, o.slices = form, depth, c_buffers, slices
    o.mb, o.nb, o.kb, o.flags = mb, nb, kb, flags
    o.b_buffers = b_buffers
    o.workspace = workspace
    o.workspace_bytes = workspace_bytes
    return o


def make_opts(**kw):
    """An ooc_opts with the given fields (the rest zero = automatic)."""
    return _opts(**kw)


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return x.ctypes.data


def _ld(x):
    """Leading dimension (elements between rows) of a row-major 2-D tensor / array whose rows
    are contiguous; raises ValueError for views with strided rows (the C ABI cannot express them)."""
    if hasattr(x, "stride"):
        if x.dim() == 2 and x.shape[1] > 1 and x.stride(1) != 1:
            raise ValueError("rows must be contiguous (stride 1 along the last dimension), got strides %s"
                             % (tuple(x.stride()),))
        return x.stride(0) if x.dim() == 2 and x.shape[0] > 1 else max(1, x.shape[-1])
    if x.ndim == 2 and x.shape[1] > 1 and x.strides[1] != x.itemsize:
        raise ValueError("rows must be contiguous (stride 1 along the last dimension), got strides %s"
                         % (tuple(x.strides),))
    return x.strides[0] // x.itemsize if x.shape[0] > 1 else max(1, x.shape[-1])


def _check(rc, fn):
    if rc != OOC_OK:
        raise OocError(rc, fn)


def ooc_dgemm(transA, transB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, budget, opts=None,
              stats=None):
    """C ABI ooc_dgemm; returns the status code (pointers may be tensors/arrays or ints)."""
    lib = load()
    return lib.ooc_dgemm(transA.encode(), transB.encode(), M, N, K, alpha, _ptr(A), lda, _ptr(B), ldb,
                         beta, _ptr(C), ldc, budget, ctypes.byref(opts) if opts is not None else None,
                         ctypes.byref(stats) if stats is not None else None)


def ooc_sgemm(transA, transB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, budget, opts=None,
              stats=None):
    """C ABI ooc_sgemm; returns the status code."""
    lib = load()
    return lib.ooc_sgemm(transA.encode(), transB.encode(), M, N, K, alpha, _ptr(A), lda, _ptr(B), ldb,
                         beta, _ptr(C), ldc, budget, ctypes.byref(opts) if opts is not None else None,
                         ctypes.byref(stats) if stats is not None else None)


def _ref(x):
    return ctypes.byref(x) if x is not None else None


def ooc_dgemmt(uplo, transA, transB, N, K, alpha, A, lda, B, ldb, beta, C, ldc, budget, opts=None, stats=None):
    """C ABI ooc_dgemmt (triangular part of C = alpha op(A) op(B) + beta C); returns the status code."""
    return load().ooc_dgemmt(uplo.encode(), transA.encode(), transB.encode(), N, K, alpha, _ptr(A), lda, _ptr(B),
                             ldb, beta, _ptr(C), ldc, budget, _ref(opts), _ref(stats))


def ooc_dsyrk(uplo, trans, N, K, alpha, A, lda, beta, C, ldc, budget, opts=None, stats=None):
    """C ABI ooc_dsyrk; returns the status code."""
    return load().ooc_dsyrk(uplo.encode(), trans.encode(), N, K, alpha, _ptr(A), lda, beta, _ptr(C), ldc, budget,
                            _ref(opts), _ref(stats))


def ooc_ssyrk(uplo, trans, N, K, alpha, A, lda, beta, C, ldc, budget, opts=None, stats=None):
    """C ABI ooc_ssyrk (BF16x3 form); returns the status code."""
    return load().ooc_ssyrk(uplo.encode(), trans.encode(), N, K, alpha, _ptr(A), lda, beta, _ptr(C), ldc, budget,
                            _ref(opts), _ref(stats))


def ooc_dtrsm(side, uplo, transA, diag, M, N, alpha, A, lda, B, ldb, budget, opts=None, stats=None):
    """C ABI ooc_dtrsm (X overwrites B); returns the status code."""
    return load().ooc_dtrsm(side.encode(), uplo.encode(), transA.encode(), diag.encode(), M, N, alpha, _ptr(A), lda,
                            _ptr(B), ldb, budget, _ref(opts), _ref(stats))


def ooc_dpotrf(uplo, N, A, lda, budget, opts=None, stats=None):
    """C ABI ooc_dpotrf; returns (status code, info)."""
    info = ctypes.c_int64(0)
    rc = load().ooc_dpotrf(uplo.encode(), N, _ptr(A), lda, budget, _ref(opts), _ref(stats), ctypes.byref(info))
    return rc, info.value


class Session:
    """A C-ABI session (ooc_session_*): one C accumulated over several calls."""

    def __init__(self, M, N, C, ldc, beta, budget, k_hint=0, opts=None):
        self._h = ctypes.c_void_p()
        self.rc = load().ooc_session_create(M, N, k_hint, beta, _ptr(C), ldc, budget, _ref(opts),
                                            ctypes.byref(self._h))

    def step(self, transA, transB, K, alpha, A, lda, B, ldb, stats=None):
        return load().ooc_session_step(self._h, transA.encode(), transB.encode(), K, alpha, _ptr(A), lda, _ptr(B),
                                       ldb, _ref(stats))

    def query(self):
        v = [ctypes.c_int64() for _ in range(4)] + [ctypes.c_int32()]
        _check(load().ooc_session_query(self._h, *[ctypes.byref(x) for x in v]), "ooc_session_query")
        return dict(mb=v[0].value, nb=v[1].value, resident_blocks=v[2].value, blocks=v[3].value, calls=v[4].value)

    def finish(self, stats=None):
        h, self._h = self._h, ctypes.c_void_p()
        return load().ooc_session_finish(h, _ref(stats))

    def free(self):
        if self._h:
            load().ooc_session_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.free()   # a session dropped without finish() releases its arena (nothing is written back)
        except Exception:
            pass


class Pipe:
    """A pipeline description compiled by the library (ooc_pipe_*)."""

    def __init__(self, description):
        self._h = ctypes.c_void_p()
        self.rc = load().ooc_pipe_create(description.encode(), ctypes.byref(self._h))

    def set(self, name, value):
        return load().ooc_pipe_set(self._h, name.encode(), float(value))

    def bind(self, operand, host=None, rows=None, cols=None, ld=None, elem_bytes=8):
        """Bind an operand to a pinned host tensor / array (or to dimensions only, for schedule())."""
        if host is not None and rows is None:
            rows, cols = host.shape
            ld = _ld(host)
            elem_bytes = host.element_size() if hasattr(host, "element_size") else host.itemsize
        return load().ooc_pipe_bind(self._h, operand.encode(), _ptr(host), rows, cols, ld or cols, elem_bytes)

    def schedule(self, budget):
        lib = load()
        st = ooc_stats()
        ops = _export(lambda buf, cap, n: lib.ooc_pipe_schedule(self._h, budget, ctypes.byref(st), buf, cap, n),
                      "ooc_pipe_schedule")
        return st.as_dict(), ops

    def run(self, budget, stats=None):
        return load().ooc_pipe_run(self._h, budget, _ref(stats))

    def free(self):
        if self._h:
            load().ooc_pipe_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


# The out-of-core GEMM of Section IV written in the pipeline language: block
# column j outer, block row i inner, K chunks innermost; C loaded only for beta != 0.
MMOOC_PIPELINE = """
operand A tile mb kb ring ra
operand B tile kb nb ring rb
operand C tile mb nb ring rc
for j in 0 .. tcols(C)
  for i in 0 .. trows(C)
    load C[i, j] if beta_nz
    alloc C[i, j] unless beta_nz
    for k in 0 .. tcols(A)
      load A[i, k]
      load B[k, j]
      run gemm C[i, j] A[i, k] B[k, j]
    end
    store C[i, j]
  end
end
"""


def ooc_schedule_session(M, N, K, beta_nonzero, budget, opts, resident_blocks, call):
    """C ABI ooc_schedule_session; returns (plan dict, list of operation dicts)."""
    lib = load()
    st = ooc_stats()
    o = _ref(opts)
    ops = _export(lambda buf, cap, n: lib.ooc_schedule_session(M, N, K, int(bool(beta_nonzero)), budget, o,
                                                               resident_blocks, call, ctypes.byref(st), buf, cap, n),
                  "ooc_schedule_session")
    return st.as_dict(), ops


def ooc_dgetrf(N, A, lda, ipiv, budget, opts=None, stats=None):
    """C ABI ooc_dgetrf; ipiv: an int64 array of N entries (numpy or tensor); returns (status, info)."""
    info = ctypes.c_int64(0)
    rc = load().ooc_dgetrf(N, _ptr(A), lda, _ptr(ipiv), budget, _ref(opts), _ref(stats), ctypes.byref(info))
    return rc, info.value


def ooc_dgemm_batched(descs, budget, opts=None, stats=None):
    """C ABI ooc_dgemm_batched on a list of ooc_gemm_desc; returns the status code."""
    lib = load()
    f = lib.ooc_dgemm_batched
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int32, ctypes.POINTER(ooc_gemm_desc), ctypes.c_size_t, ctypes.POINTER(ooc_opts),
                  ctypes.POINTER(ooc_stats)]
    arr = (ooc_gemm_desc * max(1, len(descs)))(*descs)
    return f(len(descs), arr, budget, ctypes.byref(opts) if opts is not None else None,
             ctypes.byref(stats) if stats is not None else None)


def gemm_desc(transA, transB, A, B, C, alpha=1.0, beta=0.0):
    """An ooc_gemm_desc for pinned host tensors (shapes as in dgemm): float64 for
    ooc_dgemm_batched, float64 or float32 for ooc_autotune (whose elem_bytes says which)."""
    M, N, K = _shape_args(transA, transB, A, B, C)
    d = ooc_gemm_desc()
    d.transA, d.transB = transA.encode(), transB.encode()
    d.M, d.N, d.K = M, N, K
    d.alpha, d.beta = alpha, beta
    d.A, d.lda = _ptr(A), _ld(A)
    d.B, d.ldb = _ptr(B), _ld(B)
    d.C, d.ldc = _ptr(C), _ld(C)
    return d


def ooc_dgemm_device(transA, transB, M, N, K, alpha, dA, lda, dB, ldb, beta, dC, ldc, stream=None):
    """C ABI ooc_dgemm_device on device pointers; returns the status code."""
    lib = load()
    return lib.ooc_dgemm_device(transA.encode(), transB.encode(), M, N, K, alpha, _ptr(dA), lda, _ptr(dB),
                                ldb, beta, _ptr(dC), ldc, stream)


def ooc_dgemm_noalloc(transA, transB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, budget, stream=None):
    """C ABI ooc_dgemm_noalloc (no device allocation; budget <= OOC_NOALLOC_MAX_BYTES); returns the status."""
    lib = load()
    f = lib.ooc_dgemm_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_char, ctypes.c_char, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_double,
                  ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_double,
                  ctypes.c_void_p, ctypes.c_int64, ctypes.c_size_t, ctypes.c_void_p]
    return f(transA.encode(), transB.encode(), M, N, K, alpha, _ptr(A), lda, _ptr(B), ldb, beta, _ptr(C), ldc,
             budget, stream)


OOC_NOALLOC_MAX_BYTES = 32 << 20


def ooc_plan(M, N, K, elem_bytes, beta_nonzero, budget, opts=None):
    """C ABI ooc_plan; returns the plan as a dict (raises on error)."""
    lib = load()
    st = ooc_stats()
    _check(lib.ooc_plan(M, N, K, elem_bytes, int(bool(beta_nonzero)), budget,
                        ctypes.byref(opts) if opts is not None else None, ctypes.byref(st)), "ooc_plan")
    return st.as_dict()


def ooc_schedule(M, N, K, elem_bytes, beta_nonzero, budget, opts=None):
    """C ABI ooc_schedule; returns the issued operations as a list of dicts."""
    lib = load()
    o = _ref(opts)
    return _export(lambda buf, cap, n: lib.ooc_schedule(M, N, K, elem_bytes, int(bool(beta_nonzero)), budget, o,
                                                        buf, cap, n), "ooc_schedule")


def ooc_schedule_gemmt(uplo, N, K, elem_bytes, beta_nonzero, budget, opts=None):
    """C ABI ooc_schedule_gemmt; returns (plan dict, list of operation dicts)."""
    lib = load()
    o = _ref(opts)
    st = ooc_stats()
    ops = _export(lambda buf, cap, n: lib.ooc_schedule_gemmt(uplo.encode(), N, K, elem_bytes,
                                                             int(bool(beta_nonzero)), budget, o, ctypes.byref(st),
                                                             buf, cap, n), "ooc_schedule_gemmt")
    return st.as_dict(), ops


def _export(call, name):
    n = ctypes.c_int64(0)
    rc = call(None, 0, ctypes.byref(n))
    if rc not in (OOC_OK, OOC_ERR_CAPACITY):
        _check(rc, name)
    buf = (ooc_sched_op * max(1, n.value))()
    _check(call(buf, n.value, ctypes.byref(n)), name)
    out = []
    for k in range(n.value):
        e = buf[k]
        out.append(dict(kind=e.kind, stream=e.stream, event=e.event, nreads=e.nreads,
                        write_slot=e.write_slot, write_tag=tuple(e.write_tag),
                        read_slot=[e.read_slot[r] for r in range(e.nreads)],
                        read_tag=[tuple(e.read_tag[r]) for r in range(e.nreads)]))
    return out


def _fp(a):
    return ctypes.cast(ctypes.c_void_p(_ptr(a)), ctypes.POINTER(ctypes.c_float))


def ooc_plan_candidates(M, N, K, elem_bytes, beta_nonzero, budget, opts=None, capacity=32):
    """C ABI ooc_plan_candidates; returns a list of ooc_plan_candidate."""
    lib = load()
    f = lib.ooc_plan_candidates
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int64] * 3 + [ctypes.c_int32, ctypes.c_int32, ctypes.c_size_t, ctypes.POINTER(ooc_opts),
                                         ctypes.POINTER(ooc_plan_candidate), ctypes.c_int32,
                                         ctypes.POINTER(ctypes.c_int32)]
    buf = (ooc_plan_candidate * capacity)()
    n = ctypes.c_int32(0)
    _check(f(M, N, K, elem_bytes, int(bool(beta_nonzero)), budget, ctypes.byref(opts) if opts is not None else None,
             buf, capacity, ctypes.byref(n)), "ooc_plan_candidates")
    return [buf[i] for i in range(n.value)]


def ooc_autotune(desc, elem_bytes, budget, opts=None, max_candidates=16):
    """C ABI ooc_autotune; returns [(candidate, seconds)] in candidate order."""
    lib = load()
    f = lib.ooc_autotune
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.POINTER(ooc_gemm_desc), ctypes.c_int32, ctypes.c_size_t, ctypes.POINTER(ooc_opts),
                  ctypes.c_int32, ctypes.POINTER(ooc_plan_candidate), ctypes.POINTER(ctypes.c_double),
                  ctypes.POINTER(ctypes.c_int32)]
    buf = (ooc_plan_candidate * max_candidates)()
    sec = (ctypes.c_double * max_candidates)()
    n = ctypes.c_int32(0)
    _check(f(ctypes.byref(desc), elem_bytes, budget, ctypes.byref(opts) if opts is not None else None,
             max_candidates, buf, sec, ctypes.byref(n)), "ooc_autotune")
    return [(buf[i], sec[i]) for i in range(n.value)]


def ooc_mlp_forward(params, X):
    """C ABI ooc_mlp_forward on float32 numpy arrays; returns predictions."""
    import numpy as np
    lib = load()
    params = np.ascontiguousarray(params, dtype=np.float32)
    X = np.ascontiguousarray(X, dtype=np.float32)
    y = np.empty(X.shape[0], dtype=np.float32)
    f = lib.ooc_mlp_forward
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
    _check(f(params.ctypes.data, X.ctypes.data, X.shape[0], y.ctypes.data), "ooc_mlp_forward")
    return y


def ooc_mlp_loss_grad(params, X, t):
    """C ABI ooc_mlp_loss_grad; returns (loss, grad)."""
    import numpy as np
    lib = load()
    params = np.ascontiguousarray(params, dtype=np.float32)
    X = np.ascontiguousarray(X, dtype=np.float32)
    t = np.ascontiguousarray(t, dtype=np.float32)
    g = np.empty_like(params)
    loss = ctypes.c_float(0)
    f = lib.ooc_mlp_loss_grad
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int64, ctypes.c_void_p, ctypes.POINTER(ctypes.c_float)]
    _check(f(params.ctypes.data, X.ctypes.data, t.ctypes.data, X.shape[0], g.ctypes.data, ctypes.byref(loss)),
           "ooc_mlp_loss_grad")
    return loss.value, g


def ooc_mlp_train(params, X, t, epochs=200, batch=64, lr=3e-3, seed=1, weight_decay=0.0):
    """C ABI ooc_mlp_train; returns (trained params, final loss)."""
    import numpy as np
    lib = load()
    p = np.array(params, dtype=np.float32, copy=True)
    X = np.ascontiguousarray(X, dtype=np.float32)
    t = np.ascontiguousarray(t, dtype=np.float32)
    loss = ctypes.c_float(0)
    f = lib.ooc_mlp_train
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_float,
                                          ctypes.c_float, ctypes.c_uint64, ctypes.POINTER(ctypes.c_float)]
    _check(f(p.ctypes.data, X.ctypes.data, t.ctypes.data, X.shape[0], epochs, batch, lr, weight_decay, seed,
             ctypes.byref(loss)), "ooc_mlp_train")
    return p, loss.value


def ooc_costmodel_set(params):
    """C ABI ooc_costmodel_set (None clears)."""
    import numpy as np
    lib = load()
    f = lib.ooc_costmodel_set
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64]
    if params is None:
        _check(f(None, 0), "ooc_costmodel_set")
        return
    global _model_keepalive
    _model_keepalive = np.ascontiguousarray(params, dtype=np.float32)
    _check(f(_model_keepalive.ctypes.data, _model_keepalive.size), "ooc_costmodel_set")


_model_keepalive = None


def ooc_query_device():
    """C ABI ooc_query_device: (free_bytes, h2d_gbps, d2h_gbps)."""
    lib = load()
    f, h, d = ctypes.c_size_t(0), ctypes.c_double(0), ctypes.c_double(0)
    _check(lib.ooc_query_device(ctypes.byref(f), ctypes.byref(h), ctypes.byref(d)), "ooc_query_device")
    return f.value, h.value, d.value


def ooc_query_fp64_peak(seconds=1.0):
    """C ABI ooc_query_fp64_peak: the device's measured FP64 (mma.sync f64) peak in TFLOP/s."""
    lib = load()
    f = lib.ooc_query_fp64_peak
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_double, ctypes.POINTER(ctypes.c_double)]
    t = ctypes.c_double(0)
    _check(f(seconds, ctypes.byref(t)), "ooc_query_fp64_peak")
    return t.value


def ooc_strerror(code):
    return load().ooc_strerror(code).decode()


def ooc_last_error():
    return load().ooc_last_error().decode()


# ------------------------------------------------------------------ helpers --
def _shape_args(transA, transB, A, B, C, itemsize=(4, 8)):
    """M, N, K of C = op(A) op(B) for 2-D operands; ValueError when the shapes do not chain, or the
    three operands are not floating point of one element size allowed by the call (8 for dgemm,
    4 for sgemm, either for a batched / autotune descriptor)."""
    allowed = (itemsize,) if isinstance(itemsize, int) else tuple(itemsize)
    sizes = set()
    for name, x in (("A", A), ("B", B), ("C", C)):
        if len(x.shape) != 2:
            raise ValueError("%s must be 2-D, got shape %s" % (name, tuple(x.shape)))
        es = x.element_size() if hasattr(x, "element_size") else x.itemsize
        if es not in allowed or not _is_float(x):
            raise ValueError("%s must hold floating-point elements of %s bytes, got %s" % (
                name, " or ".join(map(str, allowed)), x.dtype))
        sizes.add(es)
    if len(sizes) != 1:
        raise ValueError("A, B and C must have one element type")
    M = A.shape[0] if transA in "Nn" else A.shape[1]
    K = A.shape[1] if transA in "Nn" else A.shape[0]
    N = B.shape[1] if transB in "Nn" else B.shape[0]
    KB = B.shape[0] if transB in "Nn" else B.shape[1]
    if KB != K or tuple(C.shape) != (M, N):
        raise ValueError("shapes do not chain: op(A) %dx%d, op(B) %dx%d, C %s" % (M, K, KB, N, tuple(C.shape)))
    return M, N, K


def _is_float(x):
    if hasattr(x, "is_floating_point"):
        return x.is_floating_point() and not x.is_complex()
    return x.dtype.kind == "f"


def dgemm(A, B, C, alpha=1.0, beta=0.0, budget=4 << 30, transA="N", transB="N", opts=None):
    """In place C = alpha*op(A)*op(B) + beta*C on pinned float64 host tensors; returns stats dict."""
    M, N, K = _shape_args(transA, transB, A, B, C, 8)
    st = ooc_stats()
    _check(ooc_dgemm(transA, transB, M, N, K, alpha, A, _ld(A), B, _ld(B), beta, C, _ld(C), budget,
                     opts, st), "ooc_dgemm")
    return st.as_dict()


def sgemm(A, B, C, alpha=1.0, beta=0.0, budget=4 << 30, transA="N", transB="N", opts=None):
    """In place FP32 C = alpha*op(A)*op(B) + beta*C (BF16x3 form) on pinned float32 host tensors."""
    M, N, K = _shape_args(transA, transB, A, B, C, 4)
    st = ooc_stats()
    _check(ooc_sgemm(transA, transB, M, N, K, alpha, A, _ld(A), B, _ld(B), beta, C, _ld(C), budget,
                     opts, st), "ooc_sgemm")
    return st.as_dict()
