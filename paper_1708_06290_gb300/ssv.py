"""Python binding of ``libssv.so`` (the C ABI of ``include/ssv.h``).

Argument marshalling only: every step of the reduction and the solve runs in
the library's CUDA kernels.  PyTorch provides device memory and streams; the
tensors passed in must live on the current CUDA device.  Matrices are
column-major: a (rows, cols) tensor with stride (1, ld), ld >= rows, e.g. made
by :func:`colmajor`.  There is no CPU path: without the built library and a
CUDA device every call raises.
"""
import ctypes
import os

import torch

from . import build as _build

SSV_OK = 0
SSV_EINVAL = -1
SSV_ENOMEM = -2
SSV_ECUDA = -3
SSV_ETIMEOUT = -4
SSV_ENOTSUP = -5
SSV_ESCRATCH = -6

SHIFT_OK = 0
SHIFT_SINGULAR = 1
SHIFT_NOT_CONVERGED = 2
SHIFT_NONFINITE = 3

FP64 = 0
MIXED = 1
DFLOAT = 2

G = 0
TF = 1
XHAT = 2
X = 3

_MODES = {"g": G, "tf": TF, "xhat": XHAT, "x": X}
SPLIT = 3
_PREC = {"fp64": FP64, "mixed": MIXED, "dfloat": DFLOAT, "split": SPLIT}


class SsvError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        msg = "%s failed: %s (%d)" % (what, strerror(code), code)
        if code == SSV_ECUDA and _lib is not None:
            msg += ", cuda error %d" % _lib.ssv_last_cuda_error()
        super().__init__(msg)


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("mode", ctypes.c_int), ("nb", ctypes.c_int),
                ("max_refine", ctypes.c_int), ("tol", ctypes.c_double),
                ("panel", ctypes.c_int), ("first", ctypes.c_int)]


EXPORTS = ("ssv_default_opts", "ssv_reduce", "ssv_solve", "ssv_apply_q", "ssv_get_reduced",
           "ssv_dims", "ssv_footprint", "ssv_handle_bytes", "ssv_destroy", "ssv_strerror",
           "ssv_last_cuda_error", "ssv_kernel_launches", "ssv_peak_probe", "ssv_load_reduced", "ssv_solve_noalloc", "ssv_solve_many",
           "ssv_batch_create", "ssv_batch_run", "ssv_batch_destroy", "ssv_autotune",
           "ssv_trace_enable", "ssv_trace_reset", "ssv_trace_read", "ssv_selftest_barrier",
           "ssv_solve_rhs", "ssv_solve_trans", "ssv_givens_schedule", "ssv_tf_norm2",
           "ssv_backward_error", "ssv_refine_counts", "ssv_pool_trim", "ssv_reduce_arith")

_lib = None


def lib_path():
    return _build.LIB


def load(build_if_missing=True):
    """Load (building first if needed) the shared library and declare its ABI."""
    global _lib
    if _lib is not None:
        return _lib
    # SSV_LIBRARY may name another build of the same library (the bounds-checked
    # debug copy); it is used as is, never built here
    path = os.environ.get("SSV_LIBRARY") or _build.LIB
    if path == _build.LIB and build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError("libssv.so is not built (%s); run paper_1708_06290_gb300/build.py" % path)
    L = ctypes.CDLL(path)
    P = ctypes.c_void_p
    I = ctypes.c_int
    LL = ctypes.c_longlong
    L.ssv_default_opts.argtypes = [ctypes.POINTER(Opts)]
    L.ssv_default_opts.restype = None
    L.ssv_reduce.argtypes = [I, I, I, P, LL, P, LL, P, LL, P, ctypes.POINTER(P)]
    L.ssv_reduce_arith.argtypes = [I, I, I, P, LL, P, LL, P, LL, I, P, ctypes.POINTER(P)]
    L.ssv_load_reduced.argtypes = [I, I, I, P, LL, P, LL, P, LL, P, ctypes.POINTER(P)]
    L.ssv_solve.argtypes = [P, I, P, ctypes.POINTER(Opts), P, LL, P, P, P]
    L.ssv_solve_noalloc.argtypes = [P, I, P, ctypes.POINTER(Opts), P, LL, P, P]
    L.ssv_solve_rhs.argtypes = [P, I, P, P, LL, ctypes.POINTER(Opts), P, LL, P, P]
    L.ssv_solve_trans.argtypes = [P, I, P, P, LL, ctypes.POINTER(Opts), P, LL, P, P]
    L.ssv_givens_schedule.argtypes = [I, I, P, I, P, I, ctypes.POINTER(I)]
    L.ssv_tf_norm2.argtypes = [P, I, P, ctypes.POINTER(Opts), P, P, P]
    L.ssv_backward_error.argtypes = [P, I, P, P, LL, I, P, P]
    L.ssv_refine_counts.argtypes = [ctypes.POINTER(LL), ctypes.POINTER(LL), I]
    L.ssv_pool_trim.argtypes = [ctypes.c_size_t]
    L.ssv_pool_trim.restype = I
    PP = ctypes.POINTER(ctypes.c_void_p)
    L.ssv_solve_many.argtypes = [I, PP, ctypes.POINTER(I), PP, ctypes.POINTER(Opts), PP,
                                 ctypes.POINTER(LL), PP, P]
    L.ssv_batch_create.argtypes = [I, PP, ctypes.POINTER(I), PP, ctypes.POINTER(Opts), PP,
                                   ctypes.POINTER(LL), PP, ctypes.POINTER(P)]
    L.ssv_batch_run.argtypes = [P, P]
    L.ssv_batch_destroy.argtypes = [P]
    L.ssv_batch_destroy.restype = None
    L.ssv_autotune.argtypes = [P, I, P, ctypes.POINTER(Opts), P, LL, P, ctypes.POINTER(I),
                               ctypes.POINTER(ctypes.c_float)]
    L.ssv_selftest_barrier.argtypes = [LL, P]
    L.ssv_selftest_barrier.restype = I
    L.ssv_trace_enable.argtypes = [I]
    L.ssv_trace_reset.argtypes = []
    L.ssv_trace_read.argtypes = [I, ctypes.c_char_p, I, ctypes.POINTER(ctypes.c_float),
                                 ctypes.POINTER(I), ctypes.POINTER(I)]
    for f in ("ssv_trace_enable", "ssv_trace_reset", "ssv_trace_read", "ssv_selftest_barrier",
           "ssv_solve_rhs", "ssv_solve_trans", "ssv_givens_schedule", "ssv_tf_norm2",
           "ssv_backward_error", "ssv_refine_counts"):
        getattr(L, f).restype = I
    L.ssv_apply_q.argtypes = [P, I, P, LL, P, LL, P]
    L.ssv_get_reduced.argtypes = [P, P, LL, P, LL, P, LL, P]
    L.ssv_dims.argtypes = [P, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I)]
    L.ssv_footprint.argtypes = [I, I, I, I, ctypes.POINTER(Opts), ctypes.POINTER(ctypes.c_size_t)]
    L.ssv_handle_bytes.argtypes = [I, I, I, ctypes.POINTER(ctypes.c_size_t)]
    L.ssv_destroy.argtypes = [P]
    L.ssv_destroy.restype = None
    L.ssv_strerror.argtypes = [I]
    L.ssv_strerror.restype = ctypes.c_char_p
    L.ssv_last_cuda_error.argtypes = []
    L.ssv_kernel_launches.argtypes = []
    L.ssv_kernel_launches.restype = ctypes.c_longlong
    L.ssv_peak_probe.argtypes = [I, P, ctypes.POINTER(ctypes.c_double)]
    for f in ("ssv_reduce", "ssv_load_reduced", "ssv_solve", "ssv_solve_noalloc",
              "ssv_solve_many", "ssv_batch_create", "ssv_batch_run", "ssv_autotune", "ssv_apply_q", "ssv_get_reduced", "ssv_dims",
              "ssv_footprint", "ssv_handle_bytes", "ssv_last_cuda_error", "ssv_peak_probe"):
        getattr(L, f).restype = I
    _lib = L
    return L


def strerror(code):
    if _lib is None:
        return "code %d" % code
    return _lib.ssv_strerror(code).decode()


def _check(rc, what):
    if rc != SSV_OK:
        raise SsvError(rc, what)


def colmajor(t):
    """Column-major copy of a 2-D tensor (stride (1, rows))."""
    return t.t().contiguous().t()


def _ld(t, rows):
    """Leading dimension of a column-major 2-D tensor (strides of size-1 dims are ignored)."""
    if t.dim() != 2:
        raise ValueError("expected a 2-D tensor")
    if t.shape[0] > 1 and t.stride(0) != 1:
        raise ValueError("tensor must be column-major (stride(0) == 1)")
    ld = t.stride(1) if t.shape[1] > 1 else max(rows, 1)
    ld = max(ld, 1)
    if t.shape[1] > 1 and ld < max(rows, 1):
        raise ValueError("leading dimension %d < rows %d" % (ld, rows))
    return ld


def _stream_ptr(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _need_cuda(t, dtype, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise ValueError("%s must be %s" % (name, dtype))


_PANELS = {"householder": 0, "givens": 1}


_FIRST = {"dfloat": 0, "c64": 1, "tensor": 2}


def opts(precision="fp64", mode="g", nb=0, max_refine=8, tol=1e-13, panel="householder",
         first="tensor"):
    o = Opts()
    load().ssv_default_opts(ctypes.byref(o))
    o.precision = _PREC[precision] if isinstance(precision, str) else int(precision)
    o.mode = _MODES[mode] if isinstance(mode, str) else int(mode)
    o.nb = nb
    o.max_refine = max_refine
    o.tol = tol
    o.panel = _PANELS[panel] if isinstance(panel, str) else int(panel)
    o.first = _FIRST[first] if isinstance(first, str) else int(first)
    return o


def pool_trim(keep_bytes=0):
    """Return the library's pooled scratch memory on the current device beyond keep_bytes."""
    _check(load().ssv_pool_trim(int(keep_bytes)), "ssv_pool_trim")


def refine_counts(reset=False):
    """(correction shift-sweeps, FP64 re-solves) of the mixed path on the current
    device, accumulated since the last reset (synchronises the device)."""
    L = load()
    c = ctypes.c_longlong()
    r = ctypes.c_longlong()
    _check(L.ssv_refine_counts(ctypes.byref(c), ctypes.byref(r), 1 if reset else 0),
           "ssv_refine_counts")
    return int(c.value), int(r.value)


def givens_schedule(rows, m):
    """The library's greedy Givens schedule (Algorithm 9) for a rows x (rows + m)
    block: list of steps, each a list of (r, c1, c2), 1-based.  Host only."""
    L = load()
    nrot = rows * m
    rot = (ctypes.c_int * (3 * max(nrot, 1)))()
    off = (ctypes.c_int * (nrot + 2))()
    ns = ctypes.c_int()
    rc = L.ssv_givens_schedule(rows, m, ctypes.cast(rot, ctypes.c_void_p), nrot,
                               ctypes.cast(off, ctypes.c_void_p), nrot + 1, ctypes.byref(ns))
    _check(min(rc, 0), "ssv_givens_schedule")
    return [[tuple(rot[3 * j:3 * j + 3]) for j in range(off[t], off[t + 1])] for t in range(ns.value)]


class Handle:
    """A reduced system (H, R, Ct, Q) resident on the GPU."""

    def __init__(self, ptr, n, m, p, stream):
        self._ptr = ptr
        self.n, self.m, self.p = n, m, p
        self._stream = stream

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def close(self):
        if getattr(self, "_ptr", None):
            _lib.ssv_destroy(self._ptr)
            self._ptr = None

    @property
    def ptr(self):
        if not self._ptr:
            raise RuntimeError("handle is closed")
        return self._ptr

    def out_rows(self, mode):
        return self.p if _MODES.get(mode, mode) in (G, TF) else self.n

    def solve(self, shifts, mode="g", precision="fp64", nb=0, max_refine=8, tol=1e-13,
              out=None, status=None, resid=None, want_resid=False, stream=None, panel="householder",
              first="tensor"):
        """Solve all shifts.  Returns (out, status, resid).

        out is a column-major complex128 (rows, s*m) tensor, rows = p for
        mode g/tf and n for xhat/x; block j holds the result for shifts[j].
        """
        L = load()
        _need_cuda(shifts, torch.complex128, "shifts")
        s = shifts.numel()
        o = opts(precision, mode, nb, max_refine, tol, panel, first)
        rows = self.out_rows(o.mode)
        dev = shifts.device
        if out is None:
            out = torch.empty((s * self.m, max(rows, 1)), dtype=torch.complex128, device=dev).t()
        _need_cuda(out, torch.complex128, "out")
        ldo = _ld(out, rows)
        if status is None:
            status = torch.empty(s, dtype=torch.int32, device=dev)
        if resid is None and want_resid:
            resid = torch.empty(s, dtype=torch.float64, device=dev)
        rc = L.ssv_solve(self.ptr, s, ctypes.c_void_p(shifts.data_ptr()), ctypes.byref(o),
                         ctypes.c_void_p(out.data_ptr()), ldo,
                         ctypes.c_void_p(status.data_ptr()),
                         ctypes.c_void_p(resid.data_ptr()) if resid is not None else None,
                         _stream_ptr(stream))
        _check(rc, "ssv_solve")
        return out, status, resid

    def solve_rhs(self, shifts, bhat, mode="x", nb=0, out=None, status=None, stream=None):
        """One right-hand side B bhat[:, l] per shift (Sec. 3.3).  bhat: complex128
        (m, s) CUDA tensor (column-major or contiguous columns).  Returns (out, status)
        with out (rows, s): rows = n for x / xhat, p for g / tf."""
        L = load()
        _need_cuda(shifts, torch.complex128, "shifts")
        _need_cuda(bhat, torch.complex128, "bhat")
        s = shifts.numel()
        if tuple(bhat.shape) != (self.m, s):
            raise ValueError("bhat must be (m, s) = (%d, %d)" % (self.m, s))
        o = opts("fp64", mode, nb, 0, 0.0)
        rows = self.out_rows(o.mode)
        dev = shifts.device
        if out is None:
            out = torch.empty((s, max(rows, 1)), dtype=torch.complex128, device=dev).t()
        _need_cuda(out, torch.complex128, "out")
        if status is None:
            status = torch.empty(s, dtype=torch.int32, device=dev)
        rc = L.ssv_solve_rhs(self.ptr, s, ctypes.c_void_p(shifts.data_ptr()),
                             ctypes.c_void_p(bhat.data_ptr()), _ld(bhat, self.m), ctypes.byref(o),
                             ctypes.c_void_p(out.data_ptr()), _ld(out, rows),
                             ctypes.c_void_p(status.data_ptr()), _stream_ptr(stream))
        _check(rc, "ssv_solve_rhs")
        return out, status

    def solve_trans(self, shifts, chat, mode="x", nb=0, out=None, status=None, stream=None):
        """Transposed systems (A - sigma_l I)^T x_l = C^T chat[:, l] (Sec. 3.3).
        chat: complex128 (p, s) CUDA tensor.  Returns (out, status), out (n, s):
        x_l (mode x) or Q^T x_l (mode xhat)."""
        L = load()
        _need_cuda(shifts, torch.complex128, "shifts")
        _need_cuda(chat, torch.complex128, "chat")
        s = shifts.numel()
        if tuple(chat.shape) != (self.p, s):
            raise ValueError("chat must be (p, s) = (%d, %d)" % (self.p, s))
        o = opts("fp64", mode, nb, 0, 0.0)
        dev = shifts.device
        if out is None:
            out = torch.empty((s, self.n), dtype=torch.complex128, device=dev).t()
        _need_cuda(out, torch.complex128, "out")
        if status is None:
            status = torch.empty(s, dtype=torch.int32, device=dev)
        rc = L.ssv_solve_trans(self.ptr, s, ctypes.c_void_p(shifts.data_ptr()),
                               ctypes.c_void_p(chat.data_ptr()), _ld(chat, self.p), ctypes.byref(o),
                               ctypes.c_void_p(out.data_ptr()), _ld(out, self.n),
                               ctypes.c_void_p(status.data_ptr()), _stream_ptr(stream))
        _check(rc, "ssv_solve_trans")
        return out, status

    def tf_norm2(self, shifts, precision="fp64", nb=0, stream=None):
        """||C (sigma_j I - A)^{-1} B||_2 per shift (structured pseudospectra, Sec. 1).
        Returns (norms float64 (s,), status int32 (s,))."""
        L = load()
        _need_cuda(shifts, torch.complex128, "shifts")
        s = shifts.numel()
        o = opts(precision, "g", nb)
        norms = torch.empty(s, dtype=torch.float64, device=shifts.device)
        status = torch.empty(s, dtype=torch.int32, device=shifts.device)
        rc = L.ssv_tf_norm2(self.ptr, s, ctypes.c_void_p(shifts.data_ptr()), ctypes.byref(o),
                            ctypes.c_void_p(norms.data_ptr()), ctypes.c_void_p(status.data_ptr()),
                            _stream_ptr(stream))
        _check(rc, "ssv_tf_norm2")
        return norms, status

    def backward_error(self, shifts, xhat, method="tensor", stream=None):
        """Normwise backward error of solutions Xhat of (H - sigma_j I) Xhat = R per shift.
        xhat: complex128 (n, s*m) CUDA tensor, column-major blocks (the mode "xhat"
        output layout).  method "tensor" (Ozaki-split BF16 products on the tensor
        cores) or "fp64".  Returns eta float64 (s,)."""
        L = load()
        _need_cuda(shifts, torch.complex128, "shifts")
        _need_cuda(xhat, torch.complex128, "xhat")
        s = shifts.numel()
        meth = {"fp64": 0, "tensor": 1}[method]
        eta = torch.empty(s, dtype=torch.float64, device=shifts.device)
        rc = L.ssv_backward_error(self.ptr, s, ctypes.c_void_p(shifts.data_ptr()),
                                  ctypes.c_void_p(xhat.data_ptr()), _ld(xhat, self.n), meth,
                                  ctypes.c_void_p(eta.data_ptr()), _stream_ptr(stream))
        _check(rc, "ssv_backward_error")
        return eta

    def apply_q(self, xhat, out=None, stream=None):
        L = load()
        _need_cuda(xhat, torch.complex128, "xhat")
        ncols = xhat.shape[1]
        if out is None:
            out = torch.empty((ncols, self.n), dtype=torch.complex128, device=xhat.device).t()
        rc = L.ssv_apply_q(self.ptr, ncols, ctypes.c_void_p(xhat.data_ptr()), _ld(xhat, self.n),
                           ctypes.c_void_p(out.data_ptr()), _ld(out, self.n), _stream_ptr(stream))
        _check(rc, "ssv_apply_q")
        return out

    def reduced(self, stream=None):
        """Return (H, R, Ct) as column-major float64 CUDA tensors (explicit zeros)."""
        L = load()
        dev = torch.device("cuda", torch.cuda.current_device())
        n, m, p = self.n, self.m, self.p
        H = torch.empty((n, n), dtype=torch.float64, device=dev).t()
        R = torch.empty((m, n), dtype=torch.float64, device=dev).t()
        Ct = torch.empty((n, max(p, 1)), dtype=torch.float64, device=dev).t()
        rc = L.ssv_get_reduced(self.ptr, ctypes.c_void_p(H.data_ptr()), n,
                               ctypes.c_void_p(R.data_ptr()), n, ctypes.c_void_p(Ct.data_ptr()),
                               max(p, 1), _stream_ptr(stream))
        _check(rc, "ssv_get_reduced")
        return H, R, Ct[:p]


REDUCE_FP64, REDUCE_TENSOR = 0, 1
_ARITH = {"fp64": REDUCE_FP64, "tensor": REDUCE_TENSOR}


def reduce(A, B, C, stream=None, arith="fp64"):
    """Controller-Hessenberg reduction of (A, B, C) on the GPU; returns a Handle.

    arith: "fp64" (every product on the FP64 pipe, ssv_reduce) or "tensor"
    (two-level blocking with the bulk products as FP64-accurate BF16 digit
    products on the tensor cores, ssv_reduce_arith)."""
    L = load()
    for t, nm in ((A, "A"), (B, "B"), (C, "C")):
        _need_cuda(t, torch.float64, nm)
    if arith not in _ARITH:
        raise ValueError("arith must be one of %s" % sorted(_ARITH))
    n = A.shape[0]
    m = B.shape[1]
    p = C.shape[0]
    h = ctypes.c_void_p()
    rc = L.ssv_reduce_arith(n, m, p, ctypes.c_void_p(A.data_ptr()), _ld(A, n),
                            ctypes.c_void_p(B.data_ptr()), _ld(B, n), ctypes.c_void_p(C.data_ptr()),
                            _ld(C, p) if p > 0 else 1, _ARITH[arith], _stream_ptr(stream),
                            ctypes.byref(h))
    _check(rc, "ssv_reduce_arith")
    return Handle(h, n, m, p, stream)


def load_reduced(H, R, Ct, stream=None):
    """Handle from a stored reduced triple (H m-Hessenberg, R upper triangular, Ct); no Q."""
    L = load()
    for t, nm in ((H, "H"), (R, "R"), (Ct, "Ct")):
        _need_cuda(t, torch.float64, nm)
    n = H.shape[0]
    m = R.shape[1]
    p = Ct.shape[0]
    h = ctypes.c_void_p()
    rc = L.ssv_load_reduced(n, m, p, ctypes.c_void_p(H.data_ptr()), _ld(H, n),
                            ctypes.c_void_p(R.data_ptr()), _ld(R, n),
                            ctypes.c_void_p(Ct.data_ptr()), _ld(Ct, p) if p > 0 else 1,
                            _stream_ptr(stream), ctypes.byref(h))
    _check(rc, "ssv_load_reduced")
    return Handle(h, n, m, p, stream)


def footprint(n, m, p, s, **kw):
    L = load()
    o = opts(**kw)
    b = ctypes.c_size_t()
    _check(L.ssv_footprint(n, m, p, s, ctypes.byref(o), ctypes.byref(b)), "ssv_footprint")
    return b.value


def handle_bytes(n, m, p):
    L = load()
    b = ctypes.c_size_t()
    _check(L.ssv_handle_bytes(n, m, p, ctypes.byref(b)), "ssv_handle_bytes")
    return b.value


def kernel_launches():
    """Kernels the library has launched in this process so far."""
    return load().ssv_kernel_launches()


def peak_probe(kind="fp64", stream=None):
    """Measured FMA throughput of the current GPU in TFLOP/s (kind "fp64" or "fp32")."""
    L = load()
    v = ctypes.c_double()
    _check(L.ssv_peak_probe({"fp64": 0, "fp32": 1}[kind], _stream_ptr(stream), ctypes.byref(v)),
           "ssv_peak_probe")
    return v.value


def _many_args(handles, shifts, outs, statuses):
    n = len(handles)
    VP = ctypes.c_void_p * n
    hs = VP(*[h.ptr for h in handles])
    ss = (ctypes.c_int * n)(*[int(x.numel()) for x in shifts])
    sp = VP(*[x.data_ptr() for x in shifts])
    op = VP(*[o.data_ptr() for o in outs])
    ld = (ctypes.c_longlong * n)(*[_ld(o, o.shape[0]) for o in outs])
    st = VP(*[x.data_ptr() for x in statuses])
    cast = lambda a: ctypes.cast(a, ctypes.POINTER(ctypes.c_void_p))  # noqa: E731
    return n, cast(hs), ss, cast(sp), cast(op), ld, cast(st)


def _alloc_outputs(handles, shifts, mode):
    outs, sts = [], []
    for h, x in zip(handles, shifts):
        rows = h.out_rows(mode)
        outs.append(torch.empty((x.numel() * h.m, max(rows, 1)), dtype=torch.complex128,
                                device=x.device).t())
        sts.append(torch.empty(x.numel(), dtype=torch.int32, device=x.device))
    return outs, sts


def solve_many(handles, shifts, mode="g", precision="fp64", nb=0, stream=None):
    """Solve many systems (list of Handles, list of complex128 CUDA shift vectors) in one
    batched launch.  Returns (outs, statuses), one entry per system."""
    L = load()
    for x in shifts:
        _need_cuda(x, torch.complex128, "shifts")
    outs, sts = _alloc_outputs(handles, shifts, mode)
    o = opts(precision, mode, nb)
    n, hs, ss, sp, op, ld, st = _many_args(handles, shifts, outs, sts)
    _check(L.ssv_solve_many(n, hs, ss, sp, ctypes.byref(o), op, ld, st, _stream_ptr(stream)),
           "ssv_solve_many")
    return outs, sts


class BatchPlan:
    """A fixed FP64 (or double-float) multi-system solve: run() is one kernel launch with constant
    arguments (capturable in a CUDA graph).  Rewrite the shift tensors in place
    between runs; outputs land in .outs / .statuses."""

    def __init__(self, handles, shifts, mode="g", nb=0, precision="fp64"):
        L = load()
        self.handles = list(handles)
        self.shifts = list(shifts)
        self.outs, self.statuses = _alloc_outputs(self.handles, self.shifts, mode)
        o = opts(precision, mode, nb)
        n, hs, ss, sp, op, ld, st = _many_args(self.handles, self.shifts, self.outs, self.statuses)
        b = ctypes.c_void_p()
        _check(L.ssv_batch_create(n, hs, ss, sp, ctypes.byref(o), op, ld, st, ctypes.byref(b)),
               "ssv_batch_create")
        self._b = b

    def run(self, stream=None):
        _check(load().ssv_batch_run(self._b, _stream_ptr(stream)), "ssv_batch_run")

    def close(self):
        if getattr(self, "_b", None):
            load().ssv_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def autotune(handle, shifts, mode="g", precision="fp64", stream=None):
    """Pick and cache the block width n_b for this system; returns (nb, ms)."""
    L = load()
    _need_cuda(shifts, torch.complex128, "shifts")
    rows = handle.out_rows(mode)
    out = torch.empty((shifts.numel() * handle.m, max(rows, 1)), dtype=torch.complex128,
                      device=shifts.device).t()
    o = opts(precision, mode)
    nb = ctypes.c_int()
    ms = ctypes.c_float()
    _check(L.ssv_autotune(handle.ptr, shifts.numel(), ctypes.c_void_p(shifts.data_ptr()),
                          ctypes.byref(o), ctypes.c_void_p(out.data_ptr()), _ld(out, rows),
                          _stream_ptr(stream), ctypes.byref(nb), ctypes.byref(ms)), "ssv_autotune")
    return nb.value, ms.value


def trace(on=True):
    """Enable / disable the library's phase tracer (CUDA events per internal phase)."""
    L = load()
    if on:
        L.ssv_trace_reset()
    L.ssv_trace_enable(1 if on else 0)


def trace_read():
    """{phase: (total_ms, calls)} for the spans recorded since trace(True)."""
    L = load()
    mx, ln = 32, 48
    names = ctypes.create_string_buffer(mx * ln)
    tot = (ctypes.c_float * mx)()
    calls = (ctypes.c_int * mx)()
    cnt = ctypes.c_int()
    _check(L.ssv_trace_read(mx, names, ln, tot, calls, ctypes.byref(cnt)), "ssv_trace_read")
    out = {}
    for k in range(min(cnt.value, mx)):
        nm = names.raw[k * ln:(k + 1) * ln].split(b"\0", 1)[0].decode()
        out[nm] = (tot[k], calls[k])
    return out


def selftest_barrier(spin_limit=100000, stream=None):
    """Run the bounded-barrier timeout self-test; returns the library's return code
    (SSV_ETIMEOUT when the timeout path works)."""
    return load().ssv_selftest_barrier(int(spin_limit), _stream_ptr(stream))
