"""ctypes binding of libp3dfft_gb300.so (include/p3dfft_gb300.h).

Argument marshalling only: every step of the transform runs in the library's
CUDA kernels.  The functions keep the C names; `Plan` wraps them for torch
tensors (device memory and streams come from PyTorch).  If the library has
not been built, the first call raises: there is no other implementation to
fall back to.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libp3dfft_gb300.so")

(P3_OK, P3_ERR_INVALID, P3_ERR_UNSUPPORTED, P3_ERR_NOMEM, P3_ERR_CUDA, P3_ERR_TIMEOUT, P3_ERR_WORKSPACE,
 P3_ERR_HOOK) = range(8)
P3_F32, P3_F64 = 0, 1
P3_FFT, P3_CHEB, P3_EMPTY, P3_SINE = 0, 1, 2, 3
P3_LAYOUT_ZYX, P3_LAYOUT_XYZ = 0, 1
P3_FLAG_TC_SPLIT = 1
P3_FLAG_PADDED_REAL = 2
P3_FLAG_NO_FUSE = 4
P3_FLAG_TUNE = 8
P3_FLAG_NO_TMA = 16
P3_WAIT_FUSED_QUEUE, P3_WAIT_COPY = 1, 2

EXPORTS = ("p3_plan_create", "p3_plan_destroy", "p3_ftran_r2c", "p3_btran_c2r", "p3_ftran_r2c_noalloc",
           "p3_plan_get_dims",
           "p3_plan_workspace_bytes", "p3_plan_scale", "p3_plan_set_stage_events", "p3_plan_describe",
           "p3_plan_launches", "p3_plan_factor", "p3_plan_set_z_hook", "p3_plan_wait_status", "p3_plan_wait_flags",
           "p3_plan_set_wait_limits",
           "p3_plan_set_fused_lag", "p3_batch_create", "p3_batch_destroy", "p3_batch_ftran_r2c",
           "p3_batch_btran_c2r", "p3_batch_wait_status", "p3_batch_set_wait_limits", "p3_batch_launches",
           "p3_status_string", "p3_version")

# int hook(void* data, int n, long long nlines, long long line_stride, long long elem_stride,
#          int dir, void* stream, void* user)
Z_HOOK = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong, ctypes.c_longlong,
                          ctypes.c_longlong, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p)

_lib = None


class P3Error(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__("%s: %s (status %d)" % (what, p3_status_string(status), status))


def load():
    """Load the library (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libp3dfft_gb300.so is not built (%s); run "
                           "paper_1905_02803_gb300.build.build() first" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    I, U, P, D = ctypes.c_int, ctypes.c_uint, ctypes.c_void_p, ctypes.c_double
    lib.p3_plan_create.argtypes = [ctypes.POINTER(P), I, I, I, I, ctypes.POINTER(I), I, U]
    lib.p3_plan_destroy.argtypes = [P]
    lib.p3_ftran_r2c.argtypes = [P, P, P, P, P]
    lib.p3_btran_c2r.argtypes = [P, P, P, P, P]
    lib.p3_ftran_r2c_noalloc.argtypes = [P, P, P, P]
    lib.p3_plan_get_dims.argtypes = [P, ctypes.POINTER(I), ctypes.POINTER(I)]
    lib.p3_plan_workspace_bytes.argtypes = [P, ctypes.POINTER(ctypes.c_size_t)]
    lib.p3_plan_scale.argtypes = [P, ctypes.POINTER(D)]
    lib.p3_plan_set_stage_events.argtypes = [P, ctypes.POINTER(P), I]
    lib.p3_plan_describe.argtypes = [P, ctypes.c_char_p, ctypes.c_size_t]
    lib.p3_plan_launches.argtypes = [P, I, ctypes.POINTER(I)]
    lib.p3_plan_factor.argtypes = [I, I, ctypes.POINTER(I), I, ctypes.POINTER(I)]
    lib.p3_plan_set_z_hook.argtypes = [P, Z_HOOK, P]
    lib.p3_plan_wait_status.argtypes = [P]
    lib.p3_plan_wait_flags.argtypes = [P, ctypes.POINTER(U)]
    lib.p3_plan_set_wait_limits.argtypes = [P, U, U]
    lib.p3_plan_set_fused_lag.argtypes = [P, I]
    lib.p3_batch_create.argtypes = [ctypes.POINTER(P), I, ctypes.POINTER(P), I]
    lib.p3_batch_destroy.argtypes = [P]
    lib.p3_batch_ftran_r2c.argtypes = [P, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P), P]
    lib.p3_batch_btran_c2r.argtypes = [P, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P), P]
    lib.p3_batch_wait_status.argtypes = [P]
    lib.p3_batch_set_wait_limits.argtypes = [P, U, U]
    lib.p3_batch_launches.argtypes = [P, I, ctypes.POINTER(I)]
    lib.p3_status_string.argtypes = [I]
    lib.p3_status_string.restype = ctypes.c_char_p
    lib.p3_version.argtypes = []
    for name in EXPORTS:
        if name not in ("p3_status_string",):
            getattr(lib, name).restype = I
    _lib = lib
    return lib


def _check(st: int, what: str):
    if st != P3_OK:
        raise P3Error(st, what)


def p3_status_string(status: int) -> str:
    return load().p3_status_string(int(status)).decode()


def p3_version() -> int:
    return load().p3_version()


def p3_plan_create(nx, ny, nz, prec, ttype, layout, flags=0, check=True):
    """Returns (status, plan handle or None)."""
    h = ctypes.c_void_p()
    tt = None if ttype is None else (ctypes.c_int * 3)(*ttype)
    st = load().p3_plan_create(ctypes.byref(h), int(nx), int(ny), int(nz), int(prec), tt, int(layout),
                               int(flags))
    if check:
        _check(st, "p3_plan_create")
    return st, (h.value if st == P3_OK else None)


def p3_plan_destroy(plan):
    return load().p3_plan_destroy(plan)


def p3_ftran_r2c(plan, in_ptr, out_ptr, ws_ptr, stream, check=True):
    st = load().p3_ftran_r2c(plan, in_ptr, out_ptr, ws_ptr, stream)
    if check:
        _check(st, "p3_ftran_r2c")
    return st


def p3_btran_c2r(plan, in_ptr, out_ptr, ws_ptr, stream, check=True):
    st = load().p3_btran_c2r(plan, in_ptr, out_ptr, ws_ptr, stream)
    if check:
        _check(st, "p3_btran_c2r")
    return st


# Bytes of the library's built-in scratch array (include/p3dfft_gb300.h).
P3_NOALLOC_SCRATCH_BYTES = 64 << 20


def p3_plan_set_z_hook(plan, hook, user=None, check=True):
    """hook: a Z_HOOK instance (keep a reference while it is set) or None."""
    st = load().p3_plan_set_z_hook(plan, hook if hook is not None else Z_HOOK(), user)
    if check:
        _check(st, "p3_plan_set_z_hook")
    return st


def p3_plan_wait_status(plan) -> int:
    """P3_OK, or P3_ERR_TIMEOUT when a bounded device wait gave up since the
    last check (synchronises with the device)."""
    return load().p3_plan_wait_status(plan)


def p3_plan_wait_flags(plan, check=True) -> int:
    """Which kinds of bounded wait gave up since the last check: an OR of
    P3_WAIT_FUSED_QUEUE and P3_WAIT_COPY, 0 when none (clears the marks)."""
    f = ctypes.c_uint(0)
    st = load().p3_plan_wait_flags(plan, ctypes.byref(f))
    if check:
        _check(st, "p3_plan_wait_flags")
    return f.value


def p3_plan_set_wait_limits(plan, spin_limit, extra=0, check=True):
    st = load().p3_plan_set_wait_limits(plan, int(spin_limit), int(extra))
    if check:
        _check(st, "p3_plan_set_wait_limits")
    return st


def p3_plan_set_fused_lag(plan, lag, check=True):
    st = load().p3_plan_set_fused_lag(plan, int(lag))
    if check:
        _check(st, "p3_plan_set_fused_lag")
    return st


def _ptrs(vals):
    return (ctypes.c_void_p * len(vals))(*[ctypes.c_void_p(v) if v else None for v in vals])


def p3_batch_create(plans, nstreams, check=True):
    """plans: list of plan handles.  Returns (status, batch handle or None)."""
    h = ctypes.c_void_p()
    arr = None if plans is None else _ptrs(plans)
    st = load().p3_batch_create(ctypes.byref(h), 0 if plans is None else len(plans), arr, int(nstreams))
    if check:
        _check(st, "p3_batch_create")
    return st, (h.value if st == P3_OK else None)


def p3_batch_destroy(batch):
    return load().p3_batch_destroy(batch)


def p3_batch_ftran_r2c(batch, ins, outs, wss, stream, check=True):
    st = load().p3_batch_ftran_r2c(batch, None if ins is None else _ptrs(ins), None if outs is None else _ptrs(outs),
                                   None if wss is None else _ptrs(wss), stream)
    if check:
        _check(st, "p3_batch_ftran_r2c")
    return st


def p3_batch_btran_c2r(batch, ins, outs, wss, stream, check=True):
    st = load().p3_batch_btran_c2r(batch, None if ins is None else _ptrs(ins), None if outs is None else _ptrs(outs),
                                   None if wss is None else _ptrs(wss), stream)
    if check:
        _check(st, "p3_batch_btran_c2r")
    return st


def p3_batch_wait_status(batch) -> int:
    """P3_OK, or P3_ERR_TIMEOUT when a persistent batch's bounded wait gave
    up since the last check (synchronises with the device)."""
    return load().p3_batch_wait_status(batch)


def p3_batch_set_wait_limits(batch, spin_limit, extra=0, check=True):
    st = load().p3_batch_set_wait_limits(batch, int(spin_limit), int(extra))
    if check:
        _check(st, "p3_batch_set_wait_limits")
    return st


def p3_batch_launches(batch, direction: int) -> int:
    v = ctypes.c_int()
    _check(load().p3_batch_launches(batch, int(direction), ctypes.byref(v)), "p3_batch_launches")
    return v.value


def p3_ftran_r2c_noalloc(plan, in_ptr, out_ptr, stream, check=True):
    """Forward transform whose workspace is the library's built-in device
    array: for callers that must not allocate device memory at call time."""
    st = load().p3_ftran_r2c_noalloc(plan, in_ptr, out_ptr, stream)
    if check:
        _check(st, "p3_ftran_r2c_noalloc")
    return st


def p3_plan_get_dims(plan):
    a, b = (ctypes.c_int * 3)(), (ctypes.c_int * 3)()
    _check(load().p3_plan_get_dims(plan, a, b), "p3_plan_get_dims")
    return tuple(a), tuple(b)


def p3_plan_workspace_bytes(plan) -> int:
    v = ctypes.c_size_t()
    _check(load().p3_plan_workspace_bytes(plan, ctypes.byref(v)), "p3_plan_workspace_bytes")
    return v.value


def p3_plan_scale(plan) -> float:
    v = ctypes.c_double()
    _check(load().p3_plan_scale(plan, ctypes.byref(v)), "p3_plan_scale")
    return v.value


def p3_plan_set_stage_events(plan, events):
    if events is None:
        _check(load().p3_plan_set_stage_events(plan, None, 0), "p3_plan_set_stage_events")
        return
    arr = (ctypes.c_void_p * len(events))(*events)
    _check(load().p3_plan_set_stage_events(plan, arr, len(events)), "p3_plan_set_stage_events")


def p3_plan_describe(plan) -> str:
    buf = ctypes.create_string_buffer(1 << 14)
    _check(load().p3_plan_describe(plan, buf, len(buf)), "p3_plan_describe")
    return buf.value.decode()


def p3_plan_factor(n: int, precision: str = "f32"):
    """Radix sequence of the generic-kernel stages of an n-point line (no GPU
    needed); None when n has a prime factor above 7."""
    prec = {"f32": P3_F32, "f64": P3_F64}[precision]
    buf = (ctypes.c_int * 32)()
    cnt = ctypes.c_int()
    rc = load().p3_plan_factor(int(n), prec, buf, 32, ctypes.byref(cnt))
    if rc == P3_ERR_UNSUPPORTED:
        return None
    _check(rc, "p3_plan_factor")
    return [buf[i] for i in range(cnt.value)]


def p3_plan_launches(plan, direction: int) -> int:
    v = ctypes.c_int()
    _check(load().p3_plan_launches(plan, int(direction), ctypes.byref(v)), "p3_plan_launches")
    return v.value


# ---------------------------------------------------------------------------
# torch-facing wrapper
# ---------------------------------------------------------------------------

_TT = {"fft": P3_FFT, "cheb": P3_CHEB, "empty": P3_EMPTY, "sine": P3_SINE}
_LAYOUT = {"zyx": P3_LAYOUT_ZYX, "xyz": P3_LAYOUT_XYZ}


class Plan:
    """A plan for an (nx, ny, nz) grid.  Real arrays are torch tensors of shape
    (nz, ny, nx); complex arrays (nz, ny, H) for layout 'xyz' or (H, ny, nz)
    for 'zyx', H = nx // 2 + 1."""

    def __init__(self, nx, ny, nz, precision="f32", ttypes=("fft", "fft", "fft"), layout="zyx", device=None,
                 flags=0):
        import torch
        self.torch = torch
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.H = self.nx // 2 + 1
        self.precision = precision
        self.ttypes = tuple(ttypes)
        self.layout = layout
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        with torch.cuda.device(self.device):
            _, self.handle = p3_plan_create(self.nx, self.ny, self.nz, P3_F32 if precision == "f32" else P3_F64,
                                            [_TT[t] for t in self.ttypes], _LAYOUT[layout], flags)
        self.real_dtype = torch.float32 if precision == "f32" else torch.float64
        self.complex_dtype = torch.complex64 if precision == "f32" else torch.complex128
        self.flags = int(flags)
        self.padded = bool(self.flags & P3_FLAG_PADDED_REAL)
        self.ws_bytes = p3_plan_workspace_bytes(self.handle)
        self.scale = p3_plan_scale(self.handle)
        self._ws = None
        self._hook = None       # (python function, ctypes callback) while a Z hook is set
        self._bufs = {}         # device pointer -> tensor, for the current call
        self._hook_error = None

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and _lib is not None:
            p3_plan_destroy(h)
            self.handle = None

    @property
    def real_shape(self):
        """(nz, ny, nx), or (nz, ny, 2H) with padded real rows."""
        return (self.nz, self.ny, 2 * self.H if self.padded else self.nx)

    @property
    def complex_shape(self):
        return (self.nz, self.ny, self.H) if self.layout == "xyz" else (self.H, self.ny, self.nz)

    def empty_real(self):
        return self.torch.empty(self.real_shape, dtype=self.real_dtype, device=self.device)

    def empty_complex(self):
        return self.torch.empty(self.complex_shape, dtype=self.complex_dtype, device=self.device)

    def workspace(self):
        if self.ws_bytes == 0:
            return None
        if self._ws is None:
            self._ws = self.torch.empty(self.ws_bytes, dtype=self.torch.uint8, device=self.device)
        return self._ws

    def describe(self) -> str:
        return p3_plan_describe(self.handle)

    def set_z_hook(self, fn):
        """Run fn(lines, direction) in place of the EMPTY third-dimension
        transform: lines is a strided complex view [H*Ny, Nz] of the device
        data (one row per Z line) that fn transforms in place, on the current
        stream; direction is 0 forward, 1 inverse.  fn=None clears it."""
        if fn is None:
            p3_plan_set_z_hook(self.handle, None)
            self._hook = None
            return
        torch = self.torch

        def tramp(data, n, nlines, ls, es, direction, stream, user):
            try:
                base = self._bufs[data]
                flat = base.view(-1).view(self.complex_dtype) if base.dtype != self.complex_dtype else base.view(-1)
                lines = flat.as_strided((nlines, n), (ls, es))
                st = (torch.cuda.ExternalStream(stream, device=self.device) if stream
                      else torch.cuda.default_stream(self.device))
                with torch.cuda.stream(st):
                    fn(lines, direction)
                return 0
            except BaseException as exc:  # reported after the C call returns
                self._hook_error = exc
                return 1

        cb = Z_HOOK(tramp)
        p3_plan_set_z_hook(self.handle, cb)
        self._hook = (fn, cb)

    def _call(self, c_fn, inp, out, ws, stream):
        self._bufs = {t.data_ptr(): t for t in (ws, out) if t is not None}
        self._hook_error = None
        try:
            st = c_fn(self.handle, inp.data_ptr(), out.data_ptr(), None if ws is None else ws.data_ptr(),
                      self._stream(stream), check=False)
        finally:
            self._bufs = {}
        if st == P3_ERR_HOOK and self._hook_error is not None:
            raise P3Error(st, c_fn.__name__) from self._hook_error
        _check(st, c_fn.__name__)

    def launches(self, direction: int) -> int:
        return p3_plan_launches(self.handle, direction)

    def _stream(self, stream):
        s = stream if stream is not None else self.torch.cuda.current_stream(self.device)
        return ctypes.c_void_p(s.cuda_stream)

    def _check_tensor(self, t, shape, dtype, what):
        if t.device != self.device or t.dtype != dtype or tuple(t.shape) != tuple(shape) or not t.is_contiguous():
            raise ValueError("%s must be a contiguous %s tensor of shape %s on %s" % (what, dtype, shape, self.device))

    def forward(self, x, out=None, ws=None, stream=None):
        self._check_tensor(x, self.real_shape, self.real_dtype, "input")
        out = self.empty_complex() if out is None else out
        self._check_tensor(out, self.complex_shape, self.complex_dtype, "output")
        ws = self.workspace() if ws is None else ws
        self._call(p3_ftran_r2c, x, out, ws, stream)
        return out

    def complex_view(self, x):
        """The complex array sharing storage with a padded real array (in place)."""
        return self.torch.view_as_complex(x.view(self.nz, self.ny, self.H, 2))

    def real_view(self, X):
        """The padded real array sharing storage with a complex array (in place)."""
        return self.torch.view_as_real(X).view(self.nz, self.ny, 2 * self.H)

    def backward(self, X, out=None, ws=None, stream=None):
        self._check_tensor(X, self.complex_shape, self.complex_dtype, "input")
        out = self.empty_real() if out is None else out
        self._check_tensor(out, self.real_shape, self.real_dtype, "output")
        ws = self.workspace() if ws is None else ws
        self._call(p3_btran_c2r, X, out, ws, stream)
        return out


class Batch:
    """Independent plans in one batch (p3_batch_*): nstreams = 0 runs every
    call as one persistent launch, nstreams >= 1 spreads the plans' own
    launches over that many internal streams.  forward(xs) / backward(Xs)
    take one tensor per plan."""

    def __init__(self, plans, nstreams=8):
        self.plans = list(plans)
        self.torch = self.plans[0].torch
        self.nstreams = int(nstreams)
        _, self.handle = p3_batch_create([p.handle for p in self.plans], nstreams)

    def launches(self, direction: int) -> int:
        return p3_batch_launches(self.handle, direction)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and _lib is not None:
            p3_batch_destroy(h)
            self.handle = None

    def _stream(self, stream):
        s = stream if stream is not None else self.torch.cuda.current_stream(self.plans[0].device)
        return ctypes.c_void_p(s.cuda_stream)

    def forward(self, xs, outs=None, stream=None):
        outs = [p.empty_complex() for p in self.plans] if outs is None else outs
        for p, x, o in zip(self.plans, xs, outs):
            p._check_tensor(x, p.real_shape, p.real_dtype, "input")
            p._check_tensor(o, p.complex_shape, p.complex_dtype, "output")
        wss = [p.workspace() for p in self.plans]
        p3_batch_ftran_r2c(self.handle, [x.data_ptr() for x in xs], [o.data_ptr() for o in outs],
                           [0 if w is None else w.data_ptr() for w in wss], self._stream(stream))
        return outs

    def backward(self, Xs, outs=None, stream=None):
        outs = [p.empty_real() for p in self.plans] if outs is None else outs
        for p, X, o in zip(self.plans, Xs, outs):
            p._check_tensor(X, p.complex_shape, p.complex_dtype, "input")
            p._check_tensor(o, p.real_shape, p.real_dtype, "output")
        wss = [p.workspace() for p in self.plans]
        p3_batch_btran_c2r(self.handle, [X.data_ptr() for X in Xs], [o.data_ptr() for o in outs],
                           [0 if w is None else w.data_ptr() for w in wss], self._stream(stream))
        return outs
