"""Thin Python binding of libnufft45 (non-iterative type-4/5 NUFFTs, GB300).

Argument marshalling only: every step of every transform runs in the CUDA
library.  The C entry points are available under their own names
(``nufft_plan``, ``nufft_inv5``, ``nufft_inv4``, ``nufft_fwd1``,
``nufft_fwd2``, ``nufft_destroy``, ...) on the object returned by ``lib()``;
``Plan`` wraps them for torch tensors (device memory, streams) and
``autograd`` adds the differentiable inverses.

There is no CPU fallback: importing the transforms without the built
library raises.
"""
import ctypes
import os

__all__ = ["lib", "Plan", "Batch", "NufftError", "FP32", "FP64", "REFINE", "DEFER_CHECK", "TOEPLITZ", "Params", "build", "library_path", "ProfileEntry", "check"]

FP32 = 1
FP64 = 2
REFINE = 0x100   # OR into the precision: one refinement step per inverse (Sec. V)
DEFER_CHECK = 0x200   # OR into the precision: the plan call does not wait for the duplicate-node check
TOEPLITZ = 0x400   # OR into the precision: middle stage as a linear convolution with L (no rho^-m scaling)

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "lib", "libnufft45.so")
_lib = None


def library_path():
    return _LIB_PATH


def build(force=False):
    from . import _build
    return _build.build(force=force)


class NufftError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (status, message))
        self.status = status


class PlanInfo(ctypes.Structure):
    _fields_ = [
        ("N", ctypes.c_int64), ("prec", ctypes.c_int), ("tol", ctypes.c_double),
        ("gamma", ctypes.c_double), ("a", ctypes.c_double), ("rho", ctypes.c_double),
        ("eta", ctypes.c_int), ("R", ctypes.c_int64), ("grid_solve", ctypes.c_int64),
        ("grid_plan", ctypes.c_int64), ("w_solve", ctypes.c_int), ("w_plan", ctypes.c_int),
        ("beta_solve", ctypes.c_double), ("beta_plan", ctypes.c_double),
        ("batch_chunk", ctypes.c_int64),
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class Instance(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("x", ctypes.c_void_p), ("inp", ctypes.c_void_p), ("out", ctypes.c_void_p),
                ("kind", ctypes.c_int)]


class Params(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("eta", ctypes.c_int), ("w_plan", ctypes.c_int),
                ("w_solve", ctypes.c_int)]


class ProfileEntry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64), ("ms", ctypes.c_double),
                ("bytes", ctypes.c_double)]


def lib():
    """Load libnufft45.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise ImportError("libnufft45.so is not built (%s); run paper_1604_06236_gb300.build()" % _LIB_PATH)
        L = ctypes.CDLL(_LIB_PATH)
        vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
        L.nufft_plan.argtypes = [i64, vp, dbl, i32, vp, ctypes.POINTER(vp)]
        L.nufft_plan_ex.argtypes = [i64, vp, dbl, i32, ctypes.POINTER(Params), vp, ctypes.POINTER(vp)]
        L.nufft_plan_ex.restype = i32
        L.nufft_plan_tune.argtypes = [i64, vp, dbl, i32, i64, vp, ctypes.POINTER(Params), ctypes.POINTER(dbl)]
        L.nufft_plan_tune.restype = i32
        L.nufft_plan_save.argtypes = [vp, vp, vp, vp]
        L.nufft_plan_save.restype = i32
        L.nufft_plan_restore.argtypes = [i64, vp, dbl, i32, ctypes.POINTER(Params), vp, vp, vp, ctypes.POINTER(vp)]
        L.nufft_plan_restore.restype = i32
        for name in ("nufft_inv5", "nufft_inv4", "nufft_fwd1", "nufft_fwd2", "nufft_fwd2_deriv"):
            getattr(L, name).argtypes = [vp, vp, vp, i64, vp]
        L.nufft_destroy.argtypes = [vp]
        L.nufft_plan_set_batch_chunk.argtypes = [vp, i64]
        L.nufft_plan_set_batch_chunk.restype = i32
        L.nufft_batch_create.argtypes = [i64, ctypes.POINTER(Instance), dbl, vp, ctypes.POINTER(vp)]
        L.nufft_batch_run.argtypes = [vp, vp]
        L.nufft_batch_status.argtypes = [vp, vp, vp]
        L.nufft_batch_destroy.argtypes = [vp]
        L.nufft_batch_tune.argtypes = [vp, vp, ctypes.POINTER(dbl)]
        L.nufft_batch_config.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32)]
        L.nufft_batch_params.argtypes = [vp, ctypes.POINTER(Params)]
        L.nufft_batch_params.restype = i32
        for name in ("nufft_batch_create", "nufft_batch_run", "nufft_batch_status", "nufft_batch_destroy",
                     "nufft_batch_tune", "nufft_batch_config"):
            getattr(L, name).restype = i32
        for name in ("nufft_inv5_grad_nodes", "nufft_inv4_grad_nodes"):
            getattr(L, name).argtypes = [vp, vp, vp, i64, vp, vp]
            getattr(L, name).restype = i32
        L.nufft_plan_info.argtypes = [vp, ctypes.POINTER(PlanInfo)]
        L.nufft_plan_export.argtypes = [vp, i32, vp, vp]
        L.nufft_cache_clear.argtypes = []
        L.nufft_stream_check.argtypes = [vp]
        L.nufft_plan_check.argtypes = [vp]
        L.nufft_profile_enable.argtypes = [i32]
        L.nufft_profile_enable.restype = i32
        L.nufft_profile_read.argtypes = [ctypes.POINTER(ProfileEntry), i32, ctypes.POINTER(ctypes.c_int)]
        L.nufft_profile_read.restype = i32
        L.nufft_launch_count.argtypes = []
        L.nufft_launch_count.restype = i64
        L.nufft_measure_fma.argtypes = [i32, ctypes.POINTER(ctypes.c_double), vp]
        L.nufft_measure_fma.restype = i32
        L.nufft_status_string.argtypes = [i32]
        L.nufft_status_string.restype = ctypes.c_char_p
        L.nufft_last_error_message.argtypes = []
        L.nufft_last_error_message.restype = ctypes.c_char_p
        for name in ("nufft_plan", "nufft_inv5", "nufft_inv4", "nufft_fwd1", "nufft_fwd2", "nufft_fwd2_deriv",
                     "nufft_destroy",
                     "nufft_plan_info", "nufft_plan_export", "nufft_cache_clear", "nufft_stream_check", "nufft_plan_check"):
            getattr(L, name).restype = i32
        _lib = L
    return _lib


def check(status):
    if status != 0:
        L = lib()
        raise NufftError(L.nufft_status_string(status).decode(), L.nufft_last_error_message().decode())


def _stream_handle(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def plan_tune(x, tol=None, prec=FP32, batch=8, stream=None):
    """Choose (gamma, eta, plan width) for these nodes and tol (nufft_plan_tune);
    returns (params dict, best milliseconds).  Later plans with the same
    (N, prec, tol) use the result."""
    import torch
    if not isinstance(x, torch.Tensor):
        x = torch.as_tensor(x)
    x = x.to(torch.float64).contiguous()
    if tol is None:
        tol = 1e-5 if prec == FP32 else 1e-10
    q = Params()
    ms = ctypes.c_double()
    check(lib().nufft_plan_tune(x.numel(), _ptr(x), float(tol), int(prec), int(batch), _stream_handle(stream),
                                ctypes.byref(q), ctypes.byref(ms)))
    return {"gamma": q.gamma, "eta": q.eta, "w_plan": q.w_plan, "w_solve": q.w_solve}, ms.value


def measure_fma(prec=FP32, stream=None):
    """Sustained fused multiply-add rate of the device in TFLOP/s, float32
    (FP32) or float64 (FP64) (nufft_measure_fma; a measurement utility)."""
    r = ctypes.c_double()
    check(lib().nufft_measure_fma(prec, ctypes.byref(r), _stream_handle(stream)))
    return r.value


def stream_check(stream=None):
    """Synchronise the stream and the library's copy streams (pinned host
    outputs are then complete); raise NufftError(NUFFT_ERR_TIMEOUT) if a
    bounded wait inside a library kernel gave up since the last check."""
    check(lib().nufft_stream_check(_stream_handle(stream)))


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


class Plan:
    """A plan for N nodes (radians), float64 tensor on the GPU or host.

    prec FP32: complex64 data, float64 node weights; prec FP64: complex128.
    """

    def __init__(self, x, tol=None, prec=FP32, stream=None, gamma=None, eta=None, w_plan=None, w_solve=None,
                 saved=None):
        """saved: (K, D, params) from Plan.save() of a plan on the same node
        values, tol and precision; the plan is then restored from them
        (nufft_plan_restore: only the node geometry, phases and weights are
        computed)."""
        import torch
        if not isinstance(x, torch.Tensor):
            x = torch.as_tensor(x)
        x = x.to(torch.float64).contiguous()
        if tol is None:
            tol = 1e-5 if (prec & 0xFF) == FP32 else 1e-10
        self.N = x.numel()
        self.prec = prec
        self.tol = tol
        self.dtype = torch.complex64 if (prec & 0xFF) == FP32 else torch.complex128
        self.device = x.device if x.is_cuda else torch.device("cuda", torch.cuda.current_device())
        self._h = ctypes.c_void_p()
        self._x_keep = x
        if saved is not None:
            K, D, prm = saved
            self._saved_keep = (K, D)
            q = Params(float(prm["gamma"]), int(prm["eta"]), int(prm["w_plan"]), int(prm["w_solve"]))
            check(lib().nufft_plan_restore(self.N, _ptr(x), float(tol), int(prec), ctypes.byref(q), _ptr(K), _ptr(D),
                                           _stream_handle(stream), ctypes.byref(self._h)))
        elif gamma is None and eta is None and w_plan is None and w_solve is None:
            check(lib().nufft_plan(self.N, _ptr(x), float(tol), int(prec), _stream_handle(stream),
                                   ctypes.byref(self._h)))
        else:
            # explicit method parameters (Sec. V); None keeps the tol-derived value
            q = Params(float(gamma or 0.0), int(eta or 0), int(w_plan or 0), int(w_solve or 0))
            check(lib().nufft_plan_ex(self.N, _ptr(x), float(tol), int(prec), ctypes.byref(q),
                                      _stream_handle(stream), ctypes.byref(self._h)))

    def check(self):
        """Wait for the plan; raise NufftError(NUFFT_ERR_DUP_NODES) if two nodes
        coincide (the way a DEFER_CHECK plan reports it)."""
        check(lib().nufft_plan_check(self._h))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().nufft_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_batch_chunk(self, chunk):
        check(lib().nufft_plan_set_batch_chunk(self._h, int(chunk)))

    def info(self):
        inf = PlanInfo()
        check(lib().nufft_plan_info(self._h, ctypes.byref(inf)))
        return inf.as_dict()

    def save(self, stream=None):
        """(K, D, params): the kernel samples K_q and the derivative samples
        L'(z_p) as complex128 device tensors (nufft_plan_save, stream
        ordered) and the method parameters, enough to restore the plan."""
        import torch
        K = torch.empty(self.N, dtype=torch.complex128, device=self.device)
        D = torch.empty_like(K)
        check(lib().nufft_plan_save(self._h, _ptr(K), _ptr(D), _stream_handle(stream)))
        inf = self.info()
        return K, D, {k: inf[k] for k in ("gamma", "eta", "w_plan", "w_solve")}

    def export(self, which, stream=None):
        import torch
        out = torch.empty(self.N, dtype=torch.complex128, device=self.device)
        check(lib().nufft_plan_export(self._h, int(which), _ptr(out), _stream_handle(stream)))
        return out

    def _run(self, fname, inp, out=None, stream=None):
        import torch
        if inp.dtype != self.dtype:
            raise TypeError("expected %s data, got %s" % (self.dtype, inp.dtype))
        if inp.shape[-1] != self.N:
            raise ValueError("last dimension must be N = %d" % self.N)
        inp = inp.contiguous()
        if out is None:
            out = torch.empty_like(inp)
        batch = inp.numel() // self.N
        check(getattr(lib(), fname)(self._h, _ptr(inp), _ptr(out), batch, _stream_handle(stream)))
        return out

    def inv5(self, f, out=None, stream=None):
        """Type-5: coefficients S (k = 0..N-1) from samples at the nodes (Eq. 48)."""
        return self._run("nufft_inv5", f, out, stream)

    def inv4(self, A, out=None, stream=None):
        """Type-4: node amplitudes a from spectral samples A(k), k = 0..N-1 (Eq. 47)."""
        return self._run("nufft_inv4", A, out, stream)

    def fwd1(self, a, out=None, stream=None):
        """Type-1: A(k) = sum_p a_p e^{-j 2 pi k t_p} (Eq. 32)."""
        return self._run("nufft_fwd1", a, out, stream)

    def fwd2(self, c, out=None, stream=None):
        """Type-2: s(t_p) = sum_m c_m e^{j 2 pi m t_p} (Eq. 34)."""
        return self._run("nufft_fwd2", c, out, stream)

    def fwd2_deriv(self, c, out=None, stream=None):
        """d/dt of the type-2 sum: sum_m (j 2 pi m) c_m e^{j 2 pi m t_p}."""
        return self._run("nufft_fwd2_deriv", c, out, stream)

    def _grad_nodes(self, fname, p1, p2, stream=None):
        import torch
        for t in (p1, p2):
            if t.dtype != self.dtype or t.shape[-1] != self.N:
                raise TypeError("expected %s tensors with last dimension %d" % (self.dtype, self.N))
        p1 = p1.contiguous()
        p2 = p2.contiguous()
        batch = p1.numel() // self.N
        if p2.numel() != p1.numel():
            raise ValueError("both operands need the same batch")
        out = torch.empty(self.N, dtype=torch.float64, device=p1.device)
        check(getattr(lib(), fname)(self._h, _ptr(p1), _ptr(p2), batch, _ptr(out), _stream_handle(stream)))
        return out

    def inv5_grad_nodes(self, u, S, stream=None):
        """dL/dx for S = inv5(f): u = gradient w.r.t. f (inv4 of dL/dS), S the solution."""
        return self._grad_nodes("nufft_inv5_grad_nodes", u, S, stream)

    def inv4_grad_nodes(self, w, a, stream=None):
        """dL/dx for a = inv4(A): w = gradient w.r.t. A (inv5 of dL/da), a the solution."""
        return self._grad_nodes("nufft_inv4_grad_nodes", w, a, stream)


class Batch:
    """Many independent type-5 / type-4 inverses of uneven size, one persistent
    launch per run.  `items` is a list of (x, data, kind) with x float64 nodes
    (N,), data complex64 (N,) on the GPU and kind 5 or 4; outputs are
    allocated here.  run() re-plans and solves every instance."""

    def __init__(self, items, tol=1e-5, stream=None):
        import torch
        self.keep = []
        self.outs = []
        arr = (Instance * len(items))()
        for i, (x, d, kind) in enumerate(items):
            x = x.to(torch.float64).contiguous()
            d = d.to(torch.complex64).contiguous()
            o = torch.empty_like(d)
            self.keep += [x, d]
            self.outs.append(o)
            arr[i] = Instance(x.numel(), x.data_ptr(), d.data_ptr(), o.data_ptr(), int(kind))
        self.count = len(items)
        self._h = ctypes.c_void_p()
        check(lib().nufft_batch_create(self.count, arr, float(tol), _stream_handle(stream), ctypes.byref(self._h)))

    def run(self, stream=None):
        check(lib().nufft_batch_run(self._h, _stream_handle(stream)))
        return self.outs

    def tune(self, stream=None):
        """Autotune the launch shape on this batch; returns (ms, ctas, threads, max_radix)."""
        ms = ctypes.c_double()
        check(lib().nufft_batch_tune(self._h, _stream_handle(stream), ctypes.byref(ms)))
        c, t, r = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        check(lib().nufft_batch_config(self._h, ctypes.byref(c), ctypes.byref(t), ctypes.byref(r)))
        return ms.value, c.value, t.value, r.value

    def params(self):
        """The method's parameters in use: gamma, eta, w_plan, w_solve (Sec. V)."""
        q = Params()
        check(lib().nufft_batch_params(self._h, ctypes.byref(q)))
        return {"gamma": q.gamma, "eta": q.eta, "w_plan": q.w_plan, "w_solve": q.w_solve}

    def status(self, stream=None):
        import torch
        st = torch.empty(self.count, dtype=torch.int32)
        check(lib().nufft_batch_status(self._h, ctypes.c_void_p(st.data_ptr()), _stream_handle(stream)))
        return st

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().nufft_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
