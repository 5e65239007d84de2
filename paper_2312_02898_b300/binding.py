"""Thin Python binding of the C ABI in include/me.h (argument marshalling only).

Every step of the computation runs in libme_b300.so; PyTorch supplies device memory
and streams.  There is no CPU path: without the built library (or without a CUDA
device) every call raises.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libme_b300.so")

ME_OK, ME_ERR_ARG, ME_ERR_MODE, ME_ERR_NOMEM, ME_ERR_CUDA, ME_ERR_TIMEOUT = 0, -1, -2, -3, -4, -5
PRECISIONS = {"fp64": 0, "fp32": 1, "mixed": 2, "dfloat": 3}

# the C-ABI entry points declared in include/me.h
EXPORTS = ("me_default_params", "me_init", "me_compute", "me_compute_host", "me_info", "me_good_helicities",
           "me_flops", "me_plan", "me_reserve", "me_launch_shape", "me_set_config", "me_last_error", "me_free",
           "me_compute_noalloc", "me_unweight", "me_rambo", "me_uniforms", "me_probe_alu_peak", "me_sync_status",
           "me_set_wait_limit", "me_compute_channels", "me_compute_unweight")


class SMParams(ctypes.Structure):
    _fields_ = [("mZ", ctypes.c_double), ("wZ", ctypes.c_double), ("mt", ctypes.c_double),
                ("wt", ctypes.c_double), ("aEWM1", ctypes.c_double), ("Gf", ctypes.c_double),
                ("alphas_default", ctypes.c_double), ("precision", ctypes.c_int),
                ("zero_width_tchan", ctypes.c_int), ("rescue_kappa", ctypes.c_double)]


class MEError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"[{code}] {msg}")
        self.code = code


_lib = None


def load(path: str = LIB_PATH):
    """Load libme_b300.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: run `python -m paper_2312_02898_b300.build`")
    lib = ctypes.CDLL(path)
    vp, i64 = ctypes.c_void_p, ctypes.c_int64
    ip = ctypes.POINTER(ctypes.c_int)
    lib.me_default_params.argtypes = [ctypes.POINTER(SMParams)]
    lib.me_default_params.restype = None
    lib.me_init.argtypes = [ctypes.c_char_p, ctypes.POINTER(SMParams), ctypes.POINTER(vp)]
    lib.me_compute.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.me_compute_host.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.me_compute_noalloc.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.me_reserve.argtypes = [vp, i64, vp]
    lib.me_launch_shape.argtypes = [vp, i64, ip, ip, ip, ip]
    lib.me_unweight.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp, vp, vp]
    u64 = ctypes.c_uint64
    lib.me_rambo.argtypes = [vp, i64, u64, u64, ctypes.c_double, vp, vp]
    lib.me_uniforms.argtypes = [i64, u64, u64, ctypes.c_int, ctypes.c_double, ctypes.c_double, vp, vp]
    lib.me_info.argtypes = [vp, ip, ip, ip, ip, ip]
    lib.me_good_helicities.argtypes = [vp, ctypes.POINTER(ctypes.c_int32)]
    lib.me_flops.argtypes = [vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
    lib.me_set_config.argtypes = [vp, ctypes.c_int]
    lib.me_sync_status.argtypes = [vp, vp]
    lib.me_compute_channels.argtypes = [ctypes.POINTER(vp), ctypes.c_int, i64] + [vp] * 9
    lib.me_compute_unweight.argtypes = [vp, i64] + [vp] * 14
    lib.me_set_wait_limit.argtypes = [vp, i64]
    lib.me_plan.argtypes = [vp, i64, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
    lib.me_probe_alu_peak.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]
    lib.me_last_error.argtypes = [vp]
    lib.me_last_error.restype = ctypes.c_char_p
    lib.me_free.argtypes = [vp]
    lib.me_free.restype = None
    for f in ("me_init", "me_compute", "me_compute_host", "me_compute_noalloc", "me_info", "me_good_helicities",
              "me_flops", "me_set_config", "me_plan", "me_reserve", "me_launch_shape", "me_unweight",
              "me_rambo", "me_uniforms", "me_probe_alu_peak", "me_sync_status", "me_set_wait_limit",
              "me_compute_channels", "me_compute_unweight"):
        getattr(lib, f).restype = ctypes.c_int
    _lib = lib
    return lib


def default_params() -> SMParams:
    p = SMParams()
    load().me_default_params(ctypes.byref(p))
    return p


def alu_peak(precision: str, seconds: float = 0.3) -> float:
    """measured FMA throughput (flop/s) of the current device for 'fp64', 'fp32' or
    'fp32x2' (packed pairs, two FMAs per instruction)"""
    v = ctypes.c_double()
    code = {"fp64": 0, "fp32": 1, "fp32x2": 2}[precision]
    rc = load().me_probe_alu_peak(code, seconds, ctypes.byref(v))
    if rc != ME_OK:
        raise MEError(rc, "ALU probe failed")
    return v.value


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _check_tensor(name, t, dtype, shape, device, required=False):
    """raise ValueError unless t (a torch tensor, or None where allowed) has the dtype,
    shape and device the C ABI expects and is contiguous: the library reads raw pointers,
    and a temporary contiguous copy made here could be recycled by the caching allocator
    before a kernel on another stream has read it"""
    if t is None:
        if required:
            raise ValueError(f"{name} is required")
        return
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, not {t.dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, not {tuple(t.shape)}")
    if t.device != device:
        raise ValueError(f"{name} must be on {device}, not {t.device}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def device_uniforms(nevt, seed, first_event, stream_id, offset=0.0, scale=1.0, stream=None):
    """offset + scale * u for events first_event .. first_event + nevt - 1, generated on
    the device (the same numbers as phasespace.uniforms)"""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    out = torch.empty(nevt, dtype=torch.float64, device=s.device)
    rc = load().me_uniforms(nevt, seed, first_event, stream_id, offset, scale, _ptr(out), ctypes.c_void_p(s.cuda_stream))
    if rc != ME_OK:
        raise MEError(rc, load().me_last_error(None).decode())
    return out


def compute_channels(handles, channel, momenta, alphas=None, rnd_hel=None, rnd_col=None, out=None, stream=None):
    """Per-event subprocess dispatch (me_compute_channels): event e is evaluated by
    handles[channel[e]] (MatrixElement objects with the same number of particles, FP64 or
    FP32).  Device tensors in and out, asynchronous on ``stream``."""
    import torch
    if not handles:
        raise ValueError("at least one channel handle is required")
    h0 = handles[0]
    if not momenta.is_cuda:
        raise ValueError("momenta must be a CUDA tensor")
    nevt = momenta.shape[0]
    dev = momenta.device
    _check_tensor("channel", channel, torch.int32, (nevt,), dev, required=True)
    if out is None:
        me = torch.empty(nevt, dtype=torch.float64, device=dev)
        sh = torch.empty(nevt, dtype=torch.int32, device=dev) if rnd_hel is not None else None
        sc = torch.empty(nevt, dtype=torch.int32, device=dev) if rnd_col is not None else None
    else:
        me, sh, sc = out
    h0._check_args(momenta, alphas, rnd_hel, rnd_col, (me, sh, sc), dev)
    arr = (ctypes.c_void_p * len(handles))(*[h.handle.value for h in handles])
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    h0._check(h0.lib.me_compute_channels(arr, len(handles), nevt, _ptr(channel), _ptr(momenta), _ptr(alphas),
                                         _ptr(rnd_hel), _ptr(rnd_col), _ptr(me), _ptr(sh), _ptr(sc),
                                         ctypes.c_void_p(s.cuda_stream)))
    return me, sh, sc


class MatrixElement:
    """One process on the current CUDA device.

    >>> m = MatrixElement("g g > t t~ g g", precision="fp32")
    >>> me, sel_hel, sel_col = m.compute(momenta, alphas, rnd_hel, rnd_col)
    """

    def __init__(self, process: str, precision: str = "fp64", config: int | None = None, **params):
        self.lib = load()
        p = default_params()
        p.precision = PRECISIONS[precision]
        for k, v in params.items():
            setattr(p, "alphas_default" if k == "alphas" else k, v)
        h = ctypes.c_void_p()
        rc = self.lib.me_init(process.encode(), ctypes.byref(p), ctypes.byref(h))
        if rc != ME_OK:
            raise MEError(rc, self.lib.me_last_error(None).decode())
        self.handle = h
        self.process = process
        self.precision = precision
        self.params = p
        v = [ctypes.c_int() for _ in range(5)]
        self.lib.me_info(h, *[ctypes.byref(x) for x in v])
        self.npar, self.ncomb, self.ngood, self.ncol, self.ndiag = (x.value for x in v)
        fa, fc = ctypes.c_int64(), ctypes.c_int64()
        self.lib.me_flops(h, ctypes.byref(fa), ctypes.byref(fc))
        self.flops_amp_per_hel, self.flops_col_per_hel = fa.value, fc.value
        self.nconfig = self.lib.me_set_config(h, -1)
        if config is not None:
            self.set_config(config)

    def plan(self, nevt: int):
        """(kernel launches, workspace bytes) of a compute call of nevt events"""
        n, w = ctypes.c_int64(), ctypes.c_int64()
        self._check(self.lib.me_plan(self.handle, nevt, ctypes.byref(n), ctypes.byref(w)))
        return n.value, w.value

    def reserve(self, nevt: int, stream=None):
        """size the workspace of ``stream`` for calls of up to nevt events (before graph capture)"""
        import torch
        s = stream if stream is not None else torch.cuda.current_stream()
        self._check(self.lib.me_reserve(self.handle, nevt, ctypes.c_void_p(s.cuda_stream)))

    def launch_shape(self, nevt: int):
        """(grid blocks, threads per block, resident blocks per SM, SMs) of the main pass"""
        v = [ctypes.c_int() for _ in range(4)]
        self._check(self.lib.me_launch_shape(self.handle, nevt, *[ctypes.byref(x) for x in v]))
        return tuple(x.value for x in v)

    def set_config(self, config: int):
        self._check(self.lib.me_set_config(self.handle, config))

    def good_helicities(self):
        arr = (ctypes.c_int32 * self.ncomb)()
        self.lib.me_good_helicities(self.handle, arr)
        return list(arr)[: self.ngood]

    def flops_per_event(self) -> int:
        """generator-counted real flops of one event (amplitudes + colour sum, all kept helicities)"""
        return self.ngood * (self.flops_amp_per_hel + self.flops_col_per_hel)

    def _check(self, rc):
        if rc != ME_OK:
            raise MEError(rc, self.lib.me_last_error(self.handle).decode())

    def _check_args(self, momenta, alphas, rnd_hel, rnd_col, out, device):
        """dtype, shape, device and contiguity of every tensor argument (ValueError)"""
        import torch
        nevt = momenta.shape[0] if momenta.dim() else -1
        f64, i32 = torch.float64, torch.int32
        _check_tensor("momenta", momenta, f64, (nevt, self.npar, 4), device, required=True)
        for name, t in (("alphas", alphas), ("rnd_hel", rnd_hel), ("rnd_col", rnd_col)):
            _check_tensor(name, t, f64, (nevt,), device)
        me, sh, sc = out
        _check_tensor("me", me, f64, (nevt,), device, required=True)
        _check_tensor("sel_hel", sh, i32, (nevt,), device)
        _check_tensor("sel_col", sc, i32, (nevt,), device)
        if (sh is not None and rnd_hel is None) or (sc is not None and rnd_col is None):
            raise ValueError("a selection output needs its random numbers")
        return nevt

    def compute(self, momenta, alphas=None, rnd_hel=None, rnd_col=None, out=None, stream=None):
        """Device tensors in, device tensors out (asynchronous on ``stream``).  Every
        tensor must be contiguous, of the documented dtype and length, and on the
        device of ``momenta``."""
        import torch
        if not momenta.is_cuda:
            raise ValueError("momenta must be a CUDA tensor (use compute_host for host arrays)")
        nevt = momenta.shape[0]
        dev = momenta.device
        if out is None:
            me = torch.empty(nevt, dtype=torch.float64, device=dev)
            sh = torch.empty(nevt, dtype=torch.int32, device=dev) if rnd_hel is not None else None
            sc = torch.empty(nevt, dtype=torch.int32, device=dev) if rnd_col is not None else None
        else:
            me, sh, sc = out
        self._check_args(momenta, alphas, rnd_hel, rnd_col, (me, sh, sc), dev)
        s = stream if stream is not None else torch.cuda.current_stream(dev)
        rc = self.lib.me_compute(self.handle, nevt, _ptr(momenta), _ptr(alphas), _ptr(rnd_hel), _ptr(rnd_col),
                                 _ptr(me), _ptr(sh), _ptr(sc), ctypes.c_void_p(s.cuda_stream))
        self._check(rc)
        return me, sh, sc

    def unweight(self, me, wgt, rnd=None, stream=None, want_w=True, want_accept=True):
        """GPU-assisted batch unweighting of device tensors: (w, accept, w_max, n_accept),
        all device tensors (w_max and n_accept one element each); asynchronous."""
        import torch
        n = me.shape[0]
        dev = me.device
        w = torch.empty(n, dtype=torch.float64, device=dev) if want_w else None
        acc = torch.empty(n, dtype=torch.uint8, device=dev) if (want_accept and rnd is not None) else None
        wmax = torch.empty(1, dtype=torch.float64, device=dev)
        nacc = torch.empty(1, dtype=torch.int64, device=dev) if rnd is not None else None
        s = stream if stream is not None else torch.cuda.current_stream(dev)
        self._check(self.lib.me_unweight(self.handle, n, _ptr(me), _ptr(wgt), _ptr(rnd), _ptr(w), _ptr(acc),
                                         _ptr(wmax), _ptr(nacc), ctypes.c_void_p(s.cuda_stream)))
        return w, acc, wmax, nacc

    def compute_unweight(self, momenta, alphas, rnd_hel, rnd_col, wgt, rnd, stream=None):
        """me_compute_unweight on device tensors: (me, sel_hel, sel_col, w, accept, w_max,
        n_accept), asynchronous on ``stream``"""
        import torch
        nevt = momenta.shape[0]
        dev = momenta.device
        out = (torch.empty(nevt, dtype=torch.float64, device=dev),
               torch.empty(nevt, dtype=torch.int32, device=dev) if rnd_hel is not None else None,
               torch.empty(nevt, dtype=torch.int32, device=dev) if rnd_col is not None else None)
        self._check_args(momenta, alphas, rnd_hel, rnd_col, out, dev)
        _check_tensor("wgt", wgt, torch.float64, (nevt,), dev, required=True)
        _check_tensor("rnd", rnd, torch.float64, (nevt,), dev)
        w = torch.empty(nevt, dtype=torch.float64, device=dev)
        acc = torch.empty(nevt, dtype=torch.uint8, device=dev) if rnd is not None else None
        wmax = torch.empty(1, dtype=torch.float64, device=dev)
        nacc = torch.empty(1, dtype=torch.int64, device=dev) if rnd is not None else None
        s = stream if stream is not None else torch.cuda.current_stream(dev)
        self._check(self.lib.me_compute_unweight(self.handle, nevt, _ptr(momenta), _ptr(alphas), _ptr(rnd_hel),
                                                 _ptr(rnd_col), _ptr(wgt), _ptr(rnd), _ptr(out[0]), _ptr(out[1]),
                                                 _ptr(out[2]), _ptr(w), _ptr(acc), _ptr(wmax), _ptr(nacc),
                                                 ctypes.c_void_p(s.cuda_stream)))
        return out + (w, acc, wmax, nacc)

    def rambo(self, nevt, seed=0, first_event=0, sqrt_s=1500.0, stream=None):
        """RAMBO momenta for this process generated on the device: a [nevt][npar][4] tensor"""
        import torch
        s = stream if stream is not None else torch.cuda.current_stream()
        mom = torch.empty((nevt, self.npar, 4), dtype=torch.float64, device=s.device)
        self._check(self.lib.me_rambo(self.handle, nevt, seed, first_event, sqrt_s, _ptr(mom),
                                      ctypes.c_void_p(s.cuda_stream)))
        return mom

    def compute_raw(self, nevt, momenta_ptr, alphas_ptr, rnd_hel_ptr, rnd_col_ptr, me_ptr, sel_hel_ptr,
                    sel_col_ptr, stream_ptr):
        """Raw device pointers (integers or None)."""
        rc = self.lib.me_compute(self.handle, nevt, momenta_ptr, alphas_ptr, rnd_hel_ptr, rnd_col_ptr, me_ptr,
                                 sel_hel_ptr, sel_col_ptr, stream_ptr)
        self._check(rc)

    def compute_host(self, momenta, alphas=None, rnd_hel=None, rnd_col=None, out=None, stream=None):
        """Host (ideally pinned) tensors in and out; the copies happen inside the library.
        Every tensor must be a contiguous CPU tensor of the documented dtype and length."""
        import torch
        nevt = momenta.shape[0]
        if out is None:
            me = torch.empty(nevt, dtype=torch.float64).pin_memory()
            sh = torch.empty(nevt, dtype=torch.int32).pin_memory() if rnd_hel is not None else None
            sc = torch.empty(nevt, dtype=torch.int32).pin_memory() if rnd_col is not None else None
        else:
            me, sh, sc = out
        self._check_args(momenta, alphas, rnd_hel, rnd_col, (me, sh, sc), torch.device("cpu"))
        s = stream if stream is not None else torch.cuda.current_stream()
        rc = self.lib.me_compute_host(self.handle, nevt, _ptr(momenta), _ptr(alphas), _ptr(rnd_hel), _ptr(rnd_col),
                                      _ptr(me), _ptr(sh), _ptr(sc), ctypes.c_void_p(s.cuda_stream))
        self._check(rc)
        return me, sh, sc

    def sync_status(self, stream=None):
        """wait for ``stream``; raise MEError(ME_ERR_TIMEOUT) if a device-side wait of an
        earlier call on this handle ran out (the flag is cleared by reporting it)"""
        import torch
        s = stream if stream is not None else torch.cuda.current_stream()
        self._check(self.lib.me_sync_status(self.handle, ctypes.c_void_p(s.cuda_stream)))

    def set_wait_limit(self, polls: int):
        """testing hook: polls of the mixed kernel's MMA wait (negative: default; 0: give up at once)"""
        self._check(self.lib.me_set_wait_limit(self.handle, polls))

    def close(self):
        if getattr(self, "handle", None):
            self.lib.me_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
