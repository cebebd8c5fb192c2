"""GB300 (sm_103a) MFA value/gradient queries and MFA ray casting.

Thin Python binding over the C ABI of libmfa (include/mfa.h): the functions here only
marshal arguments -- every step of a query or a render runs in the library's CUDA
kernels.  PyTorch provides device memory and the current CUDA stream; nothing else.

    import paper_2312_15073_gb300 as mfa
    m = mfa.Model((3, 3, 3), (128, 128, 128), None, ctrl_numpy)   # clamped uniform knots
    val, grad = mfa.decode(m, pts_cuda)                             # (n,), (n, 3)
    img = mfa.render(m, camera, tf, 1024, 1024, 1024)               # (H, W, 4) premultiplied

The library must have been built (``paper_2312_15073_gb300.build.build()``); a missing
library raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import math
import os
from ctypes import POINTER, c_double, c_float, c_int, c_longlong, c_size_t, c_ulonglong, c_void_p

import numpy as np

__all__ = ["Model", "decode", "locate_spans", "render", "lib", "MFA_F64", "MFA_F32", "MFA_F16", "MFA_BF16",
           "MfaError", "camera", "transfer_fn", "Request", "Batch", "render_batch", "render_batch_static", "Server", "server_now", "tune_render", "tune_batch", "tune_save", "tune_load"]

MFA_F64, MFA_F32, MFA_F16, MFA_BF16 = 0, 1, 2, 3
MFA_WINDOW_AUTO, MFA_WINDOW_F32, MFA_WINDOW_COMPACT, MFA_WINDOW_PATCH = 0, 1, 2, 3
_PKG = os.path.dirname(os.path.abspath(__file__))
# The library the binding loads: libmfa.so, or the file MFA_LIB names (e.g. the debug
# build libmfa_debug.so).  A missing library raises; there is no fallback.
LIB_PATH = os.environ.get("MFA_LIB") or os.path.join(_PKG, "libmfa.so")


class MfaError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"mfa error {code}: {msg}")
        self.code = code


class _Camera(ctypes.Structure):
    _fields_ = [("projection", c_int), ("eye", c_double * 3), ("target", c_double * 3), ("up", c_double * 3),
                ("fov_y_deg", c_double), ("ortho_height", c_double)]


class _TF(ctypes.Structure):
    _fields_ = [("n_entries", c_int), ("rgba", c_void_p), ("vmin", c_float), ("vmax", c_float),
                ("shading", c_int), ("ka", c_float), ("kd", c_float), ("ks", c_float), ("shininess", c_float),
                ("ert_alpha", c_float)]


class _Opts(ctypes.Structure):
    _fields_ = [("samples_out", c_void_p), ("variant", c_int), ("tile_shape", c_int), ("use_tuned", c_int),
                ("reserved", c_int * 5)]


class _TuneResult(ctypes.Structure):
    _fields_ = [("variant", c_int), ("tile_shape", c_int), ("ms", c_float)]


class _Request(ctypes.Structure):
    _fields_ = [("model", c_void_p), ("camera", _Camera), ("tf", c_void_p), ("width", c_int), ("height", c_int),
                ("n_samples", c_int), ("rgba_out", c_void_p), ("samples_out", c_void_p)]


class _ServerConfig(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", c_size_t), ("max_slots", c_int), ("max_queue", c_int),
                ("priority_levels", c_int), ("variant", c_int), ("tile_shape", c_int), ("use_tuned", c_int),
                ("mode", c_int), ("urgency_rate", c_double)]


class _ServeRequest(ctypes.Structure):
    _fields_ = [("model", c_void_p), ("camera", _Camera), ("tf", c_void_p), ("width", c_int), ("height", c_int),
                ("n_samples", c_int), ("arrival_time_s", c_double)]


class _ServerStats(ctypes.Structure):
    _fields_ = [(n, c_longlong) for n in ("submitted", "completed", "failed", "rejected_busy", "cancelled",
                                          "peak_in_flight", "peak_arena_bytes", "in_flight", "queued",
                                          "arena_bytes_in_use")]


class _Peaks(ctypes.Structure):
    _fields_ = [("fp32_tflops", ctypes.c_double), ("fp32x2_tflops", ctypes.c_double),
                ("l2_gather_gbs", ctypes.c_double), ("fma_clock_mhz", ctypes.c_double), ("sm_count", c_int)]


class _MlSignal(ctypes.Structure):
    _fields_ = [("f_m", ctypes.c_double), ("alpha", ctypes.c_double)]


class _Quality(ctypes.Structure):
    _fields_ = [("mse", ctypes.c_double), ("psnr_db", ctypes.c_double), ("ssim", ctypes.c_double)]


class _EncodeConfig(ctypes.Structure):
    _fields_ = [("err_max", ctypes.c_double), ("max_ctrl", c_int * 3), ("max_iter", c_int)]


class _EncodeResult(ctypes.Structure):
    _fields_ = [("iterations", c_int), ("max_err", ctypes.c_double), ("nctrl", c_int * 3)]


class _Info(ctypes.Structure):
    _fields_ = [("degree", c_int * 3), ("nctrl", c_int * 3), ("storage", c_int), ("vmin", c_float),
                ("vmax", c_float), ("device_bytes", c_size_t), ("device", c_int), ("cardinal", c_int),
                ("window", c_int)]


_lib = None


def lib():
    """The loaded libmfa (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2312_15073_gb300.build.build() "
                               "(there is no fallback implementation)")
        L = ctypes.CDLL(LIB_PATH)
        L.mfa_last_error.restype = ctypes.c_char_p
        L.mfa_last_error.argtypes = []
        L.mfa_set_stream.restype = c_int
        L.mfa_set_stream.argtypes = [c_void_p]
        L.mfa_model_create_opts.restype = c_void_p
        L.mfa_model_create_opts.argtypes = [POINTER(c_int * 3), POINTER(c_int * 3), POINTER(c_void_p * 3), c_void_p,
                                            c_int, c_int, c_int]
        L.mfa_model_create_ex.restype = c_void_p
        L.mfa_model_create_ex.argtypes = [POINTER(c_int * 3), POINTER(c_int * 3), POINTER(c_void_p * 3), c_void_p,
                                          c_int, c_int]
        L.mfa_model_create.restype = c_void_p
        L.mfa_model_create.argtypes = [POINTER(c_int * 3), POINTER(c_int * 3), POINTER(c_void_p * 3), c_void_p, c_int]
        L.mfa_model_destroy.restype = None
        L.mfa_model_destroy.argtypes = [c_void_p]
        L.mfa_model_get_info.restype = c_int
        L.mfa_model_get_info.argtypes = [c_void_p, POINTER(_Info)]
        L.mfa_decode.restype = c_int
        L.mfa_decode.argtypes = [c_void_p, c_void_p, c_longlong, c_void_p, c_void_p]
        L.mfa_locate_spans.restype = c_int
        L.mfa_locate_spans.argtypes = [c_void_p, c_void_p, c_longlong, c_void_p]
        L.mfa_render.restype = c_int
        L.mfa_render.argtypes = [c_void_p, POINTER(_Camera), POINTER(_TF), c_int, c_int, c_int, c_void_p]
        L.mfa_render_ex.restype = c_int
        L.mfa_render_ex.argtypes = [c_void_p, POINTER(_Camera), POINTER(_TF), c_int, c_int, c_int, c_void_p,
                                    POINTER(_Opts)]
        L.mfa_fit_ctrl.restype = c_int
        L.mfa_fit_ctrl.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]
        L.mfa_model_fit.restype = c_void_p
        L.mfa_model_fit.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_void_p]
        L.mfa_model_encode.restype = c_void_p
        L.mfa_model_encode.argtypes = [c_void_p, c_void_p, c_void_p, c_int, POINTER(_EncodeConfig),
                                       POINTER(_EncodeResult)]
        L.mfa_render_iso.restype = c_int
        L.mfa_render_iso.argtypes = [c_void_p, POINTER(_Camera), POINTER(_TF), c_int, c_int, c_int, c_float, c_void_p,
                                     c_void_p, POINTER(_Opts)]
        L.mfa_render_segments.restype = c_int
        L.mfa_render_segments.argtypes = [c_void_p, POINTER(_Camera), POINTER(_TF), c_int, c_int, c_int, c_void_p,
                                          c_void_p, POINTER(_Opts)]
        L.mfa_debug_build.restype = c_int
        L.mfa_debug_build.argtypes = []
        L.mfa_debug_status.restype = c_int
        L.mfa_debug_status.argtypes = [POINTER(ctypes.c_uint), POINTER(ctypes.c_uint)]
        L.mfa_model_get_ctrl.restype = c_int
        L.mfa_model_get_ctrl.argtypes = [c_void_p, c_void_p]
        L.mfa_model_save.restype = c_int
        L.mfa_model_save.argtypes = [c_void_p, ctypes.c_char_p]
        L.mfa_model_load.restype = c_void_p
        L.mfa_model_load.argtypes = [ctypes.c_char_p]
        L.mfa_render_ml.restype = c_int
        L.mfa_render_ml.argtypes = [POINTER(_MlSignal), POINTER(_Camera), POINTER(_TF), c_int, c_int, c_int, c_void_p,
                                    POINTER(_Opts)]
        L.mfa_image_compare.restype = c_int
        L.mfa_image_compare.argtypes = [c_void_p, c_void_p, c_int, c_int, POINTER(_Quality)]
        L.mfa_measure_peaks.restype = c_int
        L.mfa_measure_peaks.argtypes = [POINTER(_Peaks)]
        L.mfa_decode_host.restype = c_int
        L.mfa_decode_host.argtypes = [c_void_p, c_void_p, c_longlong, c_void_p, c_void_p]
        L.mfa_render_host.restype = c_int
        L.mfa_render_host.argtypes = [c_void_p, POINTER(_Camera), POINTER(_TF), c_int, c_int, c_int, c_void_p,
                                      POINTER(_Opts)]
        L.mfa_batch_create.restype = c_void_p
        L.mfa_batch_create.argtypes = [c_int]
        L.mfa_batch_configure.restype = c_int
        L.mfa_batch_configure.argtypes = [c_void_p, c_int, c_int]
        L.mfa_batch_render.restype = c_int
        L.mfa_batch_render.argtypes = [c_void_p, c_void_p, c_int]
        L.mfa_batch_destroy.restype = None
        L.mfa_batch_destroy.argtypes = [c_void_p]
        L.mfa_render_batch.restype = c_int
        L.mfa_render_batch.argtypes = [c_void_p, c_int]
        L.mfa_server_now.restype = c_double
        L.mfa_server_now.argtypes = []
        L.mfa_server_create.restype = c_void_p
        L.mfa_server_create.argtypes = [POINTER(_ServerConfig)]
        L.mfa_server_submit.restype = c_int
        L.mfa_server_submit.argtypes = [c_void_p, POINTER(_ServeRequest), POINTER(c_longlong)]
        L.mfa_server_poll.restype = c_int
        L.mfa_server_poll.argtypes = [c_void_p, c_longlong, POINTER(c_int), POINTER(c_double)]
        L.mfa_server_wait.restype = c_int
        L.mfa_server_wait.argtypes = [c_void_p, c_longlong, c_double, POINTER(c_double)]
        L.mfa_server_result.restype = c_int
        L.mfa_server_result.argtypes = [c_void_p, c_longlong, POINTER(c_void_p)]
        L.mfa_server_copy_result.restype = c_int
        L.mfa_server_copy_result.argtypes = [c_void_p, c_longlong, c_void_p, c_size_t]
        L.mfa_server_release.restype = c_int
        L.mfa_server_release.argtypes = [c_void_p, c_longlong]
        L.mfa_server_get_stats.restype = c_int
        L.mfa_server_get_stats.argtypes = [c_void_p, POINTER(_ServerStats)]
        L.mfa_server_destroy.restype = None
        L.mfa_server_destroy.argtypes = [c_void_p]
        L.mfa_tune_render.restype = c_int
        L.mfa_tune_render.argtypes = [c_void_p, POINTER(_Camera), POINTER(_TF), c_int, c_int, c_int, c_void_p, c_int,
                                      POINTER(_TuneResult), c_void_p, c_int, POINTER(c_int)]
        L.mfa_tune_batch.restype = c_int
        L.mfa_tune_batch.argtypes = [c_void_p, c_void_p, c_int, c_int, POINTER(_TuneResult)]
        L.mfa_tune_lookup.restype = c_int
        L.mfa_tune_lookup.argtypes = [c_void_p, c_int, c_int, c_int, POINTER(_TuneResult)]
        L.mfa_tune_save.restype = c_int
        L.mfa_tune_save.argtypes = [ctypes.c_char_p]
        L.mfa_tune_load.restype = c_int
        L.mfa_tune_load.argtypes = [ctypes.c_char_p]
        L.mfa_render_batch_static.restype = c_int
        L.mfa_render_batch_static.argtypes = [c_void_p, c_int]
        _lib = L
    return _lib


def _check(rc: int):
    if rc != 0:
        raise MfaError(rc, lib().mfa_last_error().decode())


def _bind_stream():
    import torch
    lib().mfa_set_stream(c_void_p(torch.cuda.current_stream().cuda_stream))


_NP2MFA = {np.dtype(np.float64): MFA_F64, np.dtype(np.float32): MFA_F32, np.dtype(np.float16): MFA_F16}


class Model:
    """An MFA model on the current CUDA device (owns its device memory).

    ctrl: host array (n_z, n_y, n_x).  Its numpy dtype gives the input type (float64,
    float32, float16; pass `in_dtype=MFA_BF16` with a uint16 array for BF16 bits).
    knots: None for clamped uniform, or a list of three FP64 arrays (entries may be None).
    storage: MFA_F32 / MFA_F16 / MFA_BF16 (default: F32 for 64/32-bit input).
    window: MFA_WINDOW_AUTO (the storage type's own window values), MFA_WINDOW_F32 (FP32
    window values whatever the storage type: a 16-bit model at FP32 speed),
    MFA_WINDOW_COMPACT (no layer-pair window: the control points at 1-1.6x) or
    MFA_WINDOW_PATCH (degree 3: the FP32 window plus each knot-span cell's polynomial,
    rendered by variant 8; about 7x the window's bytes).
    """

    def __init__(self, degree, nctrl, knots, ctrl, storage: int | None = None, in_dtype: int | None = None,
                 window: int = 0):
        import torch  # noqa: F401  (makes sure the CUDA context exists on the current device)
        ctrl = np.ascontiguousarray(ctrl)
        if in_dtype is None:
            if ctrl.dtype not in _NP2MFA:
                raise TypeError(f"unsupported control-point dtype {ctrl.dtype}")
            in_dtype = _NP2MFA[ctrl.dtype]
        if storage is None:
            storage = {MFA_F64: MFA_F32, MFA_F32: MFA_F32, MFA_F16: MFA_F16, MFA_BF16: MFA_BF16}[in_dtype]
        deg = (c_int * 3)(*[int(d) for d in degree])
        nc = (c_int * 3)(*[int(n) for n in nctrl])
        self._knots = None
        kp = None
        if knots is not None:
            self._knots = [None if k is None else np.ascontiguousarray(k, dtype=np.float64) for k in knots]
            kp = (c_void_p * 3)(*[None if k is None else k.ctypes.data for k in self._knots])
        self._ctrl_keep = ctrl
        _bind_stream()
        h = lib().mfa_model_create_opts(ctypes.byref(deg), ctypes.byref(nc),
                                        ctypes.byref(kp) if kp is not None else None, ctrl.ctypes.data, in_dtype,
                                        storage, int(window))
        self._ctrl_keep = None
        if not h:
            raise MfaError(-1, lib().mfa_last_error().decode())
        self._h = h
        self.degree = tuple(int(d) for d in degree)
        self.nctrl = tuple(int(n) for n in nctrl)
        self.storage = storage

    @classmethod
    def _wrap(cls, h, storage: int) -> "Model":
        """A Model owning an existing handle (made by the library, e.g. by a fit)."""
        m = cls.__new__(cls)
        m._h = h
        m._knots = None
        m._ctrl_keep = None
        i = _Info()
        _check(lib().mfa_model_get_info(h, ctypes.byref(i)))
        m.degree = tuple(i.degree)
        m.nctrl = tuple(i.nctrl)
        m.storage = storage
        return m

    @property
    def handle(self) -> int:
        return self._h

    def info(self) -> dict:
        i = _Info()
        _check(lib().mfa_model_get_info(self._h, ctypes.byref(i)))
        return dict(degree=tuple(i.degree), nctrl=tuple(i.nctrl), storage=i.storage, vmin=i.vmin, vmax=i.vmax,
                    device_bytes=i.device_bytes, device=i.device, cardinal=bool(i.cardinal), window=i.window)

    def ctrl(self) -> np.ndarray:
        """The stored control points (n_z, n_y, n_x): float32, float16, or uint16 BF16 bits."""
        n = self.nctrl
        dt = {MFA_F32: np.float32, MFA_F16: np.float16, MFA_BF16: np.uint16}[self.storage]
        out = np.empty((n[2], n[1], n[0]), dtype=dt)
        _bind_stream()
        _check(lib().mfa_model_get_ctrl(self._h, out.ctypes.data))
        return out

    def save(self, path: str):
        """Writes the model (degrees, FP64 knots, stored control points) to a file."""
        _bind_stream()
        _check(lib().mfa_model_save(self._h, os.fsencode(path)))

    @classmethod
    def load(cls, path: str) -> "Model":
        """A model read from a file written by save(), on the current device."""
        _bind_stream()
        h = lib().mfa_model_load(os.fsencode(path))
        if not h:
            raise MfaError(-1, lib().mfa_last_error().decode())
        i = _Info()
        _check(lib().mfa_model_get_info(h, ctypes.byref(i)))
        return cls._wrap(h, i.storage)

    def close(self):
        if getattr(self, "_h", None):
            lib().mfa_model_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _dev_ptr(t, dtype, shape_tail, name):
    import torch
    if t is None:
        return None
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous CUDA tensor of {dtype}")
    if shape_tail is not None and tuple(t.shape[1:]) != tuple(shape_tail):
        raise ValueError(f"{name} must have shape (n, {', '.join(map(str, shape_tail))})")
    return t.data_ptr()


def decode(model: Model, pts, val=None, grad=None, want_grad: bool = True):
    """Value (n,) and gradient (n, 3) at pts (n, 3) FP32 CUDA; outputs allocated if not given."""
    import torch
    n = pts.shape[0]
    if val is None:
        val = torch.empty(n, device=pts.device, dtype=torch.float32)
    if grad is None and want_grad:
        grad = torch.empty((n, 3), device=pts.device, dtype=torch.float32)
    _bind_stream()
    _check(lib().mfa_decode(model.handle, _dev_ptr(pts, torch.float32, (3,), "pts"), n,
                            _dev_ptr(val, torch.float32, None, "val"), _dev_ptr(grad, torch.float32, (3,), "grad")))
    return val, grad


def locate_spans(model: Model, pts, spans=None):
    import torch
    n = pts.shape[0]
    if spans is None:
        spans = torch.empty((n, 3), device=pts.device, dtype=torch.int32)
    _bind_stream()
    _check(lib().mfa_locate_spans(model.handle, _dev_ptr(pts, torch.float32, (3,), "pts"), n,
                                  _dev_ptr(spans, torch.int32, (3,), "spans")))
    return spans


def camera(cam: dict) -> _Camera:
    c = _Camera()
    c.projection = int(cam["projection"])
    for a in range(3):
        c.eye[a] = float(cam["eye"][a])
        c.target[a] = float(cam["target"][a])
        c.up[a] = float(cam["up"][a])
    c.fov_y_deg = float(cam.get("fov_y_deg", 0.0))
    c.ortho_height = float(cam.get("ortho_height", 0.0))
    return c


class transfer_fn:
    """Transfer function + shading parameters (the table stays alive with this object)."""

    def __init__(self, rgba, *, shading=False, ka=0.3, kd=0.6, ks=0.3, shininess=32.0, ert_alpha=0.99,
                 vmin=math.nan, vmax=math.nan):
        self.table = np.ascontiguousarray(rgba, dtype=np.float32).reshape(-1, 4)
        s = _TF()
        s.n_entries = self.table.shape[0]
        s.rgba = self.table.ctypes.data
        s.vmin, s.vmax = vmin, vmax
        s.shading = 1 if shading else 0
        s.ka, s.kd, s.ks, s.shininess = ka, kd, ks, shininess
        s.ert_alpha = ert_alpha
        self.struct = s


def render(model: Model, cam, tf: transfer_fn, width: int, height: int, n_samples: int, out=None,
           samples_out=None, variant: int = 0, tile_shape: int = 0, use_tuned: bool = False):
    """Premultiplied RGBA image (height, width, 4) FP32 on the current device.
    samples_out: optional 1-element int64 CUDA tensor to which the number of evaluated
    samples is added."""
    import torch
    if out is None:
        out = torch.empty((height, width, 4), device="cuda", dtype=torch.float32)
    if not (out.is_cuda and out.dtype == torch.float32 and out.is_contiguous() and out.numel() == height * width * 4):
        raise ValueError("out must be a contiguous (height, width, 4) FP32 CUDA tensor")
    c = cam if isinstance(cam, _Camera) else camera(cam)
    opts = _Opts()
    opts.variant = int(variant)
    opts.tile_shape = int(tile_shape)
    opts.use_tuned = 1 if use_tuned else 0
    if samples_out is not None:
        if not (samples_out.is_cuda and samples_out.dtype == torch.int64):
            raise TypeError("samples_out must be an int64 CUDA tensor")
        opts.samples_out = samples_out.data_ptr()
    _bind_stream()
    _check(lib().mfa_render_ex(model.handle, ctypes.byref(c), ctypes.byref(tf.struct), width, height, n_samples,
                               out.data_ptr(), ctypes.byref(opts)))
    return out


def debug_status() -> dict:
    """Device-side index checks of a debug build (libmfa_debug.so): the flags raised and the
    number of bad indices since the last call (both 0 in a release build)."""
    f, c = ctypes.c_uint(), ctypes.c_uint()
    _check(lib().mfa_debug_status(ctypes.byref(f), ctypes.byref(c)))
    return {"debug_build": bool(lib().mfa_debug_build()), "flags": f.value, "count": c.value}


def measure_peaks() -> dict:
    """Calibration kernels for the roofline denominators on the current device: FP32 FMA
    rate (scalar and packed FP32x2) and the L2 rate of random 32-byte gathers."""
    p = _Peaks()
    _bind_stream()
    _check(lib().mfa_measure_peaks(ctypes.byref(p)))
    return dict(fp32_tflops=p.fp32_tflops, fp32x2_tflops=p.fp32x2_tflops, l2_gather_gbs=p.l2_gather_gbs,
                fma_clock_mhz=p.fma_clock_mhz, sm_count=p.sm_count)


def _host_ptr(t, shape_tail, name):
    import torch
    if t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous FP32 CPU tensor")
    if shape_tail is not None and tuple(t.shape[1:]) != shape_tail:
        raise ValueError(f"{name} must have shape (n, {shape_tail[0]})")
    return t.data_ptr()


def decode_host(model: Model, pts, val=None, grad=None, want_grad: bool = True, sync: bool = True):
    """decode() for HOST data: pts (n, 3) FP32 CPU tensor (page-locked for overlapped copies);
    returns CPU tensors val (n,) and grad (n, 3) (allocated page-locked if not given).  The
    library stages and pipelines the copies; with sync=False the call only enqueues the work
    on the current stream, which must be synchronised before the outputs are read."""
    import torch
    n = pts.shape[0]
    pin = pts.is_pinned()
    if val is None:
        val = torch.empty(n, dtype=torch.float32, pin_memory=pin)
    if grad is None and want_grad:
        grad = torch.empty((n, 3), dtype=torch.float32, pin_memory=pin)
    _bind_stream()
    _check(lib().mfa_decode_host(model.handle, _host_ptr(pts, (3,), "pts"), n, _host_ptr(val, None, "val"),
                                 _host_ptr(grad, (3,), "grad") if grad is not None else None))
    if sync:
        torch.cuda.current_stream().synchronize()
    return val, grad


def render_host(model: Model, cam, tf: transfer_fn, width: int, height: int, n_samples: int, out=None,
                samples_out=None, variant: int = 0, tile_shape: int = 0, use_tuned: bool = False, sync: bool = True):
    """render() into a HOST image: out (height, width, 4) FP32 CPU tensor (allocated
    page-locked if not given).  With sync=False the call only enqueues the work on the
    current stream, which must be synchronised before the image is read."""
    import torch
    if out is None:
        out = torch.empty((height, width, 4), dtype=torch.float32, pin_memory=True)
    if out.numel() != height * width * 4:
        raise ValueError("out must hold (height, width, 4) FP32 values")
    c = cam if isinstance(cam, _Camera) else camera(cam)
    opts = _Opts()
    opts.variant = int(variant)
    opts.tile_shape = int(tile_shape)
    opts.use_tuned = 1 if use_tuned else 0
    if samples_out is not None:
        if not (samples_out.is_cuda and samples_out.dtype == torch.int64):
            raise TypeError("samples_out must be an int64 CUDA tensor")
        opts.samples_out = samples_out.data_ptr()
    _bind_stream()
    _check(lib().mfa_render_host(model.handle, ctypes.byref(c), ctypes.byref(tf.struct), width, height, n_samples,
                                 _host_ptr(out, None, "out"), ctypes.byref(opts)))
    if sync:
        torch.cuda.current_stream().synchronize()
    return out


def _fit_data(data):
    import torch
    if not (data.is_cuda and data.dtype == torch.float32 and data.is_contiguous() and data.dim() == 3):
        raise ValueError("data must be a contiguous (m_z, m_y, m_x) FP32 CUDA tensor")
    mz, my, mx = data.shape
    return (c_int * 3)(int(mx), int(my), int(mz))


def _knot_ptrs(knots):
    if knots is None:
        return None, None
    keep = [None if k is None else np.ascontiguousarray(k, dtype=np.float64) for k in knots]
    return keep, (c_void_p * 3)(*[None if k is None else k.ctypes.data for k in keep])


def fit_ctrl(degree, nctrl, knots, data):
    """Least-squares control points (n_z, n_y, n_x) FP64 CUDA tensor of a fit to data
    (m_z, m_y, m_x) FP32 CUDA tensor at uniform parameters."""
    import torch
    md = _fit_data(data)
    deg = (c_int * 3)(*[int(d) for d in degree])
    nc = (c_int * 3)(*[int(n) for n in nctrl])
    keep, kp = _knot_ptrs(knots)
    out = torch.empty((int(nctrl[2]), int(nctrl[1]), int(nctrl[0])), device="cuda", dtype=torch.float64)
    _bind_stream()
    _check(lib().mfa_fit_ctrl(ctypes.byref(deg), ctypes.byref(nc), ctypes.byref(kp) if kp is not None else None,
                              ctypes.byref(md), data.data_ptr(), out.data_ptr()))
    return out


def model_fit(degree, nctrl, knots, data, storage: int = MFA_F32):
    """(Model of the least-squares fit, largest error at the data points)."""
    md = _fit_data(data)
    deg = (c_int * 3)(*[int(d) for d in degree])
    nc = (c_int * 3)(*[int(n) for n in nctrl])
    keep, kp = _knot_ptrs(knots)
    err = ctypes.c_double()
    _bind_stream()
    h = lib().mfa_model_fit(ctypes.byref(deg), ctypes.byref(nc), ctypes.byref(kp) if kp is not None else None,
                            ctypes.byref(md), data.data_ptr(), int(storage), ctypes.byref(err))
    if not h:
        raise MfaError(-1, lib().mfa_last_error().decode())
    return Model._wrap(h, storage), err.value


def model_encode(degree, data, err_max: float, max_ctrl=(0, 0, 0), max_iter: int = 64, storage: int = MFA_F32):
    """Adaptive encoding of data (m_z, m_y, m_x) FP32 CUDA tensor: (Model, result dict with
    iterations, max_err, nctrl)."""
    md = _fit_data(data)
    deg = (c_int * 3)(*[int(d) for d in degree])
    cfg = _EncodeConfig(float(err_max), (c_int * 3)(*[int(x) for x in max_ctrl]), int(max_iter))
    res = _EncodeResult()
    _bind_stream()
    h = lib().mfa_model_encode(ctypes.byref(deg), ctypes.byref(md), data.data_ptr(), int(storage), ctypes.byref(cfg),
                               ctypes.byref(res))
    if not h:
        raise MfaError(-1, lib().mfa_last_error().decode())
    return Model._wrap(h, storage), dict(iterations=res.iterations, max_err=res.max_err, nctrl=tuple(res.nctrl))


def render_iso(model: Model, cam, tf: transfer_fn, width: int, height: int, n_samples: int, iso: float, out=None,
               depth=None, samples_out=None, tile_shape: int = 0):
    """Isosurface f = iso: (rgba (height, width, 4), depth (height, width)) CUDA tensors;
    opaque shaded hits, transparent black and depth +inf where a ray has no crossing."""
    import torch
    if out is None:
        out = torch.empty((height, width, 4), device="cuda", dtype=torch.float32)
    if depth is None:
        depth = torch.empty((height, width), device="cuda", dtype=torch.float32)
    for t, name, n in ((out, "out", height * width * 4), (depth, "depth", height * width)):
        if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous() and t.numel() == n):
            raise ValueError(f"{name} must be a contiguous FP32 CUDA tensor of {n} values")
    c = cam if isinstance(cam, _Camera) else camera(cam)
    opts = _Opts()
    opts.tile_shape = int(tile_shape)
    if samples_out is not None:
        if not (samples_out.is_cuda and samples_out.dtype == torch.int64):
            raise TypeError("samples_out must be an int64 CUDA tensor")
        opts.samples_out = samples_out.data_ptr()
    _bind_stream()
    _check(lib().mfa_render_iso(model.handle, ctypes.byref(c), ctypes.byref(tf.struct), width, height, n_samples,
                                float(iso), out.data_ptr(), depth.data_ptr(), ctypes.byref(opts)))
    return out, depth


def render_ml(cam, tf: transfer_fn, width: int, height: int, n_samples: int, f_m: float = 6.0, alpha: float = 0.25,
              out=None, samples_out=None, tile_shape: int = 0):
    """Render of the closed-form Marschner-Lobb signal (the render-quality ground truth) with
    the rays, samples, shading and compositing of render(): a (height, width, 4) CUDA tensor."""
    import torch
    if out is None:
        out = torch.empty((height, width, 4), device="cuda", dtype=torch.float32)
    if not (out.is_cuda and out.dtype == torch.float32 and out.is_contiguous() and out.numel() == height * width * 4):
        raise ValueError("out must be a contiguous (height, width, 4) FP32 CUDA tensor")
    c = cam if isinstance(cam, _Camera) else camera(cam)
    sig = _MlSignal(float(f_m), float(alpha))
    opts = _Opts()
    opts.tile_shape = int(tile_shape)
    if samples_out is not None:
        if not (samples_out.is_cuda and samples_out.dtype == torch.int64):
            raise TypeError("samples_out must be an int64 CUDA tensor")
        opts.samples_out = samples_out.data_ptr()
    _bind_stream()
    _check(lib().mfa_render_ml(ctypes.byref(sig), ctypes.byref(c), ctypes.byref(tf.struct), width, height, n_samples,
                               out.data_ptr(), ctypes.byref(opts)))
    return out


def image_compare(test, ref) -> dict:
    """MSE, PSNR (dB) and SSIM of two (height, width, 4) FP32 CUDA images (RGB on the
    0..255 display scale)."""
    for t, name in ((test, "test"), (ref, "ref")):
        if not (t.is_cuda and t.dtype.is_floating_point and t.element_size() == 4 and t.is_contiguous()
                and t.dim() == 3 and t.shape[2] == 4):
            raise ValueError(f"{name} must be a contiguous (height, width, 4) FP32 CUDA tensor")
    if test.shape != ref.shape:
        raise ValueError("images differ in shape")
    q = _Quality()
    _bind_stream()
    _check(lib().mfa_image_compare(test.data_ptr(), ref.data_ptr(), test.shape[1], test.shape[0], ctypes.byref(q)))
    return {"mse": q.mse, "psnr_db": q.psnr_db, "ssim": q.ssim}


def render_segments(model: Model, cam, tf: transfer_fn, width: int, height: int, n_samples: int, blocks, out=None,
                    samples_out=None, variant: int = 0, tile_shape: int = 0):
    """render() with the object-space decomposition: the box split into blocks[0] x
    blocks[1] x blocks[2] blocks, each rendering its ray segments into a partial image,
    merged with over nearest segment first."""
    import torch
    if out is None:
        out = torch.empty((height, width, 4), device="cuda", dtype=torch.float32)
    if not (out.is_cuda and out.dtype == torch.float32 and out.is_contiguous() and out.numel() == height * width * 4):
        raise ValueError("out must be a contiguous (height, width, 4) FP32 CUDA tensor")
    c = cam if isinstance(cam, _Camera) else camera(cam)
    g = (c_int * 3)(*[int(b) for b in blocks])
    opts = _Opts()
    opts.variant = int(variant)
    opts.tile_shape = int(tile_shape)
    if samples_out is not None:
        if not (samples_out.is_cuda and samples_out.dtype == torch.int64):
            raise TypeError("samples_out must be an int64 CUDA tensor")
        opts.samples_out = samples_out.data_ptr()
    _bind_stream()
    _check(lib().mfa_render_segments(model.handle, ctypes.byref(c), ctypes.byref(tf.struct), width, height, n_samples,
                                     ctypes.byref(g), out.data_ptr(), ctypes.byref(opts)))
    return out


class Request:
    """One image of a batch: the arguments of one render() call."""

    def __init__(self, model: Model, cam, tf: transfer_fn, width: int, height: int, n_samples: int, out=None,
                 samples_out=None):
        import torch
        self.model, self.cam, self.tf = model, cam, tf
        self.width, self.height, self.n_samples = int(width), int(height), int(n_samples)
        self.out = out if out is not None else torch.empty((height, width, 4), device="cuda", dtype=torch.float32)
        if not (self.out.is_cuda and self.out.dtype == torch.float32 and self.out.is_contiguous()
                and self.out.numel() == height * width * 4):
            raise ValueError("out must be a contiguous (height, width, 4) FP32 CUDA tensor")
        self.samples_out = samples_out

    def _struct(self) -> _Request:
        r = _Request()
        r.model = self.model.handle
        r.camera = self.cam if isinstance(self.cam, _Camera) else camera(self.cam)
        r.tf = ctypes.addressof(self.tf.struct)
        r.width, r.height, r.n_samples = self.width, self.height, self.n_samples
        r.rgba_out = self.out.data_ptr()
        r.samples_out = self.samples_out.data_ptr() if self.samples_out is not None else None
        return r


def _request_array(requests):
    arr = (_Request * len(requests))()
    for i, q in enumerate(requests):
        arr[i] = q._struct()
    return arr


class Batch:
    """Reusable batch context (mfa_batch_*): each render() is one CUDA-graph launch of a
    persistent kernel over the ray tiles of all requests."""

    def __init__(self, max_requests: int):
        import torch  # noqa: F401
        h = lib().mfa_batch_create(int(max_requests))
        if not h:
            raise MfaError(-1, lib().mfa_last_error().decode())
        self._h = h
        self.max_requests = int(max_requests)

    def configure(self, tile_shape: int = 0, grid_ctas: int = 0):
        _check(lib().mfa_batch_configure(self._h, int(tile_shape), int(grid_ctas)))

    def render(self, requests):
        arr = _request_array(requests)
        _bind_stream()
        _check(lib().mfa_batch_render(self._h, ctypes.addressof(arr), len(requests)))
        return [q.out for q in requests]

    def close(self):
        if getattr(self, "_h", None):
            lib().mfa_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def render_batch(requests):
    """One-shot batched render (thread-local context)."""
    arr = _request_array(requests)
    _bind_stream()
    _check(lib().mfa_render_batch(ctypes.addressof(arr), len(requests)))
    return [q.out for q in requests]


def render_batch_static(requests):
    """Batched render that allocates nothing (mfa_render_batch_static): at most 32
    requests; the work table lives in a fixed array in the library's device memory."""
    arr = _request_array(requests)
    _bind_stream()
    _check(lib().mfa_render_batch_static(ctypes.addressof(arr), len(requests)))
    return [q.out for q in requests]


TICKET_QUEUED, TICKET_RUNNING, TICKET_DONE, TICKET_FAILED = 0, 1, 2, 3


def server_now() -> float:
    """The monotonic clock (seconds) the server stamps arrivals and completions with."""
    return lib().mfa_server_now()


class Server:
    """Render server (mfa_server_*): resident models, requests admitted by an HBM budget as
    slots free up, then drawn tile by tile from a device work queue by persistent kernels
    (mode 0) or launched on priority streams (mode 1)."""

    QUEUE, STREAMS = 0, 1

    def __init__(self, hbm_budget_bytes: int, max_slots: int = 16, max_queue: int = 4096, priority_levels: int = 4,
                 variant: int = 0, tile_shape: int = 0, use_tuned: bool = False, mode: int = 0,
                 urgency_rate: float = 0.0):
        import torch  # noqa: F401
        cfg = _ServerConfig(int(hbm_budget_bytes), int(max_slots), int(max_queue), int(priority_levels), int(variant),
                            int(tile_shape), 1 if use_tuned else 0, int(mode), float(urgency_rate))
        h = lib().mfa_server_create(ctypes.byref(cfg))
        if not h:
            raise MfaError(-1, lib().mfa_last_error().decode())
        self._h = h
        self._keep = {}

    def submit(self, model: Model, cam, tf: transfer_fn, width: int, height: int, n_samples: int,
               arrival_time: float = 0.0) -> int:
        r = _ServeRequest()
        r.model = model.handle
        r.camera = cam if isinstance(cam, _Camera) else camera(cam)
        r.tf = ctypes.addressof(tf.struct)
        r.width, r.height, r.n_samples = int(width), int(height), int(n_samples)
        r.arrival_time_s = float(arrival_time)
        t = c_longlong()
        _check(lib().mfa_server_submit(self._h, ctypes.byref(r), ctypes.byref(t)))
        self._keep[t.value] = (width, height)
        return t.value

    def poll(self, ticket: int):
        st, lat = c_int(), c_double()
        _check(lib().mfa_server_poll(self._h, ticket, ctypes.byref(st), ctypes.byref(lat)))
        return st.value, lat.value

    def wait(self, ticket: int, timeout_ms: float = 60000.0) -> float:
        lat = c_double()
        _check(lib().mfa_server_wait(self._h, ticket, float(timeout_ms), ctypes.byref(lat)))
        return lat.value

    def result(self, ticket: int, out=None):
        """Copies the done ticket's image into a (H, W, 4) FP32 CUDA tensor."""
        import torch
        w, h = self._keep[ticket]
        if out is None:
            out = torch.empty((h, w, 4), device="cuda", dtype=torch.float32)
        _bind_stream()
        _check(lib().mfa_server_copy_result(self._h, ticket, out.data_ptr(), out.numel() * 4))
        return out

    def release(self, ticket: int):
        _check(lib().mfa_server_release(self._h, ticket))
        self._keep.pop(ticket, None)

    def stats(self) -> dict:
        s = _ServerStats()
        _check(lib().mfa_server_get_stats(self._h, ctypes.byref(s)))
        return {n: getattr(s, n) for n, _ in _ServerStats._fields_}

    def close(self):
        if getattr(self, "_h", None):
            lib().mfa_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tune_render(model: Model, cam, tf: transfer_fn, width: int, height: int, n_samples: int, reps: int = 3):
    """Autotunes (variant, tile shape) for this render's workload class; returns
    (best dict, list of all measured candidates)."""
    import torch
    out = torch.empty((height, width, 4), device="cuda", dtype=torch.float32)
    best = _TuneResult()
    allr = (_TuneResult * 32)()
    n = c_int()
    c = cam if isinstance(cam, _Camera) else camera(cam)
    _bind_stream()
    _check(lib().mfa_tune_render(model.handle, ctypes.byref(c), ctypes.byref(tf.struct), width, height, n_samples,
                                 out.data_ptr(), reps, ctypes.byref(best), ctypes.addressof(allr), 32, ctypes.byref(n)))
    conv = lambda r: dict(variant=r.variant, tile_shape=r.tile_shape, ms=r.ms)
    return conv(best), [conv(allr[i]) for i in range(n.value)]


def tune_batch(batch: "Batch", requests, reps: int = 2) -> dict:
    arr = _request_array(requests)
    best = _TuneResult()
    _bind_stream()
    _check(lib().mfa_tune_batch(batch._h, ctypes.addressof(arr), len(requests), reps, ctypes.byref(best)))
    return dict(variant=best.variant, tile_shape=best.tile_shape, ms=best.ms)


def tune_save(path: str):
    _check(lib().mfa_tune_save(path.encode()))


def tune_load(path: str):
    _check(lib().mfa_tune_load(path.encode()))
