"""FP64 CPU oracle for MFA value/gradient queries and MFA ray casting (ctypes shim).

TEST INFRASTRUCTURE ONLY.  Only `tests/`, `__graft_entry__.smoke()` and the CPU
baseline of `bench.py` may import this package.  The GPU library never does, and this
package never imports the GPU library: the two share no code.  The arithmetic lives in
`oracle.c` (plain C, FP64, one query or one ray at a time); this file compiles it with
gcc, loads it and marshals numpy arrays.

Each function cites what it follows:
  * `find_span`, `basis`, `basis_direct*`: the textbook Cox-de Boor definition of the
    B-spline basis, which the paper's MFA model (Sec. III-A) is built from;
  * `eval_points` (decode): the value and analytic gradient of the tensor-product
    B-spline volume (Sec. III-B, Sec. V-D.3);
  * `render`: MFA-VV ray casting with the over operation between neighbouring samples
    (Sec. IV-A.4) and user-set transfer function and shading (Sec. IV-B);
  * `ml_eval`, `render_ml`: the closed-form Marschner-Lobb signal (Sec. V-A.1, Eq. 1) and
    its direct render, the ground truth the paper compares renders against (Sec. V-D.3);
  * `quality` (module): MSE, PSNR and SSIM between two images (Table II's metrics).

Pins (see tests/test_oracle_*.py): partition of unity, the derivative sum, the
Bernstein closed form, degree-1 trilinear interpolation, exact reproduction of linear
fields from Greville control points, brute-force recursion on tiny models, central
finite differences, the derivative-spline identity, brute-force span search, the slab
closed forms and the constant-density compositing closed form.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from ctypes import POINTER, c_double, c_float, c_int, c_longlong, c_void_p

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so with gcc (portable C, no -march flags,
    no FMA contraction, so x86 and Arm hosts compute the same FP64 results)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm", "-lpthread"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Model(ctypes.Structure):
    _fields_ = [("p", c_int * 3), ("n", c_int * 3), ("U", c_void_p * 3), ("P", c_void_p)]


class _Camera(ctypes.Structure):
    _fields_ = [("projection", c_int), ("eye", c_double * 3), ("target", c_double * 3),
                ("up", c_double * 3), ("fov_y_deg", c_double), ("ortho_height", c_double)]


class _TF(ctypes.Structure):
    _fields_ = [("n_entries", c_int), ("rgba", c_void_p), ("vmin", c_double), ("vmax", c_double),
                ("shading", c_int), ("ka", c_double), ("kd", c_double), ("ks", c_double),
                ("shininess", c_double), ("ert_alpha", c_double)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.orc_find_span.restype = c_int
        lib.orc_find_span.argtypes = [c_int, c_int, c_void_p, c_double]
        lib.orc_basis.restype = None
        lib.orc_basis.argtypes = [c_int, c_double, c_int, c_void_p, c_void_p, c_void_p]
        lib.orc_basis_direct.restype = c_double
        lib.orc_basis_direct.argtypes = [c_int, c_int, c_double, c_void_p, c_int]
        lib.orc_basis_direct_deriv.restype = c_double
        lib.orc_basis_direct_deriv.argtypes = [c_int, c_int, c_double, c_void_p, c_int]
        lib.orc_eval.restype = None
        lib.orc_eval.argtypes = [POINTER(_Model), c_void_p, c_void_p, c_void_p]
        lib.orc_eval_direct.restype = None
        lib.orc_eval_direct.argtypes = [POINTER(_Model), c_void_p, c_void_p]
        lib.orc_decode.restype = c_int
        lib.orc_decode.argtypes = [POINTER(_Model), c_void_p, c_longlong, c_void_p, c_void_p, c_void_p, c_int]
        lib.orc_ray.restype = None
        lib.orc_ray.argtypes = [POINTER(_Camera), c_int, c_int, c_int, c_int, c_void_p, c_void_p]
        lib.orc_clip_unit_box.restype = c_int
        lib.orc_clip_unit_box.argtypes = [c_void_p, c_void_p, POINTER(c_double), POINTER(c_double)]
        lib.orc_render.restype = c_longlong
        lib.orc_render.argtypes = [POINTER(_Model), POINTER(_Camera), POINTER(_TF), c_int, c_int, c_int,
                                   c_void_p, c_longlong, c_void_p, c_int]
        lib.orc_render_segments.restype = c_longlong
        lib.orc_render_segments.argtypes = [POINTER(_Model), POINTER(_Camera), POINTER(_TF), c_int, c_int, c_int,
                                            c_void_p, c_void_p, c_longlong, c_void_p, c_int]
        lib.orc_render_iso.restype = c_longlong
        lib.orc_render_iso.argtypes = [POINTER(_Model), POINTER(_Camera), POINTER(_TF), c_int, c_int, c_int, c_double,
                                       c_void_p, c_longlong, c_void_p, c_void_p, c_int]
        lib.orc_block_range.restype = None
        lib.orc_block_range.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_double, c_double, c_int,
                                        POINTER(c_int), POINTER(c_int)]
        lib.orc_ml_eval.argtypes = [c_double, c_double, c_void_p, c_void_p]
        lib.orc_ml_eval.restype = None
        lib.orc_render_ml.argtypes = [c_double, c_double, POINTER(_Camera), POINTER(_TF), c_int, c_int, c_int,
                                      c_void_p, c_longlong, c_void_p, c_int]
        lib.orc_render_ml.restype = c_longlong
        _lib = lib
    return _lib


def default_threads() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


# ------------------------------------------------------------------------------------------
# basis level
# ------------------------------------------------------------------------------------------

def find_span(U, p: int, u: float) -> int:
    U = _f64(U)
    n = len(U) - p - 1
    return _load().orc_find_span(n, p, _ptr(U), float(u))


def basis(U, p: int, u: float, span: int | None = None):
    """(span, N[0..p], dN[0..p]) at u (u must already lie in the domain)."""
    U = _f64(U)
    if span is None:
        span = find_span(U, p, u)
    N = np.zeros(p + 1)
    D = np.zeros(p + 1)
    _load().orc_basis(int(span), float(u), int(p), _ptr(U), _ptr(N), _ptr(D))
    return span, N, D


def basis_direct(U, p: int, i: int, u: float) -> float:
    U = _f64(U)
    return _load().orc_basis_direct(int(i), int(p), float(u), _ptr(U), len(U))


def basis_direct_deriv(U, p: int, i: int, u: float) -> float:
    U = _f64(U)
    return _load().orc_basis_direct_deriv(int(i), int(p), float(u), _ptr(U), len(U))


# ------------------------------------------------------------------------------------------
# model level
# ------------------------------------------------------------------------------------------

class Model:
    """FP64 MFA model: degrees (px,py,pz), counts (nx,ny,nz), knots, ctrl[nz][ny][nx]."""

    def __init__(self, degree, nctrl, knots, ctrl):
        self.degree = tuple(int(d) for d in degree)
        self.nctrl = tuple(int(n) for n in nctrl)
        self.knots = [_f64(k) for k in knots]
        self.ctrl = _f64(ctrl).reshape(self.nctrl[2], self.nctrl[1], self.nctrl[0])
        for a in range(3):
            if len(self.knots[a]) != self.nctrl[a] + self.degree[a] + 1:
                raise ValueError("knot vector length must be n+p+1")
        self._s = _Model()
        for a in range(3):
            self._s.p[a] = self.degree[a]
            self._s.n[a] = self.nctrl[a]
            self._s.U[a] = _ptr(self.knots[a])
        self._s.P = _ptr(self.ctrl)

    @staticmethod
    def from_spec(spec, ctrl64=None) -> "Model":
        return Model(spec.degree, spec.nctrl, spec.knots, spec.ctrl64 if ctrl64 is None else ctrl64)

    def eval(self, uvw):
        """(f, grad[3], spans[3]) at one point."""
        x = _f64(uvw)
        out = np.zeros(4)
        sp = np.zeros(3, dtype=np.int32)
        _load().orc_eval(ctypes.byref(self._s), _ptr(x), _ptr(out), _ptr(sp))
        return out[0], out[1:].copy(), sp

    def eval_direct(self, uvw):
        x = _f64(uvw)
        out = np.zeros(4)
        _load().orc_eval_direct(ctypes.byref(self._s), _ptr(x), _ptr(out))
        return out[0], out[1:].copy()

    def decode(self, pts, grad: bool = True, spans: bool = False, nthreads: int | None = None):
        """Value (n,), gradient (n,3) and optionally knot spans (n,3) at FP32 points,
        each evaluated at the exact FP64 value of its FP32 coordinates."""
        pts = np.ascontiguousarray(pts, dtype=np.float32).reshape(-1, 3)
        n = pts.shape[0]
        val = np.zeros(n)
        g = np.zeros((n, 3)) if grad else None
        sp = np.zeros((n, 3), dtype=np.int32) if spans else None
        _load().orc_decode(ctypes.byref(self._s), _ptr(pts), n, _ptr(val),
                           _ptr(g) if g is not None else None, _ptr(sp) if sp is not None else None,
                           nthreads or default_threads())
        out = [val, g]
        if spans:
            out.append(sp)
        return tuple(out)


def _camera(cam: dict) -> _Camera:
    c = _Camera()
    c.projection = int(cam["projection"])
    for a in range(3):
        c.eye[a] = cam["eye"][a]
        c.target[a] = cam["target"][a]
        c.up[a] = cam["up"][a]
    c.fov_y_deg = cam.get("fov_y_deg", 0.0)
    c.ortho_height = cam.get("ortho_height", 0.0)
    return c


def ray(cam: dict, W: int, H: int, col: int, row: int):
    o = np.zeros(3)
    d = np.zeros(3)
    c = _camera(cam)
    _load().orc_ray(ctypes.byref(c), W, H, col, row, _ptr(o), _ptr(d))
    return o, d


def clip_unit_box(o, d):
    o = _f64(o)
    d = _f64(d)
    t0 = c_double()
    t1 = c_double()
    hit = _load().orc_clip_unit_box(_ptr(o), _ptr(d), ctypes.byref(t0), ctypes.byref(t1))
    return bool(hit), t0.value, t1.value


def render(model: Model, cam: dict, tf_rgba, width: int, height: int, n_samples: int, *,
           shading: bool = False, ka=0.3, kd=0.6, ks=0.3, shininess=32.0, ert_alpha=0.99,
           vmin=math.nan, vmax=math.nan, pixels=None, nthreads: int | None = None):
    """Premultiplied RGBA in FP64: (H, W, 4) for the full image, or (len(pixels), 4) for
    the listed pixel indices (row*W + col).  Returns (rgba, samples evaluated)."""
    tf_rgba = np.ascontiguousarray(tf_rgba, dtype=np.float32).reshape(-1, 4)
    tf = _TF()
    tf.n_entries = tf_rgba.shape[0]
    tf.rgba = _ptr(tf_rgba)
    tf.vmin = vmin
    tf.vmax = vmax
    tf.shading = 1 if shading else 0
    tf.ka, tf.kd, tf.ks, tf.shininess = ka, kd, ks, shininess
    tf.ert_alpha = ert_alpha
    cam_s = _camera(cam)
    if pixels is None:
        out = np.zeros((height, width, 4))
        npix, pix_ptr = width * height, None
    else:
        pixels = np.ascontiguousarray(pixels, dtype=np.int64)
        out = np.zeros((len(pixels), 4))
        npix, pix_ptr = len(pixels), _ptr(pixels)
    ns = _load().orc_render(ctypes.byref(model._s), ctypes.byref(cam_s), ctypes.byref(tf), width, height,
                            n_samples, pix_ptr, npix, _ptr(out), nthreads or default_threads())
    return out, int(ns)


def render_segments(model: Model, cam: dict, tf_rgba, width: int, height: int, n_samples: int, blocks, *,
                    shading: bool = False, ka=0.3, kd=0.6, ks=0.3, shininess=32.0, ert_alpha=0.99,
                    vmin=math.nan, vmax=math.nan, pixels=None, nthreads: int | None = None):
    """render() with the volume split into blocks[0] x blocks[1] x blocks[2] equal blocks,
    each rendering its segment of every ray (early termination per segment), the partial
    images merged with over nearest segment first.  Returns (rgba, samples evaluated)."""
    tf_rgba = np.ascontiguousarray(tf_rgba, dtype=np.float32).reshape(-1, 4)
    tf = _TF()
    tf.n_entries = tf_rgba.shape[0]
    tf.rgba = _ptr(tf_rgba)
    tf.vmin = vmin
    tf.vmax = vmax
    tf.shading = 1 if shading else 0
    tf.ka, tf.kd, tf.ks, tf.shininess = ka, kd, ks, shininess
    tf.ert_alpha = ert_alpha
    cam_s = _camera(cam)
    g = np.ascontiguousarray(blocks, dtype=np.int32)
    if pixels is None:
        out = np.zeros((height, width, 4))
        npix, pix_ptr = width * height, None
    else:
        pixels = np.ascontiguousarray(pixels, dtype=np.int64)
        out = np.zeros((len(pixels), 4))
        npix, pix_ptr = len(pixels), _ptr(pixels)
    ns = _load().orc_render_segments(ctypes.byref(model._s), ctypes.byref(cam_s), ctypes.byref(tf), width, height,
                                     n_samples, _ptr(g), pix_ptr, npix, _ptr(out), nthreads or default_threads())
    if ns < 0:
        raise ValueError("blocks must be >= 1 per axis and at most 512 in total")
    return out, int(ns)


def render_iso(model: Model, cam: dict, tf_rgba, width: int, height: int, n_samples: int, iso: float, *,
               shading: bool = True, ka=0.3, kd=0.6, ks=0.3, shininess=32.0, vmin=math.nan, vmax=math.nan,
               pixels=None, nthreads: int | None = None):
    """Isosurface f = iso: first crossing along each ray's samples, refined by bracketed
    Newton steps, shaded opaque.  Returns (rgba, depth, queries): rgba (H, W, 4) or
    (len(pixels), 4), depth the hit parameter t (+inf on a miss)."""
    tf_rgba = np.ascontiguousarray(tf_rgba, dtype=np.float32).reshape(-1, 4)
    tf = _TF()
    tf.n_entries = tf_rgba.shape[0]
    tf.rgba = _ptr(tf_rgba)
    tf.vmin = vmin
    tf.vmax = vmax
    tf.shading = 1 if shading else 0
    tf.ka, tf.kd, tf.ks, tf.shininess = ka, kd, ks, shininess
    tf.ert_alpha = 1.0
    cam_s = _camera(cam)
    if pixels is None:
        out = np.zeros((height, width, 4))
        depth = np.zeros((height, width))
        npix, pix_ptr = width * height, None
    else:
        pixels = np.ascontiguousarray(pixels, dtype=np.int64)
        out = np.zeros((len(pixels), 4))
        depth = np.zeros(len(pixels))
        npix, pix_ptr = len(pixels), _ptr(pixels)
    nq = _load().orc_render_iso(ctypes.byref(model._s), ctypes.byref(cam_s), ctypes.byref(tf), width, height,
                                n_samples, float(iso), pix_ptr, npix, _ptr(out), _ptr(depth),
                                nthreads or default_threads())
    return out, depth, int(nq)


def ml_eval(uvw, f_m: float = 6.0, alpha: float = 0.25) -> np.ndarray:
    """{F, dF/du, dF/dv, dF/dw} of the Marschner-Lobb signal at a point of the unit box."""
    x = _f64(uvw)
    out = np.zeros(4)
    _load().orc_ml_eval(f_m, alpha, _ptr(x), _ptr(out))
    return out


def render_ml(cam: dict, tf_rgba, width: int, height: int, n_samples: int, *, f_m: float = 6.0,
              alpha: float = 0.25, shading: bool = False, ka=0.3, kd=0.6, ks=0.3, shininess=32.0,
              ert_alpha=0.99, vmin=math.nan, vmax=math.nan, pixels=None, nthreads: int | None = None):
    """render() of the closed-form Marschner-Lobb signal (vmin / vmax default to its range
    [0, 1]).  Returns (rgba, samples evaluated)."""
    tf_rgba = np.ascontiguousarray(tf_rgba, dtype=np.float32).reshape(-1, 4)
    tf = _TF()
    tf.n_entries = tf_rgba.shape[0]
    tf.rgba = _ptr(tf_rgba)
    tf.vmin = vmin
    tf.vmax = vmax
    tf.shading = 1 if shading else 0
    tf.ka, tf.kd, tf.ks, tf.shininess = ka, kd, ks, shininess
    tf.ert_alpha = ert_alpha
    cam_s = _camera(cam)
    if pixels is None:
        out = np.zeros((height, width, 4))
        npix, pix_ptr = width * height, None
    else:
        pixels = np.ascontiguousarray(pixels, dtype=np.int64)
        out = np.zeros((len(pixels), 4))
        npix, pix_ptr = len(pixels), _ptr(pixels)
    ns = _load().orc_render_ml(f_m, alpha, ctypes.byref(cam_s), ctypes.byref(tf), width, height, n_samples,
                               pix_ptr, npix, _ptr(out), nthreads or default_threads())
    return out, int(ns)


def block_range(blocks, block, o, d, t0: float, dt: float, n_samples: int):
    """Sample index range [kb, ke) that block `block` of the blocks grid renders on the ray
    (o, d) whose samples sit at t0 + (k + 1/2) dt."""
    g = np.ascontiguousarray(blocks, dtype=np.int32)
    bi = np.ascontiguousarray(block, dtype=np.int32)
    o, d = _f64(o), _f64(d)
    kb, ke = c_int(), c_int()
    _load().orc_block_range(_ptr(g), _ptr(bi), _ptr(o), _ptr(d), float(t0), float(dt), int(n_samples),
                            ctypes.byref(kb), ctypes.byref(ke))
    return kb.value, ke.value


# ------------------------------------------------------------------------------------------
# storage rounding (the reduced-precision control points the GPU stores)
# ------------------------------------------------------------------------------------------

def round_to_f16(P) -> np.ndarray:
    """FP64 -> FP16 in one round-to-nearest-even step (numpy converts double bits to
    half bits directly), returned as FP64."""
    return _f64(P).astype(np.float16).astype(np.float64)


def round_to_bf16(P) -> np.ndarray:
    """FP64 -> BF16 in one round-to-nearest-even step: keep the top 7 of the 52 FP64
    mantissa bits (round at bit 45), with no detour through FP32.  Valid for finite
    values within the BF16 normal range, which covers every generated field."""
    b = _f64(P).view(np.int64).copy()
    lsb = (b >> 45) & 1
    b = (b + ((1 << 44) - 1) + lsb) & ~np.int64((1 << 45) - 1)
    return b.view(np.float64)
