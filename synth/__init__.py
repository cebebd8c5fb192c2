"""Seeded synthetic inputs for MFA value/gradient queries and MFA ray casting.

This module builds INPUTS only: knot vectors, Greville sample sites, analytic
fields sampled at those sites (which become the control points), transfer-function
tables, camera descriptions and query points.  It holds none of the method's
arithmetic -- no knot-span search, no basis function, no control-point contraction,
no ray casting, no compositing -- so the FP64 oracle and the GPU path can both take
their inputs from here without sharing any of the computation they are compared on.

The paper's workloads (Marschner-Lobb, Fuel, Nucleon, Aneurysm, Bonsai and RMI,
Sec. V-A) are not available here.  They are stood in for by seeded fields with the
shapes of the five workload configurations below:

* Gaussian sums  g(x) = sum_m a_m exp(-|x - c_m|^2 / (2 sigma_m^2)),
  c_m ~ U[0,1]^3, sigma_m ~ U[0.05, 0.2], a_m ~ U[0.5, 1], sampled at the Greville
  abscissae of the knot vectors, plus iid N(0, 0.01^2) noise per control point;
* a turbulence-like field  sum_{m<256} A_m sin(2 pi kappa_m w_m . x + phi_m) with w_m
  uniform on the sphere, kappa_m log-uniform in [1, 64] cycles per unit length,
  A_m proportional to kappa_m^(-5/3) (normalised so sum A_m = 1), phi_m ~ U[0, 2 pi).

Configuration k draws from numpy's PCG64 seeded with 20231215 + k, in the order
documented on each builder, so every run sees the same inputs.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

SEED_BASE = 20231215


def rng_for(config: int) -> np.random.Generator:
    """Generator for workload configuration `config` (1-based)."""
    return np.random.Generator(np.random.PCG64(SEED_BASE + int(config)))


# ----------------------------------------------------------------------------------------
# knot vectors and sample sites
# ----------------------------------------------------------------------------------------

def knots_uniform(n: int, p: int) -> np.ndarray:
    """Clamped knot vector with p+1 end knots at 0 and 1 and n-p equal spans.

    Length n+p+1; interior knots i/(n-p), i = 1..n-p-1.
    """
    if n < p + 1:
        raise ValueError("need n >= p+1")
    m = n - p
    interior = np.arange(1, m, dtype=np.float64) / m
    return np.concatenate([np.zeros(p + 1), interior, np.ones(p + 1)])


def knots_nonuniform(n: int, p: int, rng: np.random.Generator, ratio: float = 4.0) -> np.ndarray:
    """Clamped knot vector whose n-p span lengths are exp(U(0, ln ratio)), normalised.

    All spans are non-empty, so interior knots are distinct.  Draws n-p uniforms.
    """
    m = n - p
    lens = np.exp(rng.uniform(0.0, math.log(ratio), size=m))
    edges = np.cumsum(lens) / lens.sum()
    interior = edges[:-1]
    return np.concatenate([np.zeros(p + 1), interior, np.ones(p + 1)])


def greville(U: np.ndarray, p: int) -> np.ndarray:
    """Greville abscissae xi_i = (U[i+1] + ... + U[i+p]) / p for i = 0..n-1.

    These are the sites at which control points are sampled from a field; for
    p = 0 the sites are the span midpoints.
    """
    U = np.asarray(U, dtype=np.float64)
    n = len(U) - p - 1
    if p == 0:
        return 0.5 * (U[:-1] + U[1:])[:n]
    csum = np.concatenate([[0.0], np.cumsum(U)])
    i = np.arange(n)
    return (csum[i + p + 1] - csum[i + 1]) / p


# ----------------------------------------------------------------------------------------
# analytic fields, evaluated on tensor grids (separably, so large grids stay cheap)
# ----------------------------------------------------------------------------------------

@dataclass
class GaussianSum:
    centres: np.ndarray  # (m, 3)
    sigma: np.ndarray    # (m,)
    amp: np.ndarray      # (m,)

    @staticmethod
    def draw(rng: np.random.Generator, m: int) -> "GaussianSum":
        """Draws centres (3m uniforms), then sigmas (m), then amplitudes (m)."""
        c = rng.uniform(0.0, 1.0, size=(m, 3))
        s = rng.uniform(0.05, 0.2, size=m)
        a = rng.uniform(0.5, 1.0, size=m)
        return GaussianSum(c, s, a)

    def grid(self, xs: np.ndarray, ys: np.ndarray, zs: np.ndarray) -> np.ndarray:
        """Field on the tensor grid, shape (len(zs), len(ys), len(xs)), x fastest."""
        inv = 1.0 / (2.0 * self.sigma ** 2)
        gx = np.exp(-((xs[None, :] - self.centres[:, 0:1]) ** 2) * inv[:, None])
        gy = np.exp(-((ys[None, :] - self.centres[:, 1:2]) ** 2) * inv[:, None])
        gz = np.exp(-((zs[None, :] - self.centres[:, 2:3]) ** 2) * inv[:, None])
        out = np.empty((len(zs), len(ys), len(xs)))
        for k in range(len(zs)):
            w = (self.amp * gz[:, k])[:, None] * gy          # (m, ny)
            out[k] = w.T @ gx                                 # (ny, nx)
        return out

    def at(self, pts: np.ndarray) -> np.ndarray:
        """Field at scattered points (n, 3)."""
        d2 = ((pts[:, None, :] - self.centres[None, :, :]) ** 2).sum(-1)
        return (self.amp[None, :] * np.exp(-d2 / (2.0 * self.sigma[None, :] ** 2))).sum(-1)


@dataclass
class Turbulence:
    kvec: np.ndarray   # (m, 3) wave vectors in cycles per unit length
    amp: np.ndarray    # (m,)
    phase: np.ndarray  # (m,)

    @staticmethod
    def draw(rng: np.random.Generator, m: int = 256, kmin: float = 1.0, kmax: float = 64.0) -> "Turbulence":
        """Draws directions (3m normals), magnitudes (m), phases (m)."""
        w = rng.normal(size=(m, 3))
        w /= np.linalg.norm(w, axis=1, keepdims=True)
        kap = np.exp(rng.uniform(math.log(kmin), math.log(kmax), size=m))
        ph = rng.uniform(0.0, 2.0 * math.pi, size=m)
        a = kap ** (-5.0 / 3.0)
        a /= a.sum()
        return Turbulence(w * kap[:, None], a, ph)

    def grid(self, xs: np.ndarray, ys: np.ndarray, zs: np.ndarray) -> np.ndarray:
        """sum_m A_m sin(2 pi k_m . x + phi_m) on a tensor grid, via the separable
        complex form Im(e^{i phi} e^{i kx x} e^{i ky y} e^{i kz z})."""
        tp = 2.0 * math.pi
        ex = np.exp(1j * tp * self.kvec[:, 0:1] * xs[None, :])
        ey = np.exp(1j * tp * self.kvec[:, 1:2] * ys[None, :])
        ez = np.exp(1j * tp * self.kvec[:, 2:3] * zs[None, :])
        c = self.amp * np.exp(1j * self.phase)
        out = np.empty((len(zs), len(ys), len(xs)))
        for k in range(len(zs)):
            w = (c * ez[:, k])[:, None] * ey
            out[k] = (w.T @ ex).imag
        return out

    def at(self, pts: np.ndarray) -> np.ndarray:
        arg = 2.0 * math.pi * (pts @ self.kvec.T) + self.phase[None, :]
        return (self.amp[None, :] * np.sin(arg)).sum(-1)


# ----------------------------------------------------------------------------------------
# transfer function, cameras, query points
# ----------------------------------------------------------------------------------------

def ramp_tf(n: int = 256, a_max: float = 0.05) -> np.ndarray:
    """n-entry RGBA table (float32, non-premultiplied); entry i sits at t = i/(n-1):
    rgb = (t, 1 - |2t - 1|, 1 - t), alpha = a_max * t."""
    t = np.arange(n, dtype=np.float64) / max(n - 1, 1)
    rgba = np.stack([t, 1.0 - np.abs(2.0 * t - 1.0), 1.0 - t, a_max * t], axis=1)
    return rgba.astype(np.float32)


def constant_tf(rgba, n: int = 2) -> np.ndarray:
    return np.tile(np.asarray(rgba, dtype=np.float32)[None, :], (n, 1))


def camera_ortho(eye, target, up, height: float) -> dict:
    return dict(projection=0, eye=tuple(map(float, eye)), target=tuple(map(float, target)),
                up=tuple(map(float, up)), fov_y_deg=0.0, ortho_height=float(height))


def camera_persp(eye, target, up, fov_y_deg: float) -> dict:
    return dict(projection=1, eye=tuple(map(float, eye)), target=tuple(map(float, target)),
                up=tuple(map(float, up)), fov_y_deg=float(fov_y_deg), ortho_height=0.0)


def random_direction(rng: np.random.Generator) -> np.ndarray:
    """Uniform on the sphere (draws 3 normals)."""
    v = rng.normal(size=3)
    return v / np.linalg.norm(v)


def view_up_for(direction: np.ndarray) -> tuple:
    """+y, unless the view direction is within ~8 degrees of it (then +z)."""
    return (0.0, 0.0, 1.0) if abs(direction[1]) > 0.99 else (0.0, 1.0, 0.0)


@dataclass
class MarschnerLobb:
    """The Marschner-Lobb test signal with the paper's constants (f_M = 6, alpha = 0.25):
        F(x, y, z) = (1 - sin(pi z / 2) + alpha (1 + rho(sqrt(x^2 + y^2)))) / (2 (1 + alpha)),
        rho(r) = cos(2 pi f_M cos(pi r / 2)),
    on its standard domain [-1, 1]^3, to which the unit parameter box maps linearly."""
    f_m: float = 6.0
    alpha: float = 0.25

    def _f(self, X, Y, Z):
        x, y, z = 2.0 * X - 1.0, 2.0 * Y - 1.0, 2.0 * Z - 1.0
        rho = np.cos(2.0 * np.pi * self.f_m * np.cos(np.pi * np.sqrt(x * x + y * y) / 2.0))
        return (1.0 - np.sin(np.pi * z / 2.0) + self.alpha * (1.0 + rho)) / (2.0 * (1.0 + self.alpha))

    def grid(self, xs: np.ndarray, ys: np.ndarray, zs: np.ndarray) -> np.ndarray:
        """Field on the tensor grid, shape (len(zs), len(ys), len(xs)), x fastest."""
        Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
        return self._f(X, Y, Z)

    def at(self, pts: np.ndarray) -> np.ndarray:
        pts = np.asarray(pts, dtype=np.float64)
        return self._f(pts[:, 0], pts[:, 1], pts[:, 2])

    def grid_device(self, m: int, device="cuda"):
        """The field at the m^3 uniform grid parameters i / (m - 1), as an (m, m, m) FP32
        torch tensor built on `device` (FP64 arithmetic; the signal is a z term plus an
        (x, y) term, so only their sum is m^3 work)."""
        import torch
        u = torch.arange(m, dtype=torch.float64, device=device) / (m - 1)
        x = 2.0 * u - 1.0
        den = 2.0 * (1.0 + self.alpha)
        r = torch.sqrt(x[:, None] ** 2 + x[None, :] ** 2)                      # [y][x]
        rho = torch.cos(2.0 * math.pi * self.f_m * torch.cos(math.pi * r / 2.0))
        fxy = (self.alpha * (1.0 + rho) / den).to(torch.float32)
        fz = ((1.0 - torch.sin(math.pi * x / 2.0)) / den).to(torch.float32)
        return fz[:, None, None] + fxy[None, :, :]


def marschner_lobb_model(n: int = 256, degree: int = 2, dtype=np.float32) -> ModelSpec:
    """Degree-p clamped-uniform model with n^3 control points: the Marschner-Lobb signal at
    the Greville sites (a stand-in for the paper's MFA encoding of the sampled signal)."""
    knots = [knots_uniform(n, degree)] * 3
    f = MarschnerLobb()
    P = sample_ctrl(f, knots, (degree,) * 3, None, 0.0)
    return ModelSpec((degree,) * 3, (n, n, n), knots, P.astype(dtype), f)


def orbit_camera(centre, dist: float, azimuth: float, elevation: float, fov_y_deg: float) -> dict:
    """Perspective camera on a sphere of radius `dist` around `centre`."""
    d = np.array([math.cos(elevation) * math.cos(azimuth), math.sin(elevation),
                  math.cos(elevation) * math.sin(azimuth)])
    eye = np.asarray(centre) + dist * d
    return camera_persp(eye, centre, view_up_for(d), fov_y_deg)


def uniform_points(rng: np.random.Generator, n: int) -> np.ndarray:
    """n query points ~ U[0,1)^3 as float32, shape (n, 3)."""
    return rng.random((n, 3), dtype=np.float32)


# ----------------------------------------------------------------------------------------
# models
# ----------------------------------------------------------------------------------------

@dataclass
class ModelSpec:
    degree: tuple
    nctrl: tuple                  # (nx, ny, nz)
    knots: List[np.ndarray]       # per axis, FP64, clamped
    ctrl: np.ndarray              # (nz, ny, nx), dtype = the input dtype handed to create
    field_: object = None

    @property
    def ctrl64(self) -> np.ndarray:
        """Control points as the FP64 values the model holds (the input's exact values)."""
        return np.asarray(self.ctrl, dtype=np.float64)


def sample_ctrl(field_obj, knots, degree, rng: Optional[np.random.Generator], noise: float) -> np.ndarray:
    """Field at the Greville tensor grid, plus iid N(0, noise^2) per point (drawn after
    the field's own parameters, in C order of the (nz, ny, nx) array)."""
    xs, ys, zs = (greville(knots[a], degree[a]) for a in range(3))
    P = field_obj.grid(xs, ys, zs)
    if noise > 0:
        P = P + rng.normal(0.0, noise, size=P.shape)
    return P


def gaussian_model(rng, degree, nctrl, m, noise=0.01, knots=None, dtype=np.float64) -> ModelSpec:
    f = GaussianSum.draw(rng, m)
    if knots is None:
        knots = [knots_uniform(nctrl[a], degree[a]) for a in range(3)]
    P = sample_ctrl(f, knots, degree, rng, noise)
    return ModelSpec(tuple(degree), tuple(nctrl), knots, P.astype(dtype), f)


def turbulence_model(rng, degree, nctrl, knots, m=256, noise=0.0, dtype=np.float64) -> ModelSpec:
    f = Turbulence.draw(rng, m)
    P = sample_ctrl(f, knots, degree, rng, noise)
    return ModelSpec(tuple(degree), tuple(nctrl), knots, P.astype(dtype), f)


# ----------------------------------------------------------------------------------------
# the five workload configurations
# ----------------------------------------------------------------------------------------

@dataclass
class RenderJob:
    camera: dict
    width: int
    height: int
    n_samples: int
    tf: np.ndarray
    shading: bool
    ka: float = 0.3
    kd: float = 0.6
    ks: float = 0.3
    shininess: float = 32.0
    ert_alpha: float = 0.99


@dataclass
class Workload:
    name: str
    model: ModelSpec
    render: Optional[RenderJob]
    decode_points: Optional[np.ndarray] = None
    extra: dict = field(default_factory=dict)


def config1() -> Workload:
    """Degree 3, 32^3 FP64 control points, clamped uniform knots, 8 Gaussians plus
    N(0, 0.01^2) noise; orthographic 256^2 view down -z, 128 samples per ray, 256-entry
    ramp (a_max 0.05), no shading, early termination at alpha 0.99."""
    rng = rng_for(1)
    m = gaussian_model(rng, (3, 3, 3), (32, 32, 32), 8, noise=0.01, dtype=np.float64)
    cam = camera_ortho((0.5, 0.5, 2.5), (0.5, 0.5, 0.5), (0.0, 1.0, 0.0), 1.0)
    job = RenderJob(cam, 256, 256, 128, ramp_tf(256, 0.05), shading=False)
    return Workload("mfa_render_p3_32cube_ortho256_ns128", m, job)


def config2(decode_n: int = 1 << 24, with_points: bool = True) -> Workload:
    """Degree 3, 128^3 FP32 control points from 64 Gaussians plus noise; perspective
    1024^2 (fov_y 30 deg, eye 2.5 from the centre along a seeded direction), 1024
    samples per ray, Phong; plus 2^24 uniform decode points (value + gradient)."""
    rng = rng_for(2)
    m = gaussian_model(rng, (3, 3, 3), (128, 128, 128), 64, noise=0.01, dtype=np.float32)
    d = random_direction(rng)
    c = np.array([0.5, 0.5, 0.5])
    cam = camera_persp(c + 2.5 * d, c, view_up_for(d), 30.0)
    job = RenderJob(cam, 1024, 1024, 1024, ramp_tf(256, 0.05), shading=True)
    pts = uniform_points(rng, decode_n) if with_points else None
    return Workload("mfa_render_p3_128cube_persp1024_ns1024_phong+decode_2^24", m, job, pts)


def config3(dtype_in=np.float64, nctrl=(512, 512, 256), decode_n: int = 1 << 22,
            with_points: bool = True) -> Workload:
    """Degree 3, 512x512x256 control points, non-uniform clamped knots (spacings
    log-uniform in 1:4), turbulence field; perspective 2048^2, 2048 samples, Phong,
    ramp a_max 0.02; plus 2^22 decode points."""
    rng = rng_for(3)
    knots = [knots_nonuniform(nctrl[a], 3, rng, 4.0) for a in range(3)]
    m = turbulence_model(rng, (3, 3, 3), nctrl, knots, 256, 0.0, dtype=dtype_in)
    d = random_direction(rng)
    c = np.array([0.5, 0.5, 0.5])
    cam = camera_persp(c + 2.5 * d, c, view_up_for(d), 30.0)
    job = RenderJob(cam, 2048, 2048, 2048, ramp_tf(256, 0.02), shading=True)
    pts = uniform_points(rng, decode_n) if with_points else None
    return Workload("mfa_precision_p3_512x512x256_nonuniform_persp2048_ns2048", m, job, pts)


def ctrl_minmax(P: np.ndarray):
    P = np.asarray(P, dtype=np.float64)
    return float(P.min()), float(P.max())


def config4(size_scale: float = 1.0, rng_draws: bool = True) -> list:
    """Batched workload: 16 models, per-axis control-point counts log-uniform integers in
    [32, 256] (times size_scale), degrees cycling 2, 3, 4, uniform knots for even models
    and non-uniform (1:4) for odd ones, FP32, Gaussian-sum fields (16 Gaussians + noise).
    Each model gets one request: square image of side drawn from {256, 384, 512, 768,
    1024}, 256..1024 samples per ray, Phong, ramp a_max 0.05, seeded perspective view.
    Returns a list of (ModelSpec, RenderJob)."""
    rng = rng_for(4)
    out = []
    for i in range(16):
        p = (2, 3, 4)[i % 3]
        n = tuple(max(p + 1, int(round(size_scale * math.exp(rng.uniform(math.log(32), math.log(256))))))
                  for _ in range(3))
        if i % 2 == 0:
            knots = [knots_uniform(n[a], p) for a in range(3)]
        else:
            knots = [knots_nonuniform(n[a], p, rng) for a in range(3)]
        m = gaussian_model(rng, (p, p, p), n, 16, noise=0.01, knots=knots, dtype=np.float32)
        side = int(rng.choice([256, 384, 512, 768, 1024]))
        ns = int(rng.integers(256, 1025))
        d = random_direction(rng)
        c = np.array([0.5, 0.5, 0.5])
        cam = camera_persp(c + 2.5 * d, c, view_up_for(d), 30.0)
        out.append((m, RenderJob(cam, side, side, ns, ramp_tf(256, 0.05), shading=True)))
    return out


SERVE_SIZES = [(128, 128, 128), (192, 192, 192), (256, 256, 256), (320, 320, 320), (384, 384, 384),
               (512, 384, 256), (512, 512, 192), (512, 512, 256)]


def config5_models(size_scale: float = 1.0) -> list:
    """Serving workload models: 8 resident degree-3 models of the listed sizes (times
    size_scale), turbulence (even index) and Gaussian-sum (odd) fields alternating,
    stored as FP16 control points.  Returns ModelSpecs with FP64 control points."""
    rng = rng_for(5)
    out = []
    for i, n in enumerate(SERVE_SIZES):
        n = tuple(max(4, int(round(size_scale * x))) for x in n)
        knots = [knots_uniform(n[a], 3) for a in range(3)]
        if i % 2 == 0:
            out.append(turbulence_model(rng, (3, 3, 3), n, knots, 64, 0.0, dtype=np.float64))
        else:
            out.append(gaussian_model(rng, (3, 3, 3), n, 32, noise=0.01, knots=knots, dtype=np.float64))
    return out


def config5_requests(rate_hz: float, duration_s: float, n_models: int = 8, seed_offset: int = 0,
                     sides=(512, 1024, 1536, 2048), ns_range=(512, 2048)):
    """Poisson request stream: arrival times (exponential gaps at rate_hz), a model index,
    a square image side from `sides`, samples per ray uniform in ns_range, and an orbit
    camera that advances along a seeded path per model.  Returns a list of dicts."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 5 + 1000 * (1 + seed_offset)))
    t, out = 0.0, []
    phase = rng.uniform(0, 2 * math.pi, size=n_models)
    elev = rng.uniform(-0.5, 0.5, size=n_models)
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t >= duration_s:
            break
        m = int(rng.integers(0, n_models))
        phase[m] += 0.05
        out.append(dict(t=t, model=m, side=int(rng.choice(sides)), n_samples=int(rng.integers(ns_range[0], ns_range[1] + 1)),
                        camera=orbit_camera((0.5, 0.5, 0.5), 2.5, float(phase[m]), float(elev[m]), 30.0)))
    return out
