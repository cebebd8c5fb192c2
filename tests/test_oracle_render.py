"""Pins of the oracle's ray casting (CPU only).

Closed forms: camera rays, slab clipping for axis-aligned and diagonal rays, the
constant-density slab A = 1 - (1-a)^n with C = rgb A, the early-termination stop
index k* = ceil(ln(1 - alpha_T) / ln(1 - a)), transfer-function interpolation through
a single sample, Phong with a constant normal, the zero-gradient rule, and symmetry
(a field varying in z only, viewed orthographically along z, gives identical pixels).
"""
import math

import numpy as np
import pytest

from synth import camera_ortho, camera_persp, constant_tf, knots_uniform

ORTHO = camera_ortho((0.5, 0.5, 2.5), (0.5, 0.5, 0.5), (0, 1, 0), 1.0)


def _f32(v):
    """Transfer-function rows are FP32; closed forms use the same rounded values."""
    return np.asarray(v, dtype=np.float32).astype(np.float64)


def _const_model(orc, c, n=6, p=3):
    knots = [knots_uniform(n, p)] * 3
    return orc.Model((p, p, p), (n, n, n), knots, np.full((n, n, n), c))


def _linear_model(orc, coef, n=7, p=2):
    from synth import greville
    knots = [knots_uniform(n, p)] * 3
    g = greville(knots[0], p)
    a0, b, c, d = coef
    P = a0 + b * g[None, None, :] + c * g[None, :, None] + d * g[:, None, None]
    return orc.Model((p, p, p), (n, n, n), knots, P)


def test_rays_orthographic_and_perspective(orc):
    W, H = 4, 2
    o, d = orc.ray(ORTHO, W, H, 0, 0)
    # ortho height 1 -> width 2 for a 2:1 image; pixel (0,0) centre at sx=-3/4, sy=+1/2
    np.testing.assert_allclose(o, [0.5 - 0.75, 0.5 + 0.25, 2.5], atol=1e-15)
    np.testing.assert_allclose(d, [0, 0, -1], atol=1e-15)
    cam = camera_persp((0.5, 0.5, 2.5), (0.5, 0.5, 0.5), (0, 1, 0), 60.0)
    th = math.tan(math.radians(30.0))
    for col, row in [(0, 0), (3, 1), (2, 0)]:
        o, d = orc.ray(cam, W, H, col, row)
        sx = 2 * (col + 0.5) / W - 1
        sy = 1 - 2 * (row + 0.5) / H
        v = np.array([sx * th * W / H, sy * th, -1.0])
        np.testing.assert_allclose(o, [0.5, 0.5, 2.5], atol=0)
        np.testing.assert_allclose(d, v / np.linalg.norm(v), atol=1e-15)


def test_slab_clip_closed_forms(orc):
    hit, t0, t1 = orc.clip_unit_box([0.5, 0.5, 2.5], [0, 0, -1])
    assert hit and t0 == pytest.approx(1.5, abs=1e-15) and t1 == pytest.approx(2.5, abs=1e-15)
    s = 1 / math.sqrt(3)
    hit, t0, t1 = orc.clip_unit_box([-1, -1, -1], [s, s, s])
    assert hit and t0 == pytest.approx(math.sqrt(3), rel=1e-15) and t1 == pytest.approx(2 * math.sqrt(3), rel=1e-15)
    assert not orc.clip_unit_box([2, 0.5, 0.5], [0, 0, 1])[0]          # parallel, outside
    assert not orc.clip_unit_box([0.5, 0.5, 2.0], [0, 0, 1])[0]        # box behind the eye
    hit, t0, t1 = orc.clip_unit_box([0.5, 0.5, 0.5], [1, 0, 0])        # eye inside
    assert hit and t0 == 0.0 and t1 == pytest.approx(0.5)
    # a diagonal ray that passes beside the box corner (x + y = 1.4 > 1 at z = 0.5 ... misses)
    assert not orc.clip_unit_box([2.0, 0.6, 0.5], [-1 / math.sqrt(2), 1 / math.sqrt(2), 0])[0]


@pytest.mark.parametrize("ns", [1, 7, 50])
def test_constant_density_slab(orc, ns):
    m = _const_model(orc, 0.7)
    rgba = _f32((0.2, 0.5, 0.9, 0.05))
    img, count = orc.render(m, ORTHO, constant_tf(rgba), 8, 8, ns, ert_alpha=1.0)
    A = 1 - (1 - rgba[3]) ** ns
    np.testing.assert_allclose(img[..., 3], A, rtol=0, atol=1e-14)
    for ch in range(3):
        np.testing.assert_allclose(img[..., ch], rgba[ch] * A, rtol=0, atol=1e-14)
    assert count == 64 * ns


def test_early_termination_stop_index(orc):
    m = _const_model(orc, 0.1)
    a = float(np.float32(0.05))
    kstar = math.ceil(math.log(1 - 0.99) / math.log(1 - a))
    img, count = orc.render(m, ORTHO, constant_tf((1, 1, 1, a)), 8, 8, 128, ert_alpha=0.99)
    assert count == 64 * kstar
    np.testing.assert_allclose(img[..., 3], 1 - (1 - a) ** kstar, rtol=0, atol=1e-14)


def test_perspective_hits_and_equal_opacity(orc):
    """Without opacity correction every ray through a constant field ends with the same
    alpha; rays that miss the box stay transparent black, as the slab test predicts."""
    m = _const_model(orc, 0.3)
    cam = camera_persp((0.5, 0.5, 3.0), (0.5, 0.5, 0.5), (0, 1, 0), 40.0)
    img, _ = orc.render(m, cam, constant_tf((1, 0, 0, 0.1)), 24, 16, 10, ert_alpha=1.0)
    for row in range(16):
        for col in range(24):
            o, d = orc.ray(cam, 24, 16, col, row)
            hit = orc.clip_unit_box(o, d)[0]
            want = 1 - (1 - _f32(0.1)) ** 10 if hit else 0.0
            assert img[row, col, 3] == pytest.approx(want, abs=1e-14)


def test_transfer_function_interpolation_single_sample(orc):
    m = _const_model(orc, 0.3)
    tf = np.array([[0, 0, 0, 0], [0.1, 0.2, 0.3, 0.4], [0.5, 0.6, 0.7, 0.8], [1, 1, 1, 1], [0, 1, 0, 1]], np.float32)
    img, _ = orc.render(m, ORTHO, tf, 2, 2, 1, vmin=0.0, vmax=1.0, ert_alpha=1.0)
    c = 0.8 * tf[1].astype(np.float64) + 0.2 * tf[2].astype(np.float64)   # x = 0.3 * 4 = 1.2
    np.testing.assert_allclose(img[0, 0], [c[0] * c[3], c[1] * c[3], c[2] * c[3], c[3]], atol=1e-14)
    # values beyond the range clamp to the end rows
    img, _ = orc.render(m, ORTHO, tf, 2, 2, 1, vmin=0.5, vmax=0.9, ert_alpha=1.0)
    np.testing.assert_allclose(img[1, 1], [0, 0, 0, 0], atol=1e-15)
    img, _ = orc.render(m, ORTHO, tf, 2, 2, 1, vmin=-1.0, vmax=0.0, ert_alpha=1.0)
    np.testing.assert_allclose(img[1, 1], [0, 1, 0, 1], atol=1e-15)


def test_phong_with_constant_normal(orc):
    coef = (0.2, 0.3, -0.4, 1.2)
    m = _linear_model(orc, coef)
    rgba = _f32((0.4, 0.6, 0.8, 0.07))
    ns = 20
    ka, kd, ks, s = 0.3, 0.6, 0.3, 32.0
    img, _ = orc.render(m, ORTHO, constant_tf(rgba), 4, 4, ns, shading=True, ka=ka, kd=kd, ks=ks,
                        shininess=s, ert_alpha=1.0)
    g = np.array(coef[1:])
    ndl = abs(g[2]) / np.linalg.norm(g)            # L = -d = +z
    spec = max(0.0, 2 * ndl * ndl - 1) ** s
    col = np.clip(np.array(rgba[:3]) * (ka + kd * ndl) + ks * spec, 0, 1)
    A = 1 - (1 - rgba[3]) ** ns
    np.testing.assert_allclose(img[..., 3], A, atol=1e-14)
    for ch in range(3):
        np.testing.assert_allclose(img[..., ch], col[ch] * A, atol=1e-13)


def test_zero_gradient_uses_ambient_plus_diffuse(orc):
    m = _const_model(orc, 0.5)
    rgba = _f32((0.9, 0.5, 0.1, 0.2))
    img, _ = orc.render(m, ORTHO, constant_tf(rgba), 2, 2, 3, shading=True, ert_alpha=1.0)
    A = 1 - (1 - rgba[3]) ** 3
    col = np.clip(np.array(rgba[:3]) * (0.3 + 0.6), 0, 1)
    np.testing.assert_allclose(img[0, 0], list(col * A) + [A], atol=1e-14)


def test_z_only_field_gives_identical_pixels(orc):
    rng = np.random.default_rng(31)
    n, p = 9, 3
    knots = [knots_uniform(n, p)] * 3
    P = np.broadcast_to(rng.normal(size=(n, 1, 1)), (n, n, n)).copy()
    m = orc.Model((p, p, p), (n, n, n), knots, P)
    from synth import ramp_tf
    img, _ = orc.render(m, ORTHO, ramp_tf(256, 0.05), 16, 16, 64, shading=True)
    np.testing.assert_allclose(img, np.broadcast_to(img[0, 0], img.shape), rtol=0, atol=1e-13)
    assert img[0, 0, 3] > 0.01


def test_pixel_subset_matches_full_image(orc):
    rng = np.random.default_rng(32)
    n = 8
    knots = [knots_uniform(n, 3)] * 3
    m = orc.Model((3, 3, 3), (n, n, n), knots, rng.uniform(0, 1, (n, n, n)))
    from synth import ramp_tf
    cam = camera_persp((1.9, 1.2, 2.4), (0.5, 0.5, 0.5), (0, 1, 0), 35.0)
    full, c1 = orc.render(m, cam, ramp_tf(256, 0.2), 20, 12, 40, shading=True)
    pix = rng.choice(240, 50, replace=False)
    sub, _ = orc.render(m, cam, ramp_tf(256, 0.2), 20, 12, 40, shading=True, pixels=pix, nthreads=3)
    np.testing.assert_array_equal(sub, full.reshape(-1, 4)[pix])


def test_sample_positions_are_midpoints(orc):
    """f = z viewed down -z through [0,1]: with ns samples the k-th sits at
    z = 1 - (k + 1/2)/ns; a two-row table with alpha = colour = t makes each sample's
    alpha equal to its z, so the composite is a closed-form product."""
    m = _linear_model(orc, (0.0, 0.0, 0.0, 1.0), n=4, p=1)
    tf = np.array([[0, 0, 0, 0], [1, 1, 1, 1]], np.float32)
    for ns in (1, 4, 9):
        img, _ = orc.render(m, ORTHO, tf, 2, 2, ns, vmin=0.0, vmax=1.0, ert_alpha=1.0)
        C, A = 0.0, 0.0
        for k in range(ns):
            z = 1 - (k + 0.5) / ns
            C += (1 - A) * z * z
            A += (1 - A) * z
        np.testing.assert_allclose(img[1, 0], [C, C, C, A], atol=1e-14)
